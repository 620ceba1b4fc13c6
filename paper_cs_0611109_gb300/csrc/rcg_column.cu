// rcg_column.cu -- the column kernel: bit-sliced stripes of a small prime
// (p <= 7, at most 6 rows per strip) without shared memory.
//
// A thread owns one 16-byte column of a stripe across all p-1 rows of every
// strip: it loads them with coalesced 16-byte loads (the columns of a warp
// are adjacent), keeps the lifted accumulators of F2[x]/(x^p - 1) in
// registers -- p rows, row p-1 the imaginary row -- and writes the results.
// Multiplication by x is a rotation of the register rows, so Q is
// accumulated by Horner's rule, Q = d + x Q, over the data strips from the
// last to the first (Section 4.2), with a second Horner sum for the extended
// strips k >= p of equation (qext) (weights 1 + x^(k-p+1)).  Reduction modulo
// f = 1 + ... + x^(p-1) folds row p-1 into every other row (Lemma 3.4.1's
// conditional all-ones fold).  Recovery follows Lemma 3.1.2's four cases with
// one multiplication by an inverse -- of w_i (data + P) or of w_i + w_j (two
// data strips) -- from a host-computed table of exponent masks.  The degraded
// read is the recovery of the strip alone, written to the caller's buffer;
// the small write adds (old + new) to P and w_i (old + new) to Q.
//
// Why a second kernel: the tile engine streams one strip tile per pipeline
// stage, and at p = 5 with 1 KiB rows a stage is 4 KB, so its fixed cost per
// stage and per tile dominates small stripes.  Here a column is one DRAM round
// trip per thread.  Single-operation launches stride the columns of one job
// over the grid; batches give each warp a contiguous range of 32-column
// chunks of their jobs, each job a self-contained 128-byte record
// (persistent grid, one kernel per variant: p = 3, 5, 5 with extended
// strips, 7).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/rcg.h"
#include "rcg_internal.h"

namespace rcg {

namespace {

constexpr int kColPrimes = 3;  // p = 3, 5, 7
constexpr int kColMaxN = 9;    // 2p - 1 for p = 5

__constant__ uint32_t c_col_inv_w[kColPrimes][kColMaxN];
__constant__ uint32_t c_col_inv_pair[kColPrimes][kColMaxN][kColMaxN];

// A lane's column is 16 bytes (a uint4; the helpers take the vector type
// as a template parameter).  8-byte columns (half the registers, three CTAs
// per SM) measured slower on GB300: the p = 5 geometry's 16-operation batch
// 0.68 against 0.69 of peak, p = 5 jobs in the uneven batches 0.49 against 0.53.
__device__ __forceinline__ uint4 xr(uint4 a, uint4 b) {
    return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
}

template <class V>
__device__ __forceinline__ V vzero();
template <>
__device__ __forceinline__ uint4 vzero<uint4>() { return make_uint4(0, 0, 0, 0); }

template <class V>
__device__ __forceinline__ V ld_col(const uint8_t *p);
template <>
__device__ __forceinline__ uint4 ld_col<uint4>(const uint8_t *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ void st_col(uint8_t *p, uint4 v) {
    asm volatile("st.global.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

// acc <- x acc + d in the lift (d has p-1 rows; its row p-1 is zero)
template <int P, class V>
__device__ __forceinline__ void horner_step(V (&acc)[P], const V (&d)[P - 1]) {
    const V top = acc[P - 1];
    acc[P - 1] = acc[P - 2];
#pragma unroll
    for (int r = P - 2; r >= 1; --r) acc[r] = xr(acc[r - 1], d[r]);
    acc[0] = xr(top, d[0]);
}

// out += x^m a in the lift, m in [0, p): a rotation of the rows
template <int P, int M = 0, class V>
__device__ __forceinline__ void add_rot(const V (&a)[P], uint32_t m, V (&out)[P]) {
    if constexpr (M < P) {
        if (m == M) {
#pragma unroll
            for (int r = 0; r < P; ++r) out[(r + M) % P] = xr(out[(r + M) % P], a[r]);
        } else {
            add_rot<P, M + 1>(a, m, out);
        }
    }
}

// out = w_k a (weight of data strip k: x^k, or 1 + x^(k-p+1) when k >= p)
template <int P, class V>
__device__ __forceinline__ void mul_w(const V (&a)[P], uint32_t k, V (&out)[P]) {
#pragma unroll
    for (int r = 0; r < P; ++r) out[r] = vzero<V>();
    if (k < static_cast<uint32_t>(P)) {
        add_rot<P>(a, k, out);
    } else {
#pragma unroll
        for (int r = 0; r < P; ++r) out[r] = a[r];
        add_rot<P>(a, k - P + 1, out);
    }
}

// out = (sum over the mask's exponents m of x^m) a
template <int P, class V>
__device__ __forceinline__ void mul_mask(const V (&a)[P], uint32_t mask, V (&out)[P]) {
#pragma unroll
    for (int r = 0; r < P; ++r) out[r] = vzero<V>();
    while (mask) {
        const uint32_t m = __ffs(mask) - 1;
        mask &= mask - 1;
        add_rot<P>(a, m, out);
    }
}

template <int P, class V>
__device__ __forceinline__ void store_folded(uint8_t *strip, uint64_t rs, const V (&a)[P]) {
#pragma unroll
    for (int r = 0; r < P - 1; ++r) st_col(strip + r * rs, xr(a[r], a[P - 1]));
}

template <int P, class V>
__device__ __forceinline__ void store_rows(uint8_t *strip, uint64_t rs, const V (&a)[P - 1]) {
#pragma unroll
    for (int r = 0; r < P - 1; ++r) st_col(strip + r * rs, a[r]);
}

template <int P, class V>
__device__ __forceinline__ void lift(const V (&a)[P - 1], V (&out)[P]) {
#pragma unroll
    for (int r = 0; r < P - 1; ++r) out[r] = a[r];
    out[P - 1] = vzero<V>();
}

template <int P>
__host__ __device__ constexpr int table_slot() {
    return P == 3 ? 0 : P == 5 ? 1 : 2;
}

// The small write on column v (sizeof(V) bytes) of stripe s: with D = old d_i + new d_i,
// P += D, Q += w_i D (reduced), d_i = new.
template <int P, class V>
__device__ __forceinline__ void column_update(const ColJob &J, uint64_t s, uint32_t v) {
    constexpr int R = P - 1;
    uint8_t *const col = J.base + s * J.st + v * static_cast<uint64_t>(sizeof(V));
    const uint8_t *const nw = J.aux + s * J.ass + v * static_cast<uint64_t>(sizeof(V));
    const uint32_t N = J.N, a = J.i;
    const uint64_t rs = J.rs, ss = J.ss;
    V od[R], nv[R], pv[R], qv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        od[r] = ld_col<V>(col + a * ss + r * rs);
        nv[r] = ld_col<V>(nw + r * J.ars);
        pv[r] = ld_col<V>(col + N * ss + r * rs);
        qv[r] = ld_col<V>(col + (N + 1) * ss + r * rs);
    }
    V dl[P], t[P];
#pragma unroll
    for (int r = 0; r < R; ++r) dl[r] = xr(od[r], nv[r]);
    dl[R] = vzero<V>();
    mul_w<P>(dl, a, t);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        st_col(col + a * ss + r * rs, nv[r]);
        st_col(col + N * ss + r * rs, xr(pv[r], dl[r]));
        st_col(col + (N + 1) * ss + r * rs, xr(qv[r], xr(t[r], t[R])));
    }
}

// One column v (sizeof(V) bytes) of stripe s of a job: every operation but the small write.
template <int P, bool EXT, class V>
__device__ __forceinline__ void column_unit(const ColJob &J, uint64_t s, uint32_t v, uint32_t *status) {
    constexpr int R = P - 1;
    constexpr int KB = P == 7 ? 2 : 4;  // strips per batch of loads
    constexpr int slot = table_slot<P>();
    if (J.op == OP_UPDATE) {
        column_update<P, V>(J, s, v);
        return;
    }
    const uint32_t N = J.N;
    const uint64_t rs = J.rs, ss = J.ss;
    const bool deg = J.op == OP_DEGRADED;
    // strips a < b that are not read: the erased pair; (N, N+1) for encode;
    // a degraded read of data strip j is the recovery of (j, Q) without the
    // writes, of P or Q the encode without them
    uint32_t a, b;
    if (J.op == OP_ENCODE) {
        a = N;
        b = N + 1;
    } else if (deg) {
        a = J.j < N ? J.j : N;
        b = N + 1;
    } else {
        a = J.i;
        b = J.j;
        if (J.pairs) {
            a = J.pairs[2 * s];
            b = J.pairs[2 * s + 1];
        }
        if (!(a < b && b <= N + 1)) {
            if (v == 0 && status) atomicOr(status, RCG_DEV_BADPAIR);
            return;
        }
    }
    uint8_t *const col = J.base + s * J.st + v * static_cast<uint64_t>(sizeof(V));
    const bool read_p = a != N && b != N, read_q = a != N + 1 && b != N + 1;
    // dP starts as P (when read).  The Horner sum of the data strips starts
    // as x^(-h) Q, h = the number of Horner steps it takes (N, or p when the
    // extended strips have their own sum; x^p = 1 in the lift), so that it
    // ends as Q + sum of x^k d_k.  x^(-h) is applied to the load addresses:
    // lifted row t of x^(-h) Q is row t + h (mod p) of Q, the imaginary row 0.
    // Every load of a column is issued before any of them is used.
    V dp[R], hl[P];
#pragma unroll
    for (int r = 0; r < R; ++r) dp[r] = read_p ? ld_col<V>(col + N * ss + r * rs) : vzero<V>();
    const uint32_t h = (EXT ? static_cast<uint32_t>(P) : N) % static_cast<uint32_t>(P);
#pragma unroll
    for (int t = 0; t < P; ++t) {
        uint32_t row = static_cast<uint32_t>(t) + h;
        if (row >= static_cast<uint32_t>(P)) row -= P;
        hl[t] = (read_q && row < static_cast<uint32_t>(R)) ? ld_col<V>(col + (N + 1) * ss + row * rs) : vzero<V>();
    }
    // Horner from the last data strip down (erased strips count as zero)
    V hx[P], ex[R];
#pragma unroll
    for (int r = 0; r < P; ++r) hx[r] = vzero<V>();
#pragma unroll
    for (int r = 0; r < R; ++r) ex[r] = vzero<V>();
    for (int k0 = static_cast<int>(N); k0 > 0; k0 -= KB) {
        V d[KB][R];  // a batch of strips, every row, loads in flight together
#pragma unroll
        for (int q = 0; q < KB; ++q) {
            const int k = k0 - 1 - q;
            const bool live = k >= 0 && static_cast<uint32_t>(k) != a && static_cast<uint32_t>(k) != b;
#pragma unroll
            for (int r = 0; r < R; ++r)
                d[q][r] = live ? ld_col<V>(col + static_cast<uint64_t>(k) * ss + r * rs) : vzero<V>();
        }
#pragma unroll
        for (int q = 0; q < KB; ++q) {
            const int k = k0 - 1 - q;
            if (k < 0) break;
#pragma unroll
            for (int r = 0; r < R; ++r) dp[r] = xr(dp[r], d[q][r]);
            if (EXT && static_cast<uint32_t>(k) >= static_cast<uint32_t>(P)) {
                horner_step<P>(hx, d[q]);
#pragma unroll
                for (int r = 0; r < R; ++r) ex[r] = xr(ex[r], d[q][r]);
            } else {
                horner_step<P>(hl, d[q]);
            }
        }
    }
    // dq (lifted) = Q + sum of w_k d_k over the surviving data strips
    V dq[P];
#pragma unroll
    for (int r = 0; r < P; ++r) dq[r] = hl[r];
    if (EXT) {
        const V top = hx[P - 1];  // x hx: rotate by one
#pragma unroll
        for (int r = P - 1; r >= 1; --r) dq[r] = xr(dq[r], hx[r - 1]);
        dq[0] = xr(dq[0], top);
#pragma unroll
        for (int r = 0; r < R; ++r) dq[r] = xr(dq[r], ex[r]);
    }

    if (deg) {  // the strip alone, to the caller's buffer
        uint8_t *const out = J.aux + s * J.ass + v * static_cast<uint64_t>(sizeof(V));
        if (J.j == N + 1)
            store_folded<P>(out, J.ars, dq);
        else
            store_rows<P>(out, J.ars, dp);
        return;
    }
    V lp[P], t[P], o[P];
    if (a == N) {                     // P and Q (encode)
        store_rows<P>(col + N * ss, rs, dp);
        store_folded<P>(col + (N + 1) * ss, rs, dq);
    } else if (b == N + 1) {          // data a and Q: RAID-5, then Q
        store_rows<P>(col + a * ss, rs, dp);
        lift<P>(dp, lp);
        mul_w<P>(lp, a, t);
#pragma unroll
        for (int r = 0; r < P; ++r) t[r] = xr(t[r], dq[r]);
        store_folded<P>(col + (N + 1) * ss, rs, t);
    } else if (b == N) {              // data a and P: w_a D_a = dQ
        mul_mask<P>(dq, c_col_inv_w[slot][a], o);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const V da = xr(o[r], o[P - 1]);
            st_col(col + a * ss + r * rs, da);
            st_col(col + N * ss + r * rs, xr(dp[r], da));
        }
    } else {                          // two data: (w_a + w_b) D_b = w_a dP + dQ
        lift<P>(dp, lp);
        mul_w<P>(lp, a, t);
#pragma unroll
        for (int r = 0; r < P; ++r) t[r] = xr(t[r], dq[r]);
        mul_mask<P>(t, c_col_inv_pair[slot][a][b], o);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const V db = xr(o[r], o[P - 1]);
            st_col(col + b * ss + r * rs, db);
            st_col(col + a * ss + r * rs, xr(db, dp[r]));
        }
    }
}

template <int P, bool EXT>
__host__ __device__ constexpr int variant_of() {
    return P == 3 ? 0 : P == 5 ? (EXT ? 2 : 1) : 3;
}

template <int P, bool EXT>
using ColVec = uint4;

// Registers: two 256-thread CTAs per SM where the accumulators fit 128
// registers (p = 3, 5), one otherwise.
template <int P, bool EXT>
__host__ __device__ constexpr int col_ctas_per_sm() {
    return (P == 7 || EXT) ? 1 : 2;
}

// One operation over n_stripes stripes of one job: columns strided over the grid.
template <int P, bool EXT>
__global__ void __launch_bounds__(256, col_ctas_per_sm<P, EXT>())
    rcg_column_kernel(const ColJob J, uint64_t n_stripes, uint32_t *status) {
    using V = ColVec<P, EXT>;
    const uint32_t cols = J.vps * static_cast<uint32_t>(16 / sizeof(V));  // lane columns per row
    const uint64_t total = n_stripes * cols;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t u = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; u < total; u += stride) {
        const uint64_t s = u / cols;
        const uint32_t v = static_cast<uint32_t>(u - s * cols);
        column_unit<P, EXT, V>(J, s, v, status);
    }
}

// A batch's columns of one variant: warp w of W takes the contiguous chunks
// (one lane column per lane) whose start falls in [Ct w / W, Ct (w+1) / W) of
// the variant's total cost Ct (rows moved), so every warp moves about the same
// bytes.  The job of its first chunk is found by binary search over the
// variant's ColJob records.  A job's
// 128-byte record is read by the warp in one coalesced load (a word per lane)
// into a per-warp copy in shared memory (kept out of registers, which the
// column needs), and the next two records are prefetched into L1 meanwhile;
// each record holds its job's end chunk, so a switch between small jobs reads
// only records already on their way and makes no dependent global round
// trip.  The
// table is a device buffer, or (IN_PARAMS) the launch's own parameter block,
// which is read through the same generic pointer and needs no prefetch.
template <int P, bool EXT, bool IN_PARAMS>
__device__ __forceinline__ void column_batch_body(const uint8_t *__restrict__ table, uint32_t *status) {
    using V = ColVec<P, EXT>;
    const auto *bh = reinterpret_cast<const BatchHeader *>(table);
    constexpr int g = variant_of<P, EXT>();
    const uint32_t n_runs = bh->col_count[g];
    const uint64_t total = bh->col_chunks[g];
    const auto *runs = reinterpret_cast<const ColJob *>(table + bh->col_items_offset) + bh->col_begin[g];
    const uint32_t lane = threadIdx.x & 31;
    if (n_runs == 0 || total == 0) return;
    const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (blockDim.x >> 5);
    const uint64_t w = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    // Warps split the variant's cost evenly -- the rows its chunks move,
    // (N+2)(p-1) per chunk -- rather than its chunk count: chunk c of job r
    // starts at cost0_r + (c - chunk0_r) (N_r+2)(p-1) and belongs to the warp
    // whose range [A, B) holds that start.  (Equal chunk counts left the
    // busiest warp 13 % above the mean on jobs of N = 3 and 4.)
    const ColJob &last = runs[n_runs - 1];
    const uint64_t cost_total = last.cost0 + (last.chunk_end - last.chunk0) * (last.N + 2ull) * (P - 1);
    const uint64_t A = cost_total * w / warps, B = cost_total * (w + 1) / warps;
    if (A >= B) return;
    // the last job whose cost0 <= A (the first job's is 0)
    uint32_t lo = 0, hi = n_runs;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (runs[mid].cost0 <= A) lo = mid; else hi = mid;
    }
    // the warp's job, its bookkeeping and the table's run list, in shared
    // memory: only the job switch reads them, and the column needs the registers
    struct WarpState {
        ColJob J;
        const ColJob *runs;
        uint64_t next, units, total, B, rows;
        uint32_t r, valid, n_runs;
    };
    __shared__ WarpState ws_all[8];
    WarpState &ws = ws_all[threadIdx.x >> 5];
    if (lane == 0) {
        ws.runs = runs;
        ws.total = total;
        ws.n_runs = n_runs;
        ws.B = B;
    }
    __syncwarp();
    auto load_job = [&](uint32_t r) {
        const ColJob *const rl = ws.runs;
        const uint32_t word = reinterpret_cast<const uint32_t *>(rl + r)[lane];
        if constexpr (!IN_PARAMS) {  // the next two records into L1
            if (lane < 2 && r + 1 + lane < ws.n_runs)
                asm volatile("prefetch.global.L1 [%0];" ::"l"(reinterpret_cast<uint64_t>(rl + r + 1 + lane)));
        }
        __syncwarp();
        reinterpret_cast<uint32_t *>(&ws.J)[lane] = word;
        __syncwarp();
        if (lane == 0) {
            const ColJob &J = ws.J;
            ws.r = r;
            ws.next = J.chunk_end;
            ws.rows = (J.N + 2ull) * (P - 1);
            ws.units = J.n_stripes * J.vps * (16 / sizeof(V));  // lane columns of the job
            // device-side guard: the job is this variant's and its chunks cover it
            const bool valid = J.p == static_cast<uint32_t>(P) && (J.N > static_cast<uint32_t>(P)) == EXT &&
                               J.N >= 1 && ws.units > 0 && J.op <= OP_UPDATE && J.chunk_end > J.chunk0 &&
                               J.chunk_end <= ws.total &&
                               J.chunk_end - J.chunk0 == (ws.units + kColChunk - 1) / kColChunk;
            ws.valid = valid;
            if (!valid && status) atomicOr(status, RCG_DEV_BADJOB);
        }
        __syncwarp();
    };
    load_job(lo);
    // the job's first chunk that starts at or after A
    uint64_t c = ws.J.chunk0 + (A > ws.J.cost0 ? (A - ws.J.cost0 + ws.rows - 1) / ws.rows : 0);
#pragma unroll 1
    for (;; ++c) {
        if (c >= ws.total) break;  // a hard bound, whatever the records hold
        if (c >= ws.next) {
            // the job holding chunk c (bounded by the number of jobs)
            uint32_t r = ws.r;
            uint64_t next = ws.next;
            while (c >= next && r + 1 < ws.n_runs) {
                ++r;
                next = ws.runs[r].chunk_end;  // the record prefetched at the last switch
            }
            if (c >= next) break;
            load_job(r);
        }
        if (c < ws.J.chunk0 || ws.J.cost0 + (c - ws.J.chunk0) * ws.rows >= ws.B) break;  // the next warp's
        if (!ws.valid) continue;
        const uint64_t u = (c - ws.J.chunk0) * kColChunk + lane;
        if (u >= ws.units) continue;
        const uint32_t cols = ws.J.vps * static_cast<uint32_t>(16 / sizeof(V));
        const uint64_t s = u / cols;
        column_unit<P, EXT, V>(ws.J, s, static_cast<uint32_t>(u - s * cols), status);
    }
}

template <int P, bool EXT>
__global__ void __launch_bounds__(256, col_ctas_per_sm<P, EXT>())
    rcg_column_batch(const uint8_t *__restrict__ table, uint32_t *status) {
    column_batch_body<P, EXT, false>(table, status);
}

template <int P, bool EXT, uint32_t SZ>
__global__ void __launch_bounds__(256, col_ctas_per_sm<P, EXT>())
    rcg_column_batch_param(uint32_t *status, const __grid_constant__ ParamTable<SZ> t) {
    column_batch_body<P, EXT, true>(t.bytes, status);
}

template <class K>
int resident_ctas(K kernel, int sm_count) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess) per_sm = 1;
    return sm_count * std::max(per_sm, 1);
}

// Launches made per call ask the occupancy once per kernel (the answer
// depends on the kernel only), keyed by the kernel's address: kernels of the
// same signature share a function-pointer type.
template <class K>
int resident_ctas_cached(K kernel, int sm_count) {
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> known;
    const void *key = reinterpret_cast<const void *>(kernel);
    std::lock_guard<std::mutex> lock(mu);
    for (const auto &k : known)
        if (k.first == key) return sm_count * k.second;
    const int per_sm = resident_ctas(kernel, 1);
    known.emplace_back(key, per_sm);
    return sm_count * per_sm;
}

}  // namespace

cudaError_t upload_column_tables() {
    static uint32_t inv_w[kColPrimes][kColMaxN];
    static uint32_t inv_pair[kColPrimes][kColMaxN][kColMaxN];
    static std::once_flag built;
    std::call_once(built, [] {
        memset(inv_w, 0, sizeof(inv_w));
        memset(inv_pair, 0, sizeof(inv_pair));
        const uint32_t primes[kColPrimes] = {3, 5, 7};
        for (int t = 0; t < kColPrimes; ++t) {
            const uint32_t p = primes[t], n_max = max_data_strips(p);
            auto weight = [&](uint32_t k) -> uint64_t {  // reduced modulo f
                if (k < p) return ring_reduce(p, 1ull << k);
                return ring_reduce(p, 1ull ^ (1ull << (k - p + 1)));
            };
            for (uint32_t a = 0; a < n_max; ++a) {
                inv_w[t][a] = static_cast<uint32_t>(ring_inverse(p, weight(a)));
                for (uint32_t b = a + 1; b < n_max; ++b)
                    inv_pair[t][a][b] = static_cast<uint32_t>(ring_inverse(p, weight(a) ^ weight(b)));
            }
        }
    });
    cudaError_t e = cudaMemcpyToSymbol(c_col_inv_w, inv_w, sizeof(inv_w));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_col_inv_pair, inv_pair, sizeof(inv_pair));
    return e;
}

cudaError_t launch_column(const ColJob &job, uint32_t p, uint64_t n_stripes, uint32_t *status, int sm_count,
                          cudaStream_t stream) {
    const uint64_t total = n_stripes * job.vps;
    if (total == 0) return cudaSuccess;
    auto go = [&](auto kernel) -> cudaError_t {
        const uint64_t resident = static_cast<uint64_t>(resident_ctas_cached(kernel, sm_count));
        const unsigned g = static_cast<unsigned>(std::min<uint64_t>((total + 255) / 256, resident));
        kernel<<<g, 256, 0, stream>>>(job, n_stripes, status);
        return cudaGetLastError();
    };
    const bool ext = job.N > p;
    switch (p) {
        case 3: return go(rcg_column_kernel<3, false>);
        case 5: return ext ? go(rcg_column_kernel<5, true>) : go(rcg_column_kernel<5, false>);
        case 7: return go(rcg_column_kernel<7, false>);
        default: return cudaErrorInvalidValue;
    }
}

const void *column_batch_function(int variant) {
    switch (variant) {
        case 0: return reinterpret_cast<const void *>(rcg_column_batch<3, false>);
        case 1: return reinterpret_cast<const void *>(rcg_column_batch<5, false>);
        case 2: return reinterpret_cast<const void *>(rcg_column_batch<5, true>);
        case 3: return reinterpret_cast<const void *>(rcg_column_batch<7, false>);
        default: return nullptr;
    }
}

template <uint32_t SZ>
static cudaError_t column_batch_param_sized(int variant, const uint8_t *table_host, size_t bytes, uint32_t *status,
                                           int sm_count, cudaStream_t stream) {
    ParamTable<SZ> t;
    memcpy(t.bytes, table_host, bytes);
    memset(t.bytes + bytes, 0, SZ - bytes);
    auto go = [&](auto kernel) -> cudaError_t {
        kernel<<<resident_ctas_cached(kernel, sm_count), 256, 0, stream>>>(status, t);
        return cudaGetLastError();
    };
    switch (variant) {
        case 0: return go(rcg_column_batch_param<3, false, SZ>);
        case 1: return go(rcg_column_batch_param<5, false, SZ>);
        case 2: return go(rcg_column_batch_param<5, true, SZ>);
        case 3: return go(rcg_column_batch_param<7, false, SZ>);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_column_batch_param(int variant, const uint8_t *table_host, size_t bytes, uint32_t *status,
                                      int sm_count, cudaStream_t stream) {
    if (bytes <= kParamTableSmall)
        return column_batch_param_sized<kParamTableSmall>(variant, table_host, bytes, status, sm_count, stream);
    if (bytes <= kParamTableLarge)
        return column_batch_param_sized<kParamTableLarge>(variant, table_host, bytes, status, sm_count, stream);
    return cudaErrorInvalidValue;
}

cudaError_t launch_column_batch(int variant, const uint8_t *table_dev, uint32_t *status, int sm_count,
                                cudaStream_t stream) {
    auto go = [&](auto kernel) -> cudaError_t {
        kernel<<<resident_ctas(kernel, sm_count), 256, 0, stream>>>(table_dev, status);
        return cudaGetLastError();
    };
    switch (variant) {
        case 0: return go(rcg_column_batch<3, false>);
        case 1: return go(rcg_column_batch<5, false>);
        case 2: return go(rcg_column_batch<5, true>);
        case 3: return go(rcg_column_batch<7, false>);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rcg
