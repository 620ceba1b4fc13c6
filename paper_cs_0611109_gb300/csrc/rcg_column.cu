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
// data strips) -- from a host-computed table of exponent masks.
//
// Why a second kernel: the tile engine streams one strip tile per pipeline
// stage, and at p = 5 with 1 KiB rows a stage is 4 KB, so its fixed cost per
// stage and per tile dominates small launches.  Here a launch is one DRAM
// round trip per thread.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/rcg.h"
#include "rcg_internal.h"

namespace rcg {

namespace {

constexpr int kColPrimes = 3;  // p = 3, 5, 7
constexpr int kColMaxN = 9;    // 2p - 1 for p = 5

__constant__ uint32_t c_col_inv_w[kColPrimes][kColMaxN];
__constant__ uint32_t c_col_inv_pair[kColPrimes][kColMaxN][kColMaxN];

struct ColParams {
    uint8_t *base;
    const uint8_t *pairs;  // per-stripe (i, j), or nullptr: use i, j
    uint64_t row_stride, strip_stride, stripe_stride;
    uint64_t n_stripes;
    uint32_t vps;          // 16-byte columns per row
    uint32_t N, i, j;
    uint32_t *status;
};

__device__ __forceinline__ uint4 xr(uint4 a, uint4 b) {
    return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
}

__device__ __forceinline__ uint4 zero4() { return make_uint4(0, 0, 0, 0); }

__device__ __forceinline__ uint4 ld_col(const uint8_t *p) {
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
template <int P>
__device__ __forceinline__ void horner_step(uint4 (&acc)[P], const uint4 (&d)[P - 1]) {
    const uint4 top = acc[P - 1];
    acc[P - 1] = acc[P - 2];
#pragma unroll
    for (int r = P - 2; r >= 1; --r) acc[r] = xr(acc[r - 1], d[r]);
    acc[0] = xr(top, d[0]);
}

// out += x^m a in the lift, m in [0, p): a rotation of the rows
template <int P, int M = 0>
__device__ __forceinline__ void add_rot(const uint4 (&a)[P], uint32_t m, uint4 (&out)[P]) {
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
template <int P>
__device__ __forceinline__ void mul_w(const uint4 (&a)[P], uint32_t k, uint4 (&out)[P]) {
#pragma unroll
    for (int r = 0; r < P; ++r) out[r] = zero4();
    if (k < static_cast<uint32_t>(P)) {
        add_rot<P>(a, k, out);
    } else {
#pragma unroll
        for (int r = 0; r < P; ++r) out[r] = a[r];
        add_rot<P>(a, k - P + 1, out);
    }
}

// out = (sum over the mask's exponents m of x^m) a
template <int P>
__device__ __forceinline__ void mul_mask(const uint4 (&a)[P], uint32_t mask, uint4 (&out)[P]) {
#pragma unroll
    for (int r = 0; r < P; ++r) out[r] = zero4();
    while (mask) {
        const uint32_t m = __ffs(mask) - 1;
        mask &= mask - 1;
        add_rot<P>(a, m, out);
    }
}

template <int P>
__device__ __forceinline__ void store_folded(uint8_t *strip, uint64_t rs, const uint4 (&a)[P]) {
#pragma unroll
    for (int r = 0; r < P - 1; ++r) st_col(strip + r * rs, xr(a[r], a[P - 1]));
}

template <int P>
__device__ __forceinline__ void store_rows(uint8_t *strip, uint64_t rs, const uint4 (&a)[P - 1]) {
#pragma unroll
    for (int r = 0; r < P - 1; ++r) st_col(strip + r * rs, a[r]);
}

template <int P>
__device__ __forceinline__ void lift(const uint4 (&a)[P - 1], uint4 (&out)[P]) {
#pragma unroll
    for (int r = 0; r < P - 1; ++r) out[r] = a[r];
    out[P - 1] = zero4();
}

// Registers: two 256-thread CTAs per SM where the accumulators fit 128
// registers without spilling (p = 3, 5), one otherwise.
template <int P, bool EXT>
__global__ void __launch_bounds__(256, (P == 7 || EXT) ? 1 : 2) rcg_column_kernel(const ColParams prm) {
    constexpr int R = P - 1;
    constexpr int KB = P == 3 ? 4 : 2;  // strips per batch of loads
    constexpr int slot = P == 3 ? 0 : P == 5 ? 1 : 2;
    const uint32_t N = prm.N;
    const uint64_t rs = prm.row_stride, ss = prm.strip_stride;
    const uint64_t total = prm.n_stripes * prm.vps;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t u = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; u < total; u += stride) {
        const uint64_t s = u / prm.vps;
        const uint32_t v = static_cast<uint32_t>(u - s * prm.vps);
        uint32_t a = prm.i, b = prm.j;
        if (prm.pairs) {
            a = prm.pairs[2 * s];
            b = prm.pairs[2 * s + 1];
        }
        if (!(a < b && b <= N + 1)) {
            if (v == 0 && prm.status) atomicOr(prm.status, RCG_DEV_BADPAIR);
            continue;
        }
        uint8_t *const col = prm.base + s * prm.stripe_stride + v * 16ull;
        const bool read_p = a != N && b != N, read_q = a != N + 1 && b != N + 1;
        uint4 pv[R], qv[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            pv[r] = read_p ? ld_col(col + N * ss + r * rs) : zero4();
            qv[r] = read_q ? ld_col(col + (N + 1) * ss + r * rs) : zero4();
        }
        // Horner from the last data strip down (erased strips count as zero)
        uint4 dp[R], hl[P], hx[P], ex[R];
#pragma unroll
        for (int r = 0; r < P; ++r) hl[r] = hx[r] = zero4();
#pragma unroll
        for (int r = 0; r < R; ++r) dp[r] = ex[r] = zero4();
        for (int k0 = static_cast<int>(N); k0 > 0; k0 -= KB) {
            uint4 d[KB][R];  // a batch of strips, every row, loads in flight together
#pragma unroll
            for (int q = 0; q < KB; ++q) {
                const int k = k0 - 1 - q;
                const bool live = k >= 0 && static_cast<uint32_t>(k) != a && static_cast<uint32_t>(k) != b;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    d[q][r] = live ? ld_col(col + static_cast<uint64_t>(k) * ss + r * rs) : zero4();
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
        // dq (lifted) = sum of w_k d_k over the surviving data strips + Q
        uint4 dq[P];
#pragma unroll
        for (int r = 0; r < P; ++r) dq[r] = hl[r];
        if (EXT) {
            const uint4 top = hx[P - 1];  // x hx: rotate by one
#pragma unroll
            for (int r = P - 1; r >= 1; --r) dq[r] = xr(dq[r], hx[r - 1]);
            dq[0] = xr(dq[0], top);
#pragma unroll
            for (int r = 0; r < R; ++r) dq[r] = xr(dq[r], ex[r]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            dp[r] = xr(dp[r], pv[r]);
            dq[r] = xr(dq[r], qv[r]);
        }

        uint4 lp[P], t[P], o[P];
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
                const uint4 da = xr(o[r], o[P - 1]);
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
                const uint4 db = xr(o[r], o[P - 1]);
                st_col(col + b * ss + r * rs, db);
                st_col(col + a * ss + r * rs, xr(db, dp[r]));
            }
        }
    }
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

cudaError_t launch_column(uint8_t *base, uint32_t p, uint32_t N, uint64_t C, uint64_t row_stride,
                          uint64_t strip_stride, uint64_t stripe_stride, uint64_t n_stripes, uint32_t i, uint32_t j,
                          const uint8_t *pairs, uint32_t *status, int sm_count, cudaStream_t stream) {
    ColParams prm;
    prm.base = base;
    prm.pairs = pairs;
    prm.row_stride = row_stride;
    prm.strip_stride = strip_stride;
    prm.stripe_stride = stripe_stride;
    prm.n_stripes = n_stripes;
    prm.vps = static_cast<uint32_t>(C / 16);
    prm.N = N;
    prm.i = i;
    prm.j = j;
    prm.status = status;
    const uint64_t total = n_stripes * prm.vps;
    if (total == 0) return cudaSuccess;
    auto go = [&](auto kernel) -> cudaError_t {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0);
        if (e != cudaSuccess) return e;
        const uint64_t resident = static_cast<uint64_t>(sm_count) * static_cast<uint64_t>(std::max(per_sm, 1));
        const unsigned g = static_cast<unsigned>(std::min<uint64_t>((total + 255) / 256, resident));
        kernel<<<g, 256, 0, stream>>>(prm);
        return cudaGetLastError();
    };
    const bool ext = N > p;
    switch (p) {
        case 3: return go(rcg_column_kernel<3, false>);
        case 5: return ext ? go(rcg_column_kernel<5, true>) : go(rcg_column_kernel<5, false>);
        case 7: return go(rcg_column_kernel<7, false>);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rcg
