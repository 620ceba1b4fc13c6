// rcg_horizontal.cu -- the code on stripes in the horizontal representation
// of Section 4.5: one ring element per (p-1)-bit lane of a machine word.  For
// p = 17 a 16-bit word holds y_0..y_15, the coefficients of x^0..x^15 (bit r
// = coefficient of x^r); for p = 5 a nibble, for p = 3 two bits.  Element e of
// a strip is the little-endian bit field [e(p-1), (e+1)(p-1)) of the strip.
//
// Arithmetic.  Multiplication by x^k is the word formula of Section 4.6,
//     x^k y = (y << k) ^ (y >> (p - k)) ^ (bit p-1-k of y ? all ones : 0),
// shifts within the lane (the right shift logical), done lane-wise on 32-bit
// registers (SWAR): per-lane masks keep the shifted bits inside their lane and
// the sign bit is spread over its lane by a multiply.  x itself (k = 1) is
// Section 4.5's doubling with the sign mask.
//
// Kernel.  A thread owns one 16-byte column of a stripe (8 elements at
// p = 17) and streams it through every strip with coalesced 16-byte loads,
// four strips in flight, four 256-thread CTAs per SM; shared memory holds only
// the product tables of a recovery's inverse (p = 17).  Q is
// accumulated by Horner's rule over the data strips from the last to the
// first (Section 4.2, Q = d + g Q),
// a second Horner sum covering the extended strips k >= p of equation (qext)
// (weights 1 + x^(k-p+1)).  Lemma 3.1.2's four cases then need, per erasure
// pair, at most one multiplication by an inverse -- of w_i (data + P) or of
// w_i + w_j (two data strips) -- by its exponent mask, precomputed on the host
// for every pair and kept in constant memory.  The erased strips are never
// read and are written in place.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/rcg.h"
#include "rcg_internal.h"

namespace rcg {

namespace {

constexpr int kHPrimes = 3;          // p = 3, 5, 17
constexpr int kHMaxN = 2 * 17 - 1;   // data strips at most (p = 17, extended)

// Inverse masks per prime slot: w_k^(-1) and (w_a + w_b)^(-1), reduced
// modulo f (bits 0..p-2).  Slot 0: p = 3, 1: p = 5, 2: p = 17.
__constant__ uint32_t c_h_inv_w[kHPrimes][kHMaxN];
__constant__ uint32_t c_h_inv_pair[kHPrimes][kHMaxN][kHMaxN];

struct HParams {
    uint8_t *base;
    const uint8_t *pairs;      // per-stripe (i, j), or nullptr: use i, j
    uint64_t strip_stride, stripe_stride;
    uint64_t n_stripes;
    uint32_t vps;              // 16-byte vectors per strip
    uint32_t N, i, j;
    uint32_t *status;
    uint32_t contiguous;       // 1: each CTA walks a contiguous range of blocks; 0: blocks interleaved
};

template <int E>
struct Lanes {
    static constexpr int P = E + 1;
    static constexpr uint32_t LSB = E == 16 ? 0x00010001u : E == 4 ? 0x11111111u : 0x55555555u;
    static constexpr uint32_t LANE = (1u << E) - 1;

    // x * y, lane-wise (Section 4.5): shift up by one, bit 0 takes the old top bit,
    // and a set top bit flips the whole lane.
    static __device__ __forceinline__ uint32_t mulx(uint32_t y) {
        return ((y << 1) & ~LSB) ^ (((y >> (E - 1)) & LSB) * LANE);
    }
    // x^k * y, 0 <= k <= E, lane-wise (Section 4.6).
    static __device__ __forceinline__ uint32_t mulxk(uint32_t y, uint32_t k) {
        if (k == 0) return y;
        const uint32_t below_k = ((1u << k) - 1) * LSB;         // lane bits < k
        const uint32_t below_k1 = ((1u << (k - 1)) - 1) * LSB;  // lane bits < k-1
        uint32_t r = (y << k) & ~below_k;
        r ^= (y >> (E + 1 - k)) & below_k1;
        r ^= ((y >> (E - k)) & LSB) * LANE;
        return r;
    }
};

// 16-bit lanes: the sign of each lane spreads over the lane with one byte
// permute (prmt's sign-replicating selectors: bytes 0-1 take the sign of
// byte 1, bytes 2-3 the sign of byte 3), so x y is three instructions.
__device__ __forceinline__ uint32_t lane_signs16(uint32_t y) {
    uint32_t r;
    asm("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(r) : "r"(y));
    return r;
}

template <>
__device__ __forceinline__ uint32_t Lanes<16>::mulx(uint32_t y) {
    return ((y << 1) & 0xFFFEFFFEu) ^ lane_signs16(y);
}

template <>
__device__ __forceinline__ uint32_t Lanes<16>::mulxk(uint32_t y, uint32_t k) {
    if (k == 0) return y;
    const uint32_t below_k = ((1u << k) - 1) * LSB;
    const uint32_t below_k1 = ((1u << (k - 1)) - 1) * LSB;
    // the bit p-1-k = 16-k of each lane is the top bit of that lane of y << (k-1)
    return ((y << k) & ~below_k) ^ ((y >> (17 - k)) & below_k1) ^ lane_signs16(y << (k - 1));
}

__device__ __forceinline__ uint4 x4(uint4 a, uint4 b) {
    return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
}

template <int E>
__device__ __forceinline__ uint4 mulx4(uint4 v) {
    using L = Lanes<E>;
    return make_uint4(L::mulx(v.x), L::mulx(v.y), L::mulx(v.z), L::mulx(v.w));
}

template <int E>
__device__ __forceinline__ uint4 mulxk4(uint4 v, uint32_t k) {
    using L = Lanes<E>;
    return make_uint4(L::mulxk(v.x, k), L::mulxk(v.y, k), L::mulxk(v.z, k), L::mulxk(v.w, k));
}

// sum over the mask's exponents m of x^m v
template <int E>
__device__ __forceinline__ uint4 mulmask4(uint4 v, uint32_t mask) {
    uint4 acc = make_uint4(0, 0, 0, 0);
    while (mask) {
        const uint32_t m = __ffs(mask) - 1;
        mask &= mask - 1;
        acc = x4(acc, mulxk4<E>(v, m));
    }
    return acc;
}

// w_k * v: x^k (k < p) or (1 + x^(k-p+1)) (equation qext)
template <int E>
__device__ __forceinline__ uint4 mulw4(uint4 v, uint32_t k) {
    constexpr uint32_t P = E + 1;
    if (k < P) return mulxk4<E>(v, k);
    return x4(v, mulxk4<E>(v, k - P + 1));
}

__device__ __forceinline__ uint4 ldg_stream(const uint8_t *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ void stg4(uint8_t *p, uint4 v) {
    asm volatile("st.global.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

constexpr int kBatch = 4;  // strips whose loads are in flight together (measured best with 4 CTAs per SM)

// Multiplication of 16-bit elements by a fixed ring element through two
// 256-entry tables of its products (low byte, high byte): R is linear over
// GF(2), so c*y = c*(y & 0xff) + c*(y & 0xff00).  Four table reads per 32-bit
// word instead of about nine lane-wise x^m.
__device__ __forceinline__ uint32_t tab_mul(const uint32_t (&tab)[2][256], uint32_t y) {
    const uint32_t lo = tab[0][y & 0xffu] ^ tab[1][(y >> 8) & 0xffu];
    const uint32_t hi = tab[0][(y >> 16) & 0xffu] ^ tab[1][y >> 24];
    return lo | (hi << 16);
}

__device__ __forceinline__ uint4 tab_mul4(const uint32_t (&tab)[2][256], uint4 v) {
    return make_uint4(tab_mul(tab, v.x), tab_mul(tab, v.y), tab_mul(tab, v.z), tab_mul(tab, v.w));
}

// EXT: the layout has extended strips (N > p); without them the second
// Horner sum and its registers drop out.
//
// Work: 256-column blocks (a block lies in one stripe), a thread one 16-byte
// column of a block.  At p = 17 the inverse a recovery multiplies by (per
// stripe, uniform over a block) goes into the CTA's shared-memory product
// tables, rebuilt only when it changes; for such launches a CTA takes a
// contiguous range of blocks, so consecutive blocks mostly share a stripe.
template <int E, bool EXT>
__global__ void __launch_bounds__(256, 4) rcg_h_kernel(const HParams prm) {
    constexpr uint32_t P = E + 1;
    constexpr int slot = E == 2 ? 0 : E == 4 ? 1 : 2;
    constexpr bool TABLES = E == 16;
    __shared__ uint32_t tab[2][256];
    uint32_t key = 0;  // the multiplier the tables hold (0: none); the same in every thread
    const uint32_t N = prm.N;
    const uint32_t bps = (prm.vps + 255) / 256;  // blocks per stripe
    const uint64_t blocks = prm.n_stripes * bps;
    // contiguous ranges keep a CTA on one stripe (and its tables) for several
    // blocks; launches that need no tables interleave blocks over the CTAs,
    // which streams a little better
    const uint64_t per = (blocks + gridDim.x - 1) / gridDim.x;
    const uint64_t first = prm.contiguous ? blockIdx.x * per : blockIdx.x;
    const uint64_t last = prm.contiguous ? (first + per < blocks ? first + per : blocks) : blocks;
    const uint64_t step = prm.contiguous ? 1 : gridDim.x;
    for (uint64_t blk = first; blk < last; blk += step) {
        const uint64_t s = blk / bps;
        const uint32_t v = static_cast<uint32_t>(blk - s * bps) * 256 + threadIdx.x;
        uint32_t a = prm.i, b = prm.j;
        if (prm.pairs) {
            a = prm.pairs[2 * s];
            b = prm.pairs[2 * s + 1];
        }
        if (!(a < b && b <= N + 1)) {  // uniform over the block
            if (v == 0 && prm.status) atomicOr(prm.status, RCG_DEV_BADPAIR);
            continue;
        }
        // the inverse this stripe needs: of w_a (data + P) or of w_a + w_b (two data)
        const uint32_t mul = (b == N) ? c_h_inv_w[slot][a] : (b < N) ? c_h_inv_pair[slot][a][b] : 0u;
        if (TABLES && mul != 0 && mul != key) {
            __syncthreads();  // every read of the old tables is done
            const uint32_t t = threadIdx.x;
            tab[0][t] = mulmask4<E>(make_uint4(t, 0, 0, 0), mul).x;
            tab[1][t] = mulmask4<E>(make_uint4(t << 8, 0, 0, 0), mul).x;
            __syncthreads();
            key = mul;
        }
        if (v >= prm.vps) continue;
        uint8_t *const col = prm.base + s * prm.stripe_stride + v * 16ull;
        const uint64_t ss = prm.strip_stride;
        // the surviving parities, in flight while the data strips stream
        const bool read_p = a != N && b != N, read_q = a != N + 1 && b != N + 1;
        uint4 pv = make_uint4(0, 0, 0, 0), qv = make_uint4(0, 0, 0, 0);
        if (read_p) pv = ldg_stream(col + N * ss);
        if (read_q) qv = ldg_stream(col + (N + 1) * ss);

        // Horner from the last data strip down: hx = sum_{k>=p} x^(k-p) d_k,
        // ex = sum_{k>=p} d_k, hl = sum_{k<p} x^k d_k; dp = sum d_k.  Erased
        // strips count as zero.
        uint4 hl = make_uint4(0, 0, 0, 0), hx = hl, ex = hl, dp = hl;
        for (int k0 = static_cast<int>(N); k0 > 0; k0 -= kBatch) {
            uint4 d[kBatch];
#pragma unroll
            for (int q = 0; q < kBatch; ++q) {
                const int k = k0 - 1 - q;
                d[q] = make_uint4(0, 0, 0, 0);
                if (k >= 0 && static_cast<uint32_t>(k) != a && static_cast<uint32_t>(k) != b)
                    d[q] = ldg_stream(col + static_cast<uint64_t>(k) * ss);
            }
#pragma unroll
            for (int q = 0; q < kBatch; ++q) {
                const int k = k0 - 1 - q;
                if (k < 0) break;
                dp = x4(dp, d[q]);
                if (EXT && static_cast<uint32_t>(k) >= P) {
                    hx = x4(mulx4<E>(hx), d[q]);
                    ex = x4(ex, d[q]);
                } else {
                    hl = x4(mulx4<E>(hl), d[q]);
                }
            }
        }
        uint4 dq = hl;  // sum of w_k d_k over the survivors
        if (EXT) dq = x4(x4(dq, ex), mulx4<E>(hx));
        dp = x4(dp, pv);
        dq = x4(dq, qv);

        if (a == N) {                      // P and Q (encode)
            stg4(col + N * ss, dp);
            stg4(col + (N + 1) * ss, dq);
        } else if (b == N + 1) {           // data a and Q: RAID-5, then Q
            stg4(col + a * ss, dp);
            stg4(col + (N + 1) * ss, x4(dq, mulw4<E>(dp, a)));
        } else if (b == N) {               // data a and P: w_a D_a = dQ
            const uint4 da = TABLES ? tab_mul4(tab, dq) : mulmask4<E>(dq, mul);
            stg4(col + a * ss, da);
            stg4(col + N * ss, x4(dp, da));
        } else {                           // two data: (w_a + w_b) D_b = w_a dP + dQ
            const uint4 t = x4(mulw4<E>(dp, a), dq);
            const uint4 db = TABLES ? tab_mul4(tab, t) : mulmask4<E>(t, mul);
            stg4(col + b * ss, db);
            stg4(col + a * ss, x4(db, dp));
        }
    }
}

}  // namespace

int h_prime_slot(uint32_t p) { return p == 3 ? 0 : p == 5 ? 1 : p == 17 ? 2 : -1; }

cudaError_t upload_h_tables() {
    static uint32_t inv_w[kHPrimes][kHMaxN];
    static uint32_t inv_pair[kHPrimes][kHMaxN][kHMaxN];
    static std::once_flag built;
    std::call_once(built, [] {
        memset(inv_w, 0, sizeof(inv_w));
        memset(inv_pair, 0, sizeof(inv_pair));
        const uint32_t primes[kHPrimes] = {3, 5, 17};
        for (int t = 0; t < kHPrimes; ++t) {
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
    cudaError_t e = cudaMemcpyToSymbol(c_h_inv_w, inv_w, sizeof(inv_w));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_h_inv_pair, inv_pair, sizeof(inv_pair));
    return e;
}

cudaError_t launch_h(uint8_t *base, uint32_t p, uint32_t N, uint64_t strip_bytes, uint64_t strip_stride,
                     uint64_t stripe_stride, uint64_t n_stripes, uint32_t i, uint32_t j, const uint8_t *pairs,
                     uint32_t *status, int sm_count, cudaStream_t stream) {
    HParams prm;
    prm.base = base;
    prm.pairs = pairs;
    prm.strip_stride = strip_stride;
    prm.stripe_stride = stripe_stride;
    prm.n_stripes = n_stripes;
    prm.vps = static_cast<uint32_t>(strip_bytes / 16);
    prm.N = N;
    prm.i = i;
    prm.j = j;
    prm.status = status;
    // product tables are used by per-stripe pairs and by fixed two-data or data + P pairs
    prm.contiguous = (pairs != nullptr || (i < N && j <= N)) ? 1u : 0u;
    const uint64_t total = n_stripes * prm.vps;
    if (total == 0) return cudaSuccess;
    // a resident grid (every block of the grid-stride loop runs from the start)
    auto go = [&](auto kernel) -> cudaError_t {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0);
        if (e != cudaSuccess) return e;
        const uint64_t resident = static_cast<uint64_t>(sm_count) * static_cast<uint64_t>(std::max(per_sm, 1));
        const uint64_t blocks = n_stripes * ((prm.vps + 255) / 256);
        const unsigned g = static_cast<unsigned>(std::min<uint64_t>(blocks, resident));
        kernel<<<g, 256, 0, stream>>>(prm);
        return cudaGetLastError();
    };
    const bool ext = N > p;
    switch (p) {
        case 3: return go(rcg_h_kernel<2, false>);  // 3 has no extension
        case 5: return ext ? go(rcg_h_kernel<4, true>) : go(rcg_h_kernel<4, false>);
        case 17: return ext ? go(rcg_h_kernel<16, true>) : go(rcg_h_kernel<16, false>);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rcg
