// rcg_h257.cu -- Z_257 (Section 3.4) in the horizontal representation of
// Section 4.5: one ring element of R = F2[x]/(1 + x + ... + x^256) per 256-bit
// (32-byte) field of a strip, little-endian, bit r = coefficient of x^r.
//
// A thread owns one element of a stripe (eight 32-bit words in registers) and
// streams it through every strip with one 32-byte load per strip (a warp reads
// 1 KB contiguous), four strips in flight.  Q is Horner's rule over the data
// strips from the last to the first (Section 4.2), Q = d + x Q, where x y is
// Section 4.5's doubling with the sign spread: a one-bit funnel shift across
// the eight words and, when bit 255 was set, all 256 bits flipped.
//
// x^m y for a run-time m (the rotations a recovery needs) is Section 4.6's
// word formula on 256 bits, (y << m) ^ (y >> (257 - m)) ^ (bit 256-m of y ?
// all ones : 0), with the word part of each shift chosen by a switch on m/32
// (m is the same for a whole block: a block lies in one stripe).
//
// Recovery follows Lemma 3.1.2.  Two data strips a < b, z = b - a: the
// system (x^a + x^b) D_b = x^a dP + dQ times x^(-a) is (1 + x^z) D_b = T,
// T = dP + x^(-a) dQ.  Lemma 3.3.1 gives R = GF(2^16)^16 (ord_257(2) = 16),
// so the Frobenius map u -> u^2 has order 16 and, since 2^8 = -1 mod 257,
// (1 + x^z)^(2^8) = 1 + x^(-z) = x^(-z) (1 + x^z): (1 + x^z)^255 = x^(-z) and
//     (1 + x^z)^(-1) = x^z (1 + x^z)^254 = x^z prod_{k=1}^{7} (1 + x^(2^k z)).
// So D_b is seven "add a rotated copy" steps and one rotation -- not the 129
// terms of Section 4.6's closed form -- and D_a = D_b + dP.  Data a and P:
// D_a = x^(-a) dQ.  Data a and Q: D_a = dP (RAID-5), then Q.  P and Q: encode.
// Base code only (N <= 257).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/rcg.h"
#include "rcg_internal.h"

namespace rcg {

namespace {

constexpr uint32_t kP = 257;
constexpr int kWords = 8;        // 32-bit words of an element
constexpr int kBatch257 = 4;     // strips whose loads are in flight together

struct H257Params {
    uint8_t *base;
    const uint16_t *pairs;       // per-stripe (i, j) as 16-bit numbers, or nullptr: use i, j
    uint64_t strip_stride, stripe_stride;
    uint64_t n_stripes;
    uint32_t eps;                // elements (32 bytes) per strip
    uint32_t N, i, j;
    uint32_t *status;
};

struct El {
    uint32_t w[kWords];
};

__device__ __forceinline__ El zero_el() {
    El e;
#pragma unroll
    for (int i = 0; i < kWords; ++i) e.w[i] = 0;
    return e;
}

__device__ __forceinline__ El ld_el(const uint8_t *p) {
    El e;
    asm volatile("ld.global.nc.L1::no_allocate.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(e.w[0]), "=r"(e.w[1]), "=r"(e.w[2]), "=r"(e.w[3]), "=r"(e.w[4]), "=r"(e.w[5]),
                   "=r"(e.w[6]), "=r"(e.w[7])
                 : "l"(p));
    return e;
}

__device__ __forceinline__ void st_el(uint8_t *p, const El &e) {
    asm volatile("st.global.v8.u32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(e.w[0]), "r"(e.w[1]),
                 "r"(e.w[2]), "r"(e.w[3]), "r"(e.w[4]), "r"(e.w[5]), "r"(e.w[6]), "r"(e.w[7])
                 : "memory");
}

__device__ __forceinline__ El xor_el(const El &a, const El &b) {
    El e;
#pragma unroll
    for (int i = 0; i < kWords; ++i) e.w[i] = a.w[i] ^ b.w[i];
    return e;
}

// x y + d (Section 4.5): shift up one bit across the words; bit 255 set
// flips the whole element.
__device__ __forceinline__ El mulx_add(const El &y, const El &d) {
    const uint32_t sign = static_cast<uint32_t>(static_cast<int32_t>(y.w[kWords - 1]) >> 31);
    El e;
#pragma unroll
    for (int i = kWords - 1; i >= 1; --i) e.w[i] = __funnelshift_l(y.w[i - 1], y.w[i], 1) ^ sign ^ d.w[i];
    e.w[0] = (y.w[0] << 1) ^ sign ^ d.w[0];
    return e;
}

// Bits of y << (32 Q + r) at words 0..8 (word 8 = bits 256..287), r < 32.
template <int Q>
__device__ __forceinline__ void shl_words(const El &y, uint32_t r, uint32_t (&o)[kWords + 1]) {
#pragma unroll
    for (int i = 0; i <= kWords; ++i) {
        const int hi = i - Q, lo = i - Q - 1;
        const uint32_t h = (hi >= 0 && hi < kWords) ? y.w[hi] : 0u;
        const uint32_t l = (lo >= 0 && lo < kWords) ? y.w[lo] : 0u;
        o[i] = __funnelshift_l(l, h, r);
    }
}

// Words 0..7 of y >> (32 Q + r), r < 32.
template <int Q>
__device__ __forceinline__ void shr_words(const El &y, uint32_t r, uint32_t (&o)[kWords]) {
#pragma unroll
    for (int i = 0; i < kWords; ++i) {
        const int lo = i + Q, hi = i + Q + 1;
        const uint32_t l = lo < kWords ? y.w[lo] : 0u;
        const uint32_t h = hi < kWords ? y.w[hi] : 0u;
        o[i] = __funnelshift_r(l, h, r);
    }
}

__device__ __forceinline__ void shl_any(const El &y, uint32_t m, uint32_t (&o)[kWords + 1]) {
    const uint32_t r = m & 31;
    switch (m >> 5) {
        case 0: shl_words<0>(y, r, o); break;
        case 1: shl_words<1>(y, r, o); break;
        case 2: shl_words<2>(y, r, o); break;
        case 3: shl_words<3>(y, r, o); break;
        case 4: shl_words<4>(y, r, o); break;
        case 5: shl_words<5>(y, r, o); break;
        case 6: shl_words<6>(y, r, o); break;
        case 7: shl_words<7>(y, r, o); break;
        default: shl_words<8>(y, r, o); break;
    }
}

__device__ __forceinline__ void shr_any(const El &y, uint32_t m, uint32_t (&o)[kWords]) {
    const uint32_t r = m & 31;
    switch (m >> 5) {
        case 0: shr_words<0>(y, r, o); break;
        case 1: shr_words<1>(y, r, o); break;
        case 2: shr_words<2>(y, r, o); break;
        case 3: shr_words<3>(y, r, o); break;
        case 4: shr_words<4>(y, r, o); break;
        case 5: shr_words<5>(y, r, o); break;
        case 6: shr_words<6>(y, r, o); break;
        case 7: shr_words<7>(y, r, o); break;
        default: shr_words<8>(y, r, o); break;
    }
}

// x^m y, 0 <= m < 257 (Section 4.6's word formula on 256 bits): bit 256-m of
// y is the bit that y << m pushes to position 256.
__device__ __forceinline__ El rot(const El &y, uint32_t m) {
    if (m == 0) return y;
    uint32_t l[kWords + 1], h[kWords];
    shl_any(y, m, l);
    shr_any(y, kP - m, h);
    const uint32_t fold = 0u - (l[kWords] & 1u);
    El e;
#pragma unroll
    for (int i = 0; i < kWords; ++i) e.w[i] = l[i] ^ h[i] ^ fold;
    return e;
}

// Blocks of 256 elements of one strip position of one stripe, interleaved
// over a resident grid.
__global__ void __launch_bounds__(256, 3) rcg_h257_kernel(const H257Params prm) {
    const uint32_t N = prm.N;
    const uint32_t bps = (prm.eps + 255) / 256;  // blocks of 256 elements per strip
    const uint64_t blocks = prm.n_stripes * bps;
    for (uint64_t blk = blockIdx.x; blk < blocks; blk += gridDim.x) {
        const uint64_t s = blk / bps;
        const uint32_t e = static_cast<uint32_t>(blk - s * bps) * 256 + threadIdx.x;
        uint32_t a = prm.i, b = prm.j;
        if (prm.pairs) {
            a = prm.pairs[2 * s];
            b = prm.pairs[2 * s + 1];
        }
        if (!(a < b && b <= N + 1)) {  // uniform over the block
            if (e == 0 && prm.status) atomicOr(prm.status, RCG_DEV_BADPAIR);
            continue;
        }
        if (e >= prm.eps) continue;
        uint8_t *const el = prm.base + s * prm.stripe_stride + e * 32ull;
        const uint64_t ss = prm.strip_stride;
        const bool read_p = a != N && b != N, read_q = a != N + 1 && b != N + 1;
        El dp = read_p ? ld_el(el + N * ss) : zero_el();
        const El qv = read_q ? ld_el(el + (N + 1) * ss) : zero_el();
        // Horner from the last data strip down (erased strips count as zero)
        El hq = zero_el();
        for (int k0 = static_cast<int>(N); k0 > 0; k0 -= kBatch257) {
            El d[kBatch257];
#pragma unroll
            for (int q = 0; q < kBatch257; ++q) {
                const int k = k0 - 1 - q;
                d[q] = (k >= 0 && static_cast<uint32_t>(k) != a && static_cast<uint32_t>(k) != b)
                           ? ld_el(el + static_cast<uint64_t>(k) * ss)
                           : zero_el();
            }
#pragma unroll
            for (int q = 0; q < kBatch257; ++q) {
                if (k0 - 1 - q < 0) break;
                dp = xor_el(dp, d[q]);
                hq = mulx_add(hq, d[q]);
            }
        }
        const El dq = xor_el(hq, qv);  // Q + sum of x^k d_k over the survivors

        if (a == N) {                    // P and Q (encode)
            st_el(el + N * ss, dp);
            st_el(el + (N + 1) * ss, dq);
        } else if (b == N + 1) {         // data a and Q: RAID-5, then Q
            st_el(el + a * ss, dp);
            st_el(el + (N + 1) * ss, xor_el(dq, rot(dp, a)));
        } else if (b == N) {             // data a and P: D_a = x^(-a) dQ
            const El da = rot(dq, a == 0 ? 0u : kP - a);
            st_el(el + a * ss, da);
            st_el(el + N * ss, xor_el(dp, da));
        } else {                         // two data: (1 + x^z) D_b = dP + x^(-a) dQ
            const uint32_t z = b - a;
            El t = xor_el(dp, rot(dq, a == 0 ? 0u : kP - a));
            uint32_t m = z;
#pragma unroll 1
            for (int k = 1; k <= 7; ++k) {   // times (1 + x^(2^k z))
                m = (2 * m) % kP;
                t = xor_el(t, rot(t, m));
            }
            const El db = rot(t, z);
            st_el(el + b * ss, db);
            st_el(el + a * ss, xor_el(db, dp));
        }
    }
}

}  // namespace

cudaError_t launch_h257(uint8_t *base, uint32_t N, uint64_t strip_bytes, uint64_t strip_stride,
                        uint64_t stripe_stride, uint64_t n_stripes, uint32_t i, uint32_t j, const uint16_t *pairs,
                        uint32_t *status, int sm_count, cudaStream_t stream) {
    H257Params prm;
    prm.base = base;
    prm.pairs = pairs;
    prm.strip_stride = strip_stride;
    prm.stripe_stride = stripe_stride;
    prm.n_stripes = n_stripes;
    prm.eps = static_cast<uint32_t>(strip_bytes / 32);
    prm.N = N;
    prm.i = i;
    prm.j = j;
    prm.status = status;
    const uint64_t blocks = n_stripes * ((prm.eps + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    auto go = [&](auto kernel) -> cudaError_t {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0);
        if (e != cudaSuccess) return e;
        const uint64_t resident = static_cast<uint64_t>(sm_count) * static_cast<uint64_t>(std::max(per_sm, 1));
        kernel<<<static_cast<unsigned>(std::min<uint64_t>(blocks, resident)), 256, 0, stream>>>(prm);
        return cudaGetLastError();
    };
    return go(rcg_h257_kernel);
}

}  // namespace rcg
