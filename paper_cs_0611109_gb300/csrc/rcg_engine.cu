// rcg_engine.cu -- the tile engine: one persistent, warp-specialised kernel
// that runs every stripe operation of the cyclic-group RAID-6 code
// (Corollary 3.2.4 encode; Lemma 3.1.2 recovery classes; the degraded read and
// the small write) on GB300 (sm_103a).
//
// Data path.  A work unit is a tile: W bytes of columns of one stripe (all
// p-1 rows of every strip it needs).  The producer warp streams the tile's
// strips, one strip per shared-memory ring slot, each with one 4-D tensor copy
// (cp.async.bulk.tensor: a (W/8) x (p-1) box of 8-byte elements; per-row 1-D
// bulk copies where the driver refuses the layout), completion counted on an
// mbarrier.  Consumer warps XOR each slot into register accumulators:
//   accP[r]            ^= strip[r]                      (P, first equation of (znparity))
//   accQ[(r + k) mod p] ^= strip_k[r]                   (x^k d_k in F2[x]/(x^p - 1))
// A consumer owns fixed accumulator rows, so x^k is a read of the slot at the
// row rotated by k: an index remap, no data movement.  Row p-1 of the lift is
// the imaginary row; reducing modulo f = 1 + ... + x^(p-1) XORs it into every
// other row (the "conditional all-ones fold" of Lemma 3.4.1's (powers); the
// EVENODD adjuster).  The epilogue of each tile exchanges rows through shared
// memory and writes the results straight to global memory.
//
// Two-data recovery (Sections 4.3, 4.6): with z = j - i,
//   T   = dP + x^(-i) dQ,     D_j = (1 + x^z)^(-1) T,     D_i = D_j + dP.
// By default the epilogue solves (1 + x^z) D_j = T by one walk along the rows
// p-1, p-1+z, p-1+2z, ... (mod p); the alternative multiplies by
// (1 + x^z)^(-1) = sum_{t=0}^{(p-1)/2} x^(2tz), a per-p host table kept in
// constant memory.
//
// Extended Q-parity (Section 3.3, equation qext).  For primes that satisfy
// Theorem 3.3.3 a stripe may hold up to 2p - 1 data strips; strip k >= p is
// weighted in Q by 1 + x^m, m = k - p + 1.  Such a strip feeds the lifted Q
// accumulator twice (rotations m and 0) -- a second index remap of the same
// slot.  Recovery multiplies the system of Lemma 3.1.2 by a monomial so that
// it keeps the shape (1 + x^z) D = T wherever it can; the one case that
// cannot (one regular and one extended data strip) multiplies T by the
// inverse of a trinomial 1 + x^u + x^v, read from a host-computed table.
//
// Every wait is bounded (mbarrier try_wait against %globaltimer); an expired
// wait sets RCG_DEV_TIMEOUT in the status word and the thread returns after
// the copies it issued have landed.  No trap, no unbounded spin.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/rcg.h"
#include "rcg_internal.h"

namespace rcg {

__constant__ uint64_t c_inv[kMaxP + 1][kMaxP + 1];

// (1 + x^u + x^v)^(-1) for the primes that allow the extension: entry
// c_tri_off[p] + u * p + v of g_tri; c_tri_off[p] = ~0u for the other primes.
constexpr bool odd_prime_c(uint32_t p) {
    if (p < 3 || (p & 1) == 0) return false;
    for (uint32_t d = 3; d * d <= p; d += 2)
        if (p % d == 0) return false;
    return true;
}
constexpr uint32_t tri_entries() {
    uint32_t n = 0;
    for (uint32_t p = 3; p <= static_cast<uint32_t>(kMaxP); ++p)
        if (odd_prime_c(p)) n += p * p;
    return n;
}
constexpr uint32_t kTriEntries = tri_entries();
__constant__ uint32_t c_tri_off[kMaxP + 1];
__device__ uint64_t g_tri[kTriEntries];

namespace {

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait with a suspend-time hint: the thread sleeps until the phase
// completes or the hint (ns) passes, instead of polling.
__device__ __forceinline__ bool mbar_test_sleep(uint32_t bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of `bar` with the given parity to complete, for at most
// timeout_ns.  try_wait itself suspends for a hardware-chosen interval, so
// the loop does not spin hot.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t timeout_ns) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_test_sleep(bar, parity, 100000u)) {
        if (global_ns() - t0 > timeout_ns) return false;
    }
    return true;
}

// L2 policy of the strip-tile loads: normal priority.  Measured on GB300
// against evict-first, whole launches ran 7 % faster on rows whose stride is
// a multiple of 128 bytes and 10-15 % faster on other strides (where two
// neighbouring tiles read the same boundary lines).
__device__ __forceinline__ uint64_t l2_tile_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// 1-D bulk copy global -> shared; completion (bytes) counted on `bar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar), "l"(policy)
        : "memory");
}

// 4-D tiled tensor copy global -> shared (box given by the tensor map),
// completion counted on `bar`.  Coordinates innermost first.
__device__ __forceinline__ void tensor_load_4d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                               int z, int w, uint32_t bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        ".L2::cache_hint [%0], [%1, {%2, %3, %4, %5}], [%6], %7;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar), "l"(policy)
        : "memory");
}

// Bring a tensor map into the TMA unit's descriptor cache ahead of its first use.
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// A batch's tensor maps live in a device table that a copy rewrites before
// each launch, at the same addresses as the previous batch's maps: acquire
// the map through the tensor-map proxy before the TMA unit reads it, so no
// descriptor cached from an earlier batch is used.
__device__ __forceinline__ void acquire_tmap(const CUtensorMap *map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
}

// Bit e of m moved to bit (p - e) mod p, for exponent sets of p bits: the
// exponents of x^(-e).
__device__ __forceinline__ uint64_t reflect_exponents(uint64_t m, uint32_t p) {
    return (m & 1ull) | (__brevll(m & ~1ull) >> (63 - p));
}

__device__ __forceinline__ uint4 xor4(uint4 a, uint4 b) {
    return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
}

// Rows per block of the chain solve's walk (loads in flight together): as
// many as the shape's registers hold without spilling (wide 8, pair 2).
template <class S>
__host__ __device__ constexpr int chain_block() {
    return S::kCtasPerSm == 1 ? 8 : 2;
}

__device__ __forceinline__ uint4 xor3(uint4 a, uint4 b, uint4 c) {
    return make_uint4(a.x ^ b.x ^ c.x, a.y ^ b.y ^ c.y, a.z ^ b.z ^ c.z, a.w ^ b.w ^ c.w);
}

__device__ __forceinline__ uint4 lds(const uint8_t *p) {
    return *reinterpret_cast<const uint4 *>(p);
}

// 16-byte shared-memory load by 32-bit shared address
__device__ __forceinline__ uint4 lds_a(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr));
    return v;
}

__device__ __forceinline__ void sts(uint8_t *p, uint4 v) { *reinterpret_cast<uint4 *>(p) = v; }

__device__ __forceinline__ void sts_a(uint32_t addr, uint4 v) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

__device__ __forceinline__ void stg(uint8_t *p, uint4 v) {
    asm volatile("st.global.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}

// --------------------------------------------------------- slot protocol

enum : uint8_t {
    F_P = 1,      // XOR the slot into the P accumulators
    F_Q = 2,      // XOR the slot, rotated by `rot`, into the lifted Q accumulators
    F_COPY = 4,   // also store the slot to the job's data strip i (small write)
    F_FIRST = 8,  // first slot of a tile
    F_LAST = 16,  // last slot of a tile: run the epilogue after it
    F_Q2 = 32,    // also XOR the slot, rotated by `rot2`, into the lifted Q accumulators
    F_END = 128   // no more tiles for this CTA
};

// Epilogue classes.
enum : uint8_t {
    E_ENC = 0,   // write P = accP, Q = fold(accQ)  (encode, P+Q recovery, small write)
    E_DD = 1,    // two data strips (Section 4.6)
    E_DP = 2,    // data strip i and P
    E_DQ = 3,    // data strip i and Q
    E_DEGP = 4,  // degraded read of a data strip or P: out = accP
    E_DEGQ = 5,  // degraded read of Q: out = fold(accQ)
    E_DDC = 6,   // two data strips, solved by the chain along x^z (same result as E_DD)
    E_DQX = 7,   // extended data strip i and Q: Q = fold(accQ + (1 + x^z) D_i)
    E_DPXC = 8,  // extended data strip i and P: (1 + x^z) D_i = dQ by the chain
    E_DPX = 9    // the same by the table, (1 + x^z)^(-1) dQ
};

// Slot header.  The first 16 bytes are read (one 16-byte load) for every
// slot; the rest -- everything a tile's consumers need, so they never read a
// job descriptor from global memory -- only on a tile's first slot.
struct SlotHdr {
    uint8_t flags;    // F_* bits
    uint8_t rot;      // x^rot for F_Q
    uint16_t w;       // tile width, bytes
    uint32_t off;     // byte offset of the stage in the ring
    uint32_t rot2;    // x^rot2 for F_Q2
    uint32_t pad1;
    uint8_t cls;      // epilogue class
    uint8_t p;
    uint8_t a, b;     // strips the epilogue writes (the erased pair, or i / j of the op)
    uint16_t pitch;   // bytes between rows in the slot (the job's tile width W)
    uint8_t spare;
    uint8_t z;        // chain solves: the z of (1 + x^z); data + Q: the rotation of D_i's weight
    uint64_t base;            // the tile's column c0 of strip 0 of its stripe
    uint64_t strip_stride;
    uint64_t row_stride;
    uint64_t out;             // degraded read: the tile's column of the output;
                              // table solves: the exponent mask of the inverse
    uint64_t out_row_stride;
};
static_assert(sizeof(SlotHdr) == 64, "slot header is 64 bytes");

struct Smem {
    uint64_t *full;   // [kMaxSlots] producer -> consumers (tx-counted)
    uint64_t *empty;  // [kMaxSlots] consumers -> producer
    uint64_t *ep;     // epilogue barrier among consumer warps
    uint8_t *terms;   // table solves: the inverse's reflected exponents, listed (64 bytes)
    SlotHdr *hdr;     // [kMaxSlots]
    uint8_t *xb;      // exchange buffer [p][nvec] x 16 B
    uint8_t *fold;    // two rows [2][nvec] x 16 B, used alternately by successive tiles
    uint8_t *ring;    // byte ring: stages of any size, up to n_slots in flight
};

template <class S>
__device__ __forceinline__ Smem carve(uint8_t *smem) {
    Smem s;
    s.full = reinterpret_cast<uint64_t *>(smem);
    s.empty = s.full + kMaxSlots;
    s.ep = s.empty + kMaxSlots;
    s.terms = smem + 640;  // after the barriers (520 bytes), before the slot headers at 1 KB
    s.hdr = reinterpret_cast<SlotHdr *>(smem + 1024);
    s.xb = smem + kCtlBytes;
    s.fold = s.xb + S::kXBytes;
    s.ring = s.fold + 2 * kFoldBytes;
    return s;
}

__device__ __forceinline__ void set_status(uint32_t *status, uint32_t bits) {
    if (status) atomicOr(status, bits);
}

// Role of strip k (0..N-1 data, N = P, N+1 = Q, N+2 = the small write's new
// strip) in a tile of class `cls` with erased (or replaced) strips a < b:
// returns flags (0 = not read) and the rotations for Q.  Data strip k is
// weighted in Q by x^k (k < p) or 1 + x^(k-p+1) (k >= p, equation qext): one
// or two rotations.  The tile's pre-rotation x^(-s) multiplies every Q weight
// (so the lifted accumulator holds x^(-s) times the sum); with `pone` the data
// weights become 1 + w_k and P feeds Q as well (the accumulator then holds
// x^(-s) (dP + dQ)).
__device__ __forceinline__ uint32_t strip_role(uint8_t cls, bool update, uint32_t k, uint32_t N,
                                               uint32_t a, uint32_t b, uint32_t p, uint32_t s, bool pone,
                                               uint32_t *rot, uint32_t *rot2) {
    *rot = 0;
    *rot2 = 0;
    if (update) {  // old d_a, P, Q, new d_a (last, so d_a is read before it is overwritten)
        if (k == a || k == N + 2) {
            const uint32_t cp = k == N + 2 ? F_COPY : 0u;
            if (a < p) { *rot = a; return F_P | F_Q | cp; }
            *rot = a - p + 1;
            return F_P | F_Q | F_Q2 | cp;  // rot2 = 0
        }
        if (k == N) return F_P;
        if (k == N + 1) return F_Q;
        return 0;
    }
    bool skip_a = true, skip_b = false, read_p = false, read_q = false;
    uint32_t dflags = F_P | F_Q;
    switch (cls) {
        case E_ENC: skip_a = false; break;
        case E_DEGQ: skip_a = false; dflags = F_Q; break;
        case E_DEGP: return (k <= N && k != b) ? F_P : 0u;  // data or P from the first equation
        case E_DQ: case E_DQX: read_p = true; break;
        case E_DP: case E_DPX: case E_DPXC: read_q = true; break;
        default: skip_b = true; read_p = true; read_q = true; break;  // two data strips
    }
    const uint32_t back = s ? p - s : 0u;  // x^(-s), in [0, p)
    if (k < N) {
        if ((skip_a && k == a) || (skip_b && k == b)) return 0;
        // the weight's one or two exponents (1 + w_k when pone)
        const bool ext = k >= p;
        const uint32_t e1 = (ext ? k - p + 1 : k) + back;
        const bool two = ext != pone;  // x^k + 1, or 1 + x^m
        *rot = e1 >= p ? e1 - p : e1;
        if (!two) return dflags;
        *rot2 = back;
        return dflags | F_Q2;
    }
    if (k == N && read_p) {
        if (!pone) return F_P;
        *rot = back;
        return F_P | F_Q;
    }
    if (k == N + 1 && read_q) {
        *rot = back;
        return F_Q;
    }
    return 0;
}

// A batch's jobs follow its table header; a single launch has job0.
__device__ __forceinline__ const Job &job_ref(const LaunchParams &prm, const Job *jobs, uint32_t idx) {
    return jobs ? jobs[idx] : prm.job0;
}

// ---------------------------------------------------------------- producer

// Ring position: slot index and the parity of its current phase.
struct RingPos {
    uint32_t slot = 0, phase = 0;
    __device__ __forceinline__ void next(uint32_t n_slots) {
        if (++slot == n_slots) {
            slot = 0;
            phase ^= 1u;
        }
    }
};

// bh: the batch table (null for single launches), in device memory or, when
// in_params, in the launch's parameter block -- whose tensor maps need no
// acquire (nothing rewrites them while the grid runs) and whose items are
// dealt round-robin (no counter).
template <class S>
__device__ void producer(const LaunchParams &prm, const Smem &sm, const BatchHeader *bh, bool in_params,
                         uint64_t total_units, uint32_t ring_bytes, uint32_t n_slots) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t policy = l2_tile_policy();
    const uint64_t timeout = prm.timeout_ns;
    const uint32_t ring0 = smem_addr(sm.ring);
    // batches: work items (a run of one job's tiles); single launches: one
    // tile per unit; both strided over the grid
    const WorkItem *items =
        bh ? reinterpret_cast<const WorkItem *>(reinterpret_cast<const uint8_t *>(bh) + bh->items_offset)
           : nullptr;
    const Job *jobs = bh ? reinterpret_cast<const Job *>(reinterpret_cast<const uint8_t *>(bh) + sizeof(BatchHeader))
                         : nullptr;
    RingPos pos;
    uint32_t issued = 0;    // stages handed to the consumers
    uint32_t released = 0;  // stages known to be released (all earlier ones are)
    RingPos rel;            // descriptor slot and phase of stage `released`
    uint32_t head = 0;      // next free byte of the ring
    // single launches have one stage size: slot k sits at k * slot bytes
    // fixed slots: single launches, and batches laid out with equal slots;
    // otherwise a byte ring of stages of any size
    const uint32_t fixed_slot = (bh && !bh->fixed_slots) ? 0u : ring_bytes / n_slots;
    bool ok = true;
    uint64_t next_static = blockIdx.x;

    // Batches, static: items u = blockIdx.x, blockIdx.x + grid, ...; dynamic:
    // the next item index comes from the global counter.  Either way the next
    // item's 128 bytes are requested while the current one streams.
    const bool dynamic = bh && bh->dynamic && !in_params;
    auto next_index = [&]() -> uint64_t {
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(prm.tile_counter, 1ull);
        return __shfl_sync(0xffffffffu, v, 0);
    };
    // The next item is held spread over the warp, word `lane` of its 128
    // bytes in each lane (one coalesced load); fields come out by shuffles.
    auto fetch = [&](uint64_t idx) -> uint32_t {
        return reinterpret_cast<const uint32_t *>(items + idx)[lane];
    };
    uint64_t u = items ? (dynamic ? next_index() : blockIdx.x) : 0;
    // Static batches with fewer items than CTAs (small batches): the CTAs
    // b = u, u + n, u + 2n, ... (n items) share item u, each taking every
    // share-th of its tiles, so a small batch still spreads over the grid.
    uint32_t share = 1, share_idx = 0;
    if (items && !dynamic && total_units > 0 && total_units < gridDim.x) {
        const uint32_t n = static_cast<uint32_t>(total_units);
        u = blockIdx.x % n;
        share_idx = blockIdx.x / n;
        share = (gridDim.x - 1 - static_cast<uint32_t>(u)) / n + 1;
    }
    uint32_t nxt = 0;
    if (items && u < total_units) nxt = fetch(u);
    uint32_t acquired = ~0u;  // job whose tensor map this CTA last acquired

    for (;;) {
        // the fields of this unit, in registers
        uint32_t ji, nt, p, N, tps, W, C, n_stripes, op, use_tmap, dd_solve, ji_i, ji_j;
        uint64_t lt0, strip_stride, row_stride, stripe_stride, aux_rs, aux_ss;
        const uint8_t *pairs;
        uint8_t *base, *aux;
        if (items) {
            if (u >= total_units) break;
            const uint32_t cur = nxt;
            u = dynamic ? next_index() : u + gridDim.x;
            if (u < total_units) nxt = fetch(u);  // prefetch
            // word offsets of the WorkItem fields
            auto w32 = [&](int i) { return __shfl_sync(0xffffffffu, cur, i); };
            auto w64 = [&](int i) { return static_cast<uint64_t>(w32(i)) | (static_cast<uint64_t>(w32(i + 1)) << 32); };
            base = reinterpret_cast<uint8_t *>(w64(0));
            aux = reinterpret_cast<uint8_t *>(w64(2));
            pairs = reinterpret_cast<const uint8_t *>(w64(4));
            strip_stride = w64(6); row_stride = w64(8); stripe_stride = w64(10);
            aux_rs = w64(12); aux_ss = w64(14);
            lt0 = w32(16); nt = w32(17); tps = w32(18); W = w32(19); C = w32(20); n_stripes = w32(21);
            ji = w32(22);
            const uint32_t b0 = w32(23), b1 = w32(24);
            p = b0 & 0xffu; N = (b0 >> 8) & 0xffu; op = (b0 >> 16) & 0xffu; ji_i = b0 >> 24;
            ji_j = b1 & 0xffu; use_tmap = (b1 >> 8) & 0xffu; dd_solve = (b1 >> 16) & 0xffu;
        } else {
            if (next_static >= total_units) break;
            ji = 0;
            lt0 = next_static;
            nt = 1;
            next_static += gridDim.x;
            const Job &J0 = prm.job0;
            p = J0.p; N = J0.n; tps = J0.tiles_per_stripe; W = J0.W; C = J0.C; n_stripes = J0.n_stripes;
            op = J0.op; use_tmap = J0.use_tmap; dd_solve = J0.dd_solve; ji_i = J0.i; ji_j = J0.j;
            pairs = J0.pairs; base = J0.base; aux = J0.aux;
            strip_stride = J0.strip_stride; row_stride = J0.row_stride; stripe_stride = J0.stripe_stride;
            aux_rs = J0.aux_row_stride; aux_ss = J0.aux_stripe_stride;
        }
        const Job &J = job_ref(prm, jobs, ji);  // only its tensor map is used, in place
        const uint32_t rows = p - 1;
        if (items && use_tmap && ji != acquired) {
            if (lane == 0 && !in_params) acquire_tmap(&J.tmap);
            acquired = ji;
        }

        for (uint32_t q = share_idx; q < nt && ok; q += share) {
            if (q == share_idx && items && u < total_units) {  // the next item's descriptor
                const uint32_t njob = __shfl_sync(0xffffffffu, nxt, 22);
                const uint32_t ntm = (__shfl_sync(0xffffffffu, nxt, 24) >> 8) & 0xffu;
                if (ntm && njob != acquired) {
                    if (lane == 0 && !in_params) {
                        acquire_tmap(&jobs[njob].tmap);
                        prefetch_tmap(&jobs[njob].tmap);
                    }
                    acquired = njob;
                }
            }
            const uint64_t local = lt0 + q;
            const uint32_t stripe = static_cast<uint32_t>(local / tps);
            const uint32_t c0 = static_cast<uint32_t>(local % tps) * W;
            const uint32_t w = min(W, C - c0);
            // device-side guard: a tile must fit its slot and the item budget
            if (p < 3 || p > kMaxP || N < 1 || N > 2 * p - 1 || (w & 15) || w == 0 || W > kMaxTileBytes ||
                (W & 15) || rows * W > ring_bytes || p * (w >> 4) > static_cast<uint32_t>(S::kMaxItems) ||
                stripe >= n_stripes) {
                if (lane == 0) set_status(prm.status, RCG_DEV_BADJOB);
                continue;
            }

            uint8_t cls = E_ENC;
            uint32_t a = ji_i, b = ji_j;
            uint32_t s = 0;         // pre-rotation x^(-s) of the Q weights
            bool pone = false;      // Q weights 1 + w_k, P feeds Q
            uint32_t z = 0;         // chain: (1 + x^z); data + Q: rotation of D_a's weight
            uint64_t mask = 0;      // table solves: exponents of the inverse
            uint32_t oa, ob;        // strips the epilogue writes
            const bool update = op == OP_UPDATE;
            if (op == OP_RECOVER) {
                if (pairs) {
                    a = pairs[2ull * stripe];
                    b = pairs[2ull * stripe + 1];
                }
                if (!(a < b && b <= N + 1)) {
                    if (lane == 0) set_status(prm.status, RCG_DEV_BADPAIR);
                    continue;
                }
                if (b < N) {  // two data strips: (w_a + w_b) D_b = w_a dP + dQ
                    if (b < p) {           // x^(-a): (1 + x^(b-a)) D_b = dP + x^(-a) dQ
                        s = a;
                        z = b - a;
                        cls = dd_solve ? E_DD : E_DDC;
                    } else if (a >= p) {   // x^(-m_a): (1 + x^(b-a)) D_b = dP + x^(-m_a)(dP + dQ)
                        s = a - p + 1;
                        pone = true;
                        z = b - a;
                        cls = dd_solve ? E_DD : E_DDC;
                    } else {               // x^(-a): (1 + x^(-a) + x^(m_b-a)) D_b = dP + x^(-a) dQ
                        s = a;
                        cls = E_DD;
                        const uint32_t off = c_tri_off[p];
                        const uint32_t u = p - a == p ? 0u : p - a, v = (b - p + 1 + p - a) % p;
                        mask = off == ~0u ? 0ull : g_tri[off + u * p + v];
                        if (mask == 0) {  // p does not allow the extension
                            if (lane == 0) set_status(prm.status, RCG_DEV_BADJOB);
                            continue;
                        }
                    }
                    if (cls == E_DD && z) mask = c_inv[p][z];
                    oa = a;
                    ob = b;
                } else if (a == N) {      // P and Q: encode
                    cls = E_ENC;
                    oa = N;
                    ob = N;
                } else if (b == N) {      // data a and P
                    if (a < p) {
                        cls = E_DP;
                        s = a;
                        oa = a;
                        ob = N;
                    } else {              // (1 + x^m_a) D_a = dQ, P = dP + D_a
                        z = a - p + 1;
                        cls = dd_solve ? E_DPX : E_DPXC;
                        if (dd_solve) mask = c_inv[p][z];
                        oa = N;           // receives D + accP
                        ob = a;           // receives D
                    }
                } else {                  // data a and Q
                    cls = a < p ? E_DQ : E_DQX;
                    z = a < p ? a : a - p + 1;
                    oa = a;
                    ob = N + 1;
                }
            } else if (op == OP_DEGRADED) {
                cls = (b == N + 1) ? E_DEGQ : E_DEGP;
                oa = a;
                ob = b;
            } else {
                if (update && a >= N) {
                    if (lane == 0) set_status(prm.status, RCG_DEV_BADJOB);
                    continue;
                }
                oa = a;
                ob = N;  // P and Q are strips N and N+1
            }
            if (cls == E_ENC) ob = N;

            // chain solves: the rows r_t = p-1 + t z (mod p) at odd positions t
            // of the walk, as a mask (the epilogue adds c to those rows)
            uint64_t odd_rows = 0;
            if (cls == E_DDC || cls == E_DPXC) {
                const uint32_t zz = z % p;
                uint32_t r = p - 1;
                for (uint32_t t = 1; t < p; ++t) {
                    r += zz;
                    if (r >= p) r -= p;
                    if (t & 1u) odd_rows |= 1ull << r;
                }
            }

            // strips streamed per tile: N for every class (the other N survivors,
            // or the N inputs of a rebuild), 4 for the small write
            const uint32_t count = update ? 4u : N;
            uint32_t rot, rot2;

            uint8_t *const stripe_base = base + stripe * stripe_stride + c0;
            const uint8_t *aux_base = aux + stripe * aux_ss + c0;
            // rows sit W bytes apart in a slot; a tensor copy always lands the full
            // W-wide box (columns past C are zero-filled), row copies land w bytes
            const uint32_t tx_tensor = rows * W, tx_rows = rows * w;
            uint32_t emitted = 0;
            for (uint32_t k = 0; k < N + 3; ++k) {
                const uint32_t fl = strip_role(cls, update, k, N, a, b, p, s, pone, &rot, &rot2);
                if (!fl) continue;
                // a free descriptor (its previous stage released) ...
                if (!mbar_wait(smem_addr(&sm.empty[pos.slot]), pos.phase ^ 1u, timeout)) {
                    ok = false;
                    break;
                }
                uint32_t start = pos.slot * fixed_slot;  // single launches: fixed slots
                if (!fixed_slot) {
                    // batches: room for the stage in the byte ring -- the oldest
                    // stages in flight are released, in order, until it fits
                    // after head (or at 0)
                    if (issued >= n_slots && released < issued - n_slots + 1) {  // the descriptor wait released these
                        while (released < issued - n_slots + 1) {
                            ++released;
                            rel.next(n_slots);
                        }
                    }
                    const uint32_t B = (rows * W + 127) & ~127u;
                    // The fewest oldest stages whose release makes room, found
                    // from their offsets alone (where a stage goes does not
                    // depend on when stages finish); then ONE wait, on the last
                    // of them -- releases come in order -- and the copy issues
                    // right after it, as with fixed slots.
                    uint32_t need = released;  // stages [released, need) must be released
                    RingPos scan = rel;        // descriptor slot and phase of stage `need`
                    RingPos last = rel;        // ... of stage need - 1
                    for (;;) {
                        if (need == issued) {  // the ring would be empty
                            start = head + B <= ring_bytes ? head : 0;
                            break;
                        }
                        uint32_t t_off;  // offset of the oldest stage still in flight then
                        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(t_off) : "r"(smem_addr(&sm.hdr[scan.slot].off)));
                        bool fits = false;
                        if (t_off < head) {         // occupied [t_off, head)
                            if (head + B <= ring_bytes) { start = head; fits = true; }
                            else if (B <= t_off) { start = 0; fits = true; }
                        } else if (t_off > head) {  // occupied [t_off, end) and [0, head)
                            if (head + B <= t_off) { start = head; fits = true; }
                        }                           // t_off == head: full
                        if (fits) break;
                        last = scan;
                        ++need;
                        scan.next(n_slots);
                    }
                    if (need > released) {
                        if (!mbar_wait(smem_addr(&sm.empty[last.slot]), last.phase, timeout)) {
                            ok = false;
                            break;
                        }
                        released = need;
                        rel = scan;
                    }
                    head = start + B;
                }
                const uint32_t full = smem_addr(&sm.full[pos.slot]);
                const bool tensor = use_tmap && k < N + 2;
                if (lane == 0) {
                    // hot 16 bytes every stage; the tile part only on its first
                    SlotHdr &h = sm.hdr[pos.slot];
                    const uint32_t first = emitted == 0;
                    const uint32_t fl2 = fl | (first ? F_FIRST : 0) | (emitted + 1 == count ? F_LAST : 0);
                    const uint4 hot = make_uint4(fl2 | (rot << 8) | (w << 16), start, rot2, 0u);
                    *reinterpret_cast<uint4 *>(&h) = hot;
                    if (first) {
                        h.cls = cls;
                        h.p = static_cast<uint8_t>(p);
                        h.a = static_cast<uint8_t>(oa);
                        h.b = static_cast<uint8_t>(ob);
                        h.pitch = static_cast<uint16_t>(W);
                        h.z = static_cast<uint8_t>(z);
                        h.base = reinterpret_cast<uint64_t>(stripe_base);
                        h.strip_stride = strip_stride;
                        h.row_stride = row_stride;
                        // table solves: the inverse's exponents reflected (see the
                        // epilogue); chain solves: the odd positions' rows
                        h.out = (cls == E_DD || cls == E_DPX)     ? reflect_exponents(mask, p)
                                : (cls == E_DDC || cls == E_DPXC) ? odd_rows
                                                                  : reinterpret_cast<uint64_t>(aux_base);
                        h.out_row_stride = aux_rs;
                    }
                    mbar_arrive_tx(full, tensor ? tx_tensor : tx_rows);
                }
                __syncwarp();
                const uint32_t dst = ring0 + start;
                if (tensor) {
                    // one tensor copy: box (W/8 x p-1) at column c0, strip k, stripe
                    if (lane == 0)
                        tensor_load_4d(dst, &J.tmap, static_cast<int>(c0 >> 3), 0, static_cast<int>(k),
                                       static_cast<int>(stripe), full, policy);
                } else {
                    const uint8_t *src = (k == N + 2) ? aux_base : stripe_base + k * strip_stride;
                    const uint64_t rs = (k == N + 2) ? aux_rs : row_stride;
                    for (uint32_t r = lane; r < rows; r += 32)
                        bulk_load(dst + r * W, src + r * rs, w, full, policy);
                }
                pos.next(n_slots);
                ++issued;
                ++emitted;
            }
        }
        if (!ok) break;
    }

    if (ok) {  // end marker
        if (mbar_wait(smem_addr(&sm.empty[pos.slot]), pos.phase ^ 1u, timeout)) {
            if (lane == 0) {
                SlotHdr h = {};
                h.flags = F_END;
                sm.hdr[pos.slot] = h;
                mbar_arrive(smem_addr(&sm.full[pos.slot]));
            }
            pos.next(n_slots);
            ++issued;
        } else {
            ok = false;
        }
    }
    if (!ok && lane == 0) set_status(prm.status, RCG_DEV_TIMEOUT);
    // Do not leave while a bulk copy may still be writing this CTA's shared
    // memory: wait (bounded) for the last use of every slot to complete.
    const uint32_t first = issued > n_slots ? issued - n_slots : 0;
    for (uint32_t s = first; s < issued; ++s)
        if (!mbar_wait(smem_addr(&sm.full[s % n_slots]), (s / n_slots) & 1u, timeout)) {
            if (lane == 0) set_status(prm.status, RCG_DEV_TIMEOUT);
            break;
        }
}

// ---------------------------------------------------------------- consumers

struct Tile {
    uint8_t *base;      // stripe base + c0
    uint8_t *out;       // degraded read output + c0 (stripe applied); table solves: the mask;
                        // chain solves: the rows of odd walk positions
    uint64_t strip_stride, row_stride, out_row_stride;
    uint32_t p, nvec, w;
    uint8_t cls, a, b, z;
};

// Epilogue barrier among the consumer warps (bounded).
__device__ __forceinline__ bool ep_sync(const Smem &sm, uint32_t &phase, uint64_t timeout_ns) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(smem_addr(sm.ep));
    const bool ok = mbar_wait(smem_addr(sm.ep), phase, timeout_ns);
    phase ^= 1u;
    return ok;
}

// Buffer discipline (no barrier on entry): every read of the exchange buffer
// happens before a barrier all consumers pass before the next tile's writes;
// the fold row alternates between two buffers, so a tile's fold writes never
// meet the previous fold-using tile's reads, which sit after its own barrier.
template <class S>
__device__ bool epilogue(const Smem &sm, const Tile &T, const uint4 (&accP)[S::kItems],
                         uint4 (&accQ)[S::kItems], const int (&row)[S::kItems], uint32_t &ep_phase,
                         uint32_t &fold_par, uint64_t timeout_ns) {
    // column of item t: item index minus row * nvec (recomputed, not kept in registers)
    const int ctid = static_cast<int>(threadIdx.x) - 32;
    int col[S::kItems];
#pragma unroll
    for (int t = 0; t < S::kItems; ++t) col[t] = ctid + t * S::kConsumers - row[t] * static_cast<int>(T.nvec);
    const int p = static_cast<int>(T.p);
    const uint32_t nv = T.nvec;
    auto X = [&](uint8_t *buf, int r, int c) { return buf + (static_cast<size_t>(r) * nv + c) * 16; };
    auto strip_row = [&](uint32_t k, int r, int c) {
        return T.base + k * T.strip_stride + static_cast<uint64_t>(r) * T.row_stride + c * 16;
    };
    uint8_t *const fold = sm.fold + fold_par * kFoldBytes;
    if (T.cls != E_DEGP) fold_par ^= 1u;

    switch (T.cls) {
        case E_ENC:
        case E_DEGQ: {
            #pragma unroll
            for (int t = 0; t < S::kItems; ++t)
                if (row[t] == p - 1) sts(fold + col[t] * 16, accQ[t]);
            if (!ep_sync(sm, ep_phase, timeout_ns)) return false;
            #pragma unroll
            for (int t = 0; t < S::kItems; ++t) {
                if (row[t] >= p - 1) continue;
                const uint4 q = xor4(accQ[t], lds(fold + col[t] * 16));
                if (T.cls == E_ENC) {
                    stg(strip_row(T.b, row[t], col[t]), accP[t]);      // P = strip N
                    stg(strip_row(T.b + 1, row[t], col[t]), q);        // Q = strip N+1
                } else {
                    stg(T.out + static_cast<uint64_t>(row[t]) * T.out_row_stride + col[t] * 16, q);
                }
            }
            break;
        }
        case E_DEGP: {
            #pragma unroll
            for (int t = 0; t < S::kItems; ++t)
                if (row[t] < p - 1)
                    stg(T.out + static_cast<uint64_t>(row[t]) * T.out_row_stride + col[t] * 16, accP[t]);
            break;
        }
        case E_DP: {  // accQ = x^(-a) dQ (lifted): D_a = fold(accQ), P = accP + D_a
#pragma unroll
            for (int t = 0; t < S::kItems; ++t)
                if (row[t] == p - 1) sts(fold + col[t] * 16, accQ[t]);
            if (!ep_sync(sm, ep_phase, timeout_ns)) return false;
#pragma unroll
            for (int t = 0; t < S::kItems; ++t) {
                if (row[t] >= p - 1) continue;
                const uint4 d = xor4(accQ[t], lds(fold + col[t] * 16));
                stg(strip_row(T.a, row[t], col[t]), d);
                stg(strip_row(T.b, row[t], col[t]), xor4(accP[t], d));
            }
            break;
        }
        case E_DQ:      // D_a = accP; Q = fold(accQ + x^z D_a), z = a
        case E_DQX: {   // extended a: Q = fold(accQ + (1 + x^z) D_a), z = a - p + 1
            const uint4 zero = make_uint4(0, 0, 0, 0);
            #pragma unroll
            for (int t = 0; t < S::kItems; ++t)
                if (row[t] < p) sts(X(sm.xb, row[t], col[t]), row[t] < p - 1 ? accP[t] : zero);
            if (!ep_sync(sm, ep_phase, timeout_ns)) return false;
            const int z = T.z;
            const bool ext = T.cls == E_DQX;
            #pragma unroll
            for (int t = 0; t < S::kItems; ++t) {
                if (row[t] >= p) continue;
                int s = row[t] - z;
                if (s < 0) s += p;
                accQ[t] = xor4(accQ[t], lds(X(sm.xb, s, col[t])));
                if (ext && row[t] < p - 1) accQ[t] = xor4(accQ[t], accP[t]);
                if (row[t] == p - 1) sts(fold + col[t] * 16, accQ[t]);
            }
            if (!ep_sync(sm, ep_phase, timeout_ns)) return false;
            #pragma unroll
            for (int t = 0; t < S::kItems; ++t) {
                if (row[t] >= p - 1) continue;
                stg(strip_row(T.a, row[t], col[t]), accP[t]);
                stg(strip_row(T.b, row[t], col[t]), xor4(accQ[t], lds(fold + col[t] * 16)));
            }
            break;
        }
        case E_DDC:
        case E_DPXC: {
            // (1 + x^z) D = T in R, T = accP + accQ (two data strips) or accQ
            // (extended data strip + P).  Lifted to F2[x]/(x^p - 1) the
            // solution with D[p-1] = 0 satisfies D[r] + D[r-z] = T[r] + c, where
            // c (the XOR of all p rows of T) makes T + c*f vanish at x = 1.
            // One thread per column walks r_t = p-1 + t z (t = 1..p-1), turning
            // T into its prefix XOR E_t in place; then D[r_t] = E_t + (t odd) c.
            // D goes to strip b, D + accP to strip a.
            const uint4 zero = make_uint4(0, 0, 0, 0);
            const bool tp = T.cls == E_DDC;
#pragma unroll
            for (int t = 0; t < S::kItems; ++t)
                if (row[t] < p)
                    sts(X(sm.xb, row[t], col[t]), (tp && row[t] < p - 1) ? xor4(accP[t], accQ[t]) : accQ[t]);
            if (!ep_sync(sm, ep_phase, timeout_ns)) return false;
            const int z = T.z;
            if (ctid < static_cast<int>(nv)) {
                // the walk in blocks of kB rows: a block's loads are
                // issued together (they never alias its stores), so the walk
                // pays one shared-memory latency per block, not per row
                const uint32_t cell0 = smem_addr(sm.xb) + ctid * 16, row_bytes = nv * 16;
                uint4 e = zero;
                int r = p - 1;
                int t = 1;
                constexpr int kB = chain_block<S>();
                for (; t + kB <= p; t += kB) {
                    uint32_t a[kB];
                    uint4 v[kB];
#pragma unroll
                    for (int q = 0; q < kB; ++q) {
                        r += z;
                        if (r >= p) r -= p;
                        a[q] = cell0 + r * row_bytes;
                        v[q] = lds_a(a[q]);
                    }
#pragma unroll
                    for (int q = 0; q < kB; ++q) {
                        e = xor4(e, v[q]);
                        sts_a(a[q], e);
                    }
                }
                for (; t < p; ++t) {
                    r += z;
                    if (r >= p) r -= p;
                    const uint32_t a = cell0 + r * row_bytes;
                    e = xor4(e, lds_a(a));
                    sts_a(a, e);
                }
                sts(fold + ctid * 16, xor4(e, lds(X(sm.xb, p - 1, ctid))));  // c
            }
            if (!ep_sync(sm, ep_phase, timeout_ns)) return false;
            // D[r_t] = E_t, plus c where the walk position t of the row is odd
            const uint64_t odd_rows = reinterpret_cast<uint64_t>(T.out);
#pragma unroll
            for (int t = 0; t < S::kItems; ++t) {
                if (row[t] >= p - 1) continue;
                uint4 dj = lds(X(sm.xb, row[t], col[t]));
                if ((odd_rows >> row[t]) & 1ull) dj = xor4(dj, lds(fold + col[t] * 16));
                stg(strip_row(T.b, row[t], col[t]), dj);
                stg(strip_row(T.a, row[t], col[t]), xor4(dj, accP[t]));
            }
            break;
        }
        case E_DD:
        case E_DPX: {
            // accQ = x^(-s) dQ (lifted), so T = dP + x^(-s) dQ is formed in place
            // (row p-1 of dP is zero), or T = accQ (extended data strip + P);
            // D_b = c^(-1) T needs every row of T.  The exponent set of c^(-1)
            // -- (1 + x^z)^(-1) of Section 4.6, or a trinomial's inverse --
            // comes in the tile header reflected (e -> p - e): row r of D_b is
            // the XOR of rows (e' + r) mod p of T over the reflected exponents
            // e'.  The consumers list those exponents once per tile; each thread
            // then walks the list once for all its items.
            const uint4 zero = make_uint4(0, 0, 0, 0);
            const bool tp = T.cls == E_DD;
            const uint64_t mref = reinterpret_cast<uint64_t>(T.out) & ((1ull << p) - 1);  // exponents < p
            if (ctid < p && ((mref >> ctid) & 1ull))
                sm.terms[__popcll(mref & ((1ull << ctid) - 1))] = static_cast<uint8_t>(ctid);
#pragma unroll
            for (int t = 0; t < S::kItems; ++t)
                if (row[t] < p)
                    sts(X(sm.xb, row[t], col[t]), (tp && row[t] < p - 1) ? xor4(accP[t], accQ[t]) : accQ[t]);
            if (!ep_sync(sm, ep_phase, timeout_ns)) return false;
            const int n_terms = __popcll(mref);
            const uint32_t row_bytes = nv * 16;
            const uint32_t xb0 = smem_addr(sm.xb);
#pragma unroll
            for (int t = 0; t < S::kItems; ++t) accQ[t] = zero;
            // two exponents per pass: each word takes one three-input XOR for
            // both rows (the product is instruction-bound)
            int k = 0;
            for (; k + 1 < n_terms; k += 2) {
                const int e0 = sm.terms[k], e1 = sm.terms[k + 1];  // the same in every thread
#pragma unroll
                for (int t = 0; t < S::kItems; ++t) {
                    const int r = row[t];
                    if (r >= p) continue;
                    int j0 = e0 + r, j1 = e1 + r;
                    if (j0 >= p) j0 -= p;
                    if (j1 >= p) j1 -= p;
                    accQ[t] = xor3(accQ[t], lds_a(xb0 + j0 * row_bytes + col[t] * 16),
                                   lds_a(xb0 + j1 * row_bytes + col[t] * 16));
                }
            }
            if (k < n_terms) {
                const int e = sm.terms[k];
#pragma unroll
                for (int t = 0; t < S::kItems; ++t) {
                    const int r = row[t];
                    if (r >= p) continue;
                    int j = e + r;
                    if (j >= p) j -= p;
                    accQ[t] = xor4(accQ[t], lds_a(xb0 + j * row_bytes + col[t] * 16));
                }
            }
#pragma unroll
            for (int t = 0; t < S::kItems; ++t)
                if (row[t] == p - 1) sts(fold + col[t] * 16, accQ[t]);
            if (!ep_sync(sm, ep_phase, timeout_ns)) return false;
#pragma unroll
            for (int t = 0; t < S::kItems; ++t) {
                if (row[t] >= p - 1) continue;
                const uint4 dj = xor4(accQ[t], lds(fold + col[t] * 16));
                stg(strip_row(T.b, row[t], col[t]), dj);
                stg(strip_row(T.a, row[t], col[t]), xor4(dj, accP[t]));
            }
            break;
        }
    }
    return true;
}

template <class S>
__device__ void consumer(const LaunchParams &prm, const Smem &sm, uint32_t n_slots) {
    const int ctid = static_cast<int>(threadIdx.x) - 32;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t timeout = prm.timeout_ns;
    const uint32_t ring0 = smem_addr(sm.ring);
    const uint32_t hdr0 = smem_addr(sm.hdr);
    uint4 accP[S::kItems], accQ[S::kItems];
    int row[S::kItems];
    uint32_t off[S::kItems];   // byte offset of the item's own row in a slot
    Tile T = {};
    uint8_t *copy_dst = nullptr;  // small write: data strip a of the tile
    uint32_t ep_phase = 0, fold_par = 0;
    int p = 3;
    uint32_t pitch = 16, pw = 48;
    RingPos pos;

    for (;;) {
        if (!mbar_wait(smem_addr(&sm.full[pos.slot]), pos.phase, timeout)) {
            if (lane == 0) set_status(prm.status, RCG_DEV_TIMEOUT);
            return;
        }
        const uint4 hv = lds_a(hdr0 + pos.slot * static_cast<uint32_t>(sizeof(SlotHdr)));
        const uint32_t flags = hv.x & 0xffu;
        if (flags & F_END) break;
        if (flags & F_FIRST) {
            const uint32_t ha = hdr0 + pos.slot * static_cast<uint32_t>(sizeof(SlotHdr));
            const uint4 tv = lds_a(ha + 16), bv = lds_a(ha + 32), ov = lds_a(ha + 48);
            T.w = hv.x >> 16;
            T.nvec = T.w >> 4;
            T.cls = static_cast<uint8_t>(tv.x);
            T.p = (tv.x >> 8) & 0xffu;
            T.a = static_cast<uint8_t>(tv.x >> 16);
            T.b = static_cast<uint8_t>(tv.x >> 24);
            T.base = reinterpret_cast<uint8_t *>(static_cast<uint64_t>(tv.z) | (static_cast<uint64_t>(tv.w) << 32));
            T.strip_stride = static_cast<uint64_t>(bv.x) | (static_cast<uint64_t>(bv.y) << 32);
            T.row_stride = static_cast<uint64_t>(bv.z) | (static_cast<uint64_t>(bv.w) << 32);
            T.out = reinterpret_cast<uint8_t *>(static_cast<uint64_t>(ov.x) | (static_cast<uint64_t>(ov.y) << 32));
            T.out_row_stride = static_cast<uint64_t>(ov.z) | (static_cast<uint64_t>(ov.w) << 32);
            copy_dst = T.base + static_cast<uint64_t>(T.a) * T.strip_stride;
            p = static_cast<int>(T.p);
            pitch = tv.y & 0xffffu;
            T.z = static_cast<uint8_t>(tv.y >> 24);
            pw = p * pitch;
            for (int t = 0; t < S::kItems; ++t) {
                const int item = ctid + t * S::kConsumers;
                const int r = item / static_cast<int>(T.nvec);
                row[t] = r < p ? r : 0x7fff;
                off[t] = r * pitch + (item - r * static_cast<int>(T.nvec)) * 16;
                accP[t] = make_uint4(0, 0, 0, 0);
                accQ[t] = make_uint4(0, 0, 0, 0);
            }
        }
        const uint32_t stage = ring0 + hv.y;  // the stage's offset in the byte ring
        const int rot = (hv.x >> 8) & 0xff;
        // row r of x^rot * strip is row r - rot (mod p) of the strip; the item
        // row whose source is the imaginary row p-1 is vrow = (p-1+rot) mod p
        const uint32_t qbase = stage - rot * pitch;  // + p*pitch for rows r < rot
        const int vrow = rot == 0 ? p - 1 : rot - 1;
        const uint32_t fsel = flags & (F_P | F_Q | F_Q2 | F_COPY);
        if (fsel == (F_P | F_Q) || (S::kItems > 4 && fsel == F_P)) {
            // a data strip feeding both accumulators: the common case; in the
            // 6-item shape also P alone (a separate loop there costs a spill)
            const bool with_q = fsel & F_Q;
#pragma unroll
            for (int t = 0; t < S::kItems; ++t) {
                const int r = row[t];  // invalid items carry a row >= p
                if (r < p - 1) accP[t] = xor4(accP[t], lds_a(stage + off[t]));
                if (with_q && r < p && r != vrow)
                    accQ[t] = xor4(accQ[t], lds_a(qbase + off[t] + (r < rot ? pw : 0u)));
            }
        } else if (fsel == F_P) {
            // P alone: every stage of a degraded read from P, the P strip of a
            // recovery (the 4-item shape)
#pragma unroll
            for (int t = 0; t < S::kItems; ++t)
                if (row[t] < p - 1) accP[t] = xor4(accP[t], lds_a(stage + off[t]));
        } else if (fsel == F_Q) {
            // Q alone: every stage of a degraded read of Q, the Q strip of a recovery
#pragma unroll
            for (int t = 0; t < S::kItems; ++t) {
                const int r = row[t];
                if (r < p && r != vrow) accQ[t] = xor4(accQ[t], lds_a(qbase + off[t] + (r < rot ? pw : 0u)));
            }
        } else if (fsel == (F_P | F_Q | F_Q2) && hv.z == 0) {
            // an extended data strip (weight 1 + x^rot) feeding both accumulators
#pragma unroll
            for (int t = 0; t < S::kItems; ++t) {
                const int r = row[t];
                if (r < p - 1) {
                    const uint4 v = lds_a(stage + off[t]);
                    accP[t] = xor4(accP[t], v);
                    accQ[t] = xor4(accQ[t], v);
                }
                if (r < p && r != vrow) accQ[t] = xor4(accQ[t], lds_a(qbase + off[t] + (r < rot ? pw : 0u)));
            }
        } else {
            const bool fp = flags & F_P, fq = flags & F_Q, fq2 = flags & F_Q2, fc = flags & F_COPY;
            const int rot2 = static_cast<int>(hv.z);
            const uint32_t qbase2 = stage - rot2 * pitch;
            const int vrow2 = rot2 == 0 ? p - 1 : rot2 - 1;
#pragma unroll
            for (int t = 0; t < S::kItems; ++t) {
                const int r = row[t];
                if (r >= p) continue;
                if (fp && r < p - 1) {
                    const uint4 v = lds_a(stage + off[t]);
                    accP[t] = xor4(accP[t], v);
                    if (fc) stg(copy_dst + static_cast<uint64_t>(r) * T.row_stride + (off[t] - r * pitch), v);
                }
                if (fq && r != vrow) accQ[t] = xor4(accQ[t], lds_a(qbase + off[t] + (r < rot ? pw : 0u)));
                if (fq2 && r != vrow2) accQ[t] = xor4(accQ[t], lds_a(qbase2 + off[t] + (r < rot2 ? pw : 0u)));
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&sm.empty[pos.slot]));
        pos.next(n_slots);
        if (flags & F_LAST) {
            if (!epilogue<S>(sm, T, accP, accQ, row, ep_phase, fold_par, timeout)) {
                if (lane == 0) set_status(prm.status, RCG_DEV_TIMEOUT);
                return;
            }
        }
    }
}

// ------------------------------------------------------------------ kernel

template <class S>
__device__ __forceinline__ void engine_body(const LaunchParams &prm, const BatchHeader *bh, bool in_params) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const Smem sm = carve<S>(smem_raw);

    // single launches: n_slots stages of slot_bytes; batches: a byte ring of
    // stages of any size, at most n_slots of them in flight
    uint32_t n_slots = prm.n_slots;
    uint64_t ring_bytes = static_cast<uint64_t>(prm.n_slots) * prm.slot_bytes;
    uint64_t total = prm.total_tiles;  // units: tiles of a single launch, or batch work items
    if (bh) {
        n_slots = bh->n_slots;
        ring_bytes = bh->ring_bytes;
        total = bh->n_items;
    }
    const uint32_t my_shape = S::kCtasPerSm == 2 ? SHAPE_PAIR : SHAPE_WIDE;
    if ((bh && bh->shape != my_shape) || n_slots == 0 || n_slots > kMaxSlots || ring_bytes < 128 ||
        ring_bytes > S::kRingBytes || (ring_bytes & 127)) {
        if (threadIdx.x == 0) set_status(prm.status, RCG_DEV_BADJOB);
        return;
    }

    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < n_slots; ++s) {
            mbar_init(smem_addr(&sm.full[s]), 1);
            mbar_init(smem_addr(&sm.empty[s]), S::kConsumerWarps);
        }
        mbar_init(smem_addr(sm.ep), S::kConsumerWarps);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (threadIdx.x < 32)
        producer<S>(prm, sm, bh, in_params, total, static_cast<uint32_t>(ring_bytes), n_slots);
    else
        consumer<S>(prm, sm, n_slots);
}

// Single launches (bh null) and batches with a device table.
template <class S>
__global__ void __launch_bounds__(S::kThreads, S::kCtasPerSm)
    rcg_tile_engine(const __grid_constant__ LaunchParams prm, const BatchHeader *bh) {
    engine_body<S>(prm, bh, false);
}

// Batches whose table travels in the parameter block.
template <class S, uint32_t SZ>
__global__ void __launch_bounds__(S::kThreads, S::kCtasPerSm)
    rcg_tile_engine_param(const __grid_constant__ LaunchParams prm, const __grid_constant__ ParamTable<SZ> t) {
    engine_body<S>(prm, reinterpret_cast<const BatchHeader *>(t.bytes), true);
}

// --------------------------------------------------- bounded-wait self test

// One thread waits, with the engine's own bounded wait, on an mbarrier that
// nothing will complete: the wait runs out after timeout_ns, the kernel
// records RCG_DEV_TIMEOUT and returns -- no trap, no hang.
__global__ void rcg_wait_probe_kernel(uint32_t *status, uint64_t timeout_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_addr(&bar);
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(b, 0, timeout_ns)) set_status(status, RCG_DEV_TIMEOUT);
}

// ------------------------------------------------------ test-data generator

__device__ __forceinline__ uint64_t splitmix_word(uint64_t seed, uint64_t w) {
    uint64_t z = (seed << 40) + (w + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void rcg_fill_kernel(uint8_t *dst, uint64_t nbytes, uint64_t seed, uint64_t word0) {
    const uint64_t n_pairs = (nbytes + 15) / 16;
    for (uint64_t q = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; q < n_pairs;
         q += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t w0 = splitmix_word(seed, word0 + 2 * q);
        const uint64_t w1 = splitmix_word(seed, word0 + 2 * q + 1);
        const uint64_t off = 16 * q;
        if (off + 16 <= nbytes) {
            uint4 v = make_uint4(static_cast<uint32_t>(w0), static_cast<uint32_t>(w0 >> 32),
                                 static_cast<uint32_t>(w1), static_cast<uint32_t>(w1 >> 32));
            *reinterpret_cast<uint4 *>(dst + off) = v;
        } else {
            for (uint64_t b = off; b < nbytes; ++b) {
                const uint64_t w = (b - off) < 8 ? w0 : w1;
                dst[b] = static_cast<uint8_t>(w >> (8 * ((b - off) & 7)));
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------- host side

void inverse_masks(uint32_t p, uint64_t *masks) {
    // Section 4.6: (1 + x^z)^(-1) = sum_{t=0}^{(p-1)/2} x^(2tz), exponents mod p.
    masks[0] = 0;
    for (uint32_t z = 1; z < p; ++z) {
        uint64_t m = 0;
        for (uint32_t t = 0; t <= (p - 1) / 2; ++t) m |= 1ull << ((2ull * t * z) % p);
        masks[z] = m;
    }
}

static bool is_odd_prime(uint32_t p) {
    if (p < 3 || (p & 1) == 0) return false;
    for (uint32_t d = 3; d * d <= p; d += 2)
        if (p % d == 0) return false;
    return true;
}

cudaError_t upload_inverse_tables() {
    // built once per process, uploaded to every device that asks
    static uint64_t table[kMaxP + 1][kMaxP + 1];
    static uint64_t tri[kTriEntries];
    static uint32_t tri_off[kMaxP + 1];
    static std::once_flag built;
    std::call_once(built, [] {
        uint32_t n = 0;
        for (uint32_t p = 0; p <= static_cast<uint32_t>(kMaxP); ++p) {
            for (uint32_t z = 0; z <= static_cast<uint32_t>(kMaxP); ++z) table[p][z] = 0;
            tri_off[p] = ~0u;
            if (!is_odd_prime(p)) continue;
            inverse_masks(p, table[p]);
            if (cone_extends(p)) {
                tri_off[p] = n;
                trinomial_inverses(p, tri + n);
            }
            n += p * p;
        }
    });
    cudaError_t e = cudaMemcpyToSymbol(c_inv, table, sizeof(table));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tri_off, tri_off, sizeof(tri_off));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tri, tri, sizeof(tri));
    return e;
}

cudaError_t engine_init_attributes() {
    const int wide = static_cast<int>(ShapeWide::kSmemLimit), pair = static_cast<int>(ShapePair::kSmemLimit);
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(rcg_tile_engine<ShapeWide>, attr, wide);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(rcg_tile_engine<ShapePair>, attr, pair);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(rcg_tile_engine_param<ShapeWide, kParamTableSmall>, attr, wide);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(rcg_tile_engine_param<ShapePair, kParamTableSmall>, attr, pair);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(rcg_tile_engine_param<ShapeWide, kParamTableLarge>, attr, wide);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(rcg_tile_engine_param<ShapePair, kParamTableLarge>, attr, pair);
    return e;
}

template <class S>
static cudaError_t launch_shape(const LaunchParams &prm, const BatchHeader *bh, size_t smem, int grid,
                                cudaStream_t stream) {
    rcg_tile_engine<S><<<grid, S::kThreads, smem, stream>>>(prm, bh);
    return cudaGetLastError();
}

cudaError_t launch_engine(const LaunchParams &prm, uint32_t shape, int grid, cudaStream_t stream) {
    const ShapeInfo si = shape_info(shape);
    const size_t smem = si.fixed_smem + static_cast<size_t>(prm.n_slots) * prm.slot_bytes;
    return shape == SHAPE_PAIR ? launch_shape<ShapePair>(prm, nullptr, smem, grid, stream)
                               : launch_shape<ShapeWide>(prm, nullptr, smem, grid, stream);
}

cudaError_t launch_batch(const uint8_t *table_dev, uint32_t *status, unsigned long long *counter,
                         uint64_t timeout_ns, uint32_t shape, int grid, cudaStream_t stream) {
    LaunchParams prm = {};
    prm.dynamic_sched = 1;
    prm.tile_counter = counter;
    prm.status = status;
    prm.timeout_ns = timeout_ns;
    const auto *bh = reinterpret_cast<const BatchHeader *>(table_dev);
    const ShapeInfo si = shape_info(shape);
    return shape == SHAPE_PAIR ? launch_shape<ShapePair>(prm, bh, si.smem_limit, grid, stream)
                               : launch_shape<ShapeWide>(prm, bh, si.smem_limit, grid, stream);
}

template <class S, uint32_t SZ>
static cudaError_t launch_param_sized(const uint8_t *table_host, size_t bytes, const LaunchParams &prm, size_t smem,
                                     int grid, cudaStream_t stream) {
    ParamTable<SZ> t;
    memcpy(t.bytes, table_host, bytes);
    memset(t.bytes + bytes, 0, SZ - bytes);
    rcg_tile_engine_param<S, SZ><<<grid, S::kThreads, smem, stream>>>(prm, t);
    return cudaGetLastError();
}

cudaError_t launch_batch_param(const uint8_t *table_host, size_t bytes, uint32_t *status, uint64_t timeout_ns,
                               uint32_t shape, int grid, cudaStream_t stream) {
    if (bytes > kParamTableLarge || bytes < sizeof(BatchHeader)) return cudaErrorInvalidValue;
    LaunchParams prm = {};
    prm.dynamic_sched = 0;
    prm.tile_counter = nullptr;
    prm.status = status;
    prm.timeout_ns = timeout_ns;
    const size_t smem = shape_info(shape).smem_limit;
    const bool small = bytes <= kParamTableSmall;
    if (shape == SHAPE_PAIR)
        return small ? launch_param_sized<ShapePair, kParamTableSmall>(table_host, bytes, prm, smem, grid, stream)
                     : launch_param_sized<ShapePair, kParamTableLarge>(table_host, bytes, prm, smem, grid, stream);
    return small ? launch_param_sized<ShapeWide, kParamTableSmall>(table_host, bytes, prm, smem, grid, stream)
                 : launch_param_sized<ShapeWide, kParamTableLarge>(table_host, bytes, prm, smem, grid, stream);
}

cudaError_t launch_wait_probe(uint32_t *status, uint64_t timeout_ns, cudaStream_t stream) {
    rcg_wait_probe_kernel<<<1, 32, 0, stream>>>(status, timeout_ns);
    return cudaGetLastError();
}

cudaError_t launch_fill(void *dev, uint64_t nbytes, uint64_t seed, uint64_t byte_offset,
                        cudaStream_t stream) {
    if (nbytes == 0) return cudaSuccess;
    const uint64_t pairs = (nbytes + 15) / 16;
    const int threads = 256;
    uint64_t blocks = (pairs + threads - 1) / threads;
    if (blocks > 152ull * 16) blocks = 152ull * 16;
    rcg_fill_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
        static_cast<uint8_t *>(dev), nbytes, seed, byte_offset / 8);
    return cudaGetLastError();
}

}  // namespace rcg
