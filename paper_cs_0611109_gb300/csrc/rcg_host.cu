// rcg_host.cu -- encode and recovery of stripes that live in (page-locked)
// HOST memory: the data are streamed through context-owned device staging
// buffers in chunks of stripes, on three internal streams, so the upload of
// one chunk, the tile engine on another and the download of a third overlap.
//
//   encode:   the data strips in -> rcg_encode on the chunk -> P and Q out
//   recovery: the N surviving strips of each stripe in (the erased strips are
//             never moved) -> rcg_recover_many on the chunk -> the two rebuilt
//             strips out.
// A gather kernel reads the strips from the host stripes through their
// device-visible (mapped) addresses and a write-back kernel writes the results
// straight into them.
// The host link, not HBM, bounds this path (about 211 GB/s host to device on
// GB300, the same for copy engines and for kernel loads), so what counts is
// the bytes that cross it: N strips in and 2 out per stripe.
//
// The caller's stream orders the call: the internal streams wait for it on
// entry and it waits for them on exit.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "../../include/rcg.h"
#include "rcg_internal.h"

namespace {

// Copy the rebuilt strips (i, j) of each stripe of a device chunk back to the
// host stripes (mapped device addresses).  Same shape as the gather below: a
// CTA takes whole units (stripe, one of its two strips), so a few CTAs keep
// the link busy and leave the SMs to the gather and the tile engine of the
// neighbouring chunks.  Pairs that are not a valid erasure pair (the engine
// skipped those stripes) are skipped here too.
__global__ void writeback_kernel(const uint8_t *chunk, uint64_t chunk_stripe_bytes, uint64_t strip_bytes,
                                 uint8_t *host_dev, uint64_t h_row, uint64_t h_strip, uint64_t h_stripe,
                                 const uint8_t *pairs, uint32_t fi, uint32_t fj, uint32_t n_stripes,
                                 uint32_t rows, uint32_t nvec, uint32_t n_total) {
    const uint64_t units = 2ull * n_stripes;
    const uint32_t row_bytes = nvec * 16;
    for (uint64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const uint32_t s = static_cast<uint32_t>(u >> 1);
        const uint32_t a = pairs ? pairs[2ull * s] : fi, b = pairs ? pairs[2ull * s + 1] : fj;
        if (!(a < b && b <= n_total + 1)) continue;
        const uint32_t k = (u & 1) ? b : a;
        const uint8_t *src = chunk + s * chunk_stripe_bytes + k * strip_bytes;
        uint8_t *dst = host_dev + s * h_stripe + k * h_strip;
        if (h_row == row_bytes) {  // one contiguous run
            const uint4 *sv = reinterpret_cast<const uint4 *>(src);
            uint4 *dv = reinterpret_cast<uint4 *>(dst);
            const uint32_t n = rows * nvec;
            for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) dv[t] = sv[t];
        } else {
            for (uint32_t r = 0; r < rows; ++r)
                for (uint32_t v = threadIdx.x; v < nvec; v += blockDim.x)
                    reinterpret_cast<uint4 *>(dst + r * h_row)[v] =
                        reinterpret_cast<const uint4 *>(src + static_cast<uint64_t>(r) * row_bytes)[v];
        }
    }
}

// Copy the surviving strips (all but the pair's two) of each stripe from the
// host stripes (mapped device addresses) into the packed chunk.  Reads over
// the host link have a long latency under load: keeping the link busy takes
// several MB of loads in flight, from every SM.  A CTA takes whole units
// (stripe, surviving strip); a strip whose rows are packed is one contiguous
// run, copied with GATHER_UNROLL independent 16-byte loads in flight per
// thread.  Stripes whose pair is invalid move nothing (the engine skips them
// and records the error).
constexpr int GATHER_UNROLL = 8;

__global__ void gather_kernel(const uint8_t *host_dev, uint64_t h_row, uint64_t h_strip, uint64_t h_stripe,
                              uint8_t *chunk, uint64_t chunk_stripe_bytes, uint64_t strip_bytes,
                              const uint8_t *pairs, uint32_t fi, uint32_t fj, uint32_t n_stripes,
                              uint32_t rows, uint32_t nvec, uint32_t n_total) {
    const uint64_t units = static_cast<uint64_t>(n_stripes) * n_total;
    const uint32_t row_bytes = nvec * 16;
    for (uint64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const uint32_t s = static_cast<uint32_t>(u / n_total);
        uint32_t k = static_cast<uint32_t>(u - static_cast<uint64_t>(s) * n_total);
        const uint32_t a = pairs ? pairs[2ull * s] : fi, b = pairs ? pairs[2ull * s + 1] : fj;
        if (!(a < b && b <= n_total + 1)) continue;
        if (k >= a) ++k;  // the k-th surviving strip
        if (k >= b) ++k;
        const uint8_t *src = host_dev + s * h_stripe + k * h_strip;
        uint8_t *dst = chunk + s * chunk_stripe_bytes + k * strip_bytes;
        if (h_row == row_bytes) {  // one contiguous run of rows * nvec vectors
            const uint4 *sv = reinterpret_cast<const uint4 *>(src);
            uint4 *dv = reinterpret_cast<uint4 *>(dst);
            const uint32_t n = rows * nvec, step = blockDim.x;
            uint32_t t = threadIdx.x;
            for (; t + (GATHER_UNROLL - 1) * step < n; t += GATHER_UNROLL * step) {
                uint4 v[GATHER_UNROLL];
#pragma unroll
                for (int q = 0; q < GATHER_UNROLL; ++q) v[q] = sv[t + q * step];
#pragma unroll
                for (int q = 0; q < GATHER_UNROLL; ++q) dv[t + q * step] = v[q];
            }
            for (; t < n; t += step) dv[t] = sv[t];
        } else {
            for (uint32_t r = 0; r < rows; ++r)
                for (uint32_t v = threadIdx.x; v < nvec; v += blockDim.x)
                    reinterpret_cast<uint4 *>(dst + static_cast<uint64_t>(r) * row_bytes)[v] =
                        reinterpret_cast<const uint4 *>(src + r * h_row)[v];
        }
    }
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

struct HostGeo {
    uint32_t p, N;
    uint64_t C, rs, ss, st;
    uint64_t strip_bytes;   // packed strip in the staging chunk: (p-1) * C
    uint64_t stripe_bytes;  // packed stripe in the staging chunk: (N+2) * strip_bytes
};

bool host_geo(const rcg_layout *L, HostGeo *g) {
    if (!L || !L->base) return false;
    g->p = L->p;
    g->N = L->n_data;
    g->C = L->row_bytes;
    if (g->p < 3 || g->p > 61 || g->N < 1 || g->N > rcg::max_data_strips(g->p) || g->C == 0 || (g->C & 15))
        return false;
    g->rs = L->row_stride ? L->row_stride : g->C;
    g->ss = L->strip_stride ? L->strip_stride : (g->p - 1) * g->rs;
    g->st = L->stripe_stride ? L->stripe_stride : (g->N + 2) * g->ss;
    if (g->rs < g->C || (g->rs & 15) || (g->ss & 15) || (g->st & 15) || !aligned16(L->base)) return false;
    g->strip_bytes = (g->p - 1) * g->C;
    g->stripe_bytes = (g->N + 2) * g->strip_bytes;
    return true;
}

}  // namespace

namespace rcg {

// CTAs of the gather kernel (512 threads each): the host link needs loads in
// flight from every SM.  The write-back's stores are posted, so a few CTAs
// keep its direction busy and leave the SMs to the gather and the engine.
constexpr unsigned kGatherCtas = 152;
constexpr unsigned kWritebackCtas = 32;

// Context-owned staging for the host path (see rcg_api.cu for the owner).
struct HostStaging {
    uint8_t *buf[3] = {nullptr, nullptr, nullptr};
    uint8_t *pairs[3] = {nullptr, nullptr, nullptr};
    cudaStream_t stream[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_in = nullptr, ev_out[3] = {nullptr, nullptr, nullptr};
    uint64_t bytes = 0;        // per chunk buffer
    uint64_t pair_bytes = 0;   // per chunk pairs buffer
};

HostStaging *host_staging_create() { return new HostStaging(); }

void host_staging_destroy(HostStaging *h) {
    if (!h) return;
    for (int k = 0; k < 3; ++k) {
        if (h->stream[k]) cudaStreamSynchronize(h->stream[k]);
        if (h->buf[k]) cudaFree(h->buf[k]);
        if (h->pairs[k]) cudaFree(h->pairs[k]);
        if (h->stream[k]) cudaStreamDestroy(h->stream[k]);
        if (h->ev_out[k]) cudaEventDestroy(h->ev_out[k]);
    }
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    delete h;
}

static cudaError_t staging_ready(HostStaging *h, uint64_t bytes, uint64_t pair_bytes) {
    if (!h->stream[0]) {
        for (int k = 0; k < 3; ++k) {
            cudaError_t e = cudaStreamCreateWithFlags(&h->stream[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out[k], cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    if (h->bytes < bytes || h->pair_bytes < pair_bytes) {
        for (int k = 0; k < 3; ++k) {
            cudaStreamSynchronize(h->stream[k]);
            if (h->buf[k]) cudaFree(h->buf[k]);
            if (h->pairs[k]) cudaFree(h->pairs[k]);
            h->buf[k] = h->pairs[k] = nullptr;
        }
        h->bytes = h->pair_bytes = 0;
        for (int k = 0; k < 3; ++k) {
            cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&h->buf[k]), bytes);
            if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&h->pairs[k]), pair_bytes);
            if (e != cudaSuccess) return e;
        }
        h->bytes = bytes;
        h->pair_bytes = pair_bytes;
    }
    return cudaSuccess;
}

// Shared driver of the two host-path calls.  encode_fn / recover_fn run the
// tile engine on a packed device chunk of n stripes.
rcg_status host_path(HostStaging *h, const rcg_layout *L, uint64_t first, uint64_t n_stripes,
                     const uint8_t *pairs_host, cudaStream_t caller, uint64_t chunk_bytes,
                     rcg_status (*run)(void *, const rcg_layout *, uint64_t, const uint8_t *, cudaStream_t),
                     void *run_arg) {
    HostGeo g;
    if (!h || !host_geo(L, &g)) return RCG_EINVAL;
    if (n_stripes == 0) return RCG_OK;
    // the host stripes must be page-locked and visible to the device
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, L->base) != cudaSuccess || attr.type != cudaMemoryTypeHost ||
        !attr.devicePointer) {
        cudaGetLastError();
        return RCG_EINVAL;
    }
    uint8_t *host_dev = static_cast<uint8_t *>(attr.devicePointer);
    // the gather and write-back kernels index a strip's vectors with 32 bits
    if (g.strip_bytes / 16 > 0xffffffffull) return RCG_EINVAL;
    const uint64_t per_chunk = std::max<uint64_t>(1, chunk_bytes / g.stripe_bytes);
    cudaError_t e = staging_ready(h, per_chunk * g.stripe_bytes, 2 * per_chunk);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? RCG_ENOMEM : RCG_ECUDA;

    e = cudaEventRecord(h->ev_in, caller);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(h->stream[k], h->ev_in, 0);
    rcg_status st = RCG_OK;
    uint64_t c = 0;
    for (uint64_t s0 = 0; s0 < n_stripes && e == cudaSuccess && st == RCG_OK; s0 += per_chunk, ++c) {
        const int k = static_cast<int>(c % 3);
        cudaStream_t s = h->stream[k];
        const uint64_t n = std::min(per_chunk, n_stripes - s0);
        rcg_layout dl;
        memset(&dl, 0, sizeof(dl));
        dl.base = h->buf[k];
        dl.p = g.p;
        dl.n_data = g.N;
        dl.row_bytes = g.C;
        // Both directions go through kernels that address the host stripes by
        // their mapped device addresses: encode is the pair (P, Q) for every
        // stripe (its data strips in, P and Q out), recovery a per-stripe pair.
        // (The copy engines move bytes as fast, but 2-D copy-engine uploads
        // showed occasional stalls of 0.1-0.2 s on the GB300 machine; the kernel
        // path never did.)
        const uint32_t rows = g.p - 1, nvec = static_cast<uint32_t>(g.C / 16);
        const uint8_t *pairs_dev = nullptr;
        if (pairs_host) {
            e = cudaMemcpyAsync(h->pairs[k], pairs_host + 2 * s0, 2 * n, cudaMemcpyHostToDevice, s);
            pairs_dev = h->pairs[k];
        }
        if (e == cudaSuccess) {
            gather_kernel<<<kGatherCtas, 512, 0, s>>>(host_dev + (first + s0) * g.st, g.rs, g.ss, g.st, h->buf[k],
                                                     g.stripe_bytes, g.strip_bytes, pairs_dev, g.N, g.N + 1,
                                                     static_cast<uint32_t>(n), rows, nvec, g.N);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) st = run(run_arg, &dl, n, pairs_dev, s);
        if (e == cudaSuccess && st == RCG_OK) {
            writeback_kernel<<<kWritebackCtas, 512, 0, s>>>(h->buf[k], g.stripe_bytes, g.strip_bytes,
                                                            host_dev + (first + s0) * g.st, g.rs, g.ss, g.st,
                                                            pairs_dev, g.N, g.N + 1, static_cast<uint32_t>(n), rows,
                                                            nvec, g.N);
            e = cudaGetLastError();
        }
    }
    for (int k = 0; k < 3; ++k) {
        cudaError_t e2 = cudaEventRecord(h->ev_out[k], h->stream[k]);
        if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(caller, h->ev_out[k], 0);
        if (e == cudaSuccess) e = e2;
    }
    if (st != RCG_OK) return st;
    return e == cudaSuccess ? RCG_OK : RCG_ECUDA;
}

}  // namespace rcg
