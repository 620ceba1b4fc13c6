// rcg_internal.h -- definitions shared by the host side (rcg_api.cu) and the
// tile engine (rcg_engine.cu) of librcg.  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rcg.h"

namespace rcg {

// ---------------------------------------------------------------- geometry
// A CTA of the tile engine is one producer warp (issues the bulk copies) and
// kConsumerWarps consumer warps.  A consumer thread owns up to kItems
// "items": one 16-byte column vector of one row, for P and for the lifted Q
// accumulator (rows 0..p-1, row p-1 being the imaginary row of the lift to
// F2[x]/(x^p - 1)).  A tile of W bytes of a p-row stripe has p * W/16 items.
#ifndef RCG_CONSUMER_WARPS
#define RCG_CONSUMER_WARPS 15
#endif
#ifndef RCG_ITEMS
#define RCG_ITEMS 4
#endif
#ifndef RCG_CTAS_PER_SM
#define RCG_CTAS_PER_SM 1
#endif
constexpr int kCtasPerSm = RCG_CTAS_PER_SM;
constexpr int kConsumerWarps = RCG_CONSUMER_WARPS;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kThreads = kConsumers + 32;
constexpr int kItems = RCG_ITEMS;
constexpr int kMaxItems = kItems * kConsumers;  // items per tile (2048 by default)
constexpr uint32_t kMaxTileBytes = 2048;        // a TMA box row is at most 256 8-byte elements
constexpr int kMaxSlots = 32;
constexpr int kMaxP = 61;
constexpr uint32_t kMaxSlotBytes = 32 * 1024;

// Dynamic shared memory: control block, exchange buffers, then the ring.
constexpr uint32_t kCtlBytes = 2048;                       // barriers + slot headers
constexpr uint32_t kXBytes = kMaxItems * 16;               // the p x W exchange buffer
constexpr uint32_t kFoldBytes = kMaxTileBytes;             // one row of W bytes
constexpr uint32_t kFixedSmem = kCtlBytes + kXBytes + 2 * kFoldBytes;  // two fold rows
// 228 KB of shared memory per SM, 1 KB of it reserved per resident CTA
constexpr uint32_t kSmemLimit = (228 / kCtasPerSm - 1) * 1024;
constexpr uint32_t kRingBytes = kSmemLimit - kFixedSmem;

enum Op : uint8_t { OP_ENCODE = 0, OP_RECOVER = 1, OP_DEGRADED = 2, OP_UPDATE = 3 };

// Device-side job: a run of stripes with one geometry and one operation.
// tmap is a 4-D tiled TMA descriptor over (8-byte column, row, strip, stripe)
// of the job's stripes with a (W/8) x (p-1) x 1 x 1 box: one tensor copy
// brings a whole strip tile into a ring slot.
struct alignas(128) Job {
    CUtensorMap tmap;
    uint8_t *base;           // stripe 0 of this job (first_stripe already applied)
    uint8_t *aux;            // update: new strips (read); degraded read: output (written)
    const uint8_t *pairs;    // recover: per-stripe (i, j) bytes, or nullptr
    uint64_t row_stride, strip_stride, stripe_stride;
    uint64_t aux_row_stride, aux_stripe_stride;
    uint64_t tile_begin;     // first global tile index of this job
    uint32_t n_stripes;
    uint32_t C;              // row bytes
    uint32_t W;              // tile width, bytes
    uint32_t tiles_per_stripe;
    uint8_t p, n, op, i, j;
    uint8_t use_tmap;        // 0: the driver refused this layout; fall back to row copies
    uint8_t dd_solve;        // two-data solve: 0 = chain along x^z, 1 = Section 4.6 table
    uint8_t pad[1];
};

struct LaunchParams {
    const Job *jobs;                 // device table, or nullptr: use job0
    Job job0;
    uint32_t n_jobs;
    uint32_t slot_bytes;
    uint32_t n_slots;
    uint32_t dynamic_sched;          // 1: tiles from *tile_counter; 0: static stride
    uint64_t total_tiles;
    unsigned long long *tile_counter;
    uint32_t *status;                // device status word (RCG_DEV_* bits)
    uint64_t timeout_ns;
};

// Header of a batch descriptor table: the graph-replayed batch kernel reads
// its sizes from here so the captured kernel node never changes.
struct alignas(128) BatchHeader {
    uint64_t total_tiles;
    uint32_t n_jobs;
    uint32_t slot_bytes;
    uint32_t n_slots;
    uint32_t pad[27];
};
static_assert(sizeof(BatchHeader) == 128, "the job table after the header stays 128-byte aligned");
static_assert(sizeof(Job) % 128 == 0, "jobs keep their tensor maps 128-byte aligned");

struct Plan {
    uint32_t W, tiles_per_stripe, slot_bytes, n_slots;
};

// Host: tiling for one (p, C).  Returns false when out of range.
bool make_plan(uint32_t p, uint64_t C, Plan *out);

// Host: upload the per-p inverse tables to the current device (once).
cudaError_t upload_inverse_tables();

// Host launchers (rcg_engine.cu).
cudaError_t launch_engine(const LaunchParams &prm, int grid, cudaStream_t stream);
cudaError_t launch_batch(const uint8_t *table_dev, uint32_t *status, unsigned long long *counter,
                         uint64_t timeout_ns, int grid, cudaStream_t stream);
cudaError_t engine_init_attributes();
cudaError_t launch_fill(void *dev, uint64_t nbytes, uint64_t seed, uint64_t byte_offset,
                        cudaStream_t stream);

void inverse_masks(uint32_t p, uint64_t *masks);

// Host: validate one public job and build its device descriptor with the
// default copy mode and two-data solve (used by rcg_batch_submit_noalloc).
bool noalloc_build_job(const rcg_job &in, Job *out, Plan *pl);

}  // namespace rcg
