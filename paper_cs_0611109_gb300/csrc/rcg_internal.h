// rcg_internal.h -- definitions shared by the host side (rcg_api.cu) and the
// tile engine (rcg_engine.cu) of librcg.  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/rcg.h"

namespace rcg {

// ---------------------------------------------------------------- geometry
// A CTA of the tile engine is one producer warp (issues the tensor copies)
// and CW consumer warps.  A consumer thread owns up to IT "items": one 16-byte
// column vector of one row, for P and for the lifted Q accumulator (rows
// 0..p-1, row p-1 being the imaginary row of the lift to F2[x]/(x^p - 1)).
// A tile of W bytes of a p-row stripe has p * W/16 items.
//
// Two shapes are built:
//   wide: 1 CTA per SM, 15 consumer warps x 4 items, 227 KB of shared memory
//         (deep ring: the best choice when slots are large, e.g. p = 59);
//   pair: 2 CTAs per SM, 6 consumer warps x 6 items, 113 KB each (one CTA's
//         epilogue overlaps the other's streaming).
constexpr uint32_t kMaxTileBytes = 2048;  // a TMA box row is at most 256 8-byte elements
constexpr int kMaxSlots = 32;
constexpr int kMaxP = 61;
constexpr uint32_t kMaxSlotBytes = 32 * 1024;
constexpr uint32_t kCtlBytes = 3072;            // barriers (1 KB) + 32 slot headers of 64 B
constexpr uint32_t kFoldBytes = kMaxTileBytes;  // one row of W bytes (two are kept)

template <int CW, int IT, int CT, int MINSLOTS>
struct EngineShape {
    static constexpr int kConsumerWarps = CW;
    static constexpr int kConsumers = CW * 32;
    static constexpr int kThreads = kConsumers + 32;
    static constexpr int kItems = IT;
    static constexpr int kMaxItems = IT * CW * 32;
    static constexpr int kCtasPerSm = CT;
    static constexpr int kMinSlots = MINSLOTS;  // a plan keeps at least this ring depth
    // 228 KB of shared memory per SM, 1 KB of it reserved per resident CTA
    static constexpr uint32_t kSmemLimit = (228 / CT - 1) * 1024;
    static constexpr uint32_t kXBytes = kMaxItems * 16;  // the p x W exchange buffer
    static constexpr uint32_t kFixedSmem = kCtlBytes + kXBytes + 2 * kFoldBytes;
    static constexpr uint32_t kRingBytes = kSmemLimit - kFixedSmem;
};
using ShapeWide = EngineShape<15, 4, 1, 2>;
using ShapePair = EngineShape<6, 6, 2, 4>;
enum Shape : uint32_t { SHAPE_WIDE = 0, SHAPE_PAIR = 1 };

struct ShapeInfo {
    uint32_t max_items, ring_bytes, fixed_smem, smem_limit, ctas_per_sm, min_slots;
};
template <class S>
constexpr ShapeInfo shape_info_of() {
    return {static_cast<uint32_t>(S::kMaxItems), S::kRingBytes, S::kFixedSmem, S::kSmemLimit,
            static_cast<uint32_t>(S::kCtasPerSm), static_cast<uint32_t>(S::kMinSlots)};
}
inline ShapeInfo shape_info(uint32_t shape) {
    return shape == SHAPE_PAIR ? shape_info_of<ShapePair>() : shape_info_of<ShapeWide>();
}

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
    Job job0;                        // single launches; batches read their jobs after the table header
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
// A unit of work in a batch: a run of tiles of one job (sized by bytes), with every field
// the producer needs copied in, so one 128-byte load (prefetched while the
// previous item streams) starts it.  Items are dealt to CTAs round-robin;
// larger jobs' items come first, so the tail of a batch is made of small items.
struct alignas(128) WorkItem {
    uint64_t base, aux, pairs;
    uint64_t strip_stride, row_stride, stripe_stride, aux_row_stride, aux_stripe_stride;
    uint32_t tile0;   // first tile of the job (local index: stripe * tiles_per_stripe + column tile)
    uint32_t ntiles;
    uint32_t tiles_per_stripe, W, C, n_stripes;
    uint32_t job;     // index of the job (for its tensor map)
    uint8_t p, n, op, i, j, use_tmap, dd_solve, pad0;
    uint8_t pad[20];
};
static_assert(sizeof(WorkItem) == 128, "work items are 128 bytes");
// the producer reads a work item as 32 words spread over a warp
static_assert(offsetof(WorkItem, aux) == 8 && offsetof(WorkItem, pairs) == 16 &&
                  offsetof(WorkItem, strip_stride) == 24 && offsetof(WorkItem, row_stride) == 32 &&
                  offsetof(WorkItem, stripe_stride) == 40 && offsetof(WorkItem, aux_row_stride) == 48 &&
                  offsetof(WorkItem, aux_stripe_stride) == 56 && offsetof(WorkItem, tile0) == 64 &&
                  offsetof(WorkItem, ntiles) == 68 && offsetof(WorkItem, tiles_per_stripe) == 72 &&
                  offsetof(WorkItem, W) == 76 && offsetof(WorkItem, C) == 80 &&
                  offsetof(WorkItem, n_stripes) == 84 && offsetof(WorkItem, job) == 88 &&
                  offsetof(WorkItem, p) == 92 && offsetof(WorkItem, n) == 93 && offsetof(WorkItem, op) == 94 &&
                  offsetof(WorkItem, i) == 95 && offsetof(WorkItem, j) == 96 && offsetof(WorkItem, use_tmap) == 97 &&
                  offsetof(WorkItem, dd_solve) == 98,
              "WorkItem word layout");

struct alignas(128) BatchHeader {
    uint64_t total_tiles;
    uint32_t n_jobs;
    uint32_t slot_bytes;
    uint32_t n_slots;
    uint32_t shape;         // the engine shape the table was planned for
    uint32_t n_items;       // work items after the jobs
    uint32_t ring_bytes;    // shared-memory byte ring shared by up to n_slots stages in flight
    uint64_t items_offset;  // bytes from the header to the first WorkItem
    uint32_t dynamic;       // 0: items dealt round-robin; 1: taken from the global counter
    uint32_t fixed_slots;   // 1: n_slots equal slots of slot_bytes (as single launches); 0: byte ring
    // jobs of p <= 7 run in the column kernel: one ColJob record per job from
    // col_items_offset, grouped by kernel variant (p = 3; p = 5; p = 5 with
    // extended strips; p = 7); col_chunks: the variant's 32-column chunks
    uint64_t col_items_offset;
    uint32_t col_begin[4];
    uint32_t col_count[4];
    uint32_t col_chunks[4];
    uint32_t pad[6];
};
static_assert(sizeof(BatchHeader) == 128, "the job table after the header stays 128-byte aligned");

constexpr uint32_t kColChunk = 32;  // columns per chunk: one per lane
constexpr int kColVariants = 4;

// A small batch table travels in the launch's own parameter block instead of
// a device buffer: no host-to-device copy before the kernels, no graph, no
// counter reset.  Two size classes (a launch copies its whole parameter
// block); the larger leaves room for the engine's LaunchParams within the
// 32764 bytes a kernel's parameters may take.
constexpr uint32_t kParamTableSmall = 8192;
constexpr uint32_t kParamTableLarge = 31744;
template <uint32_t SZ>
struct alignas(128) ParamTable {
    uint8_t bytes[SZ];
};
static_assert(sizeof(LaunchParams) + 128 + kParamTableLarge <= 32764, "kernel parameter block limit");

// The column-kernel variant of a geometry (index into col_begin / col_count),
// or -1 when p > 7.
inline int column_variant(uint32_t p, uint32_t N) {
    if (p == 3) return 0;
    if (p == 5) return N > 5 ? 2 : 1;
    if (p == 7) return 3;
    return -1;
}
static_assert(sizeof(Job) % 128 == 0, "jobs keep their tensor maps 128-byte aligned");

struct Plan {
    uint32_t W, tiles_per_stripe, slot_bytes, n_slots, shape;
};

// Host: tiling for one (p, C) on one engine shape.  Returns false when out of range.
// tile_div > 1 narrows the widest tile the constraints allow by that factor
// (a batch autotuning knob).
bool make_plan(uint32_t p, uint64_t C, uint32_t shape, Plan *out, uint32_t tile_div = 1);

// Host: upload the per-p inverse tables to the current device (once).
cudaError_t upload_inverse_tables();

// Host launchers (rcg_engine.cu).  grid = SMs x ctas_per_sm of the shape (or fewer).
cudaError_t launch_engine(const LaunchParams &prm, uint32_t shape, int grid, cudaStream_t stream);
cudaError_t launch_batch(const uint8_t *table_dev, uint32_t *status, unsigned long long *counter,
                         uint64_t timeout_ns, uint32_t shape, int grid, cudaStream_t stream);
// The tile engine over a small batch table passed as a kernel parameter
// (bytes <= kParamTableLarge): items dealt round-robin, no counter.
cudaError_t launch_batch_param(const uint8_t *table_host, size_t bytes, uint32_t *status, uint64_t timeout_ns,
                               uint32_t shape, int grid, cudaStream_t stream);
cudaError_t engine_init_attributes();
cudaError_t launch_fill(void *dev, uint64_t nbytes, uint64_t seed, uint64_t byte_offset,
                        cudaStream_t stream);
cudaError_t launch_wait_probe(uint32_t *status, uint64_t timeout_ns, cudaStream_t stream);

void inverse_masks(uint32_t p, uint64_t *masks);

// Host ring arithmetic in R = F2[x]/(1 + ... + x^(p-1)) (rcg_ring.cu).
uint64_t ring_reduce(uint32_t p, uint64_t a);
uint32_t order_of_two(uint32_t p);
uint64_t ring_inverse(uint32_t p, uint64_t u);       // 0 when u is not a unit
void trinomial_inverses(uint32_t p, uint64_t *masks);  // [u * p + v] = (1 + x^u + x^v)^(-1)
bool cone_extends(uint32_t p);                        // Theorem 3.3.3 holds for p
// Largest number of data strips for p: 2p - 1 where the extended Q-parity of
// Section 3.3 applies (Theorem 3.3.3), else p (Corollary 3.2.4).
inline uint32_t max_data_strips(uint32_t p) { return cone_extends(p) ? 2 * p - 1 : p; }

// Horizontal representation (rcg_horizontal.cu): the per-prime inverse masks
// (uploaded to the current device), and one launch over n_stripes stripes of
// recovery pair (i, j) or per-stripe pairs; i = N, j = N+1 encodes.
cudaError_t upload_h_tables();
cudaError_t launch_h(uint8_t *base, uint32_t p, uint32_t N, uint64_t strip_bytes, uint64_t strip_stride,
                     uint64_t stripe_stride, uint64_t n_stripes, uint32_t i, uint32_t j, const uint8_t *pairs,
                     uint32_t *status, int sm_count, cudaStream_t stream);

// Z_257 in the horizontal representation (rcg_h257.cu): 32-byte elements,
// base code (N <= 257); per-stripe pairs are 16-bit; i = N, j = N+1 encodes.
cudaError_t launch_h257(uint8_t *base, uint32_t N, uint64_t strip_bytes, uint64_t strip_stride,
                        uint64_t stripe_stride, uint64_t n_stripes, uint32_t i, uint32_t j, const uint16_t *pairs,
                        uint32_t *status, int sm_count, cudaStream_t stream);

// Column kernel (rcg_column.cu): bit-sliced stripes of p <= 7 without shared
// memory.  One job: op OP_ENCODE, OP_RECOVER (pair i < j, or per-stripe
// pairs), OP_DEGRADED (strip j into aux) or OP_UPDATE (data strip i replaced
// by aux).  The record is the kernel parameter of a single launch and, in a
// batch table, the self-contained description of one job: its columns
// (unit = stripe * vps + 16-byte column) are cut into chunks of 32, one column
// per lane, numbered across the variant's jobs from chunk0; a warp loads the
// 128 bytes with one coalesced read.
struct alignas(128) ColJob {
    uint8_t *base;         // stripe 0 of the job
    const uint8_t *pairs;  // recovery: per-stripe (i, j) bytes, or nullptr
    uint8_t *aux;          // degraded read: output; small write: the new strips
    uint64_t rs, ss, st;   // row, strip and stripe strides
    uint64_t ars, ass;     // aux row and stripe strides
    uint64_t chunk0;       // batches: the job's first chunk in its variant's numbering
    uint64_t chunk_end;    // batches: one past its last chunk (the next job's chunk0)
    uint64_t cost0;        // batches: rows the variant's earlier jobs move, (N+2)(p-1) per chunk
    uint64_t n_stripes;
    uint32_t vps;          // 16-byte columns per row, C / 16
    uint32_t N, i, j, op, p;
    uint32_t pad[2];
};
static_assert(sizeof(ColJob) == 128, "a column job is one 128-byte record");
cudaError_t upload_column_tables();
cudaError_t launch_column(const ColJob &job, uint32_t p, uint64_t n_stripes, uint32_t *status, int sm_count,
                          cudaStream_t stream);
// Batches: the column kernel of one variant over the table's ColJob records of that
// variant (persistent grid); the variant's kernel function for graph nodes.
cudaError_t launch_column_batch(int variant, const uint8_t *table_dev, uint32_t *status, int sm_count,
                                cudaStream_t stream);
const void *column_batch_function(int variant);
// The same over a small table passed as a kernel parameter (bytes <= kParamTableLarge).
cudaError_t launch_column_batch_param(int variant, const uint8_t *table_host, size_t bytes, uint32_t *status,
                                      int sm_count, cudaStream_t stream);
// Every kernel of a batch table on `stream`, skipping kernels with no work:
// the column kernels of its p <= 7 jobs, then the tile engine (the path of
// rcg_batch_submit_noalloc; context batches replay the same in a graph).
cudaError_t launch_batch_all(const uint8_t *table_dev, const uint8_t *table_host, uint32_t *status,
                             unsigned long long *counter, uint64_t timeout_ns, uint32_t shape, int sm_count,
                             cudaStream_t stream);
// Every kernel of a small table (bytes <= kParamTableLarge), the table passed
// as a kernel parameter.  With both column and engine work, the column
// kernels run on `side` (forked from and joined back to `stream` by the two
// events) beside the engine, as in the batch graph; side may be null when the
// table has one kind of work.
cudaError_t launch_batch_all_param(const uint8_t *table_host, size_t bytes, uint32_t *status, uint64_t timeout_ns,
                                   uint32_t shape, int sm_count, cudaStream_t stream, cudaStream_t side,
                                   cudaEvent_t fork, cudaEvent_t join);

// Host: the CUDA device of a context.
int ctx_device(const rcg_ctx *ctx);

// Host: validate public jobs and build the batch descriptor table with the
// default copy mode, two-data solve, engine shape and column kernel (used by
// rcg_batch_submit_noalloc), keeping col_capacity bytes of the table for
// column items; *shape receives the shape to launch.
bool noalloc_build_table(const rcg_job *jobs, uint32_t n_jobs, uint8_t *table, size_t capacity,
                         size_t col_capacity, size_t *bytes, uint32_t *shape);



}  // namespace rcg
