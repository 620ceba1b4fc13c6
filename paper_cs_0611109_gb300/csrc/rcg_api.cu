// rcg_api.cu -- host side of librcg: the C ABI declared in include/rcg.h.
// Argument validation, tiling plans, per-context device state (status word,
// inverse tables, batch descriptor tables and their CUDA graphs) and kernel
// launches.  All stripe arithmetic runs in rcg_engine.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/rcg.h"
#include "rcg_internal.h"

using namespace rcg;

namespace {

// Batches in flight per context before a launch waits for the oldest (a
// served stream keeps up to eight batches in flight on its own streams).
constexpr int kBatchRing = 16;

struct BatchSlot {
    uint8_t *host = nullptr;  // pinned descriptor table (header + jobs)
    uint8_t *dev = nullptr;   // device copy read by the kernel
    unsigned long long *counter = nullptr;
    size_t cap_bytes = 0;      // size of the host and device table buffers
    size_t bytes = 0;          // bytes the captured memcpy node copies
    cudaStream_t capture = nullptr;
    cudaGraph_t graph = nullptr;       // kept alive: exec updates name its nodes
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t copy_node = nullptr;
    cudaGraphNode_t col_nodes[kColVariants] = {};  // column kernels of the p <= 7 jobs
    cudaGraphNode_t engine_node = nullptr;         // the tile engine
    int enabled = -1;  // bit v: column variant v enabled; bit 4: tile engine; -1 unknown
    cudaEvent_t done = nullptr;
    uint32_t shape = 0;  // engine shape the graph's kernel node was captured with
    uint64_t ticket = 0;
    bool used = false;
};

}  // namespace

namespace rcg {
struct HostStaging;
HostStaging *host_staging_create();
void host_staging_destroy(HostStaging *h);
rcg_status host_path(HostStaging *h, const rcg_layout *L, uint64_t first, uint64_t n_stripes,
                     const uint8_t *pairs_host, cudaStream_t caller, uint64_t chunk_bytes,
                     rcg_status (*run)(void *, const rcg_layout *, uint64_t, const uint8_t *, cudaStream_t),
                     void *run_arg);
}  // namespace rcg

// A prepared batch: the descriptor-table image and the engine shape.
struct rcg_batch {
    std::vector<uint8_t> image;
    uint32_t shape = 0;
    uint32_t n_jobs = 0;
};

struct rcg_ctx {
    int device = 0;
    int sm_count = 0;
    uint32_t *status = nullptr;
    uint64_t timeout_ns = 2000000000ull;
    int copy_mode = RCG_COPY_AUTO;
    int dd_solve = RCG_SOLVE_CHAIN;
    int shape = RCG_SHAPE_AUTO;
    int batch_schedule = RCG_SCHED_DYNAMIC;
    int column = RCG_COLUMN_AUTO;
    int batch_tables = RCG_TABLES_AUTO;
    // small-table batches with column and engine work: the column kernels on a
    // side stream beside the engine (created on first use)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    // batch tuning (rcg_batch_autotune / rcg_set_batch_tuning)
    int tune_shape = RCG_SHAPE_AUTO;  // engine shape of batches; AUTO = the size rule
    uint64_t tune_item_bytes = 0;     // work-item size; 0 = the rule in build_table
    uint32_t tune_tile_div = 1;       // narrower tiles than the widest allowed
    int tune_ring = RCG_RING_FIXED;   // shared-memory stage discipline of batches
    uint64_t next_ticket = 1;
    BatchSlot slots[kBatchRing];
    rcg::HostStaging *host = nullptr;  // staging of the host-memory calls (lazy)
    uint64_t host_chunk_bytes = 256ull << 20;
};

namespace {

// Switch to the context's device for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

thread_local char g_last_error[256] = "";

rcg_status from_cuda(cudaError_t e, const char *where = "") {
    if (e == cudaSuccess) return RCG_OK;
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", where, cudaGetErrorString(e),
             cudaGetErrorName(e));
    if (e == cudaErrorMemoryAllocation) return RCG_ENOMEM;
    return RCG_ECUDA;
}

bool is_odd_prime(uint32_t p) {
    if (p < 3 || (p & 1) == 0) return false;
    for (uint32_t d = 3; d * d <= p; d += 2)
        if (p % d == 0) return false;
    return true;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

struct Geo {
    uint32_t p, N;
    uint64_t C, rs, ss, st;
};

rcg_status check_layout(const rcg_layout *L, Geo *g) {
    if (!L || !L->base || !aligned16(L->base)) return RCG_EINVAL;
    if (!is_odd_prime(L->p) || L->p > static_cast<uint32_t>(kMaxP)) return RCG_EINVAL;
    if (L->n_data < 1 || L->n_data > max_data_strips(L->p)) return RCG_EINVAL;
    const uint64_t C = L->row_bytes;
    if (C == 0 || (C & 15) || C > 0xffffffffull) return RCG_EINVAL;
    g->p = L->p;
    g->N = L->n_data;
    g->C = C;
    g->rs = L->row_stride ? L->row_stride : C;
    g->ss = L->strip_stride ? L->strip_stride : (L->p - 1) * g->rs;
    g->st = L->stripe_stride ? L->stripe_stride : (L->n_data + 2) * g->ss;
    if (g->rs < C || (g->rs & 15) || (g->ss & 15) || (g->st & 15)) return RCG_EINVAL;
    return RCG_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once (no link against libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// 4-D tiled tensor map over (8-byte column, row, strip, stripe) with a
// (W/8) x (p-1) x 1 x 1 box.  A layout the driver refuses (e.g. strides it
// does not accept) keeps use_tmap = 0 and is served by per-row bulk copies.
// L2 promotion 64 B: measured on GB300 against 256 B, the same on rows whose
// stride is a multiple of 128 bytes, and 3-4 % faster single launches and 10 %
// faster mixed batches at p = 59 where rows start off a line (a 512-byte box
// row there spans five lines).
void attach_tensor_map(Job &J, const Geo &g) {
    J.use_tmap = 0;
    auto encode = tensor_map_encoder();
    if (!encode || J.W > kMaxTileBytes || J.n_stripes == 0) return;
    const cuuint64_t dims[4] = {g.C / 8, g.p - 1, g.N + 2, J.n_stripes};
    const cuuint64_t strides[3] = {g.rs, g.ss, g.st};
    const cuuint32_t box[4] = {J.W / 8, g.p - 1, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(&J.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, J.base, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_64B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    J.use_tmap = r == CUDA_SUCCESS ? 1 : 0;
}

Job base_job(const rcg_ctx *ctx, const rcg_layout *L, const Geo &g, uint64_t first_stripe,
             uint64_t n_stripes, const Plan &pl, bool want_tmap = true) {
    Job J;
    memset(&J, 0, sizeof(J));
    J.base = static_cast<uint8_t *>(L->base) + first_stripe * g.st;
    J.row_stride = g.rs;
    J.strip_stride = g.ss;
    J.stripe_stride = g.st;
    J.n_stripes = static_cast<uint32_t>(n_stripes);
    J.C = static_cast<uint32_t>(g.C);
    J.W = pl.W;
    J.tiles_per_stripe = pl.tiles_per_stripe;
    J.p = static_cast<uint8_t>(g.p);
    J.n = static_cast<uint8_t>(g.N);
    if (want_tmap && ctx->copy_mode == RCG_COPY_AUTO) attach_tensor_map(J, g);
    J.dd_solve = ctx->dd_solve == RCG_SOLVE_TABLE ? 1 : 0;
    return J;
}

rcg_status launch_single(rcg_ctx *ctx, const Job &J, const Plan &pl, cudaStream_t stream) {
    LaunchParams prm;
    memset(&prm, 0, sizeof(prm));
    prm.job0 = J;
    prm.n_jobs = 1;
    prm.slot_bytes = pl.slot_bytes;
    prm.n_slots = pl.n_slots;
    prm.dynamic_sched = 0;
    prm.total_tiles = static_cast<uint64_t>(J.n_stripes) * J.tiles_per_stripe;
    prm.status = ctx->status;
    prm.timeout_ns = ctx->timeout_ns;
    if (prm.total_tiles == 0) return RCG_OK;
    const uint64_t grid = std::min<uint64_t>(
        prm.total_tiles, static_cast<uint64_t>(ctx->sm_count) * shape_info(pl.shape).ctas_per_sm);
    return from_cuda(launch_engine(prm, pl.shape, static_cast<int>(grid), stream));
}

// The column kernel serves single-operation launches of p <= 7 unless the
// context asks for the tile engine.
bool use_column(const rcg_ctx *ctx, const Geo &g) { return ctx->column == RCG_COLUMN_AUTO && g.p <= 7; }

ColJob column_job(const rcg_layout *L, const Geo &g, uint64_t first, uint32_t op, uint32_t i, uint32_t j,
                  const uint8_t *pairs, void *aux = nullptr, uint64_t ars = 0) {
    ColJob J;
    memset(&J, 0, sizeof(J));
    J.base = static_cast<uint8_t *>(L->base) + first * g.st;
    J.pairs = pairs;
    J.aux = static_cast<uint8_t *>(aux);
    J.rs = g.rs;
    J.ss = g.ss;
    J.st = g.st;
    J.ars = ars;
    J.ass = (g.p - 1) * ars;
    J.vps = static_cast<uint32_t>(g.C / 16);
    J.N = g.N;
    J.i = i;
    J.j = j;
    J.op = op;
    J.p = g.p;
    return J;
}

rcg_status launch_column_op(rcg_ctx *ctx, const ColJob &J, const Geo &g, uint64_t n, cudaStream_t stream) {
    DeviceGuard guard(ctx->device);
    return from_cuda(launch_column(J, g.p, n, ctx->status, ctx->sm_count, stream), "column kernel launch");
}

uint64_t now_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return static_cast<uint64_t>(ts.tv_sec) * 1000000000ull + ts.tv_nsec;
}

void sleep_us(long us) {
    timespec ts = {0, us * 1000};
    nanosleep(&ts, nullptr);
}

// Poll an event until it completes or timeout_ns passes.
rcg_status wait_event(cudaEvent_t ev, uint64_t timeout_ns) {
    const uint64_t t0 = now_ns();
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return RCG_OK;
        if (e != cudaErrorNotReady) return from_cuda(e);
        if (now_ns() - t0 > timeout_ns) return RCG_ETIMEOUT;
        sleep_us(20);
    }
}

void free_slot(BatchSlot &s) {
    if (s.exec) cudaGraphExecDestroy(s.exec);
    if (s.graph) cudaGraphDestroy(s.graph);
    if (s.host) cudaFreeHost(s.host);
    if (s.dev) cudaFree(s.dev);
    if (s.counter) cudaFree(s.counter);
    if (s.done) cudaEventDestroy(s.done);
    if (s.capture) cudaStreamDestroy(s.capture);
    s = BatchSlot();
}

}  // namespace

// ====================================================================== plan

bool rcg::make_plan(uint32_t p, uint64_t C, uint32_t shape, Plan *out, uint32_t tile_div) {
    if (!is_odd_prime(p) || p > static_cast<uint32_t>(kMaxP) || C == 0 || (C & 15) || tile_div == 0) return false;
    const ShapeInfo si = shape_info(shape);
    const uint64_t nvec_total = C / 16;
    uint64_t nvec_max = si.max_items / p;                                  // items per tile
    nvec_max = std::min<uint64_t>(nvec_max, kMaxSlotBytes / ((p - 1) * 16ull));
    nvec_max = std::min<uint64_t>(nvec_max, kMaxTileBytes / 16);           // TMA box row
    nvec_max = std::min<uint64_t>(nvec_max, si.ring_bytes / si.min_slots / ((p - 1) * 16ull));
    if (nvec_max == 0) return false;
    nvec_max = std::max<uint64_t>(1, nvec_max / tile_div);
    for (;;) {
        const uint64_t tiles = (nvec_total + nvec_max - 1) / nvec_max;
        if (tiles > 0xffffffffull) return false;
        const uint64_t nvec = (nvec_total + tiles - 1) / tiles;  // balanced tile widths
        out->W = static_cast<uint32_t>(nvec * 16);
        out->tiles_per_stripe = static_cast<uint32_t>(tiles);
        out->slot_bytes = static_cast<uint32_t>(((p - 1) * out->W + 127) & ~127u);
        out->n_slots = std::min<uint32_t>(kMaxSlots, si.ring_bytes / out->slot_bytes);
        out->shape = shape;
        if (out->n_slots >= si.min_slots) return true;
        if (--nvec_max == 0) return false;  // rounding of the slot size: narrow the tile
    }
}

// The engine shape for a launch: the context's explicit choice, else pair
// (two CTAs per SM: more CTAs in flight, epilogues overlapping streaming)
// for launches under 256 MB of traffic, and wide (one CTA per SM with the
// deepest ring) above that, where streaming throughput decides.
constexpr uint64_t kSmallLaunchBytes = 256ull << 20;

uint32_t choose_shape(const rcg_ctx *ctx, uint64_t launch_bytes) {
    if (ctx->shape == RCG_SHAPE_WIDE) return SHAPE_WIDE;
    if (ctx->shape == RCG_SHAPE_PAIR) return SHAPE_PAIR;
    return launch_bytes < kSmallLaunchBytes ? SHAPE_PAIR : SHAPE_WIDE;
}

uint64_t launch_bytes(const Geo &g, uint64_t n_stripes) {
    return (g.N + 2ull) * (g.p - 1) * g.C * n_stripes;
}

// =================================================================== C ABI

extern "C" {

uint32_t rcg_abi_version(void) { return RCG_ABI_VERSION; }

const char *rcg_last_error(void) { return g_last_error; }

const char *rcg_status_str(rcg_status s) {
    switch (s) {
        case RCG_OK: return "ok";
        case RCG_EINVAL: return "invalid argument";
        case RCG_ENOMEM: return "out of memory";
        case RCG_ECUDA: return "CUDA runtime error";
        case RCG_ETIMEOUT: return "timed out";
        case RCG_EBUSY: return "busy";
        case RCG_EUNSUPPORTED: return "unsupported device or parameter";
        case RCG_EDEVICE: return "device-side error";
    }
    return "unknown status";
}

rcg_status rcg_inverse_table(uint32_t p, uint64_t *masks) {
    if (!masks || !is_odd_prime(p) || p > static_cast<uint32_t>(kMaxP)) return RCG_EINVAL;
    inverse_masks(p, masks);
    return RCG_OK;
}

rcg_status rcg_prime_info(uint32_t p, rcg_prime_info_t *out) {
    if (!out || !is_odd_prime(p) || p > static_cast<uint32_t>(kMaxP)) return RCG_EINVAL;
    out->ord2 = order_of_two(p);
    out->is_field = out->ord2 == p - 1 ? 1u : 0u;
    out->extends = cone_extends(p) ? 1u : 0u;
    out->max_data = max_data_strips(p);
    return RCG_OK;
}

rcg_status rcg_ring_inverse(uint32_t p, uint64_t a, uint64_t *inv) {
    if (!inv || !is_odd_prime(p) || p > static_cast<uint32_t>(kMaxP)) return RCG_EINVAL;
    if (a >> (p - 1)) return RCG_EINVAL;  // not a residue modulo f
    *inv = ring_inverse(p, a);
    return *inv ? RCG_OK : RCG_EINVAL;
}

rcg_status rcg_plan(uint32_t p, uint64_t row_bytes, rcg_plan_info *out) {
    Plan pl;
    static const rcg_ctx defaults;
    if (!out || !is_odd_prime(p) || p > static_cast<uint32_t>(kMaxP)) return RCG_EINVAL;
    if (!make_plan(p, row_bytes, choose_shape(&defaults, ~0ull), &pl)) return RCG_EINVAL;
    const ShapeInfo si = shape_info(pl.shape);
    out->tile_bytes = pl.W;
    out->tiles_per_stripe = pl.tiles_per_stripe;
    out->slot_bytes = pl.slot_bytes;
    out->n_slots = pl.n_slots;
    out->max_items = si.max_items;
    out->smem_bytes = si.fixed_smem + pl.n_slots * pl.slot_bytes;
    out->ctas_per_sm = si.ctas_per_sm;
    out->shape = pl.shape;
    return RCG_OK;
}

rcg_status rcg_create(int device, rcg_ctx **out) {
    if (!out) return RCG_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return RCG_EUNSUPPORTED;
    DeviceGuard guard(device);
    if (!guard.ok) return RCG_ECUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return RCG_ECUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return RCG_EUNSUPPORTED;
    rcg_ctx *ctx = new (std::nothrow) rcg_ctx();
    if (!ctx) return RCG_ENOMEM;
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    rcg_status st = from_cuda(upload_inverse_tables());
    if (st == RCG_OK) st = from_cuda(upload_h_tables(), "horizontal tables");
    if (st == RCG_OK) st = from_cuda(upload_column_tables(), "column kernel tables");
    if (st == RCG_OK) st = from_cuda(engine_init_attributes());
    if (st == RCG_OK) st = from_cuda(cudaMalloc(&ctx->status, 256));
    if (st == RCG_OK) st = from_cuda(cudaMemset(ctx->status, 0, 256));
    if (st == RCG_OK) st = from_cuda(cudaDeviceSynchronize());
    if (st != RCG_OK) {
        if (ctx->status) cudaFree(ctx->status);
        delete ctx;
        return st;
    }
    *out = ctx;
    return RCG_OK;
}

rcg_status rcg_destroy(rcg_ctx *ctx) {
    if (!ctx) return RCG_EINVAL;
    DeviceGuard guard(ctx->device);
    for (auto &s : ctx->slots) {
        if (s.done) cudaEventSynchronize(s.done);
        free_slot(s);
    }
    host_staging_destroy(ctx->host);
    if (ctx->side) cudaStreamSynchronize(ctx->side);
    if (ctx->fork) cudaEventDestroy(ctx->fork);
    if (ctx->join) cudaEventDestroy(ctx->join);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->status) cudaFree(ctx->status);
    delete ctx;
    return RCG_OK;
}

rcg_status rcg_set_copy_mode(rcg_ctx *ctx, int mode) {
    if (!ctx || (mode != RCG_COPY_AUTO && mode != RCG_COPY_ROWS)) return RCG_EINVAL;
    ctx->copy_mode = mode;
    return RCG_OK;
}

rcg_status rcg_set_dd_solve(rcg_ctx *ctx, int solve) {
    if (!ctx || (solve != RCG_SOLVE_CHAIN && solve != RCG_SOLVE_TABLE)) return RCG_EINVAL;
    ctx->dd_solve = solve;
    return RCG_OK;
}

rcg_status rcg_set_engine_shape(rcg_ctx *ctx, int shape) {
    if (!ctx || (shape != RCG_SHAPE_AUTO && shape != RCG_SHAPE_WIDE && shape != RCG_SHAPE_PAIR))
        return RCG_EINVAL;
    ctx->shape = shape;
    return RCG_OK;
}

rcg_status rcg_set_column_kernel(rcg_ctx *ctx, int mode) {
    if (!ctx || (mode != RCG_COLUMN_AUTO && mode != RCG_COLUMN_OFF)) return RCG_EINVAL;
    ctx->column = mode;
    return RCG_OK;
}

rcg_status rcg_set_batch_tables(rcg_ctx *ctx, int mode) {
    if (!ctx || (mode != RCG_TABLES_AUTO && mode != RCG_TABLES_DEVICE)) return RCG_EINVAL;
    ctx->batch_tables = mode;
    return RCG_OK;
}

rcg_status rcg_set_batch_schedule(rcg_ctx *ctx, int schedule) {
    if (!ctx || (schedule != RCG_SCHED_STATIC && schedule != RCG_SCHED_DYNAMIC)) return RCG_EINVAL;
    ctx->batch_schedule = schedule;
    return RCG_OK;
}

rcg_status rcg_set_host_chunk(rcg_ctx *ctx, uint64_t bytes) {
    if (!ctx || bytes < 4096) return RCG_EINVAL;
    ctx->host_chunk_bytes = bytes;
    return RCG_OK;
}

rcg_status rcg_set_timeout(rcg_ctx *ctx, uint64_t timeout_ns) {
    if (!ctx || timeout_ns == 0) return RCG_EINVAL;
    ctx->timeout_ns = timeout_ns;
    return RCG_OK;
}

rcg_status rcg_last_device_status(rcg_ctx *ctx, uint32_t *code) {
    if (!ctx || !code) return RCG_EINVAL;
    DeviceGuard guard(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return from_cuda(e);
    uint32_t v = 0;
    e = cudaMemcpy(&v, ctx->status, sizeof(v), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof(v));
    if (e != cudaSuccess) return from_cuda(e);
    *code = v;
    return v ? RCG_EDEVICE : RCG_OK;
}

rcg_status rcg_encode(rcg_ctx *ctx, const rcg_layout *L, uint64_t first_stripe, uint64_t n_stripes,
                      void *stream) {
    Geo g;
    if (!ctx) return RCG_EINVAL;
    rcg_status st = check_layout(L, &g);
    if (st) return st;
    if (n_stripes == 0) return RCG_OK;
    if (n_stripes > 0x7fffffffull) return RCG_EINVAL;
    if (use_column(ctx, g))
        return launch_column_op(ctx, column_job(L, g, first_stripe, OP_ENCODE, 0, 0, nullptr), g, n_stripes,
                                static_cast<cudaStream_t>(stream));
    Plan pl;
    if (!make_plan(g.p, g.C, choose_shape(ctx, launch_bytes(g, n_stripes)), &pl)) return RCG_EINVAL;
    Job J = base_job(ctx, L, g, first_stripe, n_stripes, pl);
    J.op = OP_ENCODE;
    DeviceGuard guard(ctx->device);
    return launch_single(ctx, J, pl, static_cast<cudaStream_t>(stream));
}

rcg_status rcg_recover(rcg_ctx *ctx, const rcg_layout *L, uint64_t stripe, uint32_t i, uint32_t j,
                       void *stream) {
    Geo g;
    if (!ctx) return RCG_EINVAL;
    rcg_status st = check_layout(L, &g);
    if (st) return st;
    if (!(i < j && j <= g.N + 1)) return RCG_EINVAL;
    if (use_column(ctx, g))
        return launch_column_op(ctx, column_job(L, g, stripe, OP_RECOVER, i, j, nullptr), g, 1,
                                static_cast<cudaStream_t>(stream));
    Plan pl;
    if (!make_plan(g.p, g.C, choose_shape(ctx, launch_bytes(g, 1)), &pl)) return RCG_EINVAL;
    Job J = base_job(ctx, L, g, stripe, 1, pl);
    J.op = OP_RECOVER;
    J.i = static_cast<uint8_t>(i);
    J.j = static_cast<uint8_t>(j);
    DeviceGuard guard(ctx->device);
    return launch_single(ctx, J, pl, static_cast<cudaStream_t>(stream));
}

rcg_status rcg_recover_many(rcg_ctx *ctx, const rcg_layout *L, uint64_t first_stripe,
                            uint64_t n_stripes, const uint8_t *pairs, void *stream) {
    Geo g;
    if (!ctx || !pairs) return RCG_EINVAL;
    rcg_status st = check_layout(L, &g);
    if (st) return st;
    if (n_stripes == 0) return RCG_OK;
    if (n_stripes > 0x7fffffffull) return RCG_EINVAL;
    if (use_column(ctx, g))
        return launch_column_op(ctx, column_job(L, g, first_stripe, OP_RECOVER, 0, 0, pairs), g, n_stripes,
                                static_cast<cudaStream_t>(stream));
    Plan pl;
    if (!make_plan(g.p, g.C, choose_shape(ctx, launch_bytes(g, n_stripes)), &pl)) return RCG_EINVAL;
    Job J = base_job(ctx, L, g, first_stripe, n_stripes, pl);
    J.op = OP_RECOVER;
    J.pairs = pairs;
    DeviceGuard guard(ctx->device);
    return launch_single(ctx, J, pl, static_cast<cudaStream_t>(stream));
}

rcg_status rcg_update(rcg_ctx *ctx, const rcg_layout *L, uint64_t stripe, uint32_t i,
                      const void *new_strip, uint64_t new_row_stride, void *stream) {
    Geo g;
    if (!ctx || !new_strip || !aligned16(new_strip)) return RCG_EINVAL;
    rcg_status st = check_layout(L, &g);
    if (st) return st;
    if (i >= g.N) return RCG_EINVAL;
    const uint64_t ars = new_row_stride ? new_row_stride : g.C;
    if (ars < g.C || (ars & 15)) return RCG_EINVAL;
    if (use_column(ctx, g))
        return launch_column_op(ctx, column_job(L, g, stripe, OP_UPDATE, i, 0, nullptr, const_cast<void *>(new_strip), ars),
                                g, 1, static_cast<cudaStream_t>(stream));
    Plan pl;
    if (!make_plan(g.p, g.C, choose_shape(ctx, launch_bytes(g, 1)), &pl)) return RCG_EINVAL;
    Job J = base_job(ctx, L, g, stripe, 1, pl);
    J.op = OP_UPDATE;
    J.i = static_cast<uint8_t>(i);
    J.aux = static_cast<uint8_t *>(const_cast<void *>(new_strip));
    J.aux_row_stride = ars;
    J.aux_stripe_stride = (g.p - 1) * ars;
    DeviceGuard guard(ctx->device);
    return launch_single(ctx, J, pl, static_cast<cudaStream_t>(stream));
}

rcg_status rcg_degraded_read(rcg_ctx *ctx, const rcg_layout *L, uint64_t stripe, uint32_t j,
                             void *out, uint64_t out_row_stride, void *stream) {
    Geo g;
    if (!ctx || !out || !aligned16(out)) return RCG_EINVAL;
    rcg_status st = check_layout(L, &g);
    if (st) return st;
    if (j > g.N + 1) return RCG_EINVAL;
    const uint64_t ors = out_row_stride ? out_row_stride : g.C;
    if (ors < g.C || (ors & 15)) return RCG_EINVAL;
    if (use_column(ctx, g))
        return launch_column_op(ctx, column_job(L, g, stripe, OP_DEGRADED, 0, j, nullptr, out, ors), g, 1,
                                static_cast<cudaStream_t>(stream));
    Plan pl;
    if (!make_plan(g.p, g.C, choose_shape(ctx, launch_bytes(g, 1)), &pl)) return RCG_EINVAL;
    Job J = base_job(ctx, L, g, stripe, 1, pl);
    J.op = OP_DEGRADED;
    J.j = static_cast<uint8_t>(j);
    J.aux = static_cast<uint8_t *>(out);
    J.aux_row_stride = ors;
    J.aux_stripe_stride = (g.p - 1) * ors;
    DeviceGuard guard(ctx->device);
    return launch_single(ctx, J, pl, static_cast<cudaStream_t>(stream));
}

// ================================================== horizontal representation

static rcg_status check_hlayout(const rcg_hlayout *L, uint64_t *ss, uint64_t *st) {
    if (!L || !L->base || !aligned16(L->base)) return RCG_EINVAL;
    if (L->p != 3 && L->p != 5 && L->p != 17 && L->p != 257) return RCG_EINVAL;
    if (L->p == 257) {  // 32-byte elements, base code
        if ((reinterpret_cast<uintptr_t>(L->base) & 31) || L->n_data < 1 || L->n_data > 257 ||
            L->strip_bytes == 0 || (L->strip_bytes & 31) || L->strip_bytes / 32 > 0xffffffffull)
            return RCG_EINVAL;
        *ss = L->strip_stride ? L->strip_stride : L->strip_bytes;
        *st = L->stripe_stride ? L->stripe_stride : (L->n_data + 2ull) * *ss;
        if (*ss < L->strip_bytes || (*ss & 31) || (*st & 31)) return RCG_EINVAL;
        return RCG_OK;
    }
    if (L->n_data < 1 || L->n_data > max_data_strips(L->p)) return RCG_EINVAL;
    if (L->strip_bytes == 0 || (L->strip_bytes & 15) || L->strip_bytes / 16 > 0xffffffffull) return RCG_EINVAL;
    *ss = L->strip_stride ? L->strip_stride : L->strip_bytes;
    *st = L->stripe_stride ? L->stripe_stride : (L->n_data + 2ull) * *ss;
    if (*ss < L->strip_bytes || (*ss & 15) || (*st & 15)) return RCG_EINVAL;
    return RCG_OK;
}

static rcg_status h_launch(rcg_ctx *ctx, const rcg_hlayout *L, uint64_t first, uint64_t n, uint32_t i, uint32_t j,
                           const uint8_t *pairs, void *stream) {
    uint64_t ss, st;
    if (!ctx) return RCG_EINVAL;
    rcg_status s = check_hlayout(L, &ss, &st);
    if (s) return s;
    if (n == 0) return RCG_OK;
    DeviceGuard guard(ctx->device);
    if (L->p == 257)
        return from_cuda(launch_h257(static_cast<uint8_t *>(L->base) + first * st, L->n_data, L->strip_bytes, ss, st,
                                     n, i, j, reinterpret_cast<const uint16_t *>(pairs), ctx->status, ctx->sm_count,
                                     static_cast<cudaStream_t>(stream)),
                         "Z_257 kernel launch");
    return from_cuda(launch_h(static_cast<uint8_t *>(L->base) + first * st, L->p, L->n_data, L->strip_bytes, ss, st,
                              n, i, j, pairs, ctx->status, ctx->sm_count, static_cast<cudaStream_t>(stream)),
                     "horizontal kernel launch");
}

rcg_status rcg_h_encode(rcg_ctx *ctx, const rcg_hlayout *L, uint64_t first_stripe, uint64_t n_stripes,
                        void *stream) {
    if (!L) return RCG_EINVAL;
    return h_launch(ctx, L, first_stripe, n_stripes, L->n_data, L->n_data + 1, nullptr, stream);
}

rcg_status rcg_h_recover(rcg_ctx *ctx, const rcg_hlayout *L, uint64_t stripe, uint32_t i, uint32_t j,
                         void *stream) {
    if (!L || !(i < j && j <= L->n_data + 1)) return RCG_EINVAL;
    return h_launch(ctx, L, stripe, 1, i, j, nullptr, stream);
}

rcg_status rcg_h_recover_many(rcg_ctx *ctx, const rcg_hlayout *L, uint64_t first_stripe, uint64_t n_stripes,
                              const uint8_t *pairs, void *stream) {
    if (!L || !pairs) return RCG_EINVAL;
    if (L->p == 257 && (reinterpret_cast<uintptr_t>(pairs) & 3)) return RCG_EINVAL;  // 16-bit pairs
    return h_launch(ctx, L, first_stripe, n_stripes, 0, 0, pairs, stream);
}

// ================================================================= batches

// want_tmap = false: the job runs in the column kernel, which needs no tensor map.
static rcg_status build_job(const rcg_ctx *ctx, const rcg_job &in, uint32_t shape, Job *out, Plan *pl,
                            bool want_tmap = true) {
    Geo g;
    rcg_status st = check_layout(&in.layout, &g);
    if (st) return st;
    if (in.n_stripes == 0 || in.n_stripes > 0x7fffffffull) return RCG_EINVAL;
    if (!make_plan(g.p, g.C, shape, pl, ctx->tune_tile_div)) return RCG_EINVAL;
    Job J = base_job(ctx, &in.layout, g, in.first_stripe, in.n_stripes, *pl, want_tmap);
    const uint64_t ars = in.aux_row_stride ? in.aux_row_stride : g.C;
    const uint64_t ass = in.aux_stripe_stride ? in.aux_stripe_stride : (g.p - 1) * ars;
    switch (in.op) {
        case RCG_OP_ENCODE:
            J.op = OP_ENCODE;
            break;
        case RCG_OP_RECOVER:
            if (!(in.i < in.j && in.j <= g.N + 1)) return RCG_EINVAL;
            J.op = OP_RECOVER;
            J.i = static_cast<uint8_t>(in.i);
            J.j = static_cast<uint8_t>(in.j);
            break;
        case RCG_OP_DEGRADED_READ:
        case RCG_OP_UPDATE:
            if (in.op == RCG_OP_DEGRADED_READ ? in.j > g.N + 1 : in.i >= g.N) return RCG_EINVAL;
            if (!in.aux || !aligned16(in.aux) || ars < g.C || (ars & 15) || (ass & 15)) return RCG_EINVAL;
            J.op = in.op == RCG_OP_UPDATE ? OP_UPDATE : OP_DEGRADED;
            J.i = static_cast<uint8_t>(in.i);
            J.j = static_cast<uint8_t>(in.j);
            J.aux = static_cast<uint8_t *>(const_cast<void *>(in.aux));
            J.aux_row_stride = ars;
            J.aux_stripe_stride = ass;
            break;
        default:
            return RCG_EINVAL;
    }
    *out = J;
    return RCG_OK;
}

// Capture the slot's graph: descriptor-table copy -> tile-counter reset ->
// {the column kernels of the four p <= 7 variants, the persistent tile engine
// of the given shape}, each kernel depending on the reset directly (they work
// on different jobs).  A launch enables only the kernels its table has work
// for.
static rcg_status capture_slot(rcg_ctx *ctx, BatchSlot &s, uint32_t shape) {
    if (s.exec) cudaGraphExecDestroy(s.exec);
    if (s.graph) cudaGraphDestroy(s.graph);
    s.exec = nullptr;
    s.graph = nullptr;
    s.copy_node = nullptr;
    s.engine_node = nullptr;
    for (auto &n : s.col_nodes) n = nullptr;
    s.enabled = -1;
    const size_t bytes = s.cap_bytes;
    s.bytes = bytes;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaSuccess;
    const char *where = "graph capture";
    // fan-out: every kernel node depends on the counter reset (which follows
    // the table copy) directly, never through a node a launch may disable
    cudaStream_t side[kColVariants] = {};
    cudaEvent_t fork = nullptr, join[kColVariants] = {};
    for (int v = 0; v < kColVariants && e == cudaSuccess; ++v) {
        e = cudaStreamCreateWithFlags(&side[v], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[v], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(s.capture, cudaStreamCaptureModeThreadLocal);
    else where = "capture streams";
    if (e == cudaSuccess) {
        cudaError_t e1 = cudaMemcpyAsync(s.dev, s.host, bytes, cudaMemcpyHostToDevice, s.capture);
        cudaError_t e2 = cudaMemsetAsync(s.counter, 0, sizeof(unsigned long long), s.capture);
        cudaError_t e3 = cudaEventRecord(fork, s.capture);
        for (int v = 0; v < kColVariants && e3 == cudaSuccess; ++v) {
            e3 = cudaStreamWaitEvent(side[v], fork, 0);
            if (e3 == cudaSuccess) e3 = launch_column_batch(v, s.dev, ctx->status, ctx->sm_count, side[v]);
            if (e3 == cudaSuccess) e3 = cudaEventRecord(join[v], side[v]);
        }
        if (e3 == cudaSuccess)
            e3 = launch_batch(s.dev, ctx->status, s.counter, ctx->timeout_ns, shape,
                              ctx->sm_count * static_cast<int>(shape_info(shape).ctas_per_sm), s.capture);
        for (int v = 0; v < kColVariants && e3 == cudaSuccess; ++v) e3 = cudaStreamWaitEvent(s.capture, join[v], 0);
        e = cudaStreamEndCapture(s.capture, &graph);
        if (e1 != cudaSuccess) { e = e1; where = "captured table copy"; }
        else if (e2 != cudaSuccess) { e = e2; where = "captured counter reset"; }
        else if (e3 != cudaSuccess) { e = e3; where = "captured kernel launch"; }
    }
    for (int v = 0; v < kColVariants; ++v) {
        if (join[v]) cudaEventDestroy(join[v]);
        if (side[v]) cudaStreamDestroy(side[v]);
    }
    if (fork) cudaEventDestroy(fork);
    if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&s.exec, graph, 0);
        where = "graph instantiate";
    }
    if (e == cudaSuccess) {
        size_t n = 0;
        cudaGraphGetNodes(graph, nullptr, &n);
        std::vector<cudaGraphNode_t> nodes(n);
        cudaGraphGetNodes(graph, nodes.data(), &n);
        for (auto nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) != cudaSuccess) continue;
            if (t == cudaGraphNodeTypeMemcpy) s.copy_node = nd;
            if (t != cudaGraphNodeTypeKernel) continue;
            cudaKernelNodeParams kp;
            if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
            bool col = false;
            for (int v = 0; v < kColVariants; ++v)
                if (kp.func == column_batch_function(v)) {
                    s.col_nodes[v] = nd;
                    col = true;
                }
            if (!col) s.engine_node = nd;
        }
        bool all = s.copy_node && s.engine_node;
        for (auto nd : s.col_nodes) all = all && nd;
        if (!all) e = cudaErrorUnknown;
        where = "graph nodes";
    }
    s.graph = graph;
    if (e != cudaSuccess) {
        free_slot(s);
        return from_cuda(e, where);
    }
    s.shape = shape;
    return RCG_OK;
}

// Enable the graph's kernels that the table has work for (bit v: column
// variant v; bit 4: the tile engine).  Only kernel nodes are switched: the
// table copy and the counter reset always run.  Measured on GB300: with the
// counter reset (the memset between the copy and the kernels) disabled, a
// kernel of a back-to-back batch could start before its table copy had
// landed (1 to 4 of 400 column-only batches read the previous table).
static cudaError_t set_enabled(BatchSlot &s, int mask) {
    if (mask == s.enabled) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < kColVariants && e == cudaSuccess; ++v)
        e = cudaGraphNodeSetEnabled(s.exec, s.col_nodes[v], (mask >> v) & 1);
    if (e == cudaSuccess) e = cudaGraphNodeSetEnabled(s.exec, s.engine_node, (mask >> 4) & 1);
    s.enabled = e == cudaSuccess ? mask : -1;
    return e;
}

static int work_mask(const BatchHeader &h) {
    int m = h.n_items ? 16 : 0;
    for (int v = 0; v < kColVariants; ++v)
        if (h.col_count[v]) m |= 1 << v;
    return m;
}

// (Re)allocate a batch slot for a table of `bytes`; recapture its graph when
// the engine shape changes.
static rcg_status prepare_slot(rcg_ctx *ctx, BatchSlot &s, size_t bytes, uint32_t shape) {
    if (s.cap_bytes >= bytes && s.exec) return s.shape == shape ? RCG_OK : capture_slot(ctx, s, shape);
    free_slot(s);
    const size_t cap = std::max<size_t>(bytes, 64 * 1024);
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void **>(&s.host), cap, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&s.dev), cap);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&s.counter), sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        free_slot(s);
        return from_cuda(e, "batch slot allocation");
    }
    memset(s.host, 0, cap);
    s.cap_bytes = cap;
    return capture_slot(ctx, s, shape);
}

// One engine shape for a whole batch: the context's explicit choice, else
// by the batch's total traffic.
static uint32_t batch_shape(const rcg_ctx *ctx, const rcg_job *jobs, uint32_t n_jobs) {
    if (ctx->tune_shape == RCG_SHAPE_WIDE) return SHAPE_WIDE;
    if (ctx->tune_shape == RCG_SHAPE_PAIR) return SHAPE_PAIR;
    uint64_t bytes = 0;
    for (uint32_t k = 0; k < n_jobs; ++k) {
        Geo g;
        if (check_layout(&jobs[k].layout, &g) == RCG_OK) bytes += launch_bytes(g, jobs[k].n_stripes);
    }
    return choose_shape(ctx, bytes);
}

// The descriptor table of a batch for one engine shape, built in `out`:
// header, the tile-engine jobs (with their tensor maps), work items of the
// tile engine (runs of tiles of one job of
// roughly equal bytes; the items of larger jobs come first so the batch ends
// on small items), then the column items of the p <= 7 jobs (when the
// context uses the column kernel), grouped by variant.  max_items (0: no
// limit) coarsens the work items to fit a fixed table; more column items
// than max_col_items (0: no limit) is RCG_EINVAL.
static rcg_status build_table(const rcg_ctx *ctx, const rcg_job *jobs, uint32_t n_jobs, uint32_t shape,
                              uint64_t max_items, std::vector<uint8_t> &out, uint64_t max_col_items = 0) {
    std::vector<Job> table(n_jobs);
    std::vector<uint64_t> tiles(n_jobs);
    std::vector<int> variant(n_jobs, -1);
    uint64_t total = 0;
    uint32_t slot_bytes = 0;
    for (uint32_t k = 0; k < n_jobs; ++k) {
        Plan pl;
        if (ctx->column == RCG_COLUMN_AUTO) variant[k] = column_variant(jobs[k].layout.p, jobs[k].layout.n_data);
        rcg_status st = build_job(ctx, jobs[k], shape, &table[k], &pl, variant[k] < 0);
        if (st) return st;
        if (variant[k] >= 0) {
            tiles[k] = 0;
            continue;
        }
        tiles[k] = static_cast<uint64_t>(table[k].n_stripes) * table[k].tiles_per_stripe;
        table[k].tile_begin = total;
        total += tiles[k];
        slot_bytes = std::max(slot_bytes, pl.slot_bytes);
    }
    // Item size by bytes: about 1/16 of a CTA's share of the batch, clamped to
    // [256 KB, 2 MB], so the largest stripes do not leave one CTA working
    // alone at the end; max_items (the no-allocation table) can only raise it.
    uint64_t batch_bytes = 0;
    for (uint32_t k = 0; k < n_jobs; ++k)
        if (variant[k] < 0)
            batch_bytes += static_cast<uint64_t>(table[k].n_stripes) * (table[k].n + 2u) * (table[k].p - 1u) * table[k].C;
    const uint64_t ctas = static_cast<uint64_t>(ctx->sm_count ? ctx->sm_count : 152) * shape_info(shape).ctas_per_sm;
    const uint64_t target = ctx->tune_item_bytes
                                ? ctx->tune_item_bytes
                                : std::min<uint64_t>(2ull << 20, std::max<uint64_t>(256ull << 10, batch_bytes / (ctas * 16)));
    std::vector<uint64_t> per(n_jobs, 1);
    uint64_t n_items_est = 0;
    for (uint32_t k = 0; k < n_jobs; ++k) {
        if (variant[k] >= 0) continue;
        const uint64_t tile_bytes = (table[k].n + 2ull) * (table[k].p - 1u) * table[k].W;
        per[k] = std::max<uint64_t>(1, target / tile_bytes);
        n_items_est += (tiles[k] + per[k] - 1) / per[k];
    }
    if (max_items && n_items_est > max_items) {  // coarser items to fit the table
        const uint64_t scale = (n_items_est + max_items - 1) / max_items + 1;
        for (uint32_t k = 0; k < n_jobs; ++k) per[k] *= scale;
    }
    std::vector<uint32_t> order(n_jobs);
    for (uint32_t k = 0; k < n_jobs; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
        return table[x].n_stripes * static_cast<uint64_t>(table[x].p - 1) * table[x].C * (table[x].n + 2u) >
               table[y].n_stripes * static_cast<uint64_t>(table[y].p - 1) * table[y].C * (table[y].n + 2u);
    });
    // the Job entries (tensor maps) of tile-engine jobs only, in job order
    std::vector<uint32_t> tile_index(n_jobs, 0);
    std::vector<Job> tile_jobs;
    for (uint32_t k = 0; k < n_jobs; ++k)
        if (variant[k] < 0) {
            tile_index[k] = static_cast<uint32_t>(tile_jobs.size());
            tile_jobs.push_back(table[k]);
        }
    std::vector<WorkItem> items;
    for (uint32_t k : order) {
        if (variant[k] >= 0) continue;
        const Job &J = table[k];
        WorkItem w;
        memset(&w, 0, sizeof(w));
        w.base = reinterpret_cast<uint64_t>(J.base);
        w.aux = reinterpret_cast<uint64_t>(J.aux);
        w.pairs = reinterpret_cast<uint64_t>(J.pairs);
        w.strip_stride = J.strip_stride;
        w.row_stride = J.row_stride;
        w.stripe_stride = J.stripe_stride;
        w.aux_row_stride = J.aux_row_stride;
        w.aux_stripe_stride = J.aux_stripe_stride;
        w.tiles_per_stripe = J.tiles_per_stripe;
        w.W = J.W;
        w.C = J.C;
        w.n_stripes = J.n_stripes;
        w.job = tile_index[k];
        w.p = J.p;
        w.n = J.n;
        w.op = J.op;
        w.i = J.i;
        w.j = J.j;
        w.use_tmap = J.use_tmap;
        w.dd_solve = J.dd_solve;
        for (uint64_t t = 0; t < tiles[k]; t += per[k]) {
            w.tile0 = static_cast<uint32_t>(t);
            w.ntiles = static_cast<uint32_t>(std::min<uint64_t>(per[k], tiles[k] - t));
            items.push_back(w);
        }
    }
    for (uint32_t k = 0; k < n_jobs; ++k)
        if (tiles[k] > 0xffffffffull) return RCG_EINVAL;
    if (items.size() > 0xffffffffull) return RCG_EINVAL;
    // column items: one self-contained record per p <= 7 job, grouped by
    // variant, numbering the variant's 32-column chunks
    std::vector<ColJob> col_items;
    uint32_t col_begin[kColVariants] = {}, col_count[kColVariants] = {}, col_chunks[kColVariants] = {};
    for (int v = 0; v < kColVariants; ++v) {
        col_begin[v] = static_cast<uint32_t>(col_items.size());
        uint64_t chunks = 0, cost = 0;
        for (uint32_t k = 0; k < n_jobs; ++k) {
            if (variant[k] != v) continue;
            const Job &J = table[k];
            ColJob cj;
            memset(&cj, 0, sizeof(cj));
            cj.base = J.base;
            cj.pairs = J.pairs;
            cj.aux = J.aux;
            cj.rs = J.row_stride;
            cj.ss = J.strip_stride;
            cj.st = J.stripe_stride;
            cj.ars = J.aux_row_stride;
            cj.ass = J.aux_stripe_stride;
            cj.chunk0 = chunks;
            cj.n_stripes = J.n_stripes;
            cj.vps = J.C / 16;
            cj.N = J.n;
            cj.i = J.i;
            cj.j = J.j;
            cj.op = J.op;
            cj.p = J.p;
            cj.cost0 = cost;
            const uint64_t n_chunks = (static_cast<uint64_t>(J.n_stripes) * (J.C / 16) + kColChunk - 1) / kColChunk;
            chunks += n_chunks;
            cost += n_chunks * (J.n + 2ull) * (J.p - 1u);
            cj.chunk_end = chunks;
            col_items.push_back(cj);
        }
        if (chunks > 0xffffffffull) return RCG_EINVAL;
        col_count[v] = static_cast<uint32_t>(col_items.size()) - col_begin[v];
        col_chunks[v] = static_cast<uint32_t>(chunks);
    }
    if (max_col_items && col_items.size() > max_col_items) return RCG_EINVAL;
    BatchHeader hdr;
    memset(&hdr, 0, sizeof(hdr));
    hdr.total_tiles = total;
    hdr.n_jobs = static_cast<uint32_t>(tile_jobs.size());  // the Job entries (tile-engine jobs)
    if (slot_bytes == 0) slot_bytes = 128;  // no tile-engine job
    hdr.slot_bytes = slot_bytes;  // the largest stage
    if (ctx->tune_ring == RCG_RING_FIXED) {
        // equal slots of the largest stage, as many as the ring holds (the
        // single-launch discipline: one wait per slot reuse)
        const uint32_t slot = (slot_bytes + 127) & ~127u;
        hdr.n_slots = std::min<uint32_t>(kMaxSlots, (shape_info(shape).ring_bytes & ~127u) / slot);
        hdr.ring_bytes = hdr.n_slots * slot;
        hdr.fixed_slots = 1;
    } else {
        hdr.n_slots = kMaxSlots;  // stages of any size, up to 32 in flight, share the byte ring
        hdr.ring_bytes = shape_info(shape).ring_bytes & ~127u;
        hdr.fixed_slots = 0;
    }
    hdr.dynamic = ctx->batch_schedule == RCG_SCHED_DYNAMIC ? 1u : 0u;
    hdr.shape = shape;
    hdr.n_items = static_cast<uint32_t>(items.size());
    hdr.items_offset = sizeof(BatchHeader) + static_cast<uint64_t>(tile_jobs.size()) * sizeof(Job);
    hdr.col_items_offset = hdr.items_offset + items.size() * sizeof(WorkItem);  // 128-byte aligned
    for (int v = 0; v < kColVariants; ++v) {
        hdr.col_begin[v] = col_begin[v];
        hdr.col_count[v] = col_count[v];
        hdr.col_chunks[v] = col_chunks[v];
    }
    out.resize(hdr.col_items_offset + col_items.size() * sizeof(ColJob));
    memcpy(out.data(), &hdr, sizeof(hdr));
    memcpy(out.data() + sizeof(hdr), tile_jobs.data(), tile_jobs.size() * sizeof(Job));
    memcpy(out.data() + hdr.items_offset, items.data(), items.size() * sizeof(WorkItem));
    memcpy(out.data() + hdr.col_items_offset, col_items.data(), col_items.size() * sizeof(ColJob));
    return RCG_OK;
}

rcg_status rcg_batch_prepare(rcg_ctx *ctx, const rcg_job *jobs, uint32_t n_jobs, rcg_batch **out) {
    if (!ctx || !out || (n_jobs && !jobs)) return RCG_EINVAL;
    *out = nullptr;
    rcg_batch *b = new (std::nothrow) rcg_batch();
    if (!b) return RCG_ENOMEM;
    b->n_jobs = n_jobs;
    if (n_jobs) {
        DeviceGuard guard(ctx->device);
        b->shape = batch_shape(ctx, jobs, n_jobs);
        rcg_status st = build_table(ctx, jobs, n_jobs, b->shape, 0, b->image);
        if (st) {
            delete b;
            return st;
        }
    }
    *out = b;
    return RCG_OK;
}

rcg_status rcg_batch_free(rcg_batch *b) {
    if (!b) return RCG_EINVAL;
    delete b;
    return RCG_OK;
}

// The host half of a batch launch: the slot of the next ticket made ready for
// `b` -- it waits for the slot's previous batch; a table in device memory also
// grows the slot, re-captures its graph for a new engine shape, copies the
// table into its pinned buffer and updates the graph's copy size and enabled
// kernels.  *in_params: the table travels in the kernels' parameter blocks.
static rcg_status launch_host(rcg_ctx *ctx, const rcg_batch *b, BatchSlot **slot, bool *in_params) {
    BatchSlot &s = ctx->slots[ctx->next_ticket % kBatchRing];
    *slot = &s;
    if (s.used && s.done) {
        rcg_status st = wait_event(s.done, ctx->timeout_ns);
        if (st == RCG_ETIMEOUT) return RCG_EBUSY;
        if (st) return st;
    }
    const size_t bytes = b->image.size();
    const auto &hdr = *reinterpret_cast<const BatchHeader *>(b->image.data());
    cudaError_t e = cudaSuccess;
    const char *where = "batch event";
    *in_params = ctx->batch_tables == RCG_TABLES_AUTO && bytes <= kParamTableLarge;
    if (*in_params) {
        // a small table travels in the kernels' parameter blocks: no table
        // copy, no graph, no counter reset before the kernels
        if (!s.done) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        const int mask = work_mask(hdr);
        if (e == cudaSuccess && (mask & 15) && (mask & 16) && !ctx->side) {
            where = "side stream";
            e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->join, cudaEventDisableTiming);
        }
        return e == cudaSuccess ? RCG_OK : from_cuda(e, where);
    }
    rcg_status st = prepare_slot(ctx, s, bytes, b->shape);
    if (st) return st;
    memcpy(s.host, b->image.data(), bytes);
    where = "graph copy-size update";
    if (bytes != s.bytes) {
        // copy only the live part of the table: update the captured node
        cudaMemcpy3DParms mp;
        e = cudaGraphMemcpyNodeGetParams(s.copy_node, &mp);
        if (e == cudaSuccess) {
            mp.extent.width = bytes;
            mp.srcPtr.pitch = bytes;
            mp.srcPtr.xsize = bytes;
            mp.dstPtr.pitch = bytes;
            mp.dstPtr.xsize = bytes;
            e = cudaGraphExecMemcpyNodeSetParams(s.exec, s.copy_node, &mp);
        }
        if (e == cudaSuccess) {
            s.bytes = bytes;
        } else {
            // keep copying the whole table (the kernel reads n_jobs entries)
            cudaGetLastError();
            e = cudaSuccess;
        }
    }
    if (e == cudaSuccess) {
        e = set_enabled(s, work_mask(hdr));
        where = "graph node enable";
    }
    return e == cudaSuccess ? RCG_OK : from_cuda(e, where);
}

// The GPU half: the batch's kernels (or its graph) on `stream`, the slot's
// event after them, and the ticket handed out.
static rcg_status launch_enqueue(rcg_ctx *ctx, const rcg_batch *b, BatchSlot &s, bool in_params,
                                 cudaStream_t stream, uint64_t *ticket) {
    cudaError_t e;
    const char *where;
    if (in_params) {
        e = launch_batch_all_param(b->image.data(), b->image.size(), ctx->status, ctx->timeout_ns, b->shape,
                                   ctx->sm_count, stream, ctx->side, ctx->fork, ctx->join);
        where = "batch launch";
    } else {
        e = cudaGraphLaunch(s.exec, stream);
        where = "graph launch";
    }
    if (e == cudaSuccess) {
        e = cudaEventRecord(s.done, stream);
        where = "event record";
    }
    if (e != cudaSuccess) return from_cuda(e, where);
    const uint64_t tk = ctx->next_ticket;
    s.used = true;
    s.ticket = tk;
    ctx->next_ticket = tk + 1;
    *ticket = tk;
    return RCG_OK;
}

rcg_status rcg_batch_launch(rcg_ctx *ctx, const rcg_batch *b, void *stream, uint64_t *ticket) {
    if (!ctx || !b || !ticket) return RCG_EINVAL;
    *ticket = 0;
    if (b->n_jobs == 0) return RCG_OK;
    DeviceGuard guard(ctx->device);
    BatchSlot *s = nullptr;
    bool in_params = false;
    rcg_status st = launch_host(ctx, b, &s, &in_params);
    if (st) return st;
    return launch_enqueue(ctx, b, *s, in_params, static_cast<cudaStream_t>(stream), ticket);
}

rcg_status rcg_batch_submit(rcg_ctx *ctx, const rcg_job *jobs, uint32_t n_jobs, void *stream,
                            uint64_t *ticket) {
    if (!ctx || !ticket || (n_jobs && !jobs)) return RCG_EINVAL;
    *ticket = 0;
    if (n_jobs == 0) return RCG_OK;
    rcg_batch *b = nullptr;
    rcg_status st = rcg_batch_prepare(ctx, jobs, n_jobs, &b);
    if (st) return st;
    st = rcg_batch_launch(ctx, b, stream, ticket);
    rcg_batch_free(b);
    return st;
}

rcg_status rcg_set_batch_tuning(rcg_ctx *ctx, const rcg_batch_tuning *t) {
    if (!ctx) return RCG_EINVAL;
    if (!t) {
        ctx->tune_shape = RCG_SHAPE_AUTO;
        ctx->batch_schedule = RCG_SCHED_DYNAMIC;
        ctx->tune_item_bytes = 0;
        ctx->tune_tile_div = 1;
        ctx->tune_ring = RCG_RING_FIXED;
        return RCG_OK;
    }
    if ((t->shape != RCG_SHAPE_AUTO && t->shape != RCG_SHAPE_WIDE && t->shape != RCG_SHAPE_PAIR) ||
        (t->schedule != RCG_SCHED_STATIC && t->schedule != RCG_SCHED_DYNAMIC) ||
        (t->item_bytes != 0 && t->item_bytes < (64u << 10)) || t->tile_div < 1 || t->tile_div > 8 ||
        (t->ring != RCG_RING_FIXED && t->ring != RCG_RING_BYTES))
        return RCG_EINVAL;
    ctx->tune_shape = static_cast<int>(t->shape);
    ctx->batch_schedule = static_cast<int>(t->schedule);
    ctx->tune_item_bytes = t->item_bytes;
    ctx->tune_tile_div = t->tile_div;
    ctx->tune_ring = static_cast<int>(t->ring);
    return RCG_OK;
}

// Time one configuration: prepare under the context's current tuning, then
// one untimed and `reps` timed launches (CUDA events on `stream`); the best.
static rcg_status time_batch(rcg_ctx *ctx, const rcg_job *jobs, uint32_t n_jobs, cudaStream_t stream, int reps,
                             cudaEvent_t e0, cudaEvent_t e1, float *best_ms) {
    rcg_batch *b = nullptr;
    rcg_status st = rcg_batch_prepare(ctx, jobs, n_jobs, &b);
    if (st) return st;
    float best = -1.0f;
    for (int r = 0; r <= reps && st == RCG_OK; ++r) {
        // the host half (a slot growing or re-capturing its graph) stays
        // outside the timed region: the events time the GPU's work only
        uint64_t ticket = 0;
        BatchSlot *slot = nullptr;
        bool in_params = false;
        st = b->n_jobs ? launch_host(ctx, b, &slot, &in_params) : RCG_EINVAL;
        if (st) break;
        cudaError_t e = cudaEventRecord(e0, stream);
        if (e == cudaSuccess) st = launch_enqueue(ctx, b, *slot, in_params, stream, &ticket);
        if (st == RCG_OK && e == cudaSuccess) e = cudaEventRecord(e1, stream);
        if (st == RCG_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (st == RCG_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) st = from_cuda(e, "autotune timing");
        if (st == RCG_OK && r > 0 && (best < 0.0f || ms < best)) best = ms;
    }
    rcg_batch_free(b);
    *best_ms = best;
    return st;
}

rcg_status rcg_batch_autotune(rcg_ctx *ctx, const rcg_job *jobs, uint32_t n_jobs, void *stream,
                              rcg_batch_tuning *out) {
    if (!ctx || !jobs || n_jobs == 0 || !out) return RCG_EINVAL;
    for (uint32_t k = 0; k < n_jobs; ++k) {  // timing relaunches the batch: only idempotent ops
        Geo g;
        if (check_layout(&jobs[k].layout, &g) != RCG_OK) return RCG_EINVAL;
    }
    DeviceGuard guard(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return RCG_ECUDA;
    }
    rcg_batch_tuning cur;
    cur.shape = static_cast<uint32_t>(ctx->tune_shape);
    cur.schedule = static_cast<uint32_t>(ctx->batch_schedule);
    cur.item_bytes = ctx->tune_item_bytes;
    cur.tile_div = ctx->tune_tile_div;
    cur.ring = static_cast<uint32_t>(ctx->tune_ring);
    cur.ms = 0.0f;
    rcg_status st = rcg_set_batch_tuning(ctx, &cur);
    float best_ms = -1.0f;
    if (st == RCG_OK) st = time_batch(ctx, jobs, n_jobs, s, 2, e0, e1, &best_ms);
    // coordinate descent: one knob at a time, keeping the best value of each
    const uint32_t shapes[] = {RCG_SHAPE_WIDE, RCG_SHAPE_PAIR};
    const uint32_t schedules[] = {RCG_SCHED_DYNAMIC, RCG_SCHED_STATIC};
    const uint64_t items[] = {0, 256ull << 10, 1ull << 20, 4ull << 20};
    const uint32_t divs[] = {1, 2, 4};
    const uint32_t rings[] = {RCG_RING_FIXED, RCG_RING_BYTES};
    for (int knob = 0; knob < 5 && st == RCG_OK; ++knob) {
        const int n_vals = knob == 0 ? 2 : knob == 1 ? 2 : knob == 2 ? 4 : knob == 3 ? 3 : 2;
        for (int v = 0; v < n_vals && st == RCG_OK; ++v) {
            rcg_batch_tuning cand = cur;
            if (knob == 0) cand.shape = shapes[v];
            if (knob == 1) cand.schedule = schedules[v];
            if (knob == 2) cand.item_bytes = items[v];
            if (knob == 3) cand.tile_div = divs[v];
            if (knob == 4) cand.ring = rings[v];
            if (memcmp(&cand, &cur, sizeof(cand)) == 0) continue;
            st = rcg_set_batch_tuning(ctx, &cand);
            float ms = -1.0f;
            if (st == RCG_OK) st = time_batch(ctx, jobs, n_jobs, s, 2, e0, e1, &ms);
            if (st == RCG_EINVAL) {  // a plan that does not fit this shape: skip it
                st = RCG_OK;
                continue;
            }
            if (st == RCG_OK && ms >= 0.0f && (best_ms < 0.0f || ms < best_ms)) {
                best_ms = ms;
                cur = cand;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cur.ms = best_ms;
    const rcg_status st2 = rcg_set_batch_tuning(ctx, &cur);  // apply the best
    if (st) return st;
    *out = cur;
    return st2;
}

rcg_status rcg_batch_wait(rcg_ctx *ctx, uint64_t ticket, uint64_t timeout_ns) {
    if (!ctx || ticket == 0 || ticket >= ctx->next_ticket) return RCG_EINVAL;
    DeviceGuard guard(ctx->device);
    BatchSlot &s = ctx->slots[ticket % kBatchRing];
    if (!s.used || s.ticket != ticket) return RCG_OK;  // slot reused: that batch finished
    return wait_event(s.done, timeout_ns);
}

// ===================================================== host-memory stripes

static rcg_status run_encode(void *c, const rcg_layout *L, uint64_t n, const uint8_t *, cudaStream_t s) {
    return rcg_encode(static_cast<rcg_ctx *>(c), L, 0, n, s);
}

static rcg_status run_recover(void *c, const rcg_layout *L, uint64_t n, const uint8_t *pairs,
                              cudaStream_t s) {
    return rcg_recover_many(static_cast<rcg_ctx *>(c), L, 0, n, pairs, s);
}

rcg_status rcg_encode_host(rcg_ctx *ctx, const rcg_layout *L, uint64_t first_stripe, uint64_t n_stripes,
                           void *stream) {
    if (!ctx) return RCG_EINVAL;
    DeviceGuard guard(ctx->device);
    if (!ctx->host) ctx->host = host_staging_create();
    return host_path(ctx->host, L, first_stripe, n_stripes, nullptr, static_cast<cudaStream_t>(stream),
                     ctx->host_chunk_bytes, run_encode, ctx);
}

rcg_status rcg_recover_many_host(rcg_ctx *ctx, const rcg_layout *L, uint64_t first_stripe,
                                 uint64_t n_stripes, const uint8_t *pairs, void *stream) {
    if (!ctx || !pairs) return RCG_EINVAL;
    DeviceGuard guard(ctx->device);
    if (!ctx->host) ctx->host = host_staging_create();
    return host_path(ctx->host, L, first_stripe, n_stripes, pairs, static_cast<cudaStream_t>(stream),
                     ctx->host_chunk_bytes, run_recover, ctx);
}

// =============================================================== utilities

rcg_status rcg_selftest_wait_timeout(rcg_ctx *ctx, uint64_t timeout_ns, void *stream) {
    if (!ctx || timeout_ns == 0 || timeout_ns > 10000000000ull) return RCG_EINVAL;
    DeviceGuard guard(ctx->device);
    return from_cuda(launch_wait_probe(ctx->status, timeout_ns, static_cast<cudaStream_t>(stream)),
                     "wait probe");
}

rcg_status rcg_fill_random(void *dev, uint64_t nbytes, uint64_t seed, uint64_t byte_offset,
                           void *stream) {
    if ((!dev && nbytes) || !aligned16(dev) || (byte_offset & 7))
        return RCG_EINVAL;
    return from_cuda(launch_fill(dev, nbytes, seed, byte_offset, static_cast<cudaStream_t>(stream)));
}

}  // extern "C"

// Descriptor table for rcg_batch_submit_noalloc (default copy mode, solve,
// shape and column kernel; no context), written into `table` of `capacity`
// bytes, of which col_capacity bytes are kept for column items.  Returns the
// engine shape through *shape.
bool rcg::noalloc_build_table(const rcg_job *jobs, uint32_t n_jobs, uint8_t *table, size_t capacity,
                              size_t col_capacity, size_t *bytes, uint32_t *shape) {
    static const rcg_ctx defaults;
    *shape = batch_shape(&defaults, jobs, n_jobs);
    const uint64_t max_items =
        (capacity - col_capacity - sizeof(BatchHeader) - n_jobs * sizeof(Job)) / sizeof(WorkItem) - n_jobs;
    std::vector<uint8_t> image;
    if (build_table(&defaults, jobs, n_jobs, *shape, max_items, image, col_capacity / sizeof(ColJob)) != RCG_OK ||
        image.size() > capacity)
        return false;
    memcpy(table, image.data(), image.size());
    *bytes = image.size();
    return true;
}

cudaError_t rcg::launch_batch_all(const uint8_t *table_dev, const uint8_t *table_host, uint32_t *status,
                                  unsigned long long *counter, uint64_t timeout_ns, uint32_t shape, int sm_count,
                                  cudaStream_t stream) {
    const auto &h = *reinterpret_cast<const BatchHeader *>(table_host);
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < kColVariants && e == cudaSuccess; ++v)
        if (h.col_count[v]) e = launch_column_batch(v, table_dev, status, sm_count, stream);
    if (e == cudaSuccess && h.n_items)
        e = launch_batch(table_dev, status, counter, timeout_ns, shape,
                         sm_count * static_cast<int>(shape_info(shape).ctas_per_sm), stream);
    return e;
}

cudaError_t rcg::launch_batch_all_param(const uint8_t *table_host, size_t bytes, uint32_t *status,
                                        uint64_t timeout_ns, uint32_t shape, int sm_count, cudaStream_t stream,
                                        cudaStream_t side, cudaEvent_t fork, cudaEvent_t join) {
    if (bytes < sizeof(BatchHeader) || bytes > kParamTableLarge) return cudaErrorInvalidValue;
    const auto &h = *reinterpret_cast<const BatchHeader *>(table_host);
    bool cols = false;
    for (int v = 0; v < kColVariants; ++v) cols = cols || h.col_count[v] != 0;
    const bool beside = cols && h.n_items && side && fork && join;
    cudaStream_t cs = beside ? side : stream;
    cudaError_t e = cudaSuccess;
    if (beside) {
        e = cudaEventRecord(fork, stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, fork, 0);
    }
    for (int v = 0; v < kColVariants && e == cudaSuccess; ++v)
        if (h.col_count[v]) e = launch_column_batch_param(v, table_host, bytes, status, sm_count, cs);
    if (e == cudaSuccess && h.n_items)
        e = launch_batch_param(table_host, bytes, status, timeout_ns, shape,
                               sm_count * static_cast<int>(shape_info(shape).ctas_per_sm), stream);
    if (e == cudaSuccess && beside) {
        e = cudaEventRecord(join, side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, join, 0);
    }
    return e;
}

int rcg::ctx_device(const rcg_ctx *ctx) { return ctx ? ctx->device : 0; }
