// rcg_noalloc.cu -- rcg_batch_submit_noalloc: the batched engine for callers
// that cannot allocate device memory.
//
// Who needs it.  Some callers may not call cudaMalloc or cudaFree at all:
// a framework whose caching allocator already owns all of the device's memory
// (a cudaMalloc behind its back can fail or fragment its pool), and latency-
// critical submit paths where the implicit device synchronisation of
// cudaMalloc/cudaFree is not allowed.  rcg_batch_submit needs a context, and
// creating one allocates its status word and descriptor tables.  This entry
// point needs no context and allocates nothing: its scratch -- the batch
// descriptor table, the tile counter and a fallback status word -- lives in
// one file-scope device array of fixed size that every GPU loading the
// library holds until the process exits.
//
// The array's name is a host-side stand-in in host code, never a device
// address, so the set-up below asks the runtime for the real address once per
// device (with that device current) and passes that pointer to the kernel.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/rcg.h"
#include "rcg_internal.h"

namespace {

using namespace rcg;

// header, up to RCG_NOALLOC_MAX_JOBS jobs, 2 x RCG_NOALLOC_MAX_JOBS work items
// of the tile engine and one 128-byte column-kernel record per job (~165 KB)
constexpr uint32_t kColTableBytes = RCG_NOALLOC_MAX_JOBS * sizeof(ColJob);
constexpr uint32_t kTableBytes = sizeof(BatchHeader) + RCG_NOALLOC_MAX_JOBS * sizeof(Job) +
                                 2 * RCG_NOALLOC_MAX_JOBS * sizeof(WorkItem) + kColTableBytes;
constexpr uint32_t kCounterOff = (kTableBytes + 255) / 256 * 256;
constexpr uint32_t kStatusOff = kCounterOff + 256;
constexpr uint32_t kScratchBytes = kStatusOff + 256;

// The scratch: [descriptor table | tile counter | fallback status word].
static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

struct DeviceState {
    bool ready = false;
    uint8_t *scratch = nullptr;  // device address of g_noalloc_scratch
    int sm_count = 0;
};

constexpr int kMaxDevices = 64;
DeviceState g_dev[kMaxDevices];
std::mutex g_setup_lock;

// Host image of the descriptor table, reused by every call.
alignas(128) uint8_t g_host_table[kTableBytes];

// Once per device, with that device current: the scratch address, the
// per-p inverse tables of the tile engine and the column kernel in constant
// memory and the engine's shared-memory attribute.  None of these allocates.
rcg_status setup_device(int dev, DeviceState **out) {
    if (dev < 0 || dev >= kMaxDevices) return RCG_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_lock);
    DeviceState &d = g_dev[dev];
    if (!d.ready) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return RCG_ECUDA;
        if (!(prop.major == 10 && prop.minor == 3)) return RCG_EUNSUPPORTED;
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return RCG_ECUDA;
        if (upload_inverse_tables() != cudaSuccess) return RCG_ECUDA;
        if (upload_column_tables() != cudaSuccess) return RCG_ECUDA;
        if (engine_init_attributes() != cudaSuccess) return RCG_ECUDA;
        d.scratch = static_cast<uint8_t *>(ptr);
        d.sm_count = prop.multiProcessorCount;
        d.ready = true;
    }
    *out = &d;
    return RCG_OK;
}

}  // namespace

extern "C" rcg_status rcg_batch_submit_noalloc(const rcg_job *jobs, uint32_t n_jobs,
                                               uint32_t *status_dev, void *stream) {
    if (n_jobs > RCG_NOALLOC_MAX_JOBS) return RCG_EINVAL;  // beyond the scratch table
    if (n_jobs && !jobs) return RCG_EINVAL;
    if (n_jobs == 0) return RCG_OK;

    uint32_t shape = SHAPE_WIDE;
    size_t bytes = 0;
    if (!noalloc_build_table(jobs, n_jobs, g_host_table, kTableBytes, kColTableBytes, &bytes, &shape))
        return RCG_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RCG_ECUDA;
    DeviceState *d = nullptr;
    rcg_status st = setup_device(dev, &d);
    if (st) return st;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *table_dev = d->scratch;
    auto *counter = reinterpret_cast<unsigned long long *>(d->scratch + kCounterOff);
    uint32_t *status = status_dev ? status_dev : reinterpret_cast<uint32_t *>(d->scratch + kStatusOff);
    cudaError_t e = cudaSuccess;
    if (bytes <= kParamTableLarge) {
        // a small table travels in the kernels' parameter blocks: no copy into
        // the scratch, no counter
        e = launch_batch_all_param(g_host_table, bytes, status, 2000000000ull, shape, d->sm_count, s, nullptr,
                                   nullptr, nullptr);
    } else {
        // The host table is pageable: the copy has left it by the time the call returns.
        e = cudaMemcpyAsync(table_dev, g_host_table, bytes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
        if (e == cudaSuccess)
            e = launch_batch_all(table_dev, g_host_table, status, counter, 2000000000ull, shape, d->sm_count, s);
    }
    return e == cudaSuccess ? RCG_OK : RCG_ECUDA;
}
