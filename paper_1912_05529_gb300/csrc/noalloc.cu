// noalloc.cu -- fxmig_migrate_noalloc: the persistent depth loop for callers
// that cannot allocate device memory themselves.
//
// Some callers can hand the library only their own input and output buffers:
// code that runs inside a host application whose memory arena owns the whole
// device, plug-ins that are given buffers but no allocator, and real-time
// paths that must not call cudaMalloc because it can synchronise the device.
// They cannot provide the scratch workspace fxmig_migrate needs (the status
// word, the expanded operator table, the slowness field and the wavefield
// norms of the image scale).  This entry point keeps that scratch in a fixed
// file-scope device array instead: every GPU that loads the library holds it
// until the process exits.
#include <mutex>

#include "fxmig_internal.cuh"

namespace fxmig_impl {

// Fixed scratch: the persistent form's workspace without its second
// wavefield (migrate_ws_bytes_persistent): status head, expanded table,
// slowness field [nz][nx rounded up to 8], frequency norms.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the symbol name is only a host-side handle).  The address is
// cached for the life of the process: after cudaDeviceReset on a device the
// cached address is stale, so callers that reset devices must not use this
// entry point afterwards.
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}
}  // namespace

}  // namespace fxmig_impl

using namespace fxmig_impl;

extern "C" int fxmig_migrate_noalloc(const fxmig_desc* d, void* slab, const float* vel, const void* table,
                                     float* partials, int nparts, int z_begin, int z_end, void* stream) {
    if (!desc_valid(d) || !slab || !vel || !table || !partials) return FXMIG_EINVAL;
    const uintptr_t s8 = reinterpret_cast<uintptr_t>(slab), v4 = reinterpret_cast<uintptr_t>(vel);
    const uintptr_t t8 = reinterpret_cast<uintptr_t>(table), p16 = reinterpret_cast<uintptr_t>(partials);
    if ((s8 & 7) || (v4 & 3) || (t8 & 7) || (p16 & 15)) return FXMIG_EINVAL;
    if (z_begin < 0 || z_end < z_begin || z_end > d->nz) return FXMIG_EINVAL;
    fxmig_launch launch = {};
    launch.mode = FXMIG_MODE_PERSISTENT;
    MigratePlan plan;
    const int rc = plan_migrate(d, &launch, &plan);
    if (rc != FXMIG_OK) return rc;
    if (nparts < plan.nparts) return FXMIG_ENOSPC;
    // the persistent form's scratch must fit the fixed array
    if (migrate_ws_bytes_persistent(d) > kNoAllocScratchBytes) return FXMIG_ENOSPC;
    void* ws = nullptr;
    cudaError_t e = scratch_address(&ws);
    if (e != cudaSuccess) return record_cuda_error(e, "fxmig_migrate_noalloc");
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (z_begin == z_end) return FXMIG_OK;
    // launch_migrate clears the status head and rewrites the table, slowness
    // and norms regions on every call, so stale contents from an earlier call
    // are never read.
    e = launch_migrate(d, plan, slab, vel, table, partials, z_begin, z_end, ws, s, true);
    return e == cudaSuccess ? FXMIG_OK : record_cuda_error(e, "fxmig_migrate_noalloc");
}
