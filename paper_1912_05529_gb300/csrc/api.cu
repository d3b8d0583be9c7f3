// api.cu -- the C ABI of libfxmig (include/fxmig.h): argument checks on the
// host, then asynchronous launches on the caller's stream.  No allocation, no
// synchronisation (fxmig_check excepted), no exception crosses the boundary.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <utility>

#include "fxmig_internal.cuh"
#include "mlp_internal.cuh"

using namespace fxmig_impl;

namespace fxmig_impl {

cudaError_t kernel_smem_attr(const void* func, size_t bytes, bool nonportable_cluster) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, std::pair<size_t, bool>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    auto& st = done[{dev, func}];
    if (bytes > st.first) {
        e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        st.first = bytes;
    }
    if (nonportable_cluster && !st.second) {
        e = cudaFuncSetAttribute(func, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        st.second = true;
    }
    return cudaSuccess;
}

bool desc_valid(const fxmig_desc* d) {
    if (!d) return false;
    if (d->nx < 1 || d->nz < 1 || d->nt < 2 || d->nw < 1 || d->L < 0 || d->nk < 1) return false;
    if (d->i0 < 1 || (long long)d->i0 + d->nw > (long long)((d->nt - 1) / 2) + 1) return false;
    if (!(d->dx > 0) || !(d->dz >= 0) || !(d->dt > 0) || !isfinite(d->dx) || !isfinite(d->dz) || !isfinite(d->dt))
        return false;
    if (!(d->theta_max_deg >= 0 && d->theta_max_deg <= 90)) return false;
    if (!(d->k_max >= 0) || !isfinite(d->k_max)) return false;
    if (d->nk > 1 && !(d->k_max > 0)) return false;
    if (compiled_half_length(d->L) < 0) return false;
    // sizes that must fit 32-bit indexing of one line / one image plane
    if ((long long)d->nx * d->nz > (1LL << 31) || (long long)d->nx * d->nw > (1LL << 31)) return false;
    return true;
}

}  // namespace fxmig_impl

static thread_local char g_last_error[256] = "";

static int cuda_fail(cudaError_t e, const char* where) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
    return FXMIG_ECUDA;
}

namespace fxmig_impl {
int record_cuda_error(cudaError_t e, const char* where) { return cuda_fail(e, where); }
}  // namespace fxmig_impl

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

extern "C" {

int fxmig_version(void) { return FXMIG_VERSION; }

const char* fxmig_strerror(int code) {
    switch (code) {
        case FXMIG_OK: return "ok";
        case FXMIG_EINVAL: return "invalid argument";
        case FXMIG_ENOSPC: return "workspace or partial-image buffer too small";
        case FXMIG_ECUDA: return "CUDA error";
        case FXMIG_ETIMEOUT: return "a bounded wait on the device gave up";
        case FXMIG_EVELOCITY: return "velocity sample not finite and positive";
        case FXMIG_ERANGE: return "image contribution beyond the accumulator's range";
        default: return "unknown error";
    }
}

const char* fxmig_last_error(void) { return g_last_error; }

size_t fxmig_workspace_bytes(const fxmig_desc* d, int kind) {
    if (!desc_valid(d)) return 0;
    if (kind == FXMIG_WS_T2F) return t2f_ws_bytes(d);
    if (kind == FXMIG_WS_MIGRATE) return migrate_ws_bytes(d);
    if (kind == FXMIG_WS_MLP_MIGRATE) return mlp_migrate_ws_bytes(d);
    return 0;
}

int fxmig_num_partials(const fxmig_desc* d, const fxmig_launch* launch) {
    if (!desc_valid(d)) return FXMIG_EINVAL;
    MigratePlan p;
    const int rc = plan_migrate(d, launch, &p);
    return rc == FXMIG_OK ? p.nparts : rc;
}

int fxmig_launch_shape(const fxmig_desc* d, const fxmig_launch* launch, fxmig_shape* out) {
    if (!desc_valid(d) || !out) return FXMIG_EINVAL;
    MigratePlan p;
    const int rc = plan_migrate(d, launch, &p);
    if (rc != FXMIG_OK) return rc;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        sms = 148;
    }
    out->mode = p.mode;
    out->cluster = p.cluster;
    out->groups = p.groups;
    if (p.mode == FXMIG_MODE_PER_DEPTH) {
        out->ctas = p.groups * ((d->nx + 255) / 256);
        out->warps = p.warps;
        out->items_per_lane = 1;
        out->waves = 1;
        out->ctas_per_sm = 0;
    } else {
        out->ctas = p.groups * p.cluster;
        out->warps = p.warps;
        out->items_per_lane = p.nr;
        const int resident = p.occ * (p.cluster == 1 ? sms : 2 * (sms / 2));
        out->waves = (out->ctas + resident - 1) / resident;
        out->ctas_per_sm = p.occ;
    }
    out->smem_bytes = p.smem;
    return FXMIG_OK;
}

int fxmig_design_operators(const fxmig_desc* d, void* table, void* table64, void* stream) {
    if (!desc_valid(d) || !table || !aligned(table, 8) || (table64 && !aligned(table64, 16))) return FXMIG_EINVAL;
    const cudaError_t e = launch_design(d, nullptr, d->nk, table, table64, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FXMIG_OK : cuda_fail(e, "fxmig_design_operators");
}

int fxmig_t2f(const fxmig_desc* d, const float* section, void* slab, void* ws, size_t ws_bytes, void* stream) {
    if (!desc_valid(d) || !section || !slab || !ws) return FXMIG_EINVAL;
    if (!aligned(section, 4) || !aligned(slab, 8) || !aligned(ws, 256)) return FXMIG_EINVAL;
    if (!t2f_supported(d->nt)) return FXMIG_EINVAL;
    if (ws_bytes < t2f_ws_bytes(d)) return FXMIG_ENOSPC;
    const cudaError_t e = launch_t2f(d, section, slab, ws, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FXMIG_OK : cuda_fail(e, "fxmig_t2f");
}

int fxmig_migrate_ex(const fxmig_desc* d, const fxmig_launch* launch, void* slab, const float* vel,
                     const void* table, float* partials, int nparts, int z_begin, int z_end, void* ws,
                     size_t ws_bytes, void* stream) {
    if (!desc_valid(d) || !slab || !vel || !table || !partials || !ws) return FXMIG_EINVAL;
    if (!aligned(slab, 8) || !aligned(vel, 4) || !aligned(table, 8) || !aligned(partials, 16) || !aligned(ws, 256))
        return FXMIG_EINVAL;
    if (z_begin < 0 || z_end < z_begin || z_end > d->nz) return FXMIG_EINVAL;
    MigratePlan plan;
    const int rc = plan_migrate(d, launch, &plan);
    if (rc != FXMIG_OK) return rc;
    if (nparts < plan.nparts || ws_bytes < migrate_ws_bytes(d)) return FXMIG_ENOSPC;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (z_begin == z_end) {
        const cudaError_t e = cudaMemsetAsync(ws, 0, 16, s);
        return e == cudaSuccess ? FXMIG_OK : cuda_fail(e, "fxmig_migrate");
    }
    const cudaError_t e = launch_migrate(d, plan, slab, vel, table, partials, z_begin, z_end, ws, s, true);
    return e == cudaSuccess ? FXMIG_OK : cuda_fail(e, "fxmig_migrate");
}

int fxmig_migrate(const fxmig_desc* d, void* slab, const float* vel, const void* table, float* partials,
                  int nparts, int z_begin, int z_end, void* ws, size_t ws_bytes, void* stream) {
    return fxmig_migrate_ex(d, nullptr, slab, vel, table, partials, nparts, z_begin, z_end, ws, ws_bytes, stream);
}

int fxmig_image(const fxmig_desc* d, const float* partials, int nparts, float* image, void* stream) {
    if (!desc_valid(d) || !partials || !image) return FXMIG_EINVAL;
    if (!aligned(partials, 16) || !aligned(image, 4)) return FXMIG_EINVAL;
    if (nparts < image_planes(d->nx)) return FXMIG_ENOSPC;
    const cudaError_t e = launch_image(d, partials, nparts, image, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FXMIG_OK : cuda_fail(e, "fxmig_image");
}

int fxmig_mlp_param_count(int L) {
    if (L < 0 || L > kMlpMaxL) return FXMIG_EINVAL;
    return mlp_param_count(L);
}

size_t fxmig_mlp_train_ws_bytes(int L, int n) {
    if (L < 0 || L > kMlpMaxL || n < 1) return 0;
    return mlp_train_ws_bytes(L, n);
}

int fxmig_design_at(const fxmig_desc* d, const double* k, int n, void* taps, void* taps64, void* stream) {
    if (!desc_valid(d) || n < 0 || (n > 0 && (!k || !taps))) return FXMIG_EINVAL;
    if ((k && !aligned(k, 8)) || (taps && !aligned(taps, 8)) || (taps64 && !aligned(taps64, 16))) return FXMIG_EINVAL;
    const cudaError_t e = launch_design(d, k, n, taps, taps64, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FXMIG_OK : cuda_fail(e, "fxmig_design_at");
}

static int mlp_train_args_ok(const fxmig_desc* d, const double* k, const void* taps, int n, void* ws) {
    if (!desc_valid(d) || d->L > kMlpMaxL || !(d->k_max > 0) || n < 1 || !k || !taps || !ws) return FXMIG_EINVAL;
    if (!aligned(k, 8) || !aligned(taps, 8) || !aligned(ws, 256)) return FXMIG_EINVAL;
    return FXMIG_OK;
}

int fxmig_mlp_train(const fxmig_desc* d, float* params, float* adam_m, float* adam_v, int step0, int nsteps,
                    float lr_max, float lr_min, int schedule_steps, const double* k, const void* taps, int n,
                    float* loss, void* ws, size_t ws_bytes, void* stream) {
    int rc = mlp_train_args_ok(d, k, taps, n, ws);
    if (rc != FXMIG_OK) return rc;
    if (!params || !adam_m || !adam_v || step0 < 0 || nsteps < 0 || !(lr_max >= 0) || !(lr_min >= 0))
        return FXMIG_EINVAL;
    if (!aligned(params, 4) || !aligned(adam_m, 4) || !aligned(adam_v, 4) || (loss && !aligned(loss, 4)))
        return FXMIG_EINVAL;
    if (ws_bytes < mlp_train_ws_bytes(d->L, n)) return FXMIG_ENOSPC;
    const cudaError_t e = launch_mlp_train(d->L, params, adam_m, adam_v, step0, nsteps, lr_max, lr_min,
                                           schedule_steps, k, d->k_max, static_cast<const float*>(taps), n, loss,
                                           nullptr, ws, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FXMIG_OK : cuda_fail(e, "fxmig_mlp_train");
}

int fxmig_mlp_grad(const fxmig_desc* d, const float* params, const double* k, const void* taps, int n,
                   float* grad, float* loss, void* ws, size_t ws_bytes, void* stream) {
    int rc = mlp_train_args_ok(d, k, taps, n, ws);
    if (rc != FXMIG_OK) return rc;
    if (!params || !grad || !aligned(params, 4) || !aligned(grad, 4) || (loss && !aligned(loss, 4)))
        return FXMIG_EINVAL;
    if (ws_bytes < mlp_train_ws_bytes(d->L, n)) return FXMIG_ENOSPC;
    // the gradient-only step reads the parameters and writes grad, never params
    const cudaError_t e = launch_mlp_train(d->L, const_cast<float*>(params), nullptr, nullptr, 0, 1, 0.f, 0.f, 0, k,
                                           d->k_max, static_cast<const float*>(taps), n, loss, grad, ws,
                                           static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FXMIG_OK : cuda_fail(e, "fxmig_mlp_grad");
}

int fxmig_mlp_taps(const fxmig_desc* d, const float* params, const double* k, int n, void* taps, void* stream) {
    if (!desc_valid(d) || d->L > kMlpMaxL || !(d->k_max > 0) || !params || n < 0) return FXMIG_EINVAL;
    if (n > 0 && (!k || !taps || !aligned(k, 8) || !aligned(taps, 8))) return FXMIG_EINVAL;
    const cudaError_t e = launch_mlp_taps(d->L, params, k, d->k_max, n, taps, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FXMIG_OK : cuda_fail(e, "fxmig_mlp_taps");
}

int fxmig_mlp_num_partials(const fxmig_desc* d) {
    if (!desc_valid(d)) return FXMIG_EINVAL;
    MlpMigratePlan p;
    const int rc = plan_mlp_migrate(d, &p);
    return rc == FXMIG_OK ? p.nparts : rc;
}

int fxmig_mlp_migrate(const fxmig_desc* d, void* slab, const float* vel, const float* params, float* partials,
                      int nparts, int z_begin, int z_end, void* ws, size_t ws_bytes, void* stream) {
    if (!desc_valid(d) || !slab || !vel || !params || !partials || !ws) return FXMIG_EINVAL;
    if (!aligned(slab, 8) || !aligned(vel, 4) || !aligned(params, 4) || !aligned(partials, 16) || !aligned(ws, 256))
        return FXMIG_EINVAL;
    if (z_begin < 0 || z_end < z_begin || z_end > d->nz) return FXMIG_EINVAL;
    MlpMigratePlan plan;
    const int rc = plan_mlp_migrate(d, &plan);
    if (rc != FXMIG_OK) return rc;
    if (nparts < plan.nparts || ws_bytes < mlp_migrate_ws_bytes(d)) return FXMIG_ENOSPC;
    const cudaError_t e = launch_mlp_migrate(d, plan, slab, vel, params, partials, z_begin, z_end, ws,
                                             static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FXMIG_OK : cuda_fail(e, "fxmig_mlp_migrate");
}

size_t fxmig_batch_workspace_bytes(const fxmig_line* lines, int n, int autotune) {
    if (!batch_lines_valid(lines, n)) return 0;
    return batch_ws_bytes(lines, n, autotune != 0);
}

int fxmig_batch_num_partials(const fxmig_line* lines, int n, const fxmig_batch_plan* plan, int* nparts) {
    if (!batch_descs_valid(lines, n) || !nparts) return FXMIG_EINVAL;
    return batch_num_partials(lines, n, plan, nparts);
}

static bool batch_plan_ok(const fxmig_batch_plan* p) {
    return !p || ((p->cluster == 0 || p->cluster == 1 || p->cluster == 2 || p->cluster == 4 || p->cluster == 8) &&
                  p->lines_cap >= 0);
}

int fxmig_batch_autotune(const fxmig_line* lines, int n, fxmig_batch_plan* plan, float* best_ms, void* ws,
                         size_t ws_bytes, void* stream) {
    if (!batch_lines_valid(lines, n) || !plan || !ws || !aligned(ws, 256)) return FXMIG_EINVAL;
    if (ws_bytes < batch_ws_bytes(lines, n, true)) return FXMIG_ENOSPC;
    const int rc = batch_autotune(lines, n, plan, ws, static_cast<cudaStream_t>(stream), best_ms);
    if (rc == FXMIG_ECUDA) return cuda_fail(cudaGetLastError(), "fxmig_batch_autotune");
    return rc;
}

int fxmig_migrate_batch(const fxmig_line* lines, int n, const fxmig_batch_plan* plan, void* ws, size_t ws_bytes,
                        void* stream) {
    if (!batch_lines_valid(lines, n) || !batch_plan_ok(plan) || !ws || !aligned(ws, 256)) return FXMIG_EINVAL;
    if (ws_bytes < batch_ws_bytes(lines, n, false)) return FXMIG_ENOSPC;
    fxmig_batch_plan p = {2, 0};
    if (plan) {
        p = *plan;
        if (p.cluster == 0) p.cluster = 2;
    }
    {  // every line must be plannable (shared memory, cluster width)
        int np[FXMIG_BATCH_MAX_LINES];
        if (batch_num_partials(lines, n, &p, np) != FXMIG_OK) return FXMIG_EINVAL;
    }
    const cudaError_t e = launch_batch(lines, n, p, ws, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FXMIG_OK : cuda_fail(e, "fxmig_migrate_batch");
}

int fxmig_selftest_timeout(void* ws, int polls, void* stream) {
    if (!ws || !aligned(ws, 256) || polls < 1 || polls > (1 << 20)) return FXMIG_EINVAL;
    const cudaError_t e = launch_selftest_timeout(ws, polls, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FXMIG_OK : cuda_fail(e, "fxmig_selftest_timeout");
}

int fxmig_check(const void* ws, void* stream) {
    if (!ws) return FXMIG_EINVAL;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "fxmig_check");
    int status = 0;
    e = cudaMemcpy(&status, ws, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "fxmig_check");
    if (status & kStatusTimeout) return FXMIG_ETIMEOUT;
    if (status & kStatusVelocity) return FXMIG_EVELOCITY;
    if (status & kStatusOverflow) return FXMIG_ERANGE;
    return FXMIG_OK;
}

}  // extern "C"
