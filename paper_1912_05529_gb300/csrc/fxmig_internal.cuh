// fxmig_internal.cuh -- device helpers and internal host interfaces shared by
// the CUDA translation units of libfxmig (sm_103a only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fxmig.h"

#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ < 1000)
#error "libfxmig targets Blackwell (sm_103a)"
#endif

namespace fxmig_impl {

// ----------------------------------------------------------------- status word
// Bits OR-ed into the workspace status word by kernels; fxmig_check maps them
// to return codes.
enum : int {
    kStatusTimeout = 1,   // a bounded mbarrier wait gave up
    kStatusVelocity = 2,  // a velocity sample was not finite and > 0
    kStatusOverflow = 4,  // an image contribution beyond the fixed-point accumulator's range
};
// Workspace head: status word, then the image scale exponent and the
// counter of the line-norm blocks (image.cu), padded to 256 bytes.
constexpr size_t kStatusBytes = 256;
constexpr int kWsScaleExp = 1;   // int index of the image scale exponent e
constexpr int kWsNormCount = 2;  // int index of the finished line-norm blocks

// ---------------------------------------------------------- image accumulator
// The depth loops add every image row into a fixed-point accumulator that the
// caller owns as `partials` (image_planes(nx) planes of [nz][nx] floats): it
// starts with acc[nz][slow_pitch(nx)] int64 (value = acc * 2^-e[z]; rows padded
// to a multiple of 8 so that bulk reductions start on 64 bytes), followed by
// e[nz] int32.  Every frequency's contribution is converted on its own
// (image_fixed) and the integer sums do not depend on the order of the
// additions, so the image is deterministic whatever the launch shape.
// Within a row the four value pairs of 8-value chunk c are stored in the order
// p ^ ((c >> 1) & 3) (acc_slot): when the lanes of a warp store pair p of 32
// consecutive chunks (16 bytes each) into a shared-memory copy of the row,
// every 8 lanes cover all 32 banks (4 wavefronts, the minimum, instead of 16),
// and every chunk still occupies its own 64 bytes, so a run of chunks is one
// contiguous bulk reduction.
inline int slow_pitch(int nx) { return (nx + 7) & ~7; }
__host__ __device__ __forceinline__ int acc_slot(int x) {
    const int c = x >> 3;
    return (c << 3) | ((((x >> 1) & 3) ^ ((c >> 1) & 3)) << 1) | (x & 1);
}
inline int image_planes(int nx) {
    const long long bytes = 8LL * slow_pitch(nx) + 4;  // per depth row
    return (int)((bytes + 4LL * nx - 1) / (4LL * nx));
}
// Largest |contribution * 2^e| that converts to int32 (below 2^31).
constexpr float kImageFixedMax = 2147483520.0f;
// One frequency's contribution v to a pixel in fixed point (rint(v * scale)
// as a 32-bit integer, widened); sets `over` for values beyond the range.
__device__ __forceinline__ long long image_fixed(float v, float scale, bool& over) {
    float t = v * scale;
    if (!(fabsf(t) < kImageFixedMax)) {
        over = true;
        t = 0.f;
    }
    return (long long)__float2int_rn(t);
}

// Largest operator half-length compiled into the extrapolation kernels; other
// L are rounded up to the next compiled length with zero taps.
constexpr int kMaxL = 32;
int compiled_half_length(int L);  // smallest compiled LT >= L, or -1

// ------------------------------------------------------------ packed FP32 ops
// Blackwell executes two FP32 operations per lane with one f32x2 instruction.
// A u64 register holds (lo, hi) = (re, im) of a complex64 value.
typedef unsigned long long u64;

__device__ __forceinline__ u64 f2_pack(float lo, float hi) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(u64 v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ u64 f2_add(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 f2_mul(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 f2_fma(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// 16-byte read-only global load returning two packed pairs.
__device__ __forceinline__ void ldg_nc_v2(const void* p, u64& a, u64& b) {
    asm volatile("ld.global.nc.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p));
}

// ------------------------------------------------------------ mbarrier + bulk copy
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// 1-D bulk copy global -> own shared memory, completion counted on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// Bounded wait for phase `parity` of `bar`.  Returns false (and leaves the
// caller to record a timeout) after `max_iter` unsuccessful polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t max_iter) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < max_iter; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}
constexpr uint32_t kWaitPolls = 1u << 22;  // try_wait suspends between polls: seconds in total
// Halo waits: a neighbour is never more than one depth step behind, so a
// much smaller bound still leaves orders of magnitude of slack.
constexpr uint32_t kHaloPolls = 1u << 18;

// ------------------------------------------------------------------- clusters
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Split cluster barrier: arrive (release) early, wait (acquire) later; the
// work between the two overlaps the barrier latency.
__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
// Arrive without ordering this thread's earlier memory operations (for threads
// that wrote nothing the rest of the cluster reads after the barrier).
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of the same shared-memory variable in CTA `rank` of this cluster,
// as a shared::cluster address usable with st.shared::cluster.
__device__ __forceinline__ uint32_t map_cluster_rank(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}
// Remote store of 8 bytes into another CTA's shared memory that counts its
// bytes on that CTA's mbarrier (complete_tx), so the receiver learns of the
// data from its own barrier without any cluster-wide synchronisation.
__device__ __forceinline__ void st_async_v2(uint32_t addr, float2 v, uint32_t remote_bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];"
                 :: "r"(addr), "f"(v.x), "f"(v.y), "r"(remote_bar) : "memory");
}
// Bulk copy of `bytes` from this CTA's shared memory into another CTA's of
// the cluster (dst and remote_bar are shared::cluster addresses), counted on
// that CTA's mbarrier; 16-byte aligned addresses, bytes a multiple of 16.
// The copy engine moves the data: the issuing thread does not wait.
__device__ __forceinline__ void bulk_s2cluster(uint32_t dst, const void* src, uint32_t bytes, uint32_t remote_bar) {
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "r"(smem_u32(src)), "r"(bytes), "r"(remote_bar) : "memory");
}
// Bounded wait with cluster-scope acquire (data written by other CTAs).
__device__ __forceinline__ bool mbar_wait_cluster_bounded(uint64_t* bar, uint32_t parity, uint32_t max_iter) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < max_iter; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void st_cluster_v2(uint32_t addr, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" :: "r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// ------------------------------------------------------------ kernel attributes
// Dynamic shared memory limit (and, for cluster kernels, the non-portable
// cluster size permission) of a kernel on the current device, set once and
// raised only when a launch needs more: a launch repeated inside a stream
// capture then makes no attribute call.
cudaError_t kernel_smem_attr(const void* func, size_t bytes, bool nonportable_cluster);
template <class F>
inline cudaError_t ensure_smem(F* func, size_t bytes, bool nonportable_cluster = false) {
    return kernel_smem_attr(reinterpret_cast<const void*>(func), bytes, nonportable_cluster);
}

// ------------------------------------------------------------ host interfaces
struct MigratePlan {
    int mode;      // FXMIG_MODE_PERSISTENT or FXMIG_MODE_PER_DEPTH
    int precision; // FXMIG_PREC_*
    int LT;        // compiled half-length >= L
    int cluster;   // persistent: CTAs per frequency group (1, or a cluster of 2)
    int groups;    // persistent: frequency groups; per-depth: frequency tiles
    int warps;     // persistent: compute warps; per-depth: warps per CTA
    int nr;        // persistent: 8-output items per compute lane and depth step (1 or 2)
    int extra;     // persistent: the launch has cut lines (extra warp per CTA)
    int lines;     // persistent: max lines per group
    size_t smem;   // dynamic shared memory bytes per CTA
    int nparts;    // planes of the image accumulator (image_planes(nx))
    int occ;       // persistent: CTAs resident per SM the kernel is compiled for (1, or 2 for whole lines)
    int fixw;      // persistent: a fixup warp per CTA recomputes the outputs whose operator changes
};

// slow_pitch(nx) is also the row pitch of the slowness field in the
// workspace (floats), so every staged row range starts and ends on 16 bytes.

bool desc_valid(const fxmig_desc* d);
// Records a CUDA error for fxmig_last_error() and returns FXMIG_ECUDA.
int record_cuda_error(cudaError_t e, const char* where);
int plan_migrate(const fxmig_desc* d, const fxmig_launch* launch, MigratePlan* plan);
size_t migrate_ws_bytes(const fxmig_desc* d);
// The part of the FXMIG_WS_MIGRATE workspace the persistent form uses (no
// second wavefield).
size_t migrate_ws_bytes_persistent(const fxmig_desc* d);
size_t t2f_ws_bytes(const fxmig_desc* d);
bool t2f_supported(int nt);

// Plan of the persistent depth loop (depth.cuh) for storage of esize bytes
// per value; req_*: requested cluster size, groups, compute warps, CTAs per
// SM (0 = auto).
int plan_depth(const fxmig_desc* d, int LT, int esize, int req_c, int req_g, int req_w, int req_o, MigratePlan* p);
// Per call, before a depth loop: the image scale exponent from the wavefield
// (written to ws[kWsScaleExp] and to the scale rows [z_begin, z_end) of the
// accumulator) and zeroed accumulator rows.  norms: nw doubles of scratch;
// the workspace head (status, exponent, counter) must be zero.
cudaError_t launch_image_prep(const fxmig_desc* d, const void* slab, float* partials, int z_begin, int z_end,
                              void* ws, double* norms, cudaStream_t s);
// Slowness s = fl32(1/v) of rows [z_begin, z_end) into slow[nz][slow_pitch(nx)]
// (pitch padding repeats the last sample); flags bad velocities.
cudaError_t launch_slowness(const fxmig_desc* d, const float* vel, float* slow, int z_begin, int z_end,
                            int* status, cudaStream_t s);

// kvals == nullptr: the nk-entry table grid (n == nk); else n wavenumbers kvals.
cudaError_t launch_design(const fxmig_desc* d, const double* kvals, int n, void* table, void* table64,
                          cudaStream_t s);
cudaError_t launch_t2f(const fxmig_desc* d, const float* section, void* slab, void* ws, cudaStream_t s);
// precompute_slowness: write fl32(1/vel) into the workspace first and stage
// slowness rows (needs the full FXMIG_WS_MIGRATE workspace); false: convert
// velocity rows inside the depth loop (only status + table in the workspace).
cudaError_t launch_migrate(const fxmig_desc* d, const MigratePlan& plan, void* slab, const float* vel,
                           const void* table, float* partials, int z_begin, int z_end, void* ws,
                           cudaStream_t s, bool precompute_slowness);
// 16-bit storage forms of the persistent kernel (migrate_rp.cu)
struct DepthArgs;
bool rp_compiled(int LT);
cudaError_t expand_taps_rp(int precision, const float2* table, int nk, int L, int LT, void* taps, cudaStream_t s);
cudaError_t launch_depth_rp(const MigratePlan& plan, const DepthArgs& a, cudaStream_t s);
// many lines in one persistent launch (batch.cu)
bool batch_descs_valid(const fxmig_line* lines, int n);
bool batch_lines_valid(const fxmig_line* lines, int n);
size_t batch_ws_bytes(const fxmig_line* lines, int n, bool scratch);
int batch_num_partials(const fxmig_line* lines, int n, const fxmig_batch_plan* plan, int* out);
cudaError_t launch_batch(const fxmig_line* lines, int n, const fxmig_batch_plan& plan, void* ws, cudaStream_t s);
int batch_autotune(const fxmig_line* lines, int n, fxmig_batch_plan* out, void* ws, cudaStream_t s,
                   float* best_ms);
cudaError_t launch_selftest_timeout(void* ws, int polls, cudaStream_t s);
// Expand a [nk][L+1] complex64 table into the kernel layout [nk][LT+1] of
// (hr, hr, hi, hi), zero taps beyond L.
cudaError_t launch_expand_taps(const float2* table, int nk, int L, int LT, float4* taps, cudaStream_t s);
cudaError_t launch_image(const fxmig_desc* d, const float* partials, int nparts, float* image,
                         cudaStream_t s);

}  // namespace fxmig_impl
