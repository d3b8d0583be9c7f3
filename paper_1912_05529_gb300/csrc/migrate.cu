// migrate.cu -- depth loop of explicit f-x poststack depth migration
// (Algorithm 1; Eq. 1; Sec. III per-point operator lookup) for sm_103a:
// planning, the per-depth-launch form, and the FP32 persistent form (the
// kernel itself is in depth.cuh; the 16-bit storage forms are compiled in
// migrate_rp.cu).
//
//  * persistent (one launch): frequency lines stay in shared memory for all
//    depth steps (depth.cuh).
//  * per-depth (one launch per depth step): the wavefield streams through
//    L2/HBM; a CTA computes a 256-point x tile of a frequency tile.
//
// Compute kernel shared by both: a lane produces 8 consecutive outputs of one
// line from a register window of 8 + 2L values read out of shared memory.
// Shared-memory line layout: position p (p = x - x_seg + L) lives at
// p + 2 (p / 8), i.e. groups of 8 complex values padded by 2, so that the
// window loads of a warp (lane stride 8 outputs = 10 values) hit distinct
// banks.  Both forms add the image rows into the fixed-point accumulator of
// image.cu.
#include <float.h>
#include <math.h>

#include <string.h>

#include <algorithm>
#include <mutex>

#include "depth.cuh"
#include "fir.cuh"
#include "fxmig_internal.cuh"

namespace fxmig_impl {

int compiled_half_length(int L) {
    static const int kLs[] = {4, 8, 12, 16, 17, 20};
    for (int v : kLs)
        if (v >= L) return v;
    return -1;
}

// ------------------------------------------------------------ per-depth form
constexpr int kStepWarps = 8;
constexpr int kStepTile = 256;  // x outputs per CTA (32 lanes x 8)

struct StepArgs {
    int nx, nw, nk, G, i0, nt, z, nxp;
    double dt, dk;
    const float2* in;
    float2* out;
    const float* slow;         // [nz][nxp] slowness
    const float4* taps;        // [nk][LT+1] (hr, hr, hi, hi)
    unsigned long long* acc;   // [nz][nx] image accumulator
    const int* scale_exp;
    int* status;
};

template <int LT>
__global__ void __launch_bounds__(kStepWarps * 32) k_migrate_step(const StepArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int SP = ((kStepTile + 2 * LT + 7) >> 3) * 10;
    float* srow = reinterpret_cast<float*>(smem);                               // [256]
    long long* imgw = reinterpret_cast<long long*>(srow + kStepTile);           // [warps][256]
    float2* buf = reinterpret_cast<float2*>(imgw + kStepWarps * kStepTile);     // [warps][SP]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = blockIdx.x * kStepTile;
    const int lb = (int)(((long long)blockIdx.y * a.nw) / a.G);
    const int le = (int)(((long long)(blockIdx.y + 1) * a.nw) / a.G);
    const int z = a.z;
    {
        const int x = x0 + tid;
        srow[tid] = x < a.nxp ? a.slow[(size_t)z * a.nxp + x] : 0.f;
    }
    __syncthreads();
    // image: every frequency's contribution in fixed point, summed exactly
    long long acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const float scale = depth_scale(*a.scale_exp);
    bool over = false;
    float2* wb = buf + (size_t)warp * SP;
    float s8[8];
    load_s8(srow + lane * 8, s8);
    for (int l = lb + warp; l < le; l += kStepWarps) {
        const float2* src = a.in + (size_t)l * a.nx;
        for (int pos = lane; pos < kStepTile + 2 * LT; pos += 32) {
            const int x = x0 - LT + pos;
            wb[phys(pos)] = (x >= 0 && x < a.nx) ? src[x] : make_float2(0.f, 0.f);
        }
        __syncwarp();
        float re[8];
        u64 res[8];
        // one tap load per tap for 8 outputs where the whole warp's outputs
        // share their operator; per-output operators otherwise
        const float q = q_of_line(a.i0, l, a.nt, a.dt, a.dk);
        const int idx0 = table_index(q, s8[0], a.nk);
        bool uni = true;
#pragma unroll
        for (int r = 1; r < 8; ++r) uni &= table_index(q, s8[r], a.nk) == idx0;
        if (__all_sync(0xffffffffu, uni))
            fir8_shared_taps<LT, WsF32, TapF32>(wb + lane * 10, a.taps + (size_t)idx0 * (LT + 1), res, re);
        else
            fir8<LT>(wb + lane * 10, s8, q, a.nk, a.taps, res, re);
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[r] += image_fixed(re[r], scale, over);
        float2* dst = a.out + (size_t)l * a.nx;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int x = x0 + lane * 8 + r;
            if (x < a.nx) dst[x] = f2_unpack(res[r]);
        }
        __syncwarp();
    }
    if (over) atomicOr(a.status, kStatusOverflow);
#pragma unroll
    for (int r = 0; r < 8; ++r) imgw[warp * kStepTile + lane * 8 + r] = acc[r];
    __syncthreads();
    {
        const int x = x0 + tid;
        if (x < a.nx) {
            long long s = 0;
            for (int w = 0; w < kStepWarps; ++w) s += imgw[w * kStepTile + tid];
            if (s) depth_red_add_u64(a.acc + (size_t)z * a.nxp + acc_slot(x), s);
        }
    }
}

// Slowness s = fl32(1/v) of every velocity sample of rows [z0, z1) into the
// pitched field slow[z][nxp] (one pass per call, so the depth loops never
// divide); the pitch padding repeats the row's last sample.  Flags samples
// that are not finite and > 0.
__global__ void k_slowness(const float* __restrict__ vel, int nx, int nxp, int z0, int z1, float* __restrict__ slow,
                           int* status) {
    bool bad = false;
    const size_t n = (size_t)(z1 - z0) * nxp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int z = z0 + (int)(i / (size_t)nxp);
        const int x = (int)(i % (size_t)nxp);
        const float v = vel[(size_t)z * nx + (x < nx ? x : nx - 1)];
        if (x < nx) bad |= !(v > 0.f && v <= FLT_MAX);
        slow[(size_t)z * nxp + x] = __frcp_rn(v);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusVelocity);
}

cudaError_t launch_slowness(const fxmig_desc* d, const float* vel, float* slow, int z_begin, int z_end, int* status,
                            cudaStream_t s) {
    const int nxp = slow_pitch(d->nx);
    const size_t n = (size_t)(z_end - z_begin) * nxp;
    if (n == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t blocks = (n + 255) / 256;
    const size_t cap = (size_t)(sms > 0 ? sms : 148) * 8;
    if (blocks > cap) blocks = cap;
    k_slowness<<<(unsigned)blocks, 256, 0, s>>>(vel, d->nx, nxp, z_begin, z_end, slow, status);
    return cudaGetLastError();
}

// Expand the public [nk][L+1] complex64 table into the kernel layout
// [nk][LT+1] of (hr, hr, hi, hi), zero taps beyond L.
__global__ void k_expand_taps(const float2* __restrict__ table, int nk, int L, int LT, float4* __restrict__ taps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nk * (LT + 1)) return;
    const int k = i / (LT + 1), n = i - k * (LT + 1);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n <= L) {
        const float2 h = table[(size_t)k * (L + 1) + n];
        v = make_float4(h.x, h.x, h.y, h.y);
    }
    taps[i] = v;
}

cudaError_t launch_expand_taps(const float2* table, int nk, int L, int LT, float4* taps, cudaStream_t s) {
    const int n = nk * (LT + 1);
    if (n == 0) return cudaSuccess;
    k_expand_taps<<<(n + 255) / 256, 256, 0, s>>>(table, nk, L, LT, taps);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- host side
namespace {
size_t r256(size_t v) { return (v + 255) & ~size_t(255); }

// Workspace of FXMIG_WS_MIGRATE: head (status, image scale exponent, norm
// counter), expanded table, slowness field [nz][nxp], line norms [nw], a second
// wavefield (per-depth form).
struct MigrateWs {
    size_t taps, slow, norms, slab2, total;
};
MigrateWs migrate_ws_layout(const fxmig_desc* d, int LT) {
    MigrateWs w;
    size_t o = kStatusBytes;
    w.taps = o;
    o += r256((size_t)d->nk * (LT + 1) * 16);
    w.slow = o;
    o += r256((size_t)d->nz * slow_pitch(d->nx) * 4);
    w.norms = o;
    o += r256((size_t)d->nw * 8);
    w.slab2 = o;
    o += r256((size_t)d->nw * d->nx * 8);
    w.total = o;
    return w;
}

int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 148;
}
int device_smem_optin() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v > 0 ? v : 227 * 1024;
}
// dynamic shared memory each of two CTAs resident on one SM may use
int device_smem_half() {
    int dev = 0, sm = 0, res = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&res, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (sm <= 0) sm = 228 * 1024;
    if (res < 0) res = 1024;
    return sm / 2 - res;
}
}  // namespace

size_t migrate_ws_bytes(const fxmig_desc* d) {
    const int LT = compiled_half_length(d->L);
    if (LT < 0) return 0;
    return migrate_ws_layout(d, LT).total;
}

size_t migrate_ws_bytes_persistent(const fxmig_desc* d) {
    const int LT = compiled_half_length(d->L);
    if (LT < 0) return 0;
    return migrate_ws_layout(d, LT).slab2;
}

int plan_depth(const fxmig_desc* d, int LT, int esize, int req_c, int req_g, int req_w, int req_o,
               MigratePlan* p) {
    const int sms = device_sms();
    const size_t smax = (size_t)device_smem_optin();
    const size_t shalf = (size_t)std::max(0, device_smem_half());
    const int nxp = slow_pitch(d->nx);
    double best = 1e300;
    bool found = false;
    // (cluster, CTAs per SM): cut lines in clusters of 2, whole lines one or
    // two CTAs per SM
    const int cand[3][2] = {{2, 1}, {1, 1}, {1, 2}};
    for (const auto& cc : cand) {
        const int C = cc[0], occ = cc[1];
        if (req_c && C != req_c) continue;
        if (req_o && occ != req_o) continue;
        const int per_wave = std::max(1, occ * (C == 1 ? sms : sms / 2));
        const int wmax = occ == 2 ? DepthWarps<1, 2>::kMaxCompute : DepthWarps<1>::kMaxCompute;
        const int m_max = std::min(d->nw, 2 * kDepthMaxSegs - 2);
        for (int m = 1; m <= m_max; ++m) {
            const int G = req_g ? std::min(req_g, d->nw) : (d->nw + m - 1) / m;
            if (!req_g && m > 1 && G == (d->nw + m - 2) / (m - 1)) continue;  // same G as m - 1
            int maxch = 0, cut = 0;
            size_t smem = 0;
            bool ok = true;
            DepthLayout L;
            for (int g = 0; g < G && ok; ++g)
                for (int r = 0; r < C && ok; ++r) {
                    ok = depth_layout(d->nx, nxp, d->nw, G, C, g, r, LT, esize, L, occ == 2);
                    if (!ok) break;
                    maxch = std::max(maxch, L.nchunks);
                    cut |= L.cutseg >= 0 ? 1 : 0;
                    smem = std::max(smem, L.total);
                }
            if (!ok || smem > (occ == 2 ? shalf : smax) || maxch == 0) {
                if (req_g) break;
                continue;
            }
            int nr = 0, ncw = 0;
            if (maxch <= 32 * wmax) {
                nr = 1;
                ncw = (maxch + 31) / 32;
            } else if (occ == 1 && maxch <= 64 * DepthWarps<2>::kMaxCompute) {
                nr = 2;
                ncw = (maxch + 63) / 64;
            }
            if (req_w) {
                if (req_w * 32 >= maxch && req_w <= wmax) {
                    nr = 1;
                    ncw = req_w;
                } else if (occ == 1 && req_w * 64 >= maxch && req_w <= DepthWarps<2>::kMaxCompute) {
                    nr = 2;
                    ncw = req_w;
                } else {
                    nr = 0;
                }
            }
            // one CTA per SM: a fixup warp and its queue (one item per lane:
            // required; two: where the queue fits, else the in-warp rounds)
            int fixw = 0;
            if (occ == 1 && (nr == 1 || nr == 2)) {
                size_t sf = 0;
                int bufmax = 0;
                for (int g = 0; g < G; ++g)
                    for (int r = 0; r < C; ++r) {
                        depth_layout(d->nx, nxp, d->nw, G, C, g, r, LT, esize, L, false, true);
                        sf = std::max(sf, L.total);
                        bufmax = std::max(bufmax, L.buf);
                    }
                // queue entries hold a window base in 16 bits
                if (sf <= smax && bufmax < 65536) {
                    fixw = 1;
                    smem = sf;
                } else if (nr == 1) {
                    nr = 0;
                }
            }
            if (nr == 0) {
                if (req_g) break;
                continue;
            }
            // per depth step: warp items on the busiest SM sub-partition, plus
            // the step's fixed costs (barrier, imaging, operator changes; with
            // a cut, the extra warp's exchange); waves of groups run one after
            // another.  Calibrated on 2048-trace lines (221 frequencies): the
            // cut plan (1.5 lines per SM) 2.55 ms, two whole-line CTAs per SM
            // 3.07 ms.
            const int waves = (G + per_wave - 1) / per_wave;
            const int resident = std::min(occ, (G + (C == 1 ? sms : sms / 2) - 1) / (C == 1 ? sms : sms / 2));
            const double fixed = (occ == 2 ? 1.0 : 0.35) + ((C > 1 && cut) ? 0.5 : 0.0);
            const double cost = (double)waves * (nr * ((resident * ncw + 3) / 4) + fixed);
            if (cost < best - 1e-9) {
                best = cost;
                found = true;
                p->cluster = C;
                p->groups = G;
                p->warps = ncw;
                p->nr = nr;
                p->extra = (C > 1 && cut) ? 1 : 0;
                p->lines = (d->nw + G - 1) / G;
                p->smem = smem;
                p->nparts = image_planes(d->nx);
                p->occ = occ;
                p->fixw = fixw;
            }
            if (req_g) break;
        }
    }
    return found ? FXMIG_OK : FXMIG_EINVAL;
}

static int precision_of(const fxmig_launch* launch) { return launch ? launch->precision : FXMIG_PREC_FP32; }

int plan_migrate(const fxmig_desc* d, const fxmig_launch* launch, MigratePlan* p) {
    const int LT = compiled_half_length(d->L);
    if (LT < 0) return FXMIG_EINVAL;
    const int mode = (launch && launch->mode) ? launch->mode : FXMIG_MODE_PERSISTENT;
    if (mode != FXMIG_MODE_PERSISTENT && mode != FXMIG_MODE_PER_DEPTH) return FXMIG_EINVAL;
    const int prec = precision_of(launch);
    if (prec < FXMIG_PREC_FP32 || prec > FXMIG_PREC_BF16_SPLIT) return FXMIG_EINVAL;
    if (prec != FXMIG_PREC_FP32 && (mode != FXMIG_MODE_PERSISTENT || !rp_compiled(LT))) return FXMIG_EINVAL;
    *p = MigratePlan();
    p->mode = mode;
    p->LT = LT;
    p->precision = prec;
    p->nparts = image_planes(d->nx);
    if (mode == FXMIG_MODE_PER_DEPTH) {
        int G = (launch && launch->groups > 0) ? launch->groups : std::max(1, std::min(d->nw, 16));
        G = std::min(G, std::max(1, d->nw));
        p->cluster = 1;
        p->groups = G;
        p->warps = kStepWarps;
        p->lines = (d->nw + G - 1) / G;
        p->smem = (size_t)kStepTile * 4 + (size_t)kStepWarps * kStepTile * 8 +
                  (size_t)kStepWarps * (((kStepTile + 2 * LT + 7) >> 3) * 10) * 8;
        return FXMIG_OK;
    }
    const int req_c = launch ? launch->cluster : 0;
    if (req_c && req_c != 1 && req_c != 2) return FXMIG_EINVAL;
    const int req_w = launch ? launch->warps : 0;
    if (req_w < 0 || req_w > kDepthMaxComputeWarps) return FXMIG_EINVAL;
    const int req_g = (launch && launch->groups > 0) ? launch->groups : 0;
    const int req_o = launch ? launch->ctas_per_sm : 0;
    if (req_o < 0 || req_o > 2 || (req_o == 2 && req_c == 2)) return FXMIG_EINVAL;
    return plan_depth(d, LT, prec == FXMIG_PREC_FP32 ? 8 : 4, req_c, req_g, req_w, req_o, p);
}

DepthArgs depth_args(const fxmig_desc* d, const MigratePlan& plan, void* slab, const float* slow, const void* taps,
                     float* partials, int z_begin, int z_end, int* head) {
    DepthArgs a = {};
    a.nx = d->nx; a.nxp = slow_pitch(d->nx); a.nz = d->nz; a.nw = d->nw; a.nk = d->nk; a.L = d->L;
    a.z_begin = z_begin; a.z_end = z_end; a.i0 = d->i0; a.nt = d->nt;
    a.dt = d->dt;
    a.dk = d->nk > 1 ? d->k_max / (double)(d->nk - 1) : 0.0;
    a.slab = static_cast<float2*>(slab);
    a.slow = slow;
    a.taps = taps;
    a.acc = reinterpret_cast<unsigned long long*>(partials);
    a.scale_exp = head + kWsScaleExp;
    a.status = head;
    a.C = plan.cluster; a.G = plan.groups; a.ncw = plan.warps; a.extra = plan.extra; a.fixw = plan.fixw;
    return a;
}

// The per-depth form's launches as one CUDA graph: captured on a private
// stream the first time a given set of arguments is seen, instantiated, and
// replayed on the caller's stream (the graph's kernel arguments hold every
// pointer, so an identical call can replay it).  A few graphs are kept per
// process (least recently used dropped).  A caller stream that is itself being
// captured gets the launches directly.
namespace {
struct StepGraphKey {
    int dev, LT, nx, nz, nw, nk, i0, nt, G, z_begin, z_end;
    double dt, dk;
    const void *slab, *slow, *taps, *partials, *head, *ws_slab;
    bool operator==(const StepGraphKey& o) const { return memcmp(this, &o, sizeof(*this)) == 0; }
};
struct StepGraph {
    StepGraphKey key;
    cudaGraphExec_t exec;
    unsigned long long used;
};
std::mutex g_step_graph_mu;
StepGraph g_step_graphs[8];
int g_step_graph_n = 0;
unsigned long long g_step_graph_tick = 0;
cudaStream_t g_capture_stream[64] = {};
}  // namespace

template <int LT>
static cudaError_t enqueue_per_depth(const fxmig_desc* d, const MigratePlan& plan, void* slab, const float* slow,
                                     const float4* taps, float* partials, int z_begin, int z_end, int* head,
                                     float2* ws_slab, cudaStream_t s);

template <int LT>
static cudaError_t launch_per_depth(const fxmig_desc* d, const MigratePlan& plan, void* slab, const float* slow,
                                    const float4* taps, float* partials, int z_begin, int z_end, int* head,
                                    float2* ws_slab, cudaStream_t s) {
    cudaError_t e = ensure_smem(k_migrate_step<LT>, plan.smem);
    if (e != cudaSuccess) return e;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusNone)
        return enqueue_per_depth<LT>(d, plan, slab, slow, taps, partials, z_begin, z_end, head, ws_slab, s);
    StepGraphKey key;
    memset(&key, 0, sizeof(key));
    e = cudaGetDevice(&key.dev);
    if (e != cudaSuccess) return e;
    if (key.dev < 0 || key.dev >= 64)
        return enqueue_per_depth<LT>(d, plan, slab, slow, taps, partials, z_begin, z_end, head, ws_slab, s);
    key.LT = LT; key.nx = d->nx; key.nz = d->nz; key.nw = d->nw; key.nk = d->nk; key.i0 = d->i0; key.nt = d->nt;
    key.G = plan.groups; key.z_begin = z_begin; key.z_end = z_end;
    key.dt = d->dt; key.dk = d->nk > 1 ? d->k_max / (double)(d->nk - 1) : 0.0;
    key.slab = slab; key.slow = slow; key.taps = taps; key.partials = partials; key.head = head;
    key.ws_slab = ws_slab;
    std::lock_guard<std::mutex> lock(g_step_graph_mu);
    for (int i = 0; i < g_step_graph_n; ++i)
        if (g_step_graphs[i].key == key) {
            g_step_graphs[i].used = ++g_step_graph_tick;
            return cudaGraphLaunch(g_step_graphs[i].exec, s);
        }
    cudaStream_t& cap = g_capture_stream[key.dev];
    if (!cap) {
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t e_enq = enqueue_per_depth<LT>(d, plan, slab, slow, taps, partials, z_begin, z_end, head,
                                                    ws_slab, cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cap, &graph);
    if (e_enq != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return e_enq != cudaSuccess ? e_enq : e;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    int slot = g_step_graph_n;
    if (g_step_graph_n < 8) {
        ++g_step_graph_n;
    } else {
        slot = 0;
        for (int i = 1; i < 8; ++i)
            if (g_step_graphs[i].used < g_step_graphs[slot].used) slot = i;
        cudaGraphExecDestroy(g_step_graphs[slot].exec);
    }
    g_step_graphs[slot].key = key;
    g_step_graphs[slot].exec = exec;
    g_step_graphs[slot].used = ++g_step_graph_tick;
    return cudaGraphLaunch(exec, s);
}

template <int LT>
static cudaError_t enqueue_per_depth(const fxmig_desc* d, const MigratePlan& plan, void* slab, const float* slow,
                                     const float4* taps, float* partials, int z_begin, int z_end, int* head,
                                     float2* ws_slab, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    StepArgs a = {};
    a.nx = d->nx; a.nw = d->nw; a.nk = d->nk; a.G = plan.groups; a.i0 = d->i0; a.nt = d->nt;
    a.nxp = slow_pitch(d->nx);
    a.dt = d->dt;
    a.dk = d->nk > 1 ? d->k_max / (double)(d->nk - 1) : 0.0;
    a.slow = slow;
    a.taps = taps;
    a.acc = reinterpret_cast<unsigned long long*>(partials);
    a.scale_exp = head + kWsScaleExp;
    a.status = head;
    const dim3 grid((d->nx + kStepTile - 1) / kStepTile, plan.groups);
    float2* bufs[2] = {static_cast<float2*>(slab), ws_slab};
    const int nsteps = z_end - z_begin;
    for (int i = 0; i < nsteps; ++i) {
        a.in = bufs[i & 1];
        a.out = bufs[(i + 1) & 1];
        a.z = z_begin + i;
        k_migrate_step<LT><<<grid, kStepWarps * 32, plan.smem, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (nsteps & 1) return cudaMemcpyAsync(slab, ws_slab, (size_t)d->nw * d->nx * 8, cudaMemcpyDeviceToDevice, s);
    return cudaSuccess;
}

template <int LT>
static cudaError_t launch_fp32(const fxmig_desc* d, const MigratePlan& plan, const DepthArgs& a, float2* ws_slab,
                               cudaStream_t s) {
    if (plan.mode == FXMIG_MODE_PERSISTENT) return launch_depth<LT, WsF32, TapF32, false>(plan, a, s);
    return launch_per_depth<LT>(d, plan, a.slab, a.slow, static_cast<const float4*>(a.taps),
                                reinterpret_cast<float*>(a.acc), a.z_begin, a.z_end, a.status, ws_slab, s);
}

cudaError_t launch_migrate(const fxmig_desc* d, const MigratePlan& plan, void* slab, const float* vel,
                           const void* table, float* partials, int z_begin, int z_end, void* ws, cudaStream_t s,
                           bool /*precompute_slowness*/) {
    const int LT = plan.LT;
    const MigrateWs W = migrate_ws_layout(d, LT);
    unsigned char* wsb = static_cast<unsigned char*>(ws);
    int* head = reinterpret_cast<int*>(wsb);
    void* taps = wsb + W.taps;
    float* slow = reinterpret_cast<float*>(wsb + W.slow);
    double* norms = reinterpret_cast<double*>(wsb + W.norms);
    float2* ws_slab = reinterpret_cast<float2*>(wsb + W.slab2);
    cudaError_t e = cudaMemsetAsync(head, 0, 16, s);  // status, scale exponent, norm counter
    if (e != cudaSuccess) return e;
    if (plan.precision == FXMIG_PREC_FP32) {
        const int n = d->nk * (LT + 1);
        k_expand_taps<<<(n + 255) / 256, 256, 0, s>>>(static_cast<const float2*>(table), d->nk, d->L, LT,
                                                       static_cast<float4*>(taps));
        e = cudaGetLastError();
    } else {
        e = expand_taps_rp(plan.precision, static_cast<const float2*>(table), d->nk, d->L, LT, taps, s);
    }
    if (e != cudaSuccess) return e;
    e = launch_slowness(d, vel, slow, z_begin, z_end, head, s);
    if (e != cudaSuccess) return e;
    e = launch_image_prep(d, slab, partials, z_begin, z_end, ws, norms, s);
    if (e != cudaSuccess) return e;
    const DepthArgs a = depth_args(d, plan, slab, slow, taps, partials, z_begin, z_end, head);
    if (plan.precision != FXMIG_PREC_FP32) return launch_depth_rp(plan, a, s);
    switch (LT) {
        case 4: return launch_fp32<4>(d, plan, a, ws_slab, s);
        case 8: return launch_fp32<8>(d, plan, a, ws_slab, s);
        case 12: return launch_fp32<12>(d, plan, a, ws_slab, s);
        case 16: return launch_fp32<16>(d, plan, a, ws_slab, s);
        case 17: return launch_fp32<17>(d, plan, a, ws_slab, s);
        case 20: return launch_fp32<20>(d, plan, a, ws_slab, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fxmig_impl
