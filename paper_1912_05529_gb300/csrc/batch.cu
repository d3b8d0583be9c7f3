// batch.cu -- many independent 2-D lines (uneven Nx, Nz, band and L) in one
// persistent launch (the depth loop of Algorithm 1 for every line).
//
// A line's frequencies are split into groups (as many lines as one CTA pair
// holds, or at most a cap); a work item is one (line, group).  One kernel
// launch keeps one CTA cluster per pair of SMs (or one CTA per SM); each
// cluster takes the next item from a device counter (items ordered largest
// first) and runs the whole depth loop of that group (run_depth of the
// persistent form, with the line's own half-length by a run-time switch over
// the compiled lengths), then takes the next item.  Every group adds its image
// rows into its line's fixed-point accumulator (image.cu), so the image does
// not depend on which cluster ran which group.  The per-line arguments travel
// in the kernel parameters, so the launch needs no host-to-device copy and
// can be captured into a CUDA graph.
//
// Planning: a cluster size C (1 or 2) for the launch and, per line, the
// frequency lines per group.  The autotuner times a few (C, cap) candidates on
// scratch copies of the wavefields over the first depth rows of every line and
// keeps the fastest.
#include <algorithm>
#include <cmath>
#include <vector>

#include "depth.cuh"

namespace fxmig_impl {

// The batch kernel carries two 8-output items per compute lane (8 compute
// warps + the extra warp): one launch then fits groups of up to 512 chunks
// per CTA, which lines up to 8192 traces need (half a line per CTA).
constexpr int kBatchNR = 2;
constexpr int kBatchComputeWarps = DepthWarps<kBatchNR>::kMaxCompute;

struct BatchLineArgs {
    DepthArgs a;
    int LT;
    const float2* table;  // the line's public [nk][L+1] table (expanded into a.taps)
    const float* vel;     // the line's velocity [nz][nx] (converted into a.slow)
    double* norms;        // [nw] frequency norms of the line's wavefield (image scale)
    int* head;            // the line's scale exponent (= a.scale_exp) and norm counter
};
struct BatchArgs {
    int nlines, nitems;
    int* counter;                              // work-queue head, zero at launch
    int order[FXMIG_BATCH_MAX_LINES];          // lines in the order their items are handed out
    int item_base[FXMIG_BATCH_MAX_LINES + 1];  // first item (group) of line order[k]
    BatchLineArgs line[FXMIG_BATCH_MAX_LINES];
};

__device__ __forceinline__ void st_cluster_u32(uint32_t addr, int v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" :: "r"(addr), "r"(v) : "memory");
}

__global__ void __launch_bounds__(DepthWarps<kBatchNR>::kThreads, 1) k_migrate_batch(const __grid_constant__ BatchArgs b) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_item;
    const int C = b.line[0].a.C;  // the launch's cluster size (the same for every line)
    const uint32_t rank = C > 1 ? cluster_ctarank() : 0u;
    for (;;) {
        // the cluster's rank 0 takes the next item and hands it to every CTA
        if (rank == 0 && threadIdx.x == 0) {
            const int item = atomicAdd(b.counter, 1);
            if (C > 1) {
                for (int r = 0; r < C; ++r) st_cluster_u32(map_cluster_rank(&s_item, (uint32_t)r), item);
            } else {
                s_item = item;
            }
        }
        if (C > 1) cluster_sync_all(); else __syncthreads();
        const int item = s_item;
        if (item >= b.nitems) break;
        int k = 0;
        while (b.item_base[k + 1] <= item) ++k;
        const BatchLineArgs& L = b.line[b.order[k]];
        const int g = item - b.item_base[k];
        switch (L.LT) {
            case 4: run_depth<4, WsF32, TapF32, kBatchNR, false>(L.a, g, smem); break;
            case 8: run_depth<8, WsF32, TapF32, kBatchNR, false>(L.a, g, smem); break;
            case 12: run_depth<12, WsF32, TapF32, kBatchNR, false>(L.a, g, smem); break;
            case 16: run_depth<16, WsF32, TapF32, kBatchNR, false>(L.a, g, smem); break;
            case 17: run_depth<17, WsF32, TapF32, kBatchNR, false>(L.a, g, smem); break;
            case 20: run_depth<20, WsF32, TapF32, kBatchNR, false>(L.a, g, smem); break;
            default: break;
        }
        // s_item is rewritten for the next item only after every CTA of the
        // cluster has finished this one (run_depth ends with a cluster barrier)
        if (C > 1) cluster_sync_all(); else __syncthreads();
    }
}

// Per-line preparation of a batch, grid.y over lines: the table in the
// kernel's tap layout, the slowness field of the line's rows, zeroed
// accumulator rows.
__global__ void k_batch_prep(const __grid_constant__ BatchArgs b) {
    for (int li = blockIdx.y; li < b.nlines; li += gridDim.y) {
        const DepthArgs& a = b.line[li].a;
        const int LT = b.line[li].LT, L = a.L;
        float4* taps = static_cast<float4*>(const_cast<void*>(a.taps));
        const int n = a.nk * (LT + 1);
        const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;
        for (int i = gtid; i < n; i += gstride) {
            const int kk = i / (LT + 1), t = i - kk * (LT + 1);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (t <= L) {
                const float2 h = b.line[li].table[(size_t)kk * (L + 1) + t];
                v = make_float4(h.x, h.x, h.y, h.y);
            }
            taps[i] = v;
        }
        const float* vel = b.line[li].vel;
        float* slow = const_cast<float*>(a.slow);
        const size_t ns = (size_t)(a.z_end - a.z_begin) * a.nxp;
        bool bad = false;
        for (size_t i = gtid; i < ns; i += gstride) {
            const int z = a.z_begin + (int)(i / (size_t)a.nxp);
            const int x = (int)(i % (size_t)a.nxp);
            const float v = vel[(size_t)z * a.nx + (x < a.nx ? x : a.nx - 1)];
            if (x < a.nx) bad |= !(v > 0.f && v <= FLT_MAX);
            slow[(size_t)z * a.nxp + x] = __frcp_rn(v);
        }
        if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(a.status, kStatusVelocity);
        const size_t na = (size_t)(a.z_end - a.z_begin) * a.nxp;
        for (size_t i = gtid; i < na; i += gstride) a.acc[(size_t)a.z_begin * a.nxp + i] = 0ull;
    }
}

// Per-line image scale (grid.y over lines, grid.x over frequency lines):
// ||P(., w)||_2 per frequency, and the line's last block picks e from the
// largest of them, as in image.cu.
__global__ void __launch_bounds__(256) k_batch_norms(const __grid_constant__ BatchArgs b) {
    __shared__ double red[256];
    __shared__ bool last;
    const int li = blockIdx.y;
    if (li >= b.nlines) return;
    const DepthArgs& a = b.line[li].a;
    if ((int)blockIdx.x >= a.nw) return;
    double* norms = b.line[li].norms;
    int* head = b.line[li].head;
    const float2* p = a.slab + (size_t)blockIdx.x * a.nx;
    double s = 0.0;
    for (int x = threadIdx.x; x < a.nx; x += blockDim.x) {
        const float2 v = p[x];
        s += (double)v.x * v.x + (double)v.y * v.y;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        norms[blockIdx.x] = sqrt(red[0]);
        __threadfence();
        last = atomicAdd(&head[1], 1) == a.nw - 1;
    }
    __syncthreads();
    if (!last) return;
    __shared__ int e_sh;
    __threadfence();
    double Bt = 0.0;
    for (int j = threadIdx.x; j < a.nw; j += blockDim.x) Bt = fmax(Bt, __ldcg(norms + j));
    red[threadIdx.x] = Bt;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double B = red[0];
        int e = 0;
        if (B > 0.0 && B <= 1.0e300) {
            int k;
            frexp(B, &k);  // the largest frequency norm < 2^k
            e = 23 - k;
        }
        e = e < -126 ? -126 : (e > 127 ? 127 : e);
        // a continued depth range keeps the previous rows' exponent (image.cu)
        const int* e_prev = reinterpret_cast<const int*>(a.acc + (size_t)a.nz * a.nxp);
        if (a.z_begin > 0) {
            const int ep = e_prev[a.z_begin - 1];
            if (ep >= e - 4 && ep <= e + 4) e = ep;
        }
        e_sh = e;
        head[0] = e;
        head[1] = 0;
    }
    __syncthreads();
    int* e_rows = reinterpret_cast<int*>(a.acc + (size_t)a.nz * a.nxp);
    for (int z = a.z_begin + (int)threadIdx.x; z < a.z_end; z += blockDim.x) e_rows[z] = e_sh;
}

// ------------------------------------------------------------------ host side
namespace {

int sms_of_device() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 148;
}
// dynamic shared memory available to the batch kernel (its static part is a
// few bytes; 1 KB is kept aside)
int smem_optin() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (v > 0 ? v : 227 * 1024) - 1024;
}
size_t r256(size_t v) { return (v + 255) & ~size_t(255); }

struct LinePlan {
    int LT, G, ncw, extra;
    size_t smem;
    double cost;  // work of one group: chunks of its busiest CTA x depth rows x FP32 operations
};

// Per-line choices for cluster size C and lines-per-group cap (0 = as many
// as fit).  Returns false if the line cannot be planned.
bool plan_line(const fxmig_desc* d, int C, int cap, int smax, LinePlan* p) {
    const int LT = compiled_half_length(d->L);
    if (LT < 0) return false;
    const int nxp = slow_pitch(d->nx);
    const int mcap = std::min(d->nw, cap > 0 ? cap : 2 * kDepthMaxSegs - 2);
    for (int m = mcap; m >= 1; --m) {
        const int G = (d->nw + m - 1) / m;
        int maxch = 0, cut = 0;
        size_t smem = 0;
        bool ok = true;
        DepthLayout L;
        for (int g = 0; g < G && ok; ++g)
            for (int r = 0; r < C && ok; ++r) {
                ok = depth_layout(d->nx, nxp, d->nw, G, C, g, r, LT, 8, L);
                if (!ok) break;
                maxch = std::max(maxch, L.nchunks);
                cut |= L.cutseg >= 0 ? 1 : 0;
                smem = std::max(smem, L.total);
            }
        if (!ok || smem > (size_t)smax || maxch == 0 || maxch > 32 * kBatchNR * kBatchComputeWarps) continue;
        p->LT = LT;
        p->G = G;
        p->ncw = std::max(1, (maxch + 32 * kBatchNR - 1) / (32 * kBatchNR));
        p->extra = (C > 1 && cut) ? 1 : 0;
        p->smem = smem;
        p->cost = (double)maxch * d->nz * (6.0 * LT + 4.0);
        return true;
    }
    return false;
}

// Depth rows of a line that the autotuner runs: an eighth of the line (at
// least 8), so the items keep the proportions of the full run.
int tune_rows(const fxmig_desc& d) { return std::min(d.nz, std::max(8, (d.nz + 7) / 8)); }

// Workspace: status word and queue counter; per-line heads (scale exponent,
// norm counter); per line the expanded table, the slowness field and the
// frequency norms; (autotuner) scratch wavefields and accumulators of the
// tuning rows.
struct BatchLayout {
    size_t heads, norm_off[FXMIG_BATCH_MAX_LINES], taps_off[FXMIG_BATCH_MAX_LINES],
        slow_off[FXMIG_BATCH_MAX_LINES], norms, scratch, total;
};
BatchLayout batch_layout(const fxmig_line* lines, int n, bool scratch) {
    BatchLayout L = {};
    size_t o = kStatusBytes;
    L.heads = o;
    o += r256((size_t)n * 16);
    L.norms = o;
    long long nn = 0;
    for (int i = 0; i < n; ++i) {
        L.norm_off[i] = (size_t)nn;
        nn += lines[i].d.nw;
    }
    o += r256((size_t)nn * 8);
    for (int i = 0; i < n; ++i) {
        const int LT = compiled_half_length(lines[i].d.L);
        L.taps_off[i] = o;
        o += r256((size_t)lines[i].d.nk * (LT + 1) * 16);
        L.slow_off[i] = o;
        o += r256((size_t)lines[i].d.nz * slow_pitch(lines[i].d.nx) * 4);
    }
    L.scratch = o;
    if (scratch) {
        for (int i = 0; i < n; ++i) {
            const fxmig_desc& d = lines[i].d;
            o += r256((size_t)d.nw * d.nx * 8);                                  // wavefield copy
            o += r256((size_t)image_planes(d.nx) * tune_rows(d) * d.nx * 4);    // accumulator rows
        }
    }
    L.total = o;
    return L;
}

}  // namespace

bool batch_descs_valid(const fxmig_line* lines, int n) {
    if (!lines || n < 1 || n > FXMIG_BATCH_MAX_LINES) return false;
    for (int i = 0; i < n; ++i)
        if (!desc_valid(&lines[i].d)) return false;
    return true;
}

bool batch_lines_valid(const fxmig_line* lines, int n) {
    if (!batch_descs_valid(lines, n)) return false;
    for (int i = 0; i < n; ++i) {
        const fxmig_line& l = lines[i];
        if (!l.slab || !l.vel || !l.table || !l.partials) return false;
        if ((reinterpret_cast<uintptr_t>(l.slab) & 7) || (reinterpret_cast<uintptr_t>(l.vel) & 3) ||
            (reinterpret_cast<uintptr_t>(l.table) & 7) || (reinterpret_cast<uintptr_t>(l.partials) & 15))
            return false;
        if (l.z_begin < 0 || l.z_end < l.z_begin || l.z_end > l.d.nz) return false;
    }
    return true;
}

namespace {
bool plan_batch(const fxmig_line* lines, int n, const fxmig_batch_plan& plan, std::vector<LinePlan>* lp) {
    const int C = plan.cluster;
    if (C != 1 && C != 2) return false;
    const int smax = smem_optin();
    lp->assign(n, LinePlan());
    for (int i = 0; i < n; ++i)
        if (!plan_line(&lines[i].d, C, plan.lines_cap, smax, &(*lp)[i])) return false;
    return true;
}

// The autotuner's candidate plans: cluster sizes 2 and 1, each with as many
// lines per group as fit and with a cap of half of what fits on the
// narrowest line.
std::vector<fxmig_batch_plan> tune_candidates(const fxmig_line* lines, int n) {
    std::vector<fxmig_batch_plan> out;
    for (int C : {2, 1}) {
        std::vector<LinePlan> lp;
        const fxmig_batch_plan p0 = {C, 0};
        if (!plan_batch(lines, n, p0, &lp)) continue;
        out.push_back(p0);
        int fit_min = 1 << 30;
        for (int i = 0; i < n; ++i) fit_min = std::min(fit_min, (lines[i].d.nw + lp[i].G - 1) / lp[i].G);
        if (fit_min >= 2) out.push_back(fxmig_batch_plan{C, fit_min / 2});
    }
    return out;
}
}  // namespace

size_t batch_ws_bytes(const fxmig_line* lines, int n, bool scratch) { return batch_layout(lines, n, scratch).total; }

int batch_num_partials(const fxmig_line* lines, int n, const fxmig_batch_plan* plan, int* out) {
    fxmig_batch_plan p = {2, 0};
    if (plan) {
        p = *plan;
        if (p.cluster == 0) p.cluster = 2;
    }
    std::vector<LinePlan> lp;
    if (!plan_batch(lines, n, p, &lp)) return FXMIG_EINVAL;
    for (int i = 0; i < n; ++i) out[i] = image_planes(lines[i].d.nx);
    return FXMIG_OK;
}

// Fill the launch arguments for plan; with slabs != nullptr (autotuner)
// every line runs on a scratch wavefield and scratch accumulator over its
// first tune_rows depth rows.
static int fill_args(const fxmig_line* lines, int n, const fxmig_batch_plan& plan, unsigned char* wsb,
                     BatchArgs* b, size_t* smem_max, int* warps, const std::vector<float2*>* slabs,
                     const std::vector<float*>* accs) {
    const int C = plan.cluster;
    const BatchLayout Lw = batch_layout(lines, n, false);
    std::vector<LinePlan> lp;
    if (!plan_batch(lines, n, plan, &lp)) return FXMIG_EINVAL;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    // largest groups first
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return lp[x].cost > lp[y].cost; });
    b->nlines = n;
    b->counter = reinterpret_cast<int*>(wsb + sizeof(int));
    b->item_base[0] = 0;
    *smem_max = 0;
    int ncw = 1, extra = 0;
    for (int i = 0; i < n; ++i) {
        ncw = std::max(ncw, lp[i].ncw);
        extra |= lp[i].extra;
    }
    *warps = ncw + extra;
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        b->order[k] = i;
        b->item_base[k + 1] = b->item_base[k] + lp[i].G;
        *smem_max = std::max(*smem_max, lp[i].smem);
        const fxmig_desc& d = lines[i].d;
        DepthArgs a = {};
        a.nx = d.nx; a.nxp = slow_pitch(d.nx); a.nz = d.nz; a.nw = d.nw; a.nk = d.nk; a.L = d.L;
        a.i0 = d.i0; a.nt = d.nt;
        a.z_begin = lines[i].z_begin;
        a.z_end = lines[i].z_end;
        a.dt = d.dt;
        a.dk = d.nk > 1 ? d.k_max / (double)(d.nk - 1) : 0.0;
        a.slab = static_cast<float2*>(lines[i].slab);
        a.slow = reinterpret_cast<const float*>(wsb + Lw.slow_off[i]);
        a.taps = wsb + Lw.taps_off[i];
        a.acc = reinterpret_cast<unsigned long long*>(lines[i].partials);
        int* head = reinterpret_cast<int*>(wsb + Lw.heads) + 4 * i;
        a.scale_exp = head;
        a.status = reinterpret_cast<int*>(wsb);
        a.C = C; a.G = lp[i].G; a.ncw = ncw; a.extra = extra;
        if (slabs) {  // autotuner: scratch wavefield and accumulator rows, first rows
            a.slab = (*slabs)[i];
            a.acc = reinterpret_cast<unsigned long long*>((*accs)[i]);
            a.z_begin = 0;
            a.z_end = tune_rows(d);
            a.nz = a.z_end;  // accumulator rows are indexed by the scratch's depth count
        }
        b->line[i].a = a;
        b->line[i].LT = lp[i].LT;
        b->line[i].table = static_cast<const float2*>(lines[i].table);
        b->line[i].vel = lines[i].vel;
        b->line[i].norms = reinterpret_cast<double*>(wsb + Lw.norms) + Lw.norm_off[i];
        b->line[i].head = head;
    }
    b->nitems = b->item_base[n];
    return FXMIG_OK;
}

static cudaError_t launch_batch_kernel(const BatchArgs& b, size_t smem, int C, int warps, int* counter,
                                       cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    e = ensure_smem(k_migrate_batch, smem, false);
    if (e != cudaSuccess) return e;
    const int clusters = std::max(1, std::min(sms_of_device() / C, b.nitems));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(clusters * C);
    cfg.blockDim = dim3(warps * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_migrate_batch, b);
}

// Everything the batch kernel reads that depends on the call: the status
// word, queue counter and per-line heads cleared; tables, slowness fields and
// zeroed accumulator rows; the image scales of the lines' wavefields.
static cudaError_t prepare(const BatchArgs& b, unsigned char* wsb, const BatchLayout& Lw, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(wsb, 0, Lw.heads + (size_t)b.nlines * 16, s);
    if (e != cudaSuccess) return e;
    k_batch_prep<<<dim3(16, std::min(b.nlines, 65535)), 256, 0, s>>>(b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int nwmax = 1;
    for (int i = 0; i < b.nlines; ++i) nwmax = std::max(nwmax, b.line[i].a.nw);
    k_batch_norms<<<dim3(nwmax, b.nlines), 256, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_batch(const fxmig_line* lines, int n, const fxmig_batch_plan& plan, void* ws, cudaStream_t s) {
    unsigned char* wsb = static_cast<unsigned char*>(ws);
    std::vector<BatchArgs> hold(1);  // ~25 KB of launch arguments
    BatchArgs& b = hold[0];
    size_t smem = 0;
    int warps = 0;
    if (fill_args(lines, n, plan, wsb, &b, &smem, &warps, nullptr, nullptr) != FXMIG_OK) return cudaErrorInvalidValue;
    const BatchLayout Lw = batch_layout(lines, n, false);
    cudaError_t e = prepare(b, wsb, Lw, s);
    if (e != cudaSuccess) return e;
    return launch_batch_kernel(b, smem, plan.cluster, warps, b.counter, s);
}

int batch_autotune(const fxmig_line* lines, int n, fxmig_batch_plan* out, void* ws, cudaStream_t s,
                   float* best_ms) {
    unsigned char* wsb = static_cast<unsigned char*>(ws);
    const BatchLayout Lw = batch_layout(lines, n, true);
    // scratch wavefields (copies of the caller's) and accumulators
    std::vector<float2*> slabs(n);
    std::vector<float*> accs(n);
    size_t o = Lw.scratch;
    for (int i = 0; i < n; ++i) {
        const fxmig_desc& d = lines[i].d;
        slabs[i] = reinterpret_cast<float2*>(wsb + o);
        o += r256((size_t)d.nw * d.nx * 8);
        accs[i] = reinterpret_cast<float*>(wsb + o);
        o += r256((size_t)image_planes(d.nx) * tune_rows(d) * d.nx * 4);
    }
    const std::vector<fxmig_batch_plan> cands = tune_candidates(lines, n);
    if (cands.empty()) return FXMIG_EINVAL;
    std::vector<BatchArgs> hold(1);
    BatchArgs& b = hold[0];
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FXMIG_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FXMIG_ECUDA;
    }
    cudaError_t e = cudaSuccess;
    float best = 1e30f;
    fxmig_batch_plan best_plan = {0, 0};
    for (const fxmig_batch_plan& p : cands) {
        size_t smem = 0;
        int warps = 0;
        if (fill_args(lines, n, p, wsb, &b, &smem, &warps, &slabs, &accs) != FXMIG_OK) continue;
        for (int i = 0; i < n && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(slabs[i], lines[i].slab, (size_t)lines[i].d.nw * lines[i].d.nx * 8,
                                cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = prepare(b, wsb, Lw, s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = launch_batch_kernel(b, smem, p.cluster, warps, b.counter, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        if (ms < best) {
            best = ms;
            best_plan = p;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return FXMIG_ECUDA;
    if (best_plan.cluster == 0) return FXMIG_EINVAL;
    *out = best_plan;
    if (best_ms) *best_ms = best;
    return FXMIG_OK;
}

}  // namespace fxmig_impl
