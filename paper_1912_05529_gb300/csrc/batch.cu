// batch.cu -- many independent 2-D lines (uneven Nx, Nz, band and L) in one
// persistent launch (the depth loop of Algorithm 1 for every line).
//
// A line's frequencies are split into groups (as many lines as fit one CTA's
// shared memory), and its groups into a few streams, sized so that the batch
// has about four streams per cluster.  Work items are (line, stream) pairs.
// One kernel launch keeps one CTA cluster per group of SMs; each cluster
// takes the next item from a device counter (largest items first) and runs
// the whole depth loop of each group of that stream in turn (run_group of
// the persistent form), adding the groups' image rows into the stream's
// partial image in a fixed order (deterministic), then takes the next item.
// The per-line arguments travel in the kernel parameters, so the launch needs
// no host-to-device copy and can be captured into a CUDA graph.
//
// Planning: a cluster size C for the launch and, per line, the segment width
// W = nx / C and the frequency lines per group (as many as fit shared memory,
// or at most a cap).  The autotuner times a few (C, cap) candidates on scratch
// copies of the wavefields over the first depth steps and keeps the fastest.
#include <algorithm>
#include <cmath>
#include <vector>

#include "persistent.cuh"

namespace fxmig_impl {

// 12 warps: with clusters of 2 or more CTAs, 11 compute warps and the edge
// warp of the depth loop (run_group); clusters of 1 compute with all 12.
// Twelve warps keep 168 registers per thread (three warps per SM
// sub-partition), which the batch kernel's switch over the compiled
// half-lengths needs more than a thirteenth warp (measured on the 64-line
// batch: 530 ms against 570 ms).
constexpr int kBatchWarps = kPersistentMaxWarps;

struct BatchLineArgs {
    MigrateArgs a;
    int LT;
    int P;                // streams of the line (its partial images)
    const float2* table;  // the line's public [nk][L+1] table (expanded into a.taps)
};
struct BatchArgs {
    int nlines, nitems;
    int* counter;                            // work-queue head, zero at launch
    int order[FXMIG_BATCH_MAX_LINES];        // lines in the order their items are handed out
    int item_base[FXMIG_BATCH_MAX_LINES + 1];  // first item (stream) of line order[k]
    BatchLineArgs line[FXMIG_BATCH_MAX_LINES];
};

__device__ __forceinline__ void st_cluster_u32(uint32_t addr, int v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" :: "r"(addr), "r"(v) : "memory");
}

template <int LT>
__device__ __forceinline__ void run_item_lt(const MigrateArgs& a, int g, unsigned char* smem, int part,
                                            bool accumulate) {
    run_group<LT, WsF32, TapF32>(a, g, smem, part, accumulate);
}

__global__ void __launch_bounds__(kBatchWarps * 32, 1) k_migrate_batch(const __grid_constant__ BatchArgs b) {
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
        const int p = item - b.item_base[k];  // the line's stream
        const int g0 = (int)(((long long)p * L.a.G) / L.P), g1 = (int)(((long long)(p + 1) * L.a.G) / L.P);
        for (int g = g0; g < g1; ++g) {
            // the groups of stream p add their rows into partial image p
            // (the line's arguments are read in place from the parameters)
            const bool acc = g > g0;
            switch (L.LT) {
                case 4: run_item_lt<4>(L.a, g, smem, p, acc); break;
                case 8: run_item_lt<8>(L.a, g, smem, p, acc); break;
                case 12: run_item_lt<12>(L.a, g, smem, p, acc); break;
                case 16: run_item_lt<16>(L.a, g, smem, p, acc); break;
                case 17: run_item_lt<17>(L.a, g, smem, p, acc); break;
                case 20: run_item_lt<20>(L.a, g, smem, p, acc); break;
                default: break;
            }
            // the next group reuses the shared memory: every CTA of the
            // cluster has finished this one (write-back included)
            if (C > 1) cluster_sync_all(); else __syncthreads();
        }
        // s_item is rewritten for the next item only after every CTA of the
        // cluster has passed the last group's final barrier (above)
    }
}

// Expand every line's [nk][L+1] table into its kernel layout (TapF32).
__global__ void k_expand_taps_batch(const __grid_constant__ BatchArgs b) {
    for (int li = blockIdx.y; li < b.nlines; li += gridDim.y) {
        const MigrateArgs& a = b.line[li].a;
        const int LT = b.line[li].LT, L = a.L;
        float4* taps = static_cast<float4*>(const_cast<void*>(a.taps));
        const int n = a.nk * (LT + 1);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            const int kk = i / (LT + 1), t = i - kk * (LT + 1);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (t <= L) {
                const float2 h = b.line[li].table[(size_t)kk * (L + 1) + t];
                v = make_float4(h.x, h.x, h.y, h.y);
            }
            taps[i] = v;
        }
    }
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
    int LT, W, lines, G, img;
    size_t smem;
    double cost;  // work of one group: points x frequencies x FP32 operations
};

// Per-line choices for cluster size C and lines-per-group cap (0 = as many
// as fit).  Returns false if some line cannot be planned.
bool plan_line(const fxmig_desc* d, int C, int cap, int smax, LinePlan* p) {
    const int LT = compiled_half_length(d->L);
    if (LT < 0) return false;
    int W = (d->nx + C - 1) / C;
    W = (W + 7) & ~7;
    if (C > 1 && W < LT) return false;
    int fit = 0;
    while (fit < d->nw && persistent_layout(W, fit + 1, LT, 8, false).total <= (size_t)smax) ++fit;
    if (fit == 0) return false;
    int m = cap > 0 ? std::min(cap, fit) : fit;
    const int G = (d->nw + m - 1) / m;
    m = (d->nw + G - 1) / G;  // balanced lines per group
    p->LT = LT;
    p->W = W;
    p->lines = m;
    p->G = G;
    p->img = persistent_layout(W, m, LT, 8, true).total <= (size_t)smax ? 1 : 0;
    p->smem = persistent_layout(W, m, LT, 8, p->img != 0).total;
    p->cost = (double)m * W * C * (double)d->nz * (6.0 * LT + 4.0);
    return true;
}

struct BatchLayout {
    size_t status, taps_off[FXMIG_BATCH_MAX_LINES], scratch, total;
};

// Depth rows of a line that the autotuner runs: an eighth of the line (at
// least 8), so the items keep the proportions of the full run.
int tune_rows(const fxmig_desc& d) { return std::min(d.nz, std::max(8, (d.nz + 7) / 8)); }

// Workspace: status word and queue counter, expanded tables, and
// (autotuner, pmax != nullptr) scratch wavefields and pmax[i] partial images
// of the tuning rows per line.
BatchLayout batch_layout(const fxmig_line* lines, int n, const int* pmax) {
    BatchLayout L = {};
    size_t o = kStatusBytes;
    for (int i = 0; i < n; ++i) {
        const int LT = compiled_half_length(lines[i].d.L);
        L.taps_off[i] = o;
        o += r256((size_t)lines[i].d.nk * (LT + 1) * 16);
    }
    L.scratch = o;
    if (pmax) {
        for (int i = 0; i < n; ++i) {
            const fxmig_desc& d = lines[i].d;
            o += r256((size_t)d.nw * d.nx * 8);                            // wavefield copy
            o += r256((size_t)pmax[i] * tune_rows(d) * d.nx * 4);          // partial rows
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
bool plan_batch(const fxmig_line* lines, int n, const fxmig_batch_plan& plan, std::vector<LinePlan>* lp,
                std::vector<int>* P);

// The autotuner's candidate plans: cluster sizes 1, 2, 4, 8, each with as
// many lines per group as fit and with half of what fits on the widest line.
std::vector<fxmig_batch_plan> tune_candidates(const fxmig_line* lines, int n) {
    std::vector<fxmig_batch_plan> out;
    for (int C : {1, 2, 4, 8}) {
        std::vector<LinePlan> lp;
        std::vector<int> P;
        const fxmig_batch_plan p0 = {C, 0};
        if (!plan_batch(lines, n, p0, &lp, &P)) continue;
        out.push_back(p0);
        int fit_min = 1 << 30;
        for (int i = 0; i < n; ++i) fit_min = std::min(fit_min, lp[i].lines);
        if (fit_min >= 2) out.push_back(fxmig_batch_plan{C, fit_min / 2});
    }
    return out;
}

// Largest stream count of every line over the candidates.
std::vector<int> tune_pmax(const fxmig_line* lines, int n) {
    std::vector<int> pmax(n, 1);
    for (const fxmig_batch_plan& p : tune_candidates(lines, n)) {
        std::vector<LinePlan> lp;
        std::vector<int> P;
        if (!plan_batch(lines, n, p, &lp, &P)) continue;
        for (int i = 0; i < n; ++i) pmax[i] = std::max(pmax[i], P[i]);
    }
    return pmax;
}
}  // namespace

size_t batch_ws_bytes(const fxmig_line* lines, int n, bool scratch) {
    if (!scratch) return batch_layout(lines, n, nullptr).total;
    const std::vector<int> pmax = tune_pmax(lines, n);
    return batch_layout(lines, n, pmax.data()).total;
}

namespace {
// Line plans and stream counts of a batch: about four streams per cluster,
// each line's share in proportion to its work.
bool plan_batch(const fxmig_line* lines, int n, const fxmig_batch_plan& plan, std::vector<LinePlan>* lp,
                std::vector<int>* P) {
    const int C = plan.cluster;
    if (C != 1 && C != 2 && C != 4 && C != 8) return false;
    const int smax = smem_optin();
    lp->assign(n, LinePlan());
    P->assign(n, 1);
    double total = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!plan_line(&lines[i].d, C, plan.lines_cap, smax, &(*lp)[i])) return false;
        total += (*lp)[i].cost * (*lp)[i].G;
    }
    const double target = total / (4.0 * std::max(1, sms_of_device() / C));
    for (int i = 0; i < n; ++i) {
        const double w = (*lp)[i].cost * (*lp)[i].G;
        (*P)[i] = std::max(1, std::min((*lp)[i].G, (int)std::lround(w / target)));
    }
    return true;
}
}  // namespace

int batch_num_partials(const fxmig_line* lines, int n, const fxmig_batch_plan* plan, int* out) {
    fxmig_batch_plan p = {2, 0};
    if (plan) {
        p = *plan;
        if (p.cluster == 0) p.cluster = 2;
    }
    std::vector<LinePlan> lp;
    std::vector<int> P;
    if (!plan_batch(lines, n, p, &lp, &P)) return FXMIG_EINVAL;
    for (int i = 0; i < n; ++i) out[i] = P[i];
    return FXMIG_OK;
}

// Fill the launch arguments for plan; with slabs != nullptr (autotuner)
// every line runs on a scratch wavefield and scratch partial rows over its
// first tune_rows depth rows.
static int fill_args(const fxmig_line* lines, int n, const fxmig_batch_plan& plan, unsigned char* wsb,
                     BatchArgs* b, size_t* smem_max, const std::vector<float2*>* slabs,
                     const std::vector<float*>* partials) {
    const int C = plan.cluster;
    const BatchLayout Lw = batch_layout(lines, n, nullptr);
    std::vector<LinePlan> lp;
    std::vector<int> P;
    if (!plan_batch(lines, n, plan, &lp, &P)) return FXMIG_EINVAL;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    // largest streams first
    auto stream_cost = [&](int i) { return lp[i].cost * lp[i].G / P[i]; };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return stream_cost(x) > stream_cost(y); });
    b->nlines = n;
    b->counter = reinterpret_cast<int*>(wsb + sizeof(int));
    b->item_base[0] = 0;
    *smem_max = 0;
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        b->order[k] = i;
        b->item_base[k + 1] = b->item_base[k] + P[i];
        *smem_max = std::max(*smem_max, lp[i].smem);
        const fxmig_desc& d = lines[i].d;
        MigrateArgs a = {};
        a.nx = d.nx; a.nz = d.nz; a.nw = d.nw; a.nk = d.nk; a.i0 = d.i0; a.nt = d.nt; a.L = d.L;
        a.z_begin = lines[i].z_begin;
        a.z_end = lines[i].z_end;
        a.dt = d.dt;
        a.dk = d.nk > 1 ? d.k_max / (double)(d.nk - 1) : 0.0;
        a.slab = static_cast<float2*>(lines[i].slab);
        a.vel = lines[i].vel;
        a.slow = nullptr;  // slowness rows converted inside the depth loop
        a.taps = wsb + Lw.taps_off[i];
        a.partials = lines[i].partials;
        a.status = reinterpret_cast<int*>(wsb);
        a.W = lp[i].W; a.C = C; a.G = lp[i].G; a.lines = lp[i].lines;
        a.img = lp[i].img;
        a.tma_ok = ((d.nx & 3) == 0) && ((reinterpret_cast<uintptr_t>(lines[i].vel) & 15) == 0);
        if (slabs) {  // autotuner: scratch wavefield and partial rows, first rows
            a.slab = (*slabs)[i];
            a.partials = (*partials)[i];
            a.z_begin = 0;
            a.z_end = tune_rows(d);
            a.nz = a.z_end;  // partial rows are indexed by the scratch's depth count
        }
        b->line[i].a = a;
        b->line[i].LT = lp[i].LT;
        b->line[i].P = P[i];
        b->line[i].table = static_cast<const float2*>(lines[i].table);
    }
    b->nitems = b->item_base[n];
    return FXMIG_OK;
}

static cudaError_t launch_batch_kernel(const BatchArgs& b, size_t smem, int C, int* counter, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    e = ensure_smem(k_migrate_batch, smem, C > 1);
    if (e != cudaSuccess) return e;
    const int clusters = std::max(1, std::min(sms_of_device() / C, b.nitems));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(clusters * C);
    cfg.blockDim = dim3(kBatchWarps * 32);
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

static cudaError_t expand_tables(int n, const BatchArgs& b, cudaStream_t s) {
    k_expand_taps_batch<<<dim3(8, std::min(n, 65535)), 256, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_batch(const fxmig_line* lines, int n, const fxmig_batch_plan& plan, void* ws, cudaStream_t s) {
    unsigned char* wsb = static_cast<unsigned char*>(ws);
    std::vector<BatchArgs> hold(1);  // ~23 KB of launch arguments
    BatchArgs& b = hold[0];
    size_t smem = 0;
    if (fill_args(lines, n, plan, wsb, &b, &smem, nullptr, nullptr) != FXMIG_OK) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(wsb, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    e = expand_tables(n, b, s);
    if (e != cudaSuccess) return e;
    return launch_batch_kernel(b, smem, plan.cluster, b.counter, s);
}

int batch_autotune(const fxmig_line* lines, int n, fxmig_batch_plan* out, void* ws, cudaStream_t s,
                   float* best_ms) {
    unsigned char* wsb = static_cast<unsigned char*>(ws);
    const std::vector<int> pmax = tune_pmax(lines, n);
    const BatchLayout Lw = batch_layout(lines, n, pmax.data());
    // scratch wavefields (copies of the caller's) and partial rows
    std::vector<float2*> slabs(n);
    std::vector<float*> parts(n);
    size_t o = Lw.scratch;
    for (int i = 0; i < n; ++i) {
        const fxmig_desc& d = lines[i].d;
        slabs[i] = reinterpret_cast<float2*>(wsb + o);
        o += r256((size_t)d.nw * d.nx * 8);
        parts[i] = reinterpret_cast<float*>(wsb + o);
        o += r256((size_t)pmax[i] * tune_rows(d) * d.nx * 4);
    }
    const std::vector<fxmig_batch_plan> cands = tune_candidates(lines, n);
    if (cands.empty()) return FXMIG_EINVAL;
    cudaError_t e = cudaMemsetAsync(wsb, 0, sizeof(int), s);
    if (e != cudaSuccess) return FXMIG_ECUDA;
    std::vector<BatchArgs> hold(1);
    BatchArgs& b = hold[0];
    {  // the expanded tables do not depend on the plan
        size_t sm0 = 0;
        if (fill_args(lines, n, cands[0], wsb, &b, &sm0, nullptr, nullptr) != FXMIG_OK) return FXMIG_EINVAL;
        if (expand_tables(n, b, s) != cudaSuccess) return FXMIG_ECUDA;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FXMIG_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FXMIG_ECUDA;
    }
    float best = 1e30f;
    fxmig_batch_plan best_plan = {0, 0};
    for (const fxmig_batch_plan& p : cands) {
        size_t smem = 0;
        if (fill_args(lines, n, p, wsb, &b, &smem, &slabs, &parts) != FXMIG_OK) continue;
        for (int i = 0; i < n && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(slabs[i], lines[i].slab, (size_t)lines[i].d.nw * lines[i].d.nx * 8,
                                cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = launch_batch_kernel(b, smem, p.cluster, b.counter, s);
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
