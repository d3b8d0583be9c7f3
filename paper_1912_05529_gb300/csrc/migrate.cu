// migrate.cu -- depth loop of explicit f-x poststack depth migration
// (Algorithm 1; Eq. 1; Sec. III per-point operator lookup) for sm_103a:
// planning, the per-depth-launch form, and the FP32 persistent form (the
// kernel itself is in persistent.cuh; the 16-bit storage forms are compiled
// in migrate_rp.cu).
//
//  * persistent (one launch): frequency lines stay in shared memory for all
//    depth steps (persistent.cuh).
//  * per-depth (one launch per depth step): the wavefield streams through
//    L2/HBM; a CTA computes a 256-point x tile of a frequency tile.
//
// Compute kernel shared by both: a lane produces 8 consecutive outputs of one
// line from a register window of 8 + 2L values read out of shared memory.
// Shared-memory line layout: position p (p = x - x_seg + L) lives at
// p + 2 (p / 8), i.e. groups of 8 complex values padded by 2, so that the
// window loads of a warp (lane stride 8 outputs = 10 values) hit distinct
// banks.
#include <float.h>
#include <math.h>

#include <algorithm>

#include "fir.cuh"
#include "fxmig_internal.cuh"
#include "persistent.cuh"

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

template <int LT>
__global__ void __launch_bounds__(kStepWarps * 32) k_migrate_step(const MigrateArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int SP = ((kStepTile + 2 * LT + 7) >> 3) * 10;
    float* srow = reinterpret_cast<float*>(smem);                               // [256]
    float* imgw = srow + kStepTile;                                             // [warps][256]
    float2* buf = reinterpret_cast<float2*>(imgw + kStepWarps * kStepTile);     // [warps][SP]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = blockIdx.x * kStepTile;
    const int lb = (int)(((long long)blockIdx.y * a.nw) / a.G);
    const int le = (int)(((long long)(blockIdx.y + 1) * a.nw) / a.G);
    const int z = a.z;
    {
        const int x = x0 + tid;
        float s = 0.f;
        if (x < a.nx) {
            const float v = a.vel[(size_t)z * a.nx + x];
            if (!(v > 0.f && v <= FLT_MAX)) atomicOr(a.status, kStatusVelocity);
            s = __frcp_rn(v);
        }
        srow[tid] = s;
    }
    __syncthreads();
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
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
        fir8<LT>(wb + lane * 10, s8, q_of_line(a.i0, l, a.nt, a.dt, a.dk), a.nk,
                 static_cast<const float4*>(a.taps), res, re);
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[r] += re[r];
        float2* dst = a.out + (size_t)l * a.nx;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int x = x0 + lane * 8 + r;
            if (x < a.nx) dst[x] = f2_unpack(res[r]);
        }
        __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) imgw[warp * kStepTile + lane * 8 + r] = acc[r];
    __syncthreads();
    {
        const int x = x0 + tid;
        if (x < a.nx) {
            float s = 0.f;
            for (int w = 0; w < kStepWarps; ++w) s += imgw[w * kStepTile + tid];
            a.partials[((size_t)blockIdx.y * a.nz + z) * a.nx + x] = s;
        }
    }
}

// Slowness field s = fl32(1/v) of every velocity sample (one pass per call,
// so the depth loop never divides); flags samples that are not finite and > 0.
__global__ void k_slowness(const float* __restrict__ vel, size_t n, float* __restrict__ slow, int* status) {
    bool bad = false;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float v = vel[i];
        bad |= !(v > 0.f && v <= FLT_MAX);
        slow[i] = __frcp_rn(v);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusVelocity);
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

// ------------------------------------------------------------------- host side
size_t migrate_ws_bytes(const fxmig_desc* d) {
    const int LT = compiled_half_length(d->L);
    if (LT < 0) return 0;
    const size_t taps = align16((size_t)d->nk * (LT + 1) * 16);
    const size_t slow = (size_t)d->nz * d->nx * 4;
    const size_t slab2 = (size_t)d->nw * d->nx * 8;
    return kStatusBytes + ((taps + 255) & ~size_t(255)) + ((slow + 255) & ~size_t(255)) + slab2;
}

static int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 148;
}
static int device_smem_optin() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v > 0 ? v : 227 * 1024;
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
    p->mode = mode;
    p->LT = LT;
    p->precision = prec;
    const int sms = device_sms();
    if (mode == FXMIG_MODE_PER_DEPTH) {
        int G = (launch && launch->groups > 0) ? launch->groups : std::max(1, std::min(d->nw, 16));
        G = std::min(G, std::max(1, d->nw));
        p->cluster = 1;
        p->groups = G;
        p->warps = kStepWarps;
        p->W = kStepTile;
        p->lines = (d->nw + G - 1) / G;
        p->smem = (size_t)(kStepTile + kStepWarps * kStepTile) * 4 +
                  (size_t)kStepWarps * (((kStepTile + 2 * LT + 7) >> 3) * 10) * 8;
        p->nparts = G;
        return FXMIG_OK;
    }
    const int esize = prec == FXMIG_PREC_FP32 ? 8 : 4;
    const int smax = device_smem_optin();
    const int req_c = (launch && launch->cluster > 0) ? launch->cluster : 0;
    if (req_c && req_c != 1 && req_c != 2 && req_c != 4 && req_c != 8) return FXMIG_EINVAL;
    const int max_warps = kPersistentMaxWarps;  // compute warps (the edge warp is added at launch)
    if (launch && launch->warps > 0 && (launch->warps > max_warps || launch->warps < 1)) return FXMIG_EINVAL;
    double best = 1e300;
    bool found = false;
    for (int C : {1, 2, 4, 8}) {
        if (req_c && C != req_c) continue;
        int W = (d->nx + C - 1) / C;
        W = (W + 7) & ~7;
        if (C > 1 && W < LT) continue;
        // lines that fit one CTA's shared memory (without imaging buffer)
        int fit = 0;
        while (fit < d->nw && persistent_layout(W, fit + 1, LT, esize, false).total <= (size_t)smax) ++fit;
        if (fit == 0) continue;
        // frequency groups: one CTA per SM when the lines fit, else as many
        // groups (in several waves of CTAs) as the shared memory needs
        int G;
        if (launch && launch->groups > 0) {
            G = std::min(launch->groups, std::max(1, d->nw));
            if ((d->nw + G - 1) / G > fit) continue;
        } else {
            G = std::max(1, sms / C);
            G = std::max(G, (d->nw + fit - 1) / fit);
            G = std::min(G, std::max(1, d->nw));
        }
        const int lines = (d->nw + G - 1) / G;
        // the imaging buffer keeps the image reduction off the critical path;
        // take it whenever the lines still fit with it
        const bool img = persistent_layout(W, lines, LT, esize, true).total <= (size_t)smax;
        const size_t smem = persistent_layout(W, lines, LT, esize, img).total;
        const int waves = (G * C + sms - 1) / sms;
        // lane items: 8 outputs of one line; the warp count with the fewest
        // idle lanes (ties: more warps)
        const long items = (long)lines * (W / 8);
        int cw = 0;
        double eff_best = -1.0;
        for (int c = max_warps; c >= 1; --c) {
            if (launch && launch->warps > 0 && c != launch->warps) continue;
            const long rounds = std::max(1L, (items + 32L * c - 1) / (32L * c));
            const double eff = (double)items / (double)(rounds * 32L * c);
            if (eff > eff_best + 1e-9) { eff_best = eff; cw = c; }
        }
        if (!cw) continue;
        const long rounds = std::max(1L, (items + 32L * cw - 1) / (32L * cw));
        // time per depth step (SM cycles): FP32-pipe work of the busiest CTA
        // (~880 cycles per warp item on one SM sub-partition, 4 per SM),
        // bounded below by one item latency per round, plus the between-step
        // work and barriers; waves of CTAs run one after another
        const double work = (double)items / 32.0 * 880.0 / 4.0;
        const double lat = (double)rounds * 3000.0;
        const double t = (double)waves * (std::max(work, lat) + (C > 1 ? 900.0 : 600.0));
        if (t < best) {
            best = t;
            found = true;
            p->cluster = C;
            p->groups = G;
            p->W = W;
            p->lines = lines;
            p->smem = smem;
            p->img = img ? 1 : 0;
            p->warps = cw;
            p->nparts = G;
        }
    }
    return found ? FXMIG_OK : FXMIG_EINVAL;
}

template <int LT>
static cudaError_t launch_lt(const MigratePlan& plan, MigrateArgs a, cudaStream_t s, float2* ws_slab) {
    if (plan.mode == FXMIG_MODE_PERSISTENT) {
        if (halo_bulk_only<LT>(plan.W, plan.cluster, plan.lines, 8))
            return launch_persistent<LT, WsF32, TapF32, false, true>(plan, a, s);
        return launch_persistent<LT, WsF32, TapF32>(plan, a, s);
    }
    auto kern = k_migrate_step<LT>;
    cudaError_t e = ensure_smem(kern, plan.smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((a.nx + kStepTile - 1) / kStepTile, plan.groups);
    float2* bufs[2] = {a.slab, ws_slab};
    const int nsteps = a.z_end - a.z_begin;
    for (int i = 0; i < nsteps; ++i) {
        a.in = bufs[i & 1];
        a.out = bufs[(i + 1) & 1];
        a.z = a.z_begin + i;
        k_migrate_step<LT><<<grid, kStepWarps * 32, plan.smem, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (nsteps & 1) return cudaMemcpyAsync(a.slab, ws_slab, (size_t)a.nw * a.nx * 8, cudaMemcpyDeviceToDevice, s);
    return cudaSuccess;
}

cudaError_t launch_migrate(const fxmig_desc* d, const MigratePlan& plan, void* slab, const float* vel,
                           const void* table, float* partials, int z_begin, int z_end, void* ws,
                           cudaStream_t s, bool precompute_slowness) {
    const int LT = plan.LT;
    unsigned char* wsb = static_cast<unsigned char*>(ws);
    int* status = reinterpret_cast<int*>(wsb);
    float4* taps = reinterpret_cast<float4*>(wsb + kStatusBytes);
    const size_t taps_bytes = (align16((size_t)d->nk * (LT + 1) * 16) + 255) & ~size_t(255);
    const size_t slow_bytes = ((size_t)d->nz * d->nx * 4 + 255) & ~size_t(255);
    float* slow = reinterpret_cast<float*>(wsb + kStatusBytes + taps_bytes);
    float2* ws_slab = reinterpret_cast<float2*>(wsb + kStatusBytes + taps_bytes + slow_bytes);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (plan.precision == FXMIG_PREC_FP32) {
        const int n = d->nk * (LT + 1);
        k_expand_taps<<<(n + 255) / 256, 256, 0, s>>>(static_cast<const float2*>(table), d->nk, d->L, LT, taps);
        e = cudaGetLastError();
    } else {
        e = expand_taps_rp(plan.precision, static_cast<const float2*>(table), d->nk, d->L, LT, taps, s);
    }
    if (e != cudaSuccess) return e;
    // precomputed slowness rows are read through the TMA ring only (the depth
    // loop's 16-byte row loads need the staged copy): with nx not a multiple
    // of 4 the rows are converted from the velocity in shared memory instead
    const bool use_slow = precompute_slowness && plan.mode == FXMIG_MODE_PERSISTENT && (d->nx & 3) == 0;
    if (use_slow) {
        // only the rows this call reads
        const size_t n_rows = (size_t)(z_end - z_begin) * d->nx;
        const int sms = device_sms();
        size_t blocks = (n_rows + 255) / 256;
        if (blocks > (size_t)sms * 8) blocks = (size_t)sms * 8;
        k_slowness<<<(unsigned)blocks, 256, 0, s>>>(vel + (size_t)z_begin * d->nx, n_rows,
                                                    slow + (size_t)z_begin * d->nx, status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    MigrateArgs a = {};
    a.nx = d->nx; a.nz = d->nz; a.nw = d->nw; a.nk = d->nk; a.L = d->L;
    a.z_begin = z_begin; a.z_end = z_end; a.i0 = d->i0; a.nt = d->nt;
    a.dt = d->dt;
    a.dk = d->nk > 1 ? d->k_max / (double)(d->nk - 1) : 0.0;
    a.slab = static_cast<float2*>(slab);
    a.vel = vel;
    a.slow = use_slow ? slow : nullptr;
    a.taps = taps;
    a.partials = partials;
    a.status = status;
    a.W = plan.W; a.C = plan.cluster; a.G = plan.groups; a.lines = plan.lines;
    a.img = plan.mode == FXMIG_MODE_PERSISTENT ? plan.img : 0;
    a.tma_ok = ((d->nx & 3) == 0) && ((reinterpret_cast<uintptr_t>(use_slow ? (const float*)slow : vel) & 15) == 0);
    if (plan.precision != FXMIG_PREC_FP32) return launch_persistent_rp(plan, a, s);
    switch (LT) {
        case 4: return launch_lt<4>(plan, a, s, ws_slab);
        case 8: return launch_lt<8>(plan, a, s, ws_slab);
        case 12: return launch_lt<12>(plan, a, s, ws_slab);
        case 16: return launch_lt<16>(plan, a, s, ws_slab);
        case 17: return launch_lt<17>(plan, a, s, ws_slab);
        case 20: return launch_lt<20>(plan, a, s, ws_slab);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fxmig_impl
