// mlp_migrate.cu -- depth loop of Algorithm 1 with operators generated by the
// network for the exact slowness of every point (no table quantisation).
//
// The network costs about ten thousand multiply-adds per operator, so it is
// evaluated once per distinct (frequency, slowness) pair of a velocity row,
// not once per point:
//   k_row_unique    per row: sorted distinct values of s = fl32(1/v), their
//                   count, and for every x the index of its value;
//   k_pair_offsets  first (frequency, value) pair of every row (prefix sums
//                   of nw * count);
//   per block of Zc rows: the network writes the operators of all pairs of
//   the block (k_mlp_infer_tc), then the block's depth steps run in the
//   persistent form (depth.cuh: the frequency lines stay in shared memory for
//   the block's rows; the staged rows hold every point's pair index instead
//   of its slowness), or, for lines too wide for it, one Eq. 1 launch per row
//   streams the wavefield through L2/HBM (k_step_pairs, 256 outputs of a
//   frequency tile per CTA, output x of line w using the operator of pair
//   (w, uidx[z][x])).
// Image rows go into the fixed-point accumulator of image.cu.
// Every launch reads its counts from device memory: no host synchronisation.
#include <float.h>

#include <algorithm>

#include "depth.cuh"
#include "fir.cuh"
#include "mlp_internal.cuh"

namespace fxmig_impl {

constexpr int kUniqueThreads = 1024;

// Distinct slowness values of velocity row z_begin + blockIdx.x.  Keys are the
// bit patterns of s = fl32(1/v) (s > 0 for valid velocities, so bit order is
// value order); padding keys 0xffffffff sort last.
// uidx rows have pitch `pitch` (slow_pitch(nx)); the padding repeats the
// row's last index, like the slowness field's.
__global__ void __launch_bounds__(kUniqueThreads) k_row_unique(const float* __restrict__ vel, int nx, int nxp,
                                                               int pitch, int z_begin, float* __restrict__ uval,
                                                               int* __restrict__ uidx, int* __restrict__ cnt,
                                                               int* status) {
    extern __shared__ uint32_t keys[];      // [nxp]
    uint32_t* uniq = keys + nxp;            // [nxp] distinct keys, ascending
    __shared__ int wsum[kUniqueThreads / 32];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int z = z_begin + blockIdx.x;
    const float* v = vel + (size_t)z * nx;
    bool bad = false;
    for (int i = tid; i < nxp; i += nth) {
        uint32_t key = 0xffffffffu;
        if (i < nx) {
            const float vv = v[i];
            bad |= !(vv > 0.f && vv <= FLT_MAX);
            key = __float_as_uint(__frcp_rn(vv));
        }
        keys[i] = key;
    }
    if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(status, kStatusVelocity);
    __syncthreads();
    // bitonic sort, ascending
    for (int k = 2; k <= nxp; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < nxp; i += nth) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint32_t a = keys[i], b = keys[ixj];
                    if ((a > b) == ((i & k) == 0)) {
                        keys[i] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    // first element of every run among the nx sorted keys; block-wide
    // exclusive scan over contiguous chunks of E = nxp / nth elements
    const int E = nxp / nth;
    const int c0 = tid * E;
    int local = 0;
    for (int i = c0; i < c0 + E; ++i) local += (i < nx && (i == 0 || keys[i] != keys[i - 1])) ? 1 : 0;
    int incl = local;
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nwarps = nth >> 5;
        int w = lane < nwarps ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nwarps) wsum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    int pos = incl - local + (warp > 0 ? wsum[warp - 1] : 0);
    for (int i = c0; i < c0 + E; ++i) {
        if (i < nx && (i == 0 || keys[i] != keys[i - 1])) {
            uniq[pos] = keys[i];
            uval[(size_t)z * nx + pos] = __uint_as_float(keys[i]);
            ++pos;
        }
    }
    const int count = wsum[(nth >> 5) - 1];
    if (tid == 0) cnt[z] = count;
    __syncthreads();
    // index of every point's value (exact match by binary search)
    for (int x = tid; x < pitch; x += nth) {
        const uint32_t key = __float_as_uint(__frcp_rn(v[x < nx ? x : nx - 1]));
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (uniq[mid] < key) lo = mid + 1; else hi = mid;
        }
        uidx[(size_t)z * pitch + x] = lo;
    }
}

// base[z] = nw * sum_{z_begin <= z' < z} cnt[z'] for z in [z_begin, z_end].
__global__ void k_pair_offsets(const int* __restrict__ cnt, int nw, int z_begin, int z_end,
                               long long* __restrict__ base) {
    if (threadIdx.x != 0) return;
    long long s = 0;
    for (int z = z_begin; z < z_end; ++z) {
        base[z] = s;
        s += (long long)nw * cnt[z];
    }
    base[z_end] = s;
}

constexpr int kPairWarps = 8;
constexpr int kPairTile = 256;  // x outputs per CTA (32 lanes x 8)

struct PairStepArgs {
    int nx, nz, nw, G, z, z0, pitch;
    const float2* in;
    float2* out;
    const int* uidx;           // [nz][pitch]
    const int* cnt;            // [nz]
    const long long* base;     // [nz+1]
    const float4* taps;        // operators of the block starting at row z0
    unsigned long long* acc;   // [nz][nx] image accumulator
    const int* scale_exp;
    int* status;
};

template <int LT>
__global__ void __launch_bounds__(kPairWarps * 32) k_step_pairs(const PairStepArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int SP = ((kPairTile + 2 * LT + 7) >> 3) * 10;
    int* urow = reinterpret_cast<int*>(smem);                                   // [256]
    long long* imgw = reinterpret_cast<long long*>(urow + kPairTile);           // [warps][256]
    float2* buf = reinterpret_cast<float2*>(imgw + kPairWarps * kPairTile);     // [warps][SP]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = blockIdx.x * kPairTile;
    const int lb = (int)(((long long)blockIdx.y * a.nw) / a.G);
    const int le = (int)(((long long)(blockIdx.y + 1) * a.nw) / a.G);
    const int z = a.z;
    {
        const int x = x0 + tid;
        urow[tid] = x < a.nx ? a.uidx[(size_t)z * a.pitch + x] : 0;
    }
    __syncthreads();
    const int c = a.cnt[z];
    const float4* row_taps = a.taps + (size_t)(a.base[z] - a.base[a.z0]) * (LT + 1);
    // image: every frequency's contribution in fixed point, summed exactly
    long long acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const float scale = depth_scale(*a.scale_exp);
    bool over = false;
    float2* wb = buf + (size_t)warp * SP;
    int u8[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) u8[r] = urow[lane * 8 + r];
    for (int l = lb + warp; l < le; l += kPairWarps) {
        const float2* src = a.in + (size_t)l * a.nx;
        for (int pos = lane; pos < kPairTile + 2 * LT; pos += 32) {
            const int x = x0 - LT + pos;
            wb[phys(pos)] = (x >= 0 && x < a.nx) ? src[x] : make_float2(0.f, 0.f);
        }
        __syncwarp();
        const float4* line_taps = row_taps + (size_t)l * c * (LT + 1);
        const float4* tp[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) tp[r] = line_taps + (size_t)u8[r] * (LT + 1);
        float re[8];
        u64 res[8];
        fir8_ptrs<LT>(wb + lane * 10, tp, res, re);
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
    for (int r = 0; r < 8; ++r) imgw[warp * kPairTile + lane * 8 + r] = acc[r];
    __syncthreads();
    {
        const int x = x0 + tid;
        if (x < a.nx) {
            long long s = 0;
            for (int w = 0; w < kPairWarps; ++w) s += imgw[w * kPairTile + tid];
            if (s) depth_red_add_u64(a.acc + (size_t)z * a.pitch + acc_slot(x), s);
        }
    }
}

// ------------------------------------------------------------------ host side
static int next_pow2(int v) {
    int p = 32;
    while (p < v) p <<= 1;
    return p;
}

int plan_mlp_migrate(const fxmig_desc* d, MlpMigratePlan* p) {
    if (d->L > kMlpMaxL || d->nx > kMlpMaxNx || !(d->k_max > 0)) return FXMIG_EINVAL;
    const int LT = compiled_half_length(d->L);
    if (LT < 0) return FXMIG_EINVAL;
    p->LT = LT;
    // persistent form (pair-index rows staged like slowness rows) when the
    // lines can be planned; one launch per row otherwise
    p->persistent = plan_depth(d, LT, 8, 0, 0, 0, 0, &p->pplan) == FXMIG_OK ? 1 : 0;
    p->groups = p->persistent ? p->pplan.groups : std::max(1, std::min(d->nw, 16));
    p->nparts = image_planes(d->nx);
    // rows per operator block: worst-case operator storage (every point of a
    // row distinct) of about 6 GiB at most, and at most the 64 rows one
    // network launch takes (fewer, longer depth-loop launches)
    const double row_bytes = (double)d->nw * d->nx * (LT + 1) * 16.0;
    p->zc = (int)std::max(1.0, std::min(64.0, std::floor(6.0 * (double)(1u << 30) / row_bytes)));
    return FXMIG_OK;
}

namespace {
struct MlpWs {
    int* head;
    int* uidx;
    float* uval;
    int* cnt;
    long long* base;
    double* norms;
    float4* taps;
    float2* slab2;
    size_t total;
};
size_t r256(size_t v) { return (v + 255) & ~size_t(255); }
MlpWs mlp_ws_layout(const fxmig_desc* d, const MlpMigratePlan& p, void* ws) {
    unsigned char* b = static_cast<unsigned char*>(ws);
    MlpWs w;
    size_t o = kStatusBytes;
    w.head = reinterpret_cast<int*>(b);
    w.uidx = reinterpret_cast<int*>(b + o);
    o += r256((size_t)d->nz * slow_pitch(d->nx) * 4);
    w.uval = reinterpret_cast<float*>(b + o);
    o += r256((size_t)d->nz * d->nx * 4);
    w.cnt = reinterpret_cast<int*>(b + o);
    o += r256((size_t)d->nz * 4);
    w.base = reinterpret_cast<long long*>(b + o);
    o += r256((size_t)(d->nz + 1) * 8);
    w.norms = reinterpret_cast<double*>(b + o);
    o += r256((size_t)d->nw * 8);
    w.taps = reinterpret_cast<float4*>(b + o);
    o += r256((size_t)p.zc * d->nw * d->nx * (p.LT + 1) * 16);
    w.slab2 = reinterpret_cast<float2*>(b + o);
    o += r256((size_t)d->nw * d->nx * 8);
    w.total = o;
    return w;
}
}  // namespace

size_t mlp_migrate_ws_bytes(const fxmig_desc* d) {
    MlpMigratePlan p;
    if (plan_mlp_migrate(d, &p) != FXMIG_OK) return 0;
    return mlp_ws_layout(d, p, nullptr).total;
}

template <int LT>
static cudaError_t launch_pair_steps(const fxmig_desc* d, const MlpMigratePlan& plan, PairStepArgs a, int z0,
                                     int z1, float2* bufs[2], int& parity, cudaStream_t s) {
    const size_t smem = (size_t)kPairTile * 4 + (size_t)kPairWarps * kPairTile * 8 +
                        (size_t)kPairWarps * (((kPairTile + 2 * LT + 7) >> 3) * 10) * 8;
    cudaError_t e = ensure_smem(k_step_pairs<LT>, smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((d->nx + kPairTile - 1) / kPairTile, plan.groups);
    a.z0 = z0;
    for (int z = z0; z < z1; ++z) {
        a.in = bufs[parity];
        a.out = bufs[parity ^ 1];
        a.z = z;
        k_step_pairs<LT><<<grid, kPairWarps * 32, smem, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        parity ^= 1;
    }
    return cudaSuccess;
}

template <int LT>
static cudaError_t launch_pairs(const MigratePlan& pp, const DepthArgs& pa, cudaStream_t s) {
    return launch_depth<LT, WsF32, TapF32, true>(pp, pa, s);
}

cudaError_t launch_mlp_migrate(const fxmig_desc* d, const MlpMigratePlan& plan, void* slab, const float* vel,
                               const float* params, float* partials, int z_begin, int z_end, void* ws,
                               cudaStream_t s) {
    const MlpWs w = mlp_ws_layout(d, plan, ws);
    cudaError_t e = cudaMemsetAsync(w.head, 0, 16, s);
    if (e != cudaSuccess || z_begin == z_end) return e;
    const int nxs = next_pow2(d->nx);
    const int pitch = slow_pitch(d->nx);
    const int nth = std::min(kUniqueThreads, nxs);
    const size_t usmem = (size_t)nxs * 8;
    e = ensure_smem(k_row_unique, usmem);
    if (e != cudaSuccess) return e;
    k_row_unique<<<z_end - z_begin, nth, usmem, s>>>(vel, d->nx, nxs, pitch, z_begin, w.uval, w.uidx, w.cnt,
                                                     w.head);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_pair_offsets<<<1, 32, 0, s>>>(w.cnt, d->nw, z_begin, z_end, w.base);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_image_prep(d, slab, partials, z_begin, z_end, ws, w.norms, s);
    if (e != cudaSuccess) return e;
    PairStepArgs a = {};
    a.nx = d->nx;
    a.nz = d->nz;
    a.nw = d->nw;
    a.G = plan.groups;
    a.pitch = pitch;
    a.uidx = w.uidx;
    a.cnt = w.cnt;
    a.base = w.base;
    a.taps = w.taps;
    a.acc = reinterpret_cast<unsigned long long*>(partials);
    a.scale_exp = w.head + kWsScaleExp;
    a.status = w.head;
    float2* bufs[2] = {static_cast<float2*>(slab), w.slab2};
    int parity = 0;
    DepthArgs pa = {};
    if (plan.persistent) {
        pa.nx = d->nx; pa.nxp = pitch; pa.nz = d->nz; pa.nw = d->nw; pa.nk = d->nk; pa.L = d->L;
        pa.i0 = d->i0; pa.nt = d->nt; pa.dt = d->dt;
        pa.slab = static_cast<float2*>(slab);
        pa.slow = reinterpret_cast<const float*>(w.uidx);  // pair indices, staged like slowness rows
        pa.taps = w.taps;
        pa.acc = reinterpret_cast<unsigned long long*>(partials);
        pa.scale_exp = w.head + kWsScaleExp;
        pa.status = w.head;
        pa.C = plan.pplan.cluster; pa.G = plan.pplan.groups; pa.ncw = plan.pplan.warps; pa.extra = plan.pplan.extra;
        pa.fixw = plan.pplan.fixw;
        pa.pair_cnt = w.cnt;
        pa.pair_base = w.base;
    }
    for (int z0 = z_begin; z0 < z_end; z0 += plan.zc) {
        const int z1 = std::min(z_end, z0 + plan.zc);
        e = launch_mlp_block_taps(d, plan.LT, params, w.uval, w.cnt, w.base, z0, z1, w.taps, s);
        if (e != cudaSuccess) return e;
        if (plan.persistent) {
            pa.z_begin = z0;
            pa.z_end = z1;
            pa.pair_z0 = z0;
            switch (plan.LT) {
                case 4: e = launch_pairs<4>(plan.pplan, pa, s); break;
                case 8: e = launch_pairs<8>(plan.pplan, pa, s); break;
                case 12: e = launch_pairs<12>(plan.pplan, pa, s); break;
                case 16: e = launch_pairs<16>(plan.pplan, pa, s); break;
                default: e = cudaErrorInvalidValue; break;
            }
            if (e != cudaSuccess) return e;
            continue;
        }
        switch (plan.LT) {
            case 4: e = launch_pair_steps<4>(d, plan, a, z0, z1, bufs, parity, s); break;
            case 8: e = launch_pair_steps<8>(d, plan, a, z0, z1, bufs, parity, s); break;
            case 12: e = launch_pair_steps<12>(d, plan, a, z0, z1, bufs, parity, s); break;
            case 16: e = launch_pair_steps<16>(d, plan, a, z0, z1, bufs, parity, s); break;
            default: e = cudaErrorInvalidValue; break;
        }
        if (e != cudaSuccess) return e;
    }
    if (parity) return cudaMemcpyAsync(slab, w.slab2, (size_t)d->nw * d->nx * 8, cudaMemcpyDeviceToDevice, s);
    return cudaSuccess;
}

}  // namespace fxmig_impl
