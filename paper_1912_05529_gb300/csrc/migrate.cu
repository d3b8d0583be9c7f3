// migrate.cu -- depth loop of explicit f-x poststack depth migration
// (Algorithm 1; Eq. 1; Sec. III per-point operator lookup) for sm_103a.
//
// Two forms of the same computation:
//
//  * persistent (one launch): a cluster of C CTAs owns a group of frequency
//    lines; CTA r of the cluster keeps x-segment r of every line of the group
//    in shared memory for ALL depth steps.  Per depth step each CTA
//      - sums Re P over its lines into its partial image row (deterministic),
//      - looks up the operator of every output point (fp32 index, Sec. III),
//      - applies Eq. 1 with symmetric-pair packed f32x2 FMAs,
//      - pushes the L edge outputs into its neighbours' halos (DSMEM),
//    and the cluster barrier replaces the paper's kernel exit (Sec. III, V).
//    The velocity row of the next depth is staged by a 1-D TMA bulk copy
//    while the current depth is computed.
//  * per-depth (one launch per depth step): the wavefield streams through
//    L2/HBM; a CTA computes a 256-point x tile of a frequency tile.
//
// Compute kernel shared by both: a lane produces 8 consecutive outputs of one
// line from a register window of 8 + 2L values read out of shared memory.
// Shared-memory line layout: position p (p = x - x_seg + L) lives at
// p + 2 (p / 8), i.e. groups of 8 complex values padded by 2, so that the
// 16-byte window loads of a warp (lane stride 8 outputs = 80 bytes) hit 32
// distinct banks per quarter warp.
#include <float.h>
#include <math.h>

#include <algorithm>

#include "fxmig_internal.cuh"

namespace fxmig_impl {

int compiled_half_length(int L) {
    static const int kLs[] = {4, 8, 12, 16, 17, 20};
    for (int v : kLs)
        if (v >= L) return v;
    return -1;
}

struct MigrateArgs {
    int nx, nz, nw, nk, z_begin, z_end, i0, nt;
    double dt, dk;
    float2* slab;           // [nw][nx]
    const float* vel;       // [nz][nx]
    const float4* taps;     // [nk][LT+1] as (hr, hr, hi, hi)
    float* partials;        // [G][nz][nx]
    int* status;
    int W, C, G, lines, tma_ok;
    // per-depth form
    const float2* in;
    float2* out;
    int z;
};

__host__ __device__ inline int seg_phys_len(int W, int LT) { return ((W + 2 * LT + 7) >> 3) * 10; }
__host__ __device__ inline int phys(int p) { return p + 2 * (p >> 3); }
__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// q_w = fl32(w / dk), w = 2 pi (i0 + j) / (nt dt), evaluated in FP64 and rounded once.
__device__ __forceinline__ float q_of_line(int i0, int j, int nt, double dt, double dk) {
    const double w = 2.0 * 3.14159265358979323846 * (double)(i0 + j) / ((double)nt * dt);
    return __double2float_rn(w / dk);
}

// Table index of Sec. III: nearest entry, rint_half_even(fl32(q s)), clamped.
__device__ __forceinline__ int table_index(float q, float s, int nk) {
    const int idx = __float2int_rn(__fmul_rn(q, s));
    return min(max(idx, 0), nk - 1);
}

// Eq. 1 for 8 consecutive outputs.  wbase points at the padded position of
// the first window value (x of the first output minus L).  Outputs are
//   out_r = h0 P_r + sum_{n=1}^{L} h_n (P_{r-n} + P_{r+n}),
// accumulated as A = sum hr * (pair) and B = sum hi * (pair) with packed
// (re, im) f32x2 operations, then out = (A.re - B.im, A.im + B.re).
template <int LT>
__device__ __forceinline__ void fir8(const float2* __restrict__ wbase, const float (&s8)[8], float q, int nk,
                                     const float4* __restrict__ taps, u64 (&res)[8], float (&re)[8]) {
    constexpr int NWIN = 8 + 2 * LT;
    u64 w[NWIN];
#pragma unroll
    for (int t = 0; t < NWIN; t += 2) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(wbase + t + 2 * (t >> 3));
        w[t] = v.x;
        w[t + 1] = v.y;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) re[r] = f2_unpack(w[LT + r]).x;
    const float4* tp[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) tp[r] = taps + (size_t)table_index(q, s8[r], nk) * (LT + 1);
    u64 A[8], B[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        u64 hr, hi;
        ldg_nc_v2(tp[r], hr, hi);
        A[r] = f2_mul(hr, w[LT + r]);
        B[r] = f2_mul(hi, w[LT + r]);
    }
#pragma unroll
    for (int n = 1; n <= LT; ++n) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            u64 hr, hi;
            ldg_nc_v2(tp[r] + n, hr, hi);
            const u64 t = f2_add(w[LT + r - n], w[LT + r + n]);
            A[r] = f2_fma(hr, t, A[r]);
            B[r] = f2_fma(hi, t, B[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const float2 a = f2_unpack(A[r]), b = f2_unpack(B[r]);
        res[r] = f2_pack(a.x - b.y, a.y + b.x);
    }
}

// Store 8 outputs at padded positions LT + r relative to the 8-aligned base.
template <int LT>
__device__ __forceinline__ void store8(float2* base, const u64 (&res)[8]) {
    if constexpr ((LT & 1) == 0) {
#pragma unroll
        for (int r = 0; r < 8; r += 2) {
            const int t = LT + r;
            *reinterpret_cast<ulonglong2*>(base + t + 2 * (t >> 3)) = make_ulonglong2(res[r], res[r + 1]);
        }
    } else {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int t = LT + r;
            *reinterpret_cast<u64*>(base + t + 2 * (t >> 3)) = res[r];
        }
    }
}

__device__ __forceinline__ void load_s8(const float* p, float (&s8)[8]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    const float4 b = *reinterpret_cast<const float4*>(p + 4);
    s8[0] = a.x; s8[1] = a.y; s8[2] = a.z; s8[3] = a.w;
    s8[4] = b.x; s8[5] = b.y; s8[6] = b.z; s8[7] = b.w;
}

struct PersistentSmem {
    size_t mbar, qs, vbuf, sbuf, img, wave, total;
};
__host__ __device__ inline PersistentSmem persistent_layout(int W, int lines, int LT) {
    PersistentSmem s;
    s.mbar = 0;
    s.qs = 16;
    s.vbuf = align16(s.qs + 4 * (size_t)lines);
    s.sbuf = s.vbuf + 2 * (size_t)W * 4;
    s.img = s.sbuf + 2 * (size_t)W * 4;
    s.wave = align16(s.img + 2 * (size_t)lines * W * 4);
    s.total = s.wave + 2 * (size_t)lines * seg_phys_len(W, LT) * 8;
    return s;
}

// ------------------------------------------------------------ persistent form
constexpr int kPersistentMaxThreads = 384;  // 12 warps, up to 168 registers per thread

template <int LT>
__global__ void __launch_bounds__(kPersistentMaxThreads, 1) k_migrate_persistent(const MigrateArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int W = a.W, m = a.lines, C = a.C;
    const int SP = seg_phys_len(W, LT);
    const PersistentSmem L = persistent_layout(W, m, LT);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L.mbar);
    float* qs = reinterpret_cast<float*>(smem + L.qs);
    float* vbuf = reinterpret_cast<float*>(smem + L.vbuf);
    float* sbuf = reinterpret_cast<float*>(smem + L.sbuf);
    float* img = reinterpret_cast<float*>(smem + L.img);
    float2* wave = reinterpret_cast<float2*>(smem + L.wave);

    const int rank = (C > 1) ? (int)cluster_ctarank() : 0;
    const int g = blockIdx.x / C;
    const int l_begin = (int)(((long long)g * a.nw) / a.G);
    const int mg = (int)(((long long)(g + 1) * a.nw) / a.G) - l_begin;
    const int x0 = rank * W;
    const int wv = max(0, min(W, a.nx - x0));
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    const int nchunks = (W + 255) >> 8;

    // ---- prologue: zero both wavefield buffers (halos outside [0, nx) stay 0)
    for (int i = tid; i < 2 * m * SP; i += nthr) wave[i] = make_float2(0.f, 0.f);
    for (int s = tid; s < m; s += nthr) qs[s] = (s < mg) ? q_of_line(a.i0, l_begin + s, a.nt, a.dt, a.dk) : 0.f;
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // wavefield at depth z_begin, with halos read from the neighbours' x range
    for (int s = 0; s < mg; ++s) {
        const float2* src = a.slab + (size_t)(l_begin + s) * a.nx;
        float2* dst = wave + (size_t)s * SP;
        for (int pos = tid; pos < W + 2 * LT; pos += nthr) {
            const int x = x0 - LT + pos;
            if (x >= 0 && x < a.nx) dst[phys(pos)] = src[x];
        }
    }

    uint32_t phase = 0;  // bit b: parity of the next wait on mbar[b]
    auto issue_row = [&](int z) {  // thread 0 only
        if (!a.tma_ok) return;
        const int b = z & 1;
        const uint32_t bytes = (uint32_t)wv * 4u;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&mbar[b], bytes);
        if (bytes) bulk_g2s(vbuf + b * W, a.vel + (size_t)z * a.nx + x0, bytes, &mbar[b]);
    };
    auto wait_row = [&](int z) {
        if (!a.tma_ok) return;
        const int b = z & 1;
        if (!mbar_wait_bounded(&mbar[b], (phase >> b) & 1u, kWaitPolls)) {
            if (tid == 0) atomicOr(a.status, kStatusTimeout);
        }
        phase ^= (1u << b);
    };
    auto convert_row = [&](int z) {  // s = fl32(1/v) for the CTA's x segment
        const float* src = a.tma_ok ? (vbuf + (z & 1) * W) : (a.vel + (size_t)z * a.nx + x0);
        float* dst = sbuf + (z & 1) * W;
        bool bad = false;
        for (int x = tid; x < W; x += nthr) {
            float s = 0.f;
            if (x < wv) {
                const float v = src[x];
                bad |= !(v > 0.f && v <= FLT_MAX);
                s = __frcp_rn(v);
            }
            dst[x] = s;
        }
        if (bad) atomicOr(a.status, kStatusVelocity);
    };
    auto reduce_image_row = [&](int zr) {  // partial[g][zr][x0 + x] = sum over lines, ascending
        const float* src = img + (size_t)(zr & 1) * m * W;
        float* dst = a.partials + ((size_t)g * a.nz + zr) * a.nx + x0;
        for (int x = tid * 4; x < wv; x += nthr * 4) {
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int s = 0; s < mg; ++s) {
                const float4 v = *reinterpret_cast<const float4*>(src + (size_t)s * W + x);
                acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
            }
            if (x + 4 <= wv && (a.nx & 3) == 0) {
                *reinterpret_cast<float4*>(dst + x) = acc;
            } else {
                const float t[4] = {acc.x, acc.y, acc.z, acc.w};
                for (int i = 0; i < 4 && x + i < wv; ++i) dst[x + i] = t[i];
            }
        }
    };

    if (tid == 0) {
        issue_row(a.z_begin);
        if (a.z_begin + 1 < a.z_end) issue_row(a.z_begin + 1);
    }
    wait_row(a.z_begin);
    convert_row(a.z_begin);
    // every CTA of the cluster has zeroed its buffers before any halo push
    if (C > 1) cluster_sync_all(); else __syncthreads();

    uint32_t nb_left = 0, nb_right = 0;  // wave base in the neighbours' shared memory
    if (C > 1) {
        if (rank > 0) nb_left = map_cluster_rank(wave, rank - 1);
        if (rank < C - 1) nb_right = map_cluster_rank(wave, rank + 1);
    }

    for (int z = a.z_begin; z < a.z_end; ++z) {
        const int zb = (z - a.z_begin) & 1;
        const float2* cur = wave + (size_t)zb * m * SP;
        float2* nxt = wave + (size_t)(zb ^ 1) * m * SP;
        const size_t nxt_off = (size_t)(zb ^ 1) * m * SP;
        if (z > a.z_begin) reduce_image_row(z - 1);

        const float* srow = sbuf + (z & 1) * W;
        float* imgz = img + (size_t)(z & 1) * m * W;
        for (int task = warp; task < mg * nchunks; task += nwarps) {
            const int s = task / nchunks;
            const int xl0 = (task - s * nchunks) * 256 + lane * 8;
            if (xl0 >= W) continue;
            float s8[8], re[8];
            u64 res[8];
            load_s8(srow + xl0, s8);
            fir8<LT>(cur + (size_t)s * SP + (xl0 >> 3) * 10, s8, qs[s], a.nk, a.taps, res, re);
            *reinterpret_cast<float4*>(imgz + (size_t)s * W + xl0) = make_float4(re[0], re[1], re[2], re[3]);
            *reinterpret_cast<float4*>(imgz + (size_t)s * W + xl0 + 4) = make_float4(re[4], re[5], re[6], re[7]);
#pragma unroll
            for (int r = 0; r < 8; ++r)
                if (xl0 + r >= wv) res[r] = 0ull;
            store8<LT>(nxt + (size_t)s * SP + (xl0 >> 3) * 10, res);
            if (C > 1) {
                if (rank > 0 && xl0 < LT) {
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        const int x = xl0 + r;
                        if (x < LT)
                            st_cluster_v2(nb_left + (uint32_t)((nxt_off + (size_t)s * SP + phys(W + LT + x)) * 8),
                                          f2_unpack(res[r]));
                    }
                }
                if (rank < C - 1 && xl0 + 8 > W - LT) {
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        const int x = xl0 + r;
                        if (x >= W - LT)
                            st_cluster_v2(nb_right + (uint32_t)((nxt_off + (size_t)s * SP + phys(x - W + LT)) * 8),
                                          f2_unpack(res[r]));
                    }
                }
            }
        }
        if (z + 1 < a.z_end) {
            wait_row(z + 1);
            convert_row(z + 1);
        }
        if (tid == 0 && z + 2 < a.z_end) issue_row(z + 2);
        if (C > 1) cluster_sync_all(); else __syncthreads();
    }

    reduce_image_row(a.z_end - 1);
    const float2* fin = wave + (size_t)((a.z_end - a.z_begin) & 1) * m * SP;
    for (int s = 0; s < mg; ++s) {
        float2* dst = a.slab + (size_t)(l_begin + s) * a.nx + x0;
        for (int x = tid; x < wv; x += nthr) dst[x] = fin[(size_t)s * SP + phys(x + LT)];
    }
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
        fir8<LT>(wb + lane * 10, s8, q_of_line(a.i0, l, a.nt, a.dt, a.dk), a.nk, a.taps, res, re);
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
    const size_t slab2 = (size_t)d->nw * d->nx * 8;
    return kStatusBytes + ((taps + 255) & ~size_t(255)) + slab2;
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

int plan_migrate(const fxmig_desc* d, const fxmig_launch* launch, MigratePlan* p) {
    const int LT = compiled_half_length(d->L);
    if (LT < 0) return FXMIG_EINVAL;
    const int mode = (launch && launch->mode) ? launch->mode : FXMIG_MODE_PERSISTENT;
    if (mode != FXMIG_MODE_PERSISTENT && mode != FXMIG_MODE_PER_DEPTH) return FXMIG_EINVAL;
    p->mode = mode;
    p->LT = LT;
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
    const int smax = device_smem_optin();
    const int req_c = (launch && launch->cluster > 0) ? launch->cluster : 0;
    if (req_c && req_c != 1 && req_c != 2 && req_c != 4 && req_c != 8) return FXMIG_EINVAL;
    double best = 1e300;
    bool found = false;
    for (int C : {1, 2, 4, 8}) {
        if (req_c && C != req_c) continue;
        int W = (d->nx + C - 1) / C;
        W = (W + 7) & ~7;
        if (C > 1 && W < LT) continue;
        // frequency groups: one CTA per SM when possible
        int G = (launch && launch->groups > 0) ? launch->groups : std::max(1, sms / C);
        G = std::min(G, std::max(1, d->nw));
        const int lines = (d->nw + G - 1) / G;
        const size_t smem = persistent_layout(W, lines, LT).total;
        if (smem > (size_t)smax) continue;
        const int waves = (G * C + sms - 1) / sms;
        // time model: per-step work of the busiest CTA plus the barrier cost
        // (a cluster barrier costs about as much as ~900 points of work)
        const double t = (double)waves * ((double)lines * W + (C > 1 ? 900.0 : 80.0));
        if (t < best) {
            best = t;
            found = true;
            p->cluster = C;
            p->groups = G;
            p->W = W;
            p->lines = lines;
            p->smem = smem;
            const int tasks = lines * ((W + 255) >> 8);
            int warps = (launch && launch->warps > 0) ? launch->warps : std::min(12, std::max(4, tasks));
            p->warps = std::min(warps, kPersistentMaxThreads / 32);
            p->nparts = G;
        }
    }
    return found ? FXMIG_OK : FXMIG_EINVAL;
}

template <int LT>
static cudaError_t launch_lt(const MigratePlan& plan, MigrateArgs a, cudaStream_t s, float2* ws_slab) {
    if (plan.mode == FXMIG_MODE_PERSISTENT) {
        auto kern = k_migrate_persistent<LT>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
        if (e != cudaSuccess) return e;
        if (plan.cluster > 1) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(plan.groups * plan.cluster);
        cfg.blockDim = dim3(plan.warps * 32);
        cfg.dynamicSmemBytes = plan.smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = plan.cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kern, a);
    }
    auto kern = k_migrate_step<LT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
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
                           cudaStream_t s) {
    const int LT = plan.LT;
    unsigned char* wsb = static_cast<unsigned char*>(ws);
    int* status = reinterpret_cast<int*>(wsb);
    float4* taps = reinterpret_cast<float4*>(wsb + kStatusBytes);
    const size_t taps_bytes = (align16((size_t)d->nk * (LT + 1) * 16) + 255) & ~size_t(255);
    float2* ws_slab = reinterpret_cast<float2*>(wsb + kStatusBytes + taps_bytes);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int n = d->nk * (LT + 1);
    k_expand_taps<<<(n + 255) / 256, 256, 0, s>>>(static_cast<const float2*>(table), d->nk, d->L, LT, taps);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    MigrateArgs a = {};
    a.nx = d->nx; a.nz = d->nz; a.nw = d->nw; a.nk = d->nk;
    a.z_begin = z_begin; a.z_end = z_end; a.i0 = d->i0; a.nt = d->nt;
    a.dt = d->dt;
    a.dk = d->nk > 1 ? d->k_max / (double)(d->nk - 1) : 0.0;
    a.slab = static_cast<float2*>(slab);
    a.vel = vel;
    a.taps = taps;
    a.partials = partials;
    a.status = status;
    a.W = plan.W; a.C = plan.cluster; a.G = plan.groups; a.lines = plan.lines;
    a.tma_ok = ((d->nx & 3) == 0) && ((reinterpret_cast<uintptr_t>(vel) & 15) == 0);
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
