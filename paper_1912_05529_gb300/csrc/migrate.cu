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

#include "fir.cuh"
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
    const float* slow;      // [nz][nx] fl32(1/vel) precomputed, or nullptr (converted in the kernel)
    const float4* taps;     // [nk][LT+1] as (hr, hr, hi, hi)
    float* partials;        // [G][nz][nx]
    int* status;
    int W, C, G, lines, tma_ok;
    int cwarps, ewarps;     // persistent: interior compute warps, edge warps
    // per-depth form
    const float2* in;
    float2* out;
    int z;
};

struct PersistentSmem {
    size_t mbar, qs, vbuf, sbuf, img, wave, total;
};
constexpr int kRowSlots = 7;  // ring of staged slowness/velocity rows
constexpr int kRowAhead = kRowSlots - 1;  // rows are staged this many depth steps ahead
__host__ __device__ inline PersistentSmem persistent_layout(int W, int lines, int LT) {
    PersistentSmem s;
    s.mbar = 0;
    s.qs = 8 * (kRowSlots + 4);  // row-staging barriers, then halo barriers [side][parity]
    s.vbuf = align16(s.qs + 4 * (size_t)lines);
    s.sbuf = s.vbuf + kRowSlots * (size_t)W * 4;
    s.img = s.sbuf + 2 * (size_t)W * 4;
    s.wave = align16(s.img + 2 * (size_t)lines * W * 4);
    s.total = s.wave + 2 * (size_t)lines * seg_phys_len(W, LT) * 8;
    return s;
}

// ------------------------------------------------------------ persistent form
constexpr int kPersistentMaxThreads = 384;  // up to 12 warps: 168 registers per thread

// Per-CTA constants of the persistent kernel.
struct SegCtx {
    int W, SP, wv, rank, C, nk;
    bool has_left, has_right;    // cluster neighbours exist on that side
    uint32_t nb_left, nb_right;  // neighbours' wave base (shared::cluster address)
    // halo barriers of the neighbours that receive this CTA's edge outputs:
    // the left neighbour's right-halo barrier and the right neighbour's
    // left-halo barrier, for the parity of the receiving depth step
    uint32_t bar_left[2], bar_right[2];
};

// Send output x of line s (value v) to the neighbours whose halo holds it.
template <int LT>
__device__ __forceinline__ void push_halo(const SegCtx& g, size_t nxt_off, int s, int x, u64 v, int pb) {
    if (g.has_left && x < LT)
        st_async_v2(g.nb_left + (uint32_t)((nxt_off + (size_t)s * g.SP + phys(g.W + LT + x)) * 8), f2_unpack(v),
                    g.bar_left[pb]);
    if (g.has_right && x >= g.W - LT)
        st_async_v2(g.nb_right + (uint32_t)((nxt_off + (size_t)s * g.SP + phys(x - g.W + LT)) * 8), f2_unpack(v),
                    g.bar_right[pb]);
}

// Write one output (local position x of line s) to the next buffer and, when
// `push` is set and it lies within LT of a segment edge, into the halo of the
// neighbour on that side (st.async, counted on the neighbour's halo barrier
// of parity pb).
template <int LT>
__device__ __forceinline__ void put_output(const SegCtx& g, float2* nxt, size_t nxt_off, int s, int x, u64 v,
                                           bool push, int pb) {
    *reinterpret_cast<u64*>(nxt + (size_t)s * g.SP + phys(x + LT)) = v;
    if (push) push_halo<LT>(g, nxt_off, s, x, v, pb);
}

// One lane item: the 8 outputs of line s at local positions xl0..xl0+7,
// extrapolated with the operator of the first output.  Returns the mask of
// outputs whose own operator differs (the velocity changes inside the 8):
// those are left unwritten for fir1.  The real parts of the current wavefield
// go to the imaging buffer.
template <int LT>
__device__ __forceinline__ uint32_t main_item(const SegCtx& g, int s, int xl0, bool edge, bool push, int pb,
                                              const float2* cur, float2* nxt, size_t nxt_off, const float* srow,
                                              const float* qs, float* imgz, const float4* __restrict__ taps) {
    float s8[8];
    load_s8(srow + xl0, s8);
    const float q = qs[s];
    const int idx0 = table_index(q, s8[0], g.nk);
    uint32_t skip = 0;
    bool same = true;
#pragma unroll
    for (int r = 1; r < 8; ++r) same &= (__float_as_uint(s8[r]) == __float_as_uint(s8[0]));
    if (!same) {
        const int nvalid = min(8, g.wv - xl0);
#pragma unroll
        for (int r = 1; r < 8; ++r)
            if (r < nvalid && table_index(q, s8[r], g.nk) != idx0) skip |= 1u << r;
    }
    u64 res[8];
    float re[8];
    fir8_shared_taps<LT>(cur + (size_t)s * g.SP + (xl0 >> 3) * 10, idx0, taps, res, re);
    *reinterpret_cast<float4*>(imgz + (size_t)s * g.W + xl0) = make_float4(re[0], re[1], re[2], re[3]);
    *reinterpret_cast<float4*>(imgz + (size_t)s * g.W + xl0 + 4) = make_float4(re[4], re[5], re[6], re[7]);
    if (xl0 + 8 > g.wv) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
            if (xl0 + r >= g.wv) res[r] = 0ull;
    }
    if (skip == 0) {
        store8<LT>(nxt + (size_t)s * g.SP + (xl0 >> 3) * 10, res);
        if (edge && push) {
#pragma unroll
            for (int r = 0; r < 8; ++r) push_halo<LT>(g, nxt_off, s, xl0 + r, res[r], pb);
        }
    } else {
#pragma unroll
        for (int r = 0; r < 8; ++r)
            if (!((skip >> r) & 1u)) put_output<LT>(g, nxt, nxt_off, s, xl0 + r, res[r], edge && push, pb);
    }
    return skip;
}

// Warp-cooperative recomputation of the outputs flagged in each lane's
// `mask` (line s, chunk at xl0): the flagged outputs of the whole warp are
// numbered and taken one per lane.  All 32 lanes must call.
template <int LT>
__device__ __forceinline__ void coop_fixups(const SegCtx& g, uint32_t mask, int s, int xl0, const float2* cur,
                                            float2* nxt, size_t nxt_off, const float* srow, const float* qs,
                                            const float4* __restrict__ taps, int lane, bool push, int pb) {
    const uint32_t cnt = __popc(mask);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    const uint32_t excl = incl - cnt;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t it = base + lane;
        int owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int cand = owner + step;
            const uint32_t ex = __shfl_sync(0xffffffffu, excl, cand);
            if (ex <= it) owner = cand;
        }
        const uint32_t ex_o = __shfl_sync(0xffffffffu, excl, owner);
        const uint32_t mask_o = __shfl_sync(0xffffffffu, mask, owner);
        const int s_o = __shfl_sync(0xffffffffu, s, owner);
        const int x0_o = __shfl_sync(0xffffffffu, xl0, owner);
        if (it < total) {
            const int r = (int)__fns(mask_o, 0, (int)(it - ex_o) + 1);
            const int x = x0_o + r;
            const int idx = table_index(qs[s_o], srow[x], g.nk);
            put_output<LT>(g, nxt, nxt_off, s_o, x, fir1<LT>(cur + (size_t)s_o * g.SP, x, idx, taps), push, pb);
        }
    }
}

template <int LT>
__global__ void __launch_bounds__(kPersistentMaxThreads, 1) k_migrate_persistent(const MigrateArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int W = a.W, m = a.lines, C = a.C;
    const int SP = seg_phys_len(W, LT);
    const int NC = W >> 3;
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
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = nthr >> 5;

    // ---- prologue: zero both wavefield buffers (halos outside [0, nx) stay 0)
    for (int i = tid; i < 2 * m * SP; i += nthr) wave[i] = make_float2(0.f, 0.f);
    for (int s = tid; s < m; s += nthr) qs[s] = (s < mg) ? q_of_line(a.i0, l_begin + s, a.nt, a.dt, a.dk) : 0.f;
    uint64_t* hbar = mbar + kRowSlots;  // [side 0 left, 1 right][parity]
    if (tid == 0) {
        for (int b = 0; b < kRowSlots + 4; ++b) mbar_init(&mbar[b], 1);
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

    // Row staging.  Row z of the slowness field (precomputed, a.slow) or of
    // the velocity (converted here) goes through slot z % kRowSlots of vbuf by
    // a 1-D bulk copy, issued kRowAhead depth steps ahead.  The k-th use of a
    // slot completes mbarrier phase k, so row z waits on parity
    // ((z - z_begin) / kRowSlots) & 1; every thread that reads the row waits.
    const float* rows = a.slow ? a.slow : a.vel;
    auto issue_row = [&](int z) {  // one thread
        if (!a.tma_ok) return;
        const int b = z % kRowSlots;
        const uint32_t bytes = (uint32_t)wv * 4u;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&mbar[b], bytes);
        if (bytes) bulk_g2s(vbuf + b * W, rows + (size_t)z * a.nx + x0, bytes, &mbar[b]);
    };
    auto wait_row = [&](int z) {
        if (!a.tma_ok) return;
        const int b = z % kRowSlots;
        if (!mbar_wait_bounded(&mbar[b], (uint32_t)(((z - a.z_begin) / kRowSlots) & 1), kWaitPolls))
            atomicOr(a.status, kStatusTimeout);
    };
    auto srow_of = [&](int z) -> const float* {
        if (a.slow) return a.tma_ok ? (vbuf + (z % kRowSlots) * W) : (a.slow + (size_t)z * a.nx + x0);
        return sbuf + (z & 1) * W;
    };
    // s = fl32(1/v) for the CTA's x segment (only without precomputed slowness)
    auto convert_row = [&](int z) {
        if (a.slow) return;
        const float* src = a.tma_ok ? (vbuf + (z % kRowSlots) * W) : (a.vel + (size_t)z * a.nx + x0);
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
    // partial[g][zr][x0 + x] = sum over the group's lines, ascending
    auto reduce_image_row = [&](int zr) {
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

    if (tid == 0)
        for (int zz = a.z_begin; zz < min(a.z_end, a.z_begin + kRowAhead); ++zz) issue_row(zz);
    wait_row(a.z_begin);
    convert_row(a.z_begin);
    // every CTA of the cluster has zeroed its buffers before any halo push
    if (C > 1) cluster_sync_all(); else __syncthreads();

    SegCtx sc;
    sc.W = W; sc.SP = SP; sc.wv = wv; sc.rank = rank; sc.C = C; sc.nk = a.nk;
    sc.has_left = C > 1 && rank > 0;
    sc.has_right = C > 1 && rank < C - 1;
    sc.nb_left = sc.has_left ? map_cluster_rank(wave, rank - 1) : 0u;
    sc.nb_right = sc.has_right ? map_cluster_rank(wave, rank + 1) : 0u;
    for (int b = 0; b < 2; ++b) {
        sc.bar_left[b] = sc.has_left ? map_cluster_rank(&hbar[2 + b], rank - 1) : 0u;   // its right halo
        sc.bar_right[b] = sc.has_right ? map_cluster_rank(&hbar[b], rank + 1) : 0u;     // its left halo
    }
    // bytes each halo barrier phase receives: LT outputs of every line
    const uint32_t halo_bytes = (uint32_t)mg * LT * 8u;

    // Work items: (line, 8-output chunk), one per lane and round.  Chunks
    // within LT of a segment edge ("edge" chunks) read the halo and send their
    // outputs to the neighbours' halos.  Halo exchange is point to point:
    // outputs go out with st.async, and a CTA waits on its own halo barrier
    // of the step's parity before it reads its halo; neighbours can never be
    // more than one step apart, so two parities suffice and no cluster-wide
    // barrier is needed.  One CTA barrier ends a depth step; the image row of
    // the step is reduced right after it, overlapping the next step's items.
    const int E = (C > 1) ? min((LT + 7) >> 3, NC) : 0;  // edge chunks per side
    const int n_items = mg * NC;

    for (int z = a.z_begin; z < a.z_end; ++z) {
        const int zb = (z - a.z_begin) & 1;
        const float2* cur = wave + (size_t)zb * m * SP;
        float2* nxt = wave + (size_t)(zb ^ 1) * m * SP;
        const size_t nxt_off = (size_t)(zb ^ 1) * m * SP;
        const float* srow = srow_of(z);
        float* imgz = img + (size_t)(z & 1) * m * W;
        const bool push = (C > 1) && (z + 1 < a.z_end);  // outputs feed a further step
        const int pb = (z + 1) & 1;                         // receivers' barrier parity
        const bool halo_wait = (C > 1) && (z > a.z_begin);
        const uint32_t hpar = (uint32_t)(((z - a.z_begin - 1) >> 1) & 1);
        if (tid == 0) {
            // row z+kRowAhead goes to the slot of row z-1, which nobody reads now
            if (z + kRowAhead < a.z_end) issue_row(z + kRowAhead);
            if (halo_wait) {
                if (sc.has_left) mbar_arrive_expect_tx(&hbar[z & 1], halo_bytes);
                if (sc.has_right) mbar_arrive_expect_tx(&hbar[2 + (z & 1)], halo_bytes);
            }
        }
        if (a.slow && z > a.z_begin) wait_row(z);  // (converted rows were synchronised)

        for (int base = warp * 32; base < n_items; base += nwarps * 32) {
            const int item = base + lane;
            int s = 0, xl0 = 0;
            bool work = false, edge = false;
            if (item < n_items) {
                s = item / NC;
                const int c = item - s * NC;
                xl0 = c << 3;
                work = xl0 < wv;
                edge = (C > 1) && (c < E || c >= NC - E);
            }
            if (halo_wait && __any_sync(0xffffffffu, edge)) {
                // the neighbours' outputs of step z-1 have landed in cur's halo
                bool ok = true;
                if (sc.has_left) ok &= mbar_wait_cluster_bounded(&hbar[z & 1], hpar, kHaloPolls);
                if (sc.has_right) ok &= mbar_wait_cluster_bounded(&hbar[2 + (z & 1)], hpar, kHaloPolls);
                if (!ok && lane == 0) atomicOr(a.status, kStatusTimeout);
            }
            uint32_t mask = 0;
            if (work) {
                mask = main_item<LT>(sc, s, xl0, edge, push, pb, cur, nxt, nxt_off, srow, qs, imgz, a.taps);
            } else if (edge && push && item < n_items) {
                // beyond the line end: the neighbours still expect zeros
#pragma unroll
                for (int r = 0; r < 8; ++r) push_halo<LT>(sc, nxt_off, s, xl0 + r, 0ull, pb);
            }
            if (__any_sync(0xffffffffu, mask != 0u))
                coop_fixups<LT>(sc, mask, s, xl0, cur, nxt, nxt_off, srow, qs, a.taps, lane, push, pb);
        }
        if (!a.slow && z + 1 < a.z_end) {
            // velocity rows are converted by the whole CTA before the next step
            wait_row(z + 1);
            convert_row(z + 1);
        }
        __syncthreads();
        reduce_image_row(z);  // img[z & 1] is next written at step z + 2
    }
    // nothing is pushed at the last step and every earlier push has been
    // waited for; the final barrier keeps the CTAs' exits ordered
    if (C > 1) cluster_sync_all(); else __syncthreads();

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
    const int max_warps = kPersistentMaxThreads / 32;
    if (launch && launch->warps > 0 && (launch->warps > max_warps || launch->warps < 1)) return FXMIG_EINVAL;
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
        // work and barriers
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
            p->warps = cw;
            p->cwarps = cw;
            p->ewarps = 0;
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
    const int n = d->nk * (LT + 1);
    k_expand_taps<<<(n + 255) / 256, 256, 0, s>>>(static_cast<const float2*>(table), d->nk, d->L, LT, taps);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const bool use_slow = precompute_slowness && plan.mode == FXMIG_MODE_PERSISTENT;
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
    a.nx = d->nx; a.nz = d->nz; a.nw = d->nw; a.nk = d->nk;
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
    a.cwarps = plan.cwarps; a.ewarps = plan.ewarps;
    a.tma_ok = ((d->nx & 3) == 0) && ((reinterpret_cast<uintptr_t>(use_slow ? (const float*)slow : vel) & 15) == 0);
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
