// persistent.cuh -- the persistent form of the depth loop (Algorithm 1; Eq. 1;
// Sec. III per-point operator lookup), templated on the half-length LT and on
// how the wavefield (WsF32 / WsF16 / WsBF16) and the operator taps
// (TapF32 / TapHalf) are stored.  Arithmetic is FP32 in every form.
//
// A cluster of C CTAs owns a group of frequency lines; CTA r of the cluster
// keeps x-segment r of every line of the group in shared memory for ALL depth
// steps.  Per depth step each CTA
//   - sums Re P over its lines into its partial image row (deterministic),
//   - looks up the operator of every output point (fp32 index, Sec. III),
//   - applies Eq. 1 with symmetric-pair packed f32x2 FMAs: the compute warps
//     take the interior of the segment as 8-output items and never wait on
//     a neighbour; one edge warp waits for the halos, computes the outputs
//     near the segment edges and sends each line's L edge outputs into its
//     neighbours' halos (DSMEM: one bulk copy per strip, st.async around it),
// and one CTA barrier replaces the paper's kernel exit (Sec. III, V).  The
// slowness (or velocity) row of a later depth is staged by a 1-D TMA bulk
// copy while the current depth is computed.
#pragma once

#include <float.h>

#include "fir.cuh"
#include "fxmig_internal.cuh"

namespace fxmig_impl {

struct MigrateArgs {
    int nx, nz, nw, nk, z_begin, z_end, i0, nt, L;
    double dt, dk;
    float2* slab;           // [nw][nx]
    const float* vel;       // [nz][nx]
    const float* slow;      // [nz][nx] fl32(1/vel) precomputed, or nullptr (converted in the kernel)
    const void* taps;       // [nk][LT+1] taps in the kernel's tap layout (TapF32 / TapHalf)
    float* partials;        // [G][nz][nx]
    int* status;
    int W, C, G, lines, tma_ok;
    int img;                // persistent: imaging buffer in shared memory (persistent_layout)
    // operators per (frequency, distinct slowness) pair instead of the table
    // (kPairs): `slow` holds every point's pair index within its row, `taps`
    // the operators of rows [pair_z0, ...) in pair order
    const int* pair_cnt;          // [nz] distinct slowness values of each row
    const long long* pair_base;   // [nz+1] first pair of each row
    int pair_z0;
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
// esize: bytes of one stored wavefield value (8 FP32 complex, 4 half complex).
// img: keep Re P of every line in an imaging buffer [2][lines][W] (reduced
// after the step barrier, off the critical path) instead of summing the
// image row from the wavefield before the barrier; costs 8 W bytes per line.
__host__ __device__ inline PersistentSmem persistent_layout(int W, int lines, int LT, int esize, bool img) {
    PersistentSmem s;
    s.mbar = 0;
    s.qs = 8 * (kRowSlots + 4);  // row-staging barriers, then halo barriers [side][parity]
    s.vbuf = align16(s.qs + 8 * (size_t)lines);  // per-line lookup factors [2][lines]
    s.sbuf = s.vbuf + kRowSlots * (size_t)W * 4;
    s.img = align16(s.sbuf + 2 * (size_t)W * 4);
    s.wave = align16(s.img + (img ? 2 * (size_t)lines * W * 4 : 0));
    s.total = s.wave + 2 * (size_t)lines * seg_phys_len(W, LT) * esize;
    return s;
}

// ------------------------------------------------------------ persistent form
// Outputs per lane of the edge warp: two outputs that share one window, each
// with its own operator (fir2).
constexpr int kEdgeOut = 2;
// Up to 12 compute warps, plus one edge warp when the CTA has cluster
// neighbours: 13 warps, 152 registers per thread.
constexpr int kPersistentMaxWarps = 12;
constexpr int kPersistentMaxThreads = (kPersistentMaxWarps + 1) * 32;

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
template <int LT, class WS>
__device__ __forceinline__ void push_halo(const SegCtx& g, size_t nxt_off, int s, int x, u64 v, int pb) {
    if (g.has_left && x < LT)
        WS::st_async(g.nb_left + (uint32_t)((nxt_off + (size_t)s * g.SP + phys(g.W + LT + x)) * WS::kBytes), v,
                     pb ? g.bar_left[1] : g.bar_left[0]);
    if (g.has_right && x >= g.W - LT)
        WS::st_async(g.nb_right + (uint32_t)((nxt_off + (size_t)s * g.SP + phys(x - g.W + LT)) * WS::kBytes), v,
                     pb ? g.bar_right[1] : g.bar_right[0]);
}

// Operator index of a point with staged row value v: the table entry of
// Sec. III for line factor q (table form), or, with kPairs, the pair index
// line offset + v (v holds the point's distinct-value index).
template <bool kPairs>
__device__ __forceinline__ int op_index(float q, float v, int nk) {
    if constexpr (kPairs) return __float_as_int(q) + __float_as_int(v);
    else return table_index(q, v, nk);
}

// Bring the operator row tp[0..LT] into L1 ahead of its use (the rows of
// operator changes are read by the fixup round after the main item).
template <int LT, class TP>
__device__ __forceinline__ void prefetch_taps(const typename TP::E* tp) {
    constexpr int kBytes = (LT + 1) * (int)sizeof(typename TP::E);
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(tp);
#pragma unroll
    for (int o = 0; o < kBytes + 127; o += 128) {
        const uintptr_t a = (a0 & ~uintptr_t(127)) + (uintptr_t)o;
        if (a < a0 + kBytes) asm volatile("prefetch.global.L1 [%0];" :: "l"(a));
    }
}

// One lane item: the 8 outputs of line s at local positions xl0..xl0+7,
// extrapolated with the operator of the first output.  Returns the mask of
// outputs whose own operator differs (the velocity changes inside the 8):
// the fixup round rewrites those, and their operator rows are prefetched
// into L1 meanwhile; idx1 receives their operator when they all
// share one (the usual single change), else -1.  With an imaging buffer
// (imgz), the real parts of the current wavefield go there.
template <int LT, class WS, class TP, bool kPairs>
__device__ __forceinline__ uint32_t main_item(const SegCtx& g, int s, int xl0, const typename WS::T* cur,
                                              typename WS::T* nxt, const float* srow, const float* qs, float* imgz,
                                              const typename TP::E* __restrict__ taps, int& idx1) {
    float s8[8];
    load_s8(srow + xl0, s8);
    const float q = qs[s];
    const int idx0 = op_index<kPairs>(q, s8[0], g.nk);
    uint32_t skip = 0;
    idx1 = -1;
    bool same = true;
#pragma unroll
    for (int r = 1; r < 8; ++r) same &= (__float_as_uint(s8[r]) == __float_as_uint(s8[0]));
    if (!same) {
        const int nvalid = min(8, g.wv - xl0);
        int last = idx0;
        bool uni = true;
#pragma unroll
        for (int r = 1; r < 8; ++r) {
            const int idx = op_index<kPairs>(q, s8[r], g.nk);
            if (r < nvalid && idx != idx0) {
                uni &= (skip == 0u) || (idx == last);
                skip |= 1u << r;
                if (idx != last) prefetch_taps<LT, TP>(taps + (size_t)idx * (LT + 1));
                last = idx;
            }
        }
        if (uni) idx1 = last;
    }
    u64 res[8];
    float re[8];
    fir8_shared_taps<LT, WS, TP>(cur + (size_t)s * g.SP + (xl0 >> 3) * 10, taps + (size_t)idx0 * (LT + 1), res,
                                 re);
    if (imgz) {  // real parts of the step's input, for the imaging buffer
        *reinterpret_cast<float4*>(imgz + (size_t)s * g.W + xl0) = make_float4(re[0], re[1], re[2], re[3]);
        *reinterpret_cast<float4*>(imgz + (size_t)s * g.W + xl0 + 4) = make_float4(re[4], re[5], re[6], re[7]);
    }
    if (xl0 + 8 > g.wv) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
            if (xl0 + r >= g.wv) res[r] = 0ull;
    }
    // all 8 outputs: those whose own operator differs (skip) are rewritten by
    // the fixup round, which a __syncwarp orders after these stores
    store8<LT, WS>(nxt + (size_t)s * g.SP + (xl0 >> 3) * 10, res);
    return skip;
}

// Position of the n-th set bit (n >= 1, counted from bit 0) of m, which
// has at least n set bits: a binary search on population counts, five
// fixed steps.
__device__ __forceinline__ int nth_set_bit(uint32_t m, int n) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (n > c) {
            n -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// Warp-cooperative recomputation of the outputs flagged in each lane's
// `mask` (line s, chunk at xl0; bit 0 is never set): the flagged outputs of
// the whole warp are numbered by output position r, then by lane, from one
// ballot per position, and taken one per lane.  idx1 is the owner's common
// operator of its flagged outputs (main_item), or -1 to look each one up.
// All 32 lanes must call.
template <int LT, class WS, class TP, bool kPairs>
__device__ __forceinline__ void coop_fixups(const SegCtx& g, uint32_t mask, int s, int xl0, int idx1,
                                            const typename WS::T* cur, typename WS::T* nxt, const float* srow,
                                            const float* qs, const typename TP::E* __restrict__ taps, int lane) {
    uint32_t bal[8];
    int pre[8];
    int total = 0;
#pragma unroll
    for (int r = 1; r < 8; ++r) {
        bal[r] = __ballot_sync(0xffffffffu, (mask >> r) & 1u);
        pre[r] = total;
        total += __popc(bal[r]);
    }
    for (int base = 0; base < total; base += 32) {
        const int it = base + lane;
        // position r of output number it: the last r whose numbering starts
        // at or before it (a position with no outputs shares its start with
        // the next one, so the last such r has it inside its range)
        int r = 1;
        uint32_t br = bal[1];
        int pr = pre[1];
#pragma unroll
        for (int q = 2; q < 8; ++q)
            if (pre[q] <= it) { r = q; br = bal[q]; pr = pre[q]; }
        const int owner = it < total ? nth_set_bit(br, it - pr + 1) : 0;
        const int s_o = __shfl_sync(0xffffffffu, s, owner);
        const int x0_o = __shfl_sync(0xffffffffu, xl0, owner);
        const int i1_o = __shfl_sync(0xffffffffu, idx1, owner);
        if (it < total) {
            const int x = x0_o + r;
            const int idx = i1_o >= 0 ? i1_o : op_index<kPairs>(qs[s_o], srow[x], g.nk);
            WS::st1(nxt + (size_t)s_o * g.SP + phys(x + LT),
                    fir1<LT, WS, TP>(cur + (size_t)s_o * g.SP, x, taps + (size_t)idx * (LT + 1)));
        }
    }
}

// Halo strips of one line in the padded layout, pads included.  The left
// strip holds outputs x in [0, LT) at slots [phys(LT), phys(2LT-1)] and
// lands phys(W) slots further on in the left neighbour's right halo; the
// right strip holds x in [W-LT, W) at slots phys(W) + [0, phys(LT-1)] and
// lands at slot 0 of the right neighbour's line (W a multiple of 8, so the
// pad pattern is the same on both sides).
template <int LT>
struct HaloStrips {
    static constexpr int kLeft0 = LT + 2 * (LT >> 3);
    static constexpr int kLeftN = (2 * LT - 1) + 2 * ((2 * LT - 1) >> 3) + 1 - kLeft0;
    static constexpr int kRightN = (LT - 1) + 2 * ((LT - 1) >> 3) + 1;
};

// Whether the halos go as whole strips (one per line and side, sent by the
// edge warp once the line's edge outputs are in shared memory): segments of
// whole 8-output chunks whose padded line length keeps a strip and its
// landing place at the same 16-byte alignment.  Otherwise every halo output
// goes by its own st.async.
__host__ __device__ inline bool halo_strips(int W, int C, int esize) {
    return C > 1 && (W & 7) == 0 && ((W + 2 * (W >> 3)) * esize) % 16 == 0;
}
// Halos of a launch arrive entirely by bulk copies (FP32 values, whole
// strips of an even number of slots at even slots): their bytes are written
// by the async proxy and complete on the receiving CTA's mbarrier, so a
// CTA-scope acquire on that barrier suffices (as for any bulk copy into a
// CTA's shared memory).  Otherwise st.async bytes, whose complete_tx
// releases at cluster scope, need a cluster-scope acquire.
template <int LT>
inline bool halo_bulk_only(int W, int C, int lines, int esize) {
    typedef HaloStrips<LT> HS;
    (void)lines;
    if (esize != 8 || !halo_strips(W, C, esize)) return false;
    return HS::kLeft0 % 2 == 0 && HS::kLeftN % 2 == 0 && HS::kRightN % 2 == 0;
}

// Send slots [0, n) of a strip from this CTA's shared memory (src) to the
// neighbour's (dst, shared::cluster), counted on the neighbour's mbarrier.
// src and dst have the same address modulo 16 bytes: the 16-byte aligned
// middle goes as one bulk copy (the copy engine moves it; the thread does not
// wait), the slots before and after it by st.async.  The caller has fenced
// the strip's shared-memory writes for the async proxy.
template <class WS>
__device__ __forceinline__ void send_strip(uint32_t dst, const typename WS::T* src, int n, uint32_t bar) {
    constexpr int kB = WS::kBytes;
    const int head = min(n, (int)(((16u - (smem_u32(src) & 15u)) & 15u) / kB));
    const int body = ((n - head) * kB / 16) * 16 / kB;
    for (int i = 0; i < head; ++i) WS::st_async(dst + (uint32_t)(i * kB), WS::ld1(src + i), bar);
    if (body > 0) bulk_s2cluster(dst + (uint32_t)(head * kB), src + head, (uint32_t)(body * kB), bar);
    for (int i = head + body; i < n; ++i) WS::st_async(dst + (uint32_t)(i * kB), WS::ld1(src + i), bar);
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(smem_u32(bar)) : "memory");
}

// The whole depth loop of frequency group g of problem a, on the CTAs of one
// cluster (all of them call it with the same arguments).  smem is the CTA's
// dynamic shared memory (persistent_layout).  The group's image rows go to
// partial image `part`, added to what it holds when `accumulate` is set.  On return every mbarrier used
// is invalidated and no copy or remote store is in flight, so the memory can
// hold the next group.
// kCtaHalo: the launch's halos arrive by bulk copies only (halo_bulk_only),
// so the halo waits acquire at CTA scope.
template <int LT, class WS, class TP, bool kPairs = false, bool kCtaHalo = false>
__device__ __forceinline__ void run_group(const MigrateArgs& a, int g, unsigned char* smem, int part,
                                          bool accumulate) {
    typedef typename WS::T T;
    const typename TP::E* __restrict__ taps_all = static_cast<const typename TP::E*>(a.taps);
    const int W = a.W, m = a.lines, C = a.C;
    const int SP = seg_phys_len(W, LT);
    const int NC = W >> 3;
    const PersistentSmem L = persistent_layout(W, m, LT, WS::kBytes, a.img != 0);
    float* img = a.img ? reinterpret_cast<float*>(smem + L.img) : nullptr;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L.mbar);
    float* qs = reinterpret_cast<float*>(smem + L.qs);
    float* vbuf = reinterpret_cast<float*>(smem + L.vbuf);
    float* sbuf = reinterpret_cast<float*>(smem + L.sbuf);
    T* wave = reinterpret_cast<T*>(smem + L.wave);

    const int rank = (C > 1) ? (int)cluster_ctarank() : 0;
    const int l_begin = (int)(((long long)g * a.nw) / a.G);
    const int mg = (int)(((long long)(g + 1) * a.nw) / a.G) - l_begin;
    const int x0 = rank * W;
    const int wv = max(0, min(W, a.nx - x0));
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = nthr >> 5;

    // ---- prologue: zero both wavefield buffers (halos outside [0, nx) stay 0)
    for (int i = tid; i < 2 * m * SP; i += nthr) wave[i] = WS::zero();
    // per-line lookup factors: the table factor q_w (constant), or with
    // kPairs the line's pair offset in the row, (line) x (distinct values of
    // the row), refreshed one step ahead in qs[(z & 1) * m + s]
    auto pair_offsets = [&](int z, float* dst) {
        const int cnt = a.pair_cnt[z];
        for (int s = tid; s < m; s += nthr) dst[s] = __int_as_float((s < mg) ? (l_begin + s) * cnt : 0);
    };
    if constexpr (kPairs) {
        pair_offsets(a.z_begin, qs + (a.z_begin & 1) * m);
    } else {
        for (int s = tid; s < m; s += nthr) qs[s] = (s < mg) ? q_of_line(a.i0, l_begin + s, a.nt, a.dt, a.dk) : 0.f;
    }
    uint64_t* hbar = mbar + kRowSlots;  // [side 0 left, 1 right][parity]
    if (tid == 0) {
        for (int b = 0; b < kRowSlots + 4; ++b) mbar_init(&mbar[b], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // wavefield at depth z_begin, with halos read from the neighbours' x range
    for (int s = 0; s < mg; ++s) {
        const float2* src = a.slab + (size_t)(l_begin + s) * a.nx;
        T* dst = wave + (size_t)s * SP;
        for (int pos = tid; pos < W + 2 * LT; pos += nthr) {
            const int x = x0 - LT + pos;
            if (x >= 0 && x < a.nx) dst[phys(pos)] = WS::from_f2(src[x]);
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
    // the row the items read (16-byte loads): the staged slowness row, or the
    // converted row in sbuf (precomputed slowness is only passed with tma_ok)
    auto srow_of = [&](int z) -> const float* {
        if (a.slow) return vbuf + (z % kRowSlots) * W;
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
    // partial[g][z][x0 + x] = sum over the group's lines (ascending) of Re P at
    // depth z, by threads t = 0..nt-1: from the imaging buffer after the step
    // barrier, or (no buffer) from the step's input wavefield, which nobody
    // writes during the step, before the barrier
    auto reduce_image_row = [&](int z, const T* cur, int t, int nt) {
        float* dst = a.partials + ((size_t)part * a.nz + z) * a.nx + x0;
        if (img) {
            const float* src = img + (size_t)(z & 1) * m * W;
            for (int x = t * 4; x < wv; x += nt * 4) {
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int s = 0; s < mg; ++s) {
                    const float4 v = *reinterpret_cast<const float4*>(src + (size_t)s * W + x);
                    acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
                }
                if (x + 4 <= wv && (a.nx & 3) == 0) {
                    if (accumulate) {
                        const float4 o = *reinterpret_cast<const float4*>(dst + x);
                        acc.x += o.x; acc.y += o.y; acc.z += o.z; acc.w += o.w;
                    }
                    *reinterpret_cast<float4*>(dst + x) = acc;
                } else {
                    for (int i = 0; i < 4 && x + i < wv; ++i) {
                        const float t = i == 0 ? acc.x : i == 1 ? acc.y : i == 2 ? acc.z : acc.w;
                        dst[x + i] = accumulate ? dst[x + i] + t : t;
                    }
                }
            }
        } else {
            for (int x = t; x < wv; x += nt) {
                float acc = 0.f;
                for (int s = 0; s < mg; ++s) acc += WS::to_f2(cur[(size_t)s * SP + phys(x + LT)]).x;
                dst[x] = accumulate ? dst[x] + acc : acc;
            }
        }
    };

    if (tid == 0)
        for (int zz = a.z_begin; zz < min(a.z_end, a.z_begin + kRowAhead); ++zz) issue_row(zz);
    wait_row(a.z_begin);
    convert_row(a.z_begin);
    // From here on one thread waits for each staged row, one step before the
    // row is read, and the step barrier publishes it to the CTA: row z + 1
    // (slowness rows, read by the items of step z + 1) or row z + 2 (velocity
    // rows, converted during step z + 1) is waited for before the barrier
    // that ends step z.
    if (!a.slow && tid == 0 && a.z_begin + 1 < a.z_end) wait_row(a.z_begin + 1);
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
    // Warps.  With cluster neighbours (C > 1) the last warp is the edge warp:
    // it alone reads the halos and computes the outputs within E chunks of a
    // segment edge that has a neighbour (the "edge" chunks), two outputs per
    // lane, each with its own operator, and sends them to the neighbours'
    // halos as soon as they are in shared memory.  The other (compute) warps
    // take every other chunk as 8-output items and never wait on a halo, so
    // the halo exchange is one short item plus the DSMEM latency per step,
    // off the compute warps' path.
    const bool edges = C > 1;
    const int ncw = edges ? nwarps - 1 : nwarps;  // compute warps
    const bool edge_warp = edges && warp == nwarps - 1;
    // The thread that stages the velocity rows, arms the halo barriers and
    // waits for each staged row: lane 0 of the edge warp, which has that
    // time while it waits for the halos (else thread 0).
    const bool duty = edges ? (edge_warp && lane == 0) : tid == 0;
    // Halo strips: one per line and side with a neighbour, sent whole by the
    // edge warp (pads included; the 16-byte aligned middle as a bulk copy,
    // the slots around it by st.async), or one st.async per output when the
    // padded line length breaks the strip alignment (halo_strips).
    typedef HaloStrips<LT> HS;
    const int physW = W + 2 * (W >> 3);
    const bool strips = halo_strips(W, C, WS::kBytes);
    const uint32_t kB = (uint32_t)WS::kBytes;

    // Edge chunks of a line: c < EL on the left and c >= NC - NR on the
    // right (E = ceil(LT / 8) chunks per side, fewer on the right when the
    // segment holds fewer than 2E chunks).  Only they read the halo (the
    // window of chunk c spans outputs 8c - LT .. 8c + 7 + LT) and only they
    // feed the neighbours' halos (outputs x < LT or x >= W - LT).  Halo
    // exchange is point to point: a CTA waits on its own halo barrier of the
    // step's parity before its edge warp reads the halo; neighbours can never
    // be more than one step apart (the edge warp's wait precedes the step
    // barrier), so two parities suffice and no cluster-wide barrier is
    // needed.  One CTA barrier ends a depth step; the image row of the step
    // is summed right after it from the imaging buffer, or without that
    // buffer just before it from the step's input wavefield.
    const int E = (C > 1) ? min((LT + 7) >> 3, NC) : 0;
    const int EL = sc.has_left ? E : 0;
    const int NR = sc.has_right ? min(E, NC - EL) : 0;
    const int n_items = mg * NC;
    // item / NC by a multiply-high with m = ceil(2^32 / NC): exact while
    // item * NC < 2^32, which n_items * NC < 2^32 guarantees; m fits 32 bits
    // only for NC >= 2 (NC = 1 divides exactly)
    const uint32_t nc_magic = (uint32_t)((0xffffffffull + (uint64_t)NC) / (uint64_t)NC);
    const bool magic_ok = NC >= 2 && (uint64_t)n_items * (uint64_t)NC < (1ull << 32);
    const bool spread = (NC & 31) == 0;  // lines of whole warps of items
    // Bytes each halo barrier phase receives: per line the neighbour's strip
    // (pads included) or its LT outputs.
    const uint32_t halo_bytes_l = (uint32_t)mg * (strips ? (uint32_t)HS::kRightN * kB : (uint32_t)LT * kB);
    const uint32_t halo_bytes_r = (uint32_t)mg * (strips ? (uint32_t)HS::kLeftN * kB : (uint32_t)LT * kB);
    // line s and chunk c of a compute item.  With `spread`, a warp's 32 items
    // of a line, j = 32a + 8q + r, take chunk 8 (q NC/32 + a) + r, so each
    // warp covers four blocks of 8 chunks a quarter of the line apart
    // (velocity changes, which cost extra work, are shared between warps); a
    // quarter-warp keeps 8 consecutive chunks (conflict-free window loads).
    auto item_chunk = [&](int item, int& s, int& c) {
        s = magic_ok ? (int)__umulhi((uint32_t)item, nc_magic) : item / NC;
        const int j = item - s * NC;
        c = spread ? ((((j >> 3) & 3) * (NC >> 5) + (j >> 5)) << 3) + (j & 7) : j;
    };
    // A compute lane's item of a round: line s, first output xl0, and whether
    // it has work (an interior chunk that starts inside the segment; edge
    // chunks belong to the edge warp).
    auto item_state = [&](int item, int& s, int& xl0, bool& work) {
        s = 0;
        xl0 = 0;
        work = false;
        if (item >= n_items) return;
        int c;
        item_chunk(item, s, c);
        xl0 = c << 3;
        work = xl0 < wv && c >= EL && c < NC - NR;
    };
    // the first round's item is the same at every step
    int s_first, xl0_first;
    bool work_first;
    item_state(warp * 32 + lane, s_first, xl0_first, work_first);
    // The edge warp's lanes: kEdgeOut outputs each, the edge chunks of a
    // line on consecutive lanes, in rounds of 32.
    const int e_per_line = 8 * (EL + NR) / kEdgeOut;  // edge lane units per line
    const int e_units = mg * e_per_line;

    for (int z = a.z_begin; z < a.z_end; ++z) {
        const int zb = (z - a.z_begin) & 1;
        const T* cur = wave + (size_t)zb * m * SP;
        T* nxt = wave + (size_t)(zb ^ 1) * m * SP;
        const float* qz = kPairs ? qs + (z & 1) * m : qs;
        const typename TP::E* __restrict__ taps =
            kPairs ? taps_all + (size_t)(a.pair_base[z] - a.pair_base[a.pair_z0]) * (LT + 1) : taps_all;
        float* imgz = img ? img + (size_t)(z & 1) * m * W : nullptr;
        const size_t nxt_off = (size_t)(zb ^ 1) * m * SP;
        const float* srow = srow_of(z);
        const bool push = (C > 1) && (z + 1 < a.z_end);  // outputs feed a further step
        const int pb = (z + 1) & 1;                         // receivers' barrier parity
        const bool halo_wait = (C > 1) && (z > a.z_begin);
        const uint32_t hpar = (uint32_t)(((z - a.z_begin - 1) >> 1) & 1);
        if (duty) {
            // row z+kRowAhead goes to the slot of row z-1, which nobody reads now
            if (z + kRowAhead < a.z_end) issue_row(z + kRowAhead);
            if (halo_wait) {
                if (sc.has_left) mbar_arrive_expect_tx(&hbar[z & 1], halo_bytes_l);
                if (sc.has_right) mbar_arrive_expect_tx(&hbar[2 + (z & 1)], halo_bytes_r);
            }
        }

        if (edge_warp) {
            if (halo_wait) {
                // the neighbours' outputs of step z-1 have landed in cur's halo
                bool ok = true;
                if constexpr (kCtaHalo) {
                    if (sc.has_left) ok &= mbar_wait_bounded(&hbar[z & 1], hpar, kHaloPolls);
                    if (sc.has_right) ok &= mbar_wait_bounded(&hbar[2 + (z & 1)], hpar, kHaloPolls);
                } else {
                    if (sc.has_left) ok &= mbar_wait_cluster_bounded(&hbar[z & 1], hpar, kHaloPolls);
                    if (sc.has_right) ok &= mbar_wait_cluster_bounded(&hbar[2 + (z & 1)], hpar, kHaloPolls);
                }
                if (!ok && lane == 0) atomicOr(a.status, kStatusTimeout);
            }
            for (int u0 = 0; u0 < e_units; u0 += 32) {
                const int u = u0 + lane;
                if (u < e_units) {
                    const int s = u / e_per_line;
                    const int rem = u - s * e_per_line;
                    const int k = rem / (8 / kEdgeOut);
                    const int c = k < EL ? k : NC - NR + (k - EL);
                    const int x = 8 * c + kEdgeOut * (rem & (8 / kEdgeOut - 1));
                    const float q = qz[s];
                    const T* cl = cur + (size_t)s * SP;
                    T* dl = nxt + (size_t)s * SP;
                    u64 o0 = 0ull, o1 = 0ull;
                    float re0 = 0.f, re1 = 0.f;
                    if (x < wv) {
                        const int i0 = op_index<kPairs>(q, srow[x], a.nk);
                        const int i1 = x + 1 < wv ? op_index<kPairs>(q, srow[x + 1], a.nk) : i0;
                        fir2<LT, WS, TP>(cl, x, taps + (size_t)i0 * (LT + 1), taps + (size_t)i1 * (LT + 1), o0,
                                         o1, re0, re1);
                        if (x + 1 >= wv) o1 = 0ull;
                    }
                    WS::st1(dl + phys(x + LT), o0);
                    WS::st1(dl + phys(x + 1 + LT), o1);
                    if (imgz) *reinterpret_cast<float2*>(imgz + (size_t)s * W + x) = make_float2(re0, re1);
                    if (push && !strips) {
                        push_halo<LT, WS>(sc, nxt_off, s, x, o0, pb);
                        push_halo<LT, WS>(sc, nxt_off, s, x + 1, o1, pb);
                    }
                }
            }
            if (push && strips) {
                // the edge outputs are in nxt; make them visible to the copy
                // engine, then send each strip whole, one (line, side) per
                // lane.  Every side with a neighbour sends its strip (a
                // segment of fewer than 2E chunks counts its chunks once, as
                // left-edge chunks, but still feeds both sides).
                fence_proxy_async_smem();
                __syncwarp();
                for (int j = lane; j < 2 * mg; j += 32) {
                    const int s = j >> 1;
                    const uint32_t line = (uint32_t)(nxt_off + (size_t)s * SP);
                    if ((j & 1) == 0 && sc.has_left)
                        send_strip<WS>(sc.nb_left + (line + physW + HS::kLeft0) * kB, nxt + (size_t)s * SP + HS::kLeft0,
                                       HS::kLeftN, pb ? sc.bar_left[1] : sc.bar_left[0]);
                    if ((j & 1) == 1 && sc.has_right)
                        send_strip<WS>(sc.nb_right + line * kB, nxt + (size_t)s * SP + physW, HS::kRightN,
                                       pb ? sc.bar_right[1] : sc.bar_right[0]);
                }
            }
        } else {
            for (int base = warp * 32; base < n_items; base += ncw * 32) {
                int s, xl0;
                bool work;
                if (base == warp * 32) {
                    s = s_first;
                    xl0 = xl0_first;
                    work = work_first;
                } else {
                    item_state(base + lane, s, xl0, work);
                }
                uint32_t mask = 0;
                int idx1 = -1;
                if (work) mask = main_item<LT, WS, TP, kPairs>(sc, s, xl0, cur, nxt, srow, qz, imgz, taps, idx1);
                if (__any_sync(0xffffffffu, mask != 0u)) {
                    __syncwarp();  // the main items' stores precede the fixups' rewrites
                    coop_fixups<LT, WS, TP, kPairs>(sc, mask, s, xl0, idx1, cur, nxt, srow, qz, taps, lane);
                }
            }
        }
        // velocity rows are converted by the whole CTA one step ahead
        if (!a.slow && z + 1 < a.z_end) convert_row(z + 1);
        if constexpr (kPairs) {
            if (z + 1 < a.z_end) pair_offsets(z + 1, qs + ((z + 1) & 1) * m);
        }
        {
            const int zw = a.slow ? z + 1 : z + 2;
            if (duty && zw < a.z_end) wait_row(zw);
        }
        if (!img) reduce_image_row(z, cur, tid, nthr);
        __syncthreads();
        // img[z & 1] is next written at step z + 2; the last row is summed
        // after the final barrier
        if (img && z + 1 < a.z_end) reduce_image_row(z, cur, tid, nthr);
    }
    // nothing is pushed at the last step and every earlier push has been
    // waited for; the final barrier keeps the CTAs' exits ordered
    if (C > 1) cluster_sync_all(); else __syncthreads();
    if (img && a.z_end > a.z_begin) reduce_image_row(a.z_end - 1, nullptr, tid, nthr);
    if (tid == 0)
        for (int b = 0; b < kRowSlots + 4; ++b) mbar_inval(&mbar[b]);

    const T* fin = wave + (size_t)((a.z_end - a.z_begin) & 1) * m * SP;
    for (int s = 0; s < mg; ++s) {
        float2* dst = a.slab + (size_t)(l_begin + s) * a.nx + x0;
        for (int x = tid; x < wv; x += nthr) dst[x] = WS::to_f2(fin[(size_t)s * SP + phys(x + LT)]);
    }
}

// One launch of the persistent form: cluster blockIdx.x / C runs group
// blockIdx.x / C of the problem.
template <int LT, class WS, class TP, bool kPairs = false, bool kCtaHalo = false>
__global__ void __launch_bounds__(kPersistentMaxThreads, 1) k_migrate_persistent(const MigrateArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int g = (int)(blockIdx.x / a.C);
    run_group<LT, WS, TP, kPairs, kCtaHalo>(a, g, smem, g, false);
}


// One launch of the persistent form for compiled LT and storage policies.
template <int LT, class WS, class TP, bool kPairs = false, bool kCtaHalo = false>
cudaError_t launch_persistent(const MigratePlan& plan, const MigrateArgs& a, cudaStream_t s) {
    auto kern = k_migrate_persistent<LT, WS, TP, kPairs, kCtaHalo>;
    cudaError_t e = ensure_smem(kern, plan.smem, plan.cluster > 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    // plan.warps compute warps, plus the edge warp when the CTAs of a
    // cluster exchange halos
    if (plan.warps < 1 || plan.warps > kPersistentMaxWarps) return cudaErrorInvalidValue;
    cfg.gridDim = dim3(plan.groups * plan.cluster);
    cfg.blockDim = dim3((plan.warps + (plan.cluster > 1 ? 1 : 0)) * 32);
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

}  // namespace fxmig_impl
