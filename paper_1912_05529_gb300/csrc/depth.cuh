// depth.cuh -- the persistent depth loop of explicit f-x migration
// (Algorithm 1; Eq. 1; Sec. III per-point operator lookup), templated on the
// compiled half-length LT, on how the wavefield (WsF32 / WsF16 / WsBF16) and
// the taps (TapF32 / TapHalf) are stored, on the number NR of 8-output items
// each compute lane carries per depth step, and on kPairs (operators per
// (frequency, distinct slowness) pair instead of the table).  Arithmetic is
// FP32 in every form.
//
// Decomposition.  A launch has G groups of C CTAs (C = 1, or a cluster of 2).
// Group g owns the consecutive frequency lines [g nw / G, (g+1) nw / G); their
// 8-output chunks are laid end to end and the sequence is cut into C equal
// pieces, one per CTA.  So a CTA holds whole lines, and with C = 2 at most one
// line is cut between the two CTAs of the cluster (none when the group has an
// even number of lines).  Each CTA keeps its pieces of lines ("segments") in
// shared memory for ALL depth steps; Eq. 1 only ever reads within a segment,
// its zero padding (outside [0, nx)) and, at a cut, a halo.
//
// Halo at a cut, one step behind.  The outputs within L of the cut on the
// other side ("redundant" outputs) are computed by this CTA too, from the
// neighbour's values one step older: at step t the extra warp pulls the
// neighbour's time-t values at distance L..2L from the cut (DSMEM loads from
// the neighbour's outbox, after an mbarrier the neighbour arrives on), and
// computes the L redundant outputs of time t+1, which the compute warps read
// at step t+1.  No compute warp ever waits on the neighbour, and the
// neighbour's values have a whole depth step to arrive.  No data is written
// into another CTA's shared memory (the only remote operations are mbarrier
// arrivals and loads), so nothing can land after a CTA has finished.
//
// Compute warps.  Lane item = 8 consecutive outputs of one segment, the same
// chunks at every step, so a lane keeps its own 8 values in registers and
// loads only the 2L halo values of its window.  The 8 outputs share the
// operator of their first point (one tap load per tap); where the slowness
// changes inside the 8, the flagged outputs are recomputed by a
// warp-cooperative round of single-output FIRs.  One CTA barrier per step
// replaces the paper's kernel exit (Sec. III, V).
//
// Imaging.  Every compute lane converts the real parts of its 8 input values
// to fixed point (2^e scale from a bound on the data) into an imaging buffer
// in shared memory; after the step barrier one thread hands each segment's
// image row to the bulk-copy engine as a reduction (add, int64) into the
// image accumulator in global memory.  The image row is the exact integer sum
// of all frequencies' rounded contributions, independent of the order of the
// additions (deterministic), and costs the SM a few stores per item: no
// reduction pass inside the CTA, no atomics from the lanes, none after the
// launch.
//
// Slowness rows are staged by 1-D bulk copies into a ring, several steps ahead.
#pragma once

#include <float.h>
#include <limits.h>

#include "fir.cuh"
#include "fxmig_internal.cuh"

namespace fxmig_impl {

constexpr int kDepthMaxSegs = 8;           // segments per CTA
constexpr int kDepthRowSlots = 4;          // ring of staged slowness rows
constexpr int kDepthMaxComputeWarps = 12;  // plus the extra warp of CTAs at a cut

enum : int { kCutLeft = 1, kCutRight = 2 };

struct DepthSeg {
    int line;   // frequency line (global index)
    int x0;     // global x of the segment's first output (multiple of 8)
    int nc;     // 8-output chunks
    int cut;    // kCutLeft (chunk 0 follows the cut), kCutRight (the cut follows the last chunk), or 0
    int lbase;  // element offset of the segment's line origin in wavefield buffer 0 (x at phys(x + LT))
    int flat;   // first chunk of the segment in the CTA's chunk order
};

struct DepthLayout {
    int nseg, nchunks, cutseg;  // segments, chunks, index of the cut segment (-1: none)
    int xu0, xu1;               // global x range covered by the segments
    int sx0, rowlen;            // staged slowness range [sx0, sx0 + rowlen) (multiples of 4)
    int buf;                    // elements of one wavefield buffer
    size_t off_mbar, off_qs, off_box, off_rows, off_img, off_wave, total;
    DepthSeg seg[kDepthMaxSegs];
};

__host__ __device__ inline int depth_ceil8(int v) { return (v + 7) & ~7; }

// Segments and shared-memory layout of CTA `rank` of group g.  Buffer origin
// of a segment: P = LT + 8 ceil(LT/8) positions left of x = 0 (so chunk
// windows start on 8-value blocks and the halo 2L fits), and 2L positions
// right of its last chunk.  Returns false if the CTA would hold more than
// kDepthMaxSegs segments or more than one cut.
__host__ __device__ inline bool depth_layout(int nx, int nxp, int nw, int G, int C, int g, int rank, int LT,
                                             int esize, DepthLayout& L) {
    const int NCL = (nx + 7) >> 3;
    const int lb = (int)(((long long)g * nw) / G), le = (int)(((long long)(g + 1) * nw) / G);
    const long long T = (long long)(le - lb) * NCL;
    const long long c0 = T * rank / C, c1 = T * (rank + 1) / C;
    const int E = (LT + 7) >> 3;
    L.nseg = 0;
    L.nchunks = 0;
    L.cutseg = -1;
    L.xu0 = INT_MAX;
    L.xu1 = 0;
    int elems = 0;
    for (int j = 0; j < le - lb; ++j) {
        const long long a = c0 > (long long)j * NCL ? c0 : (long long)j * NCL;
        const long long b = c1 < (long long)(j + 1) * NCL ? c1 : (long long)(j + 1) * NCL;
        if (a >= b) continue;
        if (L.nseg == kDepthMaxSegs) return false;
        DepthSeg& s = L.seg[L.nseg];
        const int cf = (int)(a - (long long)j * NCL);
        s.line = lb + j;
        s.nc = (int)(b - a);
        s.x0 = cf * 8;
        s.cut = (cf > 0 ? kCutLeft : 0) | (cf + s.nc < NCL ? kCutRight : 0);
        if (s.cut) {
            if (L.cutseg >= 0 || s.cut == (kCutLeft | kCutRight)) return false;
            L.cutseg = L.nseg;
        }
        const int npos = LT + 8 * E + 8 * s.nc + 2 * LT;
        s.lbase = elems + 10 * E;
        s.flat = L.nchunks;
        elems += (depth_ceil8(npos) >> 3) * 10;
        L.nchunks += s.nc;
        if (s.x0 < L.xu0) L.xu0 = s.x0;
        if (s.x0 + 8 * s.nc > L.xu1) L.xu1 = s.x0 + 8 * s.nc;
        ++L.nseg;
    }
    if (L.nseg == 0) {
        L.xu0 = L.xu1 = 0;
        L.sx0 = 0;
        L.rowlen = 0;
    } else {
        int a = L.xu0 - LT;
        a = a < 0 ? 0 : (a & ~7);
        int b = depth_ceil8(L.xu1 + LT);
        if (b > nxp) b = nxp;
        L.sx0 = a;
        L.rowlen = b - a;
    }
    L.buf = elems;
    size_t o = align16(sizeof(DepthLayout));  // the layout itself heads the CTA's shared memory
    L.off_mbar = o;
    o += 8 * (kDepthRowSlots + 2);                         // row ring, inbox [parity]
    L.off_qs = o;
    o += 4 * kDepthMaxSegs;
    L.off_box = align16(o);
    o = L.off_box + 2 * (size_t)LT * esize;                // outbox [parity][LT]
    L.off_rows = align16(o);
    o = L.off_rows + (size_t)kDepthRowSlots * L.rowlen * 4;
    L.off_img = align16(o);
    o = L.off_img + 2 * (size_t)L.nchunks * 8 * 8;  // fixed-point image rows [2][chunks][8] int64
    L.off_wave = align16(o);
    L.total = L.off_wave + 2 * (size_t)elems * esize;
    return true;
}

struct DepthArgs {
    int nx, nxp, nz, nw, nk, z_begin, z_end, i0, nt, L;
    double dt, dk;
    float2* slab;                  // [nw][nx]
    const float* slow;             // [nz][nxp] slowness fl32(1/v) (or kPairs: distinct-value index bits)
    const void* taps;              // [nk][LT+1] kernel tap layout (kPairs: operators in pair order)
    unsigned long long* acc;       // [nz][nx] image accumulator, fixed point 2^e
    const int* scale_exp;          // e, written before the launch
    int* status;
    int C, G, ncw, extra;          // cluster size, groups, compute warps, extra warp present
    // kPairs: operators per (frequency, distinct slowness) pair
    const int* pair_cnt;           // [nz] distinct values of each row
    const long long* pair_base;    // [nz+1] first pair of each row
    int pair_z0;                   // row of the first operator in taps
};

// Operator index of a point with staged row value v: the table entry of
// Sec. III for line factor q, or (kPairs) the pair index line offset + v.
template <bool kPairs>
__device__ __forceinline__ int depth_op_index(float q, float v, int nk) {
    if constexpr (kPairs) return __float_as_int(q) + __float_as_int(v);
    else return table_index(q, v, nk);
}

// Warm the operator row tp[0..LT] into L1 (rows of operator changes, read by
// the fixup round after the main items).
template <int LT, class TP>
__device__ __forceinline__ void depth_prefetch_taps(const typename TP::E* tp) {
    constexpr int kBytes = (LT + 1) * (int)sizeof(typename TP::E);
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(tp);
#pragma unroll
    for (int o = 0; o < kBytes + 127; o += 128) {
        const uintptr_t a = (a0 & ~uintptr_t(127)) + (uintptr_t)o;
        if (a < a0 + kBytes) asm volatile("prefetch.global.L1 [%0];" :: "l"(a));
    }
}

__device__ __forceinline__ void depth_red_add_u64(unsigned long long* p, long long v) {
    asm volatile("red.global.add.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

// Value as stored: FP32 storage keeps it, 16-bit storage rounds it.
template <class WS>
__device__ __forceinline__ u64 depth_stored(u64 v) {
    if constexpr (WS::kBytes == 8) return v;
    else return WS::cvt(WS::rnd(v));
}

// One compute item: the 8 outputs at window base wb (element offset of the
// chunk's block in the current buffer) from the lane's own 8 values own[]
// (updated to the outputs) and the 2L halo values of its window.  Outputs at
// or beyond nv are zero (outside the line).  The 8 outputs use the operator of
// the first point; returns the mask of outputs whose own operator differs
// (recomputed by the fixup round), idx1 their common operator (or -1).
template <int LT, class WS, class TP, bool kPairs>
__device__ __forceinline__ uint32_t depth_item(const typename WS::T* __restrict__ cur, typename WS::T* __restrict__ nxt,
                                               uint32_t wb, const float* __restrict__ srow, float q, int nk, int nv,
                                               const typename TP::E* __restrict__ taps, u64 (&own)[8], int& idx1) {
    constexpr int NWIN = 8 + 2 * LT;
    float s8[8];
    load_s8(srow, s8);
    const int idx0 = depth_op_index<kPairs>(q, s8[0], nk);
    uint32_t mask = 0;
    idx1 = -1;
    bool same = true;
#pragma unroll
    for (int r = 1; r < 8; ++r) same &= (__float_as_uint(s8[r]) == __float_as_uint(s8[0]));
    if (!same) {
        int last = idx0;
        bool uni = true;
#pragma unroll
        for (int r = 1; r < 8; ++r) {
            const int idx = depth_op_index<kPairs>(q, s8[r], nk);
            if (r < nv && idx != idx0) {
                uni &= (mask == 0u) || (idx == last);
                mask |= 1u << r;
                if (idx != last) depth_prefetch_taps<LT, TP>(taps + (size_t)idx * (LT + 1));
                last = idx;
            }
        }
        if (uni) idx1 = last;
    }
    const typename WS::T* wbase = cur + wb;
    u64 w[NWIN];
    // w[LT + r] = own[r]; the 2L halo values come from shared memory in
    // pairs (for odd LT the pairs around the own values are split)
#pragma unroll
    for (int t = 0; t < NWIN; t += 2) {
        const bool lo_own = t >= LT && t < LT + 8, hi_own = t + 1 >= LT && t + 1 < LT + 8;
        if (lo_own && hi_own) {
            w[t] = own[t - LT];
            w[t + 1] = own[t + 1 - LT];
        } else if (hi_own) {
            w[t] = WS::ld1(wbase + t + 2 * (t >> 3));
            w[t + 1] = own[t + 1 - LT];
        } else if (lo_own) {
            w[t] = own[t - LT];
            w[t + 1] = WS::ld1(wbase + (t + 1) + 2 * ((t + 1) >> 3));
        } else {
            WS::ld2(wbase + t + 2 * (t >> 3), w[t], w[t + 1]);
        }
    }
    u64 A[8], B[8];
    {
        u64 hr, hi;
        TP::ld(taps + (size_t)idx0 * (LT + 1), hr, hi);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            A[r] = f2_mul(hr, w[LT + r]);
            B[r] = f2_mul(hi, w[LT + r]);
        }
    }
    const typename TP::E* __restrict__ tp = taps + (size_t)idx0 * (LT + 1);
#pragma unroll
    for (int n = 1; n <= LT; ++n) {
        u64 hr, hi;
        TP::ld(tp + n, hr, hi);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const u64 t = f2_add(w[LT + r - n], w[LT + r + n]);
            A[r] = f2_fma(hr, t, A[r]);
            B[r] = f2_fma(hi, t, B[r]);
        }
    }
    u64 res[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const float2 a = f2_unpack(A[r]), b = f2_unpack(B[r]);
        res[r] = (r < nv) ? f2_pack(a.x - b.y, a.y + b.x) : 0ull;
    }
    store8<LT, WS>(nxt + wb, res);
#pragma unroll
    for (int r = 0; r < 8; ++r) own[r] = depth_stored<WS>(res[r]);
    return mask;
}

// The fixed-point image contributions of one item (the real parts of its 8
// input values; outputs at or beyond nv contribute 0) into the imaging buffer.
__device__ __forceinline__ void depth_image_item(long long* __restrict__ dst, const u64 (&own)[8], int nv,
                                                 float scale, bool& over) {
    long long q[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) q[r] = r < nv ? image_fixed(f2_unpack(own[r]).x, scale, over) : 0;
#pragma unroll
    for (int r = 0; r < 8; r += 2)
        *reinterpret_cast<longlong2*>(dst + r) = make_longlong2(q[r], q[r + 1]);
}

// Bulk reduction (add, int64) of `bytes` from this CTA's shared memory into
// global memory, tracked as a bulk group of the issuing thread; both
// addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void depth_bulk_reduce_add_u64(unsigned long long* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u64 [%0], [%1], %2;"
                 :: "l"(dst), "r"(smem_u32(src)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void depth_bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until the issuing thread's bulk groups have read their sources (read)
// or completed entirely.
__device__ __forceinline__ void depth_bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void depth_bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Position of the n-th set bit (n >= 1) of m, which has at least n set bits.
__device__ __forceinline__ int depth_nth_set_bit(uint32_t m, int n) {
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

// Warp-cooperative recomputation of the outputs flagged in each lane's mask
// (bit r: output r of the lane's item at window base wb): numbered by output
// position, then by lane, from one ballot per position, and taken one per
// lane with a single-output FIR and the output's own operator.  idx1 is the
// owner's common operator of its flagged outputs, or -1.  All lanes call.
template <int LT, class WS, class TP, bool kPairs>
__device__ __forceinline__ void depth_fixups(uint32_t mask, uint32_t wb, uint32_t ro, float q, int idx1,
                                             const typename WS::T* __restrict__ cur, typename WS::T* __restrict__ nxt,
                                             const float* __restrict__ row, int nk,
                                             const typename TP::E* __restrict__ taps, int lane) {
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
        int r = 1;
        uint32_t br = bal[1];
        int pr = pre[1];
#pragma unroll
        for (int k = 2; k < 8; ++k)
            if (pre[k] <= it) { r = k; br = bal[k]; pr = pre[k]; }
        const int owner = it < total ? depth_nth_set_bit(br, it - pr + 1) : 0;
        const uint32_t wb_o = __shfl_sync(0xffffffffu, wb, owner);
        const uint32_t ro_o = __shfl_sync(0xffffffffu, ro, owner);
        const float q_o = __shfl_sync(0xffffffffu, q, owner);
        const int i1_o = __shfl_sync(0xffffffffu, idx1, owner);
        if (it < total) {
            const int idx = i1_o >= 0 ? i1_o : depth_op_index<kPairs>(q_o, row[ro_o + r], nk);
            WS::st1(nxt + wb_o + phys(r + LT), fir1<LT, WS, TP>(cur + wb_o, r, taps + (size_t)idx * (LT + 1)));
        }
    }
}

__device__ __forceinline__ void depth_mbar_arrive_remote(uint32_t remote_bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" :: "r"(remote_bar) : "memory");
}
__device__ __forceinline__ u64 depth_ld_cluster_b64(uint32_t addr) {
    u64 v;
    asm volatile("ld.shared::cluster.b64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t depth_ld_cluster_b32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.b32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void depth_mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(smem_u32(bar)) : "memory");
}

// Fixed-point scale 2^e of the image accumulator as a float (e in [-126, 127]).
__device__ __forceinline__ float depth_scale(int e) { return __int_as_float((e + 127) << 23); }

// The whole depth loop of group g on the CTAs of one cluster (every CTA of
// the cluster calls it with the same arguments; blockDim = (ncw + extra) warps).
template <int LT, class WS, class TP, int NR, bool kPairs>
__device__ __forceinline__ void run_depth(const DepthArgs& a, int g, unsigned char* smem) {
    typedef typename WS::T T;
    const typename TP::E* __restrict__ taps_all = static_cast<const typename TP::E*>(a.taps);
    const int C = a.C;
    const int rank = C > 1 ? (int)cluster_ctarank() : 0;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const bool compute = warp < a.ncw;
    const bool extra_warp = a.extra && warp == a.ncw;
    // the thread that stages slowness rows: lane 0 of the extra warp, else thread 0
    const bool duty = a.extra ? (extra_warp && lane == 0) : tid == 0;

    DepthLayout& L = *reinterpret_cast<DepthLayout*>(smem);
    if (tid == 0) depth_layout(a.nx, a.nxp, a.nw, a.G, C, g, rank, LT, WS::kBytes, L);
    __syncthreads();
    const DepthSeg* segs = L.seg;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L.off_mbar);
    uint64_t* inbar = mbar + kDepthRowSlots;  // [parity]
    float* qs = reinterpret_cast<float*>(smem + L.off_qs);
    T* box = reinterpret_cast<T*>(smem + L.off_box);
    float* rows = reinterpret_cast<float*>(smem + L.off_rows);
    long long* img = reinterpret_cast<long long*>(smem + L.off_img);
    T* wave = reinterpret_cast<T*>(smem + L.off_wave);
    const int nseg = L.nseg, buf = L.buf, rowlen = L.rowlen, nchunks = L.nchunks;
    const int nsteps = a.z_end - a.z_begin;

    // ---- prologue
    for (int i = tid; i < 2 * buf; i += nthr) wave[i] = WS::zero();
    if constexpr (!kPairs) {
        if (tid < nseg) qs[tid] = q_of_line(a.i0, segs[tid].line, a.nt, a.dt, a.dk);
    }
    if (tid == 0) {
        for (int b = 0; b < kDepthRowSlots; ++b) mbar_init(&mbar[b], 1);
        for (int b = 0; b < 2; ++b) mbar_init(&inbar[b], 1);  // one lane of the neighbour's extra warp arrives
        fence_mbar_init();
    }
    __syncthreads();
    // wavefield at z_begin over each segment's buffer range (halo positions
    // included; zero outside [0, nx))
    for (int s = 0; s < nseg; ++s) {
        const int line = segs[s].line, x0 = segs[s].x0, lbase = segs[s].lbase;
        const float2* src = a.slab + (size_t)line * a.nx;
        const int P = LT + 8 * ((LT + 7) >> 3);
        const int npos = P + 8 * segs[s].nc + 2 * LT;
        for (int p = tid; p < npos; p += nthr) {
            const int x = x0 - P + p;  // global x
            if (x >= 0 && x < a.nx) wave[lbase + phys(x - x0 + LT)] = WS::from_f2(src[x]);
        }
    }
    // rows, kDepthRowSlots - 1 steps ahead: row t in slot t % kDepthRowSlots
    const uint32_t row_bytes = (uint32_t)rowlen * 4u;
    const float* row_src = a.slow + (size_t)a.z_begin * a.nxp + L.sx0;
    auto issue_row = [&](int t) {  // one thread
        const int b = t % kDepthRowSlots;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&mbar[b], row_bytes);
        if (row_bytes) bulk_g2s(rows + (size_t)b * rowlen, row_src + (size_t)t * a.nxp, row_bytes, &mbar[b]);
    };
    auto wait_row = [&](int t) {
        const int b = t % kDepthRowSlots;
        if (!mbar_wait_bounded(&mbar[b], (uint32_t)((t / kDepthRowSlots) & 1), kWaitPolls))
            atomicOr(a.status, kStatusTimeout);
    };
    if (duty) {
        for (int t = 0; t < nsteps && t < kDepthRowSlots - 1; ++t) issue_row(t);
        if (nsteps > 0) wait_row(0);
    }
    // fixed-point scale of the image accumulator
    const float scale = depth_scale(*a.scale_exp);
    // every CTA of the cluster has initialised its barriers and buffers
    if (C > 1) cluster_sync_all(); else __syncthreads();

    // Each warp role runs its own step loop (so the compute warps do not keep
    // the extra warp's halo state in registers); both end every step with the
    // same CTA barrier (barrier.sync without .aligned, reached from the two
    // loops).  Only the compute warps write global memory during the loop (the
    // extra warp's cluster-scope release then waits for nothing of theirs).
    auto step_barrier = [] { asm volatile("barrier.sync 0;" ::: "memory"); };
    // image row of step t (after its barrier): one bulk reduction per segment
    // from img[t & 1] into the accumulator row (the duty thread; the lanes
    // fenced their writes for the async proxy before the barrier).  The duty
    // thread waits for the sources to be read before the next barrier, after
    // which img[t & 1] may be written again (step t + 2).
    const int pitch = a.nxp;
    auto issue_image = [&](int t) {
        const long long* src = img + (size_t)(t & 1) * nchunks * 8;
        unsigned long long* dst = a.acc + (size_t)(a.z_begin + t) * pitch;
        for (int s = 0; s < nseg; ++s)
            depth_bulk_reduce_add_u64(dst + segs[s].x0, src + (size_t)segs[s].flat * 8, (uint32_t)segs[s].nc * 64u);
        depth_bulk_commit();
    };
    auto tap_base = [&](int z) -> const typename TP::E* {
        if constexpr (kPairs) return taps_all + (size_t)(a.pair_base[z] - a.pair_base[a.pair_z0]) * (LT + 1);
        else return taps_all;
    };

    if (compute) {
        // ---- the lane's items (the same chunks at every step)
        uint32_t wb[NR], ro[NR];
        float qv[NR];
        int nv[NR], ln[NR];
        u64 own[NR][8];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            wb[k] = ro[k] = 0u;
            qv[k] = 0.f;
            nv[k] = 0;
            ln[k] = 0;
            const int item = (k * a.ncw + warp) * 32 + lane;
            if (item < nchunks) {
                int s = 0;
                while (s + 1 < nseg && segs[s + 1].flat <= item) ++s;
                const int c = item - segs[s].flat;
                const int xg = segs[s].x0 + 8 * c;
                wb[k] = (uint32_t)(segs[s].lbase + 10 * c);
                ro[k] = (uint32_t)(xg - L.sx0);
                ln[k] = segs[s].line;
                if constexpr (!kPairs) qv[k] = qs[s];
                const int rem = a.nx - xg;
                nv[k] = rem < 8 ? rem : 8;
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) own[k][r] = nv[k] > 0 ? WS::ld1(wave + wb[k] + phys(r + LT)) : 0ull;
        }
        bool over = false;
        for (int t = 0; t < nsteps; ++t) {
            const int z = a.z_begin + t;
            const T* cur = wave + (size_t)(t & 1) * buf;
            T* nxt = wave + (size_t)((t & 1) ^ 1) * buf;
            const float* row = rows + (size_t)(t % kDepthRowSlots) * rowlen;
            const typename TP::E* __restrict__ taps = tap_base(z);
            if (duty && t + kDepthRowSlots - 1 < nsteps) issue_row(t + kDepthRowSlots - 1);
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                float qz = qv[k];
                if constexpr (kPairs) qz = __int_as_float(ln[k] * a.pair_cnt[z]);
                // image row z from the step's input values (before own[k] is overwritten)
                if (nv[k] > 0)
                    depth_image_item(img + (size_t)(t & 1) * nchunks * 8 + ((k * a.ncw + warp) * 32 + lane) * 8,
                                     own[k], nv[k], scale, over);
                int idx1 = -1;
                uint32_t mask = 0;
                if (nv[k] > 0)
                    mask = depth_item<LT, WS, TP, kPairs>(cur, nxt, wb[k], row + ro[k], qz, a.nk, nv[k], taps,
                                                          own[k], idx1);
                if (__any_sync(0xffffffffu, mask != 0u)) {
                    __syncwarp();  // the main items' stores precede the rewrites
                    depth_fixups<LT, WS, TP, kPairs>(mask, wb[k], ro[k], qz, idx1, cur, nxt, row, a.nk, taps,
                                                     lane);
                    __syncwarp();
#pragma unroll
                    for (int r = 1; r < 8; ++r)
                        if ((mask >> r) & 1u) own[k][r] = WS::ld1(nxt + wb[k] + phys(r + LT));
                }
            }
            fence_proxy_async_smem();  // the image values, for the bulk reduction
            if (duty) {
                if (t + 1 < nsteps) wait_row(t + 1);
                depth_bulk_wait_read();
            }
            step_barrier();
            if (duty) issue_image(t);
        }
        if (over) atomicOr(a.status, kStatusOverflow);
    } else {
        // ---- the extra warp (halo at the cut, row staging); warps beyond it
        // (a launch sized for wider groups) only keep the step barriers
        const int cs = L.cutseg;
        const bool halo = extra_warp && cs >= 0 && C > 1;
        int c_lbase = 0, c_x0 = 0, c_line = 0;
        float c_q = 0.f;
        int x_send = 0, x_pull = 0, x_red = 0;
        uint32_t nb_box = 0u, nb_inbar0 = 0u, nb_inbar1 = 0u;
        if (halo) {
            const bool left = (segs[cs].cut & kCutLeft) != 0;
            const int nc = segs[cs].nc;
            c_lbase = segs[cs].lbase;
            c_x0 = segs[cs].x0;
            c_line = segs[cs].line;
            if constexpr (!kPairs) c_q = qs[cs];
            // segment-local x of: the values this CTA sends (distance L..2L
            // from the cut on its side), the neighbour's values it pulls
            // (distance L..2L on the other side), its redundant outputs
            // (distance 0..L on the other side)
            x_send = left ? LT : 8 * nc - 2 * LT;
            x_pull = left ? -2 * LT : 8 * nc + LT;
            x_red = left ? -LT : 8 * nc;
            const uint32_t nb = (uint32_t)(left ? rank - 1 : rank + 1);
            nb_box = map_cluster_rank(box, nb);
            nb_inbar0 = map_cluster_rank(&inbar[0], nb);
            nb_inbar1 = map_cluster_rank(&inbar[1], nb);
        }
        bool halo_ok = true;
        for (int t = 0; t < nsteps; ++t) {
            const int z = a.z_begin + t;
            const T* cur = wave + (size_t)(t & 1) * buf;
            T* nxt = wave + (size_t)((t & 1) ^ 1) * buf;
            const float* row = rows + (size_t)(t % kDepthRowSlots) * rowlen;
            if (duty && t + kDepthRowSlots - 1 < nsteps) issue_row(t + kDepthRowSlots - 1);
            // the redundant outputs of time t + 1 (those of the last step are
            // never read)
            if (halo && t + 1 < nsteps) {
                const typename TP::E* __restrict__ taps = tap_base(z);
                if (t >= 1) {
                    // send this CTA's time-t values, which the neighbour needs at its step t
                    if (lane < LT) box[(t & 1) * LT + lane] = cur[c_lbase + phys(x_send + lane + LT)];
                    // the warp's box writes, then one release-arrive (cumulative
                    // over what the warp barrier made visible to lane 0)
                    __syncwarp();
                    if (lane == 0) depth_mbar_arrive_remote((t & 1) ? nb_inbar1 : nb_inbar0);
                    // pull the neighbour's time-t values (at step 0 they came from the slab)
                    const uint32_t par = (uint32_t)(((t - 1) >> 1) & 1);
                    bool ok = mbar_wait_cluster_bounded(&inbar[t & 1], par, halo_ok ? kHaloPolls : 1u);
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) {
                        halo_ok = false;
                        if (lane == 0) atomicOr(a.status, kStatusTimeout);
                    }
                    if (lane < LT) {
                        const uint32_t src = nb_box + (uint32_t)(((t & 1) * LT + lane) * WS::kBytes);
                        T v;
                        if constexpr (WS::kBytes == 8) {
                            const u64 u = depth_ld_cluster_b64(src);
                            v = *reinterpret_cast<const T*>(&u);
                        } else {
                            const uint32_t u = depth_ld_cluster_b32(src);
                            v = *reinterpret_cast<const T*>(&u);
                        }
                        const_cast<T*>(cur)[c_lbase + phys(x_pull + lane + LT)] = v;
                    }
                    __syncwarp();
                }
                if (lane < LT) {
                    const int x = x_red + lane;
                    const int xg = c_x0 + x;
                    u64 o = 0ull;
                    if (xg >= 0 && xg < a.nx) {
                        float qz = c_q;
                        if constexpr (kPairs) qz = __int_as_float(c_line * a.pair_cnt[z]);
                        const int idx = depth_op_index<kPairs>(qz, row[xg - L.sx0], a.nk);
                        o = fir1<LT, WS, TP>(cur + c_lbase, x, taps + (size_t)idx * (LT + 1));
                    }
                    WS::st1(nxt + c_lbase + phys(x + LT), o);
                }
            }
            if (duty) {
                if (t + 1 < nsteps) wait_row(t + 1);
                depth_bulk_wait_read();
            }
            step_barrier();
            if (duty) issue_image(t);
        }
    }
    // the last image row has reached global memory; no remote access is
    // outstanding once every CTA of the cluster is here
    if (duty) depth_bulk_wait_all();
    if (C > 1) cluster_sync_all(); else __syncthreads();
    if (tid == 0) {
        for (int b = 0; b < kDepthRowSlots + 2; ++b) depth_mbar_inval(&mbar[b]);
    }
    const T* fin = wave + (size_t)(nsteps & 1) * buf;
    for (int s = 0; s < nseg; ++s) {
        const int x0 = segs[s].x0, lbase = segs[s].lbase;
        float2* dst = a.slab + (size_t)segs[s].line * a.nx + x0;
        const int n = (a.nx - x0) < 8 * segs[s].nc ? (a.nx - x0) : 8 * segs[s].nc;
        for (int x = tid; x < n; x += nthr) dst[x] = WS::to_f2(fin[lbase + phys(x + LT)]);
    }
    // the layout header is rewritten by the next group only after every
    // thread is done with it
    __syncthreads();
}

// Threads of a depth-loop launch: ncw compute warps (at most 12 with one item
// per lane, 8 with two) and the extra warp.
template <int NR>
struct DepthWarps {
    static constexpr int kMaxCompute = NR == 1 ? kDepthMaxComputeWarps : 8;
    static constexpr int kThreads = (kMaxCompute + 1) * 32;
};

template <int LT, class WS, class TP, int NR, bool kPairs = false>
__global__ void __launch_bounds__(DepthWarps<NR>::kThreads, 1) k_depth(const DepthArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    run_depth<LT, WS, TP, NR, kPairs>(a, (int)(blockIdx.x / a.C), smem);
}

}  // namespace fxmig_impl
