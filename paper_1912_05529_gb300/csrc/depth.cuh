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
// neighbour's values one step older: at the start of step t the extra warp of
// each CTA pushes its time-t values at distance L..2L from the cut into the
// other's inbox (remote stores that count their bytes on the receiver's own
// mbarrier), waits for the neighbour's, and computes the L redundant outputs
// of time t+1, which the compute warps read at step t+1.  No compute warp
// ever waits on the neighbour.  Every message is awaited by its receiver
// before the receiver's next barrier, so none can land after a CTA has
// finished.
//
// Compute warps.  Lane item = 8 consecutive outputs of one segment, the same
// chunks at every step, so a lane keeps its own 8 values in registers and
// loads only the 2L halo values of its window.  The 8 outputs share the
// operator of their first point (one tap load per tap); where the operator
// changes inside the 8, the flagged outputs are recomputed with their own
// operators by single-output FIRs: queued per item for the fixup warp (and
// the compute warps that finish first), or, in the forms without a fixup
// warp, in warp-cooperative rounds.  One CTA barrier per step replaces the
// paper's kernel exit (Sec. III, V).
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
constexpr int kDepthLaneRowSlots = 3;      // per-lane ring of the decoupled form (rows t, t+1, t+2)
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
    size_t off_mbar, off_prog, off_qs, off_box, off_rows, off_img, off_queue, off_wave, total;
    DepthSeg seg[kDepthMaxSegs];
};

__host__ __device__ inline int depth_ceil8(int v) { return (v + 7) & ~7; }

// Segments and shared-memory layout of CTA `rank` of group g.  Buffer origin
// of a segment: P = LT + 8 ceil(LT/8) positions left of x = 0 (so chunk
// windows start on 8-value blocks and the halo 2L fits), and 2L positions
// right of its last chunk.  lane_rows: slowness staged per lane (the
// decoupled form: kDepthLaneRowSlots slots of 8 values per chunk) instead of
// whole row ranges.  fixq: a queue of the items with outputs whose operator
// differs from their item's (8 bytes each, at most one per chunk) for the
// fixup warp.
// Returns false if the CTA would hold more than kDepthMaxSegs segments or
// more than one cut.
__host__ __device__ inline bool depth_layout(int nx, int nxp, int nw, int G, int C, int g, int rank, int LT,
                                             int esize, DepthLayout& L, bool lane_rows = false, bool fixq = false) {
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
    o += 8 * (kDepthRowSlots + 3);                         // row ring, inbox [parity], fixup queue
    L.off_prog = o;
    o += 4 * kDepthMaxComputeWarps;  // decoupled form: last step done per warp; cut: halo stop flag
    L.off_qs = o;
    o += 4 * kDepthMaxSegs;
    L.off_box = align16(o);
    o = L.off_box + 2 * (size_t)LT * esize;                // outbox [parity][LT]
    L.off_rows = align16(o);
    o = L.off_rows + (lane_rows ? (size_t)kDepthLaneRowSlots * L.nchunks * 8 * 4 : (size_t)kDepthRowSlots * L.rowlen * 4);
    L.off_img = align16(o);
    o = L.off_img + 2 * (size_t)L.nchunks * 8 * 8;  // fixed-point image rows [2][chunks][8] int64
    L.off_queue = align16(o);
    o = L.off_queue + (fixq ? 16 + (size_t)L.nchunks * 8 : 0);  // counts and claim heads [parity], entries
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
    int C, G, ncw, extra, fixw;    // cluster size, groups, compute warps, extra (halo) warp, fixup warp
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

// Warm the operator row tp[0..LT] into L1 (the halo warp's redundant output,
// whose operator is known a step before its FIR).
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

// Operator analysis of one compute item (8 outputs from slowness values at
// srow): idx0, the operator of its first point, which all 8 outputs use in
// the main FIR; the returned mask flags the outputs (r < nv) whose own
// operator differs (recomputed separately), idx1 their common operator (or
// -1).  (The flagged operators' tap rows are not prefetched: every lane of
// every compute warp would issue its own prefetches at the start of the step,
// and the flood of L1 requests costs more than the later loads it saves.)
template <bool kPairs>
__device__ __forceinline__ uint32_t depth_ops(const float* __restrict__ srow, float q, int nk, int nv, int& idx0,
                                              int& idx1) {
    float s8[8];
    load_s8(srow, s8);
    idx0 = depth_op_index<kPairs>(q, s8[0], nk);
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
                last = idx;
            }
        }
        if (uni) idx1 = last;
    }
    return mask;
}

// The main FIR of one compute item: the 8 outputs at window base wb (element
// offset of the chunk's block in the current buffer) with operator idx0, from
// the lane's own 8 values own[] (updated to the outputs) and the 2L halo
// values of its window.  Outputs at or beyond nv are zero (outside the line).
// Outputs flagged in skip are not stored (another warp stores them).
template <int LT, class WS, class TP>
__device__ __forceinline__ void depth_fir(const typename WS::T* __restrict__ cur, typename WS::T* __restrict__ nxt,
                                          uint32_t wb, int idx0, int nv, const typename TP::E* __restrict__ taps,
                                          u64 (&own)[8], uint32_t skip) {
    constexpr int NWIN = 8 + 2 * LT;
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
        res[r] = f2_pack(a.x - b.y, a.y + b.x);
    }
    if (nv < 8) {  // the last chunk of a line: outputs beyond it stay zero
#pragma unroll
        for (int r = 1; r < 8; ++r)
            if (r >= nv) res[r] = 0ull;
    }
    if (skip == 0u) {
        store8<LT, WS>(nxt + wb, res);
    } else {
#pragma unroll
        for (int r = 0; r < 8; ++r)
            if (!((skip >> r) & 1u)) WS::st1(nxt + wb + phys(r + LT), res[r]);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) own[r] = depth_stored<WS>(res[r]);
}

// One compute item with in-warp recomputation of its flagged outputs left to
// the caller (depth_fixups): depth_ops, then depth_fir storing all 8.
template <int LT, class WS, class TP, bool kPairs>
__device__ __forceinline__ uint32_t depth_item(const typename WS::T* __restrict__ cur, typename WS::T* __restrict__ nxt,
                                               uint32_t wb, const float* __restrict__ srow, float q, int nk, int nv,
                                               const typename TP::E* __restrict__ taps, u64 (&own)[8], int& idx1) {
    int idx0;
    const uint32_t mask = depth_ops<kPairs>(srow, q, nk, nv, idx0, idx1);
    depth_fir<LT, WS, TP>(cur, nxt, wb, idx0, nv, taps, own, 0u);
    return mask;
}

// The fixed-point image contributions of one item (the real parts of its 8
// input values; outputs at or beyond nv contribute 0) into the chunk's 64
// bytes of the imaging buffer, value pair p at slot p ^ sw (the accumulator's
// row order, acc_slot; sw = (global chunk >> 1) & 3).
__device__ __forceinline__ void depth_image_item(long long* __restrict__ dst, const u64 (&own)[8], int nv,
                                                 float scale, bool& over, uint32_t sw) {
    long long q[8];
    (void)nv;  // own[r] is zero for r >= nv (outside the line), and so is its contribution
    // rint(v * 2^e) as int32 (the conversion saturates beyond the range; one
    // range check over the item flags it)
    float m = 0.f;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const float t = f2_unpack(own[r]).x * scale;
        m = fmaxf(m, fabsf(t));
        q[r] = (long long)__float2int_rn(t);
    }
    if (!(m < kImageFixedMax)) over = true;
#pragma unroll
    for (int p = 0; p < 4; ++p)
        *reinterpret_cast<longlong2*>(dst + 2 * (p ^ sw)) = make_longlong2(q[2 * p], q[2 * p + 1]);
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

// Drain of the operator-change queue of one step by one warp: n entries, one
// per item with flagged outputs (window base | segment << 16 | flags >> 1 <<
// 19, the item's offset in the staged slowness row) in queue[0, n); the
// warps that drain it claim 4 items at a time from the shared head counter,
// 8 lanes per item, lane r taking output r if it is flagged: its operator
// from its slowness in the step's row and its segment's line factor
// qs[segment] (with kPairs the pair offset of the segment's line, line *
// pc), and one single-output FIR.  n is uniform over the warp.
template <int LT, class WS, class TP, bool kPairs>
__device__ __forceinline__ void depth_drain_items(const uint2* __restrict__ queue, int* head, int n,
                                                  const typename WS::T* __restrict__ cur,
                                                  typename WS::T* __restrict__ nxt,
                                                  const typename TP::E* __restrict__ taps,
                                                  const float* __restrict__ row, const float* __restrict__ qs,
                                                  const DepthSeg* __restrict__ segs, int pc, int nk, int lane) {
    if (n <= 0) return;
    const int r = lane & 7;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(head, 4);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) break;
        const int i = base + (lane >> 3);
        if (i < n) {
            const uint2 e = queue[i];
            if (r > 0 && ((e.x >> (18 + r)) & 1u)) {  // flag bit r (r >= 1) sits at bit 18 + r
                const uint32_t wbo = e.x & 0xffffu;
                const int sg = (int)((e.x >> 16) & 7u);
                float q;
                if constexpr (kPairs) q = __int_as_float(segs[sg].line * pc);
                else q = qs[sg];
                const int idx = depth_op_index<kPairs>(q, row[e.y + r], nk);
                WS::st1(nxt + wbo + phys(r + LT), fir1<LT, WS, TP>(cur + wbo, r, taps + (size_t)idx * (LT + 1)));
            }
        }
    }
}

__device__ __forceinline__ void depth_mbar_arrive_remote(uint32_t remote_bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" :: "r"(remote_bar) : "memory");
}
// Remote store into another CTA's shared memory whose bytes complete on that
// CTA's mbarrier (complete_tx): the receiver learns of the data from its own
// barrier, and nothing of the sender waits for it.
__device__ __forceinline__ void depth_st_async_b64(uint32_t addr, u64 v, uint32_t remote_bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];"
                 :: "r"(addr), "l"(v), "r"(remote_bar) : "memory");
}
__device__ __forceinline__ void depth_st_async_b32(uint32_t addr, uint32_t v, uint32_t remote_bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];"
                 :: "r"(addr), "r"(v), "r"(remote_bar) : "memory");
}
__device__ __forceinline__ void depth_st_cluster_b32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared::cluster.b32 [%0], %1;" :: "r"(addr), "r"(v) : "memory");
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

__device__ __forceinline__ void depth_mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" :: "r"(smem_u32(bar)) : "memory");
}

// The whole depth loop of group g on the CTAs of one cluster (every CTA of
// the cluster calls it with the same arguments; blockDim = (ncw + extra +
// fixw) warps or more).
//
// With a fixup warp (fixw), the compute warps do not recompute the outputs
// whose operator differs from their item's: a lane whose item has such
// outputs queues the item (window base, segment, the flags, its offset in the
// staged row) right after its operator analysis, the warp arrives on the
// queue barrier, and the fixup warp starts computing the flagged outputs
// (single-output FIRs, 8 lanes per item, each taking its output's operator
// from the staged row) while the compute warps run their main FIRs, which
// leave those outputs unwritten; a compute warp that finds entries in the
// queue after its main FIR joins the drain, so the queue's tail is spread over
// the warps that finish first.  The lanes reload the flagged outputs into
// their registers after the step barrier.
template <int LT, class WS, class TP, int NR, bool kPairs, bool kFQ = (NR == 1)>
__device__ __forceinline__ void run_depth(const DepthArgs& a, int g, unsigned char* smem) {
    typedef typename WS::T T;
    const typename TP::E* __restrict__ taps_all = static_cast<const typename TP::E*>(a.taps);
    const int C = a.C;
    const int rank = C > 1 ? (int)cluster_ctarank() : 0;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    // kFQ: outputs with a different operator go to the fixup warp's queue
    // (one item per lane always; two items per lane where the queue fits in
    // shared memory), else the warp recomputes them in cooperative rounds
    constexpr bool kFixW = kFQ;
    if (kFixW != (a.fixw != 0)) {  // launch inconsistent with the compiled form (uniform: no barrier reached)
        if (threadIdx.x == 0) atomicOr(a.status, kStatusTimeout);
        return;
    }
    const bool compute = warp < a.ncw;
    const bool extra_warp = a.extra && warp == a.ncw;
    const bool fix_warp = kFixW && warp == a.ncw + a.extra;
    // the thread that stages slowness rows and hands image rows to the
    // bulk-copy engine: lane 0 of the fixup warp, else of the extra warp,
    // else thread 0
    const bool duty = kFixW ? (fix_warp && lane == 0) : a.extra ? (extra_warp && lane == 0) : tid == 0;

    DepthLayout& L = *reinterpret_cast<DepthLayout*>(smem);
    if (tid == 0) depth_layout(a.nx, a.nxp, a.nw, a.G, C, g, rank, LT, WS::kBytes, L, false, kFixW);
    __syncthreads();
    const DepthSeg* segs = L.seg;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L.off_mbar);
    uint64_t* inbar = mbar + kDepthRowSlots;  // [parity]
    uint64_t* qbar = mbar + kDepthRowSlots + 2;
    int* hstop = reinterpret_cast<int*>(smem + L.off_prog);  // cut: the neighbour gave up the exchange
    // operator-change queue: entry counts [parity], claim heads [parity]
    int* qcount = reinterpret_cast<int*>(smem + L.off_queue);
    uint2* queue = reinterpret_cast<uint2*>(smem + L.off_queue + 16);
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
        for (int b = 0; b < 2; ++b) mbar_init(&inbar[b], 1);  // the local expect_tx arrival (plus the bytes)
        mbar_init(qbar, (uint32_t)a.ncw);                      // every compute warp, once per step
        *hstop = 0;
        if (kFixW) qcount[0] = qcount[1] = qcount[2] = qcount[3] = 0;
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
        uint32_t wb[NR], ro[NR], sw[NR], sg[NR];
        float qv[NR];
        int nv[NR], ln[NR];
        u64 own[NR][8];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            wb[k] = ro[k] = sw[k] = sg[k] = 0u;
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
                sg[k] = (uint32_t)s;
                ro[k] = (uint32_t)(xg - L.sx0);
                sw[k] = (uint32_t)(xg >> 4) & 3u;
                ln[k] = segs[s].line;
                if constexpr (!kPairs) qv[k] = qs[s];
                const int rem = a.nx - xg;
                nv[k] = rem < 8 ? rem : 8;
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) own[k][r] = nv[k] > 0 ? WS::ld1(wave + wb[k] + phys(r + LT)) : 0ull;
        }
        bool over = false;
        bool qok = true;
        uint32_t pend[NR];  // outputs the queue's drainers wrote in the last step
#pragma unroll
        for (int k = 0; k < NR; ++k) pend[k] = 0u;
        for (int t = 0; t < nsteps; ++t) {
            const int z = a.z_begin + t;
            const T* cur = wave + (size_t)(t & 1) * buf;
            T* nxt = wave + (size_t)((t & 1) ^ 1) * buf;
            const float* row = rows + (size_t)(t % kDepthRowSlots) * rowlen;
            const typename TP::E* __restrict__ taps = tap_base(z);
            if (duty && t + kDepthRowSlots - 1 < nsteps) issue_row(t + kDepthRowSlots - 1);
            if constexpr (kFixW) {
                float qz[NR];
                int idx0[NR];
                uint32_t mk[NR];
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    qz[k] = qv[k];
                    if constexpr (kPairs) qz[k] = __int_as_float(ln[k] * a.pair_cnt[z]);
                    idx0[k] = 0;
                    int i1;
                    mk[k] = nv[k] > 0 ? depth_ops<kPairs>(row + ro[k], qz[k], a.nk, nv[k], idx0[k], i1) : 0u;
                }
                // queue the items with flagged outputs, one entry per item:
                // one ballot and one shared-memory atomic per warp and item
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    const uint32_t bal = __ballot_sync(0xffffffffu, mk[k] != 0u);
                    if (bal) {
                        int base = 0;
                        if (lane == 0) base = atomicAdd(&qcount[t & 1], __popc(bal));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        if (mk[k])
                            queue[base + __popc(bal & ((1u << lane) - 1u))] =
                                make_uint2(wb[k] | (sg[k] << 16) | ((mk[k] >> 1) << 19), ro[k]);
                    }
                }
                __syncwarp();
                if (lane == 0) depth_mbar_arrive(qbar);
                // image row z from the step's input values (the outputs the
                // queue's drainers wrote in the last step reloaded first) and
                // the main FIRs; with two items, item by item (the second
                // item's image stores overlap the first one's FMAs on other
                // warps)
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    if (pend[k]) {
#pragma unroll
                        for (int r = 1; r < 8; ++r)
                            if ((pend[k] >> r) & 1u) own[k][r] = WS::ld1(cur + wb[k] + phys(r + LT));
                    }
                    if (nv[k] > 0)
                        depth_image_item(img + (size_t)(t & 1) * nchunks * 8 + ((k * a.ncw + warp) * 32 + lane) * 8,
                                         own[k], nv[k], scale, over, sw[k]);
                    if constexpr (NR > 1) {
                        if (nv[k] > 0) depth_fir<LT, WS, TP>(cur, nxt, wb[k], idx0[k], nv[k], taps, own[k], mk[k]);
                        pend[k] = mk[k];
                    }
                }
                if constexpr (NR == 1) {
                    if (nv[0] > 0) depth_fir<LT, WS, TP>(cur, nxt, wb[0], idx0[0], nv[0], taps, own[0], mk[0]);
                    pend[0] = mk[0];
                }
                // then help drain the step's queue, if it has entries (a
                // glance at the count, which only grows during the step; the
                // fixup warp drains whatever the compute warps leave)
                const int qseen = __shfl_sync(0xffffffffu, *reinterpret_cast<volatile int*>(&qcount[t & 1]), 0);
                if (qok && qseen > 0) {
                    qok = __all_sync(0xffffffffu, mbar_wait_bounded(qbar, (uint32_t)(t & 1), kWaitPolls));
                    if (!qok && lane == 0) atomicOr(a.status, kStatusTimeout);
                    const int nq = __shfl_sync(0xffffffffu, qok ? *reinterpret_cast<volatile int*>(&qcount[t & 1]) : 0, 0);
                    depth_drain_items<LT, WS, TP, kPairs>(queue, &qcount[2 + (t & 1)], nq, cur, nxt, taps, row, qs,
                                                          segs, kPairs ? a.pair_cnt[z] : 0, a.nk, lane);
                }
            } else {
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                float qz = qv[k];
                if constexpr (kPairs) qz = __int_as_float(ln[k] * a.pair_cnt[z]);
                // image row z from the step's input values (before own[k] is overwritten)
                if (nv[k] > 0)
                    depth_image_item(img + (size_t)(t & 1) * nchunks * 8 + ((k * a.ncw + warp) * 32 + lane) * 8,
                                     own[k], nv[k], scale, over, sw[k]);
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
    } else if (fix_warp) {
        // ---- the fixup warp (drains the queue with the compute warps that
        // join; row staging, image hand-off, the queue counters)
        bool ok = true;
        for (int t = 0; t < nsteps; ++t) {
            const T* cur = wave + (size_t)(t & 1) * buf;
            T* nxt = wave + (size_t)((t & 1) ^ 1) * buf;
            const typename TP::E* __restrict__ taps = tap_base(a.z_begin + t);
            if (duty) {
                if (t + kDepthRowSlots - 1 < nsteps) issue_row(t + kDepthRowSlots - 1);
                if (t + 1 < nsteps) wait_row(t + 1);
            }
            // the counters of step t + 1 (last used in step t - 1, whose
            // drainers all passed the last barrier)
            if (lane == 0) qcount[(t + 1) & 1] = qcount[2 + ((t + 1) & 1)] = 0;
            if (ok) {
                ok = __all_sync(0xffffffffu, mbar_wait_bounded(qbar, (uint32_t)(t & 1), kWaitPolls));
                if (!ok && lane == 0) atomicOr(a.status, kStatusTimeout);
            }
            const int n = __shfl_sync(0xffffffffu, ok ? *reinterpret_cast<volatile int*>(&qcount[t & 1]) : 0, 0);
            depth_drain_items<LT, WS, TP, kPairs>(queue, &qcount[2 + (t & 1)], n, cur, nxt, taps,
                                                  rows + (size_t)(t % kDepthRowSlots) * rowlen, qs, segs,
                                                  kPairs ? a.pair_cnt[a.z_begin + t] : 0, a.nk, lane);
            if (duty) depth_bulk_wait_read();
            step_barrier();
            if (duty) issue_image(t);
        }
    } else {
        // ---- the extra warp (halo at the cut, row staging); warps beyond it
        // (a launch sized for wider groups) only keep the step barriers
        const int cs = L.cutseg;
        const bool halo = extra_warp && cs >= 0 && C > 1;
        int c_lbase = 0, c_x0 = 0, c_line = 0;
        float c_q = 0.f;
        int x_send = 0, x_pull = 0, x_red = 0;
        uint32_t nb_box = 0u, nb_inbar0 = 0u, nb_inbar1 = 0u, nb_hstop = 0u;
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
            nb_hstop = map_cluster_rank(hstop, nb);
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
                if (t >= 1 && halo_ok) {
                    // expect the neighbour's time-t values in this CTA's inbox
                    // [t & 1] (its remote stores count their bytes on
                    // inbar[t & 1]), and push this CTA's time-t values, which
                    // the neighbour needs at its step t, into its inbox
                    // (unless the neighbour has given up waiting)
                    if (lane == 0) mbar_arrive_expect_tx(&inbar[t & 1], (uint32_t)(LT * WS::kBytes));
                    if (lane < LT && *reinterpret_cast<volatile int*>(hstop) == 0) {
                        const T v = cur[c_lbase + phys(x_send + lane + LT)];
                        const uint32_t dst = nb_box + (uint32_t)(((t & 1) * LT + lane) * WS::kBytes);
                        const uint32_t bar = (t & 1) ? nb_inbar1 : nb_inbar0;
                        if constexpr (WS::kBytes == 8) depth_st_async_b64(dst, *reinterpret_cast<const u64*>(&v), bar);
                        else depth_st_async_b32(dst, *reinterpret_cast<const uint32_t*>(&v), bar);
                    }
                }
                // the redundant output's operator, its taps warmed into L1
                // while the neighbour's values travel
                int idx_red = -1;
                if (lane < LT) {
                    const int xg = c_x0 + x_red + lane;
                    if (xg >= 0 && xg < a.nx) {
                        float qz = c_q;
                        if constexpr (kPairs) qz = __int_as_float(c_line * a.pair_cnt[z]);
                        idx_red = depth_op_index<kPairs>(qz, row[xg - L.sx0], a.nk);
                        depth_prefetch_taps<LT, TP>(taps + (size_t)idx_red * (LT + 1));
                    }
                }
                if (t >= 1 && halo_ok) {
                    // the neighbour's time-t values (at step 0 they came from the slab)
                    const uint32_t par = (uint32_t)(((t - 1) >> 1) & 1);
                    bool ok = mbar_wait_cluster_bounded(&inbar[t & 1], par, kHaloPolls);
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) {
                        // give up the exchange for the rest of the launch: tell
                        // the neighbour to stop pushing (the results are then
                        // wrong, and the status says so)
                        halo_ok = false;
                        if (lane == 0) {
                            atomicOr(a.status, kStatusTimeout);
                            depth_st_cluster_b32(nb_hstop, 1u);
                        }
                    }
                    if (lane < LT) const_cast<T*>(cur)[c_lbase + phys(x_pull + lane + LT)] = box[(t & 1) * LT + lane];
                    __syncwarp();
                }
                if (lane < LT) {
                    const int x = x_red + lane;
                    u64 o = 0ull;
                    if (idx_red >= 0) o = fir1<LT, WS, TP>(cur + c_lbase, x, taps + (size_t)idx_red * (LT + 1));
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
        // after an abandoned exchange, give pushes the neighbour issued
        // before it saw the stop flag time to land (bounded) before this
        // CTA's shared memory is released
        if (halo && (!halo_ok || *reinterpret_cast<volatile int*>(hstop) != 0))
            for (int i = 0; i < 256; ++i) __nanosleep(1000);
    }
    // the last image row has reached global memory; no remote access is
    // outstanding once every CTA of the cluster is here
    if (duty) depth_bulk_wait_all();
    if (C > 1) cluster_sync_all(); else __syncthreads();
    if (tid == 0) {
        for (int b = 0; b < kDepthRowSlots + 3; ++b) depth_mbar_inval(&mbar[b]);
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

// ---------------------------------------------------------------- decoupled
// The depth loop with one whole-line group per CTA and no step barrier: every
// warp runs its own pipeline over its 32 chunks (lane = one 8-output item) and
// waits only for the two warps whose chunks its windows reach.  Before step
// t + 1 a warp waits until its neighbours have finished step t: their step-t
// outputs are its inputs (read after write), and they have finished reading
// the buffer its step t + 1 overwrites (write after read).  Warps may
// therefore drift apart by up to one step per warp of distance, so a warp
// slowed by operator changes delays only its neighbours for a while instead
// of the whole CTA every step.  The slowness values are staged per lane
// (cp.async, two steps ahead, ring of kDepthLaneRowSlots); each warp hands its
// own image chunks to the bulk-copy engine (reduction, add int64) and reuses
// an imaging buffer slot after that reduction has read it.
__device__ __forceinline__ void depth_cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void depth_cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void depth_cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }
__device__ __forceinline__ void depth_bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ int depth_ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
    return v;
}
__device__ __forceinline__ void depth_st_release(int* p, int v) {
    asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(p)), "r"(v) : "memory");
}
// Bounded wait (one lane) until prog[a] >= s and prog[b] >= s; false after
// about kWaitPolls polls (backing off with short sleeps).
__device__ __forceinline__ bool depth_wait_progress(const int* prog, int a, int b, int s) {
    for (uint32_t it = 0; it < kWaitPolls; ++it) {
        if (depth_ld_acquire(prog + a) >= s && depth_ld_acquire(prog + b) >= s) return true;
        if (it >= 32) __nanosleep(64);
    }
    return false;
}

template <int LT, class WS, class TP, bool kPairs>
__device__ __forceinline__ void run_depth_warps(const DepthArgs& a, int g, unsigned char* smem) {
    typedef typename WS::T T;
    const typename TP::E* __restrict__ taps_all = static_cast<const typename TP::E*>(a.taps);
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = nthr >> 5;

    DepthLayout& L = *reinterpret_cast<DepthLayout*>(smem);
    if (tid == 0) depth_layout(a.nx, a.nxp, a.nw, a.G, 1, g, 0, LT, WS::kBytes, L, true);
    __syncthreads();
    const DepthSeg* segs = L.seg;
    int* prog = reinterpret_cast<int*>(smem + L.off_prog);
    float* qs = reinterpret_cast<float*>(smem + L.off_qs);
    float* rows = reinterpret_cast<float*>(smem + L.off_rows);
    long long* img = reinterpret_cast<long long*>(smem + L.off_img);
    T* wave = reinterpret_cast<T*>(smem + L.off_wave);
    const int nseg = L.nseg, buf = L.buf, nchunks = L.nchunks;
    const int nsteps = a.z_end - a.z_begin;
    const int wfirst = warp * 32, wend = min(wfirst + 32, nchunks);
    const bool wactive = wfirst < nchunks;

    // ---- prologue: zero the buffers, line factors, wavefield at z_begin
    for (int i = tid; i < 2 * buf; i += nthr) wave[i] = WS::zero();
    if constexpr (!kPairs) {
        if (tid < nseg) qs[tid] = q_of_line(a.i0, segs[tid].line, a.nt, a.dt, a.dk);
    }
    // warps without chunks never hold their neighbours back
    if (tid < kDepthMaxComputeWarps) prog[tid] = (tid < nwarps && tid * 32 < nchunks) ? -1 : INT_MAX;
    __syncthreads();
    for (int s = 0; s < nseg; ++s) {
        const int line = segs[s].line, x0 = segs[s].x0, lbase = segs[s].lbase;
        const float2* src = a.slab + (size_t)line * a.nx;
        const int P = LT + 8 * ((LT + 7) >> 3);
        const int npos = P + 8 * segs[s].nc + 2 * LT;
        for (int p = tid; p < npos; p += nthr) {
            const int x = x0 - P + p;
            if (x >= 0 && x < a.nx) wave[lbase + phys(x - x0 + LT)] = WS::from_f2(src[x]);
        }
    }
    const float scale = depth_scale(*a.scale_exp);
    __syncthreads();

    // ---- the lane's item
    const int item = wfirst + lane;
    const bool has = item < nchunks;
    uint32_t wb = 0u, sw = 0u;
    float qv = 0.f;
    int nv = 0, ln = 0, xg = 0;
    if (has) {
        int s = 0;
        while (s + 1 < nseg && segs[s + 1].flat <= item) ++s;
        const int c = item - segs[s].flat;
        xg = segs[s].x0 + 8 * c;
        wb = (uint32_t)(segs[s].lbase + 10 * c);
        sw = (uint32_t)(xg >> 4) & 3u;
        ln = segs[s].line;
        if constexpr (!kPairs) qv = qs[s];
        const int rem = a.nx - xg;
        nv = rem < 8 ? rem : 8;
    }
    u64 own[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) own[r] = nv > 0 ? WS::ld1(wave + wb + phys(r + LT)) : 0ull;
    const uint32_t ro = (uint32_t)item * 8u;  // the item's values in a row slot
    // rows of step t: the lane's 8 values, committed as one group per step
    // (empty groups past the last step keep the count uniform)
    const float* slow_src = a.slow + (size_t)a.z_begin * a.nxp + xg;
    auto issue_rows = [&](int t) {
        if (has && t < nsteps) {
            float* dst = rows + (size_t)(t % kDepthLaneRowSlots) * nchunks * 8 + ro;
            const float* src = slow_src + (size_t)t * a.nxp;
            depth_cp_async16(dst, src);
            depth_cp_async16(dst + 4, src + 4);
        }
        depth_cp_async_commit();
    };
    auto tap_base = [&](int z) -> const typename TP::E* {
        if constexpr (kPairs) return taps_all + (size_t)(a.pair_base[z] - a.pair_base[a.pair_z0]) * (LT + 1);
        else return taps_all;
    };
    const int left = warp > 0 ? warp - 1 : warp, right = warp + 1 < kDepthMaxComputeWarps ? warp + 1 : warp;
    bool over = false, ok = true;
    if (wactive) {
        issue_rows(0);
        issue_rows(1);
        for (int t = 0; t < nsteps; ++t) {
            const int z = a.z_begin + t;
            const T* cur = wave + (size_t)(t & 1) * buf;
            T* nxt = wave + (size_t)((t & 1) ^ 1) * buf;
            const float* row = rows + (size_t)(t % kDepthLaneRowSlots) * nchunks * 8;
            long long* imgt = img + (size_t)(t & 1) * nchunks * 8;
            issue_rows(t + 2);
            depth_cp_async_wait<2>();                 // this lane's row values of step t
            if (lane == 0 && t >= 2) depth_bulk_wait_read1();  // the reduction of step t - 2 has read imgt
            __syncwarp();
            // image row z from the step's input values, handed to the bulk-copy engine
            if (has) depth_image_item(imgt + (size_t)item * 8, own, nv, scale, over, sw);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                unsigned long long* dst = a.acc + (size_t)z * a.nxp;
                for (int s = 0; s < nseg; ++s) {
                    const int lo = max(wfirst, segs[s].flat), hi = min(wend, segs[s].flat + segs[s].nc);
                    if (lo < hi)
                        depth_bulk_reduce_add_u64(dst + segs[s].x0 + 8 * (lo - segs[s].flat), imgt + (size_t)lo * 8,
                                                  (uint32_t)(hi - lo) * 64u);
                }
                depth_bulk_commit();
                // the neighbours have finished step t - 1
                if (t >= 1 && ok && !depth_wait_progress(prog, left, right, t - 1)) {
                    ok = false;
                    atomicOr(a.status, kStatusTimeout);
                }
            }
            __syncwarp();
            float qz = qv;
            if constexpr (kPairs) qz = __int_as_float(ln * a.pair_cnt[z]);
            const typename TP::E* __restrict__ taps = tap_base(z);
            int idx1 = -1;
            uint32_t mask = 0;
            if (nv > 0) mask = depth_item<LT, WS, TP, kPairs>(cur, nxt, wb, row + ro, qz, a.nk, nv, taps, own, idx1);
            if (__any_sync(0xffffffffu, mask != 0u)) {
                __syncwarp();
                depth_fixups<LT, WS, TP, kPairs>(mask, wb, ro, qz, idx1, cur, nxt, row, a.nk, taps, lane);
                __syncwarp();
#pragma unroll
                for (int r = 1; r < 8; ++r)
                    if ((mask >> r) & 1u) own[r] = WS::ld1(nxt + wb + phys(r + LT));
            }
            __syncwarp();  // the warp's outputs of step t are all written
            if (lane == 0) depth_st_release(prog + warp, t);
        }
        if (lane == 0) depth_bulk_wait_all();
    }
    depth_cp_async_wait<0>();
    if (over) atomicOr(a.status, kStatusOverflow);
    __syncthreads();
    const T* fin = wave + (size_t)(nsteps & 1) * buf;
    for (int s = 0; s < nseg; ++s) {
        const int x0 = segs[s].x0, lbase = segs[s].lbase;
        float2* dst = a.slab + (size_t)segs[s].line * a.nx + x0;
        const int n = (a.nx - x0) < 8 * segs[s].nc ? (a.nx - x0) : 8 * segs[s].nc;
        for (int x = tid; x < n; x += nthr) dst[x] = WS::to_f2(fin[lbase + phys(x + LT)]);
    }
    __syncthreads();
}

// Threads of a depth-loop launch compiled for OCC resident CTAs per SM.
// OCC = 1: ncw compute warps (at most 12 with one item per lane, 8 with two),
// the extra (halo) warp and the fixup warp.  OCC = 2 (whole lines, no cut, no extra warp): at most 8
// compute warps with one item per lane, so that two CTAs (16 warps, 4 per SM
// sub-partition at 128 registers a thread) share an SM and each one's step
// barrier, imaging and fixups overlap the other's FIR.
template <int NR, int OCC = 1>
struct DepthWarps {
    static_assert(OCC == 1 || (OCC == 2 && NR == 1), "two CTAs per SM: one item per lane");
    static constexpr int kMaxCompute = (NR == 1 && OCC == 1) ? kDepthMaxComputeWarps : 8;
    static constexpr int kThreads = OCC == 1 ? (kMaxCompute + 2) * 32 : kMaxCompute * 32;
};

template <int LT, class WS, class TP, int NR, bool kPairs = false, int OCC = 1, bool kFQ = (NR == 1)>
__global__ void __launch_bounds__(DepthWarps<NR, OCC>::kThreads, OCC) k_depth(const DepthArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    if constexpr (OCC == 2) run_depth_warps<LT, WS, TP, kPairs>(a, (int)blockIdx.x, smem);
    else run_depth<LT, WS, TP, NR, kPairs, kFQ>(a, (int)(blockIdx.x / a.C), smem);
}

// Launch of the depth loop for a plan (plan_depth): the kernel compiled for
// the plan's items per lane and CTAs per SM, clusters of plan.cluster CTAs.
template <int LT, class WS, class TP, int NR, bool kPairs, int OCC, bool kFQ = (NR == 1)>
inline cudaError_t launch_depth_nr(const MigratePlan& plan, const DepthArgs& a, cudaStream_t s) {
    auto kern = k_depth<LT, WS, TP, NR, kPairs, OCC, kFQ>;
    cudaError_t e = ensure_smem(kern, plan.smem, false);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.groups * plan.cluster);
    cfg.blockDim = dim3((plan.warps + plan.extra + plan.fixw) * 32);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = plan.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = plan.cluster > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int LT, class WS, class TP, bool kPairs>
inline cudaError_t launch_depth(const MigratePlan& plan, const DepthArgs& a, cudaStream_t s) {
    if (plan.occ == 2) {
        if (plan.nr != 1 || plan.extra || plan.cluster != 1) return cudaErrorInvalidValue;
        return launch_depth_nr<LT, WS, TP, 1, kPairs, 2>(plan, a, s);
    }
    if (plan.nr == 1) return launch_depth_nr<LT, WS, TP, 1, kPairs, 1>(plan, a, s);
    if (plan.nr == 2)
        return plan.fixw ? launch_depth_nr<LT, WS, TP, 2, kPairs, 1, true>(plan, a, s)
                         : launch_depth_nr<LT, WS, TP, 2, kPairs, 1, false>(plan, a, s);
    return cudaErrorInvalidValue;
}

}  // namespace fxmig_impl
