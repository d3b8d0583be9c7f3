// fir.cuh -- the extrapolation arithmetic of Eq. 1 shared by the depth-loop
// kernels: operator lookup (Sec. III), register-blocked 8-output FIR with
// packed f32x2 FMAs, and the single-output FIR used for operator changes.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "fxmig_internal.cuh"

namespace fxmig_impl {

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

// Eq. 1 for 8 consecutive outputs, output r with its own taps tp[r]
// ([LT+1] of (hr, hr, hi, hi)).  wbase points at the padded position of the
// first window value (x of the first output minus L).  Outputs are
//   out_r = h0 P_r + sum_{n=1}^{L} h_n (P_{r-n} + P_{r+n}),
// accumulated as A = sum hr * (pair) and B = sum hi * (pair) with packed
// (re, im) f32x2 operations, then out = (A.re - B.im, A.im + B.re).
template <int LT>
__device__ __forceinline__ void fir8_ptrs(const float2* __restrict__ wbase, const float4* const (&tp)[8],
                                          u64 (&res)[8], float (&re)[8]) {
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
    u64 A[8], B[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const ulonglong2 h = __ldg(reinterpret_cast<const ulonglong2*>(tp[r]));
        A[r] = f2_mul(h.x, w[LT + r]);
        B[r] = f2_mul(h.y, w[LT + r]);
    }
#pragma unroll
    for (int n = 1; n <= LT; ++n) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const ulonglong2 h = __ldg(reinterpret_cast<const ulonglong2*>(tp[r] + n));
            const u64 t = f2_add(w[LT + r - n], w[LT + r + n]);
            A[r] = f2_fma(h.x, t, A[r]);
            B[r] = f2_fma(h.y, t, B[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const float2 a = f2_unpack(A[r]), b = f2_unpack(B[r]);
        res[r] = f2_pack(a.x - b.y, a.y + b.x);
    }
}

// Eq. 1 for 8 consecutive outputs with the table operators of Sec. III:
// output r uses table row table_index(q, s8[r]).
template <int LT>
__device__ __forceinline__ void fir8(const float2* __restrict__ wbase, const float (&s8)[8], float q, int nk,
                                     const float4* __restrict__ taps, u64 (&res)[8], float (&re)[8]) {
    const float4* tp[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) tp[r] = taps + (size_t)table_index(q, s8[r], nk) * (LT + 1);
    fir8_ptrs<LT>(wbase, tp, res, re);
}

__device__ __forceinline__ void load_s8(const float* p, float (&s8)[8]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    const float4 b = *reinterpret_cast<const float4*>(p + 4);
    s8[0] = a.x; s8[1] = a.y; s8[2] = a.z; s8[3] = a.w;
    s8[4] = b.x; s8[5] = b.y; s8[6] = b.z; s8[7] = b.w;
}

// ------------------------------------------------- wavefield storage policies
// How the persistent kernel keeps the wavefield in shared memory.  All
// arithmetic is FP32 (packed f32x2 pairs (re, im)); the policies convert on
// load and round on store.  ld2/st2 take an even padded position, which is
// 16-byte aligned for 8-byte elements and 8-byte aligned for 4-byte ones.
struct WsF32 {  // complex64
    typedef float2 T;
    static constexpr int kBytes = 8;
    __device__ static __forceinline__ u64 ld1(const T* p) { return *reinterpret_cast<const u64*>(p); }
    __device__ static __forceinline__ void ld2(const T* p, u64& a, u64& b) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p);
        a = v.x;
        b = v.y;
    }
    __device__ static __forceinline__ void st1(T* p, u64 v) { *reinterpret_cast<u64*>(p) = v; }
    __device__ static __forceinline__ void st2(T* p, u64 a, u64 b) {
        *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(a, b);
    }
    __device__ static __forceinline__ T from_f2(float2 v) { return v; }
    __device__ static __forceinline__ float2 to_f2(T v) { return v; }
    __device__ static __forceinline__ T zero() { return make_float2(0.f, 0.f); }
    __device__ static __forceinline__ void st_async(uint32_t addr, u64 v, uint32_t bar) {
        st_async_v2(addr, f2_unpack(v), bar);
    }
};

// complex value as two 16-bit floats (re in the low half), 4 bytes
template <class H2>
struct WsHalf {
    typedef uint32_t T;
    static constexpr int kBytes = 4;
    __device__ static __forceinline__ float2 to_f2(T v) { return H2::to_f2(v); }
    __device__ static __forceinline__ T from_f2(float2 v) { return H2::from_f2(v); }
    __device__ static __forceinline__ u64 cvt(T v) {
        const float2 f = to_f2(v);
        return f2_pack(f.x, f.y);
    }
    __device__ static __forceinline__ T rnd(u64 v) { return from_f2(f2_unpack(v)); }
    __device__ static __forceinline__ u64 ld1(const T* p) { return cvt(*p); }
    __device__ static __forceinline__ void ld2(const T* p, u64& a, u64& b) {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        a = cvt(v.x);
        b = cvt(v.y);
    }
    __device__ static __forceinline__ void st1(T* p, u64 v) { *p = rnd(v); }
    __device__ static __forceinline__ void st2(T* p, u64 a, u64 b) {
        *reinterpret_cast<uint2*>(p) = make_uint2(rnd(a), rnd(b));
    }
    __device__ static __forceinline__ T zero() { return 0u; }
    __device__ static __forceinline__ void st_async(uint32_t addr, u64 v, uint32_t bar) {
        asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];"
                     :: "r"(addr), "r"(rnd(v)), "r"(bar) : "memory");
    }
};
struct H2F16 {
    __device__ static __forceinline__ float2 to_f2(uint32_t v) {
        __half2 h;
        *reinterpret_cast<uint32_t*>(&h) = v;
        return __half22float2(h);
    }
    __device__ static __forceinline__ uint32_t from_f2(float2 v) {
        const __half2 h = __floats2half2_rn(v.x, v.y);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
};
struct H2BF16 {
    __device__ static __forceinline__ float2 to_f2(uint32_t v) {
        __nv_bfloat162 h;
        *reinterpret_cast<uint32_t*>(&h) = v;
        return __bfloat1622float2(h);
    }
    __device__ static __forceinline__ uint32_t from_f2(float2 v) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
};
typedef WsHalf<H2F16> WsF16;
typedef WsHalf<H2BF16> WsBF16;

// ------------------------------------------------------- tap storage policies
// Kernel layout of one tap of the expanded operator table and its load as
// the packed pairs (hr, hr) and (hi, hi).
struct TapF32 {  // (hr, hr, hi, hi) in FP32, 16 bytes
    typedef float4 E;
    // read-only path; a plain load so that tap offsets fold into the address
    __device__ static __forceinline__ void ld(const E* p, u64& hr, u64& hi) {
        const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(p));
        hr = v.x;
        hi = v.y;
    }
};
// 16-bit taps: (hr, hi) rounded to the half type (4 bytes), or with kSplit
// the rounded pair and the rounded remainder, h = hi_part + lo_part (8 bytes).
template <class H2, bool kSplit>
struct TapHalf {
    typedef typename std::conditional<kSplit, uint2, uint32_t>::type E;
    __device__ static __forceinline__ void ld(const E* p, u64& hr, u64& hi) {
        float2 h;
        if constexpr (kSplit) {
            const uint2 v = __ldg(p);
            const float2 a = H2::to_f2(v.x), b = H2::to_f2(v.y);
            h = make_float2(a.x + b.x, a.y + b.y);
        } else {
            h = H2::to_f2(__ldg(p));
        }
        hr = f2_pack(h.x, h.x);
        hi = f2_pack(h.y, h.y);
    }
};

// Store 8 outputs at padded positions LT + r relative to the 8-aligned base.
template <int LT, class WS>
__device__ __forceinline__ void store8(typename WS::T* base, const u64 (&res)[8]) {
    if constexpr ((LT & 1) == 0) {
#pragma unroll
        for (int r = 0; r < 8; r += 2) {
            const int t = LT + r;
            WS::st2(base + t + 2 * (t >> 3), res[r], res[r + 1]);
        }
    } else {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int t = LT + r;
            WS::st1(base + t + 2 * (t >> 3), res[r]);
        }
    }
}

// Eq. 1 for 8 consecutive outputs that share one operator (taps tp[0..LT]):
// the common case, one tap load per tap for 8 outputs.  re: real parts of
// the 8 input values at the output positions.
template <int LT, class WS, class TP>
__device__ __forceinline__ void fir8_shared_taps(const typename WS::T* __restrict__ wbase,
                                                 const typename TP::E* __restrict__ tp, u64 (&res)[8],
                                                 float (&re)[8]) {
    constexpr int NWIN = 8 + 2 * LT;
    u64 w[NWIN];
#pragma unroll
    for (int t = 0; t < NWIN; t += 2) WS::ld2(wbase + t + 2 * (t >> 3), w[t], w[t + 1]);
#pragma unroll
    for (int r = 0; r < 8; ++r) re[r] = f2_unpack(w[LT + r]).x;
    u64 A[8], B[8];
    {
        u64 hr, hi;
        TP::ld(tp, hr, hi);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            A[r] = f2_mul(hr, w[LT + r]);
            B[r] = f2_mul(hi, w[LT + r]);
        }
    }
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
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const float2 a = f2_unpack(A[r]), b = f2_unpack(B[r]);
        res[r] = f2_pack(a.x - b.y, a.y + b.x);
    }
}

// Eq. 1 for one output at local position x of a line, with taps tp[0..LT].
// The window x-LT..x+LT (positions x + d, d = 0..2LT, of the line's padded
// layout) is addressed from the 8-aligned block of x: with a = x mod 8,
// phys(x + d) = 10 (x div 8) + a + d + 2 (d div 8) + 2 [a + (d mod 8) >= 8],
// so every load is one of eight base registers plus a constant.
template <int LT, class WS, class TP>
__device__ __forceinline__ u64 fir1(const typename WS::T* __restrict__ line, int x,
                                    const typename TP::E* __restrict__ tp) {
    const int a = x & 7;
    const typename WS::T* bp = line + 10 * (x >> 3) + a;
    int adj[8];
    adj[0] = 0;
#pragma unroll
    for (int m = 1; m < 8; ++m) adj[m] = (a >= 8 - m) ? 2 : 0;
    auto at = [&](int d) { return WS::ld1(bp + adj[d & 7] + d + 2 * (d >> 3)); };
    u64 hr, hi;
    TP::ld(tp, hr, hi);
    const u64 c = at(LT);
    u64 A = f2_mul(hr, c), B = f2_mul(hi, c);
#pragma unroll
    for (int n = 1; n <= LT; ++n) {
        TP::ld(tp + n, hr, hi);
        const u64 t = f2_add(at(LT - n), at(LT + n));
        A = f2_fma(hr, t, A);
        B = f2_fma(hi, t, B);
    }
    const float2 av = f2_unpack(A), bv = f2_unpack(B);
    return f2_pack(av.x - bv.y, av.y + bv.x);
}

// Eq. 1 for the two outputs x and x + 1 (x even) of a line, each with its
// own operator (taps tp0 and tp1), in the summation order of fir1 and fir8
// (n = 0, then the pairs n = 1..LT ascending).  The window x-LT..x+1+LT is
// addressed from the 8-aligned block of x as in fir1.  re0 / re1: real parts
// of the input values at x and x + 1.
template <int LT, class WS, class TP>
__device__ __forceinline__ void fir2(const typename WS::T* __restrict__ line, int x,
                                     const typename TP::E* __restrict__ tp0, const typename TP::E* __restrict__ tp1,
                                     u64& o0, u64& o1, float& re0, float& re1) {
    const int a = x & 7;
    const typename WS::T* bp = line + 10 * (x >> 3) + a;
    int adj[8];
    adj[0] = 0;
#pragma unroll
    for (int m = 1; m < 8; ++m) adj[m] = (a >= 8 - m) ? 2 : 0;
    u64 w[2 * LT + 2];
#pragma unroll
    for (int d = 0; d < 2 * LT + 2; ++d) w[d] = WS::ld1(bp + adj[d & 7] + d + 2 * (d >> 3));
    re0 = f2_unpack(w[LT]).x;
    re1 = f2_unpack(w[LT + 1]).x;
    u64 hr, hi;
    TP::ld(tp0, hr, hi);
    u64 A0 = f2_mul(hr, w[LT]), B0 = f2_mul(hi, w[LT]);
    TP::ld(tp1, hr, hi);
    u64 A1 = f2_mul(hr, w[LT + 1]), B1 = f2_mul(hi, w[LT + 1]);
#pragma unroll
    for (int n = 1; n <= LT; ++n) {
        TP::ld(tp0 + n, hr, hi);
        const u64 t0 = f2_add(w[LT - n], w[LT + n]);
        A0 = f2_fma(hr, t0, A0);
        B0 = f2_fma(hi, t0, B0);
        TP::ld(tp1 + n, hr, hi);
        const u64 t1 = f2_add(w[LT + 1 - n], w[LT + 1 + n]);
        A1 = f2_fma(hr, t1, A1);
        B1 = f2_fma(hi, t1, B1);
    }
    float2 av = f2_unpack(A0), bv = f2_unpack(B0);
    o0 = f2_pack(av.x - bv.y, av.y + bv.x);
    av = f2_unpack(A1);
    bv = f2_unpack(B1);
    o1 = f2_pack(av.x - bv.y, av.y + bv.x);
}

}  // namespace fxmig_impl
