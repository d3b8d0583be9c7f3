// fir.cuh -- the extrapolation arithmetic of Eq. 1 shared by the depth-loop
// kernels: operator lookup (Sec. III), register-blocked 8-output FIR with
// packed f32x2 FMAs, and the single-output FIR used for operator changes.
#pragma once

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

// Eq. 1 for 8 consecutive outputs that share one operator (taps of table row
// idx0): the common case, one 16-byte tap load per tap for 8 outputs.
template <int LT>
__device__ __forceinline__ void fir8_shared_taps(const float2* __restrict__ wbase, int idx0,
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
    const float4* tp = taps + (size_t)idx0 * (LT + 1);
    u64 A[8], B[8];
    {
        u64 hr, hi;
        ldg_nc_v2(tp, hr, hi);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            A[r] = f2_mul(hr, w[LT + r]);
            B[r] = f2_mul(hi, w[LT + r]);
        }
    }
#pragma unroll
    for (int n = 1; n <= LT; ++n) {
        u64 hr, hi;
        ldg_nc_v2(tp + n, hr, hi);
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

// Eq. 1 for one output at local position x with its own operator idx.
template <int LT>
__device__ __forceinline__ u64 fir1(const float2* __restrict__ line, int x, int idx, const float4* __restrict__ taps) {
    const float4* tp = taps + (size_t)idx * (LT + 1);
    u64 hr, hi;
    ldg_nc_v2(tp, hr, hi);
    const u64 c = *reinterpret_cast<const u64*>(line + phys(x + LT));
    u64 A = f2_mul(hr, c), B = f2_mul(hi, c);
#pragma unroll
    for (int n = 1; n <= LT; ++n) {
        ldg_nc_v2(tp + n, hr, hi);
        const u64 t = f2_add(*reinterpret_cast<const u64*>(line + phys(x + LT - n)),
                             *reinterpret_cast<const u64*>(line + phys(x + LT + n)));
        A = f2_fma(hr, t, A);
        B = f2_fma(hi, t, B);
    }
    const float2 a = f2_unpack(A), b = f2_unpack(B);
    return f2_pack(a.x - b.y, a.y + b.x);
}

}  // namespace fxmig_impl
