// migrate_rp.cu -- the persistent depth loop with 16-bit storage (FP16 or
// BF16 wavefield lines in shared memory, 16-bit taps with an optional hi/lo
// split); FP32 arithmetic.  Same kernel as the FP32 form (depth.cuh),
// compiled here for LT = 8, 12, 17 so the FP32 translation unit stays small.
#include "depth.cuh"

namespace fxmig_impl {

bool rp_compiled(int LT) { return LT == 8 || LT == 12 || LT == 17; }

// Public [nk][L+1] complex64 table -> kernel layout [nk][LT+1] of 16-bit taps:
// the rounded pair (hr, hi), and with kSplit also the rounded remainder.
template <class H2, bool kSplit>
__global__ void k_expand_taps_half(const float2* __restrict__ table, int nk, int L, int LT,
                                   typename TapHalf<H2, kSplit>::E* __restrict__ taps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nk * (LT + 1)) return;
    const int k = i / (LT + 1), n = i - k * (LT + 1);
    const float2 h = n <= L ? table[(size_t)k * (L + 1) + n] : make_float2(0.f, 0.f);
    const uint32_t hi = H2::from_f2(h);
    if constexpr (kSplit) {
        const float2 r = H2::to_f2(hi);
        taps[i] = make_uint2(hi, H2::from_f2(make_float2(h.x - r.x, h.y - r.y)));
    } else {
        taps[i] = hi;
    }
}

template <class H2, bool kSplit>
static cudaError_t expand(const float2* table, int nk, int L, int LT, void* taps, cudaStream_t s) {
    const int n = nk * (LT + 1);
    k_expand_taps_half<H2, kSplit><<<(n + 255) / 256, 256, 0, s>>>(
        table, nk, L, LT, static_cast<typename TapHalf<H2, kSplit>::E*>(taps));
    return cudaGetLastError();
}

cudaError_t expand_taps_rp(int precision, const float2* table, int nk, int L, int LT, void* taps, cudaStream_t s) {
    switch (precision) {
        case FXMIG_PREC_FP16: return expand<H2F16, false>(table, nk, L, LT, taps, s);
        case FXMIG_PREC_BF16: return expand<H2BF16, false>(table, nk, L, LT, taps, s);
        case FXMIG_PREC_FP16_SPLIT: return expand<H2F16, true>(table, nk, L, LT, taps, s);
        case FXMIG_PREC_BF16_SPLIT: return expand<H2BF16, true>(table, nk, L, LT, taps, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int LT, class WS, class TP>
static cudaError_t launch_one(const MigratePlan& plan, const DepthArgs& a, cudaStream_t s) {
    return launch_depth<LT, WS, TP, false>(plan, a, s);
}

template <int LT>
static cudaError_t launch_prec(const MigratePlan& plan, const DepthArgs& a, cudaStream_t s) {
    switch (plan.precision) {
        case FXMIG_PREC_FP16: return launch_one<LT, WsF16, TapHalf<H2F16, false>>(plan, a, s);
        case FXMIG_PREC_BF16: return launch_one<LT, WsBF16, TapHalf<H2BF16, false>>(plan, a, s);
        case FXMIG_PREC_FP16_SPLIT: return launch_one<LT, WsF16, TapHalf<H2F16, true>>(plan, a, s);
        case FXMIG_PREC_BF16_SPLIT: return launch_one<LT, WsBF16, TapHalf<H2BF16, true>>(plan, a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_depth_rp(const MigratePlan& plan, const DepthArgs& a, cudaStream_t s) {
    switch (plan.LT) {
        case 8: return launch_prec<8>(plan, a, s);
        case 12: return launch_prec<12>(plan, a, s);
        case 17: return launch_prec<17>(plan, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fxmig_impl
