// image.cu -- imaging (Algorithm 1, "calculate depth row by summing over
// frequencies"; Sec. III, second kernel).
//
// The depth loops add every depth row of Re P, frequency by frequency, into a
// fixed-point accumulator acc[z][x] (int64, value acc * 2^-e).
// Integer addition is associative, so the image does not depend on the order
// in which the CTAs add their rows: the result is deterministic for any launch
// shape, and no partial image per CTA group is written or read back.
//
// The scale 2^e comes from a bound on every contribution.  Each step of Eq. 1
// with the guarded operators (|H| <= 1) does not increase the energy of a
// frequency line, so the contribution of one frequency to one pixel is
// |Re P(x, z, w)| <= ||P(., z_begin, w)||_2 <= Bmax = max_w ||P(., z_begin, w)||_2.
// Every depth loop converts the contribution of each frequency on its own,
// rint(Re P * 2^e) as a 32-bit integer (the fast float-to-int32 conversion;
// float-to-int64 runs on the FP64 pipe), and adds it into the int64
// accumulator.  With Bmax < 2^k and e = 23 - k a contribution stays below 2^31
// with a growth allowance of 2^8 (laterally varying operators are not exactly
// norm-bounded); contributions beyond that are reported (FXMIG_ERANGE).  The
// rounding of a contribution is at most 2^-(e+1) = 2^(k-24) <= Bmax 2^-23, and
// the sum over nw frequencies of such independent roundings stays near the
// FP32 rounding of the image itself.
#include <math.h>

#include "fxmig_internal.cuh"

namespace fxmig_impl {

// image[z][x] = acc[z][acc_slot(x)] * 2^-e[z]  (HBM-bound: 12 bytes per pixel;
// a warp reads 32 consecutive pixels from 4 whole chunks).  The integer is
// rounded to fp32 once (round to nearest) and scaled by an exact power of two,
// so the pixel is the correctly rounded value of acc * 2^-e (outside the
// subnormal range), without FP64 arithmetic.
__device__ __forceinline__ float exp2_int(int e) {  // 2^e, e in [-149, 127]
    return e >= -126 ? __int_as_float((e + 127) << 23) : __int_as_float(1 << (e + 149));
}
__global__ void __launch_bounds__(256) k_image_fixed(const long long* __restrict__ acc, const int* __restrict__ e,
                                                      int nz, int nx, int pitch, float* __restrict__ image) {
    const size_t n = (size_t)nz * nx;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int z = (int)(i / (size_t)nx), x = (int)(i - (size_t)z * nx);
        const float v = __ll2float_rn(__ldcs(acc + (size_t)z * pitch + acc_slot(x)));
        // 2^-e in two factors when it alone would be subnormal or overflow
        const int ez = -__ldg(e + z);
        image[i] = (ez >= -126 && ez <= 127) ? v * exp2_int(ez) : (v * exp2_int(ez / 2)) * exp2_int(ez - ez / 2);
    }
}

cudaError_t launch_image(const fxmig_desc* d, const float* partials, int nparts, float* image, cudaStream_t s) {
    const size_t n = (size_t)d->nz * d->nx;
    if (n == 0) return cudaSuccess;
    (void)nparts;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
    size_t blocks = (n + 255) / 256;
    const size_t cap = (size_t)sms * 8;
    if (blocks > cap) blocks = cap;
    const int pitch = slow_pitch(d->nx);
    const long long* acc = reinterpret_cast<const long long*>(partials);
    const int* e = reinterpret_cast<const int*>(acc + (size_t)d->nz * pitch);
    k_image_fixed<<<(unsigned)blocks, 256, 0, s>>>(acc, e, d->nz, d->nx, pitch, image);
    return cudaGetLastError();
}

// Block b: ||P(., b)||_2 of frequency line b (FP64, fixed summation order).
// The last block to finish takes the largest norm, picks e, writes it to the
// workspace and to the scale rows [z_begin, z_end), and re-arms the counter.
// A call that continues a depth range (z_begin > 0) keeps the exponent of row
// z_begin - 1 when it lies within 4 bits of the one the wavefield would get, so
// that a migration split into consecutive calls gives the same image as one
// call.  With guarded operators the energy only decreases with depth (the kept
// exponent is then coarser); learned operators may let it grow a little (the
// kept exponent is finer, and at most 4 bits of the 2^8 allowance are spent).
__global__ void __launch_bounds__(256) k_line_norms(const float2* __restrict__ slab, int nx, int nw,
                                                     double* __restrict__ norms, int* ws_head, int* e_rows,
                                                     int z_begin, int z_end) {
    __shared__ double red[256];
    __shared__ bool last;
    const float2* p = slab + (size_t)blockIdx.x * nx;
    double s = 0.0;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        const float2 v = p[x];
        s += (double)v.x * v.x + (double)v.y * v.y;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        norms[blockIdx.x] = sqrt(red[0]);
        __threadfence();
        last = atomicAdd(&ws_head[kWsNormCount], 1) == nw - 1;
    }
    __syncthreads();
    if (!last) return;
    __shared__ int e_sh;
    // the largest norm (the blocks' writes are visible: each fenced before
    // its counter increment), a block-wide max in a fixed order
    __threadfence();
    double Bt = 0.0;
    for (int j = threadIdx.x; j < nw; j += blockDim.x) Bt = fmax(Bt, __ldcg(norms + j));
    red[threadIdx.x] = Bt;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double B = red[0];
        int e = 0;
        if (B > 0.0 && B <= 1.0e300) {
            int k;
            frexp(B, &k);  // Bmax < 2^k
            e = 23 - k;
        }
        e = e < -126 ? -126 : (e > 127 ? 127 : e);
        if (z_begin > 0) {
            const int ep = e_rows[z_begin - 1];
            if (ep >= e - 4 && ep <= e + 4) e = ep;
        }
        e_sh = e;
        ws_head[kWsScaleExp] = e;
        ws_head[kWsNormCount] = 0;
    }
    __syncthreads();
    for (int z = z_begin + (int)threadIdx.x; z < z_end; z += blockDim.x) e_rows[z] = e_sh;
}

cudaError_t launch_image_prep(const fxmig_desc* d, const void* slab, float* partials, int z_begin, int z_end,
                              void* ws, double* norms, cudaStream_t s) {
    const int pitch = slow_pitch(d->nx);
    long long* acc = reinterpret_cast<long long*>(partials);
    cudaError_t e = cudaMemsetAsync(acc + (size_t)z_begin * pitch, 0, (size_t)(z_end - z_begin) * pitch * 8, s);
    if (e != cudaSuccess) return e;
    int* head = static_cast<int*>(ws);
    int* e_rows = reinterpret_cast<int*>(acc + (size_t)d->nz * pitch);
    k_line_norms<<<d->nw, 256, 0, s>>>(static_cast<const float2*>(slab), d->nx, d->nw, norms, head, e_rows, z_begin,
                                       z_end);
    return cudaGetLastError();
}

}  // namespace fxmig_impl
