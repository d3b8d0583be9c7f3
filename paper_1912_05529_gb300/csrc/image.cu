// image.cu -- imaging reduction (Algorithm 1, "calculate depth row by summing
// over frequencies"; Sec. III, second kernel): the depth section is the sum of
// the partial images written by the depth loop, taken in ascending partial
// order so that the result does not depend on scheduling.  HBM-bound: reads
// nparts * nz * nx floats once, writes nz * nx.
#include "fxmig_internal.cuh"

namespace fxmig_impl {

__global__ void __launch_bounds__(256) k_image_v4(const float4* __restrict__ partials, int nparts, size_t n4,
                                                   float4* __restrict__ image) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        float4 acc = __ldcs(partials + i);
        for (int p = 1; p < nparts; ++p) {
            const float4 v = __ldcs(partials + (size_t)p * n4 + i);
            acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
        }
        image[i] = acc;
    }
}

__global__ void __launch_bounds__(256) k_image_v1(const float* __restrict__ partials, int nparts, size_t n,
                                                   float* __restrict__ image) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float acc = partials[i];
        for (int p = 1; p < nparts; ++p) acc += partials[(size_t)p * n + i];
        image[i] = acc;
    }
}

cudaError_t launch_image(const fxmig_desc* d, const float* partials, int nparts, float* image, cudaStream_t s) {
    const size_t n = (size_t)d->nz * d->nx;
    if (n == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
    const bool v4 = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(partials) & 15) == 0) &&
                    ((reinterpret_cast<uintptr_t>(image) & 15) == 0);
    const size_t items = v4 ? n / 4 : n;
    size_t blocks = (items + 255) / 256;
    const size_t cap = (size_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (nparts == 0) return cudaMemsetAsync(image, 0, n * sizeof(float), s);
    if (v4)
        k_image_v4<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const float4*>(partials), nparts, n / 4,
                                                   reinterpret_cast<float4*>(image));
    else
        k_image_v1<<<(unsigned)blocks, 256, 0, s>>>(partials, nparts, n, image);
    return cudaGetLastError();
}

}  // namespace fxmig_impl
