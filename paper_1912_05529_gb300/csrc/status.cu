// status.cu -- self-test of the device-side failure reporting: the bounded
// mbarrier wait the depth loops use, run against a barrier that nothing ever
// arrives at.  The wait gives up after `polls` polls, records
// kStatusTimeout in the workspace status word (as the depth loops do), and
// the kernel returns normally, so the context stays usable.
#include "fxmig_internal.cuh"

namespace fxmig_impl {

__global__ void k_selftest_timeout(int* status, uint32_t polls) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one arrival expected; none is ever made
        fence_mbar_init();
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0u, polls) && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(smem_u32(&bar)) : "memory");
}

cudaError_t launch_selftest_timeout(void* ws, int polls, cudaStream_t s) {
    int* status = static_cast<int*>(ws);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_selftest_timeout<<<1, 32, 0, s>>>(status, (uint32_t)polls);
    return cudaGetLastError();
}

}  // namespace fxmig_impl
