// prs_selftest.cu -- exercises the bounded-wait path of the library's kernels
// without any fault: one CTA waits on an mbarrier phase that nothing completes
// and spins on a flag that nothing sets.  Both waits give up after their time
// limit, record the error code and return, leaving the context usable.
#include <cuda_runtime.h>
#include <stdio.h>

#include "prs.h"
#include "prs_internal.h"
#include "prs_ptx.cuh"

namespace prs {
namespace {

__global__ void k_selftest_wait(unsigned int* err, const unsigned int* flag, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one arrival expected; none ever comes
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // the library's bounded mbarrier wait (2 s limit)
        if (!mbar_wait(&bar, 0, err)) atomicOr(err, 2u);
        // a flag spin with the same structure as the ensemble kernel's neighbour waits
        const unsigned long long t0 = global_ns();
        unsigned sleep = 32;
        for (;;) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
            if (v != 0u) break;
            if (global_ns() - t0 > limit_ns) {
                atomicOr(err, 4u);
                break;
            }
            __nanosleep(sleep);
            sleep = sleep < 1024 ? 2 * sleep : 1024;
        }
    }
}

}  // namespace
}  // namespace prs

using namespace prs;

extern "C" int prs_selftest_wait_timeout(void* stream, unsigned int* codes)
{
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int* d = nullptr;
    if (cudaMalloc((void**)&d, 2 * sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        return PRS_ENOMEM;
    }
    unsigned int h[2] = {0u, 0u};
    cudaError_t e = cudaMemsetAsync(d, 0, 2 * sizeof(unsigned int), st);
    if (e == cudaSuccess) {
        k_selftest_wait<<<1, 32, 0, st>>>(d, d + 1, 200000000ull /* 0.2 s */);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof msg, "prs_selftest_wait_timeout: %s", cudaGetErrorString(e));
        record_error(msg);
        return PRS_ECUDA;
    }
    if (codes) *codes = h[0];
    return h[0] == (kErrWaitTimeout | 2u | 4u) ? PRS_ETIMEOUT : PRS_ECUDA;
}
