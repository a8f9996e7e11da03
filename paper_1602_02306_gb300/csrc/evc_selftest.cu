// evc_selftest.cu -- failure detection without a GPU fault: a kernel whose
// mbarrier wait can never complete (nothing arrives on the barrier) runs the
// library's bounded wait with a short limit, gives up, records DERR_TIMEOUT in
// a device word and returns, so the host sees EVC_ETIMEOUT and the context
// stays usable.  The streaming kernels report a stalled pipeline the same way.
#include "evc_internal.cuh"
#include "evc_bulk.cuh"
#include "../../include/evc.h"

namespace evc {
namespace {

__global__ void wait_selftest_kernel(long long cycles, int* flag)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    // phase 0 of `bar` completes only after one arrival, and none is made
    const bool ok = mbar_wait_for(&bar, 0u, cycles);
    const bool all = __syncthreads_and(ok ? 1 : 0);
    if (threadIdx.x == 0) *flag = all ? DERR_NONE : DERR_TIMEOUT;
}

}  // namespace
}  // namespace evc

int evc_wait_selftest(double limit_ms, int* status)
{
    if (!status || !(limit_ms > 0.0) || limit_ms > 2000.0) return EVC_EINVAL;
    int dev = 0, khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0) {
        cudaGetLastError();
        return EVC_ECUDA;
    }
    int* flag = nullptr;
    if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return EVC_ENOMEM;
    }
    const long long cycles = (long long)(limit_ms * khz);
    evc::wait_selftest_kernel<<<1, 64>>>(cycles, flag);
    cudaError_t e = cudaGetLastError();
    int h = -1;
    if (e == cudaSuccess) e = cudaMemcpy(&h, flag, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(flag);
    if (e != cudaSuccess) return EVC_ECUDA;
    *status = h == evc::DERR_TIMEOUT ? EVC_ETIMEOUT : (h == evc::DERR_NONE ? EVC_OK : EVC_ECUDA);
    return EVC_OK;
}
