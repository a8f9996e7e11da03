// evc_static.cu -- allocation-free batched Gauss quadrature (see
// evc_gauss_quadrature_static in include/evc.h).  The eigensolver scratch
// lives in one file-scope device array instead of caller- or library-
// allocated memory, for callers that cannot allocate device memory.
#include "evc_internal.cuh"
#include "evc_tridiag.cuh"
#include "../../include/evc.h"

#include <math_constants.h>

#include <cmath>
#include <cstdio>
#include <mutex>

namespace {

// 3 * EVC_STATIC_QUAD_MAX doubles (6 MiB) on every device that loads the library.
__device__ __align__(256) double g_quad_scratch[3 * EVC_STATIC_QUAD_MAX];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
double* g_scratch_dev[kMaxDevices] = {};

// One thread per column.  A column whose size is outside [1, k] is not
// computed (NaN, status EVC_EINVAL); one whose eigensolve does not converge
// gets NaN and status EVC_ENUMERIC.  The first failure wins the status word.
__global__ void static_quad_kernel(const double* alpha, const double* beta, const int* kcol,
                                   int k, int ncol, double vnorm2, double* quad, double* scratch,
                                   int* status)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    const int kc = kcol ? kcol[c] : k;
    if (kc < 1 || kc > k) {
        quad[c] = CUDART_NAN;
        if (status) atomicCAS(status, EVC_OK, EVC_EINVAL);
        return;
    }
    bool finite = true;
    for (int t = 0; t < kc; ++t)
        finite = finite && isfinite(alpha[(int64_t)t * ncol + c]) &&
                 (t == 0 || isfinite(beta[(int64_t)t * ncol + c]));
    // scratch layout [3][k][ncol]: d, e, z, coalesced across columns
    const int64_t plane = (int64_t)k * ncol;
    double q = finite ? evc::tridiag_gauss_quadrature(alpha + c, beta + c, ncol, kc, vnorm2,
                                                      scratch + c, scratch + plane + c,
                                                      scratch + 2 * plane + c, ncol)
                      : -1.0;
    if (!(q >= 0.0)) {   // -1: non-finite input, or the eigensolver did not converge
        q = CUDART_NAN;
        if (status) atomicCAS(status, EVC_OK, EVC_ENUMERIC);
    }
    quad[c] = q;
}

int say(char* buf, size_t len, int code, const char* msg)
{
    if (buf && len) snprintf(buf, len, "%s", msg);
    return code;
}

}  // namespace

extern "C" int evc_gauss_quadrature_static(const double* d_alpha, const double* d_beta,
                                           const int* d_kcol, int k, int ncol, double vnorm2,
                                           double* d_quad, int* d_status, void* stream,
                                           char* errbuf, size_t errlen)
{
    if (!d_alpha || !d_beta || !d_quad)
        return say(errbuf, errlen, EVC_EINVAL, "null device pointer");
    if (k < 1 || k > EVC_MAX_STEPS || ncol < 1)
        return say(errbuf, errlen, EVC_EINVAL, "need 1 <= k <= EVC_MAX_STEPS and ncol >= 1");
    if ((int64_t)k * ncol > EVC_STATIC_QUAD_MAX)
        return say(errbuf, errlen, EVC_EINVAL,
                   "k * ncol exceeds EVC_STATIC_QUAD_MAX (262144): split the columns");
    if (!std::isfinite(vnorm2) || vnorm2 < 0.0)
        return say(errbuf, errlen, EVC_EINVAL, "vnorm2 must be finite and >= 0");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return say(errbuf, errlen, EVC_ECUDA, "no current CUDA device");
    }
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> g(g_lock);
        if (!g_scratch_dev[dev]) {
            // once per device, with that device current: the host-side name of the
            // array is not a device address, so look the address up.
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_quad_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return say(errbuf, errlen, EVC_ECUDA, "cudaGetSymbolAddress of the scratch failed");
            }
            g_scratch_dev[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_dev[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (d_status) {
        // the status word starts at EVC_OK for this call (a memset, no allocation)
        cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(int), st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return say(errbuf, errlen, EVC_ECUDA, cudaGetErrorString(e));
        }
    }
    static_quad_kernel<<<(ncol + 127) / 128, 128, 0, st>>>(d_alpha, d_beta, d_kcol, k, ncol,
                                                            vnorm2, d_quad, scratch, d_status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return say(errbuf, errlen, EVC_ECUDA, cudaGetErrorString(e));
    return EVC_OK;
}
