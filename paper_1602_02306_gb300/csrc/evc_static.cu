// evc_static.cu -- allocation-free batched Gauss quadrature (see
// evc_gauss_quadrature_static in include/evc.h).  The eigensolver scratch
// lives in one file-scope device array instead of caller- or library-
// allocated memory, for callers that cannot allocate device memory.
#include "evc_internal.cuh"
#include "evc_tridiag.cuh"
#include "../../include/evc.h"

#include <cstdio>
#include <mutex>

namespace {

// 3 * EVC_STATIC_QUAD_MAX doubles (6 MiB) on every device that loads the library.
__device__ __align__(256) double g_quad_scratch[3 * EVC_STATIC_QUAD_MAX];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
double* g_scratch_dev[kMaxDevices] = {};

__global__ void static_quad_kernel(const double* alpha, const double* beta, const int* kcol,
                                   int k, int ncol, double vnorm2, double* quad, double* scratch)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    int kc = kcol ? kcol[c] : k;
    kc = kc < 1 ? 1 : (kc > k ? k : kc);
    // scratch layout [3][k][ncol]: d, e, z, coalesced across columns
    const int64_t plane = (int64_t)k * ncol;
    double q = evc::tridiag_gauss_quadrature(alpha + c, beta + c, ncol, kc, vnorm2, scratch + c,
                                             scratch + plane + c, scratch + 2 * plane + c, ncol);
    quad[c] = q;   // -1 when the eigensolver did not converge
}

int say(char* buf, size_t len, int code, const char* msg)
{
    if (buf && len) snprintf(buf, len, "%s", msg);
    return code;
}

}  // namespace

extern "C" int evc_gauss_quadrature_static(const double* d_alpha, const double* d_beta,
                                           const int* d_kcol, int k, int ncol, double vnorm2,
                                           double* d_quad, void* stream, char* errbuf,
                                           size_t errlen)
{
    if (!d_alpha || !d_beta || !d_quad)
        return say(errbuf, errlen, EVC_EINVAL, "null device pointer");
    if (k < 1 || k > EVC_MAX_STEPS || ncol < 1)
        return say(errbuf, errlen, EVC_EINVAL, "need 1 <= k <= EVC_MAX_STEPS and ncol >= 1");
    if ((int64_t)k * ncol > EVC_STATIC_QUAD_MAX)
        return say(errbuf, errlen, EVC_EINVAL,
                   "k * ncol exceeds EVC_STATIC_QUAD_MAX (262144): split the columns");
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
    static_quad_kernel<<<(ncol + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(
        d_alpha, d_beta, d_kcol, k, ncol, vnorm2, d_quad, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return say(errbuf, errlen, EVC_ECUDA, cudaGetErrorString(e));
    return EVC_OK;
}
