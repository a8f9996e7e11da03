// evc_arnoldi.cu -- the kernels of the preconditioned Arnoldi-type estimator
// (Sec. 4) that the Lanczos path does not already have.
//
//  * row_scale_kernel: w <- T w for the Jacobi preconditioner used without its
//    factorisation, T = diag(m^2), m the Jacobi scales of the Lanczos path.
//  * arnoldi_quad_kernel: the Arnoldi quadrature (Eq. arnoldi_quad)
//      ||v||^2 Re(e_1^T h(H_k) e_1),  h = 1 on the open left half-plane,
//    of each column's k x k upper Hessenberg matrix.  The paper writes it
//    through the eigen-decomposition H_k = Z Theta Z^{-1}; for a real H_k
//    with no eigenvalue on the imaginary axis the same number is
//      e_1^T h(H_k) e_1 = (1 - sign(H_k)_{11}) / 2,
//    and sign(H_k) is computed by Newton's iteration
//      X <- (mu X + (mu X)^{-1}) / 2,  mu = |det X|^{-1/k}  (determinant scaling),
//    which is real for a real H_k, so the real part comes for free.  One block
//    per column, all of it in FP64 shared memory; each inverse is a
//    Gauss-Jordan elimination with partial pivoting.
#include "evc_internal.cuh"

#include <algorithm>
#include <cmath>

namespace evc {
namespace {

constexpr int AQT = 256;               // threads of the quadrature kernel

__device__ __forceinline__ int64_t tri_a(int a, int b) { return (int64_t)a * (a + 1) / 2 + b; }

template <typename T>
__global__ void __launch_bounds__(kThreads)
row_scale_kernel(T* w, int64_t cs, const T* jac, const int* shift_of, const int* chunk_active,
                 int64_t n)
{
    const int ch = blockIdx.y;
    if (!chunk_active[ch]) return;
    const int lane = threadIdx.x & 31;
    const int s = shift_of[ch * CW + lane];
    T* wc = w + ch * cs;
    const T* js = jac + (int64_t)s * n;
    const int wpb = blockDim.x / 32;
    for (int64_t row = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); row < n;
         row += (int64_t)gridDim.x * wpb) {
        const T m = js[row];
        wc[row * CW + lane] *= m * m;
    }
}

__device__ double block_sum(double v, double* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < AQT / 32; ++q) t += red[q];
    return t;
}

__global__ void __launch_bounds__(AQT)
arnoldi_quad_kernel(Run r, int i)
{
    extern __shared__ double sm[];
    __shared__ double red[AQT / 32];
    __shared__ double s_logdet, s_pv;
    __shared__ int s_piv, s_bad;
    const int c = blockIdx.x;
    if (r.sdone[r.shift_of[c]]) return;                   // uniform over the block
    const int k = r.kdone[c] ? min(r.kdone[c], i) : i;
    const int k2 = 2 * k;
    double* X = sm;                  // [k][k]
    double* G = X + k * k;           // [k][2k]: [X | I] -> [I | X^{-1}]
    double* f = G + 2 * k * k;       // [k]: column of elimination factors
    const int tid = threadIdx.x;
    // H_k: column j holds h_{1..j+1, j+1} (packed) and below it beta_{j+2}
    for (int e = tid; e < k * k; e += AQT) {
        const int row = e / k, col = e % k;
        double v = 0.0;
        if (row <= col) v = r.hess[tri_a(col, row) * r.ncol + c];
        else if (row == col + 1) v = r.beta[(int64_t)(col + 1) * r.ncol + c];
        X[e] = v;
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    // Newton's iteration converges quadratically once every eigenvalue is
    // scaled near +-1; one that has not met the tolerance after 100 steps (an
    // eigenvalue of H_k close to the imaginary axis) is reported as a numeric
    // failure instead of a quadrature from an unconverged X.
    bool converged = false;
    for (int it = 0; it < 100; ++it) {
        for (int e = tid; e < k * k2; e += AQT) {
            const int row = e / k2, col = e % k2;
            G[e] = col < k ? X[row * k + col] : (col - k == row ? 1.0 : 0.0);
        }
        if (tid == 0) s_logdet = 0.0;
        __syncthreads();
        for (int p = 0; p < k; ++p) {
            if (tid < 32) {
                double best = -1.0;
                int br = p;
                for (int rr = p + tid; rr < k; rr += 32) {
                    const double a = fabs(G[rr * k2 + p]);
                    if (a > best) {
                        best = a;
                        br = rr;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int orr = __shfl_xor_sync(0xffffffffu, br, o);
                    if (ob > best || (ob == best && orr < br)) {
                        best = ob;
                        br = orr;
                    }
                }
                if (tid == 0) {
                    s_piv = br;
                    s_pv = G[br * k2 + p];
                    if (!(best > 0.0)) s_bad = 1;
                    else s_logdet += log(best);
                }
            }
            __syncthreads();
            if (s_bad) break;
            const int pr = s_piv;
            if (pr != p) {
                for (int q = tid; q < k2; q += AQT) {
                    const double t = G[p * k2 + q];
                    G[p * k2 + q] = G[pr * k2 + q];
                    G[pr * k2 + q] = t;
                }
                __syncthreads();
            }
            const double inv = 1.0 / s_pv;
            for (int q = tid; q < k2; q += AQT) G[p * k2 + q] *= inv;
            for (int rr = tid; rr < k; rr += AQT) f[rr] = G[rr * k2 + p];   // row p unused below
            __syncthreads();
            for (int e = tid; e < k * k2; e += AQT) {
                const int rr = e / k2, q = e % k2;
                if (rr != p) G[e] -= f[rr] * G[p * k2 + q];
            }
            __syncthreads();
        }
        if (s_bad) break;
        const double mu = exp(-s_logdet / k);
        double dloc = 0.0, nloc = 0.0;
        for (int e = tid; e < k * k; e += AQT) {
            const int row = e / k, col = e % k;
            const double xn = 0.5 * (mu * X[e] + G[row * k2 + k + col] / mu);
            dloc += (xn - X[e]) * (xn - X[e]);
            nloc += xn * xn;
            X[e] = xn;
        }
        const double dn = block_sum(dloc, red);
        const double nn = block_sum(nloc, red);
        __syncthreads();
        if (!(dn > 1e-28 * nn)) {          // converged (uniform: every thread sees the same sums)
            converged = true;
            break;
        }
    }
    if (tid == 0) {
        double q = (double)r.n * 0.5 * (1.0 - X[0]);
        if (s_bad || !converged || !isfinite(q)) {
            atomicExch(r.err, DERR_NUMERIC);
            q = 0.0;
        }
        r.quad[c] = q;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_row_scale(const Run& r, void* w, int64_t cs, cudaStream_t st)
{
    const int wpb = kThreads / 32;
    const int64_t blocks = std::min<int64_t>((r.n + wpb - 1) / wpb, 4096);
    row_scale_kernel<T><<<dim3((unsigned)blocks, r.nchunk), kThreads, 0, st>>>(
        static_cast<T*>(w), cs, static_cast<const T*>(r.jac), r.shift_of, r.chunk_active, r.n);
    return cudaGetLastError();
}

template cudaError_t launch_row_scale<float>(const Run&, void*, int64_t, cudaStream_t);
template cudaError_t launch_row_scale<double>(const Run&, void*, int64_t, cudaStream_t);

cudaError_t launch_arnoldi_quad(const Run& r, int i, cudaStream_t st)
{
    if (i > kArnoldiMaxSteps) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(3 * i * i + i) * sizeof(double);
    static std::atomic<uint64_t> attr{0};
    const size_t mx = (size_t)(3 * kArnoldiMaxSteps * kArnoldiMaxSteps + kArnoldiMaxSteps) *
                      sizeof(double);
    const cudaError_t e = smem_limit_once(attr, arnoldi_quad_kernel, mx);
    if (e != cudaSuccess) return e;
    arnoldi_quad_kernel<<<r.ncol_real, AQT, smem, st>>>(r, i);
    return cudaGetLastError();
}

}  // namespace evc
