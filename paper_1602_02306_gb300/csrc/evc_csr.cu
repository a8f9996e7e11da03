// evc_csr.cu -- the preconditioned shifted operator for a CSR matrix,
//   w = M (A - sigma_c I) M q_i - beta_i q_{i-1}       (Algorithm 1, first
// line of the loop body), with M = I or the Jacobi scaling
// M = diag((|a_rr - sigma| + eps)^(-1/2)) fused as row and column scales.
//
// One warp owns one row of one 32-column chunk: lanes are the probe columns,
// so every gathered x row is one contiguous 128-byte (FP32) / 256-byte
// (FP64) segment, and the row's (col, val) pairs are read once per chunk and
// broadcast through warp shuffles.  q_i = s_i P_i is scaled on the fly.
#include "evc_internal.cuh"

namespace evc {
namespace {

struct CArgs {
    CsrOp op;
    const void* x;          // slot i-1 of the basis (P_i)
    const void* pp;         // slot i-2 (P_{i-1}) or null
    void* out;              // slot i
    int64_t chunk_stride;
    const double* insc;     // s_i per column
    const double* ppc;      // beta_i s_{i-1} per column
    const double* sigma;
    const int* shift_of;
    const void* jac;
    const int* chunk_active;
};

template <typename T, bool JAC>
__global__ void __launch_bounds__(kThreads)
csr_pass_kernel(CArgs a)
{
    const int ch = blockIdx.y;
    if (!a.chunk_active[ch]) return;
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    if (row >= a.op.n) return;
    const int c = ch * CW + lane;
    const int64_t n = a.op.n;
    const T* x = static_cast<const T*>(a.x) + ch * a.chunk_stride;
    const T* val = static_cast<const T*>(a.op.val);
    const T* jr = JAC ? static_cast<const T*>(a.jac) + (int64_t)a.shift_of[c] * n : nullptr;

    const int64_t beg = a.op.row_ptr[row], end = a.op.row_ptr[row + 1];
    T acc0 = 0, acc1 = 0;
    for (int64_t k0 = beg; k0 < end; k0 += 32) {
        const int64_t kk = k0 + lane;
        int mycol = 0;
        T myval = 0;
        if (kk < end) {
            mycol = __ldg(a.op.col + kk);
            myval = __ldg(val + kk);
        }
        const int cnt = (int)min((int64_t)32, end - k0);
        int t = 0;
        for (; t + 1 < cnt; t += 2) {
            const int ca = __shfl_sync(0xffffffffu, mycol, t);
            const int cb = __shfl_sync(0xffffffffu, mycol, t + 1);
            const T va = __shfl_sync(0xffffffffu, myval, t);
            const T vb = __shfl_sync(0xffffffffu, myval, t + 1);
            T xa = __ldg(x + (int64_t)ca * CW + lane);
            T xb = __ldg(x + (int64_t)cb * CW + lane);
            if (JAC) { xa *= __ldg(jr + ca); xb *= __ldg(jr + cb); }
            acc0 += va * xa;
            acc1 += vb * xb;
        }
        if (t < cnt) {
            const int ca = __shfl_sync(0xffffffffu, mycol, t);
            const T va = __shfl_sync(0xffffffffu, myval, t);
            T xa = __ldg(x + (int64_t)ca * CW + lane);
            if (JAC) xa *= __ldg(jr + ca);
            acc0 += va * xa;
        }
    }
    T center = __ldg(x + row * CW + lane);
    T mr = 1;
    if (JAC) { mr = __ldg(jr + row); center *= mr; }
    T res = (acc0 + acc1) - (T)a.sigma[c] * center;
    if (JAC) res *= mr;
    res *= (T)a.insc[c];
    if (a.pp) {
        const T* pp = static_cast<const T*>(a.pp) + ch * a.chunk_stride;
        res -= (T)a.ppc[c] * pp[row * CW + lane];
    }
    static_cast<T*>(a.out)[ch * a.chunk_stride + row * CW + lane] = res;
}

}  // namespace

template <typename T>
cudaError_t launch_csr_pass(const CsrOp& op, const Run& r, int i, bool jacobi, cudaStream_t st)
{
    // step i reads slot i-1 (q_i), slot i-2 (q_{i-1}) and writes slot i
    CArgs a;
    a.op = op;
    T* basis = static_cast<T*>(r.basis);
    a.x = basis + (int64_t)(i - 1) * r.slot_stride;
    a.pp = i >= 2 ? basis + (int64_t)(i - 2) * r.slot_stride : nullptr;
    a.out = basis + (int64_t)i * r.slot_stride;
    a.chunk_stride = r.chunk_stride;
    a.insc = r.scl + (int64_t)(i - 1) * r.ncol;
    a.ppc = r.ppc;
    a.sigma = r.sigma;
    a.shift_of = r.shift_of;
    a.jac = r.jac;
    a.chunk_active = r.chunk_active;
    const int rows_per_block = kThreads / 32;
    dim3 grid((unsigned)((op.n + rows_per_block - 1) / rows_per_block), r.nchunk);
    if (jacobi) csr_pass_kernel<T, true><<<grid, kThreads, 0, st>>>(a);
    else csr_pass_kernel<T, false><<<grid, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_csr_pass<float>(const CsrOp&, const Run&, int, bool, cudaStream_t);
template cudaError_t launch_csr_pass<double>(const CsrOp&, const Run&, int, bool, cudaStream_t);

}  // namespace evc
