// evc_reorth.cu -- the vector part of the Lanczos step after the operator
// apply (Algorithm 1), the batched tridiagonal eigensolve with Gauss
// quadrature (Eq. gauss_quad) and the per-shift estimator (Algorithm 2).
//
// Per step i, for every column c (w = C q_i - beta_i q_{i-1} is in slot i):
//   dots    h_j = q_j^T w and G_ij = q_j^T q_i, j = 1..i, in one sweep over
//           the basis (partials per row block)
//   reduce  h, the new Gram row, alpha_i = h_i       (FP64, fixed order)
//   coef    c = h + (I - G) h                        (FP64, per column)
//   update  w <- w - Q_i c;  ||w||^2 partials
//   finish  beta_{i+1} = ||w||, s_{i+1} = 1/beta_{i+1}, breakdown test,
//           eig(J_i) -> quadrature, per-shift mean L(i) and stop rule.
// In exact arithmetic G = I, c = h, and the single fused classical
// Gram-Schmidt sweep equals Algorithm 1's "alpha_i = q_i^T w;
// w -= alpha_i q_i; w -= Q_i (Q_i^T w)" (the second projection's i-th
// coefficient is then zero).  In floating point the stored basis is
// orthonormal only to the working precision; the term (I - G) h is the
// second Gram-Schmidt pass Q_i^T (w - Q_i h) = (I - G) h evaluated from the
// Gram matrix instead of a second sweep over the vectors, which keeps the
// FP32 basis as orthogonal as two full passes would (CGS2) at the cost of
// one pass.  The Gram row of q_i is formed in the same sweep as Q_i^T w.
//
// Reductions are deterministic: per-thread partial sums over a fixed row
// set (FP32 runs of 16 rows promoted to FP64 in mixed mode), a fixed
// shared-memory tree, then a fixed-order sum over row blocks.  A column's
// result does not depend on which other columns share the launch.
#include "evc_internal.cuh"
#include "evc_tridiag.cuh"

#include <cmath>

namespace evc {
namespace {

constexpr int JB = 8;          // basis vectors per pass of the dot kernel
constexpr int RUN = 16;        // rows per FP32 partial-sum run
constexpr int WARPS = kThreads / 32;
static_assert(JB == WARPS, "the dot kernel's warp tree maps warp q to basis vector jg + q");

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    // SplitMix64 output finaliser (Steele, Lea & Flood 2014).
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

template <typename T>
__global__ void init_probe_kernel(Run r)
{
    // slot 0 of every chunk: the Rademacher probe v (Sec. 2, Eq. trace)
    const uint64_t seed = *r.seed;
    const int64_t total = (int64_t)r.nchunk * r.n * CW;
    T* basis = static_cast<T*>(r.basis);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int lane = (int)(e % CW);
        const int64_t row = (e / CW) % r.n;
        const int ch = (int)(e / (CW * r.n));
        const int c = ch * CW + lane;
        const uint64_t j = (uint64_t)r.probe_id[c];
        const uint64_t xh = mix64(seed ^ mix64((j << 32) | (uint64_t)row));
        basis[ch * r.chunk_stride + row * CW + lane] = (xh >> 63) ? (T)-1 : (T)1;
    }
}

__global__ void init_state_kernel(Run r)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < r.ncol) {
        r.scl[t] = 1.0 / sqrt((double)r.n);   // q_1 = v/||v||, ||v||^2 = n
        r.beta[t] = 0.0;                      // beta_1 = 0
        r.ppc[t] = 0.0;
        r.colscale[t] = 0.0;
        r.kdone[t] = 0;
        r.quad[t] = 0.0;
        r.quad_final[t] = 0.0;
    }
    if (t < r.S) {
        r.sdone[t] = 0;
        r.Lprev[t] = 0.0;
        r.Lfinal[t] = 0.0;
        r.steps[t] = 0;
    }
    if (t < r.nchunk) r.chunk_active[t] = 1;
    if (t == 0) *r.err = DERR_NONE;
}

template <typename T>
__global__ void jacobi_scale_kernel(Run r, const double* diag, const T* V, double vdiag, double eps)
{
    // M = diag((|a_rr - tau| + eps)^(-1/2)) per shift
    const int64_t total = (int64_t)r.S * r.n;
    T* jac = static_cast<T*>(r.jac);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(e / r.n);
        const int64_t row = e % r.n;
        const double d = diag ? diag[row] : (double)V[row] + vdiag;
        jac[e] = (T)(1.0 / sqrt(fabs(d - r.shifts[s]) + eps));
    }
}

template <typename T> struct Acc { typedef float run; };
template <> struct Acc<double> { typedef double run; };

__device__ __forceinline__ void row_range(int64_t n, int nblk, int blk, int64_t& r0, int64_t& r1)
{
    const int64_t per = (n + nblk - 1) / nblk;
    r0 = (int64_t)blk * per;
    r1 = min(n, r0 + per);
}

// part_dot[ch][blk][j][lane]  = sum_{rows of blk} P_j[row][lane] * w[row][lane]
// part_gram[ch][blk][j][lane] = sum_{rows of blk} P_j[row][lane] * P_{i-1}[row][lane]
// for j < i.  The block walks its rows in slabs of WARPS*RTD rows; each warp
// holds RTD-row tiles of w and of P_{i-1} in registers and streams JB basis
// tiles at a time against both (independent loads).  Tile sums (FP32 runs of
// RTD rows in mixed mode) go through a fixed shared-memory tree into per-block
// FP64 accumulators, so the summation order is fixed and w is read once.
constexpr int RT = 16;          // rows per warp tile (update)
constexpr int RTD = 8;          // rows per warp tile (dots)

template <typename T>
__global__ void __launch_bounds__(kThreads)
reorth_dots_kernel(Run r, int i)
{
    const int ch = blockIdx.y, blk = blockIdx.x;
    if (!r.chunk_active[ch]) return;
    extern __shared__ double sm[];
    double* bacc = sm;                              // [i][CW]
    double* bgram = sm + (size_t)i * CW;            // [i][CW]
    double* red = sm + (size_t)2 * i * CW;          // [WARPS][2*JB][CW]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < 2 * i * CW; e += blockDim.x) sm[e] = 0.0;
    int64_t r0, r1;
    row_range(r.n, r.nblk, blk, r0, r1);
    const T* __restrict__ P = static_cast<const T*>(r.basis) + ch * r.chunk_stride;
    const T* __restrict__ w = P + (int64_t)i * r.slot_stride;
    const T* __restrict__ q = P + (int64_t)(i - 1) * r.slot_stride;
    typedef typename Acc<T>::run RTy;
    for (int64_t base = r0; base < r1; base += (int64_t)WARPS * RTD) {
        const int64_t t0 = base + (int64_t)warp * RTD;
        T wv[RTD], qv[RTD];
#pragma unroll
        for (int t = 0; t < RTD; ++t) {
            const bool ok = t0 + t < r1;
            wv[t] = ok ? __ldg(w + (t0 + t) * CW + lane) : (T)0;
            qv[t] = ok ? __ldg(q + (t0 + t) * CW + lane) : (T)0;
        }
        for (int jg = 0; jg < i; jg += JB) {
            RTy a[JB], b[JB];
#pragma unroll
            for (int jj = 0; jj < JB; ++jj) { a[jj] = 0; b[jj] = 0; }
#pragma unroll
            for (int jj = 0; jj < JB; ++jj) {
                if (jg + jj < i) {
                    const T* __restrict__ Pj = P + (int64_t)(jg + jj) * r.slot_stride + t0 * CW + lane;
#pragma unroll
                    for (int t = 0; t < RTD; ++t)
                        if (t0 + t < r1) {
                            const RTy pj = (RTy)__ldg(Pj + t * CW);
                            a[jj] += pj * (RTy)wv[t];
                            b[jj] += pj * (RTy)qv[t];
                        }
                }
            }
#pragma unroll
            for (int jj = 0; jj < JB; ++jj) {
                red[((size_t)warp * 2 * JB + jj) * CW + lane] = (double)a[jj];
                red[((size_t)warp * 2 * JB + JB + jj) * CW + lane] = (double)b[jj];
            }
            __syncthreads();
            if (jg + warp < i) {
                double sa = 0.0, sb = 0.0;
#pragma unroll
                for (int qq = 0; qq < WARPS; ++qq) {
                    sa += red[((size_t)qq * 2 * JB + warp) * CW + lane];
                    sb += red[((size_t)qq * 2 * JB + JB + warp) * CW + lane];
                }
                bacc[(size_t)(jg + warp) * CW + lane] += sa;
                bgram[(size_t)(jg + warp) * CW + lane] += sb;
            }
            __syncthreads();
        }
    }
    for (int e = threadIdx.x; e < i * CW; e += blockDim.x) {
        const int64_t o = (((int64_t)ch * r.nblk + blk) * r.kmax + e / CW) * CW + (e % CW);
        r.part_dot[o] = bacc[e];
        r.part_gram[o] = bgram[e];
    }
}

__device__ __forceinline__ int64_t tri(int a, int b)
{
    // packed lower triangle, a >= b
    return (int64_t)a * (a + 1) / 2 + b;
}

// h_j = s_j * sum_blk part_dot;  G_{i-1,j} = s_{i-1} s_j * sum_blk part_gram;
// alpha_i = h_{i-1}  (slot j holds q_{j+1})
__global__ void reorth_reduce_kernel(Run r, int i)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= r.ncol * i) return;
    const int c = t % r.ncol, j = t / r.ncol;
    const int ch = c / CW, lane = c % CW;
    if (!r.chunk_active[ch]) return;
    double sh = 0.0, sg = 0.0;
    for (int b = 0; b < r.nblk; ++b) {
        const int64_t o = (((int64_t)ch * r.nblk + b) * r.kmax + j) * CW + lane;
        sh += r.part_dot[o];
        sg += r.part_gram[o];
    }
    const double sj = r.scl[(int64_t)j * r.ncol + c];
    const double si = r.scl[(int64_t)(i - 1) * r.ncol + c];
    const double h = sh * sj;
    r.hbuf[(int64_t)j * r.ncol + c] = h;
    r.gram[tri(i - 1, j) * r.ncol + c] = sg * sj * si;
    if (j == i - 1) r.alpha[(int64_t)(i - 1) * r.ncol + c] = h;
}

// c = h + (I - G) h, g_j = c_j s_j (coefficients of the unnormalised P_j)
__global__ void reorth_coef_kernel(Run r, int i)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= r.ncol) return;
    if (!r.chunk_active[c / CW]) return;
    for (int j = 0; j < i; ++j) {
        double gh = 0.0;
        for (int l = 0; l < i; ++l) {
            const double G = r.gram[(j >= l ? tri(j, l) : tri(l, j)) * r.ncol + c];
            gh += G * r.hbuf[(int64_t)l * r.ncol + c];
        }
        const double hj = r.hbuf[(int64_t)j * r.ncol + c];
        r.g[(int64_t)j * r.ncol + c] = (2.0 * hj - gh) * r.scl[(int64_t)j * r.ncol + c];
    }
}

// w <- w - sum_{j<i} g_j P_j (in place, slot i); part_nrm = partial ||w||^2.
// Same warp tiling as the dot kernel: the w tile lives in registers while
// every P_j tile streams past it.
template <typename T>
__global__ void __launch_bounds__(kThreads)
reorth_update_kernel(Run r, int i)
{
    const int ch = blockIdx.y, blk = blockIdx.x;
    if (!r.chunk_active[ch]) return;
    extern __shared__ unsigned char smem_raw[];
    T* gs = reinterpret_cast<T*>(smem_raw);            // [i][CW]
    __shared__ double red[WARPS][CW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < i * CW; e += blockDim.x)
        gs[e] = (T)r.g[(int64_t)(e / CW) * r.ncol + ch * CW + (e % CW)];
    __syncthreads();
    int64_t r0, r1;
    row_range(r.n, r.nblk, blk, r0, r1);
    const T* __restrict__ P = static_cast<const T*>(r.basis) + ch * r.chunk_stride;
    T* __restrict__ w = static_cast<T*>(r.basis) + ch * r.chunk_stride + (int64_t)i * r.slot_stride;
    typedef typename Acc<T>::run RTy;
    double acc = 0.0;
    for (int64_t t0 = r0 + (int64_t)warp * RT; t0 < r1; t0 += (int64_t)WARPS * RT) {
        T wv[RT];
#pragma unroll
        for (int t = 0; t < RT; ++t) wv[t] = (t0 + t < r1) ? w[(t0 + t) * CW + lane] : (T)0;
#pragma unroll 2
        for (int j = 0; j < i; ++j) {
            const T gj = gs[j * CW + lane];
            const T* __restrict__ Pj = P + (int64_t)j * r.slot_stride + t0 * CW + lane;
#pragma unroll
            for (int t = 0; t < RT; ++t)
                if (t0 + t < r1) wv[t] -= gj * __ldg(Pj + t * CW);
        }
        RTy nr = 0;
#pragma unroll
        for (int t = 0; t < RT; ++t)
            if (t0 + t < r1) {
                w[(t0 + t) * CW + lane] = wv[t];
                nr += (RTy)wv[t] * (RTy)wv[t];
            }
        acc += (double)nr;
    }
    red[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < WARPS; ++q) s += red[q][lane];
        r.part_nrm[((int64_t)ch * r.nblk + blk) * CW + lane] = s;
    }
}

// Gauss quadrature of column c's J_k; eigensolver scratch in the workspace,
// [3][kmax][ncol] (coalesced across columns).
__device__ double gauss_quadrature(const Run& r, int c, int k, double vnorm2)
{
    const int64_t plane = (int64_t)r.kmax * r.ncol;
    return tridiag_gauss_quadrature(r.alpha + c, r.beta + c, r.ncol, k, vnorm2, r.eigw + c,
                                    r.eigw + plane + c, r.eigw + 2 * plane + c, r.ncol);
}

// One block per shift (block S handles the padding columns).
__global__ void __launch_bounds__(kThreads)
finish_kernel(Run r, int i, int do_quad, int last)
{
    const int s = blockIdx.x;
    const bool real = s < r.S;
    if (real && r.sdone[s]) return;
    const int cbeg = real ? s * r.m : r.ncol_real;
    const int cend = real ? cbeg + r.m : r.ncol;
    __shared__ double red[kThreads];
    __shared__ int stop;
    double lsum = 0.0;
    for (int c = cbeg + threadIdx.x; c < cend; c += blockDim.x) {
        const int ch = c / CW, lane = c % CW;
        if (r.kdone[c] == 0) {
            double nrm2 = 0.0;
            for (int b = 0; b < r.nblk; ++b)
                nrm2 += r.part_nrm[((int64_t)ch * r.nblk + b) * CW + lane];
            const double beta = sqrt(nrm2);
            const double al = r.alpha[(int64_t)(i - 1) * r.ncol + c];
            const double bprev = r.beta[(int64_t)(i - 1) * r.ncol + c];
            double sc = fmax(r.colscale[c], fmax(fabs(al), bprev));
            r.colscale[c] = sc;
            r.beta[(int64_t)i * r.ncol + c] = beta;
            if (!isfinite(beta) || !isfinite(al)) {
                if (real) atomicExch(r.err, DERR_NUMERIC);
                r.kdone[c] = i;
                r.scl[(int64_t)i * r.ncol + c] = 0.0;
                r.ppc[c] = 0.0;
            } else if (beta <= r.breakdown_rel * sc || (int64_t)i >= r.n) {
                // Lanczos breakdown: J_i is exact (Sec. 3, Proposition 1 argument)
                r.kdone[c] = i;
                r.scl[(int64_t)i * r.ncol + c] = 0.0;
                r.ppc[c] = 0.0;
            } else {
                r.scl[(int64_t)i * r.ncol + c] = 1.0 / beta;
                r.ppc[c] = beta * r.scl[(int64_t)(i - 1) * r.ncol + c];
            }
        }
        if (do_quad && real) {
            const int k = r.kdone[c] ? min(r.kdone[c], i) : i;
            double q = gauss_quadrature(r, c, k, (double)r.n);
            if (q < 0.0) {
                atomicExch(r.err, DERR_NUMERIC);
                q = 0.0;
            }
            r.quad[c] = q;
            lsum += q;
        }
    }
    if (!real || !do_quad) return;
    // L_s(i) = mean_j quad_j: fixed-shape shared-memory tree
    red[threadIdx.x] = lsum;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double L = red[0] / r.m;
        const double tol = *r.tol;
        int st = last ? 1 : 0;
        if (tol > 0.0 && i >= 2 && fabs(L - r.Lprev[s]) <= tol) st = 1;
        r.Lprev[s] = L;
        if (st) {
            r.sdone[s] = 1;
            r.steps[s] = i;
            r.Lfinal[s] = L;
        }
        stop = st;
    }
    __syncthreads();
    if (stop)
        for (int c = cbeg + threadIdx.x; c < cend; c += blockDim.x) {
            // freeze the column: its later vectors become exact zeros
            r.quad_final[c] = r.quad[c];
            r.ppc[c] = 0.0;
            for (int j = i; j <= r.kmax; ++j) r.scl[(int64_t)j * r.ncol + c] = 0.0;
            if (!r.kdone[c]) r.kdone[c] = i;
        }
}

// A chunk stays active while one of its real columns belongs to a running shift.
__global__ void active_kernel(Run r)
{
    const int ch = blockIdx.x * blockDim.x + threadIdx.x;
    if (ch >= r.nchunk) return;
    int act = 0;
    for (int l = 0; l < CW; ++l) {
        const int c = ch * CW + l;
        if (c < r.ncol_real && !r.sdone[r.shift_of[c]]) act = 1;
    }
    r.chunk_active[ch] = act;
}

}  // namespace

cudaError_t launch_init_state(const Run& r, cudaStream_t st)
{
    const int nstate = max(max(r.ncol, r.S), r.nchunk);
    init_state_kernel<<<(nstate + 255) / 256, 256, 0, st>>>(r);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_probe(const Run& r, cudaStream_t st)
{
    const int64_t total = (int64_t)r.nchunk * r.n * CW;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
    init_probe_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(r);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_jacobi_scales(const Run& r, const double* diag, const void* V, double vdiag,
                                 double eps, cudaStream_t st)
{
    const int64_t total = (int64_t)r.S * r.n;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
    jacobi_scale_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(r, diag, static_cast<const T*>(V),
                                                             vdiag, eps);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dots(const Run& r, int i, cudaStream_t st)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(reorth_dots_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((2 * kMaxSteps + 2 * WARPS * JB) * CW * sizeof(double)));
        attr_set = true;
    }
    const size_t smem = ((size_t)2 * i + 2 * WARPS * JB) * CW * sizeof(double);
    reorth_dots_kernel<T><<<dim3(r.nblk, r.nchunk), kThreads, smem, st>>>(r, i);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const Run& r, int i, cudaStream_t st)
{
    const int tot = r.ncol * i;
    reorth_reduce_kernel<<<(tot + 255) / 256, 256, 0, st>>>(r, i);
    return cudaGetLastError();
}

cudaError_t launch_coef(const Run& r, int i, cudaStream_t st)
{
    reorth_coef_kernel<<<(r.ncol + 127) / 128, 128, 0, st>>>(r, i);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update(const Run& r, int i, cudaStream_t st)
{
    const size_t smem = (size_t)i * CW * sizeof(T);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(reorth_update_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kMaxSteps * CW * sizeof(T)));
        attr_set = true;
    }
    reorth_update_kernel<T><<<dim3(r.nblk, r.nchunk), kThreads, smem, st>>>(r, i);
    return cudaGetLastError();
}

cudaError_t launch_finish(const Run& r, int i, bool do_quad, bool last, cudaStream_t st)
{
    const int nb = r.S + (r.ncol > r.ncol_real ? 1 : 0);
    finish_kernel<<<nb, kThreads, 0, st>>>(r, i, do_quad ? 1 : 0, last ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_active(const Run& r, cudaStream_t st)
{
    active_kernel<<<(r.nchunk + 127) / 128, 128, 0, st>>>(r);
    return cudaGetLastError();
}

template cudaError_t launch_init_probe<float>(const Run&, cudaStream_t);
template cudaError_t launch_init_probe<double>(const Run&, cudaStream_t);
template cudaError_t launch_jacobi_scales<float>(const Run&, const double*, const void*, double,
                                                 double, cudaStream_t);
template cudaError_t launch_jacobi_scales<double>(const Run&, const double*, const void*, double,
                                                  double, cudaStream_t);
template cudaError_t launch_dots<float>(const Run&, int, cudaStream_t);
template cudaError_t launch_dots<double>(const Run&, int, cudaStream_t);
template cudaError_t launch_update<float>(const Run&, int, cudaStream_t);
template cudaError_t launch_update<double>(const Run&, int, cudaStream_t);

}  // namespace evc
