// evc_reorth.cu -- the vector part of the Lanczos step after the operator
// apply (Algorithm 1), the batched tridiagonal eigensolve with Gauss
// quadrature (Eq. gauss_quad) and the per-shift estimator (Algorithm 2).
//
// Per step i, for every column c (w = C q_i - beta_i q_{i-1} is in slot i):
//   dots    h_j = q_j^T w and G_ij = q_j^T q_i, j = 1..i, in one sweep over
//           the basis (partials per row block)
//   reduce  sums the partials (FP64, fixed order): h, the new Gram row,
//           alpha_i = h_i
//   coef    c = h + (I - G) h
//   update  w <- w - Q_i c;  ||w||^2 partials; its last block per chunk sets
//           beta_{i+1} = ||w||, s_{i+1} = 1/beta_{i+1} and the breakdown test
//   finish  eig(J_i) -> quadrature, per-shift mean L(i) and stop rule
//           (every step under a tolerance, else once after the last step).
// T^{-1}-inner-product mode (Sec. 4, Eq. lanT1, Jacobi T = M^2): the basis
// holds y_j = M q_j, w = T (A - sigma I) y_i - beta_i y_{i-1}, and every inner
// product above is <x, y> = x^T T^{-1} y -- the dot kernel weights w and y_i
// by T^{-1} on load, the update kernel weights the norm -- so the same
// coefficients, Gram matrix and J_i come out (Y_i = M Q_i).
//
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
#include "evc_bulk.cuh"

#include <cuda_bf16.h>

#include <cmath>

namespace evc {
namespace {

constexpr int JB = 8;          // basis vectors per pass of the dot kernel
constexpr int WARPS = kThreads / 32;
static_assert(JB == WARPS, "the dot kernel's warp tree maps warp q to basis vector jg + q");

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    // SplitMix64 output finaliser (Steele, Lea & Flood 2014).
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Correctly rounded square roots in the working precision (an FP64 root per
// element would make the FP32 probe set-up FP64-bound).
__device__ __forceinline__ float sqrt_rn(float x) { return __fsqrt_rn(x); }
__device__ __forceinline__ double sqrt_rn(double x) { return __dsqrt_rn(x); }

template <typename T>
__global__ void init_probe_kernel(Run r)
{
    // slot 0 of every chunk: the Rademacher probe v (Sec. 2, Eq. trace); in
    // T^{-1} mode M v (y_1 = M q_1, Sec. 4), m = sqrt of the stored T = m^2
    const uint64_t seed = *r.seed;
    const int64_t total = (int64_t)r.nchunk * r.n * CW;
    T* basis = static_cast<T*>(r.basis);
    const T* tdiag = static_cast<const T*>(r.jac);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int lane = (int)(e % CW);
        const int64_t row = (e / CW) % r.n;
        const int ch = (int)(e / (CW * r.n));
        const int c = ch * CW + lane;
        const uint64_t j = (uint64_t)r.probe_id[c];
        const uint64_t xh = mix64(seed ^ mix64((j << 32) | (uint64_t)row));
        T v = (xh >> 63) ? (T)-1 : (T)1;
        if (r.tinv) v *= sqrt_rn(tdiag[(int64_t)r.shift_of[c] * r.n + row]);
        basis[ch * r.chunk_stride + row * CW + lane] = v;
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
    }
    if (t < r.nq) {
        r.quad[t] = 0.0;
        r.quad_final[t] = 0.0;
    }
    if (t < r.S) {
        r.sdone[t] = 0;
        r.Lprev[t] = 0.0;
        r.Lprev2[t] = 0.0;
        r.Lfinal[t] = 0.0;
        r.steps[t] = 0;
    }
    if (t <= r.kmax) r.nactive[t] = r.nchunk;
    if (t < r.nchunk) {
        r.chunk_active[t] = 1;
        r.cnt_upd[t] = 0;
    }
    if (t == 0) *r.err = DERR_NONE;
}

template <typename T>
__global__ void jacobi_scale_kernel(Run r, const double* diag, const T* V, double vdiag, double eps,
                                    int form)
{
    // M = diag((|a_rr - tau| + eps)^(-1/2)) per shift, and (CSR) the diagonal
    // of the shifted operator: (a_rr - tau) m_r^2 when M or T = M^2 scales it,
    // else a_rr - tau.  In T^{-1} mode (form PM_TLEFT) jac holds T = m_r^2 and
    // tinvd T^{-1} = |a_rr - tau| + eps.  All from the FP64 diagonal, rounded
    // once at the end: near a_rr = tau, m_r^2 = 1/(|a_rr - tau| + eps)
    // amplifies an error in a_rr by up to 1/eps, so none may be formed from
    // rounded values.
    const int64_t total = (int64_t)r.Sop * r.n;
    T* jac = static_cast<T*>(r.jac);
    T* dsh = static_cast<T*>(r.dsh);
    T* tinvd = static_cast<T*>(r.tinvd);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(e / r.n);
        const int64_t row = e % r.n;
        const double d = diag ? diag[row] : (double)V[row] + vdiag;
        const double x = d - r.opshift[s];
        const double m2 = 1.0 / (fabs(x) + eps);
        if (jac) jac[e] = (T)(form == PM_TLEFT ? m2 : sqrt(m2));
        if (dsh) dsh[e] = (T)(form != PM_NONE ? x * m2 : x);
        if (tinvd) tinvd[e] = (T)(fabs(x) + eps);
    }
}

// Bulk copy with its preconditions checked first: a 16-byte aligned source
// inside [lo, hi), a 16-byte aligned destination, a size that is a positive
// multiple of 16.  A violation records DERR_BOUNDS and skips the copy (the
// waiting consumers then give up through their bounded waits).
__device__ __forceinline__ bool checked_bulk(void* dst, const void* src, uint32_t bytes,
                                             uint64_t* bar, const void* lo, const void* hi,
                                             int* err)
{
    const char* s = static_cast<const char*>(src);
    const bool ok = bytes > 0 && (bytes & 15) == 0 && ((uintptr_t)src & 15) == 0 &&
                    ((uintptr_t)smem_addr(dst) & 15) == 0 && s >= static_cast<const char*>(lo) &&
                    s + bytes <= static_cast<const char*>(hi);
    if (!ok) {
        atomicExch(err, DERR_BOUNDS);
        return false;
    }
    bulk_g2s(dst, src, bytes, bar);
    return true;
}

template <typename T> struct Acc { typedef float run; };
template <> struct Acc<double> { typedef double run; };

__device__ __forceinline__ void row_range(int64_t n, int nblk, int blk, int64_t& r0, int64_t& r1)
{
    const int64_t per = (n + nblk - 1) / nblk;
    r0 = (int64_t)blk * per;
    r1 = min(n, r0 + per);
}

// Streaming layout of the two reorthogonalisation kernels.  Each block owns
// a contiguous row range of one chunk and walks it in row tiles.  One
// producer warp issues asynchronous bulk copies (cp.async.bulk, mbarrier
// completion) of every basis tile P_j[tile] into a ring of shared-memory
// stages, so the bytes in flight are set by shared memory, not registers;
// eight consumer warps compute from shared memory and release the stages.
constexpr int CWARPS = 8;                       // consumer warps
constexpr int DSTAGE = 4096;                    // bytes per stage, dot kernel
constexpr int NSW = 2;                          // stages per consumer warp, dot kernel
constexpr int NPROD = 2;                        // producer warps, dot kernel
constexpr int DTHREADS = (CWARPS + NPROD) * 32; // threads of the dot kernel
static_assert(CWARPS % NPROD == 0, "a consumer warp's ring must have one producer");
constexpr int DNS = CWARPS * NSW;               // stages, dot kernel
constexpr int USTAGE = 8192;                    // bytes per stage, update kernel
constexpr int UNS = 10;                         // stages, update kernel
constexpr int UWARPS = CWARPS + NPROD;          // warps of the update kernel
constexpr int UTHREADS = UWARPS * 32;           // threads of the update kernel
static_assert(UNS % NPROD == 0, "a stage of the update ring must have one producer");

// part_dot[ch][blk][j][lane]  = sum_{rows of blk} P_j[row][lane] * w[row][lane]
// part_gram[ch][blk][j][lane] = sum_{rows of blk} P_j[row][lane] * P_{i-1}[row][lane]
// for j < i.  Consumer warp q handles the basis vectors j = q, q+8, ...: it
// holds the w and P_{i-1} tiles of the current row tile in registers and
// owns the FP64 accumulators of its j's in shared memory, so every sum has a
// fixed order (tiles in row order, FP32 runs of one tile in mixed mode).
// Each consumer warp has its own ring of NSW stages, so the item a warp
// waits for is always one phase ahead of the previous item in that stage,
// which the same warp consumed (mbarrier parities cannot alias).
// TW (T^{-1}-inner-product mode): every w and q_i tile is weighted by T^{-1}.
// FP64: the second producer warp weights each tile in shared memory once it
// lands (all 32 lanes, one column each) and releases it to the consumers on
// wqready -- one pass per block and tile, where the FP64 consumer warps have
// no multiplies to spare.  FP32: each consumer warp weights its register
// copies (one load and TR shuffles per tile), which keeps the second producer
// free to issue copies (measured faster for FP32, slower for FP64).
template <typename T, bool TW>
__global__ void __launch_bounds__(DTHREADS, 2)
reorth_dots_kernel(Run r, int i)
{
    constexpr int TR = DSTAGE / (CW * (int)sizeof(T));   // rows per tile
    const int ch = blockIdx.y, blk = blockIdx.x;
    if (!r.chunk_active[ch]) return;
    extern __shared__ __align__(128) unsigned char smem[];
    T* stage = reinterpret_cast<T*>(smem);                               // [DNS][TR*CW]
    T* wq = reinterpret_cast<T*>(smem + (size_t)DNS * DSTAGE);           // [2][2][TR*CW]
    double* acc = reinterpret_cast<double*>(smem + (size_t)(DNS + 4) * DSTAGE);   // [2][i][CW]
    uint64_t* full = reinterpret_cast<uint64_t*>(acc + (size_t)2 * i * CW);
    uint64_t* empty = full + DNS;
    uint64_t* wqfull = empty + DNS;
    uint64_t* wqempty = wqfull + 2;
    uint64_t* wqready = wqempty + 2;                     // TW: weighted tiles
    __shared__ int s_fail;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t r0, r1;
    row_range(r.n, r.nblk, blk, r0, r1);
    const int ntile = r1 > r0 ? (int)((r1 - r0 + TR - 1) / TR) : 0;
    const T* P = static_cast<const T*>(r.basis) + ch * r.chunk_stride;
    const T* w = P + (int64_t)i * r.slot_stride;
    const T* q = P + (int64_t)(i - 1) * r.slot_stride;
    const void* lo = P;                                  // this chunk's basis
    const void* hi = P + r.chunk_stride;
    // T^{-1} weights of this lane's column (TW: T^{-1}-inner-product mode);
    // when the chunk's columns share one shift, lane l loads row l of the
    // tile and the others take it by shuffle (one load per tile, not TR)
    const T* wt = TW ? static_cast<const T*>(r.tinvd) +
                           (int64_t)r.shift_of[ch * CW + (threadIdx.x & 31)] * r.n
                     : nullptr;
    const bool wuni = r.S == 1 || r.m % CW == 0;
    static_assert(TR <= 32, "one weight per lane covers a tile");
    static_assert(NPROD >= 2, "the second producer warp weights the tiles");
    constexpr bool PRODW = TW && sizeof(T) == 8;         // weights applied by a producer warp
    constexpr bool CONSW = TW && sizeof(T) == 4;         // ... by each consumer warp
    if (threadIdx.x == 0) {
        for (int s = 0; s < DNS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&wqfull[b], 1);
            mbar_init(&wqempty[b], CWARPS);
            mbar_init(&wqready[b], 32);
        }
        mbar_init_fence();
        s_fail = 0;
    }
    for (int e = threadIdx.x; e < 2 * i * CW; e += blockDim.x) acc[e] = 0.0;
    __syncthreads();
    typedef typename Acc<T>::run RTy;
    bool ok = true;
    if (warp >= CWARPS) {
        // Producer p issues the items j = p, p + NPROD, ... -- the rings of the
        // consumer warps cw = j % CWARPS with cw % NPROD == p, each ring in
        // order -- so that NPROD threads issue bulk copies (one thread issues
        // about one copy per quarter microsecond); producer 0 also issues the
        // w and q_i tiles.
        const int pw = warp - CWARPS;
        const bool weigh = PRODW && pw == 1;     // the whole warp weights the w, q tiles
        if (lane == 0 || weigh) {
            int64_t lastk[DNS];                  // last item issued into each stage
            int lastt[2] = {-1, -1};             // last tile issued into each w/q buffer
            for (int s = 0; s < DNS; ++s) lastk[s] = -1;
            for (int t = 0; t < ntile && ok; ++t) {
                const int64_t row0 = r0 + (int64_t)t * TR;
                const uint32_t bytes = (uint32_t)(min((int64_t)TR, r1 - row0) * CW * sizeof(T));
                const int b = t & 1;
                if (weigh) {
                    // w <- T^{-1} w, q_i <- T^{-1} q_i in place, lane = column
                    if (!(ok = mbar_wait_warp(&wqfull[b], (t >> 1) & 1))) break;
                    const int rows = (int)min((int64_t)TR, r1 - row0);
                    T* wtile = wq + (size_t)(2 * b) * TR * CW + lane;
                    T* qtile = wq + (size_t)(2 * b + 1) * TR * CW + lane;
                    T dl = 0;
                    if (wuni && lane < rows) dl = __ldg(wt + row0 + lane);
#pragma unroll
                    for (int rr = 0; rr < TR; ++rr) {
                        T d = __shfl_sync(0xffffffffu, dl, rr);
                        if (rr < rows) {
                            if (!wuni) d = __ldg(wt + row0 + rr);
                            wtile[rr * CW] *= d;
                            qtile[rr * CW] *= d;
                        }
                    }
                    // the next bulk copy into this buffer must follow these writes
                    fence_proxy_async_smem();
                    mbar_arrive(&wqready[b]);
                }
                if (lane == 0) {
                    if (pw == 0) {
                        // (warp 0 runs this loop on lane 0 alone: the break leaves it)
                        if (t >= 2 && !(ok = mbar_wait(&wqempty[b], ((t >> 1) - 1) & 1))) break;
                        lastt[b] = t;
                        mbar_arrive_expect_tx(&wqfull[b], 2 * bytes);
                        ok = checked_bulk(wq + (size_t)(2 * b) * TR * CW, w + row0 * CW, bytes,
                                          &wqfull[b], lo, hi, r.err) &&
                             checked_bulk(wq + (size_t)(2 * b + 1) * TR * CW, q + row0 * CW, bytes,
                                          &wqfull[b], lo, hi, r.err);
                    }
                    for (int j = pw; j < i && ok; j += NPROD) {
                        // k-th item of consumer warp cw lives in stage cw*NSW + k % NSW
                        const int cw = j % CWARPS;
                        const int64_t k = (int64_t)t * ((i - cw + CWARPS - 1) / CWARPS) + j / CWARPS;
                        const int s = cw * NSW + (int)(k % NSW);
                        if (k >= NSW && !(ok = mbar_wait(&empty[s], ((k / NSW) - 1) & 1))) break;
                        lastk[s] = k;
                        mbar_arrive_expect_tx(&full[s], bytes);
                        ok = checked_bulk(stage + (size_t)s * TR * CW,
                                          P + (int64_t)j * r.slot_stride + row0 * CW, bytes,
                                          &full[s], lo, hi, r.err);
                    }
                }
                // the weighing warp leaves the loop as one
                if (weigh) ok = __shfl_sync(0xffffffffu, ok, 0);
            }
            if (!ok) {
                // let the copies already issued land before the block exits
                for (int s = 0; s < DNS; ++s)
                    if (lastk[s] >= 0) mbar_wait(&full[s], (lastk[s] / NSW) & 1);
                for (int b = 0; b < 2; ++b)
                    if (lastt[b] >= 0) mbar_wait(&wqfull[b], (lastt[b] >> 1) & 1);
            }
        }
    } else {
        for (int t = 0; t < ntile && ok; ++t) {
            const int64_t row0 = r0 + (int64_t)t * TR;
            const int rows = (int)min((int64_t)TR, r1 - row0);
            const int b = t & 1;
            if (!(ok = mbar_wait_warp(PRODW ? &wqready[b] : &wqfull[b], (t >> 1) & 1))) break;
            T wv[TR], qv[TR];
            T dl = 0;
            if (CONSW && wuni && lane < rows) dl = __ldg(wt + row0 + lane);
#pragma unroll
            for (int rr = 0; rr < TR; ++rr) {
                wv[rr] = rr < rows ? wq[(size_t)(2 * b) * TR * CW + rr * CW + lane] : (T)0;
                qv[rr] = rr < rows ? wq[(size_t)(2 * b + 1) * TR * CW + rr * CW + lane] : (T)0;
                if (CONSW) {
                    T d = __shfl_sync(0xffffffffu, dl, rr);
                    if (!wuni && rr < rows) d = __ldg(wt + row0 + rr);
                    wv[rr] *= d;
                    qv[rr] *= d;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&wqempty[b]);
            const int per = (i - warp + CWARPS - 1) / CWARPS;   // my items per tile
            for (int j = warp; j < i; j += CWARPS) {
                const int64_t k = (int64_t)t * per + j / CWARPS;
                const int s = warp * NSW + (int)(k % NSW);
                if (!(ok = mbar_wait_warp(&full[s], (k / NSW) & 1))) break;
                const T* st = stage + (size_t)s * TR * CW + lane;
                RTy a = 0, g = 0;
#pragma unroll
                for (int rr = 0; rr < TR; ++rr) {
                    // rows past the tail of a short tile hold stale shared memory
                    const RTy pv = rr < rows ? (RTy)st[rr * CW] : (RTy)0;
                    a += pv * (RTy)wv[rr];
                    g += pv * (RTy)qv[rr];
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
                acc[(size_t)j * CW + lane] += (double)a;
                acc[(size_t)(i + j) * CW + lane] += (double)g;
            }
        }
    }
    if (!ok) s_fail = 1;
    __syncthreads();
    if (s_fail) {
        if (threadIdx.x == 0) atomicCAS(r.err, DERR_NONE, DERR_TIMEOUT);
        return;
    }
    for (int e = threadIdx.x; e < i * CW; e += blockDim.x) {
        const int64_t o = (((int64_t)ch * r.nblk + blk) * r.kmax + e / CW) * CW + (e % CW);
        r.part_dot[o] = acc[e];
        r.part_gram[o] = acc[(size_t)i * CW + e];
    }
}

__device__ __forceinline__ int64_t tri(int a, int b)
{
    // packed lower triangle, a >= b
    return (int64_t)a * (a + 1) / 2 + b;
}

// h_j = s_j sum_b part_dot[ch][b][j][:], G_{i-1,j} = s_{i-1} s_j sum_b part_gram,
// alpha_i = h_{i-1}.  One block of RW warps per (chunk, j): warp q sums the row
// blocks b = q, q+RW, ... for the 32 columns (one coalesced 256-byte load per
// b), then the warps' sums are added in warp order (fixed summation order).
constexpr int RW = 4;
__global__ void __launch_bounds__(RW * 32)
reorth_reduce_kernel(Run r, int i)
{
    const int ch = blockIdx.x % r.nchunk, j = blockIdx.x / r.nchunk;
    if (!r.chunk_active[ch]) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double sh[RW][CW], sg[RW][CW];
    double ah = 0.0, ag = 0.0;
#pragma unroll 4
    for (int b = warp; b < r.nblk; b += RW) {
        const int64_t o = (((int64_t)ch * r.nblk + b) * r.kmax + j) * CW + lane;
        ah += r.part_dot[o];
        ag += r.part_gram[o];
    }
    sh[warp][lane] = ah;
    sg[warp][lane] = ag;
    __syncthreads();
    if (warp == 0) {
        double th = 0.0, tg = 0.0;
#pragma unroll
        for (int q = 0; q < RW; ++q) { th += sh[q][lane]; tg += sg[q][lane]; }
        const int c = ch * CW + lane;
        const double sj = r.scl[(int64_t)j * r.ncol + c];
        const double si = r.scl[(int64_t)(i - 1) * r.ncol + c];
        const double h = th * sj;                    // q_j . w
        r.hbuf[(int64_t)j * r.ncol + c] = h;
        r.gram[tri(i - 1, j) * r.ncol + c] = tg * sj * si;   // q_j . q_i
        if (j == i - 1) r.alpha[(int64_t)(i - 1) * r.ncol + c] = h;
    }
}

// c = h + (I - G) h;  g_j = c_j s_j multiplies the unnormalised P_j.
// One thread per (column, j).
__global__ void reorth_coef_kernel(Run r, int i)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= r.ncol * i) return;
    const int c = t % r.ncol, j = t / r.ncol;
    if (!r.chunk_active[c / CW]) return;
    double gh = 0.0;
#pragma unroll 4
    for (int l = 0; l < i; ++l) {
        const double G = r.gram[(j >= l ? tri(j, l) : tri(l, j)) * r.ncol + c];
        gh += G * r.hbuf[(int64_t)l * r.ncol + c];
    }
    const double hj = r.hbuf[(int64_t)j * r.ncol + c];
    r.g[(int64_t)j * r.ncol + c] = (2.0 * hj - gh) * r.scl[(int64_t)j * r.ncol + c];
    // Arnoldi: the full coefficient is the Hessenberg entry h_{j+1,i} (Algorithm 3)
    if (r.hess) r.hess[tri(i - 1, j) * r.ncol + c] = 2.0 * hj - gh;
}

// w <- w - sum_{j<i} g_j P_j (in place, slot i); part_nrm = partial ||w||^2.
// The producer streams, per row tile, the w tile and then every P_j tile;
// consumer warp q owns rows q*RPW.. of the tile in registers and applies
// every P_j stage to them, then writes the tile back.
template <typename T, bool TW>
__global__ void __launch_bounds__(UTHREADS, 2)
reorth_update_kernel(Run r, int i)
{
    constexpr int TR = USTAGE / (CW * (int)sizeof(T));   // rows per tile
    constexpr int RPW = TR / CWARPS;                      // rows per consumer warp
    const int ch = blockIdx.y, blk = blockIdx.x;
    if (!r.chunk_active[ch]) return;
    extern __shared__ __align__(128) unsigned char smem[];
    T* stage = reinterpret_cast<T*>(smem);                                // [UNS][TR*CW]
    T* wbuf = reinterpret_cast<T*>(smem + (size_t)UNS * USTAGE);          // [2][TR*CW]
    T* gs = reinterpret_cast<T*>(smem + (size_t)(UNS + 2) * USTAGE);      // [i][CW]
    uint64_t* full = reinterpret_cast<uint64_t*>(
        smem + (size_t)(UNS + 2) * USTAGE + (((size_t)i * CW * sizeof(T) + 15) & ~(size_t)15));
    uint64_t* empty = full + UNS;
    uint64_t* wfull = empty + UNS;
    uint64_t* wempty = wfull + 2;
    __shared__ double red[UWARPS][CW];
    __shared__ int s_fail;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < i * CW; e += blockDim.x)
        gs[e] = (T)r.g[(int64_t)(e / CW) * r.ncol + ch * CW + (e % CW)];
    int64_t r0, r1;
    row_range(r.n, r.nblk, blk, r0, r1);
    const int ntile = r1 > r0 ? (int)((r1 - r0 + TR - 1) / TR) : 0;
    const T* P = static_cast<const T*>(r.basis) + ch * r.chunk_stride;
    T* w = static_cast<T*>(r.basis) + ch * r.chunk_stride + (int64_t)i * r.slot_stride;
    const void* lo = P;
    const void* hi = P + r.chunk_stride;
    // T^{-1} weights of this lane's column (TW: the norm is <w, w> in T^{-1});
    // one load per row per warp and shuffles when the chunk has one shift
    const T* wt = TW ? static_cast<const T*>(r.tinvd) +
                           (int64_t)r.shift_of[ch * CW + (threadIdx.x & 31)] * r.n
                     : nullptr;
    const bool wuni = r.S == 1 || r.m % CW == 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < UNS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CWARPS);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&wfull[b], 1);
            mbar_init(&wempty[b], CWARPS);
        }
        mbar_init_fence();
        s_fail = 0;
    }
    __syncthreads();
    typedef typename Acc<T>::run RTy;
    bool ok = true;
    double acc = 0.0;
    if (warp >= CWARPS) {
        // Producer p issues the items with index = p (mod NPROD) -- the stages
        // s = p (mod NPROD), each in order -- so that NPROD threads issue bulk
        // copies; producer 0 also issues the w tiles.
        const int pw = warp - CWARPS;
        if (lane == 0) {
            int64_t item = 0;
            int64_t lastk[UNS];
            int lastt[2] = {-1, -1};
            for (int s = 0; s < UNS; ++s) lastk[s] = -1;
            for (int t = 0; t < ntile && ok; ++t) {
                const int64_t row0 = r0 + (int64_t)t * TR;
                const uint32_t bytes = (uint32_t)(min((int64_t)TR, r1 - row0) * CW * sizeof(T));
                const int b = t & 1;
                if (pw == 0) {
                    if (t >= 2 && !(ok = mbar_wait(&wempty[b], ((t >> 1) - 1) & 1))) break;
                    lastt[b] = t;
                    mbar_arrive_expect_tx(&wfull[b], bytes);
                    ok = checked_bulk(wbuf + (size_t)b * TR * CW, w + row0 * CW, bytes, &wfull[b],
                                      lo, hi, r.err);
                }
                for (int j = 0; j < i && ok; ++j, ++item) {
                    if ((int)(item % NPROD) != pw) continue;
                    const int s = (int)(item % UNS);
                    if (item >= UNS && !(ok = mbar_wait(&empty[s], ((item / UNS) - 1) & 1))) break;
                    lastk[s] = item;
                    mbar_arrive_expect_tx(&full[s], bytes);
                    ok = checked_bulk(stage + (size_t)s * TR * CW,
                                      P + (int64_t)j * r.slot_stride + row0 * CW, bytes, &full[s],
                                      lo, hi, r.err);
                }
            }
            if (!ok) {
                // let the copies already issued land before the block exits
                for (int s = 0; s < UNS; ++s)
                    if (lastk[s] >= 0) mbar_wait(&full[s], (lastk[s] / UNS) & 1);
                for (int b = 0; b < 2; ++b)
                    if (lastt[b] >= 0) mbar_wait(&wfull[b], (lastt[b] >> 1) & 1);
            }
        }
    } else {
        int64_t item = 0;
        for (int t = 0; t < ntile && ok; ++t) {
            const int64_t row0 = r0 + (int64_t)t * TR;
            const int rows = (int)min((int64_t)TR, r1 - row0);
            const int b = t & 1;
            if (!(ok = mbar_wait_warp(&wfull[b], (t >> 1) & 1))) break;
            T wv[RPW];
#pragma unroll
            for (int rr = 0; rr < RPW; ++rr) {
                const int row = warp * RPW + rr;
                wv[rr] = row < rows ? wbuf[(size_t)b * TR * CW + row * CW + lane] : (T)0;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&wempty[b]);
            for (int j = 0; j < i; ++j, ++item) {
                const int s = (int)(item % UNS);
                if (!(ok = mbar_wait_warp(&full[s], (item / UNS) & 1))) break;
                const T gj = gs[j * CW + lane];
                const T* st = stage + (size_t)s * TR * CW + (size_t)warp * RPW * CW + lane;
#pragma unroll
                for (int rr = 0; rr < RPW; ++rr)
                    if (warp * RPW + rr < rows) wv[rr] -= gj * st[rr * CW];
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
            if (!ok) break;
            RTy nr = 0;
            T dl = 0;
            if (TW && wuni && lane < RPW && warp * RPW + lane < rows)
                dl = __ldg(wt + row0 + warp * RPW + lane);
#pragma unroll
            for (int rr = 0; rr < RPW; ++rr) {
                const int row = warp * RPW + rr;
                T d = 0;
                if (TW) d = __shfl_sync(0xffffffffu, dl, rr);
                if (row < rows) {
                    // BF16 storage of the basis (an accuracy trial): the vector
                    // kept is the rounded one, and beta is its norm
                    if (sizeof(T) == 4 && r.basis_bf16)
                        wv[rr] = (T)__bfloat162float(__float2bfloat16_rn((float)wv[rr]));
                    w[(row0 + row) * CW + lane] = wv[rr];
                    if (TW && !wuni) d = __ldg(wt + row0 + row);
                    if (TW) nr += (RTy)(wv[rr] * d) * (RTy)wv[rr];
                    else nr += (RTy)wv[rr] * (RTy)wv[rr];
                }
            }
            acc += (double)nr;
        }
    }
    if (!ok) s_fail = 1;
    red[warp][lane] = acc;
    __syncthreads();
    if (s_fail) {
        if (threadIdx.x == 0) atomicCAS(r.err, DERR_NONE, DERR_TIMEOUT);
        return;
    }
    if (warp == 0) {
        double sum = 0.0;
#pragma unroll
        for (int qq = 0; qq < CWARPS; ++qq) sum += red[qq][lane];
        r.part_nrm[((int64_t)ch * r.nblk + blk) * CW + lane] = sum;
    }
    // The last block of this chunk forms beta_{i+1}, the new scale s_i and the
    // breakdown test for the chunk's columns (no extra launch).
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&r.cnt_upd[ch], 1) == r.nblk - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    {
        double ps = 0.0;
        for (int b = warp; b < r.nblk; b += UWARPS)
            ps += r.part_nrm[((int64_t)ch * r.nblk + b) * CW + lane];
        red[warp][lane] = ps;
    }
    __syncthreads();
    if (threadIdx.x < CW) {
        const int ln = threadIdx.x, c = ch * CW + ln;
        if (r.kdone[c] == 0) {
            double nrm2 = 0.0;
#pragma unroll
            for (int q = 0; q < UWARPS; ++q) nrm2 += red[q][ln];
            const double beta = sqrt(nrm2);
            const double al = r.alpha[(int64_t)(i - 1) * r.ncol + c];
            const double bprev = r.beta[(int64_t)(i - 1) * r.ncol + c];
            const double sc = fmax(r.colscale[c], fmax(fabs(al), bprev));
            r.colscale[c] = sc;
            r.beta[(int64_t)i * r.ncol + c] = beta;
            if (!isfinite(beta) || !isfinite(al)) {
                if (c < r.ncol_real) atomicExch(r.err, DERR_NUMERIC);
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
    }
    if (threadIdx.x == 0) r.cnt_upd[ch] = 0;
}

// Quadrature of every running column's J_i (Sec. 3, Eq. gauss_quad), or of
// the extended J~_{2i-1} of the generalized averaged rule (Sec. 3.4,
// Eq. GA_Tk) when r.ga is set.  One thread per Lanczos column; the
// eigensolver scratch (3 x rule size per column) lives in shared memory.  In
// shared mode one decomposition of the column's J_i serves every running
// shift: the quadrature of shift s sums the weights of the Ritz values below
// tau_s (J_i(A - tau I) = J_i(A) - tau I).
__global__ void quad_kernel(Run r, int i)
{
    extern __shared__ double qs[];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= r.ncol_real) return;
    bool running;
    if (r.shared) {
        running = false;
        for (int s = 0; s < r.S; ++s) running |= !r.sdone[s];
    } else {
        running = !r.sdone[r.shift_of[c]];
    }
    if (!running) return;
    const int k = r.kdone[c] ? min(r.kdone[c], i) : i;
    const int nb = blockDim.x;
    const int kk = r.ga ? 2 * r.kmax - 1 : r.kmax;
    double* d = qs + threadIdx.x;
    double* e = qs + (size_t)kk * nb + threadIdx.x;
    double* z = qs + (size_t)2 * kk * nb + threadIdx.x;
    const int kr = tridiag_fill(r.alpha + c, r.beta + c, r.ncol, k, r.ga != 0, d, e, nb);
    const bool ok = tridiag_eig_inplace(d, e, z, nb, kr);
    if (!ok) atomicExch(r.err, DERR_NUMERIC);
    if (r.shared) {
        for (int s = 0; s < r.S; ++s)
            if (!r.sdone[s])
                r.quad[(int64_t)s * r.m + c] =
                    ok && c < r.m ? quadrature_below(d, z, nb, kr, (double)r.n, r.shifts[s]) : 0.0;
    } else {
        r.quad[c] = ok ? quadrature_below(d, z, nb, kr, (double)r.n, 0.0) : 0.0;
    }
}

// Per-shift mean L_s(i) = (1/m) sum_j quad_j in a fixed tree, and the stop
// rule: a shift stops at its last step (skmax[s]) or, under its tolerance, at
// the first step i >= max(3, min_steps) with |L_s(i) - L_s(i-1)| <= tol and
// |L_s(i-1) - L_s(i-2)| <= tol.  In the normal mode a stopped shift's columns
// are frozen (their later vectors become exact zeros); in shared mode the
// Lanczos columns run on while any shift does.  One block per shift.
__global__ void __launch_bounds__(kThreads)
shift_kernel(Run r, int i)
{
    const int s = blockIdx.x;
    if (r.sdone[s]) return;
    const int cbeg = s * r.m, cend = cbeg + r.m;
    __shared__ double red[kThreads];
    __shared__ int stop;
    double lsum = 0.0;
    for (int c = cbeg + threadIdx.x; c < cend; c += blockDim.x) lsum += r.quad[c];
    red[threadIdx.x] = lsum;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double L = red[0] / r.m;
        const double tol = r.stol[s];
        int st = i >= r.skmax[s] ? 1 : 0;
        if (tol > 0.0 && i >= 3 && i >= r.min_steps && fabs(L - r.Lprev[s]) <= tol &&
            fabs(r.Lprev[s] - r.Lprev2[s]) <= tol)
            st = 1;
        r.Lprev2[s] = r.Lprev[s];
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
            r.quad_final[c] = r.quad[c];
            if (r.shared) continue;
            r.ppc[c] = 0.0;
            for (int j = i; j <= r.kmax; ++j) r.scl[(int64_t)j * r.ncol + c] = 0.0;
            if (!r.kdone[c]) r.kdone[c] = i;
        }
}

// A chunk stays active while one of its real columns belongs to a running
// shift; the number of active chunks of the next step is recorded.
__global__ void __launch_bounds__(kThreads) active_kernel(Run r, int i)
{
    __shared__ int cnt[kThreads];
    __shared__ int any_running;
    if (threadIdx.x == 0) {
        int a = 0;
        for (int s = 0; s < r.S; ++s) a |= !r.sdone[s];
        any_running = a;
    }
    __syncthreads();
    int mine = 0;
    for (int ch = threadIdx.x; ch < r.nchunk; ch += blockDim.x) {
        int act = 0;
        if (r.shared) {
            act = any_running;
        } else {
            for (int l = 0; l < CW; ++l) {
                const int c = ch * CW + l;
                if (c < r.ncol_real && !r.sdone[r.shift_of[c]]) act = 1;
            }
        }
        r.chunk_active[ch] = act;
        mine += act;
    }
    cnt[threadIdx.x] = mine;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) cnt[threadIdx.x] += cnt[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0 && i < r.kmax) r.nactive[i] = cnt[0];
}

}  // namespace

cudaError_t launch_init_state(const Run& r, cudaStream_t st)
{
    const int nstate = max(max(max(r.ncol, r.S), r.nchunk), r.kmax + 1);
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
                                 double eps, int form, cudaStream_t st)
{
    const int64_t total = (int64_t)r.Sop * r.n;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
    if ((form == PM_TLEFT) != (r.tinv != 0)) return cudaErrorInvalidValue;
    jacobi_scale_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(r, diag, static_cast<const T*>(V),
                                                             vdiag, eps, form);
    return cudaGetLastError();
}

template <typename T>
size_t dots_smem(int i)
{
    return (size_t)(DNS + 4) * DSTAGE + (size_t)2 * i * CW * sizeof(double) +
           (2 * DNS + 6) * sizeof(uint64_t);
}

template <typename T>
size_t update_smem(int i)
{
    return (size_t)(UNS + 2) * USTAGE + (((size_t)i * CW * sizeof(T) + 15) & ~(size_t)15) +
           (2 * UNS + 4) * sizeof(uint64_t);
}

template <typename T, bool TW>
cudaError_t launch_dots_w(const Run& r, int i, cudaStream_t st)
{
    static std::atomic<uint64_t> attr{0};
    const cudaError_t e = smem_limit_once(attr, reorth_dots_kernel<T, TW>, dots_smem<T>(kMaxSteps));
    if (e != cudaSuccess) return e;
    reorth_dots_kernel<T, TW><<<dim3(r.nblk, r.nchunk), DTHREADS, dots_smem<T>(i), st>>>(r, i);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dots(const Run& r, int i, cudaStream_t st)
{
    return r.tinv ? launch_dots_w<T, true>(r, i, st) : launch_dots_w<T, false>(r, i, st);
}

cudaError_t launch_reduce(const Run& r, int i, cudaStream_t st)
{
    reorth_reduce_kernel<<<r.nchunk * i, RW * 32, 0, st>>>(r, i);
    return cudaGetLastError();
}

cudaError_t launch_coef(const Run& r, int i, cudaStream_t st)
{
    const int tot = r.ncol * i;
    reorth_coef_kernel<<<(tot + 255) / 256, 256, 0, st>>>(r, i);
    return cudaGetLastError();
}

template <typename T, bool TW>
cudaError_t launch_update_w(const Run& r, int i, cudaStream_t st)
{
    static std::atomic<uint64_t> attr{0};
    const cudaError_t e =
        smem_limit_once(attr, reorth_update_kernel<T, TW>, update_smem<T>(kMaxSteps));
    if (e != cudaSuccess) return e;
    reorth_update_kernel<T, TW><<<dim3(r.nblk, r.nchunk), UTHREADS, update_smem<T>(i), st>>>(r, i);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update(const Run& r, int i, cudaStream_t st)
{
    return r.tinv ? launch_update_w<T, true>(r, i, st) : launch_update_w<T, false>(r, i, st);
}

cudaError_t launch_finish(const Run& r, int i, cudaStream_t st)
{
    // The eigensolves are chains of dependent FP64 operations: spread the
    // columns over all 152 SMs (few threads per block) so each one has an
    // SM's FP64 pipes to itself; 3 scratch vectors per thread must fit in 96 KB.
    const int kk = r.ga ? 2 * r.kmax - 1 : r.kmax;
    int qb = 1;
    while (qb < 32 && qb * 2 * 152 <= r.ncol_real) qb <<= 1;
    while (qb > 1 && (size_t)qb * 3 * kk * sizeof(double) > 96 * 1024) qb >>= 1;
    const size_t smem = (size_t)qb * 3 * kk * sizeof(double);
    static std::atomic<uint64_t> attr{0};
    const cudaError_t ea = smem_limit_once(attr, quad_kernel, 96 * 1024);
    if (ea != cudaSuccess) return ea;
    if (r.arnoldi) {
        const cudaError_t e = launch_arnoldi_quad(r, i, st);
        if (e != cudaSuccess) return e;
    } else {
        quad_kernel<<<(r.ncol_real + qb - 1) / qb, qb, smem, st>>>(r, i);
    }
    shift_kernel<<<r.S, kThreads, 0, st>>>(r, i);
    return cudaGetLastError();
}

cudaError_t launch_active(const Run& r, int i, cudaStream_t st)
{
    active_kernel<<<1, kThreads, 0, st>>>(r, i);
    return cudaGetLastError();
}

template cudaError_t launch_init_probe<float>(const Run&, cudaStream_t);
template cudaError_t launch_init_probe<double>(const Run&, cudaStream_t);
template cudaError_t launch_jacobi_scales<float>(const Run&, const double*, const void*, double,
                                                 double, int, cudaStream_t);
template cudaError_t launch_jacobi_scales<double>(const Run&, const double*, const void*, double,
                                                  double, int, cudaStream_t);
template cudaError_t launch_dots<float>(const Run&, int, cudaStream_t);
template cudaError_t launch_dots<double>(const Run&, int, cudaStream_t);
template cudaError_t launch_update<float>(const Run&, int, cudaStream_t);
template cudaError_t launch_update<double>(const Run&, int, cudaStream_t);

}  // namespace evc
