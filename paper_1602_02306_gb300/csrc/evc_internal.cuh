// evc_internal.cuh -- internal declarations shared by the libevc translation
// units (kernels + host orchestration). Not part of the C ABI.
//
// Data layout in HBM.  The (shift x probe) columns of one call are packed as
// c = s*m + j and padded to a multiple of CW = 32.  A "chunk" is CW columns;
// every block vector is stored chunk-major, row-major inside a chunk:
//     X[chunk][row][CW]      (the CW probes of a row are contiguous)
// so one grid point / CSR row of one chunk is one 128-byte (FP32) or
// 256-byte (FP64) segment, and chunks whose shift has stopped early are
// skipped as whole contiguous blocks.  The Lanczos basis of chunk ch is
//     P[ch][slot][row][CW],  slot j holding the unnormalised q_{j+1},
// with per-column scales s_j (q_{j+1} = s_j P_j), so normalisation costs no
// extra pass over the vectors.  Per-column scalars are stored [step][column].
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace evc {

// A named NVTX range over a host-side phase (graph capture, replay, set-up,
// autotuning, a server batch), visible to Nsight tools; without an attached
// tool the calls do nothing.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Raise a kernel's dynamic shared-memory limit on the current device, once per
// process and device: `done` is that kernel's bitmask of devices already set.
// Launches from several host threads (the request server's slots) may both
// set it the first time, which is harmless; the mask itself is atomic.
template <typename F>
inline cudaError_t smem_limit_once(std::atomic<uint64_t>& done, F* kernel, size_t bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev >= 0 && dev < 64 ? (uint64_t)1 << dev : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

constexpr int CW = 32;                 // columns per chunk
constexpr int kMaxSteps = 256;         // == EVC_MAX_STEPS
constexpr int kThreads = 256;          // threads per block of the streaming kernels

// Device-side error codes (mirror evc_status).
enum { DERR_NONE = 0, DERR_NUMERIC = 4, DERR_TIMEOUT = 5, DERR_BOUNDS = 7 };

// One run (a call of evc_count_slices) -- device pointers and sizes.
//
// Shared mode (identity preconditioner, Lanczos): the Krylov space of A - tau I
// does not depend on tau, and Algorithm 1 on A - tau I gives J_k(A) - tau I.
// So the run keeps m Lanczos columns on A itself (operator shift 0) and every
// shift tau_s reads its quadrature from the same J_k: sum over Ritz values
// theta < tau_s.  Per-column arrays (basis, alpha, beta, ...) then hold the m
// probes; per-(shift, probe) arrays (quad, quad_final) hold S*m entries,
// c = s*m + j, as in the normal mode.
struct Run {
    int64_t n;
    int S, m, kmax;          // shifts, probes, steps (kmax already clamped)
    int ncol, ncol_real;     // padded / real Lanczos columns (S*m, or m when shared)
    int shared;              // 1: all shifts read one Krylov run (see above)
    int nq;                  // (shift, probe) quadratures: S*m
    int Sop;                 // operator shifts: S (normal) or 1 (shared: tau = 0)
    double* opshift;         // [Sop] shift of the operator the columns run on
    int nchunk;
    int nblk;                // row blocks per chunk in the reorth kernels
    int64_t slot_stride;     // n*CW elements
    int64_t chunk_stride;    // (kmax+1)*n*CW elements
    void* basis;             // T[nchunk][kmax+1][n][CW]
    // per column
    double* sigma;           // [ncol]
    int* shift_of;           // [ncol]
    int64_t* probe_id;       // [ncol]
    double* alpha;           // [kmax][ncol]
    double* beta;            // [kmax+1][ncol]
    double* scl;             // [kmax+1][ncol]
    double* g;               // [kmax][ncol]
    double* ppc;             // [ncol]
    double* colscale;        // [ncol]
    int* kdone;              // [ncol]
    double* quad;            // [nq]  latest quadrature per (shift, probe)
    double* quad_final;      // [nq]  quadrature at the shift's stop step
    // per shift
    double* shifts;          // [S]
    double* Lprev;           // [S]  L_s(i-1)
    double* Lprev2;          // [S]  L_s(i-2)
    double* Lfinal;          // [S]
    int* steps;              // [S]
    int* sdone;              // [S]
    double* stol;            // [S]  stop tolerance per shift (<= 0: none)
    int* skmax;              // [S]  last step per shift (<= kmax)
    int* chunk_active;       // [nchunk]
    int* cnt_upd;            // [nchunk]  blocks done, update kernel (last block forms beta)
    int* nactive;            // [kmax+1]  chunks active during step i+1 (profiling)
    int* err;                // [1]
    double* part_dot;        // [nchunk][nblk][kmax][CW]  partial P_j . w
    double* part_gram;       // [nchunk][nblk][kmax][CW]  partial P_j . P_{i-1}
    double* hbuf;            // [kmax][ncol]  h_j = q_j . w of the current step
    double* gram;            // [kmax(kmax+1)/2][ncol]  G_ab = q_a . q_b, a >= b
    double* part_nrm;        // [nchunk][nblk][CW]
    void* jac;               // T[Sop][n]  Jacobi scales m_r (or m_r^2 = T in T^{-1} mode)
    void* dsh;               // T[Sop][n]  CSR contexts: the diagonal of the shifted operator,
                             //   (a_rr - sigma) m_r^2 (Lanczos with Jacobi) or a_rr - sigma,
                             //   formed in FP64 from the FP64 diagonal, then rounded
    // T^{-1}-inner-product Lanczos (Sec. 4, Eq. lanT1) with the Jacobi T = M^2:
    // the basis holds y_j = M q_j, the operator is T (A - sigma I), and every
    // inner product of the reorthogonalisation and the norm carry the weight
    // T^{-1} = diag(|a_rr - sigma| + eps), kept in tinvd.
    int tinv;
    void* tinvd;             // T[Sop][n]  T^{-1} diagonal (tinv only)
    // device scalars, rewritten before each replay
    uint64_t* seed;          // [1]
    double breakdown_rel;
    int ga;                  // 1: generalized averaged Gauss quadrature (Sec. 3.4)
    int min_steps;           // no tolerance stop before this step
    int basis_bf16;          // 1: basis vectors rounded to BF16 when stored (FP32 mode)
    int arnoldi;             // 1: Arnoldi process on T(A - sigma I) (Sec. 4)
    double* hess;            // [kmax(kmax+1)/2][ncol] Hessenberg columns (Arnoldi), or null
};

// Longest Arnoldi run: the quadrature keeps three k x k FP64 matrices in
// shared memory (evc_arnoldi.cu): 195 KB at k = 90.
constexpr int kArnoldiMaxSteps = 90;

// Coefficients of one stencil pass (see evc_stencil.cu):
//   st  = k1 * (L in)_offdiag + (k1*cd + k0 + [V_p] - [sigma_c]) * in_p
//   (Jacobi variant: in is scaled by M on load and st by M_p)
//   out = insc_c * st + a0 * xs_c * x_p - a2 * prev_p - ppc_c * pp_p
struct StencilPass {
    const void* in;   int64_t in_cs;
    const void* x;    int64_t x_cs;
    const void* prev; int64_t prev_cs;
    const void* pp;   int64_t pp_cs;
    void* out;        int64_t out_cs;
    const double* insc;     // per column or null
    const double* xs;       // per column or null
    const double* ppc;      // per column or null
    double k1, k0, a0, a2;
    int useV, useSigma;
};

struct StencilOp {
    int N, order;
    double h;
    double c1, c2, cd;      // L = -1/2 Lap_h: +-1 neighbours, +-2 neighbours, diagonal
    const void* V;          // T[n]
    int zb;                 // z planes per block (tuned; 0 = 32)
    int patch;              // points per thread: 1 (default) or 2 = a 2 x 2 patch (tuned)
    int c0, cn;             // chunks c0 .. c0+cn-1 of the launch (cn = 0: every chunk)
};

// Most concurrent chunk groups of the stencil operator (EVC_OPT_STENCIL_GROUPS).
constexpr int kMaxStencilGroups = 4;

struct CsrOp {
    int64_t n, nnz;
    const int64_t* row_ptr;
    const int32_t* col;
    const void* val;        // T[nnz]
    const double* diag;     // double[n]
    const int32_t* perm;    // [n] rows by decreasing length (visit order), or null
    int threads;            // threads per block: 128, 256 (default) or 512 (tuned)
};

// Rows per block of the reorthogonalisation kernels that a tuned context may
// use: at least kMinReorthRows, and no more blocks per chunk than
// reorth_max_blocks(n) (the workspace sizes the per-block partial sums for
// that many) -- small problems may split into up to 512 blocks, large ones
// down to 1728 rows per block.
constexpr int kMinReorthRows = 64;
inline int reorth_max_blocks(int64_t n)
{
    const int64_t big = (n + 1727) / 1728, small = (n + kMinReorthRows - 1) / kMinReorthRows;
    const int64_t m = big > (small < 512 ? small : 512) ? big : (small < 512 ? small : 512);
    return (int)(m < 65535 ? (m > 0 ? m : 1) : 65535);
}

// Kernel launchers (T = float for EVC_MIXED, double for EVC_FP64).
// Diagonal preconditioning of an operator pass: none, M (A - sigma I) M with
// the Jacobi M, or T (A - sigma I) with T = M^2 (T^{-1}-inner-product mode).
enum { PM_NONE = 0, PM_JACOBI = 1, PM_TLEFT = 2 };

template <typename T>
cudaError_t launch_stencil_pass(const StencilOp& op, const Run& r, const StencilPass& p,
                                int pmode, cudaStream_t st);
// The same pass on block tiles staged by tensor copies (evc_stencil_tma.cu):
// N a multiple of the tile (8 x 8 points FP32, 8 x 4 FP64); PM_NONE or
// PM_TLEFT.  p, shift_of, sigma and chunk_active are already moved to the
// launch's first chunk; cn chunks.
template <typename T>
bool stencil_tma_eligible(int N);
template <typename T>
cudaError_t launch_stencil_tma(const StencilOp& op, const StencilPass& p, const int* shift_of,
                               const double* sigma, const void* jac, const int* chunk_active,
                               int64_t n, int* err, int cn, int pmode, cudaStream_t st);
// Arnoldi-type estimator (evc_arnoldi.cu)
template <typename T>
cudaError_t launch_row_scale(const Run& r, void* w, int64_t cs, cudaStream_t st);
cudaError_t launch_arnoldi_quad(const Run& r, int i, cudaStream_t st);
template <typename T>
cudaError_t launch_csr_pass(const CsrOp& op, const Run& r, int i, int pmode, cudaStream_t st);
cudaError_t launch_init_state(const Run& r, cudaStream_t st);
template <typename T>
cudaError_t launch_init_probe(const Run& r, cudaStream_t st);
// form: PM_NONE (m_r and a_rr - sigma), PM_JACOBI (m_r and (a_rr - sigma) m_r^2)
// or PM_TLEFT (m_r^2, (a_rr - sigma) m_r^2 and the T^{-1} diagonal).
template <typename T>
cudaError_t launch_jacobi_scales(const Run& r, const double* diag, const void* V, double vdiag,
                                 double eps, int form, cudaStream_t st);
template <typename T>
cudaError_t launch_dots(const Run& r, int i, cudaStream_t st);
template <typename T>
cudaError_t launch_update(const Run& r, int i, cudaStream_t st);
cudaError_t launch_reduce(const Run& r, int i, cudaStream_t st);
cudaError_t launch_coef(const Run& r, int i, cudaStream_t st);
cudaError_t launch_finish(const Run& r, int i, cudaStream_t st);
cudaError_t launch_active(const Run& r, int i, cudaStream_t st);

// Host-side helpers.
int cheb_coefficients(int degree, double a, double b, double* coef);

}  // namespace evc

struct evc_ctx;
namespace evc {
evc_ctx* clone_context(const evc_ctx* src);
cudaStream_t ctx_stream(const evc_ctx* c);
// evc_count_slices with a stop tolerance and a step limit per shift (the
// request server merges requests whose tolerances and limits differ).
int count_slices_each(evc_ctx* ctx, const double* shifts, int nshift, int nprobe,
                      const int* maxsteps, const double* tol, uint64_t seed, double* n_below,
                      double* per_probe_quad, int* steps_used);
// 1 when calls with nshift shifts run in shared mode (see Run).
int shares_krylov(const evc_ctx* ctx, int nshift);

}  // namespace evc
