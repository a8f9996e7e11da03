/*
 * evc.h -- C ABI of libevc, a GB300 (sm_103a) implementation of the
 * preconditioned Lanczos eigenvalue-count estimator of Vecharynski & Yang,
 * "Preconditioned iterative methods for eigenvalue counts".
 *
 * What it computes (Sec. 2 and Sec. 3 of the paper):
 *   For a real symmetric A and a shift tau, n_-(A - tau I) = trace h(C) with
 *   C = M (A - tau I) M, T = M^2 an SPD preconditioner and h the step
 *   function of Eq. (h) (h(x) = 1 for x < 0, else 0).  For each of m seeded
 *   Rademacher probes v_j, k steps of Lanczos with full reorthogonalisation
 *   (Algorithm 1) give a tridiagonal J_k; Gauss quadrature (Eq. gauss_quad)
 *   gives v_j^T h(C) v_j ~ ||v_j||^2 sum_{theta_i < 0} z_i(1)^2 and the
 *   estimator L_tau(k, m) (Eq. rand_prec_quad, Algorithm 2) is their mean.
 *   The count in [xi, eta] is L_eta - L_xi (Sec. 3, two runs of Algorithm 2).
 *
 * Conventions
 *   - Every function returns an evc_status (0 = EVC_OK) and never aborts.
 *     evc_last_error(ctx) describes the last failure on that context.
 *   - Output arrays are caller-allocated HOST memory unless stated.
 *   - A context owns one CUDA stream binding (the caller's stream, or the
 *     legacy default stream when NULL); calls on one context must not run
 *     concurrently from several host threads.  This is deliberate: a
 *     context's captured graph, workspace and pinned staging buffers are its
 *     own state.  Concurrent callers use one context each (the request
 *     server runs a clone of each matrix's context per slot).
 *   - Probes: v_j[i] = -1 if bit 63 of x is set, else +1, where
 *     x = mix(seed ^ mix((j << 32) | i)) and mix is the SplitMix64 output
 *     finaliser.  The same probes serve every shift of one call.
 *   - Real symmetric matrices only.
 */
#ifndef EVC_H
#define EVC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct evc_ctx evc_ctx;

typedef enum {
    EVC_OK = 0,
    EVC_EINVAL = 1,        /* invalid argument (message in evc_last_error)      */
    EVC_ENOMEM = 2,        /* device or host allocation failed / workspace small */
    EVC_ECUDA = 3,         /* a CUDA runtime call failed                         */
    EVC_ENUMERIC = 4,      /* NaN/Inf in alpha/beta or eigensolver did not converge */
    EVC_ETIMEOUT = 5,      /* a bounded device wait gave up                      */
    EVC_EUNSUPPORTED = 6,  /* valid request this build does not implement        */
    EVC_EAGAIN = 7         /* a server request has not finished yet              */
} evc_status;

/* Arithmetic of the path.
 *   EVC_FP64 : matrix values, vectors and all arithmetic in float64.
 *   EVC_MIXED: matrix values, probe blocks, Lanczos basis, operator and
 *              preconditioner applies in float32; alpha, beta, the
 *              reorthogonalisation coefficients, the tridiagonal eigensolve
 *              and the quadrature weights in float64 (dot products accumulate
 *              short float32 runs and sum them in float64).  CSR contexts:
 *              the diagonal of A is kept in float64 as given, and per shift
 *              the diagonal of the shifted operator, (a_rr - tau) m_r^2 with
 *              Jacobi or a_rr - tau, and the Jacobi scales m_r are formed from
 *              it in float64 and rounded once; the stored diagonal entries do
 *              not enter the float32 row sums.  A Jacobi scale formed from a
 *              rounded a_rr would carry its error magnified by up to 1/eps.  */
enum { EVC_FP64 = 0, EVC_MIXED = 1 };

/* Preconditioners T = M^2 (Sec. 6; all SPD, so C keeps the inertia of
 * A - tau I, Sec. 2 Eq. negi_T).
 *   EVC_PREC_IDENTITY    : M = I.
 *   EVC_PREC_JACOBI      : M = diag((|a_ii - tau| + eps)^(-1/2)), per shift;
 *                          param0 = eps (> 0, default 1e-3).
 *   EVC_PREC_CHEB_KINETIC: stencil contexts only.  M = p_d(K), K = -1/2 Lap_h
 *                          + c I with the context's stencil, p_d the degree-d
 *                          Chebyshev interpolant (first-kind nodes) of
 *                          x^(-1/2) on the closed-form spectral interval
 *                          [c, c + 6/h^2] (7-point) or [c, c + 8/h^2]
 *                          (13-point) of K; shift independent (Sec. 3: one
 *                          T may serve both runs).  param0 = d (1..32),
 *                          param1 = c (> 0).  Fails with EVC_EINVAL when p_d
 *                          is not positive on the discrete spectrum of K.  */
enum { EVC_PREC_IDENTITY = 0, EVC_PREC_JACOBI = 1, EVC_PREC_CHEB_KINETIC = 2 };

/* Largest number of Lanczos steps per call. */
#define EVC_MAX_STEPS 256

/* A CSR matrix (Sec. 1: A large, sparse, symmetric).
 *   n, nnz      : order and stored entries (0 < n < 2^31, nnz < 2^62).
 *   row_ptr     : int64[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz.
 *   col         : int32[nnz], 0 <= col < n (duplicates are summed).
 *   val         : float64[nnz], or float32[nnz] when val_is_fp32 = 1.
 *   on_device   : 0 = host pointers (the library copies them into device
 *                 memory it owns); 1 = device pointers, borrowed (they must
 *                 stay valid until evc_destroy) when val's type matches the
 *                 context precision, else copied/converted.
 *   check       : 1 = validate ranges and symmetry on the host (host input
 *                 only); 0 = trust the caller.                                */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t* row_ptr;
    const int32_t* col;
    const void* val;
    int32_t val_is_fp32;
    int32_t on_device;
    int32_t check;
    int32_t reserved;
} evc_csr;

/* Create a context for a CSR matrix.  precision: EVC_FP64 or EVC_MIXED.
 * stream: a cudaStream_t (NULL = legacy default stream).  *out receives the
 * context; on failure *out is NULL.                                          */
int evc_create_csr(const evc_csr* A, int precision, void* stream, evc_ctx** out);

/* Create a context for the periodic finite-difference Hamiltonian
 * H = -1/2 Lap_h + diag(V) on an N^3 grid with spacing h (the real-space DFT
 * setting of Sec. 7).  order 2 = 7-point, order 4 = 13-point Laplacian.
 * V: N^3 values, point p = x + N*(y + N*z), float64 (or float32 when
 * V_is_fp32 = 1), host (copied) or device (on_device = 1: borrowed if its
 * type matches the precision, else converted).  N >= 2 (order 2), N >= 5
 * (order 4), N^3 < 2^31.                                                     */
int evc_create_stencil(int N, double h, int order, const void* V, int V_is_fp32,
                       int on_device, int precision, void* stream, evc_ctx** out);

/* Replace the matrix values without changing the structure: V (stencil
 * context, N^3 values) or the CSR values (nnz values), in the type given at
 * creation (val_is_fp32 / V_is_fp32).  Host (on_device = 0) or device
 * pointer; copied (converted to the context's type when it differs) into the
 * context's own device buffer on its stream; a CSR context re-forms its
 * float64 diagonal from the values as given.  Host values of the other type
 * pass through a device staging buffer the context keeps for later calls.
 * EVC_EINVAL when the context borrowed its values at creation.               */
int evc_set_values(evc_ctx* ctx, const void* values, int on_device);

/* Choose the preconditioner (see the EVC_PREC_* list above).                */
int evc_set_precond(evc_ctx* ctx, int kind, double param0, double param1);

/* Device scratch needed by a call with nshift shifts, nprobe probes and
 * maxsteps steps (bytes).  The Lanczos basis dominates:
 * (maxsteps + 1) * n * ceil(nshift*nprobe/32)*32 * (8 or 4) bytes.           */
size_t evc_workspace_bytes(const evc_ctx* ctx, int nshift, int nprobe, int maxsteps);

/* Hand the context caller-owned device scratch (for instance from a PyTorch
 * allocator).  The memory must stay valid until it is replaced or the
 * context is destroyed; bytes >= evc_workspace_bytes(...) of the calls that
 * follow, else they fail with EVC_ENOMEM.  dptr = NULL returns to scratch
 * the library allocates itself (cudaMalloc, grown on demand).                 */
int evc_set_workspace(evc_ctx* ctx, void* dptr, size_t bytes);

/* Algorithm 2 twice (Sec. 3): estimate of the number of eigenvalues of A in
 * [xi, eta] (xi < eta).
 *   nprobe      : m >= 1 probes (ids 0..m-1), the same for both shifts.
 *   maxsteps    : k, 1..EVC_MAX_STEPS, clamped to n.
 *   tol         : <= 0 runs exactly k steps; > 0 stops a shift at the first
 *                 step i >= max(3, EVC_OPT_MIN_STEPS) with
 *                 |L(i) - L(i-1)| <= tol and |L(i-1) - L(i-2)| <= tol.
 *   estimate    : L_eta - L_xi (real; the paper's count is its rounding).
 *   per_probe_quad (may be NULL): double[2*nprobe], [0..m) for xi, [m..2m) eta.
 *   steps_used  (may be NULL): int[2].
 * Blocks until the results are on the host.                                   */
int evc_count(evc_ctx* ctx, double xi, double eta, int nprobe, int maxsteps,
              double tol, uint64_t seed, double* estimate, double* per_probe_quad,
              int* steps_used);

/* Algorithm 2 for nshift shifts in one batched launch (spectrum slicing,
 * Sec. 1): n_below[s] = L_{shifts[s]}(k, m), the estimate of
 * n_-(A - shifts[s] I).  Slice counts are differences of consecutive
 * entries.  per_probe_quad: double[nshift*nprobe] (may be NULL),
 * steps_used: int[nshift] (may be NULL).                                      */
int evc_count_slices(evc_ctx* ctx, const double* shifts, int nshift, int nprobe,
                     int maxsteps, double tol, uint64_t seed, double* n_below,
                     double* per_probe_quad, int* steps_used);

/* Same as evc_count_slices, but leaves the results on the device: d_quad
 * (double[nshift*nprobe]), d_n_below (double[nshift]) and d_steps
 * (int32[nshift]) are device pointers (any may be NULL).  Enqueues the work
 * on the context's stream and returns without waiting; errors raised on the
 * device are reported by the next synchronising call.                         */
int evc_count_slices_async(evc_ctx* ctx, const double* shifts, int nshift, int nprobe,
                           int maxsteps, double tol, uint64_t seed, double* d_n_below,
                           double* d_quad, int* d_steps);

/* Wait for the context's stream and report any error raised on the device by
 * the work enqueued so far.                                                   */
int evc_sync(evc_ctx* ctx);

/* The tridiagonal matrices of the last call (Sec. 3, Eq. Tk), for
 * diagnostics: alpha[c*maxsteps + i] = alpha_{i+1}, beta[c*(maxsteps+1) + i]
 * = beta_{i+1} (beta_1 = 0) of column c = s*nprobe + j; kdone[c] = steps the
 * column completed (< maxsteps after a Lanczos breakdown or its shift's stop).
 * After a shared-Krylov call (EVC_OPT_SHARED_KRYLOV) the tridiagonal of
 * column s*nprobe + j is probe j's J_k(A) - shifts[s] I.  Host arrays of the
 * sizes implied by the last call's nshift, nprobe and maxsteps.              */
int evc_get_tridiag(evc_ctx* ctx, double* alpha, double* beta, int* kdone);

/* The computable factor of the Gauss quadrature error bound of the last call
 * (Sec. 3, Eq. qbound): per column c = s*nprobe + j, after the column's
 * k = kdone[c] steps,
 *     log10_bound[c] = log10( ||v||^2 beta_2^2 ... beta_{k+1}^2 / (2k)! ),
 * so that |eps_k| <= N_k * 10^log10_bound[c] for every smooth stand-in of the
 * step function h that agrees with it on the spectrum and the Ritz values,
 * N_k bounding its 2k-th derivative there (||v||^2 = n for the Rademacher
 * probes).  -inf when a beta_j is exactly zero (the process broke down: the
 * rule is exact, Proposition 1); NaN for a column with no steps.  Host array
 * double[nshift*nprobe] of the last call.  EVC_EUNSUPPORTED after an Arnoldi
 * call (no tridiagonal).  A diagnostic: the count does not use it.            */
int evc_get_quad_bound(evc_ctx* ctx, double* log10_bound);

/* Options.
 *   EVC_OPT_GRAPH     : 1 (default) replays the whole multi-step launch
 *                       sequence as one CUDA graph, 0 launches kernels one by one.
 *   EVC_OPT_PROFILE   : 1 brackets every kernel launch with a pair of timing
 *                       events on the context's stream (inside the graph when
 *                       graphs are on); 0 (default) records nothing.
 *   EVC_OPT_QUADRATURE: EVC_QUAD_GAUSS (default) uses the Gauss rule of J_k
 *                       (Sec. 3, Eq. gauss_quad); EVC_QUAD_GA the generalized
 *                       averaged Gauss rule, i.e. the same weights taken from
 *                       the (2k-1)-order extension of J_k built by mirroring
 *                       its coefficients around beta_{k+1} (Sec. 3.4,
 *                       Eq. GA_Tk).  Same Lanczos steps, different step 5 of
 *                       Algorithm 2.
 *   EVC_OPT_MIN_STEPS : under a tolerance (tol > 0), no shift stops before
 *                       this step (default 3, at least 3).
 *   EVC_OPT_PROBE_OFFSET: the calls that follow use probe ids offset..offset+
 *                       nprobe-1 (default 0), so that shards of one count can
 *                       run on different GPUs and be combined: the union of the
 *                       shards is the same probe set as one unsharded call.
 *   EVC_OPT_CHEB_FORM : how M = p_d(K) is applied.  EVC_CHEB_FACTORED (default)
 *                       multiplies the factors of p_d (roots found when the
 *                       preconditioner is set; a conjugate pair of roots gives
 *                       the factor (K - re)^2 + im^2, two passes that move 5
 *                       vectors); EVC_CHEB_CLENSHAW runs Clenshaw's recurrence,
 *                       one pass per degree moving 4 vectors.  The same operator
 *                       up to rounding.  When the factorisation fails its check
 *                       at EVC_PREC_CHEB_KINETIC time, Clenshaw's recurrence is
 *                       used whatever this option says.
 *   EVC_OPT_BASIS_BF16: EVC_MIXED contexts only; 1 rounds every Lanczos basis
 *                       vector to BF16 (round to nearest even) when it is
 *                       stored after reorthogonalisation, and takes beta_{i+1}
 *                       as the norm of the rounded vector: the numerics of a
 *                       BF16 basis with an FP32 working vector.  The storage
 *                       itself stays FP32, so this measures the accuracy of
 *                       BF16 storage, not its bandwidth.  Default 0.
 *   EVC_OPT_REORTH_ROWS: rows per block of the reorthogonalisation kernels
 *                       (default 0 = min(3456, max(64, ceil(n/64))); otherwise at
 *                       least 64, and at most max(ceil(n/1728), min(ceil(n/64),
 *                       512)) blocks per chunk).  It sets the summation
 *                       order of the dot products, so results may change in the
 *                       last bits; it never depends on how many columns a call
 *                       batches, so a column's result is the same alone or in
 *                       a batch for one setting.
 *   EVC_OPT_STENCIL_ZB: stencil contexts: z planes per block of the stencil
 *                       pass (default 32).  Results are unchanged.
 *   EVC_OPT_STENCIL_PATCH: stencil contexts: points per thread of the stencil
 *                       pass, 1 (default) or 2 = a 2 x 2 patch of (x, y) points
 *                       whose inner neighbours come from registers (fewer loads
 *                       per output; passes without Jacobi scaling and grids
 *                       with N even, else 1 is used), or 3 = the 2 x 2 patches
 *                       of a block tile (8 x 8 points FP32, 8 x 4 FP64) whose
 *                       input tile, stencil arms and pointwise operands are
 *                       staged in shared memory by tiled tensor copies, plane
 *                       by plane (N a multiple of the tile, else 2 is used).
 *                       2 and 3 give bitwise the same results; they agree with
 *                       1 to rounding.
 *   EVC_OPT_STENCIL_GROUPS: stencil contexts: 1 (default) to 4.  The stencil
 *                       passes of each step's operator application run as this
 *                       many groups of column chunks, each group on its own
 *                       stream (forked from and joined back into the context's
 *                       stream, inside the captured graph), so that one group's
 *                       passes fill the SMs another group's tail wave leaves
 *                       idle.  At most one group per chunk.  Results are
 *                       bitwise unchanged.  With profiling on, each segment is
 *                       timed as one span record (see evc_prof_rec).
 *   EVC_OPT_SHARED_KRYLOV: 1 (default): a call with several shifts under the
 *                       identity preconditioner (Lanczos) runs one Lanczos
 *                       process per probe, on A itself, and reads every shift's
 *                       quadrature from its J_k: the Krylov space of A - tau I
 *                       does not depend on tau and J_k(A - tau I) = J_k(A) -
 *                       tau I, so shift tau sums the Gauss weights of the Ritz
 *                       values below tau (Sec. 3, Eq. gauss_quad).  The m probe
 *                       columns run while any shift runs; a shift's stop rule
 *                       and results are its own.  Results equal per-shift runs
 *                       up to rounding.  0: one run per shift.  Other
 *                       preconditioners depend on the shift (Jacobi) or make the
 *                       operator M A M - tau M^2 (Chebyshev), whose Krylov space
 *                       moves with tau: they always run per shift.
 *   EVC_OPT_CSR_THREADS: CSR contexts: threads per block of the CSR pass, 128,
 *                       256 (default) or 512.  Results are unchanged.
 *   EVC_OPT_METHOD    : EVC_METHOD_LANCZOS (default): Algorithms 1-2 on
 *                       C = M (A - tau I) M.  EVC_METHOD_ARNOLDI: the
 *                       preconditioned Arnoldi-type estimator of Sec. 4 -- the
 *                       Arnoldi process (Algorithm 3) on C = T (A - tau I) with T
 *                       used without its factorisation (Jacobi: T = diag(1/(|a_ii
 *                       - tau| + eps)); Chebyshev: T = p_d(K)^2; identity), the
 *                       quadrature ||v||^2 Re(e_1^T h(H_k) e_1) with h = 1 on the
 *                       open left half-plane (Eq. arnoldi_quad), the same probes,
 *                       means and stop rule.  At most 90 steps; the Gauss rule
 *                       only; evc_get_tridiag does not apply.  Per-probe values
 *                       may be negative (the weights are complex).
 *   EVC_OPT_TINV_LANCZOS: 0 (default): Algorithm 1 on C = M (A - tau I) M.
 *                       1: the T^{-1}-inner-product Lanczos process of Sec. 4
 *                       (Eq. lanT1), T (A - tau I) Y_k = Y_{k+1} J_{k+1,k} with
 *                       Y^T T^{-1} Y = I, started from y_1 = M q_1, for the
 *                       Jacobi preconditioner T = M^2 = diag(1/(|a_ii - tau| +
 *                       eps)): the operator pass scales its output rows by T and
 *                       not its gathered operands, and the reorthogonalisation's
 *                       inner products and norms carry the weight T^{-1} =
 *                       diag(|a_ii - tau| + eps).  Y_k = M Q_k, so J_k, the
 *                       quadratures and the estimate equal Algorithm 1's up to
 *                       rounding.  Identity preconditioner: the same process as
 *                       Algorithm 1 (T = I).  The kinetic Chebyshev preconditioner
 *                       and the Arnoldi method return EVC_EUNSUPPORTED at the
 *                       count (the start z_1 = T^{-1} y_1 = M^{-1} q_1 would need
 *                       a solve with p_d(K)).  */
enum {
    EVC_OPT_GRAPH = 1,
    EVC_OPT_PROFILE = 2,
    EVC_OPT_QUADRATURE = 3,
    EVC_OPT_MIN_STEPS = 4,
    EVC_OPT_PROBE_OFFSET = 5,
    EVC_OPT_CHEB_FORM = 6,
    EVC_OPT_BASIS_BF16 = 7,
    EVC_OPT_REORTH_ROWS = 8,
    EVC_OPT_STENCIL_ZB = 9,
    EVC_OPT_CSR_THREADS = 10,
    EVC_OPT_METHOD = 11,
    EVC_OPT_STENCIL_PATCH = 12,
    EVC_OPT_STENCIL_GROUPS = 13,
    EVC_OPT_SHARED_KRYLOV = 14,
    EVC_OPT_TINV_LANCZOS = 15
};
enum { EVC_METHOD_LANCZOS = 0, EVC_METHOD_ARNOLDI = 1 };
enum { EVC_CHEB_FACTORED = 0, EVC_CHEB_CLENSHAW = 1 };
enum { EVC_QUAD_GAUSS = 0, EVC_QUAD_GA = 1 };
int evc_set_option(evc_ctx* ctx, int option, int64_t value);

/* Kernel classes reported by evc_get_profile.                               */
enum {
    EVC_K_INIT = 0,      /* probe generation and state reset                  */
    EVC_K_JACOBI = 1,    /* Jacobi scales per shift                           */
    EVC_K_STENCIL = 2,   /* one stencil pass (Chebyshev step / H apply)       */
    EVC_K_CSR = 3,       /* CSR operator apply                                */
    EVC_K_DOTS = 4,      /* reorthogonalisation dot products                  */
    EVC_K_REDUCE = 5,    /* dot-product reduction, alpha, coefficients        */
    EVC_K_UPDATE = 6,    /* reorthogonalisation update and norm               */
    EVC_K_FINISH = 7     /* beta, eigensolve, quadrature, stop rule           */
};

/* One kernel launch of the last call: its class, Lanczos step (0 = set-up),
 * device time in milliseconds (events on the context's stream; -1 when
 * profiling was off) and the compulsory HBM bytes of the launch (every
 * operand read once, every output written once, all chunks active).
 * With stencil chunk groups (EVC_OPT_STENCIL_GROUPS > 1) the launches of a
 * step's operator segment run concurrently on several streams: they carry
 * ms = -1 and their group's share of the bytes, and one extra record with
 * span = 1 covers the segment -- its wall time on the context's stream and
 * the compulsory bytes of all its launches.  span = 0 for a launch.          */
typedef struct {
    int32_t kind;
    int32_t step;
    double ms;
    double bytes;
    int32_t span;
    int32_t reserved;
} evc_prof_rec;

/* Launch list of the last call.  Writes min(cap, records) records to recs
 * (may be NULL) and the number of records of one call (launches plus span
 * records) to *nrec.  Synchronises the context's stream.                     */
int evc_get_profile(evc_ctx* ctx, evc_prof_rec* recs, int cap, int* nrec);

/* evc_autotune -- the library's tile-shape autotuner.  Times short counts
 * (min(maxsteps, 6) Lanczos steps, nshift placeholder shifts, nprobe probes:
 * the caller's launch shape) with a pair of timing events around every kernel,
 * and keeps, per kernel family, the fastest of
 *   stencil pass:  z planes per block 16 / 32 / 64 (EVC_OPT_STENCIL_ZB) times
 *                  points per thread 1 / 2x2 / 2x2 in tensor-copied tiles
 *                  (EVC_OPT_STENCIL_PATCH), then
 *                  1 / 2 / 4 concurrent chunk groups (EVC_OPT_STENCIL_GROUPS), and
 *                  the shapes once more if the groups changed,
 *   CSR pass:      threads per block 128 / 256 / 512 (EVC_OPT_CSR_THREADS),
 *   reorthogonalisation: rows per block 64 ... 13824 within the allowed
 *                  block counts (EVC_OPT_REORTH_ROWS),
 * tuning the operator pass first.  The choice stays in the context for later
 * calls (and contexts cloned from it); `out` (may be NULL) reports it with the
 * device time of one short count before and after.  Needs the workspace of a
 * call with (nshift, nprobe, min(maxsteps, 6)) -- a workspace set for the
 * real call is enough; every configuration fits it.  On error the previous
 * settings are restored.  Not part of the paper: tile shapes are a property of
 * the GPU, the grid and the batch. */
typedef struct {
    int stencil_zb;      /* chosen z planes per block (stencil contexts), else 0 */
    int stencil_patch;   /* chosen EVC_OPT_STENCIL_PATCH value 1, 2 or 3 (stencil contexts), else 0 */
    int stencil_groups;  /* chosen concurrent chunk groups (stencil contexts), else 0 */
    int csr_threads;     /* chosen threads per block (CSR contexts), else 0 */
    int reorth_rows;     /* chosen rows per block of the reorthogonalisation */
    int steps;           /* Lanczos steps of each timing count */
    double ms_before;    /* device time of one timing count before tuning */
    double ms_after;     /* ... and with the chosen shapes */
} evc_tuning;
int evc_autotune(evc_ctx* ctx, int nshift, int nprobe, int maxsteps, evc_tuning* out);

/* ------------------------------------------------------------------------
 * Request server: interval counts on several resident matrices, served as
 * requests arrive (the spectrum-slicing use of Sec. 1, many independent
 * counts).
 *
 * A scheduler thread keeps the waiting requests in arrival order.  Whenever
 * one of `slots` execution slots is idle it forms a batch: the oldest waiting
 * request plus later requests that can share its launch (same matrix, nprobe
 * and seed; tol and maxsteps may differ), at most max_batch of them and only
 * as many as fit the HBM budget (the batch's workspace, evc_workspace_bytes
 * of 2 shifts per request at the batch's largest maxsteps).  A batch is one
 * batched count on the slot's own stream in which every shift keeps its own
 * request's tol and maxsteps, so batches on different slots overlap on the
 * device; under the identity preconditioner the batch's shifts share one
 * Lanczos run per probe (EVC_OPT_SHARED_KRYLOV).  Memory and slots return
 * when a batch ends and waiting requests are admitted then.
 * The oldest request is never overtaken; one that cannot fit even with
 * nothing running fails with EVC_ENOMEM.  Each request's result equals the
 * result of the same request run alone (columns are independent and every
 * reduction has a batch-independent order).  A launch flags a numeric
 * failure (EVC_ENUMERIC) once for all its columns, so a merged batch that
 * fails is run again request by request: only the request whose own columns
 * fail reports it.
 * ------------------------------------------------------------------------ */
typedef struct evc_server evc_server;

typedef struct {
    int32_t status;       /* evc_status of the request                          */
    int32_t batch_size;   /* requests that shared its launch                    */
    double estimate;      /* L_eta - L_xi                                        */
    double n_below[2];    /* L_xi, L_eta                                         */
    int32_t steps[2];     /* Lanczos steps used per shift                        */
    double t_submit;      /* seconds since the server started: submission,      */
    double t_start;       /*   admission of its batch,                          */
    double t_done;        /*   completion                                       */
} evc_result;

typedef struct {
    uint64_t budget_bytes, used_bytes, peak_bytes;   /* HBM admission accounting */
    int64_t pending;      /* requests waiting                                   */
    int64_t batches;      /* batches launched                                   */
    int64_t completed;    /* requests finished                                  */
    int64_t merged;       /* requests that joined another request's batch       */
} evc_server_counters;

/* hbm_budget_bytes: device memory the workspaces of running batches may use
 * together; slots: batches in flight at once (1..64); max_batch: requests
 * per batch (1..1024).  Uses the current CUDA device.                         */
int evc_server_create(size_t hbm_budget_bytes, int slots, int max_batch, evc_server** out);

/* Register a configured context (matrix + preconditioner + options); the
 * server borrows it (it must outlive the server).  *matrix_id receives its id. */
int evc_server_add_matrix(evc_server* srv, evc_ctx* ctx, int* matrix_id);

/* Queue one count of the eigenvalues in [xi, eta] (arguments as evc_count).
 * per_probe_quad: optional host buffer of 2*nprobe doubles, filled on
 * completion; it must stay valid until then.  Returns at once.                */
int evc_server_submit(evc_server* srv, int matrix_id, double xi, double eta, int nprobe,
                      int maxsteps, double tol, uint64_t seed, double* per_probe_quad,
                      int64_t* ticket);

/* Result of a finished request: EVC_EAGAIN while it is still queued or
 * running; otherwise the request's status, *res filled and the ticket
 * released.  evc_server_wait blocks up to timeout_s seconds (< 0: forever).  */
int evc_server_poll(evc_server* srv, int64_t ticket, evc_result* res);
int evc_server_wait(evc_server* srv, int64_t ticket, double timeout_s, evc_result* res);

int evc_server_stats(evc_server* srv, evc_server_counters* stats);

/* Finish every queued request, then stop the threads and free the server.     */
void evc_server_destroy(evc_server* srv);

/* Allocation-free batched Gauss quadrature.  The paper has no counterpart.
 *
 * For callers that cannot allocate device memory at the point of the call:
 * code running while another framework is capturing a CUDA graph, code under
 * a memory pool or budget that forbids new allocations, or runtimes that
 * have no device allocator of their own.  Nothing here calls cudaMalloc,
 * cudaFree or any allocating routine; the only device memory used besides
 * the caller's inputs and outputs is one fixed scratch array compiled into
 * libevc (3 * EVC_STATIC_QUAD_MAX doubles = 6 MiB), which every GPU that
 * loads the library holds until the process exits.
 *
 * It computes the same quadrature as the last step of evc_count_slices
 * (Sec. 3, Eq. gauss_quad): for each column c, ||v||^2 sum over the negative
 * eigenvalues theta of J_kc of z(1)^2, from coefficients laid out as the
 * estimator keeps them on the device:
 *   d_alpha : double[k * ncol],     d_alpha[t*ncol + c] = alpha_{t+1}
 *   d_beta  : double[(k+1) * ncol], d_beta[t*ncol + c]  = beta_{t+1} (t >= 1 used)
 *   d_kcol  : int32[ncol] per-column sizes 1 <= kc <= k, or NULL for k
 *   vnorm2  : ||v||^2 (n for the library's Rademacher probes), finite, >= 0
 *   d_quad  : double[ncol] output
 *   d_status: int32[1] output, or NULL: set to EVC_OK on the stream before the
 *             kernel runs, then to the first failure the kernel meets --
 *             EVC_EINVAL for a d_kcol entry outside [1, k] (that column is
 *             not computed) or EVC_ENUMERIC for an eigensolve that did not
 *             converge (non-finite input); such columns get NaN in d_quad.
 * All pointers are device pointers; the call only enqueues a 4-byte memset
 * of d_status (when given) and one kernel on `stream` (NULL = legacy default
 * stream) and returns, so d_status is meaningful once the stream has reached
 * that point (synchronise, or order later work after it).
 * Limits: 1 <= k <= EVC_MAX_STEPS, ncol >= 1, k * ncol <= EVC_STATIC_QUAD_MAX;
 * larger requests return EVC_EINVAL without launching anything, with a
 * message in errbuf (optional host buffer of errlen bytes).
 * The first call on a device looks up the device address of the scratch
 * array (cudaGetSymbolAddress) with that device current, so make that first
 * call outside any stream capture.  Every call reuses the same array and the
 * kernel writes each scratch entry before reading it, so a previous call's
 * leftovers do not matter; but calls whose kernels can overlap on the GPU
 * (different streams without ordering between them) race on the array and
 * give wrong results -- serialise them.                                       */
#define EVC_STATIC_QUAD_MAX 262144
int evc_gauss_quadrature_static(const double* d_alpha, const double* d_beta, const int* d_kcol,
                                int k, int ncol, double vnorm2, double* d_quad, int* d_status,
                                void* stream, char* errbuf, size_t errlen);

/* evc_wait_selftest -- checks the failure detection of the streaming kernels
 * without making the GPU fault or hang.  Every device-side wait of the library
 * (on an mbarrier phase or a copy) gives up after a bounded number of SM clock
 * cycles, records a timeout and lets the kernel return, and the call that
 * launched it reports EVC_ETIMEOUT.  This entry runs one block whose wait can
 * never complete (nothing arrives on its barrier) with a limit of limit_ms
 * milliseconds (0 < limit_ms <= 2000, converted with the SM clock rate),
 * synchronises the device and stores in *status the status that the wait
 * produced: EVC_ETIMEOUT when the bounded wait gave up as designed.  Returns
 * EVC_OK when the launch and the read-back succeeded (the context is still
 * usable), EVC_EINVAL / EVC_ENOMEM / EVC_ECUDA otherwise.  It allocates and
 * frees 4 bytes of device memory and uses the current device.  Not part of the
 * paper: a property of this implementation. */
int evc_wait_selftest(double limit_ms, int* status);

const char* evc_last_error(const evc_ctx* ctx);
void evc_destroy(evc_ctx* ctx);
/* Library version, major*10000 + minor*100 + patch.                           */
int evc_version(void);

/* evc_cheb_kinetic -- host only, no device work: the kinetic-energy
 * Chebyshev preconditioner M = p_d(K), K = -1/2 Lap_h + cI, exactly as
 * evc_set_precond(ctx, EVC_PREC_CHEB_KINETIC, degree, c) builds it for a
 * periodic stencil of this order (2: 7-point, 4: 13-point) and spacing h
 * (Sec. 6, the kinetic-energy preconditioning of the numerical examples):
 * p_d interpolates x^(-1/2) at the d+1 Chebyshev points of the first kind on
 * [a, b] = [c, c + 6/h^2] (order 2) or [c, c + 8/h^2] (order 4), the bounds of
 * spec(K) from the stencil's symbol.
 *   info[5]    out: a, b, min of p_d over the exact spectrum of K on an N^3
 *              grid (0 when N = 0: not evaluated; evc_set_precond rejects a
 *              grid where it is not > 0), g, sign;
 *   coef[d+1]  out: p_d(x) = sum_j coef[j] T_j((2x - a - b)/(b - a));
 *   factors[3*d], *nfac  out: the factored form the stencil passes apply,
 *              p_d(x) = sign * prod over factors, a factor (re, im, 1) being
 *              g^2 ((x - re)^2 + im^2) (a conjugate pair of roots) and (r, 0, 0)
 *              being g (x - r) (a real root); pairs first, each group by
 *              ascending re.  *nfac = 0 when the factored product fails to
 *              reproduce the series to 1e-9 relative on [a, b] (the library
 *              then uses Clenshaw's recurrence).
 * All buffers are caller-owned host memory.  Returns EVC_OK, or EVC_EINVAL
 * for a null buffer, N < 0, an order other than 2 / 4, h <= 0, a degree
 * outside [1, 32] or c <= 0. */
int evc_cheb_kinetic(int order, double h, int degree, double c, int N, double* info,
                     double* coef, double* factors, int* nfac);

#ifdef __cplusplus
}
#endif
#endif /* EVC_H */
