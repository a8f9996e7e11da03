/*
 * evc_oracle.h -- plain FP64 CPU oracle of the preconditioned Lanczos
 * eigenvalue-count estimator (Vecharynski & Yang, "Preconditioned iterative
 * methods for eigenvalue counts").
 *
 * TEST INFRASTRUCTURE ONLY. This oracle exists to check the CUDA library and
 * to be timed as a CPU baseline. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header, table
 * or helper with the CUDA library.
 *
 * Everything is float64. Arrays are caller-owned. Functions return 0 on
 * success and a negative value on invalid arguments.
 */
#ifndef EVC_ORACLE_H
#define EVC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { EVO_OP_DENSE = 0, EVO_OP_CSR = 1, EVO_OP_STENCIL = 2 };
enum { EVO_PREC_NONE = 0, EVO_PREC_JACOBI = 1, EVO_PREC_CHEB = 2, EVO_PREC_DENSE = 3 };

/* The matrix A and the HPD preconditioner T = M*M (M symmetric here).
 *   op_kind DENSE   : dense[n*n], row-major.
 *   op_kind CSR     : row_ptr[n+1], col[nnz], val[nnz] (duplicates allowed).
 *   op_kind STENCIL : H = -1/2 Lap_h + diag(V) on a periodic N^3 grid, spacing
 *                     h; order 2 = 7-point, order 4 = 13-point Laplacian;
 *                     point p = x + N*(y + N*z); V[N^3].
 *   prec_kind NONE  : M = I.
 *   prec_kind JACOBI: M = diag((|a_ii - tau| + jac_eps)^(-1/2)).
 *   prec_kind CHEB  : M = p_d(K), K = -1/2 Lap_h + cheb_c I (stencil only),
 *                     p_d the degree-d Chebyshev interpolant of x^(-1/2) on
 *                     the closed-form spectral interval of K.
 *   prec_kind DENSE : M = denseM[n*n] (symmetric), for small pins.         */
typedef struct {
    int64_t n;
    int32_t op_kind;
    int32_t prec_kind;
    const double* dense;
    const int64_t* row_ptr;
    const int32_t* col;
    const double* val;
    int32_t N;
    int32_t order;
    double h;
    const double* V;
    double jac_eps;
    int32_t cheb_degree;
    int32_t reserved;
    double cheb_c;
    const double* denseM;
} evo_problem;

/* SplitMix64 output finalizer (Steele, Lea & Flood 2014). */
uint64_t evo_mix64(uint64_t z);
/* Rademacher probe entry v_j[i] in {-1, +1}: x = mix64(seed ^ mix64((j<<32)|i)),
 * -1 when bit 63 of x is set. */
double evo_probe_entry(uint64_t seed, uint64_t j, uint64_t i);
void evo_probe_vector(uint64_t seed, uint64_t j, int64_t n, double* v);

int evo_apply_A(const evo_problem* P, const double* x, double* y);
int evo_apply_M(const evo_problem* P, double tau, const double* x, double* y);
/* y = C x with C = M (A - tau I) M. */
int evo_apply_C(const evo_problem* P, double tau, const double* x, double* y);
/* Chebyshev interpolation coefficients of x^(-1/2) on [a, b]; coef[degree+1]. */
int evo_cheb_coeffs(int degree, double a, double b, double* coef);
/* Closed-form spectral interval [a, b] of K = -1/2 Lap_h + c I. */
int evo_kinetic_interval(const evo_problem* P, double* a, double* b);

/* k steps of the Lanczos procedure for C = M(A - tau I)M with start vector v.
 * alpha[k]: alpha[i-1] = alpha_i.  beta[k+1]: beta[0] = beta_1 = 0,
 * beta[i] = beta_{i+1}.  Q (optional, may be NULL): n x (k+1), column-major,
 * Q[j*n + r] = (q_{j+1})_r.  Stops early at breakdown, when
 * beta_{i+1} <= breakdown_rel * max_{j<=i}(|alpha_j|, beta_j); *k_done = the
 * number of completed steps. */
int evo_lanczos(const evo_problem* P, double tau, const double* v, int k,
                double breakdown_rel, double* alpha, double* beta, double* Q,
                int* k_done);

/* Eigen-decomposition of the k x k symmetric tridiagonal J_k (diagonal
 * alpha[0..k-1], off-diagonal beta[1..k-1], i.e. the beta layout above) by
 * the cyclic Jacobi rotation method. theta[k] ascending, z1[k] = first
 * components of the unit eigenvectors. */
int evo_tridiag_eig(int k, const double* alpha, const double* beta,
                    double* theta, double* z1);

/* Gauss quadrature ||v||^2 sum_{theta_i < 0} z_i(1)^2 from J_k. */
double evo_gauss_quad(int k, const double* alpha, const double* beta, double vnorm2);

/* Generalized averaged Gauss quadrature (Sec. 3.4, Eq. GA_Tk) from J_{k+1,k}:
 * the Gauss formula on the mirrored (2k-1) x (2k-1) extension; beta[k] =
 * beta_{k+1} is used. */
double evo_ga_quad(int k, const double* alpha, const double* beta, double vnorm2);

/* The estimator L_tau(k, m) for S shifts with m probes each.
 * Column (s, j) uses probe id probe_ids[j] (or j if probe_ids is NULL) and the
 * seeded Rademacher probe above; the same probes serve every shift.
 * tol <= 0: every shift runs kmax steps. tol > 0: shift s stops at the first
 * step i >= 3 with |L_s(i) - L_s(i-1)| <= tol and |L_s(i-1) - L_s(i-2)| <= tol
 * (kmax caps it).
 * Outputs: quad[s*m + j], steps[s], L[s] (= mean_j quad[s*m + j]).
 * nthreads <= 0: OpenMP default. */
int evo_count(const evo_problem* P, const double* shifts, int S, int m,
              const int64_t* probe_ids, int kmax, double tol, uint64_t seed,
              double breakdown_rel, int nthreads,
              double* quad, int* steps, double* L);
/* Same with the quadrature rule chosen (rule 0 = Gauss, 1 = generalized
 * averaged Gauss) and no tolerance stop before step max(3, min_steps). */
int evo_count_rule(const evo_problem* P, const double* shifts, int S, int m,
                   const int64_t* probe_ids, int kmax, double tol, uint64_t seed,
                   double breakdown_rel, int nthreads, int rule, int min_steps,
                   double* quad, int* steps, double* L);

#ifdef __cplusplus
}
#endif
#endif
