/*
 * evc_oracle.c -- plain FP64 CPU oracle of the preconditioned Lanczos
 * eigenvalue-count estimator (Vecharynski & Yang).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path. It is written for
 * obviousness, not speed: every step follows the paper's definition in the
 * paper's order, in float64, with OpenMP only across independent probes.
 *
 * Where each function comes from:
 *   probe            Sec. 2, Eq. (trace): i.i.d. zero-mean unit-variance
 *                    entries; Rademacher signs drawn by SplitMix64.
 *   apply_C          Sec. 2, Eq. (negi_T): C = M (A - tau I) M*, T = M*M.
 *   Jacobi M         diagonal HPD T = 1/(|a_ii - tau| + eps) (Sec. 6 lists
 *                    HPD choices; this one is the diagonal special case).
 *   Chebyshev M      Sec. 6 (kinetic-energy preconditioner, Teter analogue in
 *                    real space): M = p_d(K) ~ K^(-1/2), K = -1/2 Lap_h + cI.
 *   evo_lanczos      Sec. 3, Algorithm 1 (Lanczos with full
 *                    reorthogonalisation), Eq. (lan), Eq. (Tk).
 *   evo_tridiag_eig  eigenpairs of J_k (Sec. 3, Eq. gauss_quad) by cyclic
 *                    Jacobi rotations (a textbook method, not the GPU's).
 *   evo_gauss_quad   Sec. 3, Eq. (gauss_quad): ||v||^2 sum_{theta<0} z(1)^2.
 *   evo_count        Sec. 3, Algorithm 2 and Eq. (rand_prec_quad), run for
 *                    several shifts (Sec. 3, the two-run interval count).
 */
#include "evc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- probes */

uint64_t evo_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

double evo_probe_entry(uint64_t seed, uint64_t j, uint64_t i)
{
    uint64_t x = evo_mix64(seed ^ evo_mix64((j << 32) | i));
    return (x >> 63) ? -1.0 : 1.0;
}

void evo_probe_vector(uint64_t seed, uint64_t j, int64_t n, double* v)
{
    for (int64_t i = 0; i < n; ++i) v[i] = evo_probe_entry(seed, j, (uint64_t)i);
}

/* ---------------------------------------------------------------- helpers */

static double dot(int64_t n, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* -1/2 times the periodic finite-difference Laplacian of x on the N^3 grid.
 * order 2: second difference (u[-1] - 2u + u[+1]) / h^2 per axis.
 * order 4: (-u[-2] + 16u[-1] - 30u + 16u[+1] - u[+2]) / (12 h^2) per axis. */
static void minus_half_laplacian(int N, double h, int order, const double* x, double* y)
{
    const double ih2 = 1.0 / (h * h);
    for (int z = 0; z < N; ++z)
        for (int yy = 0; yy < N; ++yy)
            for (int xx = 0; xx < N; ++xx) {
                int64_t p = xx + (int64_t)N * (yy + (int64_t)N * z);
                double lap = 0.0;
                for (int axis = 0; axis < 3; ++axis) {
                    double u[5];
                    for (int o = -2; o <= 2; ++o) {
                        int cx = xx, cy = yy, cz = z;
                        if (axis == 0) cx = ((xx + o) % N + N) % N;
                        if (axis == 1) cy = ((yy + o) % N + N) % N;
                        if (axis == 2) cz = ((z + o) % N + N) % N;
                        u[o + 2] = x[cx + (int64_t)N * (cy + (int64_t)N * cz)];
                    }
                    if (order == 2)
                        lap += (u[1] - 2.0 * u[2] + u[3]) * ih2;
                    else
                        lap += (-u[0] + 16.0 * u[1] - 30.0 * u[2] + 16.0 * u[3] - u[4]) * ih2 / 12.0;
                }
                y[p] = -0.5 * lap;
            }
}

int evo_apply_A(const evo_problem* P, const double* x, double* y)
{
    const int64_t n = P->n;
    if (P->op_kind == EVO_OP_DENSE) {
        for (int64_t r = 0; r < n; ++r) y[r] = dot(n, P->dense + r * n, x);
    } else if (P->op_kind == EVO_OP_CSR) {
        for (int64_t r = 0; r < n; ++r) {
            double s = 0.0;
            for (int64_t k = P->row_ptr[r]; k < P->row_ptr[r + 1]; ++k) s += P->val[k] * x[P->col[k]];
            y[r] = s;
        }
    } else if (P->op_kind == EVO_OP_STENCIL) {
        minus_half_laplacian(P->N, P->h, P->order, x, y);
        for (int64_t r = 0; r < n; ++r) y[r] += P->V[r] * x[r];
    } else {
        return -1;
    }
    return 0;
}

static double diag_of_A(const evo_problem* P, int64_t r)
{
    if (P->op_kind == EVO_OP_DENSE) return P->dense[r * P->n + r];
    if (P->op_kind == EVO_OP_CSR) {
        double d = 0.0;
        for (int64_t k = P->row_ptr[r]; k < P->row_ptr[r + 1]; ++k)
            if (P->col[k] == r) d += P->val[k];
        return d;
    }
    /* -1/2 Lap_h has diagonal 3/h^2 (order 2) or 3 * 30/(24 h^2) (order 4). */
    double ih2 = 1.0 / (P->h * P->h);
    return P->V[r] + (P->order == 2 ? 3.0 * ih2 : 3.0 * 30.0 / 24.0 * ih2);
}

int evo_kinetic_interval(const evo_problem* P, double* a, double* b)
{
    if (P->op_kind != EVO_OP_STENCIL) return -1;
    /* Symbol of -1/2 d^2/dx^2 per axis at wavenumber theta:
     *   order 2: (1 - cos theta) / h^2,               max 2/h^2 at theta = pi;
     *   order 4: (30 - 32 cos theta + 2 cos 2theta) / (24 h^2), max 8/(3h^2).
     * Three axes, shifted by c. */
    double ih2 = 1.0 / (P->h * P->h);
    *a = P->cheb_c;
    *b = P->cheb_c + (P->order == 2 ? 6.0 * ih2 : 8.0 * ih2);
    return 0;
}

int evo_cheb_coeffs(int degree, double a, double b, double* coef)
{
    if (degree < 0 || !(b > a) || !(a > 0.0)) return -1;
    const double pi = 3.14159265358979323846;
    int np = degree + 1;
    for (int j = 0; j <= degree; ++j) {
        double s = 0.0;
        for (int k = 0; k < np; ++k) {
            double t = cos(pi * (k + 0.5) / np);           /* Chebyshev node  */
            double x = 0.5 * (b - a) * t + 0.5 * (a + b);  /* mapped to [a,b] */
            s += cos(j * pi * (k + 0.5) / np) / sqrt(x);   /* T_j(t) f(x)     */
        }
        coef[j] = 2.0 * s / np;
    }
    coef[0] *= 0.5;
    return 0;
}

/* y = p_d(K) x by the three-term recurrence T_{j+1}(K~) = 2 K~ T_j(K~) - T_{j-1}(K~),
 * K~ = (2K - (a+b) I)/(b-a), summing c_j T_j(K~) x. */
static int apply_cheb(const evo_problem* P, const double* x, double* y)
{
    const int64_t n = P->n;
    const int d = P->cheb_degree;
    double a, b;
    if (d < 0 || d > 64 || evo_kinetic_interval(P, &a, &b) != 0) return -1;
    double coef[65];
    if (evo_cheb_coeffs(d, a, b, coef) != 0) return -1;
    double* tprev = (double*)malloc(sizeof(double) * n);
    double* tcur = (double*)malloc(sizeof(double) * n);
    double* tnext = (double*)malloc(sizeof(double) * n);
    double* kx = (double*)malloc(sizeof(double) * n);
    if (!tprev || !tcur || !tnext || !kx) { free(tprev); free(tcur); free(tnext); free(kx); return -2; }
    /* K~ u = (2 (-1/2 Lap_h u + c u) - (a+b) u) / (b-a) */
    #define KTILDE(in, out)                                                         \
        do {                                                                        \
            minus_half_laplacian(P->N, P->h, P->order, (in), kx);                   \
            for (int64_t r = 0; r < n; ++r)                                          \
                (out)[r] = (2.0 * (kx[r] + P->cheb_c * (in)[r]) - (a + b) * (in)[r]) / (b - a); \
        } while (0)
    for (int64_t r = 0; r < n; ++r) { tprev[r] = x[r]; y[r] = coef[0] * x[r]; }
    if (d >= 1) {
        KTILDE(x, tcur);
        for (int64_t r = 0; r < n; ++r) y[r] += coef[1] * tcur[r];
    }
    for (int j = 2; j <= d; ++j) {
        KTILDE(tcur, tnext);
        for (int64_t r = 0; r < n; ++r) {
            tnext[r] = 2.0 * tnext[r] - tprev[r];
            y[r] += coef[j] * tnext[r];
        }
        double* t = tprev; tprev = tcur; tcur = tnext; tnext = t;
    }
    #undef KTILDE
    free(tprev); free(tcur); free(tnext); free(kx);
    return 0;
}

int evo_apply_M(const evo_problem* P, double tau, const double* x, double* y)
{
    const int64_t n = P->n;
    switch (P->prec_kind) {
    case EVO_PREC_NONE:
        memcpy(y, x, sizeof(double) * n);
        return 0;
    case EVO_PREC_JACOBI:
        for (int64_t r = 0; r < n; ++r)
            y[r] = x[r] / sqrt(fabs(diag_of_A(P, r) - tau) + P->jac_eps);
        return 0;
    case EVO_PREC_CHEB:
        return apply_cheb(P, x, y);
    case EVO_PREC_DENSE:
        for (int64_t r = 0; r < n; ++r) y[r] = dot(n, P->denseM + r * n, x);
        return 0;
    default:
        return -1;
    }
}

int evo_apply_C(const evo_problem* P, double tau, const double* x, double* y)
{
    const int64_t n = P->n;
    double* u = (double*)malloc(sizeof(double) * n);
    double* t = (double*)malloc(sizeof(double) * n);
    if (!u || !t) { free(u); free(t); return -2; }
    int rc = evo_apply_M(P, tau, x, u);                     /* u = M x           */
    if (rc == 0) rc = evo_apply_A(P, u, t);                 /* t = A u           */
    if (rc == 0) {
        for (int64_t r = 0; r < n; ++r) t[r] -= tau * u[r]; /* t = (A - tau I) u */
        rc = evo_apply_M(P, tau, t, y);                     /* y = M t           */
    }
    free(u); free(t);
    return rc;
}

/* ---------------------------------------------------------------- Lanczos */

int evo_lanczos(const evo_problem* P, double tau, const double* v, int k,
                double breakdown_rel, double* alpha, double* beta, double* Q,
                int* k_done)
{
    const int64_t n = P->n;
    if (k < 1 || n < 1) return -1;
    double* basis = Q ? Q : (double*)malloc(sizeof(double) * n * (size_t)(k + 1));
    double* w = (double*)malloc(sizeof(double) * n);
    double* hc = (double*)malloc(sizeof(double) * (size_t)(k + 1));
    if (!basis || !w || !hc) { if (!Q) free(basis); free(w); free(hc); return -2; }
    int rc = 0;
    /* Algorithm 1, first line: q1 = v/||v||, q0 = 0, beta_1 = 0, Q_1 = q1. */
    double vn = sqrt(dot(n, v, v));
    for (int64_t r = 0; r < n; ++r) basis[r] = v[r] / vn;
    beta[0] = 0.0;
    double scale = 0.0;
    int done = 0;
    for (int i = 1; i <= k; ++i) {
        const double* qi = basis + (size_t)(i - 1) * n;
        const double* qprev = (i >= 2) ? basis + (size_t)(i - 2) * n : NULL;
        /* w = M (A - tau I) M* q_i - beta_i q_{i-1} */
        rc = evo_apply_C(P, tau, qi, w);
        if (rc) break;
        if (qprev)
            for (int64_t r = 0; r < n; ++r) w[r] -= beta[i - 1] * qprev[r];
        /* alpha_i = q_i* w ; w = w - alpha_i q_i */
        alpha[i - 1] = dot(n, qi, w);
        for (int64_t r = 0; r < n; ++r) w[r] -= alpha[i - 1] * qi[r];
        /* full reorthogonalisation w = w - Q_i (Q_i* w), one classical pass */
        for (int j = 0; j < i; ++j) hc[j] = dot(n, basis + (size_t)j * n, w);
        for (int j = 0; j < i; ++j) {
            const double* qj = basis + (size_t)j * n;
            for (int64_t r = 0; r < n; ++r) w[r] -= hc[j] * qj[r];
        }
        /* beta_{i+1} = ||w|| ; q_{i+1} = w / beta_{i+1} */
        beta[i] = sqrt(dot(n, w, w));
        done = i;
        if (fabs(alpha[i - 1]) > scale) scale = fabs(alpha[i - 1]);
        if (beta[i - 1] > scale) scale = beta[i - 1];
        if (beta[i] <= breakdown_rel * scale) break;
        double* qn = basis + (size_t)i * n;
        for (int64_t r = 0; r < n; ++r) qn[r] = w[r] / beta[i];
    }
    for (int i = done + 1; i <= k; ++i) { alpha[i - 1] = 0.0; beta[i] = 0.0; }
    *k_done = done;
    if (!Q) free(basis);
    free(w); free(hc);
    return rc;
}

/* ------------------------------------------------------- tridiagonal eig */

int evo_tridiag_eig(int k, const double* alpha, const double* beta,
                    double* theta, double* z1)
{
    if (k < 1) return -1;
    double* A = (double*)calloc((size_t)k * k, sizeof(double));
    double* Z = (double*)calloc((size_t)k * k, sizeof(double));
    if (!A || !Z) { free(A); free(Z); return -2; }
    for (int i = 0; i < k; ++i) {
        A[i * k + i] = alpha[i];
        Z[i * k + i] = 1.0;
        if (i + 1 < k) { A[i * k + i + 1] = beta[i + 1]; A[(i + 1) * k + i] = beta[i + 1]; }
    }
    /* Cyclic Jacobi: rotate away each off-diagonal (p,q) in turn until the
     * off-diagonal mass is negligible against the whole matrix. */
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                tot += A[i * k + j] * A[i * k + j];
                if (i != j) off += A[i * k + j] * A[i * k + j];
            }
        if (off <= 1e-32 * tot || off == 0.0) break;
        for (int p = 0; p < k - 1; ++p)
            for (int q = p + 1; q < k; ++q) {
                double apq = A[p * k + q];
                if (apq == 0.0) continue;
                double app = A[p * k + p], aqq = A[q * k + q];
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* A <- J^T A J with J the rotation in the (p,q) plane */
                for (int r = 0; r < k; ++r) {
                    double arp = A[r * k + p], arq = A[r * k + q];
                    A[r * k + p] = c * arp - s * arq;
                    A[r * k + q] = s * arp + c * arq;
                }
                for (int r = 0; r < k; ++r) {
                    double apr = A[p * k + r], aqr = A[q * k + r];
                    A[p * k + r] = c * apr - s * aqr;
                    A[q * k + r] = s * apr + c * aqr;
                }
                /* Z <- Z J: columns of Z are the eigenvectors */
                for (int r = 0; r < k; ++r) {
                    double zrp = Z[r * k + p], zrq = Z[r * k + q];
                    Z[r * k + p] = c * zrp - s * zrq;
                    Z[r * k + q] = s * zrp + c * zrq;
                }
            }
    }
    /* sort ascending by eigenvalue (selection sort, k is small) */
    int* idx = (int*)malloc(sizeof(int) * k);
    for (int i = 0; i < k; ++i) idx[i] = i;
    for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j)
            if (A[idx[j] * k + idx[j]] < A[idx[i] * k + idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
    for (int i = 0; i < k; ++i) {
        theta[i] = A[idx[i] * k + idx[i]];
        z1[i] = Z[0 * k + idx[i]];
    }
    free(idx); free(A); free(Z);
    return 0;
}

double evo_gauss_quad(int k, const double* alpha, const double* beta, double vnorm2)
{
    double* theta = (double*)malloc(sizeof(double) * k);
    double* z1 = (double*)malloc(sizeof(double) * k);
    double s = 0.0;
    if (theta && z1 && evo_tridiag_eig(k, alpha, beta, theta, z1) == 0)
        for (int i = 0; i < k; ++i)
            if (theta[i] < 0.0) s += z1[i] * z1[i];   /* h(theta) = 1 iff theta < 0 */
    free(theta); free(z1);
    return vnorm2 * s;
}

/* Generalized averaged Gauss quadrature (Sec. 3.4, Eq. GA_Tk): the Gauss
 * formula of Eq. gauss_quad applied to the (2k-1) x (2k-1) tridiagonal with
 * diagonal (alpha_1..alpha_k, alpha_{k-1}..alpha_1) and off-diagonal
 * (beta_2..beta_k, beta_{k+1}, beta_{k-1}..beta_2).  beta[k] = beta_{k+1}. */
double evo_ga_quad(int k, const double* alpha, const double* beta, double vnorm2)
{
    if (k <= 1) return evo_gauss_quad(k, alpha, beta, vnorm2);
    const int kk = 2 * k - 1;
    double* a2 = (double*)malloc(sizeof(double) * kk);
    double* b2 = (double*)malloc(sizeof(double) * (kk + 1));
    double q = 0.0;
    if (a2 && b2) {
        /* diagonal: alpha_1 .. alpha_k, then alpha_{k-1} .. alpha_1 */
        for (int t = 0; t < k; ++t) a2[t] = alpha[t];
        for (int t = 0; t < k - 1; ++t) a2[k + t] = alpha[k - 2 - t];
        /* off-diagonal in the beta layout (b2[t] couples t-1 and t) */
        b2[0] = 0.0;
        for (int t = 1; t < k; ++t) b2[t] = beta[t];            /* beta_2 .. beta_k  */
        b2[k] = beta[k];                                         /* beta_{k+1}        */
        for (int t = 1; t < k - 1; ++t) b2[k + t] = beta[k - 1 - t]; /* beta_{k-1} .. beta_2 */
        b2[kk] = 0.0;
        q = evo_gauss_quad(kk, a2, b2, vnorm2);
    }
    free(a2); free(b2);
    return q;
}

/* ---------------------------------------------------------------- count */

int evo_count_rule(const evo_problem* P, const double* shifts, int S, int m,
                   const int64_t* probe_ids, int kmax, double tol, uint64_t seed,
                   double breakdown_rel, int nthreads, int rule, int min_steps,
                   double* quad, int* steps, double* L)
{
    const int64_t n = P->n;
    if (S < 1 || m < 1 || kmax < 1 || n < 1) return -1;
    if (kmax > n) kmax = (int)n;
    const int ncol = S * m;
    /* quad_hist[c*kmax + (i-1)]: quadrature of column c after i steps */
    double* quad_hist = (double*)calloc((size_t)ncol * kmax, sizeof(double));
    if (!quad_hist) return -2;
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    #pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int c = 0; c < ncol; ++c) {
        int s = c / m, j = c % m;
        uint64_t pid = probe_ids ? (uint64_t)probe_ids[j] : (uint64_t)j;
        double* v = (double*)malloc(sizeof(double) * n);
        double* alpha = (double*)malloc(sizeof(double) * kmax);
        double* beta = (double*)malloc(sizeof(double) * (kmax + 1));
        int kd = 0;
        if (!v || !alpha || !beta) { err = -2; free(v); free(alpha); free(beta); continue; }
        evo_probe_vector(seed, pid, n, v);
        double vn2 = dot(n, v, v);
        if (evo_lanczos(P, shifts[s], v, kmax, breakdown_rel, alpha, beta, NULL, &kd) != 0 || kd < 1) {
            err = -3;
        } else {
            for (int i = 1; i <= kmax; ++i) {
                if (tol <= 0.0 && i < kmax) continue;   /* only the last step is needed */
                int ki = i < kd ? i : kd;               /* after breakdown J stays J_kd */
                quad_hist[(size_t)c * kmax + (i - 1)] =
                    rule == 1 ? evo_ga_quad(ki, alpha, beta, vn2) : evo_gauss_quad(ki, alpha, beta, vn2);
            }
        }
        free(v); free(alpha); free(beta);
    }
    if (err) { free(quad_hist); return err; }
    for (int s = 0; s < S; ++s) {
        int ks = kmax;
        if (tol > 0.0) {
            /* stop at the first step i >= max(3, min_steps) where L changed by
             * at most tol over each of the last two steps */
            double prev = 0.0, prev2 = 0.0;
            for (int i = 1; i <= kmax; ++i) {
                double Li = 0.0;
                for (int j = 0; j < m; ++j) Li += quad_hist[(size_t)(s * m + j) * kmax + (i - 1)];
                Li /= m;
                if (i >= 3 && i >= min_steps && fabs(Li - prev) <= tol && fabs(prev - prev2) <= tol) {
                    ks = i;
                    break;
                }
                prev2 = prev;
                prev = Li;
            }
        }
        double Ls = 0.0;
        for (int j = 0; j < m; ++j) {
            quad[s * m + j] = quad_hist[(size_t)(s * m + j) * kmax + (ks - 1)];
            Ls += quad[s * m + j];
        }
        steps[s] = ks;
        L[s] = Ls / m;
    }
    free(quad_hist);
    return 0;
}

int evo_count(const evo_problem* P, const double* shifts, int S, int m,
              const int64_t* probe_ids, int kmax, double tol, uint64_t seed,
              double breakdown_rel, int nthreads,
              double* quad, int* steps, double* L)
{
    return evo_count_rule(P, shifts, S, m, probe_ids, kmax, tol, seed, breakdown_rel, nthreads, 0,
                          3, quad, steps, L);
}
