// evc_tridiag.cuh -- Gauss quadrature of a symmetric tridiagonal matrix
// (Sec. 3, Eq. gauss_quad): ||v||^2 sum_{theta_i < 0} z_i(1)^2 over the
// eigenpairs (theta_i, z_i) of J_k.  Shared by the estimator's finish kernel
// and the allocation-free quadrature entry point.
#pragma once

#include <cstdint>

namespace evc {

struct Strided {
    double* p;
    int64_t s;
    __device__ double& operator[](int t) const { return p[(int64_t)t * s]; }
};

// Eigen-decomposition of a tridiagonal already in scratch: d[0..k) diagonal,
// e[0..k-1) off-diagonal (e[t] couples t and t+1), z scratch of k entries,
// all with stride sstride.  Eigenvalues by the implicit symmetric QR
// iteration with Wilkinson shifts on the unreduced trailing block; the first
// components of the eigenvectors are carried along by applying every Givens
// rotation to the vector e_1 (Golub & Welsch).  On return d holds the
// eigenvalues theta_t and z their first components z_t(1); false if the
// iteration did not converge.
__device__ inline bool tridiag_eig_inplace(double* dp, double* ep, double* zp, int64_t sstride,
                                           int k)
{
    const Strided d{dp, sstride}, e{ep, sstride}, z{zp, sstride};
    for (int t = 0; t < k; ++t) z[t] = t == 0 ? 1.0 : 0.0;
    if (k > 0) e[k - 1] = 0.0;
    const double eps = 2.220446049250313e-16;
    int hi = k - 1;
    int iter = 0;
    const int max_iter = 40 * k + 40;
    while (hi > 0) {
        if (fabs(e[hi - 1]) <= eps * (fabs(d[hi - 1]) + fabs(d[hi]))) {
            e[hi - 1] = 0.0;
            --hi;
            continue;
        }
        if (++iter > max_iter) return false;
        int lo = hi - 1;
        while (lo > 0 && fabs(e[lo - 1]) > eps * (fabs(d[lo - 1]) + fabs(d[lo]))) --lo;
        // Wilkinson shift: eigenvalue of the trailing 2x2 closer to d[hi]
        const double dl = 0.5 * (d[hi - 1] - d[hi]);
        const double eh = e[hi - 1];
        const double den = dl + (dl >= 0.0 ? 1.0 : -1.0) * sqrt(dl * dl + eh * eh);
        const double mu = d[hi] - eh * eh / den;
        // implicit QR step on [lo, hi]: chase the bulge down the band.  The
        // entries one rotation hands to the next (d_t, e_t, z_t, the bulge)
        // stay in registers; only the untouched d_{t+1}, e_{t+1}, z_{t+1} are
        // loaded, off the dependency chain, and the chain's last values are
        // stored once after the sweep.  The eigensolve is a chain of dependent
        // FP64 operations, so its latency is the cost.
        double a = d[lo], b = e[lo], zt = z[lo];
        double xv = a - mu, yv = b;
        for (int t = lo; t < hi; ++t) {
            const double dd = d[t + 1], zn = z[t + 1];
            const double en = t + 1 < hi ? e[t + 1] : 0.0;
            // Lanczos coefficients are O(||C||): no scaling against overflow needed
            const double s2 = xv * xv + yv * yv;
            double cs = 1.0, sn = 0.0, rr = 0.0;
            if (s2 > 0.0) {
                const double inv = rsqrt(s2);
                cs = xv * inv;
                sn = yv * inv;
                rr = s2 * inv;
            }
            if (t > lo) e[t - 1] = rr;                    // (t, t-1) after the rotation
            d[t] = cs * cs * a + 2.0 * cs * sn * b + sn * sn * dd;
            const double dn = sn * sn * a - 2.0 * cs * sn * b + cs * cs * dd;
            xv = cs * sn * (dd - a) + (cs * cs - sn * sn) * b;   // new e_t
            yv = sn * en;                                        // bulge at (t+2, t)
            z[t] = cs * zt + sn * zn;
            zt = -sn * zt + cs * zn;
            a = dn;
            b = cs * en;                                         // new e_{t+1}
        }
        d[hi] = a;
        e[hi - 1] = xv;
        z[hi] = zt;
    }
    return true;
}

// Gauss quadrature of h(. - sigma) from a decomposed tridiagonal:
// vnorm2 * sum_{theta_t < sigma} z_t(1)^2 (h(x) = 1 iff x < 0, Eq. h).
__device__ inline double quadrature_below(const double* dp, const double* zp, int64_t sstride,
                                          int k, double vnorm2, double sigma)
{
    double s = 0.0;
    for (int t = 0; t < k; ++t) {
        const double th = dp[(int64_t)t * sstride], z = zp[(int64_t)t * sstride];
        if (th < sigma) s += z * z;
    }
    return vnorm2 * s;
}

// Quadrature from a tridiagonal already in scratch (see tridiag_eig_inplace):
// vnorm2 * sum_{theta<0} z(1)^2, or -1 if the iteration does not converge.
__device__ inline double tridiag_quadrature_inplace(double* dp, double* ep, double* zp,
                                                   int64_t sstride, int k, double vnorm2)
{
    if (!tridiag_eig_inplace(dp, ep, zp, sstride, k)) return -1.0;
    return quadrature_below(dp, zp, sstride, k, vnorm2, 0.0);
}

// Fill scratch with J_k (Gauss) or the extended J~_{2k-1} (GA); returns the
// order of the filled matrix.  Layouts as in the two quadratures below.
__device__ inline int tridiag_fill(const double* alpha, const double* beta, int64_t astride, int k,
                                   bool ga, double* dp, double* ep, int64_t sstride)
{
    if (!ga || k <= 1) {
        for (int t = 0; t < k; ++t) {
            dp[(int64_t)t * sstride] = alpha[(int64_t)t * astride];
            ep[(int64_t)t * sstride] = t + 1 < k ? beta[(int64_t)(t + 1) * astride] : 0.0;
        }
        return k;
    }
    const int kk = 2 * k - 1;
    for (int t = 0; t < kk; ++t) {
        const int a = t < k ? t : 2 * k - 2 - t;
        dp[(int64_t)t * sstride] = alpha[(int64_t)a * astride];
        double off = 0.0;
        if (t < k - 1) off = beta[(int64_t)(t + 1) * astride];
        else if (t == k - 1) off = beta[(int64_t)k * astride];
        else if (t < kk - 1) off = beta[(int64_t)(2 * k - 2 - t) * astride];
        ep[(int64_t)t * sstride] = off;
    }
    return kk;
}

// Gauss quadrature of J_k (Sec. 3, Eq. gauss_quad): alpha[t*astride] =
// alpha_{t+1} (t < k), beta[t*astride] = beta_{t+1} (beta[0] unused); d, e,
// z: scratch of k entries each with stride sstride.
__device__ inline double tridiag_gauss_quadrature(const double* alpha, const double* beta,
                                                  int64_t astride, int k, double vnorm2,
                                                  double* dp, double* ep, double* zp,
                                                  int64_t sstride)
{
    for (int t = 0; t < k; ++t) {
        dp[(int64_t)t * sstride] = alpha[(int64_t)t * astride];
        ep[(int64_t)t * sstride] = t + 1 < k ? beta[(int64_t)(t + 1) * astride] : 0.0;
    }
    return tridiag_quadrature_inplace(dp, ep, zp, sstride, k, vnorm2);
}

// Generalized averaged Gauss quadrature (Sec. 3.4, Eq. GA_Tk): the same rule
// on the (2k-1) x (2k-1) tridiagonal with diagonal (alpha_1..alpha_k,
// alpha_{k-1}..alpha_1) and off-diagonal (beta_2..beta_k, beta_{k+1},
// beta_{k-1}..beta_2).  Needs beta_{k+1} = beta[k*astride]; scratch of 2k-1
// entries.  For k = 1 it is the Gauss rule.
__device__ inline double tridiag_ga_quadrature(const double* alpha, const double* beta,
                                               int64_t astride, int k, double vnorm2,
                                               double* dp, double* ep, double* zp,
                                               int64_t sstride)
{
    const int kk = 2 * k - 1;
    for (int t = 0; t < kk; ++t) {
        const int a = t < k ? t : 2 * k - 2 - t;               // mirrored alpha index
        dp[(int64_t)t * sstride] = alpha[(int64_t)a * astride];
        double off = 0.0;
        if (t < k - 1) off = beta[(int64_t)(t + 1) * astride];            // beta_{t+2}
        else if (t == k - 1) off = kk > 1 ? beta[(int64_t)k * astride] : 0.0;   // beta_{k+1}
        else if (t < kk - 1) off = beta[(int64_t)(2 * k - 2 - t) * astride];   // mirrored
        ep[(int64_t)t * sstride] = off;
    }
    return tridiag_quadrature_inplace(dp, ep, zp, sstride, kk, vnorm2);
}

}  // namespace evc
