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

// alpha[t*astride] = alpha_{t+1} (t < k), beta[t*astride] = beta_{t+1}
// (beta[0] unused); d, e, z: scratch of k entries each with stride sstride.
// Eigenvalues by the implicit symmetric QR iteration with Wilkinson shifts
// on the unreduced trailing block; the first components of the eigenvectors
// are carried along by applying every Givens rotation to the vector e_1
// (Golub & Welsch).  Returns -1 if it does not converge.
__device__ inline double tridiag_gauss_quadrature(const double* alpha, const double* beta,
                                                  int64_t astride, int k, double vnorm2,
                                                  double* dp, double* ep, double* zp,
                                                  int64_t sstride)
{
    const Strided d{dp, sstride}, e{ep, sstride}, z{zp, sstride};
    for (int t = 0; t < k; ++t) {
        d[t] = alpha[(int64_t)t * astride];
        e[t] = t + 1 < k ? beta[(int64_t)(t + 1) * astride] : 0.0;
        z[t] = t == 0 ? 1.0 : 0.0;
    }
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
        if (++iter > max_iter) return -1.0;
        int lo = hi - 1;
        while (lo > 0 && fabs(e[lo - 1]) > eps * (fabs(d[lo - 1]) + fabs(d[lo]))) --lo;
        // Wilkinson shift: eigenvalue of the trailing 2x2 closer to d[hi]
        const double dl = 0.5 * (d[hi - 1] - d[hi]);
        const double eh = e[hi - 1];
        const double den = dl + (dl >= 0.0 ? 1.0 : -1.0) * hypot(dl, eh);
        const double mu = d[hi] - eh * eh / den;
        // implicit QR step on [lo, hi]: chase the bulge down the band
        double xv = d[lo] - mu, yv = e[lo];
        double bulge = 0.0;
        for (int t = lo; t < hi; ++t) {
            const double rr = hypot(xv, yv);
            const double cs = rr == 0.0 ? 1.0 : xv / rr;
            const double sn = rr == 0.0 ? 0.0 : yv / rr;
            if (t > lo) e[t - 1] = rr;                    // (t, t-1) after the rotation
            const double a = d[t], b = e[t], dd = d[t + 1];
            d[t] = cs * cs * a + 2.0 * cs * sn * b + sn * sn * dd;
            d[t + 1] = sn * sn * a - 2.0 * cs * sn * b + cs * cs * dd;
            e[t] = cs * sn * (dd - a) + (cs * cs - sn * sn) * b;
            if (t + 1 < hi) {
                bulge = sn * e[t + 1];
                e[t + 1] = cs * e[t + 1];
            }
            const double z0 = z[t], z1 = z[t + 1];
            z[t] = cs * z0 + sn * z1;
            z[t + 1] = -sn * z0 + cs * z1;
            xv = e[t];
            yv = bulge;
        }
    }
    double s = 0.0;
    for (int t = 0; t < k; ++t)
        if (d[t] < 0.0) s += z[t] * z[t];                // h(theta) = 1 iff theta < 0
    return vnorm2 * s;
}

}  // namespace evc
