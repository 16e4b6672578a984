/*
 * Oracle: LETKF analysis of the nine distribution functions
 * (arXiv 2308.03972, Section 3.2). TEST INFRASTRUCTURE ONLY; see oracle.h.
 *
 * Readings of the paper taken here:
 *  - the innovation enters with a plus sign (the generic linear update in
 *    Section 3 prints a minus; the LETKF equations themselves are
 *    sign-correct and are what is implemented);
 *  - ybar is the mean of H(x_m) over members;
 *  - R is diagonal with sigma_u^2 for u and sigma_v^2 for v observations
 *    (sigma_rho^2 for rho where density is observed as well);
 *    R-localisation divides each variance by the Gaspari-Cohn weight
 *    G(r / d_cut), r the periodic minimum-image distance from the grid
 *    point to the observation point, and drops observations with
 *    r / d_cut >= 2 or G <= 0 (the support of G);
 *  - inflation multiplies the background covariance: (k-1)/beta in P-tilde;
 *  - [(k-1) P-tilde]^{1/2} is the symmetric square root.
 * The transform is formed in ensemble space exactly as printed: the k x k
 * matrix, its eigendecomposition, its inverse and its inverse square root.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

/* Gaspari-Cohn fifth-order piecewise rational function. */
double orc_gaspari_cohn(double d) {
    if (d < 0.0) d = -d;
    if (d <= 1.0) {
        return -0.25 * pow(d, 5) + 0.5 * pow(d, 4) + 0.625 * pow(d, 3) - (5.0 / 3.0) * d * d + 1.0;
    }
    if (d < 2.0) {
        return (1.0 / 12.0) * pow(d, 5) - 0.5 * pow(d, 4) + 0.625 * pow(d, 3) + (5.0 / 3.0) * d * d
               - 5.0 * d + 4.0 - (2.0 / 3.0) / d;
    }
    return 0.0;
}

int orc_letkf_transform(int k, int p, const double *dY, const double *rloc,
                        const double *d, double beta, double *wbar, double *W) {
    size_t kk = (size_t)k * k;
    double *C = (double *)malloc(sizeof(double) * kk);
    double *Q = (double *)malloc(sizeof(double) * kk);
    double *Pt = (double *)malloc(sizeof(double) * kk);
    double *lam = (double *)malloc(sizeof(double) * k);
    double *b = (double *)malloc(sizeof(double) * k);
    /* C = (k-1)/beta I + dY^T R_loc^{-1} dY ; b = dY^T R_loc^{-1} d. */
    for (int i = 0; i < k; ++i) {
        for (int j = 0; j < k; ++j) {
            double s = 0.0;
            for (int o = 0; o < p; ++o) s += dY[(size_t)o * k + i] * rloc[o] * dY[(size_t)o * k + j];
            C[(size_t)i * k + j] = s + ((i == j) ? (k - 1) / beta : 0.0);
        }
        double s = 0.0;
        for (int o = 0; o < p; ++o) s += dY[(size_t)o * k + i] * rloc[o] * d[o];
        b[i] = s;
    }
    int status = orc_sym_eig(k, C, lam, Q);
    /* P-tilde = Q diag(1/lam) Q^T ; W = Q diag(sqrt((k-1)/lam)) Q^T. */
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            double sp = 0.0, sw = 0.0;
            for (int l = 0; l < k; ++l) {
                double qq = Q[(size_t)i * k + l] * Q[(size_t)j * k + l];
                sp += qq / lam[l];
                sw += qq * sqrt((k - 1) / lam[l]);
            }
            Pt[(size_t)i * k + j] = sp;
            W[(size_t)i * k + j] = sw;
        }
    /* wbar = P-tilde b. */
    for (int i = 0; i < k; ++i) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s += Pt[(size_t)i * k + j] * b[j];
        wbar[i] = s;
    }
    free(C);
    free(Q);
    free(Pt);
    free(lam);
    free(b);
    return status;
}

int orc_letkf_update(int nrows, int k, double *X, int p, const double *dY,
                     const double *rloc, const double *d, double beta) {
    double *wbar = (double *)malloc(sizeof(double) * k);
    double *W = (double *)malloc(sizeof(double) * k * k);
    double *dx = (double *)malloc(sizeof(double) * k);
    int status = orc_letkf_transform(k, p, dY, rloc, d, beta, wbar, W);
    for (int r = 0; r < nrows; ++r) {
        double *row = X + (size_t)r * k;
        double mean = 0.0;
        for (int m = 0; m < k; ++m) mean += row[m];
        mean /= k;
        for (int m = 0; m < k; ++m) dx[m] = row[m] - mean;
        /* x^a_m = xbar + sum_j dx_j (wbar_j + W_jm). */
        for (int m = 0; m < k; ++m) {
            double s = 0.0;
            for (int j = 0; j < k; ++j) s += dx[j] * (wbar[j] + W[(size_t)j * k + m]);
            row[m] = mean + s;
        }
    }
    free(wbar);
    free(W);
    free(dx);
    return status;
}

static int min_image(int dx, int n) {
    if (dx > n / 2) dx -= n;
    if (dx < -(n / 2)) dx += n;
    return dx;
}

int orc_local_obs_vars(int nx, int ny, int x, int y, int npts, const int *ix,
                       const int *iy, int nvar, const double *sigma, double d_cut,
                       int *idx, double *rloc) {
    int p = 0;
    for (int j = 0; j < npts; ++j) {
        int dx = min_image(ix[j] - x, nx);
        int dy = min_image(iy[j] - y, ny);
        double r = sqrt((double)dx * dx + (double)dy * dy);
        double dist = r / d_cut;
        if (!(dist < 2.0)) continue;
        double g = orc_gaspari_cohn(dist);
        if (!(g > 0.0)) continue;
        for (int q = 0; q < nvar; ++q) {
            idx[p] = nvar * j + q;
            rloc[p] = g / (sigma[q] * sigma[q]);
            ++p;
        }
    }
    return p;
}

int orc_local_obs(int nx, int ny, int x, int y, int npts, const int *ix,
                  const int *iy, double sigma_u, double sigma_v, double d_cut,
                  int *idx, double *rloc) {
    const double sigma[2] = {sigma_u, sigma_v};
    return orc_local_obs_vars(nx, ny, x, y, npts, ix, iy, 2, sigma, d_cut, idx, rloc);
}

int orc_letkf_analyze(int nx, int ny, int k, double *f, int npts,
                      const int *ix, const int *iy, const double *yo_u,
                      const double *yo_v, double sigma_u, double sigma_v,
                      double d_cut, double beta, int npoints,
                      const int *points) {
    double *yo = (double *)malloc(sizeof(double) * 2 * (npts > 0 ? npts : 1));
    for (int j = 0; j < npts; ++j) {
        yo[2 * j] = yo_u[j];
        yo[2 * j + 1] = yo_v[j];
    }
    const double sigma[2] = {sigma_u, sigma_v};
    int status = orc_letkf_analyze_vars(nx, ny, k, f, npts, ix, iy, 2, yo, sigma, d_cut, beta,
                                        npoints, points);
    free(yo);
    return status;
}

int orc_letkf_analyze_vars(int nx, int ny, int k, double *f, int npts,
                           const int *ix, const int *iy, int nvar, const double *yo,
                           const double *sigma, double d_cut, double beta, int npoints,
                           const int *points) {
    int nobs = nvar * npts;
    double *Yf = (double *)malloc(sizeof(double) * nobs * k);
    double *dYall = (double *)malloc(sizeof(double) * nobs * k);
    double *dall = (double *)malloc(sizeof(double) * nobs);
    /* y_m^f = H x_m^f; ybar = mean over members; dY = Y - ybar; d = y^o - ybar. */
    orc_observe_vars(nx, ny, k, f, npts, ix, iy, nvar, Yf);
    for (int o = 0; o < nobs; ++o) {
        double mean = 0.0;
        for (int m = 0; m < k; ++m) mean += Yf[(size_t)o * k + m];
        mean /= k;
        for (int m = 0; m < k; ++m) dYall[(size_t)o * k + m] = Yf[(size_t)o * k + m] - mean;
        dall[o] = yo[o] - mean;
    }
    int total = (npoints < 0) ? nx * ny : npoints;
    int status = 0;
    size_t plane = (size_t)nx * ny;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) reduction(| : status)
#endif
    for (int t = 0; t < total; ++t) {
        int cell = (npoints < 0) ? t : points[t];
        int x = cell % nx, y = cell / nx;
        int *idx = (int *)malloc(sizeof(int) * nobs);
        double *rloc = (double *)malloc(sizeof(double) * nobs);
        double *dY = (double *)malloc(sizeof(double) * nobs * k);
        double *d = (double *)malloc(sizeof(double) * nobs);
        double *X = (double *)malloc(sizeof(double) * 9 * k);
        int p = orc_local_obs_vars(nx, ny, x, y, npts, ix, iy, nvar, sigma, d_cut, idx, rloc);
        for (int i = 0; i < p; ++i) {
            memcpy(dY + (size_t)i * k, dYall + (size_t)idx[i] * k, sizeof(double) * k);
            d[i] = dall[idx[i]];
        }
        for (int a = 0; a < 9; ++a)
            memcpy(X + (size_t)a * k, f + ((size_t)a * plane + cell) * k, sizeof(double) * k);
        status |= orc_letkf_update(9, k, X, p, dY, rloc, d, beta);
        for (int a = 0; a < 9; ++a)
            memcpy(f + ((size_t)a * plane + cell) * k, X + (size_t)a * k, sizeof(double) * k);
        free(idx);
        free(rloc);
        free(dY);
        free(d);
        free(X);
    }
    free(Yf);
    free(dYall);
    free(dall);
    return status;
}
