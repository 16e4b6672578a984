/*
 * Oracle: diagnostics of the ensemble (arXiv 2308.03972, Section 4.1 energy
 * spectrum, Section 4.3 RMSE). TEST INFRASTRUCTURE ONLY; see oracle.h.
 *
 * Readings of the paper taken here:
 *  - u-hat(k) = N^{-1} sum_xi u(xi) exp(-i k . xi), N = nx * ny cells, with
 *    k = 2 pi (kx / nx, ky / ny) over the full integer range of each axis;
 *  - E(k') = 1/2 |u-hat(k')|^2 summed over both velocity components;
 *  - the shell of integer wavenumber s holds the k' whose magnitude
 *    |k'| = sqrt(kx'^2 + ky'^2) (signed, minimum-image integers) lies in
 *    [s - 1/2, s + 1/2): the printed inequality |k'| - k <= 1/2 would count
 *    half-integer magnitudes twice;
 *  - the ensemble's spectrum is the mean over members of each member's E(k).
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

/* Signed integer wavenumber of index j on an axis of n points. */
static int signed_wavenumber(int j, int n) { return (2 * j > n) ? j - n : j; }

void orc_energy_spectrum(int nx, int ny, int k, const double *f, int nshells, double *E) {
    size_t cells = (size_t)nx * ny;
    double *rho = (double *)malloc(sizeof(double) * cells * k);
    double *u = (double *)malloc(sizeof(double) * cells * k);
    double *v = (double *)malloc(sizeof(double) * cells * k);
    orc_lbm_moments(nx, ny, k, f, rho, u, v);
    /* Twiddles exp(-2 pi i j / n) for j = 0..n-1 of each axis; the product
     * index is reduced modulo n before the table is read. */
    double *cxr = (double *)malloc(sizeof(double) * nx), *cxi = (double *)malloc(sizeof(double) * nx);
    double *cyr = (double *)malloc(sizeof(double) * ny), *cyi = (double *)malloc(sizeof(double) * ny);
    const double two_pi = 8.0 * atan(1.0);
    for (int j = 0; j < nx; ++j) {
        cxr[j] = cos(two_pi * j / nx);
        cxi[j] = -sin(two_pi * j / nx);
    }
    for (int j = 0; j < ny; ++j) {
        cyr[j] = cos(two_pi * j / ny);
        cyi[j] = -sin(two_pi * j / ny);
    }
    double *Em = (double *)calloc((size_t)k * nshells, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int m = 0; m < k; ++m) {
        /* Row transform then column transform of both components. */
        double *ar = (double *)malloc(sizeof(double) * cells * 2);
        double *ai = (double *)malloc(sizeof(double) * cells * 2);
        for (int c = 0; c < 2; ++c) {
            const double *fld = (c == 0) ? u : v;
            for (int y = 0; y < ny; ++y)
                for (int kx = 0; kx < nx; ++kx) {
                    double sr = 0.0, si = 0.0;
                    for (int x = 0; x < nx; ++x) {
                        int t = (int)(((long long)kx * x) % nx);
                        double val = fld[((size_t)y * nx + x) * k + m];
                        sr += val * cxr[t];
                        si += val * cxi[t];
                    }
                    ar[c * cells + (size_t)y * nx + kx] = sr;
                    ai[c * cells + (size_t)y * nx + kx] = si;
                }
        }
        for (int kx = 0; kx < nx; ++kx)
            for (int ky = 0; ky < ny; ++ky) {
                double e = 0.0;
                for (int c = 0; c < 2; ++c) {
                    double sr = 0.0, si = 0.0;
                    for (int y = 0; y < ny; ++y) {
                        int t = (int)(((long long)ky * y) % ny);
                        double pr = ar[c * cells + (size_t)y * nx + kx];
                        double pi = ai[c * cells + (size_t)y * nx + kx];
                        sr += pr * cyr[t] - pi * cyi[t];
                        si += pr * cyi[t] + pi * cyr[t];
                    }
                    sr /= (double)cells;
                    si /= (double)cells;
                    e += 0.5 * (sr * sr + si * si);
                }
                int wx = signed_wavenumber(kx, nx), wy = signed_wavenumber(ky, ny);
                double mag = sqrt((double)wx * wx + (double)wy * wy);
                int s = (int)floor(mag + 0.5);
                if (s < nshells) Em[(size_t)m * nshells + s] += e;
            }
        free(ar);
        free(ai);
    }
    for (int s = 0; s < nshells; ++s) {
        double acc = 0.0;
        for (int m = 0; m < k; ++m) acc += Em[(size_t)m * nshells + s];
        E[s] = acc / k;
    }
    free(Em);
    free(cxr);
    free(cxi);
    free(cyr);
    free(cyi);
    free(rho);
    free(u);
    free(v);
}
