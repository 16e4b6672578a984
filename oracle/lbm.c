/*
 * Oracle: D2Q9 lattice-BGK LES step (arXiv 2308.03972, Section 2 and 4.1).
 * TEST INFRASTRUCTURE ONLY; see oracle.h.
 *
 * Readings of the paper taken here:
 *  - lattice units: dx = dt = c = 1, so c_s^2 = 1/3;
 *  - diagonal order alpha = 5..8 is (+,+), (-,-), (+,-), (-,+), i.e. the
 *    same "plus then minus" pairing the paper uses for alpha = 1,2 and 3,4;
 *  - |S| is evaluated from the local non-equilibrium momentum flux
 *    Pi = sum c c (f - f^eq) (unforced f^eq), which together with
 *    nu + nu_SGS = (tau - 1/2)/3 and nu_SGS = (C_s Delta)^2 |S| gives the
 *    quadratic tau^2 - tau0 tau - 9 C_s^2 Q / (2 rho) = 0, Q = sqrt(2 Pi:Pi);
 *  - u in f^eq and in the friction is sum f c / rho (no force shift);
 *  - the stored state is the pre-collision f; streaming pushes f*_alpha
 *    from xi to xi + c_alpha with periodic wrap.
 */
#include <math.h>
#include <stddef.h>
#include "oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

static const int CX[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
static const int CY[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
static const double W9[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

void orc_d2q9(int *cx, int *cy, double *w) {
    for (int a = 0; a < 9; ++a) {
        cx[a] = CX[a];
        cy[a] = CY[a];
        w[a] = W9[a];
    }
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* f^eq_alpha = rho w_alpha (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u), c = 1. */
void orc_equilibrium(double rho, double ux, double uy, double *feq) {
    double uu = ux * ux + uy * uy;
    for (int a = 0; a < 9; ++a) {
        double cu = CX[a] * ux + CY[a] * uy;
        feq[a] = rho * W9[a] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

static size_t fidx(int a, int y, int x, int m, int nx, int ny, int k) {
    return (((size_t)a * ny + y) * nx + x) * k + m;
}

/* Collision of one cell of one member: f (pre-collision) -> fs (post). */
static void collide(const double *f, double Fix, double Fiy, double tau0,
                    double cs_smag, double mu, double *fs) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < 9; ++a) {
        rho += f[a];
        jx += f[a] * CX[a];
        jy += f[a] * CY[a];
    }
    double ux = jx / rho, uy = jy / rho;
    double feq[9];
    orc_equilibrium(rho, ux, uy, feq);
    /* Non-equilibrium momentum flux Pi_ij = sum_a c_ai c_aj (f_a - f^eq_a). */
    double pxx = 0.0, pxy = 0.0, pyy = 0.0;
    for (int a = 0; a < 9; ++a) {
        double fneq = f[a] - feq[a];
        pxx += CX[a] * CX[a] * fneq;
        pxy += CX[a] * CY[a] * fneq;
        pyy += CY[a] * CY[a] * fneq;
    }
    double Q = sqrt(2.0 * (pxx * pxx + 2.0 * pxy * pxy + pyy * pyy));
    /* Filter width Delta = dx = 1. */
    double tau = 0.5 * (tau0 + sqrt(tau0 * tau0 + 18.0 * cs_smag * cs_smag * Q / rho));
    /* Acceleration F = F^i - mu u; forcing term F_a = 3 w_a rho (F . c_a). */
    double Fx = Fix - mu * ux, Fy = Fiy - mu * uy;
    for (int a = 0; a < 9; ++a) {
        double Fa = 3.0 * W9[a] * rho * (Fx * CX[a] + Fy * CY[a]);
        fs[a] = f[a] - (f[a] - feq[a]) / tau + Fa;
    }
}

void orc_lbm_step(int nx, int ny, int k, const double *f_in, double *f_out,
                  const double *force, double tau0, double cs_smag, double mu) {
    size_t plane = (size_t)nx * ny;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double Fix = force[(size_t)y * nx + x];
            double Fiy = force[plane + (size_t)y * nx + x];
            for (int m = 0; m < k; ++m) {
                double f[9], fs[9];
                for (int a = 0; a < 9; ++a) f[a] = f_in[fidx(a, y, x, m, nx, ny, k)];
                collide(f, Fix, Fiy, tau0, cs_smag, mu, fs);
                for (int a = 0; a < 9; ++a) {
                    int xd = (x + CX[a] + nx) % nx;
                    int yd = (y + CY[a] + ny) % ny;
                    f_out[fidx(a, yd, xd, m, nx, ny, k)] = fs[a];
                }
            }
        }
    }
}

void orc_lbm_moments(int nx, int ny, int k, const double *f, double *rho,
                     double *u, double *v) {
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            for (int m = 0; m < k; ++m) {
                double r = 0.0, jx = 0.0, jy = 0.0;
                for (int a = 0; a < 9; ++a) {
                    double fa = f[fidx(a, y, x, m, nx, ny, k)];
                    r += fa;
                    jx += fa * CX[a];
                    jy += fa * CY[a];
                }
                size_t c = ((size_t)y * nx + x) * k + m;
                rho[c] = r;
                u[c] = jx / r;
                v[c] = jy / r;
            }
}

void orc_set_equilibrium(int nx, int ny, int k, const double *rho,
                         const double *u, const double *v, double *f) {
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            for (int m = 0; m < k; ++m) {
                size_t c = ((size_t)y * nx + x) * k + m;
                double feq[9];
                orc_equilibrium(rho[c], u[c], v[c], feq);
                for (int a = 0; a < 9; ++a) f[fidx(a, y, x, m, nx, ny, k)] = feq[a];
            }
}

void orc_observe_vars(int nx, int ny, int k, const double *f, int npts,
                      const int *ix, const int *iy, int nvar, double *Yf) {
    for (int j = 0; j < npts; ++j)
        for (int m = 0; m < k; ++m) {
            double r = 0.0, jx = 0.0, jy = 0.0;
            for (int a = 0; a < 9; ++a) {
                double fa = f[fidx(a, iy[j], ix[j], m, nx, ny, k)];
                r += fa;
                jx += fa * CX[a];
                jy += fa * CY[a];
            }
            Yf[(size_t)(nvar * j) * k + m] = jx / r;
            Yf[(size_t)(nvar * j + 1) * k + m] = jy / r;
            if (nvar == 3) Yf[(size_t)(nvar * j + 2) * k + m] = r;
        }
}

void orc_observe(int nx, int ny, int k, const double *f, int npts,
                 const int *ix, const int *iy, double *Yf) {
    orc_observe_vars(nx, ny, k, f, npts, ix, iy, 2, Yf);
}

/* Bilinear interpolation of a periodic field on the observation lattice. */
static double interp_obs(const double *g, int nox, int noy, int px, int py, int x, int y) {
    int i0 = x / px, j0 = y / py;
    double tx = (double)(x - i0 * px) / px;
    double ty = (double)(y - j0 * py) / py;
    int i1 = (i0 + 1) % nox, j1 = (j0 + 1) % noy;
    return (1.0 - tx) * (1.0 - ty) * g[(size_t)j0 * nox + i0] + tx * (1.0 - ty) * g[(size_t)j0 * nox + i1] +
           (1.0 - tx) * ty * g[(size_t)j1 * nox + i0] + tx * ty * g[(size_t)j1 * nox + i1];
}

void orc_nudge(int nx, int ny, int k, double *f, int nox, int noy,
               const double *rho_o, const double *u_o, const double *v_o,
               double gamma) {
    int px = nx / nox, py = ny / noy;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double feq[9];
            orc_equilibrium(interp_obs(rho_o, nox, noy, px, py, x, y),
                            interp_obs(u_o, nox, noy, px, py, x, y),
                            interp_obs(v_o, nox, noy, px, py, x, y), feq);
            for (int m = 0; m < k; ++m)
                for (int a = 0; a < 9; ++a) {
                    size_t i = fidx(a, y, x, m, nx, ny, k);
                    f[i] = f[i] + gamma * (feq[a] - f[i]);
                }
        }
}
