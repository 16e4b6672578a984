/*
 * CPU oracle for the LBM-LETKF forecast-analysis cycle (arXiv 2308.03972).
 *
 * TEST INFRASTRUCTURE ONLY. This library exists to check the CUDA path. It
 * shares no code, header, table or helper with the CUDA library, and only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Everything is IEEE binary64, compiled without floating-point contraction,
 * in plain loops that follow the paper's equations in the paper's order.
 *
 * Array layouts (all row-major, member index innermost):
 *   f      [9][ny][nx][k]   distribution functions f_alpha of every member
 *   force  [2][ny][nx]      large-scale acceleration F^i (x then y component)
 *   rho, u, v [ny][nx][k]   macroscopic moments
 *   Yf     [2*npts][k]      observed (u, v) of every member; row 2j is u at
 *                           observation point j, row 2j+1 is v there (with
 *                           density observed: [3*npts][k], rows u, v, rho)
 */
#ifndef LBM_LETKF_ORACLE_H
#define LBM_LETKF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* D2Q9 velocity set and weights (Section 2, discrete velocities and w_alpha). */
void orc_d2q9(int *cx, int *cy, double *w);

/* Second-order equilibrium (Section 2, f^eq) in lattice units c = 1. */
void orc_equilibrium(double rho, double ux, double uy, double *feq);

/* One lattice-BGK step with Smagorinsky eddy viscosity and forcing
 * (Section 2, lattice Boltzmann equation; Section 4.1, F = F^i - mu u):
 * collide every member at every cell, then push f*_alpha to xi + c_alpha
 * with periodic wrap. f_in and f_out must not alias. */
void orc_lbm_step(int nx, int ny, int k, const double *f_in, double *f_out,
                  const double *force, double tau0, double cs_smag, double mu);

/* rho = sum f, u = sum f c / rho (Section 2, moments). */
void orc_lbm_moments(int nx, int ny, int k, const double *f,
                     double *rho, double *u, double *v);

/* f = f^eq(rho, u, v) at every cell and member. */
void orc_set_equilibrium(int nx, int ny, int k, const double *rho,
                         const double *u, const double *v, double *f);

/* Observation operator H (Section 3, y = [u, v] at eta): Yf as above. */
void orc_observe(int nx, int ny, int k, const double *f, int npts,
                 const int *ix, const int *iy, double *Yf);

/* Observation operator with nvar = 2 (u, v) or 3 (u, v, rho) variables per
 * point (Section 3, y = macroscopic variables at eta; Section 4.3 observes
 * the density as well): row nvar*j + q of Yf [nvar*npts][k] is variable q
 * of point j. */
void orc_observe_vars(int nx, int ny, int k, const double *f, int npts,
                      const int *ix, const int *iy, int nvar, double *Yf);

/* Gaspari-Cohn localisation weight G(d) (Section 3.2.2). */
double orc_gaspari_cohn(double d);

/* Symmetric eigendecomposition A = Q diag(lam) Q^T by Householder
 * tridiagonalisation and implicit symmetric QR with Wilkinson shift
 * (Golub & Van Loan, Matrix Computations, Section 8.3). A is n x n row-major
 * and is not modified. lam ascending; Q columns are the eigenvectors.
 * Returns 0, or 1 if the QR iteration did not converge. */
int orc_sym_eig(int n, const double *A, double *lam, double *Q);

/* LETKF ensemble-space solution (Section 3.2, Eqs. for w-bar, P-tilde and
 * delta-W with R-localisation and multiplicative inflation):
 *   Pt   = [ (k-1)/beta I + dY^T diag(rloc) dY ]^{-1}
 *   wbar = Pt dY^T diag(rloc) d
 *   W    = [ (k-1) Pt ]^{1/2}   (symmetric square root)
 * dY is p x k (perturbations of the local observations), rloc the p
 * localised inverse error variances G/sigma^2, d the p innovations.
 * Outputs wbar[k] and W[k][k]. Returns 0 or 1 (eigensolver failure). */
int orc_letkf_transform(int k, int p, const double *dY, const double *rloc,
                        const double *d, double beta, double *wbar, double *W);

/* x^a_m = xbar + dX (wbar + W_m) for nrows state components of X[nrows][k]
 * in place (Section 3.2, analysis update). Returns 0 or 1. */
int orc_letkf_update(int nrows, int k, double *X, int p, const double *dY,
                     const double *rloc, const double *d, double beta);

/* Local observation set of grid point (x, y): observation scalars whose
 * point lies at periodic minimum-image distance r with r / d_cut < 2 and
 * G(r / d_cut) > 0. Writes up to 2*npts indices (into the Yf rows) and the
 * matching rloc = G / sigma^2; returns the count. */
int orc_local_obs(int nx, int ny, int x, int y, int npts, const int *ix,
                  const int *iy, double sigma_u, double sigma_v, double d_cut,
                  int *idx, double *rloc);

/* orc_local_obs for nvar variables per point with error sigma[q] for
 * variable q; indices nvar*j + q. */
int orc_local_obs_vars(int nx, int ny, int x, int y, int npts, const int *ix,
                       const int *iy, int nvar, const double *sigma, double d_cut,
                       int *idx, double *rloc);

/* Full LETKF analysis of the nine f_alpha at grid points (Section 3.2):
 * H applied to the forecast ensemble, ybar, dY and d = y^o - ybar, then the
 * local transform and update at each selected point, in place on f.
 * points: npoints cell indices y*nx + x, or NULL with npoints < 0 for all.
 * Returns 0, or 1 if any eigensolve failed. */
int orc_letkf_analyze(int nx, int ny, int k, double *f, int npts,
                      const int *ix, const int *iy, const double *yo_u,
                      const double *yo_v, double sigma_u, double sigma_v,
                      double d_cut, double beta, int npoints,
                      const int *points);

/* orc_letkf_analyze with nvar variables per observation point (see
 * orc_observe_vars): yo [npts][nvar], sigma [nvar]. */
int orc_letkf_analyze_vars(int nx, int ny, int k, double *f, int npts,
                           const int *ix, const int *iy, int nvar, const double *yo,
                           const double *sigma, double d_cut, double beta, int npoints,
                           const int *points);

/* Nudging (Section 3.1): every member is relaxed toward the equilibrium of
 * the observed macroscopic field, f_a <- f_a + gamma (f^eq_a(rho^, u^, v^) - f_a).
 * Observations sit on the uniform periodic lattice (i nx/nox, j ny/noy),
 * arrays [noy][nox]; rho^, u^, v^ at a grid point are their bilinear
 * interpolation (linear interpolation of the sparse data). nx must
 * be a multiple of nox and ny of noy. In place on f. */
void orc_nudge(int nx, int ny, int k, double *f, int nox, int noy,
               const double *rho_o, const double *u_o, const double *v_o,
               double gamma);

/* Energy spectrum of the ensemble (Section 4.1): for each member the 2D
 * discrete Fourier transform u-hat(k') = N^{-1} sum u e^{-i k'.xi} of both
 * velocity components, E(k') = |u-hat|^2 / 2 binned into integer shells
 * s = floor(|k'| + 1/2), then the mean over members. E[nshells]; shells at
 * or beyond nshells are dropped. */
void orc_energy_spectrum(int nx, int ny, int k, const double *f, int nshells, double *E);

/* Number of OpenMP threads the oracle will use (1 without OpenMP). */
int orc_num_threads(void);
/* Threads of the following OpenMP regions (timing of the CPU baseline). */
void orc_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
