/*
 * lbm_letkf.h -- C ABI of the GB300 (sm_103a) LBM-LETKF library.
 *
 * The library runs the forecast-analysis cycle of "Continuous data
 * assimilation of large eddy simulation by lattice Boltzmann method and
 * local ensemble transform Kalman filter" (arXiv 2308.03972):
 *   - an ensemble of D2Q9 lattice-BGK LES members (Section 2) advanced
 *     together by a fused collide-and-push kernel;
 *   - the LETKF analysis (Section 3.2) applied to the nine distribution
 *     functions at every grid point, with Gaspari-Cohn R-localisation and
 *     multiplicative covariance inflation.
 *
 * Units: lattice units (dx = dt = lattice speed = 1, c_s^2 = 1/3).
 *
 * Layouts (row-major, member index innermost, all FP64 at this boundary):
 *   f      [9][ny][nx][members]  distribution functions; alpha = 0 rest,
 *                                1 (+x), 2 (-x), 3 (+y), 4 (-y),
 *                                5 (+x,+y), 6 (-x,-y), 7 (+x,-y), 8 (-x,+y)
 *   force  [2][ny][nx]           large-scale acceleration F^i (x, then y)
 *   rho, u, v [ny][nx][members]  macroscopic moments
 * The state held between calls is the pre-collision f (the paper's
 * f_alpha(xi, t)); a step collides it and pushes f*_alpha to xi + c_alpha
 * with periodic wrap.
 *
 * Ownership: the context owns every device buffer it allocates. Pointers
 * passed in are borrowed for the duration of the call only. Pointer kinds:
 * LBM_PTR_HOST (ordinary host memory) or LBM_PTR_DEVICE (CUDA device memory
 * of the current device).
 *
 * Streams and errors: all device work is queued on the stream given in the
 * config (NULL = the legacy default stream). Calls return an lbm_status; no
 * C++ exception crosses this boundary. Invalid arguments are reported at
 * once (LBM_EINVAL). Conditions found on the device (non-finite or
 * supersonic state, eigensolver without convergence, local problem larger
 * than the kernel supports) are recorded in a device flag word and reported
 * by the next call that synchronises (lbm_sync, lbm_moments and lbm_get_f
 * with host pointers). lbm_last_error gives a message for the last failure.
 *
 * Threading: a context may be used by one host thread at a time.
 */
#ifndef LBM_LETKF_H
#define LBM_LETKF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,    /* bad argument, or local problem too large (see letkf_analyze) */
    LBM_ENOMEM = 2,    /* device allocation failed */
    LBM_ECUDA = 3,     /* CUDA runtime error (launch or copy) */
    LBM_EDIVERGED = 4, /* non-finite density/velocity or |u| > 0.5 seen */
    LBM_ENOCONV = 5    /* eigensolver hit its sweep cap at some point */
} lbm_status;

typedef enum {
    LBM_FP64 = 0,  /* everything in binary64 */
    LBM_MIXED = 1  /* f stored and collided in binary32 as f - w_alpha;
                      LETKF eigensolve in binary64, products in binary32 */
} lbm_precision;

typedef enum { LBM_PTR_HOST = 0, LBM_PTR_DEVICE = 1 } lbm_ptr_kind;

typedef struct {
    int nx, ny;      /* periodic lattice, nx, ny >= 1 */
    int members;     /* ensemble size k >= 1 (k >= 2 for letkf_analyze) */
    double tau0;     /* molecular relaxation time, nu = (tau0 - 1/2)/3; > 0.5 */
    double cs_smag;  /* Smagorinsky constant C_s (paper: 0.2), >= 0 */
    double mu;       /* linear friction coefficient, F^mu = -mu u, >= 0 */
    int precision;   /* lbm_precision */
    void *stream;    /* cudaStream_t to queue work on; NULL = default stream */
} lbm_config;

/* Observation window of a variational misfit (used by lbm_misfit and
 * lbm_misfit_gradient): observations of (u, v) at npts points after every
 * obs_every steps of an nsteps forecast, i.e. at t = obs_every,
 * 2 obs_every, ..., nt obs_every with nt = nsteps / obs_every (integer
 * division). All pointers are host arrays read during the call.
 *   ix, iy      [npts] lattice coordinates (0 <= ix < nx, 0 <= iy < ny)
 *   yo_u, yo_v  [nt][npts] observed velocities, time-major
 *   sigma_u, sigma_v  observation error standard deviations (> 0)
 *   checkpoint_every  states kept by the gradient's forward pass: every
 *               checkpoint_every steps (>= 1); the backward pass recomputes
 *               the states in between one segment at a time. */
typedef struct {
    int nsteps;
    int obs_every;
    int checkpoint_every;
    int npts;
    const int *ix, *iy;
    const double *yo_u, *yo_v;
    double sigma_u, sigma_v;
} lbm_window;

/* Create a context: allocate the double-buffered ensemble state and copy the
 * initial f0 and the forcing field (Section 2; forcing Section 4.1).
 * f0 may be NULL (state set to the rest equilibrium rho = 1, u = 0);
 * force may be NULL (no large-scale forcing). *out receives the context or
 * NULL on failure. */
int lbm_init(const lbm_config *cfg, const double *f0, const double *force,
             int ptr_kind, lbm_ctx **out);

/* Set every member to the equilibrium f^eq(rho, u, v) (Section 2, f^eq).
 * rho may be NULL (rho = 1). Arrays [ny][nx][members]. */
int lbm_set_equilibrium(lbm_ctx *ctx, const double *rho, const double *u,
                        const double *v, int ptr_kind);

/* Advance all members nsteps lattice steps (Section 2, lattice Boltzmann
 * equation with Smagorinsky eddy viscosity and F = F^i - mu u). Asynchronous
 * on the context stream. nsteps >= 0. */
int lbm_forecast(lbm_ctx *ctx, int nsteps);

/* Macroscopic moments rho = sum f, u = sum f c / rho (Section 2). Any of the
 * outputs may be NULL. With LBM_PTR_HOST the call synchronises. */
int lbm_moments(lbm_ctx *ctx, double *rho, double *u, double *v, int ptr_kind);

/* Ensemble-mean velocity ubar = M^{-1} sum_m u_m, the best estimate the
 * paper scores against the truth (Section 4.3, RMSE). u, v: [ny][nx]; either
 * may be NULL. With LBM_PTR_HOST the call synchronises. */
int lbm_mean_velocity(lbm_ctx *ctx, double *u, double *v, int ptr_kind);

/* Velocity RMSE of ctx's ensemble mean against truth's (Section 4.3 scores
 * the ensemble mean against the nature run):
 *   rmse = sqrt( (nx ny)^-1 sum_xi (ubar - ubar_t)^2 + (vbar - vbar_t)^2 ),
 * ubar the member mean of each context (the truth usually has one member).
 * Both lattices must have the same size. FP64, reduced on the device in a
 * fixed order; the truth's queued work is waited for on ctx's stream.
 * rmse: one double, host or device per ptr_kind (LBM_PTR_HOST
 * synchronises). */
int lbm_velocity_rmse(lbm_ctx *ctx, lbm_ctx *truth, double *rmse, int ptr_kind);

/* Energy spectrum of the ensemble (Section 4.1, shell-averaged spectrum;
 * Section 4.3 takes the mean of the members' spectra). For every member,
 * u-hat(k') = N^{-1} sum_xi u(xi) exp(-i k'.xi) over the N = nx*ny cells for
 * both velocity components, E(k') = |u-hat(k')|^2 / 2, summed over the shell
 * s - 1/2 <= |k'| < s + 1/2 (k' in signed integer wavenumbers), then averaged
 * over members. E[nshells] receives shells s = 0 .. nshells-1; wavenumbers in
 * higher shells are dropped (floor(hypot(nx/2, ny/2) + 1/2) + 1 shells hold
 * them all). FP64 in both precisions. With LBM_PTR_HOST the call
 * synchronises; the scratch it needs is allocated and released on the
 * context stream. LBM_EINVAL if nshells < 1 or the lattice is too large for
 * the diagnostic (nx or ny beyond about 1700). */
int lbm_energy_spectrum(lbm_ctx *ctx, double *E, int nshells, int ptr_kind);

/* Observation step (Section 3, y = H x; Section 3.2, ybar and dY): record
 * npts observation points (ix[j], iy[j]) with observed velocities
 * (yo_u[j], yo_v[j]) and error standard deviations sigma_u, sigma_v, apply
 * H to every forecast member, and form dY = Y - ybar and d = y^o - ybar on
 * the device. Host pointers (read before the call returns; the values are
 * staged through a pinned buffer, so the call does not wait for the
 * device); npts >= 1; 0 <= ix < nx, 0 <= iy < ny; sigma > 0. The
 * observation vector orders scalars as (u_0, v_0, u_1, ...). */
int letkf_observe(lbm_ctx *ctx, int npts, const int *ix, const int *iy,
                  const double *yo_u, const double *yo_v, double sigma_u,
                  double sigma_v);

/* letkf_observe with the density observed as well (Section 4.3 observes
 * rho at the same points as the velocity, with its own error level): the
 * observation vector holds three scalars per point, (u_j, v_j, rho_j), with
 * error standard deviations sigma_u, sigma_v, sigma_rho; rho_m = sum_alpha
 * f_alpha of member m. Localisation gives the three scalars of a point the
 * same Gaspari-Cohn weight. Same pointer rules and errors as letkf_observe;
 * yo_rho must not be NULL and sigma_rho must be finite and > 0. The next
 * letkf_analyze assimilates all three. */
int letkf_observe_rho(lbm_ctx *ctx, int npts, const int *ix, const int *iy,
                      const double *yo_u, const double *yo_v, const double *yo_rho,
                      double sigma_u, double sigma_v, double sigma_rho);

/* Arithmetic of the local Gram matrix C = (k-1)/beta I + Yh^T Yh and of
 * b = Yh^T d-hat (Section 3.2, with Yh = R_loc^{-1/2} dY_loc) in the
 * ensemble-space form (p >= k) of a mixed-precision context's analysis:
 *   LBM_PROD_DF32  FP64-class: double-binary32 products and sums on the
 *                  binary32 units (each value split into two binary32
 *                  halves, rounding errors recovered exactly; C within
 *                  a few 1e-13 relative of FP64), the default;
 *   LBM_PROD_FP64  FP64 products and sums;
 *   LBM_PROD_FP32  binary32 products, binary32 accumulation (CUDA cores);
 *   LBM_PROD_TF32  TF32 products on the tcgen05 tensor cores, binary32
 *                  accumulation in tensor memory (rows staged by TMA);
 *   LBM_PROD_BF16  BF16 products, likewise.
 * A bounded wait of the tensor-core pass that runs out is reported by the
 * next synchronising call as LBM_ECUDA. The merged observation list of
 * eight neighbouring grid points must fit shared memory with the operand
 * tiles (about 30,000 observation points); beyond it the launch fails with
 * LBM_ECUDA.
 * The eigensolve stays FP64-accurate in every mode; the modes apply for
 * members <= 128 (larger ensembles form C in FP64 per grid point).
 * LBM_EINVAL for an unknown mode or a mode other than LBM_PROD_FP64 on an
 * FP64 context. Applies to later analyses. */
enum { LBM_PROD_FP64 = 0, LBM_PROD_FP32 = 1, LBM_PROD_TF32 = 2, LBM_PROD_BF16 = 3, LBM_PROD_DF32 = 4 };
int letkf_set_products(lbm_ctx *ctx, int mode);

/* Grid points per run of the analysis (Section 3.2: the local analyses are
 * independent, so they may be taken in any order). A run is run_len
 * consecutive grid points of one lattice row, analysed by one warp over the
 * union of their local observation sets: a scalar outside a point's
 * support enters that point with weight zero, which leaves its analysis
 * unchanged, and each point's binary32 Jacobi starts from the previous
 * point's basis. In a mixed-precision context that basis is refined to
 * FP64-class accuracy; in a double-precision context an FP64 Jacobi starts
 * from it and runs to the cold path's stopping rule, so the eigenpairs are
 * FP64's. Used when every grid point has p < members and every run's union
 * holds at most 32 scalars; otherwise, and with run_len = 0, the analysis
 * takes the cold-started path (one Jacobi per point from the identity).
 * Default 8. LBM_EINVAL outside [0, 4096]. Applies to later analyses;
 * results agree with either path to rounding. */
int letkf_set_run_length(lbm_ctx *ctx, int run_len);

/* Pipelining of the run analysis (Section 3.2's local analyses taken in
 * chunks of runs): with runs > 0 and more than one chunk, the runs are
 * taken in chunks of `runs`, the Jacobi kernel of chunk c + 1 running on a
 * second stream of the context beside the refinement (mixed precision) or
 * the FP64 kernel (double precision) of chunk c, so that the two share the
 * GPU's SMs; the result is the same as unpipelined, bit for bit. 0 turns it
 * off, the default: at 256^2 x 64 members every chunk size measured slower
 * than one pass (4.97-8.8 ms against 4.88 ms mixed, 38.1-44.5 against
 * 37.8 ms FP64 for chunks of 4096 down to 512 runs). LBM_EINVAL outside
 * [0, 2^24]. Applies to later analyses. */
int letkf_set_run_pipeline(lbm_ctx *ctx, int runs);

/* Diagnostic: count the Jacobi sweeps of every local eigensolve of later
 * analyses (enable != 0) into a 32-bin histogram (bin s: points that took s
 * sweeps, the last one rotating nothing; bin 31: 31 or more, or the sweep
 * cap). With hist (host, [32]) non-NULL the current counts are copied out
 * and reset (synchronises). Recording adds one atomic per grid point. */
int letkf_sweep_stats(lbm_ctx *ctx, int enable, int *hist);

/* Set the Smagorinsky coefficient C_s of the eddy-viscosity closure
 * (Section 2) used by the following forecasts; finite, >= 0. */
int lbm_set_closure(lbm_ctx *ctx, double cs_smag);

/* Windowed observation misfit of every member (the cost a variational
 * method minimises; the paper's Section 1 contrasts it with the ensemble
 * method): starting from the current state (left unchanged), forecast
 * nsteps steps and accumulate
 *   J_m = 1/2 sum_t sum_j [ (u_m(eta_j, t) - yo_u[t][j])^2 / sigma_u^2
 *                          + (v_m(eta_j, t) - yo_v[t][j])^2 / sigma_v^2 ].
 * J: host [members]. Synchronises. */
int lbm_misfit(lbm_ctx *ctx, const lbm_window *win, double *J);

/* lbm_misfit and its gradient by the hand-written adjoint of the forecast
 * (reverse sweep through the transposed collision Jacobian and the pulled
 * streaming, with the forward states recomputed from checkpoints). For
 * F = sum_m w_m J_m (w: [members], NULL = all ones; host or device per
 * ptr_kind, device weights are not checked for finiteness):
 *   grad_f0 [9][ny][nx][members]  dF/df at the current state (FP64; host
 *                                 or device per ptr_kind),
 *   grad_cs [members] (host)      w_m dJ_m/dC_s,
 *   dcs     [1]                   dF/dC_s = sum_m w_m dJ_m/dC_s, summed on
 *                                 the device in member order (host or
 *                                 device per ptr_kind).
 * J stays a host array [members]. Any output may be NULL. In mixed
 * precision the forecast and the adjoint run in binary32 (C_s derivative
 * summed in FP64); in FP64 mode everything is FP64. Scratch of about
 * (nsteps / checkpoint_every + checkpoint_every + 3) states is allocated
 * and released on the context stream. Synchronises. */
int lbm_misfit_gradient(lbm_ctx *ctx, const lbm_window *win, const double *w, double *J,
                        double *grad_f0, double *grad_cs, double *dcs, int ptr_kind);

/* LETKF analysis of the nine f_alpha at every grid point, in place
 * (Section 3.2: w-bar, P-tilde, delta-W = [(k-1) P-tilde]^{1/2} symmetric,
 * x^a_m = xbar + dX (w-bar + delta-W_m); R-localisation with the
 * Gaspari-Cohn weight G(r / d_cut), r the periodic distance, support
 * r < 2 d_cut; inflation P^f -> beta P^f). Uses the observations of the
 * last letkf_observe call, which it consumes. d_cut > 0, beta > 0,
 * members >= 2. Asynchronous. The local eigenproblem has size
 * n = min(k, p), p the number of local observation scalars; a grid point
 * with n > 64 (LBM_FP64) or n > 128 (LBM_MIXED) is reported as LBM_EINVAL
 * at the next synchronising call and leaves that point unchanged. */
int letkf_analyze(lbm_ctx *ctx, double d_cut, double beta);

/* Diagnostic of the mixed-precision analysis (Section 3.2: w-bar, W and the
 * transform x^a_m = xbar + sum_j dx_j (w-bar_j + W_jm)). For the grid points
 * cells[npoints] (host array of y * nx + x, 1 <= npoints <= 4096), writes
 * T[p][j][m] = w-bar_j + W[j][m] ([npoints][members][members], FP64, host or
 * device per ptr_kind) as the run analysis represents it: the same
 * warm-started binary32 bases and the same first-order refinement as
 * letkf_analyze, with the resulting matrix functions applied in FP64 instead
 * of the binary32 transform. Same arguments as the following letkf_analyze;
 * the state is not changed and the observation is not consumed. Needs a
 * mixed-precision context on the run path (run length > 0, every grid point
 * with p < members, every run's union of local sets within 32 scalars);
 * otherwise LBM_EINVAL. Synchronises. */
int letkf_probe_transform(lbm_ctx *ctx, double d_cut, double beta, int npoints, const int *cells,
                          double *T, int ptr_kind);

/* Nudging, the paper's comparison method (Section 3.1): every member is
 * relaxed toward the equilibrium of the observed macroscopic field,
 * f_alpha <- f_alpha + gamma (f^eq_alpha(rho^, u^, v^) - f_alpha), 0 <= gamma <= 1.
 * The observations sit on the uniform periodic lattice of points
 * (i nx/nobs_x, j ny/nobs_y): host arrays rho_o, u_o, v_o [nobs_y][nobs_x]
 * (copied before the call returns). rho^, u^, v^ at a grid point are their
 * bilinear interpolation (the paper's "simple linear interpolation"). nx and
 * ny must be multiples of nobs_x and nobs_y. Asynchronous. */
int lbm_nudge(lbm_ctx *ctx, int nobs_x, int nobs_y, const double *rho_o,
              const double *u_o, const double *v_o, double gamma);

/* Copy the state out (checkpoint, parity) or in (restart, fault tests).
 * Layout f [9][ny][nx][members] FP64. lbm_get_f with LBM_PTR_HOST
 * synchronises. */
int lbm_get_f(lbm_ctx *ctx, double *f, int ptr_kind);
int lbm_set_f(lbm_ctx *ctx, const double *f, int ptr_kind);

/* Wait for the context stream and report deferred device conditions
 * (LBM_EDIVERGED, LBM_ENOCONV, LBM_EINVAL for an oversized local problem).
 * The flag word is cleared after it is reported. */
int lbm_sync(lbm_ctx *ctx);

/* Message for the last failure on ctx (or, when ctx is NULL, of the last
 * failed lbm_init or letkf_analyze_noalloc on this thread). Never NULL. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Free the context and its device buffers (synchronises its stream). */
void lbm_destroy(lbm_ctx *ctx);

/* Limits of letkf_analyze_noalloc. */
#define LBM_NOALLOC_MAX_POINTS 256   /* observation points (512 scalars) */
#define LBM_NOALLOC_MAX_MEMBERS 128  /* ensemble members */

/* Allocation-free LETKF analysis, for callers that cannot call cudaMalloc
 * (an embedding whose memory manager owns the device pool, or code that
 * must not trigger an allocation's implicit synchronisation). The paper has
 * no counterpart; this is a library-interface addition. It performs the
 * same observation step and analysis as letkf_observe + letkf_analyze, on
 * an FP64 ensemble state the caller owns, without a context:
 *   f      device pointer, [9][ny][nx][members] FP64, updated in place;
 *   ix, iy, yo_u, yo_v  host arrays of npts observation points and values
 *          (checked on the host, then copied);
 *   stream cudaStream_t (NULL = legacy default stream).
 * Intermediates (dY, d, dY dY^T, positions, a flag word) live in one fixed
 * file-scope device array of about 2.6 MB that every GPU loading the
 * library holds until exit; nothing is allocated or freed. Sizes above
 * LBM_NOALLOC_MAX_POINTS / LBM_NOALLOC_MAX_MEMBERS are rejected with
 * LBM_EINVAL. The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture. Every call shares the array and overwrites
 * it; two calls that overlap on the GPU (different streams, or different
 * host threads) race on it and must be serialised by the caller. The call
 * synchronises the stream and returns LBM_OK, LBM_EINVAL (bad argument, or a
 * local problem larger than the kernel holds), LBM_ENOCONV or LBM_ECUDA;
 * lbm_last_error(NULL) gives the message. The analysis is the FP64 one, so
 * a grid point's local problem must satisfy n = min(members, 2 p) <= 64 (p
 * observation points in range): with more than 64 members, dense
 * observations are refused. On LBM_EINVAL for a too-large local problem and
 * on LBM_ENOCONV the state is partly updated: every grid point that fitted
 * or converged has been analysed, the others are unchanged. */
int letkf_analyze_noalloc(double *f, int nx, int ny, int members, int npts,
                          const int *ix, const int *iy, const double *yo_u,
                          const double *yo_v, double sigma_u, double sigma_v,
                          double d_cut, double beta, void *stream);

/* ---- Batches of independent experiments ----------------------------------
 * Many DA experiments of uneven lattice, ensemble and observation sizes
 * (the "thousands of trial-and-error experiments" of Section 1) advanced
 * together. A batch groups existing contexts (1..64, one precision, one
 * shared stream; the contexts stay owned by the caller and must outlive the
 * batch). */
typedef struct lbm_batch lbm_batch;

/* Create a batch over ctxs[0..n-1]. LBM_EINVAL if a context is NULL or
 * repeated, or the contexts differ in stream or precision. */
int lbm_batch_create(lbm_ctx *const *ctxs, int n, lbm_batch **out);

/* Advance every context nsteps LBM steps (Section 2) in ONE cooperative
 * persistent launch: the grid strides over the work items of all
 * experiments, and a grid barrier separates the steps. Each barrier wait is
 * bounded (a few seconds); a timeout is reported by lbm_batch_sync.
 * Results are identical to lbm_forecast on each context. Asynchronous. */
int lbm_batch_forecast(lbm_batch *b, int nsteps);

/* Pick the persistent launch shape (threads per block, blocks) by timing
 * candidates on the batch's own experiments: block sizes 128/256/512 times
 * 1..max co-resident blocks per SM, one step each into the spare buffers
 * (the current states are unchanged). threads/blocks may be NULL.
 * Synchronises. */
int lbm_batch_autotune(lbm_batch *b, int *threads, int *blocks);

/* Pick the run length (grid points per warp, letkf_set_run_length) of the
 * batch's analyses per size class: experiments whose analysis takes the
 * run path (every grid point with p < members) are grouped by the union
 * size of their runs (up to 8, 16, 24, 28, 32 scalars); mixed-precision
 * experiments with ensemble-space points and at most 32 members (whose
 * Jacobi kernel warm-starts along runs) by their member tile (8, 16, 24,
 * 28, 32). Each class times its analyses at run lengths 4, 8, 16 and 32,
 * best of three, keeping the fastest; a run-path class times two forms at
 * each length: batched (kernel J over every run of the class in one
 * launch, then kernel F per experiment over all its grid points) and one
 * experiment after another (each with its own launches in chunks of runs,
 * as lbm_analyze makes them).
 * lbm_batch_cycle then analyses the class in the form chosen; the results
 * are the same in both forms. The timed analyses work on copies of the
 * current states in the spare buffers: states and observations are
 * unchanged. Every context must be observed (letkf_observe) with the
 * observations the analyses will use (d_cut[i], beta[i]). run_len[i] (may
 * be NULL) receives each experiment's run length (unchanged for
 * experiments in no class); batched[i] (may be NULL) 1 if its run
 * analysis goes into the batched launches, else 0 (the default before
 * tuning is 1). Synchronises; a captured cycle is captured again. */
int lbm_batch_autotune_analysis(lbm_batch *b, const double *d_cut, const double *beta, int *run_len,
                                int *batched);

/* Set the launch form of each experiment's run analysis in lbm_batch_cycle
 * (the choice lbm_batch_autotune_analysis makes): batched[i] = 1 puts
 * experiment i's run analysis into the size class's batched launch of
 * kernel J, 0 launches it on its own (as lbm_analyze does). Results are
 * the same in both forms; experiments off the run path ignore it. One value
 * per context of the batch (host array, read before the call returns);
 * LBM_EINVAL for a value other than 0 or 1. A captured cycle is captured
 * again. */
int lbm_batch_set_analysis_form(lbm_batch *b, const int *batched);

/* One DA cycle of every experiment i: forecast nsteps (one persistent
 * launch for all), observe (u, v) at npts[i] points (ix[i], iy[i]) with
 * values yo_u[i], yo_v[i] and errors sigma[2i], sigma[2i+1], and the LETKF
 * analysis with d_cut[i], beta[i]. The analyses of experiments on the run
 * path share launches: per size class one launch of kernel J over all
 * their runs, then one launch of kernel F per experiment over all its grid
 * points (the analysis scratch of each is then sized for all its runs at
 * once); the others, and run-path experiments whose launch form is set to
 * 0 (lbm_batch_autotune_analysis, lbm_batch_set_analysis_form), are
 * analysed one by one. With use_graph, once a cycle has run
 * uncaptured with the same positions, nsteps, d_cut and beta, the next call
 * captures the whole cycle of all experiments in a CUDA graph and later
 * calls replay it, staging only the new observed values through pinned
 * memory (nsteps must be even so the state buffers return to their roles).
 * A change of plan falls back to an uncaptured cycle. Asynchronous except
 * for waiting on the previous cycle's copies; errors surface at
 * lbm_batch_sync. Host arrays are read before the call returns. */
int lbm_batch_cycle(lbm_batch *b, int nsteps, const int *npts, const int *const *ix,
                    const int *const *iy, const double *const *yo_u, const double *const *yo_v,
                    const double *sigma, const double *d_cut, const double *beta, int use_graph);

/* Wait for the batch's work; reports a timed-out grid barrier, then each
 * context's deferred status (as lbm_sync). */
int lbm_batch_sync(lbm_batch *b);

/* Bound of every grid-barrier wait of the batch's persistent forecast:
 * spin_limit rounds of a 100 ns sleep (1 .. 20,000,000, the default; about
 * 2-4 s). absent = 1 makes each barrier wait for one participant more than
 * the grid holds, so every wait runs out: the forecast stops after its first
 * step, every block returns, and lbm_batch_sync reports LBM_ECUDA ("a grid
 * barrier ... timed out"); this exercises the timeout path without a fault.
 * absent = 0 restores normal operation. Synchronises; a captured cycle is
 * captured again. LBM_EINVAL outside these ranges. */
int lbm_batch_set_barrier(lbm_batch *b, long long spin_limit, int absent);
const char *lbm_batch_last_error(const lbm_batch *b);
void lbm_batch_destroy(lbm_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* LBM_LETKF_H */
