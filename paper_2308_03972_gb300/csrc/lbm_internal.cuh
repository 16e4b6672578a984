// Internal declarations shared by the CUDA translation units of the
// LBM-LETKF library. Not part of the C ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace lbmgpu {

// Bits of the device flag word (reported by lbm_sync).
enum : int {
    FLAG_DIVERGED = 1,  // non-finite or |u| above the limit
    FLAG_NOCONV = 2,    // eigensolver sweep cap reached
    FLAG_TOOLARGE = 4,  // local problem larger than the analysis kernel holds
    FLAG_TCWAIT = 8     // a bounded wait of the tensor-core Gram ran out
};

// Arithmetic of the local Gram matrix C = a I + Yh^T Yh and b = Yh^T d-hat in
// the ensemble-space form of the mixed-precision analysis: FP64,
// double-binary32 (FP64-class, the default), or binary32 accumulation of
// binary32 / TF32 / BF16 products.
enum : int { PROD_FP64 = 0, PROD_FP32 = 1, PROD_TF32 = 2, PROD_BF16 = 3, PROD_DF32 = 4 };
// No ensemble-space grid point in this analysis: no Gram pass at all.
constexpr int PROD_NONE = -1;

// Speed limit used by the divergence check: |u| > 0.5 lattice units.
constexpr double kUMax2 = 0.25;

// D2Q9 set (arXiv 2308.03972, Section 2): rest, +-x, +-y, four diagonals.
__host__ __device__ constexpr int d2q9_cx(int a) {
    return a == 1 || a == 5 || a == 7 ? 1 : (a == 2 || a == 6 || a == 8 ? -1 : 0);
}
__host__ __device__ constexpr int d2q9_cy(int a) {
    return a == 3 || a == 5 || a == 8 ? 1 : (a == 4 || a == 6 || a == 7 ? -1 : 0);
}
__host__ __device__ constexpr double d2q9_w(int a) {
    return a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}

struct LbmParams {
    int nx, ny, k;
    double tau0;
    double cs18;  // 18 C_s^2 Delta^2 with Delta = 1
    double mu;
};

// Observation vector: nvar scalars per point, row nvar*j + q holding u
// (q = 0), v (q = 1) and, when nvar = 3, rho (q = 2) at point j.
struct ObsParams {
    int npts;          // observation points
    const int* ix;     // [npts]
    const int* iy;     // [npts]
    const double* dY;  // [nobs][k] perturbations of H(x_m), nobs = nvar npts
    const double* d;   // [nobs] innovations y^o - ybar
    const double* G;   // [nobs][nobs] dY dY^T
    double sigma_u, sigma_v;
    float* dY32;       // [nobs][k] binary32 copy of dY (mixed precision only)
    int nvar = 2;      // 2: (u, v); 3: (u, v, rho)
    double sigma_r = 1.0;
    int plmax = 0;     // capacity of one grid point's local list (0: nobs); a
                       // point with more local scalars is reported too large
    int* sweep_hist = nullptr;  // [32] Jacobi sweep counts per point, or null
};

// ---- lbm_kernels.cu -------------------------------------------------------
// One fused collide+push step. FP64: f stored as is. FP32: f stored as
// g = f - w_alpha (rest-state shift) in binary32.
cudaError_t launch_lbm_step_f64(const double* fin, double* fout, const double* force,
                                const LbmParams& p, int* flags, cudaStream_t s);
cudaError_t launch_lbm_step_f32(const float* gin, float* gout, const float* force,
                                const LbmParams& p, int* flags, cudaStream_t s);
// One experiment of a persistent multi-ensemble forecast: its state buffers
// (f[cur] holds the current state), forcing, flag word, lattice, members,
// parameters, members per work item V (1, 2 or 4; 4 means 2 in FP64) and
// its range [offset, offset + items) of the global work-item index.
struct MultiExp {
    void* f[2];
    const void* force;
    int* flags;
    int nx, ny, k, V, cur;
    double tau0, cs18, mu;
    long long offset, items;
};
constexpr int kMaxMultiExp = 64;
// Cooperative launch of `blocks` x `threads` advancing every experiment
// nsteps steps (ex_dev: device array). bar: two zeroed words (reset here);
// status: set to 1 if a grid barrier timed out. Each barrier wait spins at
// most spin_limit rounds of a 100 ns sleep; absent > 0 makes every wait run
// out (participants that never arrive).
constexpr long long kBarrierSpins = 20000000;  // default: ~2-4 s
cudaError_t launch_lbm_multi(const MultiExp* ex_dev, int nexp, long long total, int nsteps, int fp32,
                             int blocks, int threads, unsigned* bar, int* status, long long spin_limit,
                             unsigned absent, cudaStream_t s);
// Largest co-resident grid for the multi kernel (0 on error).
int lbm_multi_max_blocks(int fp32, int threads);
// Nudging toward f^eq of observations on a uniform lattice; obs = rho, u, v
// fields [3][noy][nox] in device memory.
cudaError_t launch_nudge(void* f, int fp32, int nx, int ny, int k, int nox, int noy,
                         const double* obs, double gamma, cudaStream_t s);
cudaError_t launch_moments(const void* f, int fp32, int nx, int ny, int k, double* rho,
                           double* u, double* v, int* flags, cudaStream_t s);
cudaError_t launch_mean_velocity(const void* f, int fp32, int nx, int ny, int k, double* u,
                                 double* v, int* flags, cudaStream_t s);
cudaError_t launch_set_equilibrium(void* f, int fp32, int nx, int ny, int k,
                                   const double* rho, const double* u, const double* v,
                                   cudaStream_t s);
cudaError_t launch_store_f(void* f, int fp32, const double* src, size_t n, cudaStream_t s);
cudaError_t launch_load_f(const void* f, int fp32, double* dst, size_t n, cudaStream_t s);
cudaError_t launch_store_force(void* dst, int fp32, const double* src, size_t n,
                               cudaStream_t s);

// ---- letkf_kernels.cu -----------------------------------------------------
cudaError_t launch_observe(const void* f, int fp32, int nx, int ny, int k, int npts, int nvar,
                           const int* ix, const int* iy, const double* yo, double* dY,
                           double* d, cudaStream_t s);
cudaError_t launch_obs_gram(const double* dY, int nobs, int k, double* G, cudaStream_t s);
// Second stream and events the mixed-precision analysis uses to overlap its
// binary32 Jacobi pass over one chunk of grid points with the FP64
// refinement of the previous chunk.
struct AnalyzeAux {
    cudaStream_t s2;
    cudaEvent_t start, jac_done[2], ref_done[2];
};
// Scratch the analysis needs (bytes; 0 for the FP64 path).
// nl: capacity of a local list (ObsParams::plmax, or nobs).
size_t analyze_scratch_bytes(int nx, int ny, int fp32, int nl, int nmax, int k, int prod);
// nmax: largest local problem size n = min(p, k) over the grid (sizes the
// mixed kernel's shared memory; points above it are reported as too large).
// prod: PROD_* arithmetic of the ensemble-space Gram (mixed precision only),
// PROD_NONE when no grid point uses the ensemble-space form.
// warm_run > 1 (binary32 states with a Gram pass): kernel (A) takes runs of
// warm_run consecutive grid points per warp and starts each ensemble-space
// point's Jacobi from the previous one's basis.
cudaError_t launch_analyze(void* f, int fp32, int nx, int ny, int k, const ObsParams& o,
                           double d_cut, double beta, int nmax, int prod, int warm_run, int* flags,
                           void* scratch, const AnalyzeAux* aux, cudaStream_t s);

// dst = (float) src, n elements.
cudaError_t launch_to_f32(const double* src, float* dst, size_t n, cudaStream_t s);

// ---- letkf_runs.cu --------------------------------------------------------
// Mixed-precision analysis over runs of run_len consecutive grid points of a
// row (one warp each; warm-started binary32 Jacobi over the union of the
// run's local sets), observation-space form. Valid when every grid point
// has p < k and the union of every run holds at most 32 scalars
// (maxunion: that largest union, from the host's geometry). scratch holds
// run_scratch_bytes(...) bytes: a split copy of the observation Gram and,
// per chunk of runs, every grid point's binary32 basis and eigenvalue
// estimates (handed from the Jacobi kernel to the refinement kernel).
constexpr int kRunMaxUnion = 32;
// whole: scratch for every run at once (the batched launch) rather than for
// chunks of runs within a fixed budget.
size_t run_scratch_bytes(int nx, int ny, int nobs, int run_len, int maxunion, bool whole = false);
// aux (may be null) and pipe_runs > 0: chunks of pipe_runs runs with kernel
// J on aux->s2 beside the refinement of the previous chunk on s.
cudaError_t launch_analyze_runs(float* f, int nx, int ny, int k, const ObsParams& o, double d_cut,
                                double beta, int run_len, int maxunion, int* flags, void* scratch,
                                const AnalyzeAux* aux, int pipe_runs, cudaStream_t s);
// The same runs for a double-precision context: the binary32 Jacobi of the
// run gives each grid point a starting basis, and an FP64 Jacobi from it
// (launch_run_fp64, letkf_kernels.cu) gives the eigenpairs; transform and
// update in FP64. scratch as above.
cudaError_t launch_analyze_runs_fp64(double* f, int nx, int ny, int k, const ObsParams& o, double d_cut,
                                     double beta, int run_len, int maxunion, int* flags, void* scratch,
                                     const AnalyzeAux* aux, int pipe_runs, cudaStream_t s);
// FP64 warm-started analysis of the nruns * run_len grid points of the runs
// run0.. (chunk-local basis Yg [.][ns][ns], eigenvalue estimates lamg
// [.][ns] with -1 marking a point with no observation in range, union
// lists rinfo [.][info_stride]).
cudaError_t launch_run_fp64(double* f, int nx, int ny, int k, const ObsParams& o, double d_cut, double beta,
                            int run_len, int run0, int nruns, int ns, const float* Yg, const float* lamg,
                            const int* rinfo, int info_stride, int* flags, cudaStream_t s);
// The run analyses of several experiments (one lattice, state and
// observation set each) in batched launches: kernel J over the runs of
// every experiment of a size class in one launch, then kernel F over their
// grid points in one launch (the FP64 kernel per experiment for FP64
// states). Each item's scratch holds run_scratch_bytes(..., whole = true).
struct RunItem {
    float* f;      // binary32 state, or null
    double* f64;   // FP64 state, or null
    int nx, ny, k, run_len, maxunion;
    ObsParams o;
    double d_cut, beta;
    int* flags;
    void* scratch;
};
cudaError_t launch_analyze_runs_batch(const RunItem* items, int n, cudaStream_t s);
// Diagnostic: the ensemble transform T = w-bar 1^T + W [npoints][k][k]
// (FP64) that the run analysis' refined representation gives at the listed
// grid points cells[npoints] (device), evaluated in FP64; f is not
// changed. work: probe_work_bytes(npoints, maxunion, k) bytes.
size_t probe_work_bytes(int npoints, int maxunion, int k);
cudaError_t launch_probe_runs(float* f, int nx, int ny, int k, const ObsParams& o, double d_cut, double beta,
                              int run_len, int maxunion, int* flags, void* scratch, const int* cells,
                              int npoints, double* T, double* work, cudaStream_t s);

// ---- diag_kernels.cu ------------------------------------------------------
// Member-averaged energy spectrum E[nshells] (device pointer); work holds
// spectrum_work_bytes(nx, ny, k, nshells) bytes. Lattices whose row or column
// pass does not fit shared memory give cudaErrorInvalidValue.
size_t spectrum_work_bytes(int nx, int ny, int k, int nshells);
cudaError_t launch_energy_spectrum(const void* f, int fp32, int nx, int ny, int k, double* E,
                                   int nshells, void* work, int* flags, cudaStream_t s);

// *out = sqrt(n^-1 sum_i (u1 - u2)^2 + (v1 - v2)^2), FP64, fixed summation
// order; work: rmse_work_doubles() doubles.
size_t rmse_work_doubles();
cudaError_t launch_velocity_rmse(const double* u1, const double* v1, const double* u2, const double* v2, size_t n,
                                 double* work, double* out, cudaStream_t s);

// ---- adjoint_kernels.cu ---------------------------------------------------
// Adjoint of one LBM step at the stored state f_t: lam_out = (df_{t+1}/df_t)^T
// lam_in; dJ/dCs of every member added to gcs[k] (FP64). fp32: FP32 shifted
// state and FP32 adjoint; else FP64 for both. force in the state's type.
cudaError_t launch_adjoint_step(const void* ft, const void* lam_in, void* lam_out, const void* force,
                                int fp32, const LbmParams& p, double cs, double* gcs,
                                cudaStream_t s);
// Misfit terms r[npts][k] of one observation time; yo [npts][2] (u, v).
cudaError_t launch_misfit(const void* f, int fp32, int nx, int ny, int k, int npts, const int* ix,
                          const int* iy, const double* yo, double sigma_u, double sigma_v,
                          double* r, cudaStream_t s);
// lam += w_m d(misfit of one time)/df at the observation points.
cudaError_t launch_misfit_adjoint(const void* f, void* lam, int fp32, int nx, int ny, int k, int npts,
                                  const int* ix, const int* iy, const double* yo, double sigma_u,
                                  double sigma_v, const double* w, cudaStream_t s);
// J[m] = sum_i r[i][m], i < nterms, in order.
cudaError_t launch_misfit_reduce(const double* r, int nterms, int k, double* J, cudaStream_t s);
// dst = (double) src, n elements (no shift: for adjoint fields).
cudaError_t launch_widen(const void* src, int fp32, double* dst, size_t n, cudaStream_t s);

}  // namespace lbmgpu
