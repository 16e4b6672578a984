// C ABI of the LBM-LETKF library: context management, argument checks,
// host/device marshalling and kernel launches. See include/lbm_letkf.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "../../include/lbm_letkf.h"
#include "lbm_internal.cuh"

using namespace lbmgpu;

struct lbm_ctx {
    int nx = 0, ny = 0, k = 0, precision = LBM_FP64;
    double tau0 = 0.0, cs = 0.0, mu = 0.0;
    cudaStream_t stream = nullptr;
    void* f[2] = {nullptr, nullptr};  // double-buffered state (double or float)
    int cur = 0;
    void* force = nullptr;           // [2][ny][nx] in the state's type
    int* flags = nullptr;            // device flag word
    double* stage = nullptr;         // FP64 staging [9][ny][nx][k] (lazy)
    // observations
    // nobs = nvar * npts scalars: (u, v) per point, or (u, v, rho).
    int npts = 0, nvar = 2, pts_cap = 0, nobs_cap = 0;
    int* ix = nullptr;
    int* iy = nullptr;
    double* yo = nullptr;  // [nobs] interleaved per point
    double* dY = nullptr;  // [nobs][k]
    double* d = nullptr;   // [nobs]
    double* G = nullptr;   // [nobs][nobs]
    float* dY32 = nullptr; // [nobs][k] binary32 copy (mixed precision)
    void* ana_scratch = nullptr;   // analysis scratch (mixed precision)
    size_t ana_scratch_bytes = 0;
    // Observation geometry of the last letkf_observe, and the largest local
    // problem it gives for a cached d_cut.
    std::vector<int> geo_ix, geo_iy;
    double geo_dcut = -1.0;
    int geo_nmax = 0;
    int geo_pmax = 0;  // largest local list (scalars) for geo_dcut
    bool geo_any_ens = false;  // some grid point has p >= k (ensemble-space form)
    // Largest union of local sets over runs of run_len grid points of a row
    // (the run analysis), for geo_dcut and union_rl.
    int geo_maxunion = -1;
    int union_rl = -1;
    int run_len = 8;  // grid points per run of the mixed analysis (0: chunked two-kernel path)
    AnalyzeAux aux{};              // second stream + events (mixed precision)
    bool aux_ready = false;
    double* nudge_obs = nullptr;  // [3][noy][nox] nudging observations
    size_t nudge_cap = 0;
    double* h_yo = nullptr;  // pinned staging [nobs_cap]
    int* h_ixy = nullptr;    // pinned staging [2 pts_cap] (ix then iy)
    cudaEvent_t obs_copied = nullptr;  // last staging copy done
    bool obs_pending = false;
    double sigma_u = 0.0, sigma_v = 0.0, sigma_r = 1.0;
    int prod = PROD_FP64;  // ensemble-space Gram arithmetic (mixed precision)
    int run_pipe = 0;      // runs per pipelined chunk of the run analysis (0: not pipelined)
    int run_batched = 1;   // in a batch: run analysis in the batched launches (0: launched on its own)
    int* sweep_hist = nullptr;  // [32] Jacobi sweeps per point (diagnostic)
    bool sweep_stats = false;
    bool observed = false;
    char err[512] = {0};
};

namespace {

thread_local char g_init_err[512] = "no error";

int fail(lbm_ctx* c, int code, const char* fmt, ...) {
    char* buf = c ? c->err : g_init_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
    return fail(c, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CK(ctx, call, what)                                       \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, what); \
    } while (0)

size_t elem_size(const lbm_ctx* c) { return c->precision == LBM_MIXED ? sizeof(float) : sizeof(double); }
size_t state_elems(const lbm_ctx* c) { return (size_t)9 * c->nx * c->ny * c->k; }
size_t cell_elems(const lbm_ctx* c) { return (size_t)c->nx * c->ny * c->k; }
int is_fp32(const lbm_ctx* c) { return c->precision == LBM_MIXED; }

bool ptr_kind_ok(int kind) { return kind == LBM_PTR_HOST || kind == LBM_PTR_DEVICE; }

int ensure_stage(lbm_ctx* c) {
    if (c->stage) return LBM_OK;
    CK(c, cudaMalloc(&c->stage, state_elems(c) * sizeof(double)), "allocating staging buffer");
    return LBM_OK;
}

// Copy n doubles from a host or device pointer into device memory dst.
int copy_in(lbm_ctx* c, double* dst, const double* src, size_t n, int kind) {
    CK(c, cudaMemcpyAsync(dst, src, n * sizeof(double),
                          kind == LBM_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                          c->stream),
       "copying input");
    return LBM_OK;
}

int read_flags(lbm_ctx* c) {
    int h = 0;
    CK(c, cudaMemcpyAsync(&h, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
       "reading device flags");
    CK(c, cudaStreamSynchronize(c->stream), "synchronising stream");
    if (h == 0) return LBM_OK;
    CK(c, cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream), "clearing device flags");
    CK(c, cudaStreamSynchronize(c->stream), "synchronising stream");
    if (h & FLAG_DIVERGED)
        return fail(c, LBM_EDIVERGED, "state diverged: non-finite density/velocity or |u| > 0.5");
    if (h & FLAG_TOOLARGE)
        return fail(c, LBM_EINVAL, "local analysis problem larger than the kernel supports (n = min(k, p) > 64 in FP64, > 128 in mixed precision)");
    if (h & FLAG_TCWAIT)
        return fail(c, LBM_ECUDA, "a bounded wait of the tensor-core Gram ran out (its analysis is incomplete)");
    return fail(c, LBM_ENOCONV, "eigensolver reached its sweep cap");
}

void free_obs(lbm_ctx* c) {
    if (c->obs_pending && c->obs_copied) cudaEventSynchronize(c->obs_copied);
    c->obs_pending = false;
    cudaFreeHost(c->h_yo);
    cudaFreeHost(c->h_ixy);
    c->h_yo = nullptr;
    c->h_ixy = nullptr;
    cudaFree(c->ix);
    cudaFree(c->yo);
    cudaFree(c->dY);
    cudaFree(c->d);
    cudaFree(c->G);
    cudaFree(c->dY32);
    c->dY32 = nullptr;
    c->ix = c->iy = nullptr;
    c->yo = c->dY = c->d = c->G = nullptr;
    c->pts_cap = c->nobs_cap = 0;
}

// Largest local problem n = min(p, k) over the grid for the current
// observation points and d_cut: p = 2 x (points with r / d_cut < 2), counted
// by stamping a disc around every point. The test uses a tiny margin so the
// count bounds the kernels' own (exact) selection from above.
int largest_local_problem(lbm_ctx* c, double d_cut) {
    if (c->geo_dcut == d_cut) return c->geo_nmax;
    const int nx = c->nx, ny = c->ny;
    std::vector<int> cnt((size_t)nx * ny, 0);
    const int R = (int)std::ceil(2.0 * d_cut);
    const int ox0 = -(nx / 2), ox1 = nx - 1 - nx / 2;
    const int oy0 = -(ny / 2), oy1 = ny - 1 - ny / 2;
    for (size_t j = 0; j < c->geo_ix.size(); ++j) {
        for (int dy = (oy0 > -R ? oy0 : -R); dy <= (oy1 < R ? oy1 : R); ++dy) {
            const int y = ((c->geo_iy[j] + dy) % ny + ny) % ny;
            for (int dx = (ox0 > -R ? ox0 : -R); dx <= (ox1 < R ? ox1 : R); ++dx) {
                const double r = std::sqrt((double)dx * dx + (double)dy * dy);
                if (r / d_cut < 2.0 + 1e-12) {
                    const int x = ((c->geo_ix[j] + dx) % nx + nx) % nx;
                    ++cnt[(size_t)y * nx + x];
                }
            }
        }
    }
    int nmax = 2, vmax = 0;
    for (int v : cnt) {
        const int n = (c->nvar * v < c->k) ? c->nvar * v : c->k;
        if (n > nmax) nmax = n;
        if (v > vmax) vmax = v;
    }
    c->geo_dcut = d_cut;
    c->geo_maxunion = -1;
    c->geo_nmax = nmax;
    c->geo_pmax = c->nvar * (vmax > 0 ? vmax : 1);
    c->geo_any_ens = c->nvar * vmax >= c->k;
    return nmax;
}

// Largest number of observation scalars in the union of the local sets of a
// run of run_len consecutive grid points of a row (runs start at x = 0,
// run_len, ...). An observation point belongs to a run when
// r / d_cut < 2 at some cell of it, the kernels' own test; for each point
// and row the cells in range form one interval |dx| <= dxmax(dy), and every
// run that interval meets is counted.
int largest_run_union(lbm_ctx* c, double d_cut, int run_len) {
    largest_local_problem(c, d_cut);
    if (c->geo_maxunion >= 0 && c->union_rl == run_len) return c->geo_maxunion;
    const int nx = c->nx, ny = c->ny;
    const int rx = (nx + run_len - 1) / run_len;
    std::vector<int> cnt((size_t)ny * rx, 0);
    std::vector<int> stamp((size_t)rx, -1);
    const int R = (int)std::ceil(2.0 * d_cut) + 1;
    const int hx = nx / 2, hy = ny / 2;
    for (size_t j = 0; j < c->geo_ix.size(); ++j) {
        for (int dy = -R; dy <= R; ++dy) {
            if (dy > hy || dy < -hy) continue;          // outside the minimum image
            if (ny % 2 == 0 && dy == -hy) continue;     // -n/2 maps to +n/2
            const double dy2 = (double)dy * dy;
            int dxmax = -1;
            for (int dx = 0; dx <= hx; ++dx) {
                if (std::sqrt((double)dx * dx + dy2) / d_cut < 2.0) dxmax = dx;
                else break;
            }
            if (dxmax < 0) continue;
            const int y = ((c->geo_iy[j] + dy) % ny + ny) % ny;
            int* row = cnt.data() + (size_t)y * rx;
            const int tag = (int)(j * (2 * R + 1) + (dy + R));
            if (2 * dxmax + 1 >= nx) {
                for (int q = 0; q < rx; ++q) row[q] += 1;
                continue;
            }
            for (int dx = -dxmax; dx <= dxmax; ++dx) {
                const int x = ((c->geo_ix[j] + dx) % nx + nx) % nx;
                const int q = x / run_len;
                if (stamp[q] != tag) {
                    stamp[q] = tag;
                    ++row[q];
                }
            }
        }
    }
    int vmax = 0;
    for (int v : cnt) vmax = v > vmax ? v : vmax;
    c->geo_maxunion = c->nvar * vmax;
    c->union_rl = run_len;
    return c->geo_maxunion;
}

// Observation operator for (u, v) or, with yo_r, (u, v, rho) at each point:
// checks, staging through pinned memory, H and the ensemble statistics, and
// the global Gram dY dY^T the observation-space analysis gathers from.
int observe_impl(lbm_ctx* c, int npts, const int* ix, const int* iy, const double* yo_u,
                 const double* yo_v, const double* yo_r, double sigma_u, double sigma_v,
                 double sigma_r) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (npts < 1) return fail(c, LBM_EINVAL, "npts must be >= 1");
    if (!ix || !iy || !yo_u || !yo_v) return fail(c, LBM_EINVAL, "NULL observation array");
    if (!(sigma_u > 0.0) || !(sigma_v > 0.0) || !std::isfinite(sigma_u) || !std::isfinite(sigma_v))
        return fail(c, LBM_EINVAL, "sigma_u and sigma_v must be finite and > 0");
    if (yo_r && (!(sigma_r > 0.0) || !std::isfinite(sigma_r)))
        return fail(c, LBM_EINVAL, "sigma_rho must be finite and > 0");
    const int nvar = yo_r ? 3 : 2;
    if ((long long)npts * nvar > 65535) return fail(c, LBM_EINVAL, "too many observation points");
    for (int j = 0; j < npts; ++j) {
        if (ix[j] < 0 || ix[j] >= c->nx || iy[j] < 0 || iy[j] >= c->ny)
            return fail(c, LBM_EINVAL, "observation point %d outside the lattice", j);
        if (!std::isfinite(yo_u[j]) || !std::isfinite(yo_v[j]) || (yo_r && !std::isfinite(yo_r[j])))
            return fail(c, LBM_EINVAL, "observation %d is not finite", j);
    }
    const int nobs = nvar * npts;
    if (!c->obs_copied)
        CK(c, cudaEventCreateWithFlags(&c->obs_copied, cudaEventDisableTiming), "creating event");
    if (npts > c->pts_cap || nobs > c->nobs_cap) {
        CK(c, cudaStreamSynchronize(c->stream), "synchronising");
        free_obs(c);
        const size_t no = (size_t)nobs;
        CK(c, cudaMalloc(&c->ix, 2 * npts * sizeof(int)), "allocating obs");
        c->iy = c->ix + npts;
        CK(c, cudaMalloc(&c->yo, no * sizeof(double)), "allocating obs");
        CK(c, cudaMalloc(&c->dY, no * c->k * sizeof(double)), "allocating obs");
        CK(c, cudaMalloc(&c->d, no * sizeof(double)), "allocating obs");
        CK(c, cudaMalloc(&c->G, no * no * sizeof(double)), "allocating obs");
        if (is_fp32(c)) CK(c, cudaMalloc(&c->dY32, no * c->k * sizeof(float)), "allocating obs");
        CK(c, cudaMallocHost(&c->h_yo, no * sizeof(double)), "allocating pinned staging");
        CK(c, cudaMallocHost(&c->h_ixy, 2 * npts * sizeof(int)), "allocating pinned staging");
        c->pts_cap = npts;
        c->nobs_cap = nobs;
    }
    // The staging buffer may still be read by the previous copy.
    if (c->obs_pending) CK(c, cudaEventSynchronize(c->obs_copied), "waiting for staging copy");
    for (int j = 0; j < npts; ++j) {
        c->h_yo[nvar * j] = yo_u[j];
        c->h_yo[nvar * j + 1] = yo_v[j];
        if (yo_r) c->h_yo[nvar * j + 2] = yo_r[j];
        c->h_ixy[j] = ix[j];
        c->h_ixy[npts + j] = iy[j];
    }
    c->iy = c->ix + npts;
    CK(c, cudaMemcpyAsync(c->ix, c->h_ixy, 2 * npts * sizeof(int), cudaMemcpyHostToDevice, c->stream),
       "copy positions");
    CK(c, cudaMemcpyAsync(c->yo, c->h_yo, (size_t)nobs * sizeof(double), cudaMemcpyHostToDevice,
                          c->stream),
       "copy observations");
    CK(c, cudaEventRecord(c->obs_copied, c->stream), "recording event");
    c->obs_pending = true;
    CK(c, launch_observe(c->f[c->cur], is_fp32(c), c->nx, c->ny, c->k, npts, nvar, c->ix, c->iy,
                         c->yo, c->dY, c->d, c->stream),
       "launching observation operator");
    CK(c, launch_obs_gram(c->dY, nobs, c->k, c->G, c->stream), "launching observation Gram");
    if (c->nvar != nvar || c->geo_ix.size() != (size_t)npts ||
        !std::equal(ix, ix + npts, c->geo_ix.begin()) ||
        !std::equal(iy, iy + npts, c->geo_iy.begin())) {
        c->geo_ix.assign(ix, ix + npts);
        c->geo_iy.assign(iy, iy + npts);
        c->geo_dcut = -1.0;
        c->geo_maxunion = -1;
    }
    c->npts = npts;
    c->nvar = nvar;
    c->sigma_u = sigma_u;
    c->sigma_v = sigma_v;
    c->sigma_r = sigma_r;
    c->observed = true;
    return LBM_OK;
}

// Device buffers of one misfit/gradient call, allocated and released in
// stream order on the context stream.
struct StreamScratch {
    cudaStream_t s;
    std::vector<void*> bufs;
    explicit StreamScratch(cudaStream_t st) : s(st) {}
    cudaError_t get(void** p, size_t bytes) {
        *p = nullptr;
        cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, s);
        if (e == cudaSuccess) bufs.push_back(*p);
        return e;
    }
    ~StreamScratch() {
        for (void* b : bufs) cudaFreeAsync(b, s);
    }
};

// Forward sweep of the window with the misfit, and (want_grad) the reverse
// sweep: lambda_N from the last observation, then for every segment of
// checkpoint_every steps (last first) the forward states are recomputed from
// its checkpoint and the step adjoint runs back through them, adding the
// misfit derivative at each observation time.
int misfit_impl(lbm_ctx* c, const lbm_window* win, const double* w, double* J, double* grad_f0,
                double* grad_cs, double* dcs, int ptr_kind, bool want_grad) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!win) return fail(c, LBM_EINVAL, "window is NULL");
    if (!ptr_kind_ok(ptr_kind)) return fail(c, LBM_EINVAL, "bad ptr_kind");
    const int N = win->nsteps, E = win->obs_every, C = win->checkpoint_every, np = win->npts;
    if (N < 1 || E < 1 || C < 1 || np < 0)
        return fail(c, LBM_EINVAL, "nsteps, obs_every, checkpoint_every must be >= 1 and npts >= 0");
    const int nt = N / E;
    if (np > 0) {
        if (!win->ix || !win->iy || !win->yo_u || !win->yo_v)
            return fail(c, LBM_EINVAL, "NULL observation array");
        if (!(win->sigma_u > 0.0) || !(win->sigma_v > 0.0) || !std::isfinite(win->sigma_u) ||
            !std::isfinite(win->sigma_v))
            return fail(c, LBM_EINVAL, "sigma_u and sigma_v must be finite and > 0");
        for (int j = 0; j < np; ++j)
            if (win->ix[j] < 0 || win->ix[j] >= c->nx || win->iy[j] < 0 || win->iy[j] >= c->ny)
                return fail(c, LBM_EINVAL, "observation point %d outside the lattice", j);
        for (size_t i = 0; i < (size_t)nt * np; ++i)
            if (!std::isfinite(win->yo_u[i]) || !std::isfinite(win->yo_v[i]))
                return fail(c, LBM_EINVAL, "observation %zu is not finite", i);
    }
    // Host weights are checked here; device weights (ptr_kind device) are the
    // caller's responsibility.
    const bool w_dev = w && ptr_kind == LBM_PTR_DEVICE;
    if (w && !w_dev)
        for (int m = 0; m < c->k; ++m)
            if (!std::isfinite(w[m])) return fail(c, LBM_EINVAL, "weight %d is not finite", m);
    const int fp32 = is_fp32(c);
    const size_t S = state_elems(c) * elem_size(c);
    const int k = c->k;
    const LbmParams p{c->nx, c->ny, k, c->tau0, 18.0 * c->cs * c->cs, c->mu};
    auto step = [&](const void* in, void* out) {
        return fp32 ? launch_lbm_step_f32((const float*)in, (float*)out, (const float*)c->force, p,
                                          c->flags, c->stream)
                    : launch_lbm_step_f64((const double*)in, (double*)out,
                                          (const double*)c->force, p, c->flags, c->stream);
    };
    StreamScratch sc(c->stream);
    const int nck = want_grad ? (N + C - 1) / C : 0;
    const int nseg = want_grad ? std::min(C, N) - 1 : 0;
    std::vector<void*> ck(nck), seg(nseg);
    void *tmp[2], *lam[2] = {nullptr, nullptr};
    for (auto& b : ck) CK(c, sc.get(&b, S), "allocating checkpoints");
    for (auto& b : seg) CK(c, sc.get(&b, S), "allocating segment states");
    for (auto& b : tmp) CK(c, sc.get(&b, S), "allocating forecast states");
    if (want_grad)
        for (auto& b : lam) CK(c, sc.get(&b, S), "allocating adjoint states");
    const size_t nterm = (size_t)nt * np;
    void *d_pos, *d_yo, *d_w, *d_r, *d_J, *d_gcs;
    CK(c, sc.get(&d_pos, 2 * (size_t)np * sizeof(int)), "allocating observations");
    CK(c, sc.get(&d_yo, 2 * nterm * sizeof(double)), "allocating observations");
    CK(c, sc.get(&d_w, (size_t)k * sizeof(double)), "allocating weights");
    CK(c, sc.get(&d_r, nterm * k * sizeof(double)), "allocating misfit terms");
    CK(c, sc.get(&d_J, (size_t)k * sizeof(double)), "allocating misfit");
    CK(c, sc.get(&d_gcs, (size_t)k * sizeof(double)), "allocating C_s gradient");
    // Host staging (pageable; the call synchronises before returning).
    std::vector<int> hpos(2 * (size_t)np);
    std::vector<double> hyo(2 * nterm), hw((size_t)k, 1.0);
    for (int j = 0; j < np; ++j) {
        hpos[j] = win->ix[j];
        hpos[np + j] = win->iy[j];
    }
    for (size_t i = 0; i < nterm; ++i) {
        hyo[2 * i] = win->yo_u[i];
        hyo[2 * i + 1] = win->yo_v[i];
    }
    if (w && !w_dev) std::copy(w, w + k, hw.begin());
    const int* ixd = (const int*)d_pos;
    const int* iyd = ixd + np;
    const double* yod = (const double*)d_yo;
    if (np > 0) {
        CK(c, cudaMemcpyAsync(d_pos, hpos.data(), hpos.size() * sizeof(int), cudaMemcpyHostToDevice,
                              c->stream), "copy positions");
        if (nterm)
            CK(c, cudaMemcpyAsync(d_yo, hyo.data(), hyo.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, c->stream), "copy observations");
    }
    if (w_dev)
        CK(c, cudaMemcpyAsync(d_w, w, (size_t)k * sizeof(double), cudaMemcpyDeviceToDevice, c->stream),
           "copy weights");
    else
        CK(c, cudaMemcpyAsync(d_w, hw.data(), (size_t)k * sizeof(double), cudaMemcpyHostToDevice, c->stream),
           "copy weights");
    auto obs_time = [&](int t) { return (np > 0 && t >= 1 && t % E == 0 && t / E <= nt) ? t / E - 1 : -1; };

    // Forward sweep.
    const void* prev = c->f[c->cur];
    if (want_grad) {
        CK(c, cudaMemcpyAsync(ck[0], prev, S, cudaMemcpyDeviceToDevice, c->stream), "checkpoint");
    }
    for (int t = 1; t <= N; ++t) {
        void* out = (want_grad && t % C == 0 && t < N) ? ck[t / C] : tmp[t & 1];
        CK(c, step(prev, out), "launching LBM step");
        const int r = obs_time(t);
        if (r >= 0)
            CK(c, launch_misfit(out, fp32, c->nx, c->ny, k, np, ixd, iyd, yod + 2 * (size_t)r * np,
                                win->sigma_u, win->sigma_v, (double*)d_r + (size_t)r * np * k, c->stream),
               "launching misfit");
        prev = out;
    }
    if (nterm) {
        CK(c, launch_misfit_reduce((const double*)d_r, (int)nterm, k, (double*)d_J, c->stream),
           "launching misfit reduction");
    } else {
        CK(c, cudaMemsetAsync(d_J, 0, (size_t)k * sizeof(double), c->stream), "clearing misfit");
    }
    if (J) CK(c, cudaMemcpyAsync(J, d_J, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
              "copy misfit");

    if (want_grad) {
        // Reverse sweep.
        const void* fN = prev;
        int cur = 0;
        CK(c, cudaMemsetAsync(lam[cur], 0, S, c->stream), "clearing adjoint");
        CK(c, cudaMemsetAsync(d_gcs, 0, (size_t)k * sizeof(double), c->stream), "clearing C_s gradient");
        if (obs_time(N) >= 0)
            CK(c, launch_misfit_adjoint(fN, lam[cur], fp32, c->nx, c->ny, k, np, ixd, iyd,
                                        yod + 2 * (size_t)obs_time(N) * np, win->sigma_u, win->sigma_v,
                                        (const double*)d_w, c->stream),
               "launching misfit adjoint");
        std::vector<const void*> st((size_t)std::min(C, N));
        for (int sgi = nck - 1; sgi >= 0; --sgi) {
            const int t0 = sgi * C, t1 = std::min(t0 + C, N);
            st[0] = ck[sgi];
            for (int i = 1; i < t1 - t0; ++i) {
                CK(c, step(st[i - 1], seg[i - 1]), "launching LBM step");
                st[i] = seg[i - 1];
            }
            for (int t = t1 - 1; t >= t0; --t) {
                CK(c, launch_adjoint_step(st[t - t0], lam[cur], lam[cur ^ 1], c->force, fp32, p, c->cs,
                                          (double*)d_gcs, c->stream),
                   "launching adjoint step");
                cur ^= 1;
                const int r = obs_time(t);
                if (r >= 0)
                    CK(c, launch_misfit_adjoint(st[t - t0], lam[cur], fp32, c->nx, c->ny, k, np, ixd, iyd,
                                                yod + 2 * (size_t)r * np, win->sigma_u, win->sigma_v,
                                                (const double*)d_w, c->stream),
                       "launching misfit adjoint");
            }
        }
        const size_t n = state_elems(c);
        if (grad_f0) {
            if (ptr_kind == LBM_PTR_DEVICE) {
                CK(c, launch_widen(lam[cur], fp32, grad_f0, n, c->stream), "widening gradient");
            } else {
                int st2 = ensure_stage(c);
                if (st2) return st2;
                CK(c, launch_widen(lam[cur], fp32, c->stage, n, c->stream), "widening gradient");
                CK(c, cudaMemcpyAsync(grad_f0, c->stage, n * sizeof(double), cudaMemcpyDeviceToHost,
                                      c->stream), "copy gradient");
            }
        }
        if (grad_cs)
            CK(c, cudaMemcpyAsync(grad_cs, d_gcs, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost,
                                  c->stream), "copy C_s gradient");
        if (dcs) {
            // dF/dC_s = sum_m w_m dJ_m/dC_s, summed on the device in member order.
            void* d_dcs = dcs;
            if (ptr_kind != LBM_PTR_DEVICE) CK(c, sc.get(&d_dcs, sizeof(double)), "allocating C_s gradient sum");
            CK(c, launch_misfit_reduce((const double*)d_gcs, k, 1, (double*)d_dcs, c->stream),
               "launching C_s gradient sum");
            if (ptr_kind != LBM_PTR_DEVICE)
                CK(c, cudaMemcpyAsync(dcs, d_dcs, sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                   "copy C_s gradient sum");
        }
    }
    CK(c, cudaStreamSynchronize(c->stream), "synchronising");
    return read_flags(c);
}

// Host part of an analysis: argument checks, the largest local problem of
// the geometry (cached), scratch and the mixed path's second stream. No
// device work is queued, so it may precede a stream capture.
struct AnalysisPlan {
    double d_cut = 0.0, beta = 0.0;
    int nmax = 0, plmax = 0, prod = PROD_FP64;
    int run_len = 0, maxunion = 0;  // run_len > 0: the run analysis
};

// whole: size the run analysis' scratch for every run at once (batched
// launches) instead of chunks within a fixed budget.
int analyze_prepare(lbm_ctx* c, double d_cut, double beta, AnalysisPlan* plan, bool whole = false) {
    if (c->k < 2) return fail(c, LBM_EINVAL, "the analysis needs members >= 2");
    if (!(d_cut > 0.0) || !std::isfinite(d_cut)) return fail(c, LBM_EINVAL, "d_cut must be > 0");
    if (!(beta > 0.0) || !std::isfinite(beta)) return fail(c, LBM_EINVAL, "beta must be > 0");
    const int nmax = largest_local_problem(c, d_cut);
    const int plmax = c->geo_pmax;
    // The reduced-precision Gram pass serves ensemble-space points only.
    const int prod = c->geo_any_ens ? c->prod : PROD_NONE;
    // Every grid point in observation space and every run's union within
    // one warp: the run analysis (Jacobi warm-started along runs; in double
    // precision the FP64 Jacobi starts from the run's binary32 basis).
    int run_len = 0, maxunion = 0;
    if (c->run_len > 0 && !c->geo_any_ens) {
        maxunion = largest_run_union(c, d_cut, c->run_len);
        if (maxunion <= kRunMaxUnion) run_len = c->run_len;
    }
    const size_t scratch = run_len > 0 ? run_scratch_bytes(c->nx, c->ny, c->nvar * c->npts, run_len, maxunion, whole)
                                       : analyze_scratch_bytes(c->nx, c->ny, is_fp32(c), plmax, nmax, c->k, prod);
    if (scratch > c->ana_scratch_bytes) {
        CK(c, cudaStreamSynchronize(c->stream), "synchronising");
        cudaFree(c->ana_scratch);
        c->ana_scratch = nullptr;
        c->ana_scratch_bytes = 0;
        CK(c, cudaMalloc(&c->ana_scratch, scratch), "allocating analysis scratch");
        c->ana_scratch_bytes = scratch;
    }
    if ((is_fp32(c) || run_len > 0) && !c->aux_ready) {
        CK(c, cudaStreamCreateWithFlags(&c->aux.s2, cudaStreamNonBlocking), "creating stream");
        CK(c, cudaEventCreateWithFlags(&c->aux.start, cudaEventDisableTiming), "creating event");
        for (int b = 0; b < 2; ++b) {
            CK(c, cudaEventCreateWithFlags(&c->aux.jac_done[b], cudaEventDisableTiming), "creating event");
            CK(c, cudaEventCreateWithFlags(&c->aux.ref_done[b], cudaEventDisableTiming), "creating event");
        }
        c->aux_ready = true;
    }
    *plan = AnalysisPlan{d_cut, beta, nmax, plmax, prod, run_len, maxunion};
    return LBM_OK;
}

ObsParams obs_params(lbm_ctx* c, const AnalysisPlan& pl) {
    return ObsParams{c->npts, c->ix,    c->iy,   c->dY,       c->d,
                     c->G,    c->sigma_u, c->sigma_v, c->dY32, c->nvar,
                     c->sigma_r, pl.plmax, c->sweep_stats ? c->sweep_hist : nullptr};
}

// Device part: the analysis kernels on the context stream (capturable).
int analyze_launch(lbm_ctx* c, const AnalysisPlan& pl) {
    const ObsParams o = obs_params(c, pl);
    if (pl.run_len > 0) {
        const AnalyzeAux* aux = c->aux_ready ? &c->aux : nullptr;
        if (is_fp32(c))
            CK(c, launch_analyze_runs((float*)c->f[c->cur], c->nx, c->ny, c->k, o, pl.d_cut, pl.beta, pl.run_len,
                                      pl.maxunion, c->flags, c->ana_scratch, aux, c->run_pipe, c->stream),
               "launching analysis");
        else
            CK(c, launch_analyze_runs_fp64((double*)c->f[c->cur], c->nx, c->ny, c->k, o, pl.d_cut, pl.beta,
                                           pl.run_len, pl.maxunion, c->flags, c->ana_scratch, aux, c->run_pipe,
                                           c->stream),
               "launching analysis");
        return LBM_OK;
    }
    CK(c, launch_analyze(c->f[c->cur], is_fp32(c), c->nx, c->ny, c->k, o, pl.d_cut, pl.beta, pl.nmax,
                         pl.prod, c->run_len, c->flags, c->ana_scratch, c->aux_ready ? &c->aux : nullptr,
                         c->stream),
       "launching analysis");
    return LBM_OK;
}

// Observation step from a pinned host buffer of nvar * npts values, for
// positions already on the device (set by an earlier observe_impl): the copy,
// H and the Gram, all on the context stream (capturable).
int observe_from_pinned(lbm_ctx* c, const double* h_yo) {
    const int nobs = c->nvar * c->npts;
    CK(c, cudaMemcpyAsync(c->yo, h_yo, (size_t)nobs * sizeof(double), cudaMemcpyHostToDevice, c->stream),
       "copy observations");
    CK(c, launch_observe(c->f[c->cur], is_fp32(c), c->nx, c->ny, c->k, c->npts, c->nvar, c->ix, c->iy,
                         c->yo, c->dY, c->d, c->stream),
       "launching observation operator");
    CK(c, launch_obs_gram(c->dY, nobs, c->k, c->G, c->stream), "launching observation Gram");
    return LBM_OK;
}

}  // namespace

namespace lbmgpu {
// Error message of a context-free entry point, read by lbm_last_error(NULL).
void set_context_free_error(const char* msg) { snprintf(g_init_err, sizeof g_init_err, "%s", msg); }
}  // namespace lbmgpu

extern "C" {

int lbm_init(const lbm_config* cfg, const double* f0, const double* force, int ptr_kind,
             lbm_ctx** out) {
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, LBM_EINVAL, "cfg is NULL");
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->members < 1)
        return fail(nullptr, LBM_EINVAL, "nx, ny and members must be >= 1");
    if (!((size_t)cfg->nx * cfg->ny < (1ull << 31)))
        return fail(nullptr, LBM_EINVAL, "nx * ny must be below 2^31");
    if (!(cfg->tau0 > 0.5) || !std::isfinite(cfg->tau0))
        return fail(nullptr, LBM_EINVAL, "tau0 must be finite and > 0.5");
    if (!(cfg->cs_smag >= 0.0) || !std::isfinite(cfg->cs_smag))
        return fail(nullptr, LBM_EINVAL, "cs_smag must be finite and >= 0");
    if (!(cfg->mu >= 0.0) || !std::isfinite(cfg->mu))
        return fail(nullptr, LBM_EINVAL, "mu must be finite and >= 0");
    if (cfg->precision != LBM_FP64 && cfg->precision != LBM_MIXED)
        return fail(nullptr, LBM_EINVAL, "precision must be LBM_FP64 or LBM_MIXED");
    if ((f0 || force) && !ptr_kind_ok(ptr_kind))
        return fail(nullptr, LBM_EINVAL, "ptr_kind must be LBM_PTR_HOST or LBM_PTR_DEVICE");

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    c->nx = cfg->nx;
    c->ny = cfg->ny;
    c->k = cfg->members;
    c->tau0 = cfg->tau0;
    c->cs = cfg->cs_smag;
    c->mu = cfg->mu;
    c->precision = cfg->precision;
    if (c->precision == LBM_MIXED) c->prod = PROD_DF32;
    c->stream = (cudaStream_t)cfg->stream;

    int st = LBM_OK;
    auto bail = [&](int code) {
        snprintf(g_init_err, sizeof g_init_err, "%s", c->err);
        lbm_destroy(c);
        return code;
    };
    const size_t bytes = state_elems(c) * elem_size(c);
    for (int b = 0; b < 2; ++b) {
        cudaError_t e = cudaMalloc(&c->f[b], bytes);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "allocating state"));
    }
    cudaError_t e = cudaMalloc(&c->force, (size_t)2 * c->nx * c->ny * elem_size(c));
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "allocating force"));
    e = cudaMalloc(&c->flags, sizeof(int));
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "allocating flags"));
    e = cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "clearing flags"));

    // Forcing field.
    const size_t nf = (size_t)2 * c->nx * c->ny;
    if (force) {
        double* tmp = nullptr;
        e = cudaMalloc(&tmp, nf * sizeof(double));
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "allocating force staging"));
        st = copy_in(c, tmp, force, nf, ptr_kind);
        if (st == LBM_OK) {
            e = launch_store_force(c->force, is_fp32(c), tmp, nf, c->stream);
            if (e != cudaSuccess) st = cuda_fail(c, e, "converting force");
        }
        cudaError_t e2 = cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
        if (st != LBM_OK) return bail(st);
        if (e2 != cudaSuccess) return bail(cuda_fail(c, e2, "synchronising"));
    } else {
        e = cudaMemsetAsync(c->force, 0, nf * elem_size(c), c->stream);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "clearing force"));
    }

    // Initial state.
    if (f0) {
        st = lbm_set_f(c, f0, ptr_kind);
    } else {
        e = launch_set_equilibrium(c->f[0], is_fp32(c), c->nx, c->ny, c->k, nullptr, nullptr,
                                   nullptr, c->stream);
        if (e != cudaSuccess) st = cuda_fail(c, e, "initialising state");
    }
    if (st != LBM_OK) return bail(st);
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "synchronising"));
    snprintf(c->err, sizeof c->err, "no error");
    *out = c;
    return LBM_OK;
}

int lbm_set_equilibrium(lbm_ctx* c, const double* rho, const double* u, const double* v,
                        int ptr_kind) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!ptr_kind_ok(ptr_kind)) return fail(c, LBM_EINVAL, "bad ptr_kind");
    if (!u || !v) return fail(c, LBM_EINVAL, "u and v are required");
    const size_t n = cell_elems(c);
    const double *dr = rho, *du = u, *dv = v;
    if (ptr_kind == LBM_PTR_HOST) {
        int st = ensure_stage(c);
        if (st) return st;
        double* s = c->stage;
        if (rho) {
            if ((st = copy_in(c, s, rho, n, ptr_kind))) return st;
            dr = s;
        }
        if ((st = copy_in(c, s + n, u, n, ptr_kind))) return st;
        if ((st = copy_in(c, s + 2 * n, v, n, ptr_kind))) return st;
        du = s + n;
        dv = s + 2 * n;
    }
    CK(c, launch_set_equilibrium(c->f[c->cur], is_fp32(c), c->nx, c->ny, c->k, dr, du, dv,
                                 c->stream),
       "launching equilibrium");
    if (ptr_kind == LBM_PTR_HOST) CK(c, cudaStreamSynchronize(c->stream), "synchronising");
    c->observed = false;
    return LBM_OK;
}

int lbm_forecast(lbm_ctx* c, int nsteps) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (nsteps < 0) return fail(c, LBM_EINVAL, "nsteps must be >= 0");
    LbmParams p{c->nx, c->ny, c->k, c->tau0, 18.0 * c->cs * c->cs, c->mu};
    for (int s = 0; s < nsteps; ++s) {
        cudaError_t e;
        if (is_fp32(c))
            e = launch_lbm_step_f32((const float*)c->f[c->cur], (float*)c->f[c->cur ^ 1],
                                    (const float*)c->force, p, c->flags, c->stream);
        else
            e = launch_lbm_step_f64((const double*)c->f[c->cur], (double*)c->f[c->cur ^ 1],
                                    (const double*)c->force, p, c->flags, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "launching LBM step");
        c->cur ^= 1;
    }
    if (nsteps > 0) c->observed = false;
    return LBM_OK;
}

int lbm_moments(lbm_ctx* c, double* rho, double* u, double* v, int ptr_kind) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!ptr_kind_ok(ptr_kind)) return fail(c, LBM_EINVAL, "bad ptr_kind");
    const size_t n = cell_elems(c);
    if (ptr_kind == LBM_PTR_DEVICE) {
        CK(c, launch_moments(c->f[c->cur], is_fp32(c), c->nx, c->ny, c->k, rho, u, v, c->flags,
                             c->stream),
           "launching moments");
        return LBM_OK;
    }
    int st = ensure_stage(c);
    if (st) return st;
    double* s = c->stage;
    CK(c, launch_moments(c->f[c->cur], is_fp32(c), c->nx, c->ny, c->k, rho ? s : nullptr,
                         u ? s + n : nullptr, v ? s + 2 * n : nullptr, c->flags, c->stream),
       "launching moments");
    if (rho) CK(c, cudaMemcpyAsync(rho, s, n * 8, cudaMemcpyDeviceToHost, c->stream), "copy rho");
    if (u) CK(c, cudaMemcpyAsync(u, s + n, n * 8, cudaMemcpyDeviceToHost, c->stream), "copy u");
    if (v) CK(c, cudaMemcpyAsync(v, s + 2 * n, n * 8, cudaMemcpyDeviceToHost, c->stream), "copy v");
    return read_flags(c);
}

int lbm_mean_velocity(lbm_ctx* c, double* u, double* v, int ptr_kind) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!ptr_kind_ok(ptr_kind)) return fail(c, LBM_EINVAL, "bad ptr_kind");
    const size_t n = (size_t)c->nx * c->ny;
    if (ptr_kind == LBM_PTR_DEVICE) {
        CK(c, launch_mean_velocity(c->f[c->cur], is_fp32(c), c->nx, c->ny, c->k, u, v, c->flags,
                                   c->stream),
           "launching mean velocity");
        return LBM_OK;
    }
    int st = ensure_stage(c);
    if (st) return st;
    double* s = c->stage;
    CK(c, launch_mean_velocity(c->f[c->cur], is_fp32(c), c->nx, c->ny, c->k, u ? s : nullptr,
                               v ? s + n : nullptr, c->flags, c->stream),
       "launching mean velocity");
    if (u) CK(c, cudaMemcpyAsync(u, s, n * 8, cudaMemcpyDeviceToHost, c->stream), "copy u");
    if (v) CK(c, cudaMemcpyAsync(v, s + n, n * 8, cudaMemcpyDeviceToHost, c->stream), "copy v");
    return read_flags(c);
}

int lbm_velocity_rmse(lbm_ctx* c, lbm_ctx* truth, double* rmse, int ptr_kind) {
    if (!c || !truth) return fail(c, LBM_EINVAL, "ctx is NULL");
    if (!rmse) return fail(c, LBM_EINVAL, "rmse is NULL");
    if (!ptr_kind_ok(ptr_kind)) return fail(c, LBM_EINVAL, "bad ptr_kind");
    if (truth->nx != c->nx || truth->ny != c->ny) return fail(c, LBM_EINVAL, "the two lattices differ");
    const size_t n = (size_t)c->nx * c->ny;
    // The truth's state as queued on its own stream.
    if (truth->stream != c->stream) {
        cudaEvent_t ev;
        CK(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "creating event");
        cudaError_t e = cudaEventRecord(ev, truth->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, ev, 0);
        cudaEventDestroy(ev);
        CK(c, e, "ordering the two streams");
    }
    StreamScratch sc(c->stream);
    void* buf;
    CK(c, sc.get(&buf, (4 * n + rmse_work_doubles() + 1) * sizeof(double)), "allocating RMSE scratch");
    double* b = (double*)buf;
    double* out = ptr_kind == LBM_PTR_DEVICE ? rmse : b + 4 * n + rmse_work_doubles();
    CK(c, launch_mean_velocity(c->f[c->cur], is_fp32(c), c->nx, c->ny, c->k, b, b + n, c->flags, c->stream),
       "launching mean velocity");
    CK(c, launch_mean_velocity(truth->f[truth->cur], is_fp32(truth), truth->nx, truth->ny, truth->k, b + 2 * n,
                               b + 3 * n, truth->flags, c->stream),
       "launching mean velocity");
    CK(c, launch_velocity_rmse(b, b + n, b + 2 * n, b + 3 * n, n, b + 4 * n, out, c->stream), "launching RMSE");
    if (ptr_kind == LBM_PTR_DEVICE) return LBM_OK;
    CK(c, cudaMemcpyAsync(rmse, out, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy RMSE");
    return read_flags(c);
}

int lbm_energy_spectrum(lbm_ctx* c, double* E, int nshells, int ptr_kind) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!ptr_kind_ok(ptr_kind)) return fail(c, LBM_EINVAL, "bad ptr_kind");
    if (!E) return fail(c, LBM_EINVAL, "E is NULL");
    if (nshells < 1) return fail(c, LBM_EINVAL, "nshells must be >= 1");
    // Shells past floor(hypot(nx/2, ny/2) + 1/2) hold no wavenumber.
    const int all = (int)std::floor(std::hypot((double)(c->nx / 2), (double)(c->ny / 2)) + 0.5) + 1;
    const int nsh = nshells < all ? nshells : all;
    const size_t work = spectrum_work_bytes(c->nx, c->ny, c->k, nsh);
    const size_t out = ptr_kind == LBM_PTR_HOST ? (size_t)nshells * sizeof(double) : 0;
    void* buf = nullptr;
    // Stream-ordered scratch: the diagnostic is occasional and its buffers
    // (about 1 KiB per member and lattice row) are returned right after.
    CK(c, cudaMallocAsync(&buf, work + out, c->stream), "allocating spectrum scratch");
    double* Ed = ptr_kind == LBM_PTR_HOST
                     ? reinterpret_cast<double*>(static_cast<unsigned char*>(buf) + work)
                     : E;
    cudaError_t e = launch_energy_spectrum(c->f[c->cur], is_fp32(c), c->nx, c->ny, c->k, Ed,
                                           nsh, buf, c->flags, c->stream);
    if (e == cudaSuccess && nshells > nsh)
        e = cudaMemsetAsync(Ed + nsh, 0, (size_t)(nshells - nsh) * sizeof(double), c->stream);
    if (e == cudaSuccess && ptr_kind == LBM_PTR_HOST)
        e = cudaMemcpyAsync(E, Ed, out, cudaMemcpyDeviceToHost, c->stream);
    const cudaError_t e2 = cudaFreeAsync(buf, c->stream);
    if (e == cudaErrorInvalidValue)
        return fail(c, LBM_EINVAL, "lattice too large for the spectrum diagnostic's shared memory");
    CK(c, e, "launching the energy spectrum");
    CK(c, e2, "freeing spectrum scratch");
    return ptr_kind == LBM_PTR_HOST ? read_flags(c) : LBM_OK;
}

int letkf_set_products(lbm_ctx* c, int mode) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (mode < LBM_PROD_FP64 || mode > LBM_PROD_DF32) return fail(c, LBM_EINVAL, "unknown product mode %d", mode);
    if (mode != LBM_PROD_FP64 && !is_fp32(c))
        return fail(c, LBM_EINVAL, "product modes other than FP64 need a mixed-precision context");
    c->prod = mode;
    return LBM_OK;
}

int letkf_set_run_pipeline(lbm_ctx* c, int runs) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (runs < 0 || runs > (1 << 24)) return fail(c, LBM_EINVAL, "runs must be in [0, 2^24]");
    c->run_pipe = runs;
    return LBM_OK;
}

int letkf_set_run_length(lbm_ctx* c, int run_len) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (run_len < 0 || run_len > 4096) return fail(c, LBM_EINVAL, "run_len must be in [0, 4096]");
    c->run_len = run_len;
    return LBM_OK;
}

int letkf_sweep_stats(lbm_ctx* c, int enable, int* hist) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!c->sweep_hist) {
        CK(c, cudaMalloc(&c->sweep_hist, 32 * sizeof(int)), "allocating sweep histogram");
        CK(c, cudaMemsetAsync(c->sweep_hist, 0, 32 * sizeof(int), c->stream), "clearing sweep histogram");
    }
    if (hist) {
        CK(c, cudaMemcpyAsync(hist, c->sweep_hist, 32 * sizeof(int), cudaMemcpyDeviceToHost, c->stream),
           "reading sweep histogram");
        CK(c, cudaMemsetAsync(c->sweep_hist, 0, 32 * sizeof(int), c->stream), "clearing sweep histogram");
        CK(c, cudaStreamSynchronize(c->stream), "synchronising");
    }
    c->sweep_stats = enable != 0;
    return LBM_OK;
}

int lbm_set_closure(lbm_ctx* c, double cs_smag) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!(cs_smag >= 0.0) || !std::isfinite(cs_smag)) return fail(c, LBM_EINVAL, "cs_smag must be finite and >= 0");
    c->cs = cs_smag;
    return LBM_OK;
}

int lbm_misfit(lbm_ctx* c, const lbm_window* win, double* J) {
    if (c && !J) return fail(c, LBM_EINVAL, "J is NULL");
    return misfit_impl(c, win, nullptr, J, nullptr, nullptr, nullptr, LBM_PTR_HOST, false);
}

int lbm_misfit_gradient(lbm_ctx* c, const lbm_window* win, const double* w, double* J,
                        double* grad_f0, double* grad_cs, double* dcs, int ptr_kind) {
    return misfit_impl(c, win, w, J, grad_f0, grad_cs, dcs, ptr_kind, true);
}

int letkf_observe(lbm_ctx* c, int npts, const int* ix, const int* iy, const double* yo_u,
                  const double* yo_v, double sigma_u, double sigma_v) {
    return observe_impl(c, npts, ix, iy, yo_u, yo_v, nullptr, sigma_u, sigma_v, 1.0);
}

int letkf_observe_rho(lbm_ctx* c, int npts, const int* ix, const int* iy, const double* yo_u,
                      const double* yo_v, const double* yo_rho, double sigma_u, double sigma_v,
                      double sigma_rho) {
    if (c && !yo_rho) return fail(c, LBM_EINVAL, "NULL observation array");
    return observe_impl(c, npts, ix, iy, yo_u, yo_v, yo_rho, sigma_u, sigma_v, sigma_rho);
}

int letkf_analyze(lbm_ctx* c, double d_cut, double beta) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!c->observed) return fail(c, LBM_EINVAL, "letkf_observe must precede letkf_analyze");
    AnalysisPlan plan;
    int st = analyze_prepare(c, d_cut, beta, &plan);
    if (st) return st;
    st = analyze_launch(c, plan);
    if (st) return st;
    c->observed = false;
    return LBM_OK;
}

int letkf_probe_transform(lbm_ctx* c, double d_cut, double beta, int npoints, const int* cells, double* T,
                          int ptr_kind) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!is_fp32(c)) return fail(c, LBM_EINVAL, "the transform probe covers the mixed-precision analysis");
    if (!c->observed) return fail(c, LBM_EINVAL, "letkf_observe must precede letkf_probe_transform");
    if (npoints < 1 || npoints > 4096) return fail(c, LBM_EINVAL, "npoints must be in [1, 4096]");
    if (!cells || !T) return fail(c, LBM_EINVAL, "NULL argument");
    if (!ptr_kind_ok(ptr_kind)) return fail(c, LBM_EINVAL, "bad ptr_kind");
    const long long ncell = (long long)c->nx * c->ny;
    for (int i = 0; i < npoints; ++i)
        if (cells[i] < 0 || cells[i] >= ncell) return fail(c, LBM_EINVAL, "grid point %d outside the lattice", i);
    AnalysisPlan plan;
    int st = analyze_prepare(c, d_cut, beta, &plan);
    if (st) return st;
    if (plan.run_len == 0)
        return fail(c, LBM_EINVAL,
                    "the transform probe needs the run analysis (run length > 0, every grid point with p < members, "
                    "unions of at most 32 scalars)");
    StreamScratch sc(c->stream);
    void *d_cells, *d_work, *d_T = T;
    const size_t tbytes = (size_t)npoints * c->k * c->k * sizeof(double);
    CK(c, sc.get(&d_cells, (size_t)npoints * sizeof(int)), "allocating probe points");
    CK(c, sc.get(&d_work, probe_work_bytes(npoints, plan.maxunion, c->k)), "allocating probe scratch");
    if (ptr_kind == LBM_PTR_HOST) CK(c, sc.get(&d_T, tbytes), "allocating probe output");
    CK(c, cudaMemcpyAsync(d_cells, cells, (size_t)npoints * sizeof(int), cudaMemcpyHostToDevice, c->stream),
       "copy probe points");
    ObsParams o{c->npts, c->ix, c->iy, c->dY, c->d, c->G, c->sigma_u, c->sigma_v, c->dY32,
                c->nvar, c->sigma_r, plan.plmax, nullptr};
    CK(c, launch_probe_runs((float*)c->f[c->cur], c->nx, c->ny, c->k, o, plan.d_cut, plan.beta, plan.run_len,
                            plan.maxunion, c->flags, c->ana_scratch, (const int*)d_cells, npoints, (double*)d_T,
                            (double*)d_work, c->stream),
       "launching the transform probe");
    if (ptr_kind == LBM_PTR_HOST)
        CK(c, cudaMemcpyAsync(T, d_T, tbytes, cudaMemcpyDeviceToHost, c->stream), "copy probe output");
    CK(c, cudaStreamSynchronize(c->stream), "synchronising");
    return read_flags(c);
}

int lbm_nudge(lbm_ctx* c, int nobs_x, int nobs_y, const double* rho_o, const double* u_o,
              const double* v_o, double gamma) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (nobs_x < 1 || nobs_y < 1 || c->nx % nobs_x != 0 || c->ny % nobs_y != 0)
        return fail(c, LBM_EINVAL, "nx, ny must be multiples of nobs_x, nobs_y");
    if (!rho_o || !u_o || !v_o) return fail(c, LBM_EINVAL, "NULL observation field");
    if (!(gamma >= 0.0 && gamma <= 1.0)) return fail(c, LBM_EINVAL, "gamma must be in [0, 1]");
    const size_t no = (size_t)nobs_x * nobs_y;
    for (size_t i = 0; i < no; ++i)
        if (!std::isfinite(rho_o[i]) || !std::isfinite(u_o[i]) || !std::isfinite(v_o[i]) || !(rho_o[i] > 0.0))
            return fail(c, LBM_EINVAL, "observation %zu is not finite or has rho <= 0", i);
    if (3 * no > c->nudge_cap) {
        CK(c, cudaStreamSynchronize(c->stream), "synchronising");
        cudaFree(c->nudge_obs);
        c->nudge_obs = nullptr;
        c->nudge_cap = 0;
        CK(c, cudaMalloc(&c->nudge_obs, 3 * no * sizeof(double)), "allocating nudging observations");
        c->nudge_cap = 3 * no;
    }
    // Copies from pageable memory are staged before the call returns.
    CK(c, cudaMemcpyAsync(c->nudge_obs, rho_o, no * 8, cudaMemcpyHostToDevice, c->stream), "copy rho");
    CK(c, cudaMemcpyAsync(c->nudge_obs + no, u_o, no * 8, cudaMemcpyHostToDevice, c->stream), "copy u");
    CK(c, cudaMemcpyAsync(c->nudge_obs + 2 * no, v_o, no * 8, cudaMemcpyHostToDevice, c->stream), "copy v");
    CK(c, launch_nudge(c->f[c->cur], is_fp32(c), c->nx, c->ny, c->k, nobs_x, nobs_y, c->nudge_obs,
                       gamma, c->stream),
       "launching nudging");
    c->observed = false;
    return LBM_OK;
}

int lbm_get_f(lbm_ctx* c, double* f, int ptr_kind) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!f) return fail(c, LBM_EINVAL, "f is NULL");
    if (!ptr_kind_ok(ptr_kind)) return fail(c, LBM_EINVAL, "bad ptr_kind");
    const size_t n = state_elems(c);
    if (!is_fp32(c)) {
        CK(c, cudaMemcpyAsync(f, c->f[c->cur], n * sizeof(double),
                              ptr_kind == LBM_PTR_HOST ? cudaMemcpyDeviceToHost
                                                       : cudaMemcpyDeviceToDevice,
                              c->stream),
           "copying state out");
    } else if (ptr_kind == LBM_PTR_DEVICE) {
        CK(c, launch_load_f(c->f[c->cur], 1, f, n, c->stream), "converting state");
    } else {
        int st = ensure_stage(c);
        if (st) return st;
        CK(c, launch_load_f(c->f[c->cur], 1, c->stage, n, c->stream), "converting state");
        CK(c, cudaMemcpyAsync(f, c->stage, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
           "copying state out");
    }
    if (ptr_kind == LBM_PTR_HOST) return read_flags(c);
    return LBM_OK;
}

int lbm_set_f(lbm_ctx* c, const double* f, int ptr_kind) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!f) return fail(c, LBM_EINVAL, "f is NULL");
    if (!ptr_kind_ok(ptr_kind)) return fail(c, LBM_EINVAL, "bad ptr_kind");
    const size_t n = state_elems(c);
    if (!is_fp32(c)) {
        CK(c, cudaMemcpyAsync(c->f[c->cur], f, n * sizeof(double),
                              ptr_kind == LBM_PTR_HOST ? cudaMemcpyHostToDevice
                                                       : cudaMemcpyDeviceToDevice,
                              c->stream),
           "copying state in");
    } else {
        const double* src = f;
        if (ptr_kind == LBM_PTR_HOST) {
            int st = ensure_stage(c);
            if (st) return st;
            if ((st = copy_in(c, c->stage, f, n, ptr_kind))) return st;
            src = c->stage;
        }
        CK(c, launch_store_f(c->f[c->cur], 1, src, n, c->stream), "converting state");
    }
    if (ptr_kind == LBM_PTR_HOST) CK(c, cudaStreamSynchronize(c->stream), "synchronising");
    c->observed = false;
    return LBM_OK;
}

int lbm_sync(lbm_ctx* c) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    return read_flags(c);
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err : g_init_err; }

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    cudaFree(c->f[0]);
    cudaFree(c->f[1]);
    cudaFree(c->force);
    cudaFree(c->flags);
    cudaFree(c->stage);
    cudaFree(c->ana_scratch);
    cudaFree(c->nudge_obs);
    cudaFree(c->sweep_hist);
    if (c->aux_ready) {
        cudaStreamSynchronize(c->aux.s2);
        cudaEventDestroy(c->aux.start);
        for (int b = 0; b < 2; ++b) {
            cudaEventDestroy(c->aux.jac_done[b]);
            cudaEventDestroy(c->aux.ref_done[b]);
        }
        cudaStreamDestroy(c->aux.s2);
    }
    free_obs(c);
    if (c->obs_copied) cudaEventDestroy(c->obs_copied);
    delete c;
}

}  // extern "C"

// ---- Batches of independent experiments ------------------------------------

struct lbm_batch {
    std::vector<lbm_ctx*> ctx;
    cudaStream_t stream = nullptr;
    int fp32 = 0;
    MultiExp* ex_dev = nullptr;   // device copy of the experiment table
    std::vector<MultiExp> ex;
    long long total = 0;
    unsigned* bar = nullptr;      // grid barrier words
    int* status = nullptr;        // barrier timeout flag (device)
    long long spin_limit = kBarrierSpins;  // bound of each grid-barrier wait
    unsigned absent = 0;          // arrivals that never come (timeout path)
    int threads = 256, blocks = 0;
    bool tuned = false;
    // Cycle state: fixed observation positions per experiment, pinned
    // staging of the observed values, the captured cycle graph.
    std::vector<double*> h_yo;
    std::vector<int> npts;
    std::vector<std::vector<int>> pos;
    int cycles = 0;
    int graph_steps = -1;
    std::vector<double> graph_dcut, graph_beta, graph_sigma;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    cudaStream_t cap = nullptr;   // capture stream (the shared stream may be the legacy one)
    bool launched = false;
    char err[512] = {0};
};

namespace {

int bfail(lbm_batch* b, int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b ? b->err : g_init_err, sizeof b->err, fmt, ap);
    va_end(ap);
    return code;
}

#define BK(b, call, what)                                                       \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess)                                                  \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", \
                         what, cudaGetErrorString(e_));                         \
    } while (0)

// Experiment table from the contexts' current buffers and parameters.
void batch_table(lbm_batch* b) {
    b->ex.clear();
    long long off = 0;
    for (lbm_ctx* c : b->ctx) {
        MultiExp e{};
        e.f[0] = c->f[0];
        e.f[1] = c->f[1];
        e.force = c->force;
        e.flags = c->flags;
        e.nx = c->nx;
        e.ny = c->ny;
        e.k = c->k;
        e.V = b->fp32 ? (c->k % 4 == 0 ? 4 : (c->k % 2 == 0 ? 2 : 1)) : (c->k % 2 == 0 ? 2 : 1);
        e.cur = c->cur;
        e.tau0 = c->tau0;
        e.cs18 = 18.0 * c->cs * c->cs;
        e.mu = c->mu;
        e.offset = off;
        e.items = (long long)c->nx * c->ny * (c->k / e.V);
        off += e.items;
        b->ex.push_back(e);
    }
    b->total = off;
}

int batch_forecast_impl(lbm_batch* b, int nsteps) {
    batch_table(b);
    BK(b, cudaMemcpyAsync(b->ex_dev, b->ex.data(), b->ex.size() * sizeof(MultiExp), cudaMemcpyHostToDevice,
                          b->stream),
       "copy experiment table");
    BK(b, launch_lbm_multi(b->ex_dev, (int)b->ex.size(), b->total, nsteps, b->fp32, b->blocks, b->threads,
                           b->bar, b->status, b->spin_limit, b->absent, b->stream),
       "launching persistent forecast");
    for (lbm_ctx* c : b->ctx) {
        c->cur = (c->cur + nsteps) & 1;
        c->observed = false;
    }
    return LBM_OK;
}

// The analyses of a batch on stream s: the experiments on the run path
// marked batched (the default; the analysis autotuner may unmark a size
// class) in batched launches (kernel J over all their runs, then kernel F
// over all their grid points, per size class), the others one by one. The
// plans come from analyze_prepare(..., whole = true).
int batch_analyze(lbm_batch* b, const std::vector<AnalysisPlan>& plans, const std::vector<int>& which,
                  cudaStream_t s) {
    std::vector<RunItem> items;
    for (int i : which) {
        lbm_ctx* c = b->ctx[i];
        const AnalysisPlan& pl = plans[i];
        if (pl.run_len > 0 && c->run_batched) {
            const bool f32 = is_fp32(c);
            items.push_back(RunItem{f32 ? (float*)c->f[c->cur] : nullptr, f32 ? nullptr : (double*)c->f[c->cur],
                                    c->nx, c->ny, c->k, pl.run_len, pl.maxunion, obs_params(c, pl), pl.d_cut,
                                    pl.beta, c->flags, c->ana_scratch});
        } else {
            const cudaStream_t own = c->stream;
            c->stream = s;
            const int st = analyze_launch(c, pl);
            c->stream = own;
            if (st) return bfail(b, st, "experiment %d: %s", i, c->err);
        }
    }
    if (!items.empty())
        BK(b, launch_analyze_runs_batch(items.data(), (int)items.size(), s), "launching batched run analysis");
    return LBM_OK;
}

std::vector<int> all_experiments(const lbm_batch* b) {
    std::vector<int> v(b->ctx.size());
    for (size_t i = 0; i < v.size(); ++i) v[i] = (int)i;
    return v;
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_ctx* const* ctxs, int n, lbm_batch** out) {
    if (!out) return bfail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ctxs || n < 1 || n > kMaxMultiExp) return bfail(nullptr, LBM_EINVAL, "need 1..%d contexts", kMaxMultiExp);
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return bfail(nullptr, LBM_EINVAL, "context %d is NULL", i);
        if (ctxs[i]->stream != ctxs[0]->stream)
            return bfail(nullptr, LBM_EINVAL, "the contexts of a batch must share one stream");
        if (is_fp32(ctxs[i]) != is_fp32(ctxs[0]))
            return bfail(nullptr, LBM_EINVAL, "the contexts of a batch must share one precision");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return bfail(nullptr, LBM_EINVAL, "context %d appears twice", i);
    }
    lbm_batch* b = new (std::nothrow) lbm_batch;
    if (!b) return bfail(nullptr, LBM_ENOMEM, "out of host memory");
    b->ctx.assign(ctxs, ctxs + n);
    b->stream = ctxs[0]->stream;
    b->fp32 = is_fp32(ctxs[0]);
    auto bail = [&](int code) {
        lbm_batch_destroy(b);
        return code;
    };
    cudaError_t e = cudaMalloc(&b->ex_dev, kMaxMultiExp * sizeof(MultiExp));
    if (e == cudaSuccess) e = cudaMalloc(&b->bar, 4 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&b->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, sizeof(int), b->stream);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e != cudaSuccess)
        return bail(bfail(nullptr, LBM_ECUDA, "creating batch: %s", cudaGetErrorString(e)));
    b->blocks = lbm_multi_max_blocks(b->fp32, b->threads);
    if (b->blocks < 1) return bail(bfail(nullptr, LBM_ECUDA, "no co-resident grid for the persistent kernel"));
    b->h_yo.assign(n, nullptr);
    b->npts.assign(n, 0);
    b->pos.assign(n, std::vector<int>());
    *out = b;
    return LBM_OK;
}

int lbm_batch_forecast(lbm_batch* b, int nsteps) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (nsteps < 0) return bfail(b, LBM_EINVAL, "nsteps must be >= 0");
    if (nsteps == 0) return LBM_OK;
    return batch_forecast_impl(b, nsteps);
}

int lbm_batch_autotune(lbm_batch* b, int* threads, int* blocks) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    // Candidates: block size x co-resident blocks per SM, each timed on one
    // step from the current states into the spare buffers (the current
    // states are not changed), best of three runs.
    int dev = 0, sms = 0;
    BK(b, cudaGetDevice(&dev), "querying device");
    BK(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "querying SMs");
    batch_table(b);
    BK(b, cudaMemcpyAsync(b->ex_dev, b->ex.data(), b->ex.size() * sizeof(MultiExp), cudaMemcpyHostToDevice,
                          b->stream),
       "copy experiment table");
    cudaEvent_t t0, t1;
    BK(b, cudaEventCreate(&t0), "creating event");
    BK(b, cudaEventCreate(&t1), "creating event");
    float best = 1e30f;
    int bt = b->threads, bb = b->blocks;
    const int cand_t[] = {128, 256, 512};  // the kernel's launch bound is 512
    for (int th : cand_t) {
        const int maxb = lbm_multi_max_blocks(b->fp32, th);
        if (maxb < 1) continue;
        const int per = maxb / sms;
        for (int q = 1; q <= per; ++q) {
            const int nb = q * sms;
            float tbest = 1e30f;
            for (int r = 0; r < 3; ++r) {
                cudaEventRecord(t0, b->stream);
                cudaError_t e = launch_lbm_multi(b->ex_dev, (int)b->ex.size(), b->total, 1, b->fp32, nb, th,
                                                 b->bar, b->status, b->spin_limit, b->absent, b->stream);
                cudaEventRecord(t1, b->stream);
                if (e != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess) {
                    cudaEventDestroy(t0);
                    cudaEventDestroy(t1);
                    return bfail(b, LBM_ECUDA, "autotune launch: %s", cudaGetErrorString(e));
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, t0, t1);
                if (ms < tbest) tbest = ms;
            }
            if (tbest < best) {
                best = tbest;
                bt = th;
                bb = nb;
            }
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    b->threads = bt;
    b->blocks = bb;
    b->tuned = true;
    if (threads) *threads = bt;
    if (blocks) *blocks = bb;
    return LBM_OK;
}

int lbm_batch_autotune_analysis(lbm_batch* b, const double* d_cut, const double* beta, int* run_len,
                                int* batched) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (!d_cut || !beta) return bfail(b, LBM_EINVAL, "NULL argument");
    const int n = (int)b->ctx.size();
    for (int i = 0; i < n; ++i)
        if (!b->ctx[i]->observed)
            return bfail(b, LBM_EINVAL, "experiment %d: letkf_observe must precede the analysis autotuning", i);
    // Size classes: on the run path, the union size class at the default
    // run length; with ensemble-space points (chunked path, whose kernel (A)
    // warm-starts along runs when members <= 32), the member tile (classes
    // 100 + tile). Other experiments are not tuned.
    auto tile = [](int v) { return v <= 8 ? 8 : (v <= 16 ? 16 : (v <= 24 ? 24 : (v <= 28 ? 28 : 32))); };
    std::vector<int> cls(n, -1);
    for (int i = 0; i < n; ++i) {
        lbm_ctx* c = b->ctx[i];
        if (!(d_cut[i] > 0.0) || !std::isfinite(d_cut[i]) || !(beta[i] > 0.0) || !std::isfinite(beta[i]))
            return bfail(b, LBM_EINVAL, "experiment %d: d_cut and beta must be finite and > 0", i);
        const int nmax = largest_local_problem(c, d_cut[i]);
        if (c->geo_any_ens) {
            if (is_fp32(c) && c->k <= 32 && nmax <= 32) cls[i] = 100 + tile(c->k);
            continue;
        }
        const int u = largest_run_union(c, d_cut[i], 8);
        if (u <= kRunMaxUnion) cls[i] = tile(u);
    }
    const int cand[] = {4, 8, 16, 32};
    cudaEvent_t t0, t1;
    BK(b, cudaEventCreate(&t0), "creating event");
    BK(b, cudaEventCreate(&t1), "creating event");
    int st = LBM_OK;
    std::vector<int> done(n, 0);
    for (int i0 = 0; i0 < n && st == LBM_OK; ++i0) {
        if (cls[i0] < 0 || done[i0]) continue;
        std::vector<int> which;
        for (int i = i0; i < n; ++i)
            if (cls[i] == cls[i0]) {
                which.push_back(i);
                done[i] = 1;
            }
        float best = 1e30f;
        int best_r = b->ctx[which[0]]->run_len, best_m = 1;
        // Run-path classes also time the class's analyses launched one
        // experiment at a time against the batched launches.
        const int nmodes = cls[i0] < 100 ? 2 : 1;
        for (int ci = 0; ci < 4 * nmodes && st == LBM_OK; ++ci) {
            const int r = cand[ci % 4], mode = ci < 4 ? 1 : 0;
            // Each timing analyses copies of the current states in the spare
            // buffers; the states and the observations are not changed.
            std::vector<AnalysisPlan> plans(n);
            for (int i : which) {
                lbm_ctx* c = b->ctx[i];
                c->run_len = r;
                c->run_batched = mode;
                st = analyze_prepare(c, d_cut[i], beta[i], &plans[i], true);
                if (st) break;
            }
            if (st) break;
            float tbest = 1e30f;
            for (int rep = 0; rep < 3 && st == LBM_OK; ++rep) {
                for (int i : which) {
                    lbm_ctx* c = b->ctx[i];
                    const size_t bytes = (size_t)9 * c->nx * c->ny * c->k * (is_fp32(c) ? 4 : 8);
                    if (cudaMemcpyAsync(c->f[1 - c->cur], c->f[c->cur], bytes, cudaMemcpyDeviceToDevice, b->stream) !=
                        cudaSuccess)
                        st = bfail(b, LBM_ECUDA, "copying a state for the autotuning");
                    c->cur ^= 1;
                }
                cudaEventRecord(t0, b->stream);
                if (st == LBM_OK) st = batch_analyze(b, plans, which, b->stream);
                cudaEventRecord(t1, b->stream);
                for (int i : which) b->ctx[i]->cur ^= 1;
                if (st == LBM_OK && cudaEventSynchronize(t1) != cudaSuccess)
                    st = bfail(b, LBM_ECUDA, "autotuning the analysis");
                float ms = 0.f;
                if (st == LBM_OK) cudaEventElapsedTime(&ms, t0, t1);
                if (ms < tbest) tbest = ms;
            }
            if (st) break;
            if (tbest < best) {
                best = tbest;
                best_r = r;
                best_m = mode;
            }
        }
        for (int i : which) {
            b->ctx[i]->run_len = best_r;
            b->ctx[i]->run_batched = best_m;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (st) return st;
    // A captured cycle holds the old shapes: capture again on the next cycle.
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    b->graph_steps = -1;
    for (int i = 0; i < n; ++i) {
        if (run_len) run_len[i] = b->ctx[i]->run_len;
        if (batched) batched[i] = b->ctx[i]->run_batched;
    }
    return LBM_OK;
}

int lbm_batch_cycle(lbm_batch* b, int nsteps, const int* npts, const int* const* ix, const int* const* iy,
                    const double* const* yo_u, const double* const* yo_v, const double* sigma,
                    const double* d_cut, const double* beta, int use_graph) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    const int n = (int)b->ctx.size();
    if (nsteps < 1) return bfail(b, LBM_EINVAL, "nsteps must be >= 1");
    if (!npts || !ix || !iy || !yo_u || !yo_v || !sigma || !d_cut || !beta)
        return bfail(b, LBM_EINVAL, "NULL argument");
    if (use_graph && (nsteps & 1))
        return bfail(b, LBM_EINVAL, "a captured cycle needs an even nsteps (the state buffers alternate)");
    for (int i = 0; i < n; ++i) {
        if (npts[i] < 1 || !ix[i] || !iy[i] || !yo_u[i] || !yo_v[i])
            return bfail(b, LBM_EINVAL, "experiment %d: missing observations", i);
        for (int j = 0; j < npts[i]; ++j)
            if (!std::isfinite(yo_u[i][j]) || !std::isfinite(yo_v[i][j]))
                return bfail(b, LBM_EINVAL, "experiment %d: observation %d is not finite", i, j);
    }
    const bool same_geometry = b->cycles > 0 && [&] {
        for (int i = 0; i < n; ++i) {
            if (npts[i] != b->npts[i]) return false;
            for (int j = 0; j < npts[i]; ++j)
                if (b->pos[i][j] != ix[i][j] || b->pos[i][npts[i] + j] != iy[i][j]) return false;
        }
        return true;
    }();
    const bool same_plan = same_geometry && b->graph_steps == nsteps &&
                           std::equal(d_cut, d_cut + n, b->graph_dcut.begin()) &&
                           std::equal(beta, beta + n, b->graph_beta.begin()) &&
                           std::equal(sigma, sigma + 2 * n, b->graph_sigma.begin());
    // The pinned staging may still be read by the previous graph launch.
    if (b->launched) BK(b, cudaEventSynchronize(b->done), "waiting for the previous cycle");
    if (!use_graph || !same_plan) {
        // Uncaptured cycle (also the first one, which sets positions, caches
        // the local-problem bounds and allocates scratch).
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        if (b->graph) {
            cudaGraphDestroy(b->graph);
            b->graph = nullptr;
        }
        int st = batch_forecast_impl(b, nsteps);
        if (st) return st;
        std::vector<AnalysisPlan> plans(n);
        for (int i = 0; i < n; ++i) {
            lbm_ctx* c = b->ctx[i];
            st = letkf_observe(c, npts[i], ix[i], iy[i], yo_u[i], yo_v[i], sigma[2 * i], sigma[2 * i + 1]);
            if (st) return bfail(b, st, "experiment %d: %s", i, c->err);
            st = analyze_prepare(c, d_cut[i], beta[i], &plans[i], true);
            if (st) return bfail(b, st, "experiment %d: %s", i, c->err);
        }
        st = batch_analyze(b, plans, all_experiments(b), b->stream);
        if (st) return st;
        for (int i = 0; i < n; ++i) {
            b->ctx[i]->observed = false;
            if (npts[i] > b->npts[i]) {
                if (b->h_yo[i]) cudaFreeHost(b->h_yo[i]);
                b->h_yo[i] = nullptr;
                BK(b, cudaMallocHost(&b->h_yo[i], 2 * (size_t)npts[i] * sizeof(double)), "allocating staging");
            }
            b->npts[i] = npts[i];
            b->pos[i].assign(ix[i], ix[i] + npts[i]);
            b->pos[i].insert(b->pos[i].end(), iy[i], iy[i] + npts[i]);
        }
        b->graph_steps = nsteps;
        b->graph_dcut.assign(d_cut, d_cut + n);
        b->graph_beta.assign(beta, beta + n);
        b->graph_sigma.assign(sigma, sigma + 2 * n);
        ++b->cycles;
        BK(b, cudaEventRecord(b->done, b->stream), "recording event");
        b->launched = true;
        return LBM_OK;
    }
    // Captured cycle: stage this cycle's values, then replay (capturing the
    // graph the first time with the plan of the previous, uncaptured cycle).
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < npts[i]; ++j) {
            b->h_yo[i][2 * j] = yo_u[i][j];
            b->h_yo[i][2 * j + 1] = yo_v[i][j];
        }
    }
    if (!b->exec) {
        std::vector<AnalysisPlan> plans(n);
        for (int i = 0; i < n; ++i) {
            lbm_ctx* c = b->ctx[i];
            int st = analyze_prepare(c, d_cut[i], beta[i], &plans[i], true);
            if (st) return bfail(b, st, "experiment %d: %s", i, c->err);
        }
        batch_table(b);
        BK(b, cudaMemcpyAsync(b->ex_dev, b->ex.data(), b->ex.size() * sizeof(MultiExp),
                              cudaMemcpyHostToDevice, b->stream),
           "copy experiment table");
        BK(b, cudaStreamSynchronize(b->stream), "synchronising");
        // Capture on a stream of our own (the shared stream may be the
        // legacy default stream, which cannot be captured): the contexts
        // queue on it while the capture lasts.
        if (!b->cap) BK(b, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "creating stream");
        const cudaStream_t shared = b->stream;
        for (lbm_ctx* c : b->ctx) c->stream = b->cap;
        BK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "beginning capture");
        cudaError_t e = launch_lbm_multi(b->ex_dev, n, b->total, nsteps, b->fp32, b->blocks, b->threads, b->bar,
                                         b->status, b->spin_limit, b->absent, b->cap);
        int st = e == cudaSuccess ? LBM_OK : LBM_ECUDA;
        for (int i = 0; i < n && st == LBM_OK; ++i) st = observe_from_pinned(b->ctx[i], b->h_yo[i]);
        if (st == LBM_OK) st = batch_analyze(b, plans, all_experiments(b), b->cap);
        cudaGraph_t g = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
        for (lbm_ctx* c : b->ctx) c->stream = shared;
        if (st != LBM_OK || e != cudaSuccess || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bfail(b, LBM_ECUDA, "capturing the cycle: %s",
                         cudaGetErrorString(e != cudaSuccess ? e : (ee != cudaSuccess ? ee : cudaErrorUnknown)));
        }
        b->graph = g;
        BK(b, cudaGraphInstantiate(&b->exec, b->graph, 0), "instantiating the cycle graph");
    }
    BK(b, cudaGraphLaunch(b->exec, b->stream), "launching the cycle graph");
    BK(b, cudaEventRecord(b->done, b->stream), "recording event");
    b->launched = true;
    ++b->cycles;
    return LBM_OK;
}

int lbm_batch_set_barrier(lbm_batch* b, long long spin_limit, int absent) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (spin_limit < 1 || spin_limit > kBarrierSpins) return bfail(b, LBM_EINVAL, "spin_limit out of range");
    if (absent < 0 || absent > 1) return bfail(b, LBM_EINVAL, "absent must be 0 or 1");
    BK(b, cudaStreamSynchronize(b->stream), "synchronising");
    b->spin_limit = spin_limit;
    b->absent = (unsigned)absent;
    // A captured cycle holds the old values: capture again on the next cycle.
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    b->graph_steps = -1;
    return LBM_OK;
}

int lbm_batch_set_analysis_form(lbm_batch* b, const int* batched) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (!batched) return bfail(b, LBM_EINVAL, "batched is NULL");
    const int n = (int)b->ctx.size();
    for (int i = 0; i < n; ++i)
        if (batched[i] != 0 && batched[i] != 1) return bfail(b, LBM_EINVAL, "batched[%d] must be 0 or 1", i);
    for (int i = 0; i < n; ++i) b->ctx[i]->run_batched = batched[i];
    // A captured cycle holds the old launches: capture again on the next cycle.
    if (b->exec) {
        BK(b, cudaStreamSynchronize(b->stream), "synchronising");
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    b->graph_steps = -1;
    return LBM_OK;
}

int lbm_batch_sync(lbm_batch* b) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    BK(b, cudaStreamSynchronize(b->stream), "synchronising");
    int h = 0;
    BK(b, cudaMemcpy(&h, b->status, sizeof(int), cudaMemcpyDeviceToHost), "reading barrier status");
    if (h) {
        cudaMemset(b->status, 0, sizeof(int));
        return bfail(b, LBM_ECUDA, "a grid barrier of the persistent forecast timed out");
    }
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        const int st = lbm_sync(b->ctx[i]);
        if (st) return bfail(b, st, "experiment %zu: %s", i, b->ctx[i]->err);
    }
    return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : g_init_err; }

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->done) cudaEventDestroy(b->done);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (double* p : b->h_yo)
        if (p) cudaFreeHost(p);
    cudaFree(b->ex_dev);
    cudaFree(b->bar);
    cudaFree(b->status);
    delete b;
}

}  // extern "C"
