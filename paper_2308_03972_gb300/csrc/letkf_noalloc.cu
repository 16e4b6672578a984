// Allocation-free variant of the LETKF analysis (observation operator,
// observation Gram and per-grid-point analysis) for callers that must not
// allocate device memory: code running under a memory manager that owns the
// whole device pool, inside a tightly budgeted embedding, or where a
// cudaMalloc would synchronise the device at a bad moment. The caller owns
// the ensemble state; the intermediate arrays live in one fixed file-scope
// device array instead of context buffers.
//
// The array below is part of the library image: every GPU that loads the
// library holds it (about 2.6 MB) until the process exits. Host code cannot
// use its name as a device address, so its address is looked up with
// cudaGetSymbolAddress once per device, on the first call made with that
// device current.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/lbm_letkf.h"
#include "lbm_internal.cuh"

namespace lbmgpu {
void set_context_free_error(const char* msg);
}

using namespace lbmgpu;

namespace {

constexpr int kMaxPts = LBM_NOALLOC_MAX_POINTS;
constexpr int kMaxObs = 2 * kMaxPts;
constexpr int kMaxMembers = LBM_NOALLOC_MAX_MEMBERS;

// Scratch layout, in doubles: dY [kMaxObs][kMaxMembers], G [kMaxObs][kMaxObs],
// d [kMaxObs], yo [kMaxObs], then ints: ix [kMaxPts], iy [kMaxPts], flags.
constexpr size_t kOffDY = 0;
constexpr size_t kOffG = kOffDY + (size_t)kMaxObs * kMaxMembers;
constexpr size_t kOffD = kOffG + (size_t)kMaxObs * kMaxObs;
constexpr size_t kOffYo = kOffD + kMaxObs;
constexpr size_t kOffInts = kOffYo + kMaxObs;
constexpr size_t kIntWords = 2 * (size_t)kMaxPts + 32;
constexpr size_t kScratchDoubles = kOffInts + (kIntWords + 1) / 2;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_base[kMaxDevices] = {};

int fail(int code, const char* msg) {
    set_context_free_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    set_context_free_error(buf);
    return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
}

// Device address of g_scratch on the current device (looked up once).
int scratch_base(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "querying the current device");
    if (dev < 0 || dev >= kMaxDevices) return fail(LBM_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
        double* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "looking up the scratch address");
        g_base[dev] = p;
    }
    *out = g_base[dev];
    return LBM_OK;
}

}  // namespace

extern "C" int letkf_analyze_noalloc(double* f, int nx, int ny, int members, int npts,
                                     const int* ix, const int* iy, const double* yo_u,
                                     const double* yo_v, double sigma_u, double sigma_v,
                                     double d_cut, double beta, void* stream) {
    if (!f || !ix || !iy || !yo_u || !yo_v) return fail(LBM_EINVAL, "NULL argument");
    if (nx < 1 || ny < 1 || !((long long)nx * ny < (1ll << 31)))
        return fail(LBM_EINVAL, "nx, ny must be >= 1 with nx * ny below 2^31");
    if (members < 2 || members > kMaxMembers)
        return fail(LBM_EINVAL, "members must be in [2, LBM_NOALLOC_MAX_MEMBERS]");
    if (npts < 1 || npts > kMaxPts)
        return fail(LBM_EINVAL, "npts must be in [1, LBM_NOALLOC_MAX_POINTS]");
    if (!(sigma_u > 0.0) || !(sigma_v > 0.0) || !std::isfinite(sigma_u) || !std::isfinite(sigma_v))
        return fail(LBM_EINVAL, "sigma_u and sigma_v must be finite and > 0");
    if (!(d_cut > 0.0) || !std::isfinite(d_cut)) return fail(LBM_EINVAL, "d_cut must be > 0");
    if (!(beta > 0.0) || !std::isfinite(beta)) return fail(LBM_EINVAL, "beta must be > 0");
    // Observation values and positions are host arrays, checked here so the
    // kernels never index outside the caller's state.
    double yo[kMaxObs];
    int pos[2 * kMaxPts];
    for (int j = 0; j < npts; ++j) {
        if (ix[j] < 0 || ix[j] >= nx || iy[j] < 0 || iy[j] >= ny)
            return fail(LBM_EINVAL, "observation point outside the lattice");
        if (!std::isfinite(yo_u[j]) || !std::isfinite(yo_v[j]))
            return fail(LBM_EINVAL, "observation value is not finite");
        yo[2 * j] = yo_u[j];
        yo[2 * j + 1] = yo_v[j];
        pos[j] = ix[j];
        pos[npts + j] = iy[j];
    }
    double* base = nullptr;
    int st = scratch_base(&base);
    if (st != LBM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double* dY = base + kOffDY;
    double* G = base + kOffG;
    double* d = base + kOffD;
    double* yo_d = base + kOffYo;
    int* ints = reinterpret_cast<int*>(base + kOffInts);
    int* ix_d = ints;
    int* iy_d = ints + npts;
    int* flags = ints + 2 * kMaxPts;

    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the flag word");
    e = cudaMemcpyAsync(ix_d, pos, 2 * (size_t)npts * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "copying positions");
    e = cudaMemcpyAsync(yo_d, yo, 2 * (size_t)npts * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "copying observations");
    e = launch_observe(f, 0, nx, ny, members, npts, 2, ix_d, iy_d, yo_d, dY, d, s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the observation operator");
    e = launch_obs_gram(dY, 2 * npts, members, G, s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the observation Gram");
    ObsParams o{npts, ix_d, iy_d, dY, d, G, sigma_u, sigma_v};
    // No host-side stamp of the local sets here: size the kernel for the
    // largest problem the inputs allow, min(k, p) with p = 2 * npts.
    const int nmax = members < 2 * npts ? members : 2 * npts;
    e = launch_analyze(f, 0, nx, ny, members, o, d_cut, beta, nmax, PROD_FP64, 0, flags, nullptr,
                       nullptr, s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the analysis");
    int h = 0;
    e = cudaMemcpyAsync(&h, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "reading the flag word");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "synchronising");
    if (h & FLAG_DIVERGED) return fail(LBM_EDIVERGED, "state diverged");
    if (h & FLAG_TOOLARGE) return fail(LBM_EINVAL, "local analysis problem larger than the kernel supports (min(k, p) > 64)");
    if (h & FLAG_NOCONV) return fail(LBM_ENOCONV, "eigensolver reached its sweep cap");
    return LBM_OK;
}
