// Ensemble diagnostics (arXiv 2308.03972, Section 4.1 energy spectrum):
// E(s) = mean over members of sum_{s - 1/2 <= |k'| < s + 1/2} |u-hat(k')|^2 / 2,
// u-hat(k') = N^{-1} sum_xi u(xi) exp(-i k'.xi), both velocity components.
//
// Three passes, all FP64:
//  (1) rows: per lattice row and member group, the velocity is formed from
//      the nine f's and transformed along x for kx = 0 .. nx/2 only (the field
//      is real, so u-hat(-k') is the conjugate of u-hat(k'));
//  (2) columns: per (kx, member), the x-transforms are transformed along y,
//      |u-hat|^2 / 2 is weighted by the multiplicity of kx (1 for kx = 0 and
//      the even Nyquist column, 2 otherwise) and binned by shell, in ky order,
//      into a per-(member, kx) partial row;
//  (3) reduce: per shell, the partials summed over kx and the mean over
//      members, in a fixed order (the result does not depend on scheduling).
// This is an untimed diagnostic; the direct transforms cost O(nx ny (nx + ny))
// per member and component.
#include <cmath>

#include "lbm_internal.cuh"

namespace lbmgpu {
namespace {

constexpr int kRowMembers = 8;  // members per block in the row pass

// exp(-2 pi i j / n) as (cos, -sin) with the angle reduced to j / n in [0, 1).
__device__ __forceinline__ void twiddle(int j, int n, double& c, double& s) {
    double sn, cs;
    sincospi(2.0 * (double)j / (double)n, &sn, &cs);
    c = cs;
    s = -sn;
}

// Pass 1. Grid (ny, ceil(k / kRowMembers)). Shared: u, v [nx][kRowMembers],
// twiddles [nx] (re, im). Output F1 [k][2][ny][hx] complex (re, im).
template <typename T, bool SHIFT>
__global__ void spectrum_rows_kernel(const T* __restrict__ f, int nx, int ny, int k, int hx,
                                     double2* __restrict__ F1, int* __restrict__ flags) {
    extern __shared__ double sh[];
    double* su = sh;
    double* sv = su + (size_t)nx * kRowMembers;
    double2* tw = reinterpret_cast<double2*>(sv + (size_t)nx * kRowMembers);
    const int y = blockIdx.x;
    const int m0 = blockIdx.y * kRowMembers;
    const int nm = min(kRowMembers, k - m0);
    const size_t plane = (size_t)nx * ny * k;
    for (int j = threadIdx.x; j < nx; j += blockDim.x) {
        double c, s;
        twiddle(j, nx, c, s);
        tw[j] = make_double2(c, s);
    }
    bool bad = false;
    for (int t = threadIdx.x; t < nx * kRowMembers; t += blockDim.x) {
        const int x = t / kRowMembers, ml = t % kRowMembers;
        double u = 0.0, v = 0.0;
        if (ml < nm) {
            const size_t i = ((size_t)y * nx + x) * k + m0 + ml;
            double r = SHIFT ? 1.0 : 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                const double g = (double)f[a * plane + i];
                r += g;
                jx += d2q9_cx(a) * g;
                jy += d2q9_cy(a) * g;
            }
            u = jx / r;
            v = jy / r;
            bad |= !(r > 0.0) || !(u * u + v * v <= kUMax2);
        }
        su[t] = u;
        sv[t] = v;
    }
    if (bad) atomicOr(flags, FLAG_DIVERGED);
    __syncthreads();
    for (int t = threadIdx.x; t < hx * nm; t += blockDim.x) {
        const int kx = t / nm, ml = t % nm;
        double ur = 0.0, ui = 0.0, vr = 0.0, vi = 0.0;
        int idx = 0;  // kx * x mod nx, advanced incrementally
        for (int x = 0; x < nx; ++x) {
            const double2 w = tw[idx];
            const double uu = su[x * kRowMembers + ml], vv = sv[x * kRowMembers + ml];
            ur += uu * w.x;
            ui += uu * w.y;
            vr += vv * w.x;
            vi += vv * w.y;
            idx += kx;
            if (idx >= nx) idx -= nx;
        }
        const size_t m = (size_t)(m0 + ml);
        F1[((m * 2 + 0) * ny + y) * hx + kx] = make_double2(ur, ui);
        F1[((m * 2 + 1) * ny + y) * hx + kx] = make_double2(vr, vi);
    }
}

// Pass 2. Grid (hx, k). Shared: column of both components [2][ny], twiddles
// [ny], energies [ny], shell bins [nsh]. Output P [k][hx][nsh].
__global__ void spectrum_cols_kernel(const double2* __restrict__ F1, int nx, int ny, int k,
                                     int hx, int nsh, double* __restrict__ P) {
    extern __shared__ double sh[];
    double2* col = reinterpret_cast<double2*>(sh);  // [2][ny]
    double2* tw = col + 2 * (size_t)ny;             // [ny]
    double* e = reinterpret_cast<double*>(tw + ny);  // [ny]
    double* bins = e + ny;                           // [nsh]
    const int kx = blockIdx.x;
    const size_t m = blockIdx.y;
    for (int j = threadIdx.x; j < ny; j += blockDim.x) {
        double c, s;
        twiddle(j, ny, c, s);
        tw[j] = make_double2(c, s);
        col[j] = F1[((m * 2 + 0) * ny + j) * hx + kx];
        col[ny + j] = F1[((m * 2 + 1) * ny + j) * hx + kx];
    }
    for (int s = threadIdx.x; s < nsh; s += blockDim.x) bins[s] = 0.0;
    __syncthreads();
    const double inv_n = 1.0 / ((double)nx * (double)ny);
    const double mult = (kx == 0 || 2 * kx == nx) ? 1.0 : 2.0;
    for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) {
        double ur = 0.0, ui = 0.0, vr = 0.0, vi = 0.0;
        int idx = 0;
        for (int y = 0; y < ny; ++y) {
            const double2 w = tw[idx];
            const double2 a = col[y], b = col[ny + y];
            ur += a.x * w.x - a.y * w.y;
            ui += a.x * w.y + a.y * w.x;
            vr += b.x * w.x - b.y * w.y;
            vi += b.x * w.y + b.y * w.x;
            idx += ky;
            if (idx >= ny) idx -= ny;
        }
        ur *= inv_n;
        ui *= inv_n;
        vr *= inv_n;
        vi *= inv_n;
        e[ky] = mult * 0.5 * ((ur * ur + ui * ui) + (vr * vr + vi * vi));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int ky = 0; ky < ny; ++ky) {
            const int wy = 2 * ky > ny ? ky - ny : ky;
            const double mag = sqrt((double)kx * kx + (double)wy * wy);
            const int s = (int)floor(mag + 0.5);
            if (s < nsh) bins[s] += e[ky];
        }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < nsh; s += blockDim.x) P[(m * hx + kx) * nsh + s] = bins[s];
}

// Pass 3. One thread per shell.
__global__ void spectrum_reduce_kernel(const double* __restrict__ P, int k, int hx, int nsh,
                                       double* __restrict__ E) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsh) return;
    double acc = 0.0;
    for (int m = 0; m < k; ++m) {
        double em = 0.0;
        for (int kx = 0; kx < hx; ++kx) em += P[((size_t)m * hx + kx) * nsh + s];
        acc += em;
    }
    E[s] = acc / k;
}

// RMSE of two velocity fields (Section 4.3 scores the ensemble mean
// against the truth): sum over cells of (u1 - u2)^2 + (v1 - v2)^2 in FP64,
// block partials in a fixed order, then one block sums the partials in
// order and writes sqrt(sum / n).
constexpr int kRmseBlocks = 256, kRmseThreads = 256;

__global__ void __launch_bounds__(kRmseThreads) rmse_partial_kernel(const double* __restrict__ u1,
                                                                   const double* __restrict__ v1,
                                                                   const double* __restrict__ u2,
                                                                   const double* __restrict__ v2, size_t n,
                                                                   double* __restrict__ partial) {
    __shared__ double red[kRmseThreads];
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * kRmseThreads + threadIdx.x; i < n; i += (size_t)kRmseBlocks * kRmseThreads) {
        const double du = u1[i] - u2[i], dv = v1[i] - v2[i];
        s += du * du + dv * dv;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = kRmseThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kRmseThreads) rmse_final_kernel(const double* __restrict__ partial, size_t n,
                                                                 double* __restrict__ out) {
    __shared__ double red[kRmseThreads];
    red[threadIdx.x] = threadIdx.x < kRmseBlocks ? partial[threadIdx.x] : 0.0;
    __syncthreads();
    for (int h = kRmseThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sqrt(red[0] / (double)n);
}

}  // namespace

size_t spectrum_work_bytes(int nx, int ny, int k, int nshells) {
    const size_t hx = (size_t)nx / 2 + 1;
    return (size_t)k * 2 * ny * hx * sizeof(double2) + (size_t)k * hx * nshells * sizeof(double);
}

cudaError_t launch_energy_spectrum(const void* f, int fp32, int nx, int ny, int k, double* E,
                                   int nshells, void* work, int* flags, cudaStream_t s) {
    const int hx = nx / 2 + 1;
    double2* F1 = reinterpret_cast<double2*>(work);
    double* P = reinterpret_cast<double*>(F1 + (size_t)k * 2 * ny * hx);
    const size_t sh1 = 2 * (size_t)nx * kRowMembers * sizeof(double) + (size_t)nx * sizeof(double2);
    const size_t sh2 = 3 * (size_t)ny * sizeof(double2) + (size_t)ny * sizeof(double) +
                       (size_t)nshells * sizeof(double);
    constexpr size_t kMaxShared = 227 * 1024;
    if (sh1 > kMaxShared || sh2 > kMaxShared) return cudaErrorInvalidValue;
    cudaError_t e;
    const dim3 g1((unsigned)ny, (unsigned)((k + kRowMembers - 1) / kRowMembers));
    if (fp32) {
        e = cudaFuncSetAttribute(spectrum_rows_kernel<float, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh1);
        if (e != cudaSuccess) return e;
        spectrum_rows_kernel<float, true><<<g1, 256, sh1, s>>>((const float*)f, nx, ny, k, hx, F1,
                                                               flags);
    } else {
        e = cudaFuncSetAttribute(spectrum_rows_kernel<double, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh1);
        if (e != cudaSuccess) return e;
        spectrum_rows_kernel<double, false><<<g1, 256, sh1, s>>>((const double*)f, nx, ny, k, hx,
                                                                 F1, flags);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = cudaFuncSetAttribute(spectrum_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sh2);
    if (e != cudaSuccess) return e;
    spectrum_cols_kernel<<<dim3((unsigned)hx, (unsigned)k), 256, sh2, s>>>(F1, nx, ny, k, hx,
                                                                           nshells, P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    spectrum_reduce_kernel<<<(nshells + 127) / 128, 128, 0, s>>>(P, k, hx, nshells, E);
    return cudaGetLastError();
}

size_t rmse_work_doubles() { return kRmseBlocks; }

cudaError_t launch_velocity_rmse(const double* u1, const double* v1, const double* u2, const double* v2, size_t n,
                                 double* work, double* out, cudaStream_t s) {
    if (n == 0) return cudaErrorInvalidValue;
    rmse_partial_kernel<<<kRmseBlocks, kRmseThreads, 0, s>>>(u1, v1, u2, v2, n, work);
    rmse_final_kernel<<<1, kRmseThreads, 0, s>>>(work, n, out);
    return cudaGetLastError();
}

}  // namespace lbmgpu
