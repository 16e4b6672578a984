// Adjoint (reverse mode) of the LBM forecast for a windowed observation
// misfit. The paper's Section 1 names the adjoint model as what makes
// variational assimilation costly; this is that adjoint for the forecast
// model of Section 2 / Section 4.1, written by hand:
//
//   f_{t+1}(xi + c_a, a) = f*_a(xi),
//   f*_a = f_a - omega (f_a - f^eq_a) + F_a,   omega = 1 / tau,
//   tau = (tau0 + S) / 2,  S = sqrt(tau0^2 + 18 Cs^2 Q / rho),  Q = sqrt(2 Pi:Pi),
//   Pi = sum_a c_a c_a (f_a - f^eq_a),  F_a = 3 w_a (rho F^i.c_a - mu j.c_a),
//
// with rho = sum f, j = sum f c, u = j / rho. Given lambda_{t+1} = dJ/df_{t+1},
// the step adjoint pulls g_a(xi) = lambda_{t+1}(xi + c_a, a) (the transpose
// of the push) and applies the transposed Jacobian of the collision at
// f_t(xi):
//
//   dJ/df_b = (1 - omega) g_b + omega (G_rho + G_j.c_b)          [f^eq]
//           + 3 sum_a g_a w_a F^i.c_a - 3 mu (sum_a g_a w_a c_a).c_b   [forcing]
//           + kappa ((2 / (Q rho)) D_b - Q / rho^2)                 [tau]
//
//   G_rho = sum_a g_a w_a (1 - 9/2 (c_a.u)^2 + 3/2 u.u),
//   G_j   = sum_a g_a w_a (3 c_a + 9 (c_a.u) c_a - 3 u),
//   h = sum_a g_a (f_a - f^eq_a),  kappa = h omega^2 18 Cs^2 / (4 S),
//   D_b = (c_b - u)^T Pi (c_b - u) - tr(Pi) / 3,
//
// (f^eq written as w_a (rho + 3 c.j + 9/2 (c.j)^2 / rho - 3/2 j.j / rho); dQ
// from Q^2 = 2 Pi:Pi and dPi_ab/df_b = c_ba c_bb - delta_ab / 3 - (c_ba u_b +
// u_a c_bb) + u_a u_b). Where Q = 0 (f at equilibrium) the D term is taken as
// zero: it multiplies h = 0 there. The closure coefficient enters only
// through omega: dJ/dCs += h omega^2 9 Cs Q / (rho S) per cell and member.
//
// The misfit of one observation time adds, at each observation point eta_j,
// w_m ((u - yo_u) (c_bx - u) / sigma_u^2 + (v - yo_v) (c_by - v) / sigma_v^2) / rho
// to lambda_t(eta_j, b) (the derivative of 1/2 w_m r^2 through u = j / rho).
#include <cmath>

#include "lbm_internal.cuh"
#include "vec.cuh"

namespace lbmgpu {
namespace {

__host__ __device__ constexpr double wgt(int a) { return d2q9_w(a); }

// Reciprocal and square root: IEEE in FP64; in binary32 the approximate
// hardware forms (a few ulp; the binary32 adjoint is checked against the
// FP64 one at 1e-3), without the special-case branches of the IEEE ones.
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp_(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

// Transposed collision Jacobian at one cell and member. f: the stored state
// (g = f - w with SHIFT), g: adjoint of the post-collision values (in), out:
// adjoint of the pre-collision values. Returns the C_s derivative term.
template <typename T, bool SHIFT>
__device__ __forceinline__ T collide_vjp(const T (&f)[9], const T (&g)[9], T (&out)[9], T Fix,
                                         T Fiy, T tau0, T cs, T mu) {
    T s = T(0), jx = T(0), jy = T(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        s += f[a];
        jx += T(d2q9_cx(a)) * f[a];
        jy += T(d2q9_cy(a)) * f[a];
    }
    const T rho = SHIFT ? T(1) + s : s;
    const T ir = rcp_(rho);
    const T ux = jx * ir, uy = jy * ir;
    const T uu = ux * ux + uy * uy;
    T fneq[9];
    T pxx = T(0), pxy = T(0), pyy = T(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const T cx = T(d2q9_cx(a)), cy = T(d2q9_cy(a));
        const T cu = cx * ux + cy * uy;
        const T w = T(wgt(a));
        // f - f^eq; with SHIFT, f = g + w and f^eq - w = w (s + rho (3cu +
        // 9/2 cu^2 - 3/2 uu)), s = rho - 1 (no cancellation near rest).
        const T feq_rel = w * ((SHIFT ? s : rho) + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu));
        fneq[a] = f[a] - feq_rel;
        pxx += cx * cx * fneq[a];
        pxy += cx * cy * fneq[a];
        pyy += cy * cy * fneq[a];
    }
    const T Q = sqrt_(T(2) * (pxx * pxx + T(2) * pxy * pxy + pyy * pyy));
    const T cs18 = T(18) * cs * cs;
    const T S = sqrt_(tau0 * tau0 + cs18 * Q * ir);
    const T iS = rcp_(S);
    const T om = T(2) * rcp_(tau0 + S);
    const T iQ = Q > T(0) ? rcp_(Q) : T(0);
    // Contractions of the incoming adjoint.
    T grho = T(0), gjx = T(0), gjy = T(0), gF = T(0), gcx = T(0), gcy = T(0), h = T(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const T cx = T(d2q9_cx(a)), cy = T(d2q9_cy(a));
        const T cu = cx * ux + cy * uy;
        const T gw = g[a] * T(wgt(a));
        grho += gw * (T(1) - T(4.5) * cu * cu + T(1.5) * uu);
        gjx += gw * (T(3) * cx + T(9) * cu * cx - T(3) * ux);
        gjy += gw * (T(3) * cy + T(9) * cu * cy - T(3) * uy);
        gF += gw * (Fix * cx + Fiy * cy);
        gcx += gw * cx;
        gcy += gw * cy;
        h += g[a] * fneq[a];
    }
    const T kappa = T(0.25) * h * om * om * cs18 * iS;
    const T qfac = T(2) * ir * iQ;
    const T trp3 = (pxx + pyy) * T(1.0 / 3.0);
    const T base = om * grho + T(3) * gF - kappa * Q * ir * ir;
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        const T cx = T(d2q9_cx(b)), cy = T(d2q9_cy(b));
        const T dx = cx - ux, dy = cy - uy;
        const T D = pxx * dx * dx + T(2) * pxy * dx * dy + pyy * dy * dy - trp3;
        out[b] = (T(1) - om) * g[b] + base + om * (gjx * cx + gjy * cy) -
                 T(3) * mu * (gcx * cx + gcy * cy) + kappa * qfac * D;
    }
    return h * om * om * T(9) * cs * Q * ir * iS;
}

// One adjoint step: lam_out(xi) = collision VJP at f_t(xi) of the pulled
// lam_in(xi + c_a, a). Same thread layout as the forward step (V consecutive
// members of one cell per thread). The C_s derivative of every member is
// summed per block in shared memory (FP64) and added to gcs[k] once per
// block and member.
template <typename T, int V, bool SHIFT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) adjoint_step_kernel(const T* __restrict__ ft,
                                                           const T* __restrict__ lam_in,
                                                           T* __restrict__ lam_out,
                                                           const T* __restrict__ force, int nx,
                                                           int ny, int k, T tau0, T cs, T mu,
                                                           double* __restrict__ gcs) {
    extern __shared__ unsigned char adj_smem[];
    T* part = reinterpret_cast<T*>(adj_smem);  // [blockDim][V] C_s terms
    const int kv = k / V;
    const long long total = (long long)nx * ny * kv;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    T dcs[V];
#pragma unroll
    for (int j = 0; j < V; ++j) dcs[j] = T(0);
    if (t < total) {
        int mv, x, y;
        long long cell;
        split_item(t, kv, nx, mv, cell, x, y);
        const size_t plane = (size_t)nx * ny * k;
        const size_t mo = (size_t)mv * V;
        const size_t here = (size_t)cell * k + mo;
        T f[9][V], g[9][V];
#pragma unroll
        for (int a = 0; a < 9; ++a) Vec<T, V>::ld(ft + a * plane + here, f[a]);
        const int xp = (x + 1 == nx) ? 0 : x + 1, xm = (x == 0) ? nx - 1 : x - 1;
        const int yp = (y + 1 == ny) ? 0 : y + 1, ym = (y == 0) ? ny - 1 : y - 1;
        auto src = [&](int a, int xx, int yy) {
            return lam_in + a * plane + ((size_t)yy * nx + xx) * k + mo;
        };
        // Transpose of the push: the adjoint of f*_a(xi) sits at xi + c_a.
        Vec<T, V>::ld(src(0, x, y), g[0]);
        Vec<T, V>::ld(src(1, xp, y), g[1]);
        Vec<T, V>::ld(src(2, xm, y), g[2]);
        Vec<T, V>::ld(src(3, x, yp), g[3]);
        Vec<T, V>::ld(src(4, x, ym), g[4]);
        Vec<T, V>::ld(src(5, xp, yp), g[5]);
        Vec<T, V>::ld(src(6, xm, ym), g[6]);
        Vec<T, V>::ld(src(7, xp, ym), g[7]);
        Vec<T, V>::ld(src(8, xm, yp), g[8]);
        const T Fix = __ldg(force + cell);
        const T Fiy = __ldg(force + (size_t)nx * ny + cell);
#pragma unroll
        for (int j = 0; j < V; ++j) {
            T fj[9], gj[9], oj[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                fj[a] = f[a][j];
                gj[a] = g[a][j];
            }
            dcs[j] = collide_vjp<T, SHIFT>(fj, gj, oj, Fix, Fiy, tau0, cs, mu);
#pragma unroll
            for (int a = 0; a < 9; ++a) g[a][j] = oj[a];  // g now holds the output
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) Vec<T, V>::st(lam_out + a * plane + here, g[a]);
    }
    // C_s derivative per member: the block's terms of member m sit at the
    // threads t0 with (t0 - first) % kv == m / V (slot m % V); they are summed
    // in thread order and added to gcs once per block.
#pragma unroll
    for (int j = 0; j < V; ++j) part[threadIdx.x * V + j] = dcs[j];
    __syncthreads();
    const long long first = (long long)blockIdx.x * blockDim.x;
    const int first_mv = (int)(first % kv);  // once per thread
    for (int m = threadIdx.x; m < k; m += blockDim.x) {
        const int mv = m / V, j = m % V;
        // First thread of the block holding member group mv.
        int t0 = mv - first_mv;
        if (t0 < 0) t0 += kv;
        double acc = 0.0;
        for (; t0 < (int)blockDim.x; t0 += kv) acc += (double)part[t0 * V + j];
        if (acc != 0.0) atomicAdd(&gcs[m], acc);
    }
}

// Misfit terms of one observation time: for point j and member m,
// r[j][m] = 1/2 ((u - yo_u)^2 / sigma_u^2 + (v - yo_v)^2 / sigma_v^2).
template <typename T, bool SHIFT>
__global__ void misfit_kernel(const T* __restrict__ f, int nx, int ny, int k, int npts,
                              const int* __restrict__ ix, const int* __restrict__ iy,
                              const double* __restrict__ yo, double isu2, double isv2,
                              double* __restrict__ r) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)npts * k) return;
    const int j = (int)(i / k), m = (int)(i % k);
    const size_t plane = (size_t)nx * ny * k;
    const size_t at = ((size_t)iy[j] * nx + ix[j]) * k + m;
    double s = SHIFT ? 1.0 : 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const double v = (double)f[a * plane + at];
        s += v;
        jx += d2q9_cx(a) * v;
        jy += d2q9_cy(a) * v;
    }
    const double du = jx / s - yo[2 * j], dv = jy / s - yo[2 * j + 1];
    r[i] = 0.5 * (du * du * isu2 + dv * dv * isv2);
}

// Adds the misfit derivative of one observation time to lam at the points
// (atomic, so repeated points accumulate).
template <typename T, bool SHIFT>
__global__ void misfit_adjoint_kernel(const T* __restrict__ f, T* __restrict__ lam, int nx, int ny,
                                      int k, int npts, const int* __restrict__ ix,
                                      const int* __restrict__ iy, const double* __restrict__ yo,
                                      double isu2, double isv2, const double* __restrict__ w) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)npts * k) return;
    const int j = (int)(i / k), m = (int)(i % k);
    const size_t plane = (size_t)nx * ny * k;
    const size_t at = ((size_t)iy[j] * nx + ix[j]) * k + m;
    double s = SHIFT ? 1.0 : 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const double v = (double)f[a * plane + at];
        s += v;
        jx += d2q9_cx(a) * v;
        jy += d2q9_cy(a) * v;
    }
    const double u = jx / s, v = jy / s;
    const double ru = w[m] * (u - yo[2 * j]) * isu2 / s;
    const double rv = w[m] * (v - yo[2 * j + 1]) * isv2 / s;
#pragma unroll
    for (int b = 0; b < 9; ++b)
        atomicAdd(&lam[b * plane + at], (T)(ru * (d2q9_cx(b) - u) + rv * (d2q9_cy(b) - v)));
}

// J[m] = sum over times and points of r: one block per member, strided
// partial sums then a shared-memory tree, in a fixed order.
__global__ void __launch_bounds__(256) misfit_reduce_kernel(const double* __restrict__ r, int nterms,
                                                            int k, double* __restrict__ J) {
    __shared__ double part[256];
    const int m = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < nterms; i += 256) s += r[(size_t)i * k + m];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) J[m] = part[0];
}

template <typename T>
__global__ void widen_kernel(const T* __restrict__ src, double* __restrict__ dst, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}

inline unsigned blocks_of(long long n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename T, int V, bool SHIFT>
cudaError_t adjoint_step_v(const T* ft, const T* lin, T* lout, const T* force, const LbmParams& p,
                           double cs, double* gcs, cudaStream_t s) {
    const long long total = (long long)p.nx * p.ny * (p.k / V);
    const long long nb = (total + 255) / 256;
    if (nb > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const size_t sh = (size_t)256 * V * sizeof(T);
    adjoint_step_kernel<T, V, SHIFT><<<(unsigned)nb, 256, sh, s>>>(ft, lin, lout, force, p.nx, p.ny, p.k,
                                                                   (T)p.tau0, (T)cs, (T)p.mu, gcs);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adjoint_step(const void* ft, const void* lam_in, void* lam_out, const void* force,
                                int fp32, const LbmParams& p, double cs, double* gcs,
                                cudaStream_t s) {
    if (fp32) {
        const float *f = (const float*)ft, *li = (const float*)lam_in, *fo = (const float*)force;
        float* lo = (float*)lam_out;
        if (p.k % 2 == 0) return adjoint_step_v<float, 2, true>(f, li, lo, fo, p, cs, gcs, s);
        return adjoint_step_v<float, 1, true>(f, li, lo, fo, p, cs, gcs, s);
    }
    const double *f = (const double*)ft, *li = (const double*)lam_in, *fo = (const double*)force;
    double* lo = (double*)lam_out;
    // FP64: one member per thread (the FP64 collision adjoint is bound by
    // the FP64 units; two members per thread would spill).
    return adjoint_step_v<double, 1, false>(f, li, lo, fo, p, cs, gcs, s);
}

cudaError_t launch_misfit(const void* f, int fp32, int nx, int ny, int k, int npts, const int* ix,
                          const int* iy, const double* yo, double sigma_u, double sigma_v,
                          double* r, cudaStream_t s) {
    const long long n = (long long)npts * k;
    if (n == 0) return cudaSuccess;
    const double isu2 = 1.0 / (sigma_u * sigma_u), isv2 = 1.0 / (sigma_v * sigma_v);
    if (fp32)
        misfit_kernel<float, true><<<blocks_of(n, 128), 128, 0, s>>>((const float*)f, nx, ny, k, npts, ix,
                                                                     iy, yo, isu2, isv2, r);
    else
        misfit_kernel<double, false><<<blocks_of(n, 128), 128, 0, s>>>((const double*)f, nx, ny, k, npts,
                                                                       ix, iy, yo, isu2, isv2, r);
    return cudaGetLastError();
}

cudaError_t launch_misfit_adjoint(const void* f, void* lam, int fp32, int nx, int ny, int k, int npts,
                                  const int* ix, const int* iy, const double* yo, double sigma_u,
                                  double sigma_v, const double* w, cudaStream_t s) {
    const long long n = (long long)npts * k;
    if (n == 0) return cudaSuccess;
    const double isu2 = 1.0 / (sigma_u * sigma_u), isv2 = 1.0 / (sigma_v * sigma_v);
    if (fp32)
        misfit_adjoint_kernel<float, true><<<blocks_of(n, 128), 128, 0, s>>>(
            (const float*)f, (float*)lam, nx, ny, k, npts, ix, iy, yo, isu2, isv2, w);
    else
        misfit_adjoint_kernel<double, false><<<blocks_of(n, 128), 128, 0, s>>>(
            (const double*)f, (double*)lam, nx, ny, k, npts, ix, iy, yo, isu2, isv2, w);
    return cudaGetLastError();
}

cudaError_t launch_misfit_reduce(const double* r, int nterms, int k, double* J, cudaStream_t s) {
    misfit_reduce_kernel<<<(unsigned)k, 256, 0, s>>>(r, nterms, k, J);
    return cudaGetLastError();
}

cudaError_t launch_widen(const void* src, int fp32, double* dst, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (fp32)
        widen_kernel<float><<<blocks_of((long long)n, 256), 256, 0, s>>>((const float*)src, dst, n);
    else
        widen_kernel<double><<<blocks_of((long long)n, 256), 256, 0, s>>>((const double*)src, dst, n);
    return cudaGetLastError();
}

}  // namespace lbmgpu
