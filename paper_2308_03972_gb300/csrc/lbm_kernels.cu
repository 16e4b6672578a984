// Lattice-Boltzmann kernels of the LBM-LETKF library (sm_103a).
//
// K1 fused collide+push step (arXiv 2308.03972, Section 2: lattice BGK
// equation, moments, second-order equilibrium, Smagorinsky eddy viscosity,
// forcing term; Section 4.1: F = F^i - mu u), the moments kernel, and the
// layout conversions at the C-ABI boundary.
//
// Layout: f[alpha][y][x][m], member index innermost. A thread owns V
// consecutive members of one cell, so the nine loads and the nine pushed
// stores of a warp are contiguous 16-byte vectors; a shift by one cell is a
// shift by k elements and keeps that alignment.
//
// Precision: FP64 stores f itself. FP32 stores g = f - w_alpha (the rest
// state at rho = 1 removed) so binary32 keeps the small departures from rest
// that carry the flow; the collision is written in terms of g.
#include <cmath>

#include "lbm_internal.cuh"
#include "vec.cuh"

namespace lbmgpu {
namespace {

// BGK-LES collision of one member at one cell, in place on f[9].
// SHIFT: f holds g = f - w_alpha. Returns true if the state is bad
// (non-positive or non-finite density, or |u|^2 above the limit).
template <typename T, bool SHIFT>
__device__ __forceinline__ bool collide(T (&f)[9], T Fix, T Fiy, T tau0, T cs18, T mu) {
    // Density and momentum. With SHIFT the sum is rho - 1 (sum w = 1) and
    // the momentum is unchanged (sum w c = 0).
    const T s = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    const T rho = SHIFT ? T(1) + s : s;
    const T jx = (f[1] - f[2]) + (f[5] - f[6]) + (f[7] - f[8]);
    const T jy = (f[3] - f[4]) + (f[5] - f[6]) + (f[8] - f[7]);
    const T ir = T(1) / rho;
    const T ux = jx * ir, uy = jy * ir;
    const T uu = ux * ux + uy * uy;
    // f^eq_a (or f^eq_a - w_a) = w_a (A + rho e_a), e_a = 3 c.u + 9/2 (c.u)^2,
    // A = rho (1 - 3/2 u.u) (or rho - 1 - 3/2 rho u.u).
    const T A = s - T(1.5) * rho * uu;
    T fneq[9];
    {
        fneq[0] = f[0] - T(4.0 / 9.0) * A;
        const T cu[4] = {ux, uy, ux + uy, ux - uy};
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const T q = T(4.5) * cu[p] * cu[p];
            const T l = T(3) * cu[p];
            const T w = p < 2 ? T(1.0 / 9.0) : T(1.0 / 36.0);
            const int ap = p < 2 ? 1 + 2 * p : 5 + 2 * (p - 2);  // +c direction
            fneq[ap] = f[ap] - w * (A + rho * (q + l));
            fneq[ap + 1] = f[ap + 1] - w * (A + rho * (q - l));
        }
    }
    // Non-equilibrium momentum flux and the Smagorinsky relaxation time
    // tau = (tau0 + sqrt(tau0^2 + 18 Cs^2 Q / rho)) / 2, Q = sqrt(2 Pi:Pi).
    const T d58 = (fneq[5] + fneq[6]) + (fneq[7] + fneq[8]);
    const T pxx = (fneq[1] + fneq[2]) + d58;
    const T pyy = (fneq[3] + fneq[4]) + d58;
    const T pxy = (fneq[5] + fneq[6]) - (fneq[7] + fneq[8]);
    const T Q = sqrt(T(2) * (pxx * pxx + T(2) * pxy * pxy + pyy * pyy));
    const T tau = T(0.5) * (tau0 + sqrt(tau0 * tau0 + cs18 * Q * ir));
    const T om = T(1) / tau;
    // Forcing F_a = 3 w_a rho F.c_a with F = F^i - mu u.
    const T Fx = Fix - mu * ux, Fy = Fiy - mu * uy;
    const T fx3 = rho * Fx * T(1.0 / 3.0);
    const T fy3 = rho * Fy * T(1.0 / 3.0);
    const T dp = rho * (Fx + Fy) * T(1.0 / 12.0);
    const T dm = rho * (Fx - Fy) * T(1.0 / 12.0);
    f[0] = f[0] - om * fneq[0];
    f[1] = f[1] - om * fneq[1] + fx3;
    f[2] = f[2] - om * fneq[2] - fx3;
    f[3] = f[3] - om * fneq[3] + fy3;
    f[4] = f[4] - om * fneq[4] - fy3;
    f[5] = f[5] - om * fneq[5] + dp;
    f[6] = f[6] - om * fneq[6] - dp;
    f[7] = f[7] - om * fneq[7] + dm;
    f[8] = f[8] - om * fneq[8] - dm;
    return !(uu <= T(kUMax2)) || !(rho > T(0));
}

// One work item of a step: V consecutive members (group mv) of one cell,
// item index t in [0, nx * ny * k / V). Collide, then push.
template <typename T, int V, bool SHIFT>
__device__ __forceinline__ void step_item(const T* __restrict__ fin, T* __restrict__ fout,
                                          const T* __restrict__ force, int nx, int ny, int k,
                                          T tau0, T cs18, T mu, int* __restrict__ flags,
                                          long long t) {
    const int kv = k / V;
    int mv, x, y;
    long long cell;
    split_item(t, kv, nx, mv, cell, x, y);
    const size_t plane = (size_t)nx * ny * k;  // elements per alpha
    const size_t src = (size_t)cell * k + (size_t)mv * V;

    T f[9][V];
#pragma unroll
    for (int a = 0; a < 9; ++a) Vec<T, V>::ld(fin + a * plane + src, f[a]);
    const T Fix = __ldg(force + cell);
    const T Fiy = __ldg(force + (size_t)nx * ny + cell);

    bool bad = false;
#pragma unroll
    for (int j = 0; j < V; ++j) {
        T g[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) g[a] = f[a][j];
        bad |= collide<T, SHIFT>(g, Fix, Fiy, tau0, cs18, mu);
#pragma unroll
        for (int a = 0; a < 9; ++a) f[a][j] = g[a];
    }
    if (bad) atomicOr(flags, FLAG_DIVERGED);

    // Push f*_a to xi + c_a with periodic wrap.
    const int xp = (x + 1 == nx) ? 0 : x + 1, xm = (x == 0) ? nx - 1 : x - 1;
    const int yp = (y + 1 == ny) ? 0 : y + 1, ym = (y == 0) ? ny - 1 : y - 1;
    const size_t mo = (size_t)mv * V;
    auto dst = [&](int a, int xx, int yy) {
        return fout + a * plane + ((size_t)yy * nx + xx) * k + mo;
    };
    Vec<T, V>::st(dst(0, x, y), f[0]);
    Vec<T, V>::st(dst(1, xp, y), f[1]);
    Vec<T, V>::st(dst(2, xm, y), f[2]);
    Vec<T, V>::st(dst(3, x, yp), f[3]);
    Vec<T, V>::st(dst(4, x, ym), f[4]);
    Vec<T, V>::st(dst(5, xp, yp), f[5]);
    Vec<T, V>::st(dst(6, xm, ym), f[6]);
    Vec<T, V>::st(dst(7, xp, ym), f[7]);
    Vec<T, V>::st(dst(8, xm, yp), f[8]);
}

template <typename T, int V, bool SHIFT>
__global__ void __launch_bounds__(256) lbm_step_kernel(const T* __restrict__ fin,
                                                       T* __restrict__ fout,
                                                       const T* __restrict__ force, int nx,
                                                       int ny, int k, T tau0, T cs18, T mu,
                                                       int* __restrict__ flags) {
    const long long total = (long long)nx * ny * (k / V);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    step_item<T, V, SHIFT>(fin, fout, force, nx, ny, k, tau0, cs18, mu, flags, t);
}

// ---- Many independent ensembles in one persistent launch -------------------
// Every experiment (its own lattice, members, parameters and state buffers)
// contributes nx * ny * k / V work items per step; a cooperative grid strides
// over the items of all experiments, then meets at a grid barrier before the
// next step. The barrier spins at most spin_limit rounds (with a short
// sleep): on timeout the block records it in status and the kernel stops.

template <typename T>
__device__ __forceinline__ void multi_item(const MultiExp& e, int step, long long t) {
    const int b = (e.cur + step) & 1;
    const T* fin = reinterpret_cast<const T*>(e.f[b]);
    T* fout = reinterpret_cast<T*>(e.f[b ^ 1]);
    const T* force = reinterpret_cast<const T*>(e.force);
    constexpr bool SHIFT = sizeof(T) == 4;
    if (e.V == 4)
        step_item<T, sizeof(T) == 4 ? 4 : 2, SHIFT>(fin, fout, force, e.nx, e.ny, e.k, (T)e.tau0,
                                                    (T)e.cs18, (T)e.mu, e.flags, t);
    else if (e.V == 2)
        step_item<T, 2, SHIFT>(fin, fout, force, e.nx, e.ny, e.k, (T)e.tau0, (T)e.cs18, (T)e.mu,
                               e.flags, t);
    else
        step_item<T, 1, SHIFT>(fin, fout, force, e.nx, e.ny, e.k, (T)e.tau0, (T)e.cs18, (T)e.mu,
                               e.flags, t);
}

// Sense-reversing grid barrier over gridDim.x blocks (count, gen in global
// memory, both zero before the launch), waiting for gridDim.x + absent
// arrivals: absent > 0 stands for participants that never arrive, so every
// wait runs out (the timeout path, exercised on purpose). Returns false on
// timeout.
__device__ bool grid_barrier(unsigned* count, unsigned* gen, int* status, long long spin_limit, unsigned absent) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned* vg = gen;
        const unsigned g = *vg;
        __threadfence();
        if (atomicAdd(count, 1u) == gridDim.x + absent - 1) {
            *count = 0u;
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            long long spins = 0;
            while (*vg == g) {
                if (++spins > spin_limit) {
                    atomicOr(status, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(512) lbm_multi_kernel(const MultiExp* __restrict__ ex, int nexp,
                                                        long long total, int nsteps,
                                                        unsigned* __restrict__ bar,
                                                        int* __restrict__ status, long long spin_limit,
                                                        unsigned absent) {
    __shared__ MultiExp se[kMaxMultiExp];
    for (int i = threadIdx.x; i < nexp; i += blockDim.x) se[i] = ex[i];
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int step = 0; step < nsteps; ++step) {
        int e = 0;
        for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
            while (t >= se[e].offset + se[e].items) ++e;  // items are in experiment order
            multi_item<T>(se[e], step, t - se[e].offset);
        }
        if (step + 1 < nsteps && !grid_barrier(bar, bar + 1, status, spin_limit, absent)) return;
    }
}

// Nudging (arXiv 2308.03972, Section 3.1): f_a <- f_a + gamma (f^eq_a(rho^, u^, v^) - f_a)
// for every member, with (rho^, u^, v^) the bilinear interpolation of the
// observations on the uniform periodic lattice (spacing px, py) to the cell.
template <typename T, int V, bool SHIFT>
__global__ void __launch_bounds__(256) nudge_kernel(T* __restrict__ f, int nx, int ny, int k,
                                                    int nox, int noy, const double* __restrict__ obs,
                                                    double gamma) {
    const int kv = k / V;
    const long long total = (long long)nx * ny * kv;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int mv = (int)(t % kv);
    const long long cell = t / kv;
    const int x = (int)(cell % nx), y = (int)(cell / nx);
    const int px = nx / nox, py = ny / noy;
    const int i0 = x / px, j0 = y / py;
    const double tx = (double)(x - i0 * px) / px, ty = (double)(y - j0 * py) / py;
    const int i1 = (i0 + 1 == nox) ? 0 : i0 + 1, j1 = (j0 + 1 == noy) ? 0 : j0 + 1;
    const size_t no = (size_t)nox * noy;
    const size_t c00 = (size_t)j0 * nox + i0, c01 = (size_t)j0 * nox + i1;
    const size_t c10 = (size_t)j1 * nox + i0, c11 = (size_t)j1 * nox + i1;
    const double w00 = (1.0 - tx) * (1.0 - ty), w01 = tx * (1.0 - ty);
    const double w10 = (1.0 - tx) * ty, w11 = tx * ty;
    double q[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        const double* g = obs + v * no;
        q[v] = w00 * g[c00] + w01 * g[c01] + w10 * g[c10] + w11 * g[c11];
    }
    const double rho = q[0], ux = q[1], uy = q[2];
    const double uu = ux * ux + uy * uy;
    T feq[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const double cu = d2q9_cx(a) * ux + d2q9_cy(a) * uy;
        const double w = d2q9_w(a);
        // f^eq (or f^eq - w) in FP64, then in the state's type.
        const double dev = w * ((rho - 1.0) + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
        feq[a] = SHIFT ? (T)dev : (T)(w + dev);
    }
    const size_t plane = (size_t)nx * ny * k;
    const size_t base = (size_t)cell * k + (size_t)mv * V;
    const T gm = (T)gamma;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        T v[V];
        Vec<T, V>::ld(f + a * plane + base, v);
#pragma unroll
        for (int j = 0; j < V; ++j) v[j] = v[j] + gm * (feq[a] - v[j]);
        Vec<T, V>::st(f + a * plane + base, v);
    }
}

template <typename T, int V, bool SHIFT>
cudaError_t launch_step_v(const T* fin, T* fout, const T* force, const LbmParams& p, int* flags,
                          cudaStream_t s) {
    const long long total = (long long)p.nx * p.ny * (p.k / V);
    const int bs = 256;
    const long long nb = (total + bs - 1) / bs;
    if (nb > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    lbm_step_kernel<T, V, SHIFT><<<(unsigned)nb, bs, 0, s>>>(fin, fout, force, p.nx, p.ny, p.k,
                                                             (T)p.tau0, (T)p.cs18, (T)p.mu, flags);
    return cudaGetLastError();
}

// Moments from the stored state: rho = sum f, u = sum f c / rho, in FP64.
template <typename T, bool SHIFT>
__global__ void moments_kernel(const T* __restrict__ f, int nx, int ny, int k,
                               double* __restrict__ rho, double* __restrict__ u,
                               double* __restrict__ v, int* __restrict__ flags) {
    const size_t n = (size_t)nx * ny * k;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double g[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = (double)f[a * n + i];
    double r = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        r += g[a];
        jx += d2q9_cx(a) * g[a];
        jy += d2q9_cy(a) * g[a];
    }
    if (SHIFT) r += 1.0;
    const double ux = jx / r, uy = jy / r;
    if (rho) rho[i] = r;
    if (u) u[i] = ux;
    if (v) v[i] = uy;
    if (!(ux * ux + uy * uy <= kUMax2) || !(r > 0.0)) atomicOr(flags, FLAG_DIVERGED);
}

// Ensemble-mean velocity: one warp per cell, lanes over members. A member's
// moments are taken in the precision of the stored state (FP64 here; the
// binary32 shifted state g = f - w has its own kernel below, whose moments
// match that state's storage error, ~1e-9 absolute in u); the member mean
// is summed in FP64.
template <typename T, bool SHIFT>
__global__ void mean_velocity_kernel(const T* __restrict__ f, int nx, int ny, int k,
                                     double* __restrict__ um, double* __restrict__ vm,
                                     int* __restrict__ flags) {
    const long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= (long long)nx * ny) return;
    const size_t n = (size_t)nx * ny * k;
    double su = 0.0, sv = 0.0;
    bool bad = false;
    for (int m = lane; m < k; m += 32) {
        const size_t i = (size_t)cell * k + m;
        T r = T(0), jx = T(0), jy = T(0);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const T g = f[a * n + i];
            r += g;
            jx += T(d2q9_cx(a)) * g;
            jy += T(d2q9_cy(a)) * g;
        }
        if (SHIFT) r += T(1);
        const T ux = jx / r, uy = jy / r;
        su += (double)ux;
        sv += (double)uy;
        // The divergence test in the state's precision, as the LBM step
        // makes it (0.25 is exact in binary32).
        bad |= !(ux * ux + uy * uy <= T(kUMax2)) || !(r > T(0));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        su += __shfl_xor_sync(0xffffffffu, su, o);
        sv += __shfl_xor_sync(0xffffffffu, sv, o);
    }
    if (lane == 0) {
        if (um) um[cell] = su / k;
        if (vm) vm[cell] = sv / k;
    }
    if (bad) atomicOr(flags, FLAG_DIVERGED);
}

// Knuth's TwoSum in binary32: s + e = a + b exactly.
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// (h, l) += (bh, bl) in double-binary32: the high parts by TwoSum, the low
// parts and the error in binary32.
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
    float s, e;
    two_sum_f(h, bh, s, e);
    h = s;
    l = __fadd_rn(l, __fadd_rn(bl, e));
}

// Ensemble-mean velocity of a binary32 state (g = f - w): each member's
// moments in binary32 (sum g, sum c g; rho = 1 + sum g), as the LBM step
// takes them, and the divergence test in binary32; their sum
// in double-binary32 (TwoSum per member and per step of the warp's
// butterfly), about as exact as an FP64 sum of the binary32 velocities,
// without FP64 work per member (GB300's FP64 rate is 1/64 of binary32).
// A block of 8 warps takes 8 cells; its first 16 threads form the 8 means
// of u and v in FP64.
__global__ void mean_velocity_f32_kernel(const float* __restrict__ f, int nx, int ny, int k,
                                         double* __restrict__ um, double* __restrict__ vm,
                                         int* __restrict__ flags) {
    __shared__ float2 part[2][8];  // (high, low) sums of u and v per cell of the block
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long ncell = (long long)nx * ny;
    const long long cell0 = (long long)blockIdx.x * 8;
    const long long cell = cell0 + w;
    const size_t n = (size_t)ncell * k;
    float uh = 0.0f, ul = 0.0f, vh = 0.0f, vl = 0.0f;
    bool bad = false;
    if (cell < ncell) {
        for (int m = lane; m < k; m += 32) {
            const size_t i = (size_t)cell * k + m;
            float r = 0.0f, jx = 0.0f, jy = 0.0f;
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                const float g = f[a * n + i];
                r += g;
                jx += float(d2q9_cx(a)) * g;
                jy += float(d2q9_cy(a)) * g;
            }
            r += 1.0f;
            const float ux = jx / r, uy = jy / r;
            df_add(uh, ul, ux, 0.0f);
            df_add(vh, vl, uy, 0.0f);
            bad |= !(ux * ux + uy * uy <= float(kUMax2)) || !(r > 0.0f);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ouh = __shfl_xor_sync(0xffffffffu, uh, o), oul = __shfl_xor_sync(0xffffffffu, ul, o);
        const float ovh = __shfl_xor_sync(0xffffffffu, vh, o), ovl = __shfl_xor_sync(0xffffffffu, vl, o);
        df_add(uh, ul, ouh, oul);
        df_add(vh, vl, ovh, ovl);
    }
    if (lane == 0) {
        part[0][w] = make_float2(uh, ul);
        part[1][w] = make_float2(vh, vl);
    }
    if (bad) atomicOr(flags, FLAG_DIVERGED);
    __syncthreads();
    if (threadIdx.x < 16) {
        const int q = threadIdx.x & 7, comp = threadIdx.x >> 3;
        double* out = comp ? vm : um;
        if (cell0 + q < ncell && out) {
            const float2 p = part[comp][q];
            out[cell0 + q] = ((double)p.x + (double)p.y) / k;
        }
    }
}

template <typename T, bool SHIFT>
__global__ void equilibrium_kernel(T* __restrict__ f, size_t n, const double* __restrict__ rho,
                                   const double* __restrict__ u, const double* __restrict__ v) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double r = rho ? rho[i] : 1.0;
    const double ux = u ? u[i] : 0.0, uy = v ? v[i] : 0.0;
    const double uu = ux * ux + uy * uy;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const double cu = d2q9_cx(a) * ux + d2q9_cy(a) * uy;
        const double w = d2q9_w(a);
        // f^eq - w = w ((rho - 1) + rho (3 cu + 9/2 cu^2 - 3/2 uu)).
        const double dev = w * ((r - 1.0) + r * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
        f[a * n + i] = SHIFT ? (T)dev : (T)(w + dev);
    }
}

// FP64 f [9][ny][nx][k] <-> stored representation (plane = ny nx k).
template <typename T, bool SHIFT>
__global__ void store_f_kernel(T* __restrict__ dst, const double* __restrict__ src, size_t n,
                               size_t plane) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = (int)(i / plane);
    dst[i] = SHIFT ? (T)(src[i] - d2q9_w(a)) : (T)src[i];
}

template <typename T, bool SHIFT>
__global__ void load_f_kernel(double* __restrict__ dst, const T* __restrict__ src, size_t n,
                              size_t plane) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = (int)(i / plane);
    dst[i] = SHIFT ? (double)src[i] + d2q9_w(a) : (double)src[i];
}

__global__ void store_force_f32(float* __restrict__ dst, const double* __restrict__ src, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)src[i];
}

inline unsigned blocks_for(size_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t launch_lbm_step_f64(const double* fin, double* fout, const double* force,
                                const LbmParams& p, int* flags, cudaStream_t s) {
    if (p.k % 2 == 0) return launch_step_v<double, 2, false>(fin, fout, force, p, flags, s);
    return launch_step_v<double, 1, false>(fin, fout, force, p, flags, s);
}

cudaError_t launch_lbm_step_f32(const float* gin, float* gout, const float* force,
                                const LbmParams& p, int* flags, cudaStream_t s) {
    if (p.k % 4 == 0) return launch_step_v<float, 4, true>(gin, gout, force, p, flags, s);
    if (p.k % 2 == 0) return launch_step_v<float, 2, true>(gin, gout, force, p, flags, s);
    return launch_step_v<float, 1, true>(gin, gout, force, p, flags, s);
}

cudaError_t launch_lbm_multi(const MultiExp* ex_dev, int nexp, long long total, int nsteps, int fp32,
                             int blocks, int threads, unsigned* bar, int* status, long long spin_limit,
                             unsigned absent, cudaStream_t s) {
    if (nexp < 1 || nexp > kMaxMultiExp || nsteps < 1 || blocks < 1 || spin_limit < 1) return cudaErrorInvalidValue;
    void* args[] = {(void*)&ex_dev, (void*)&nexp, (void*)&total, (void*)&nsteps, (void*)&bar,
                    (void*)&status, (void*)&spin_limit, (void*)&absent};
    cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (fp32)
        return cudaLaunchCooperativeKernel((const void*)lbm_multi_kernel<float>, dim3(blocks),
                                           dim3(threads), args, 0, s);
    return cudaLaunchCooperativeKernel((const void*)lbm_multi_kernel<double>, dim3(blocks),
                                       dim3(threads), args, 0, s);
}

int lbm_multi_max_blocks(int fp32, int threads) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    cudaError_t e = fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, lbm_multi_kernel<float>,
                                                                         threads, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, lbm_multi_kernel<double>,
                                                                         threads, 0);
    if (e != cudaSuccess) return 0;
    return per * sms;
}

cudaError_t launch_nudge(void* f, int fp32, int nx, int ny, int k, int nox, int noy,
                         const double* obs, double gamma, cudaStream_t s) {
    const int V = fp32 ? (k % 4 == 0 ? 4 : (k % 2 == 0 ? 2 : 1)) : (k % 2 == 0 ? 2 : 1);
    const long long total = (long long)nx * ny * (k / V);
    const long long nb = (total + 255) / 256;
    if (nb > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (fp32) {
        if (V == 4)
            nudge_kernel<float, 4, true><<<(unsigned)nb, 256, 0, s>>>((float*)f, nx, ny, k, nox, noy, obs, gamma);
        else if (V == 2)
            nudge_kernel<float, 2, true><<<(unsigned)nb, 256, 0, s>>>((float*)f, nx, ny, k, nox, noy, obs, gamma);
        else
            nudge_kernel<float, 1, true><<<(unsigned)nb, 256, 0, s>>>((float*)f, nx, ny, k, nox, noy, obs, gamma);
    } else {
        if (V == 2)
            nudge_kernel<double, 2, false><<<(unsigned)nb, 256, 0, s>>>((double*)f, nx, ny, k, nox, noy, obs, gamma);
        else
            nudge_kernel<double, 1, false><<<(unsigned)nb, 256, 0, s>>>((double*)f, nx, ny, k, nox, noy, obs, gamma);
    }
    return cudaGetLastError();
}

cudaError_t launch_moments(const void* f, int fp32, int nx, int ny, int k, double* rho,
                           double* u, double* v, int* flags, cudaStream_t s) {
    const size_t n = (size_t)nx * ny * k;
    if (n == 0) return cudaSuccess;
    if (fp32)
        moments_kernel<float, true><<<blocks_for(n, 256), 256, 0, s>>>(
            (const float*)f, nx, ny, k, rho, u, v, flags);
    else
        moments_kernel<double, false><<<blocks_for(n, 256), 256, 0, s>>>(
            (const double*)f, nx, ny, k, rho, u, v, flags);
    return cudaGetLastError();
}

cudaError_t launch_mean_velocity(const void* f, int fp32, int nx, int ny, int k, double* u,
                                 double* v, int* flags, cudaStream_t s) {
    const size_t threads = (size_t)nx * ny * 32;
    if (threads == 0) return cudaSuccess;
    if (fp32)
        mean_velocity_f32_kernel<<<blocks_for(threads, 256), 256, 0, s>>>((const float*)f, nx, ny, k, u, v,
                                                                          flags);
    else
        mean_velocity_kernel<double, false><<<blocks_for(threads, 256), 256, 0, s>>>(
            (const double*)f, nx, ny, k, u, v, flags);
    return cudaGetLastError();
}

cudaError_t launch_set_equilibrium(void* f, int fp32, int nx, int ny, int k, const double* rho,
                                   const double* u, const double* v, cudaStream_t s) {
    const size_t n = (size_t)nx * ny * k;
    if (n == 0) return cudaSuccess;
    if (fp32)
        equilibrium_kernel<float, true><<<blocks_for(n, 256), 256, 0, s>>>((float*)f, n, rho, u, v);
    else
        equilibrium_kernel<double, false><<<blocks_for(n, 256), 256, 0, s>>>((double*)f, n, rho, u,
                                                                            v);
    return cudaGetLastError();
}

cudaError_t launch_store_f(void* f, int fp32, const double* src, size_t n, cudaStream_t s) {
    const size_t plane = n / 9;
    if (n == 0) return cudaSuccess;
    if (fp32)
        store_f_kernel<float, true><<<blocks_for(n, 256), 256, 0, s>>>((float*)f, src, n, plane);
    else
        store_f_kernel<double, false><<<blocks_for(n, 256), 256, 0, s>>>((double*)f, src, n, plane);
    return cudaGetLastError();
}

cudaError_t launch_load_f(const void* f, int fp32, double* dst, size_t n, cudaStream_t s) {
    const size_t plane = n / 9;
    if (n == 0) return cudaSuccess;
    if (fp32)
        load_f_kernel<float, true><<<blocks_for(n, 256), 256, 0, s>>>(dst, (const float*)f, n, plane);
    else
        load_f_kernel<double, false><<<blocks_for(n, 256), 256, 0, s>>>(dst, (const double*)f, n,
                                                                       plane);
    return cudaGetLastError();
}

cudaError_t launch_store_force(void* dst, int fp32, const double* src, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (fp32) {
        store_force_f32<<<blocks_for(n, 256), 256, 0, s>>>((float*)dst, src, n);
        return cudaGetLastError();
    }
    return cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

}  // namespace lbmgpu
