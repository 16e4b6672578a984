// LETKF kernels of the LBM-LETKF library (sm_103a).
//
// K2 observation operator and ensemble observation statistics
//   (arXiv 2308.03972, Section 3: y = H x = (u, v) at the observation points;
//    Section 3.2: ybar, dY = Y - ybar, innovation d = y^o - ybar).
// K3 per-grid-point analysis, one warp per grid point
//   (Section 3.2: w-bar, P-tilde, delta-W = [(k-1) P-tilde]^{1/2}, the
//    update x^a_m = xbar + dX (w-bar + delta-W_m); R-localisation with the
//    Gaspari-Cohn weight; multiplicative inflation beta).
//
// The analysis uses whichever of two exactly equivalent forms is smaller.
// With Yh = diag(sqrt(rho)) dY_loc (p x k), C = a I + Yh^T Yh, a = (k-1)/beta:
//  * ensemble space (p >= k): eigendecompose the k x k matrix C as printed;
//  * observation space (p < k): eigendecompose the p x p matrix
//    A = Yh Yh^T = U S U^T. Then w-bar = Yh^T (a I + A)^{-1} d-hat and
//    C^{-1/2} = a^{-1/2} I + Yh^T U diag(g(s)) U^T Yh with
//    g(s) = ((a + s)^{-1/2} - a^{-1/2}) / s, so
//    x^a_m = xbar + dX Yh^T v + sqrt(beta) dx_m + sqrt(k-1) (dX Yh^T) U g U^T yh_m.
//    A is gathered from the global Gram dY dY^T, formed once per analysis.
// The symmetric eigensolve is a cyclic Jacobi method (Golub & Van Loan,
// Section 8.5) with the round-robin parallel ordering, in FP64, on a
// matrix held in shared memory, one column per lane.
#include <cmath>
#include <cstdint>
#include <cstring>

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "lbm_internal.cuh"
#include "letkf_device.cuh"
#include "tc_ptx.cuh"

namespace lbmgpu {
namespace {

constexpr int NMAX = 128;  // largest local eigenproblem of the mixed-precision analysis
constexpr int NMID = 64;   // largest held wholly in shared memory; the FP64 analysis' limit
constexpr int NREG = 32;   // largest one handled by the register Jacobi
constexpr int kMaxSweeps = 30;

// ------------------------------------------------------------------ K2
template <typename T, bool SHIFT>
__global__ void __launch_bounds__(128) observe_kernel(const T* __restrict__ f, int nx, int ny,
                                                      int k, int nvar, const int* __restrict__ ix,
                                                      const int* __restrict__ iy,
                                                      const double* __restrict__ yo,
                                                      double* __restrict__ dY,
                                                      double* __restrict__ d) {
    // One block per observation point: the nvar observed variables (u, v,
    // and rho when nvar = 3) of every member, their ensemble means, the
    // perturbations and the innovations.
    extern __shared__ double sh[];  // y[3][k], red[3 * 4]
    double* yv = sh;
    double* red = sh + 3 * k;
    const int j = blockIdx.x;
    const size_t plane = (size_t)nx * ny * k;
    const size_t base = ((size_t)iy[j] * nx + ix[j]) * k;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int m = threadIdx.x; m < k; m += blockDim.x) {
        double r = SHIFT ? 1.0 : 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const double g = (double)f[a * plane + base + m];
            r += g;
            jx += d2q9_cx(a) * g;
            jy += d2q9_cy(a) * g;
        }
        const double val[3] = {jx / r, jy / r, r};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            yv[q * k + m] = val[q];
            acc[q] += val[q];
        }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double t = warp_sum(acc[q]);
        if (l == 0) red[4 * q + w] = t;
    }
    __syncthreads();
    for (int q = 0; q < nvar; ++q) {
        const double mean = ((red[4 * q] + red[4 * q + 1]) + (red[4 * q + 2] + red[4 * q + 3])) / k;
        for (int m = threadIdx.x; m < k; m += blockDim.x)
            dY[(size_t)(nvar * j + q) * k + m] = yv[q * k + m] - mean;
        if (threadIdx.x == 0) d[nvar * j + q] = yo[nvar * j + q] - mean;
    }
}

// G = dY dY^T (nobs x nobs), one thread per entry.
__global__ void obs_gram_kernel(const double* __restrict__ dY, int nobs, int k,
                                double* __restrict__ G) {
    const int i = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nobs) return;
    const double* a = dY + (size_t)i * k;
    const double* b = dY + (size_t)j * k;
    double s = 0.0;
    for (int m = 0; m < k; ++m) s += a[m] * b[m];
    G[(size_t)i * nobs + j] = s;
}

// Sweep count of one eigensolve into the optional histogram (bin 31: 31 or
// more sweeps, or the sweep cap).
__device__ __forceinline__ void record_sweeps(const ObsParams& o, int sweeps, int lane) {
    if (o.sweep_hist && lane == 0) atomicAdd(&o.sweep_hist[(sweeps < 0 || sweeps > 31) ? 31 : sweeps], 1);
}

// Local observation set of grid point (x, y), in increasing point order:
// point j is in range when r / d_cut < 2 and G(r / d_cut) > 0; it gives the
// nvar scalars nvar*j + q (u, v, rho) with sqrt(rho-tilde) = sqrt(G) / sigma_q.
// Returns the number of scalars p; at most cap of them are stored.
// Warp-cooperative.
__device__ int local_set(const ObsParams& o, int x, int y, int nx, int ny, double d_cut, int lane,
                         int* lidx, double* lsq, int cap) {
    int count = 0;
    const long long lim2 = support_lim2(d_cut);
    for (int j0 = 0; j0 < o.npts; j0 += 32) {
        const int j = j0 + lane;
        bool in = false;
        double g = 0.0;
        if (j < o.npts) {
            const int dx = min_image(o.ix[j] - x, nx);
            const int dy = min_image(o.iy[j] - y, ny);
            // Integer prefilter well outside the support (r > 2 d_cut + 1);
            // the decision itself is r / d_cut < 2 in FP64.
            if (dist2(dx, dy) <= lim2) {
                const double d2 = (double)dx * dx + (double)dy * dy;
                const double dist = sqrt(d2) / d_cut;
                if (dist < 2.0) {
                    g = gaspari_cohn(dist);
                    in = g > 0.0;
                }
            }
        }
        const unsigned bal = __ballot_sync(kFull, in);
        if (in) {
            const int pos = o.nvar * (count + __popc(bal & ((1u << lane) - 1u)));
            const double sg = sqrt(g);
            // Entries past the capacity are counted, not stored; the caller
            // reports the point as too large.
            if (pos + o.nvar <= cap) {
                lidx[pos] = o.nvar * j;
                lidx[pos + 1] = o.nvar * j + 1;
                lsq[pos] = sg / o.sigma_u;
                lsq[pos + 1] = sg / o.sigma_v;
                if (o.nvar == 3) {
                    lidx[pos + 2] = 3 * j + 2;
                    lsq[pos + 2] = sg / o.sigma_r;
                }
            }
        }
        count += __popc(bal);
    }
    __syncwarp();
    return o.nvar * count;
}

// ------------------------------------------------------------------ K3, FP64
// Apply body(c) to the columns c a thread owns: c = lane when every problem
// fits one lane per column (WIDE = false), else c = t, t + 32 NW, ... for
// thread t of NW warps.
template <bool WIDE, int NW = 1, typename F>
__device__ __forceinline__ void for_cols(int t, int n, F&& body) {
    if (WIDE) {
        for (int c = t; c < n; c += 32 * NW) body(c);
    } else if (t < n) {
        body(t);
    }
}

// Barrier of the NW warps that share a grid point.
template <int NW>
__device__ __forceinline__ void point_sync() {
    if (NW == 1)
        __syncwarp();
    else
        __syncthreads();
}

__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

// Cyclic Jacobi (R = double) on the symmetric n x n matrix A (shared memory, row
// stride ld), round-robin order (position 0 fixed, the others rotating), one
// warp. Only what symmetry requires is updated: each rotated pair's 2 x 2
// diagonal block analytically (a_pp - t a_pq, a_qq + t a_pq, 0), the
// off-diagonal 2 x 2 blocks (P, Q), P < Q, as J_P^T X J_Q (mirrored), and the
// rows of U. A rotation is skipped when |a_pq| <= rel ||A||_F; the solve ends
// after a sweep without one. n <= 64 (at most 32 pairs). Returns the number
// of sweeps (the last one rotating nothing), or -1 if max_sweeps was reached.
template <typename R>
__device__ int jacobi_sym_warp(R* A, R* U, int n, int ld, int lane, R* rc, R* rs, int* rp,
                                int* rq, R rel, int max_sweeps) {
    const int np = n + (n & 1);
    const int half = np / 2;
    const int nb = half * (half - 1) / 2;
    R fro = R(0);
    for (int c = lane; c < n; c += 32)
        for (int i = 0; i < n; ++i) fro += A[i * ld + c] * A[i * ld + c];
    fro = warp_sum(fro);
    const R thresh = rel * sqrt(fro);
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        bool any_sweep = false;
        for (int r = 0; r + 1 < np; ++r) {
            bool rot = false;
            if (lane < half) {
                const int pa = lane, pb = np - 1 - lane;
                const int P = pa == 0 ? 0 : 1 + (pa - 1 + r) % (np - 1);
                const int Q = 1 + (pb - 1 + r) % (np - 1);
                const int p = P < Q ? P : Q, q = P < Q ? Q : P;
                R c = R(1), sn = R(0);
                if (q < n) {
                    const R apq = A[p * ld + q];
                    if (fabs(apq) > thresh) {
                        // t = phi / (theta + sgn(theta) sqrt(theta^2 + phi^2)),
                        // theta = a_qq - a_pp, phi = 2 a_pq: the smaller root of
                        // t^2 + 2 (theta / phi) t - 1 = 0.
                        const R app = A[p * ld + p], aqq = A[q * ld + q];
                        const R th = aqq - app, ph = R(2) * apq;
                        const R rr = sqrt(th * th + ph * ph);
                        const R t = ph / (th >= R(0) ? th + rr : th - rr);
                        c = rsq(R(1) + t * t);
                        sn = t * c;
                        rot = true;
                        // Diagonal block of the pair, analytically.
                        A[p * ld + p] = app - t * apq;
                        A[q * ld + q] = aqq + t * apq;
                        A[p * ld + q] = R(0);
                        A[q * ld + p] = R(0);
                    }
                }
                rp[lane] = p;
                rq[lane] = q;
                rc[lane] = c;
                rs[lane] = sn;
            }
            const unsigned any = __ballot_sync(kFull, rot);
            __syncwarp();
            if (any == 0) continue;
            any_sweep = true;
            // Off-diagonal blocks (P, Q), P < Q, of the pairs of this round.
            for (int bb = lane; bb < nb; bb += 32) {
                int P = 0, Q = bb;
                while (Q >= half - 1 - P) {
                    Q -= half - 1 - P;
                    ++P;
                }
                Q += P + 1;
                const bool rP = (any >> P) & 1u, rQ = (any >> Q) & 1u;
                if (!rP && !rQ) continue;
                const int pP = rp[P], qP = rq[P], pQ = rp[Q], qQ = rq[Q];
                // For odd n the padding player n is always the q of its pair
                // (it is the largest index); its pair does not rotate, and its
                // row and column do not exist: they read as zero and are not
                // written, while the real member of that pair is still turned
                // by the other pair's rotation.
                const bool vP = qP < n, vQ = qQ < n;
                const R cP = rc[P], sP = rs[P], cQ = rc[Q], sQ = rs[Q];
                const R x00 = A[pP * ld + pQ];
                const R x01 = vQ ? A[pP * ld + qQ] : R(0);
                const R x10 = vP ? A[qP * ld + pQ] : R(0);
                const R x11 = (vP && vQ) ? A[qP * ld + qQ] : R(0);
                // J_P^T X: rows p, q.
                const R y00 = cP * x00 - sP * x10, y01 = cP * x01 - sP * x11;
                const R y10 = sP * x00 + cP * x10, y11 = sP * x01 + cP * x11;
                // (J_P^T X) J_Q: columns p, q.
                const R z00 = cQ * y00 - sQ * y01, z01 = sQ * y00 + cQ * y01;
                const R z10 = cQ * y10 - sQ * y11, z11 = sQ * y10 + cQ * y11;
                A[pP * ld + pQ] = z00;
                A[pQ * ld + pP] = z00;
                if (vQ) {
                    A[pP * ld + qQ] = z01;
                    A[qQ * ld + pP] = z01;
                }
                if (vP) {
                    A[qP * ld + pQ] = z10;
                    A[pQ * ld + qP] = z10;
                }
                if (vP && vQ) {
                    A[qP * ld + qQ] = z11;
                    A[qQ * ld + qP] = z11;
                }
            }
            // U <- U J: rotate column pairs; lanes own rows.
            for (int row = lane; row < n; row += 32) {
                for (int t = 0; t < half; ++t) {
                    if (!((any >> t) & 1u)) continue;
                    const int p = rp[t], q = rq[t];
                    const R c = rc[t], sn = rs[t];
                    const R up = U[row * ld + p], uq = U[row * ld + q];
                    U[row * ld + p] = c * up - sn * uq;
                    U[row * ld + q] = sn * up + c * uq;
                }
            }
            __syncwarp();
        }
        if (!any_sweep) return sweep + 1;
    }
    return -1;
}

// The cyclic Jacobi of jacobi_sym_warp (same rotations, same round-robin
// order) for 33..128 (up to 64 pairs) by a block of NT = 256 threads: the
// first 64 threads choose and apply the rotations of a round's pairs; then
// every thread updates off-diagonal blocks and half a row of U (two threads
// per row, 32 pairs each). The mask of rotated pairs alternates between two
// shared slots by round parity, so it is not overwritten before every warp
// has read it. mask: 4 words, red: NT / 32 floats. Binary32.
template <int NT>
__device__ int jacobi_sym_block(float* A, float* U, int n, int ld, float* rc, float* rs, int* rp, int* rq,
                                unsigned* mask, float* red, float rel, int max_sweeps) {
    static_assert(NT == 256, "two threads per row of U for n <= 128");
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int np = n + (n & 1);
    const int half = np / 2;
    const int nb = half * (half - 1) / 2;
    float fro = 0.0f;
    for (int e = tid; e < n * n; e += NT) {
        const float v = A[(e / n) * ld + e % n];
        fro += v * v;
    }
    fro = warp_sum(fro);
    if (lane == 0) red[w] = fro;
    __syncthreads();
    fro = 0.0f;
    for (int q = 0; q < NT / 32; ++q) fro += red[q];
    const float thresh = rel * sqrtf(fro);
    const int urow = tid >> 1, ut0 = (tid & 1) * 32;  // U: this thread's row and first pair
    int parity = 0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        bool any_sweep = false;
        for (int r = 0; r + 1 < np; ++r) {
            unsigned* mk = mask + 2 * parity;
            parity ^= 1;
            if (w < 2) {
                const int pr = tid;
                bool rot = false;
                if (pr < half) {
                    const int pa = pr, pb = np - 1 - pr;
                    const int P = pa == 0 ? 0 : 1 + (pa - 1 + r) % (np - 1);
                    const int Q = 1 + (pb - 1 + r) % (np - 1);
                    const int p = P < Q ? P : Q, q = P < Q ? Q : P;
                    float c = 1.0f, sn = 0.0f;
                    if (q < n) {
                        const float apq = A[p * ld + q];
                        if (fabsf(apq) > thresh) {
                            const float app = A[p * ld + p], aqq = A[q * ld + q];
                            const float th = aqq - app, ph = 2.0f * apq;
                            const float rr = sqrtf(th * th + ph * ph);
                            const float t = ph / (th >= 0.0f ? th + rr : th - rr);
                            c = rsqrtf(1.0f + t * t);
                            sn = t * c;
                            rot = true;
                            A[p * ld + p] = app - t * apq;
                            A[q * ld + q] = aqq + t * apq;
                            A[p * ld + q] = 0.0f;
                            A[q * ld + p] = 0.0f;
                        }
                    }
                    rp[pr] = p;
                    rq[pr] = q;
                    rc[pr] = c;
                    rs[pr] = sn;
                }
                const unsigned bal = __ballot_sync(kFull, rot);
                if (lane == 0) mk[w] = bal;
            }
            __syncthreads();
            const unsigned long long any = mk[0] | ((unsigned long long)mk[1] << 32);
            if (any == 0) continue;
            any_sweep = true;
            // Off-diagonal blocks (P, Q), P < Q: block bb is entry Q0 of row
            // P of the pair matrix's upper triangle; a thread advances its
            // previous (P, Q0) by NT blocks.
            int P = 0, Q0 = 0;
            for (int bb = tid; bb < nb; bb += NT) {
                if (bb == tid) {
                    Q0 = bb;
                } else {
                    Q0 += NT;
                }
                while (Q0 >= half - 1 - P) {
                    Q0 -= half - 1 - P;
                    ++P;
                }
                const int Q = P + 1 + Q0;
                if (!((any >> P) & 1ull) && !((any >> Q) & 1ull)) continue;
                const int pP = rp[P], qP = rq[P], pQ = rp[Q], qQ = rq[Q];
                // The padding player of odd n (always a q) reads as zero and
                // is not written.
                const bool vP = qP < n, vQ = qQ < n;
                const float cP = rc[P], sP = rs[P], cQ = rc[Q], sQ = rs[Q];
                const float x00 = A[pP * ld + pQ];
                const float x01 = vQ ? A[pP * ld + qQ] : 0.0f;
                const float x10 = vP ? A[qP * ld + pQ] : 0.0f;
                const float x11 = (vP && vQ) ? A[qP * ld + qQ] : 0.0f;
                const float y00 = cP * x00 - sP * x10, y01 = cP * x01 - sP * x11;
                const float y10 = sP * x00 + cP * x10, y11 = sP * x01 + cP * x11;
                const float z00 = cQ * y00 - sQ * y01, z01 = sQ * y00 + cQ * y01;
                const float z10 = cQ * y10 - sQ * y11, z11 = sQ * y10 + cQ * y11;
                A[pP * ld + pQ] = z00;
                A[pQ * ld + pP] = z00;
                if (vQ) {
                    A[pP * ld + qQ] = z01;
                    A[qQ * ld + pP] = z01;
                }
                if (vP) {
                    A[qP * ld + pQ] = z10;
                    A[pQ * ld + qP] = z10;
                }
                if (vP && vQ) {
                    A[qP * ld + qQ] = z11;
                    A[qQ * ld + qP] = z11;
                }
            }
            // U <- U J on this thread's half row.
            if (urow < n) {
                const int t1 = ut0 + 32 < half ? ut0 + 32 : half;
                for (int t = ut0; t < t1; ++t) {
                    if (!((any >> t) & 1ull)) continue;
                    const int p = rp[t], q = rq[t];
                    const float c = rc[t], sn = rs[t];
                    const float up = U[urow * ld + p], uq = U[urow * ld + q];
                    U[urow * ld + p] = c * up - sn * uq;
                    U[urow * ld + q] = sn * up + c * uq;
                }
            }
            __syncthreads();
        }
        if (!any_sweep) return sweep + 1;
    }
    return -1;
}

// Shared memory of the FP64 analysis kernel for problems up to NM.
template <int NM>
struct AnaSmem {
    static constexpr int kLd = NM + 1;
    double* A;     // [NM][kLd]
    double* U;     // [NM][kLd]
    double* dX;    // [9][k]
    double* xbar;  // [16]
    double* lsq;   // [nl] sqrt of the localised inverse error variance
    double* ldh;   // [nl] sqrt(rho) * d
    double* v1;    // [NM]
    double* v2;    // [NM]
    double* v3;    // [NM]
    double* v4;    // [NM]
    double* v5;    // [NM]
    double* Z;     // [9][NM]
    double* B;     // [9][NM]
    double* zv;    // [16]
    double* rc;    // [NM / 2]
    double* rs;    // [NM / 2]
    int* rp;       // [NM / 2]
    int* rq;       // [NM / 2]
    int* lidx;     // [nl]

    __host__ __device__ static size_t bytes(int k, int nl) {
        const size_t d = 2 * (size_t)NM * kLd + 9 * (size_t)k + 16 + 2 * (size_t)nl + 5 * NM +
                         18 * (size_t)NM + 16 + NM;
        return d * sizeof(double) + (size_t)(NM + nl) * sizeof(int);
    }
    __device__ void carve(unsigned char* raw, int k, int nl) {
        double* p = reinterpret_cast<double*>(raw);
        A = p;
        p += NM * kLd;
        U = p;
        p += NM * kLd;
        dX = p;
        p += 9 * k;
        xbar = p;
        p += 16;
        lsq = p;
        p += nl;
        ldh = p;
        p += nl;
        v1 = p;
        p += NM;
        v2 = p;
        p += NM;
        v3 = p;
        p += NM;
        v4 = p;
        p += NM;
        v5 = p;
        p += NM;
        Z = p;
        p += 9 * NM;
        B = p;
        p += 9 * NM;
        zv = p;
        p += 16;
        rc = p;
        p += NM / 2;
        rs = p;
        p += NM / 2;
        int* ip = reinterpret_cast<int*>(p);
        rp = ip;
        ip += NM / 2;
        rq = ip;
        ip += NM / 2;
        lidx = ip;
    }
};

// Observation-space transform and update of one grid point (FP64), after
// the eigensolve: A holds S = U^T A U (nearly diagonal), U the basis;
// lidx, lsq, ldh the n local scalars (zero weight on padding), dX and
// xbar the staged state; the result goes to fc. One warp.
template <int NM>
__device__ void fp64_obs_update(AnaSmem<NM>& sm, double* __restrict__ fc, size_t plane, int k, int n,
                                double aa, double beta, const ObsParams& o, int lane) {
    constexpr int ld = AnaSmem<NM>::kLd;
    double* A = sm.A;
    double* U = sm.U;
    // With u_i = sqrt(a + s_ii), h(s) = 1/(a+s) and g(s) = ((a+s)^{-1/2} - a^{-1/2}) / s:
    //   h(S)_ii = 1/u_i^2, h(S)_ij = -s_ij / (u_i^2 u_j^2),
    //   g(S)_ii = -alpha_i / r, g(S)_ij = s_ij (u_i+u_j+r) alpha_i alpha_j / (r (u_i+u_j)),
    // alpha_i = 1 / (u_i (u_i + r)), r = sqrt(a).
    const double rr = sqrt(aa);
    const double ir = 1.0 / rr;
    for (int c = lane; c < n; c += 32) {
        const double sii = A[c * ld + c];
        const double u = sqrt(aa + sii);
        sm.v3[c] = u;
        sm.v4[c] = 1.0 / (aa + sii);      // h_i
        sm.v5[c] = 1.0 / (u * (u + rr));  // alpha_i
        double t = 0.0;
        for (int l = 0; l < n; ++l) t += U[l * ld + c] * sm.ldh[l];
        sm.v1[c] = t;  // t1 = U^T d-hat
    }
    __syncwarp();
    for (int c = lane; c < n; c += 32) {
        double t = 0.0;
        for (int j = 0; j < n; ++j)
            if (j != c) t += A[c * ld + j] * (sm.v4[j] * sm.v1[j]);
        sm.v2[c] = sm.v4[c] * (sm.v1[c] - t);  // t2 = h(S) t1
    }
    __syncwarp();
    for (int c = lane; c < n; c += 32) {
        // g(S), column c, over S (each column is read and written by one lane).
        const double ui = sm.v3[c];
        const double ai = sm.v5[c];
        for (int j = 0; j < n; ++j) {
            const double uj = sm.v3[j];
            A[j * ld + c] = (j == c) ? -ai * ir : A[j * ld + c] * (ui + uj + rr) * ai * sm.v5[j] * ir / (ui + uj);
        }
        double t = 0.0;
        for (int l = 0; l < n; ++l) t += U[c * ld + l] * sm.v2[l];
        sm.v1[c] = t;  // v = U t2 = (a I + A)^{-1} d-hat
        // Z = dX Yh^T, column c.
        const double* row = o.dY + (size_t)sm.lidx[c] * k;
        double acc[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) acc[a] = 0.0;
        for (int m = 0; m < k; ++m) {
            const double dy = row[m];
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] += sm.dX[a * k + m] * dy;
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) sm.Z[a * NM + c] = sm.lsq[c] * acc[a];
    }
    __syncwarp();
    // zv = Z v (= dX w-bar); B = Z U.
    if (lane < 9) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += sm.Z[lane * NM + i] * sm.v1[i];
        sm.zv[lane] = s;
    }
    for (int c = lane; c < n; c += 32)
        for (int a = 0; a < 9; ++a) {
            double s = 0.0;
            for (int l = 0; l < n; ++l) s += sm.Z[a * NM + l] * U[l * ld + c];
            sm.B[a * NM + c] = s;
        }
    __syncwarp();
    // Z <- (Z U) g(S).
    for (int c = lane; c < n; c += 32)
        for (int a = 0; a < 9; ++a) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += sm.B[a * NM + j] * A[j * ld + c];
            sm.Z[a * NM + c] = s;
        }
    __syncwarp();
    // B <- sqrt(k-1) Z U^T diag(sqrt(rho)), ready to meet dY.
    const double sk = sqrt((double)(k - 1));
    for (int c = lane; c < n; c += 32)
        for (int a = 0; a < 9; ++a) {
            double s = 0.0;
            for (int l = 0; l < n; ++l) s += sm.Z[a * NM + l] * U[c * ld + l];
            sm.B[a * NM + c] = sk * sm.lsq[c] * s;
        }
    __syncwarp();
    const double sb = sqrt(beta);
    for (int m = lane; m < k; m += 32) {
        double acc[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) acc[a] = sm.xbar[a] + sm.zv[a] + sb * sm.dX[a * k + m];
        for (int i = 0; i < n; ++i) {
            const double dy = o.dY[(size_t)sm.lidx[i] * k + m];
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] += sm.B[a * NM + i] * dy;
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) fc[a * plane + m] = acc[a];
    }
}

// FP64 analysis, one warp per grid point, local problems up to NM (32 or 64;
// lanes own columns c = lane, lane + 32, ...).
template <int NM>
__global__ void __launch_bounds__(32) analyze_fp64_kernel(double* __restrict__ f, int nx, int ny,
                                                          int k, ObsParams o, double d_cut,
                                                          double beta, int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int ld = AnaSmem<NM>::kLd;
    const int nobs = o.nvar * o.npts;
    const int cap = o.plmax > 0 ? o.plmax : nobs;
    AnaSmem<NM> sm;
    sm.carve(smem_raw, k, cap);
    const int lane = threadIdx.x;
    const int cell = blockIdx.x;
    const int x = cell % nx, y = cell / nx;
    const size_t plane = (size_t)nx * ny * k;
    double* fc = f + (size_t)cell * k;

    // Ensemble mean and perturbations of the nine components.
    for (int a = 0; a < 9; ++a) {
        double s = 0.0;
        for (int m = lane; m < k; m += 32) {
            const double xv = fc[a * plane + m];
            sm.dX[a * k + m] = xv;
            s += xv;
        }
        const double mean = warp_sum(s) / k;
        for (int m = lane; m < k; m += 32) sm.dX[a * k + m] -= mean;
        if (lane == 0) sm.xbar[a] = mean;
    }

    const int p = local_set(o, x, y, nx, ny, d_cut, lane, sm.lidx, sm.lsq, cap);
    if (p > cap) {
        if (lane == 0) atomicOr(flags, FLAG_TOOLARGE);
        return;
    }
    for (int i = lane; i < p; i += 32) sm.ldh[i] = sm.lsq[i] * o.d[sm.lidx[i]];
    __syncwarp();

    if (p == 0) {
        // No observation in range: x^a_m = xbar + sqrt(beta) dx_m.
        const double sb = sqrt(beta);
        for (int a = 0; a < 9; ++a)
            for (int m = lane; m < k; m += 32) fc[a * plane + m] = sm.xbar[a] + sb * sm.dX[a * k + m];
        return;
    }
    const bool obs_space = p < k;
    const int n = obs_space ? p : k;
    if (n > NM) {
        if (lane == 0) atomicOr(flags, FLAG_TOOLARGE);
        return;
    }
    const double aa = (k - 1) / beta;
    double* A = sm.A;
    double* U = sm.U;

    if (obs_space) {
        // A = Yh Yh^T gathered from the global Gram.
        for (int c = lane; c < n; c += 32) {
            const int oc = sm.lidx[c];
            const double sc = sm.lsq[c];
            for (int i = 0; i < n; ++i) A[i * ld + c] = sm.lsq[i] * o.G[(size_t)sm.lidx[i] * nobs + oc] * sc;
        }
    } else {
        // C = a I + Yh^T Yh and b = Yh^T d-hat, column c.
        for (int c = lane; c < n; c += 32) {
            for (int i = 0; i < n; ++i) {
                double s = 0.0;
                for (int l = 0; l < p; ++l) {
                    const double* row = o.dY + (size_t)sm.lidx[l] * k;
                    s += sm.lsq[l] * sm.lsq[l] * row[i] * row[c];
                }
                A[i * ld + c] = s + (i == c ? aa : 0.0);
            }
            double bj = 0.0;
            for (int l = 0; l < p; ++l) bj += sm.lsq[l] * o.dY[(size_t)sm.lidx[l] * k + c] * sm.ldh[l];
            sm.v3[c] = bj;
        }
    }
    for (int c = lane; c < n; c += 32)
        for (int i = 0; i < n; ++i) U[i * ld + c] = (i == c) ? 1.0 : 0.0;
    __syncwarp();

    // Observation space: stop once the off-diagonal is below 3e-8 ||A||_F and
    // take the matrix functions to first order in it (Daleckii-Krein; the
    // neglected second-order term is (3e-8 ||A||_F / (a + s))^2, below
    // ~1e-11 relative even for ||A||_F ~ 100 a, i.e. ~1e-13 of the state).
    // Ensemble space converges fully and uses the diagonal directly.
    const int sweeps = jacobi_sym_warp<double>(A, U, n, ld, lane, sm.rc, sm.rs, sm.rp, sm.rq,
                                               obs_space ? 3e-8 : 1e-18, kMaxSweeps);
    if (sweeps < 0 && lane == 0) atomicOr(flags, FLAG_NOCONV);
    record_sweeps(o, sweeps, lane);
    __syncwarp();

    if (obs_space) {
        fp64_obs_update<NM>(sm, fc, plane, k, n, aa, beta, o, lane);
    } else {
        // lam = diag; w-bar = U diag(1/lam) U^T b; T = W + w-bar 1^T with
        // W = sqrt(k-1) U diag(lam^{-1/2}) U^T, stored over A.
        for (int c = lane; c < n; c += 32) {
            const double lam = A[c * ld + c];
            double t = 0.0;
            for (int l = 0; l < n; ++l) t += U[l * ld + c] * sm.v3[l];
            sm.v1[c] = t / lam;
            sm.v2[c] = sqrt((double)(k - 1) / lam);
        }
        __syncwarp();
        for (int c = lane; c < n; c += 32) {
            double t = 0.0;
            for (int l = 0; l < n; ++l) t += U[c * ld + l] * sm.v1[l];
            sm.v4[c] = t;  // w-bar
        }
        __syncwarp();
        for (int c = lane; c < n; c += 32)
            for (int i = 0; i < n; ++i) {
                double s = 0.0;
                for (int l = 0; l < n; ++l) s += U[i * ld + l] * sm.v2[l] * U[c * ld + l];
                A[i * ld + c] = s + sm.v4[i];
            }
        __syncwarp();
        for (int m = lane; m < k; m += 32) {
            for (int a = 0; a < 9; ++a) {
                double s = 0.0;
                for (int j = 0; j < k; ++j) s += sm.dX[a * k + j] * A[j * ld + m];
                fc[a * plane + m] = sm.xbar[a] + s;
            }
        }
    }
}

// FP64 analysis warm-started from a binary32 basis: the run path of a
// double-precision context, one warp per grid point. The binary32 Jacobi
// over the run (kernel J in letkf_runs.cu) leaves per point a basis Y of the
// run's union of local scalars (NS x NS, row-major, Y_ic = component i of
// vector c). Union scalars outside this point's support have weight zero, so
// their rows and columns of A vanish and the result is that of the point's
// own local set (exactly, in exact arithmetic). Then:
//  1. Y1 = Y (I - E/2) with E = Y^T Y - I: Y is orthonormal to ~1e-7 in
//     binary32, Y1 to ~1e-13. E and the correction Y E run on the binary32
//     units (double-binary32 sums of exact products for E); Y1 is FP64.
// In FP64:
//  2. A' = Y1^T A Y1 (symmetrised), diagonal to ~1e-6 of ||A||.
//  3. The FP64 cyclic Jacobi of the cold path from A' with U = Y1 at the
//     start and the same stopping rule (3e-8 ||A||_F): one rotating sweep
//     where a cold start needs five or six.
//  4. The FP64 transform and update of the cold path.
// The eigenpairs are FP64's; the binary32 basis is only where the FP64
// Jacobi starts.
template <int NS>
__global__ void __launch_bounds__(32) run_fp64_kernel(double* __restrict__ f, int nx, int ny, int k, ObsParams o,
                                                      double d_cut, double beta, int R, int run0,
                                                      const float* __restrict__ Yg, const float* __restrict__ lamg,
                                                      const int* __restrict__ rinfo, int info_stride,
                                                      int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int ld = AnaSmem<NS>::kLd;
    AnaSmem<NS> sm;
    sm.carve(smem_raw, k, NS);
    double* A = sm.A;
    double* U = sm.U;
    const int lane = threadIdx.x;
    const int runs_x = (nx + R - 1) / R;
    const int lc = blockIdx.x;  // grid point within the chunk of runs
    const int rl = lc / R;
    const int run = run0 + rl;
    const int y = run / runs_x;
    const int x = (run - y * runs_x) * R + (lc - rl * R);
    if (x >= nx) return;  // past the end of a ragged last run
    const size_t cell = (size_t)y * nx + x;
    const size_t plane = (size_t)nx * ny * k;
    double* fc = f + cell * k;

    for (int a = 0; a < 9; ++a) {
        double s = 0.0;
        for (int m = lane; m < k; m += 32) {
            const double xv = fc[a * plane + m];
            sm.dX[a * k + m] = xv;
            s += xv;
        }
        const double mean = warp_sum(s) / k;
        for (int m = lane; m < k; m += 32) sm.dX[a * k + m] -= mean;
        if (lane == 0) sm.xbar[a] = mean;
    }
    const int* info = rinfo + (size_t)rl * info_stride;
    const int nu = info[0];
    if (nu < 0) return;  // reported by kernel J
    if (nu == 0 || lamg[(size_t)lc * NS] == -1.0f) {
        // No observation in range: x^a_m = xbar + sqrt(beta) dx_m.
        __syncwarp();
        const double sb = sqrt(beta);
        for (int a = 0; a < 9; ++a)
            for (int m = lane; m < k; m += 32) fc[a * plane + m] = sm.xbar[a] + sb * sm.dX[a * k + m];
        return;
    }
    // The union's scalars with this point's weights (the FP64 operations of
    // local_set; zero outside the support and on padding).
    const double lim2 = (2.0 * d_cut + 1.0) * (2.0 * d_cut + 1.0);
    for (int c = lane; c < NS; c += 32) {
        int g = 0;
        double w = 0.0;
        if (c < nu) {
            g = info[1 + c];
            const int j = g / o.nvar;
            const int dx = min_image(o.ix[j] - x, nx);
            const int dy = min_image(o.iy[j] - y, ny);
            const double d2 = (double)dx * dx + (double)dy * dy;
            if (d2 <= lim2) {
                const double dist = sqrt(d2) / d_cut;
                if (dist < 2.0) {
                    const double gc = gaspari_cohn(dist);
                    const int q = g % o.nvar;
                    if (gc > 0.0) w = sqrt(gc) / (q == 0 ? o.sigma_u : (q == 1 ? o.sigma_v : o.sigma_r));
                }
            }
        }
        sm.lidx[c] = g;
        sm.lsq[c] = w;
        sm.ldh[c] = c < nu ? w * o.d[g] : 0.0;
    }
    // 1. Y1 = Y (I - E/2), E = Y^T Y - I, on the binary32 units: Y is
    // binary32, so E comes exactly enough from double-binary32 sums of
    // exact products (|E| ~ 1e-7, kept to ~1e-15 absolute in binary32), and
    // the correction Y E / 2 (entries ~1e-7) needs only binary32 relative
    // precision (~1e-14 absolute). Y1 is then orthonormal to ~1e-13; the
    // FP64 work starts with A' below. Yf (binary32 Y) sits over A, Ef over
    // Z and B until they are used.
    float* Yf = reinterpret_cast<float*>(A);
    float* Ef = reinterpret_cast<float*>(sm.Z);
    const float* Yp = Yg + (size_t)lc * NS * NS;
    for (int e = lane; e < NS * NS; e += 32) Yf[e] = Yp[e];
    __syncwarp();
    const int c = lane < NS ? lane : NS - 1;  // lanes past NS compute a copy and store nothing
    {
        // E column c, rows in groups of 8 (two per packed register):
        // E_ic = sum_j Y_ji Y_jc, rows i..i+7 of row j of Yf.
        for (int i0 = 0; i0 < NS; i0 += 8) {
            f2x S2[4], C2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) S2[q] = C2[q] = 0ull;
#pragma unroll 2
            for (int j = 0; j < NS; ++j) {
                const float yjc = Yf[j * NS + c];
                const f2x Y2 = f2pack(yjc, yjc), NY2 = f2pack(-yjc, -yjc);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = i0 + 2 * q;
                    const f2x A2 = i + 1 < NS ? *reinterpret_cast<const f2x*>(Yf + j * NS + i)
                                              : f2pack(i < NS ? Yf[j * NS + i] : 0.0f, 0.0f);
                    df2_acc1(S2[q], C2[q], A2, Y2, NY2);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float s0, s1, c0, c1;
                f2unpack(S2[q], s0, s1);
                f2unpack(C2[q], c0, c1);
                const int i = i0 + 2 * q;
                if (lane < NS && i < NS) Ef[i * NS + c] = (float)(df_value(s0, c0) - (i == c ? 1.0 : 0.0));
                if (lane < NS && i + 1 < NS) Ef[(i + 1) * NS + c] = (float)(df_value(s1, c1) - (i + 1 == c ? 1.0 : 0.0));
            }
        }
    }
    __syncwarp();
    {
        // (Y E)_ic for column c, then Y1 = Y - (Y E) / 2 in FP64 (into U).
        float ye[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) ye[i] = 0.0f;
#pragma unroll 2
        for (int j = 0; j < NS; ++j) {
            const float ejc = Ef[j * NS + c];
#pragma unroll
            for (int i = 0; i < NS; ++i) ye[i] = fmaf(Yf[i * NS + j], ejc, ye[i]);
        }
        if (lane < NS) {
#pragma unroll
            for (int i = 0; i < NS; ++i) U[i * ld + c] = fma(-0.5, (double)ye[i], (double)Yf[i * NS + c]);
        }
    }
    __syncwarp();
    // A = Yh Yh^T from the global Gram (over E), as in the cold path.
    for (int cc = lane; cc < NS; cc += 32) {
        const int oc = sm.lidx[cc];
        const double sc = sm.lsq[cc];
        for (int i = 0; i < NS; ++i) A[i * ld + cc] = sm.lsq[i] * o.G[(size_t)sm.lidx[i] * (o.nvar * o.npts) + oc] * sc;
    }
    __syncwarp();
    // 2. A' = Y1^T (A Y1), column c; then symmetrised.
    {
        double v[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) v[i] = 0.0;
#pragma unroll 1
        for (int j = 0; j < NS; ++j) {
            const double ujc = U[j * ld + c];
#pragma unroll
            for (int i = 0; i < NS; ++i) v[i] += A[i * ld + j] * ujc;
        }
        __syncwarp();  // A is read by every lane above and rewritten below
        for (int i = 0; i < NS; ++i) {
            double s = 0.0;
#pragma unroll
            for (int j = 0; j < NS; ++j) s += U[j * ld + i] * v[j];
            if (lane < NS) A[i * ld + c] = s;
        }
    }
    __syncwarp();
    if (lane < NS) {
        for (int i = 0; i < c; ++i) {
            const double m = 0.5 * (A[i * ld + c] + A[c * ld + i]);
            A[i * ld + c] = m;
            A[c * ld + i] = m;
        }
    }
    __syncwarp();
    // 3. FP64 Jacobi from A' with U = Y1.
    const int sweeps = jacobi_sym_warp<double>(A, U, NS, ld, lane, sm.rc, sm.rs, sm.rp, sm.rq, 3e-8, kMaxSweeps);
    if (sweeps < 0 && lane == 0) atomicOr(flags, FLAG_NOCONV);
    record_sweeps(o, sweeps, lane);
    __syncwarp();
    // 4. Transform and update.
    fp64_obs_update<NS>(sm, fc, plane, k, NS, (k - 1) / beta, beta, o, lane);
}

// ------------------------------------------------------------------ K3, mixed precision
// The state is binary32 (g = f - w). The eigensolve is FP64-accurate at a
// fraction of the FP64 work, in two kernels over chunks of grid points:
//  (A) mixed_jacobi_kernel: the local set, the matrix in FP64 rounded to
//      binary32, and a binary32 cyclic Jacobi held in registers (no shared
//      memory, so many warps per SM hide its latency); above n = 32 the
//      block Jacobi in shared memory. The basis X goes to the chunk's
//      scratch.
//  (B) analyze_mixed_kernel: to FP64-class accuracy (double-binary32
//      products on the binary32 units), form the Rayleigh-Ritz matrix
//      S = X^T A X and the non-orthogonality E = X^T X - I of the binary32
//      basis, correct S to first order in E (refine_rr), and evaluate
//      f(A) = X (f(S') - E o (f_i + f_j)/2) X^T with f(S') to first order in
//      the off-diagonal of S' (Daleckii-Krein: f(S)_ii = f(s_ii),
//      f(S)_ij = s_ij f[s_ii, s_jj], divided differences in closed form).
//      The error is second order in E and in the off-diagonal of S
//      (relative ~1e-11 at these sizes). The transform products and the update run in
//      binary32 with binary32 accumulation.

constexpr int kChunkCells = 65536;  // grid points per (A)+(B) pass (at most)
constexpr int kJacWarps = 4;        // points per block in (A)

// Binary32 cyclic Jacobi with the column of A and of U held in registers.
// Lane a owns player (column) a of an NS-player round-robin tournament
// (NS even, NS >= n; players n..NS-1 are zero padding). The rows of A are
// kept in tournament-position order: in every round position t meets
// position NS-1-t, so a row rotation always acts on the fixed register pair
// (t, NS-1-t), and after the round the rows move one position
// (q -> q-1 for q >= 2, 1 -> NS-1, 0 stays), a fixed register permutation.
// Column rotations pair a lane with its partner through warp shuffles. The
// player at position q in round r is 0 for q = 0, else 1 + (q-1+r) mod (NS-1).
// On entry a[i] = A[i][lane] (row i at position i); on return u[i] holds
// U[i][lane], the eigenvector of player `lane`.
template <int NS>
__device__ int jacobi32_reg(float (&a)[NS], float (&u)[NS], int lane, float rel, int max_sweeps, float* rs) {
    // rs: the warp's rotation slots (16-byte aligned, 2 NS floats): (c, s)
    // of pair t at rs[2t], (t, a_pq) at rs[NS + 2t].
    float2* const CS = reinterpret_cast<float2*>(rs);
    float2* const TO = reinterpret_cast<float2*>(rs + NS);
    float dg = 0.0f;  // my diagonal entry A[lane][lane], tracked analytically
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        u[i] = (i == lane) ? 1.0f : 0.0f;
        if (i == lane) dg = a[i];
    }
    float fro = 0.0f;
#pragma unroll
    for (int i = 0; i < NS; ++i) fro += a[i] * a[i];
    fro = warp_sum(fro);
    const float thresh = rel * sqrtf(fro);
    const int m1 = NS - 1;
    int r = 0;  // round index modulo NS - 1
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        bool any_sweep = false;
        for (int round = 0; round < m1; ++round) {
            const int q = (lane == 0) ? 0 : 1 + ((lane - 1 - r + 2 * m1) % m1);
            const int qp = m1 - q;
            const int partner = (qp == 0) ? 0 : 1 + ((qp - 1 + r) % m1);
            const bool pside = q < NS / 2;
            float off = 0.0f;
#pragma unroll
            for (int i = 0; i < NS; ++i)
                if (i == qp) off = a[i];
            const float dp = __shfl_sync(kFull, dg, partner & 31);
            // Rotation of my pair (symmetric 2 x 2 Schur), on the p side.
            float c = 1.0f, s = 0.0f, t = 0.0f;
            bool rot = false;
            if (pside && lane < NS && fabsf(off) > thresh) {
                // The binary32 Jacobi only has to shrink the off-diagonal (the
                // FP64 refinement takes the basis from there), so the angle
                // uses the approximate reciprocal and reciprocal square root
                // (a few ulp, no special-case branches). sqrt(x) = x rsqrt(x)
                // for x in [1, 1e30]; the clamp keeps tau^2 finite, where the
                // rotation is negligible anyway (t ~ 1/(2 tau)).
                const float tau = __fdividef(dp - dg, 2.0f * off);
                const float x = fminf(fmaf(tau, tau, 1.0f), 1e30f);
                const float root = x * rsqrtf(x);
                t = __fdividef(tau >= 0.0f ? 1.0f : -1.0f, fabsf(tau) + root);
                c = rsqrtf(fmaf(t, t, 1.0f));
                s = t * c;
                rot = true;
            }
            if (__ballot_sync(kFull, rot) != 0u) {
                any_sweep = true;
                // Every pair's rotation goes to its slot (the p side writes);
                // all lanes read them back by position.
                __syncwarp();  // the previous round's reads are done
                if (pside && lane < NS) {
                    CS[q] = make_float2(c, s);
                    TO[q] = make_float2(t, off);
                }
                __syncwarp();
                // Row rotations: position t (row p) with position NS-1-t (row q).
#pragma unroll
                for (int tt = 0; tt < NS / 2; ++tt) {
                    const float4 cs2 = reinterpret_cast<const float4*>(CS)[tt >> 1];
                    const float ct = (tt & 1) ? cs2.z : cs2.x;
                    const float st = (tt & 1) ? cs2.w : cs2.y;
                    const float x0 = a[tt], x1 = a[NS - 1 - tt];
                    a[tt] = ct * x0 - st * x1;
                    a[NS - 1 - tt] = st * x0 + ct * x1;
                }
                // Column rotations with the partner lane; the diagonal moves
                // by -/+ t a_pq on the p/q side.
                const int pair = lane < NS ? (pside ? q : qp) : 0;
                const float2 csm = CS[pair];
                const float2 tom = TO[pair];
                const float cm = csm.x, sm_ = csm.y, tm = tom.x, om = tom.y;
                dg = pside ? dg - tm * om : dg + tm * om;
                const float sg = pside ? -sm_ : sm_;
                // The rotated off-diagonal entry (row position qp) is zero by
                // construction; it is set so in the same pass.
                const int zq = (sm_ != 0.0f) ? qp : -1;
#pragma unroll
                for (int i = 0; i < NS; ++i) {
                    const float th = __shfl_sync(kFull, a[i], partner & 31);
                    a[i] = (i == zq) ? 0.0f : cm * a[i] + sg * th;
                    const float tu = __shfl_sync(kFull, u[i], partner & 31);
                    u[i] = cm * u[i] + sg * tu;
                }
            }
            // Rows move one tournament position.
            {
                const float a1 = a[1];
#pragma unroll
                for (int i = 1; i < NS - 1; ++i) a[i] = a[i + 1];
                a[NS - 1] = a1;
            }
            r = (r + 1 == m1) ? 0 : r + 1;
        }
        if (!any_sweep) return sweep + 1;
    }
    return -1;
}

// One point of kernel (A): build column `lane` of the matrix (FP64, rounded
// to binary32), run the Jacobi, store X = U (row i of X at Xp + i * xr).
template <int NS>
__device__ void jacobi_point(const ObsParams& o, int k, int n, int p, bool obs_space, double aa,
                             const int* lidx, const double* lsq, int lane, float* __restrict__ Xp,
                             int /*xr = NREG*/, int* flags, const float* __restrict__ Cp,
                             const double* __restrict__ Cd, float* rs) {
    const int nobs = o.nvar * o.npts;
    float a[NS], u[NS];
    if (obs_space) {
        const bool own = lane < n;
        const int ol = own ? lidx[lane] : 0;
        const double sl = own ? lsq[lane] : 0.0;
#pragma unroll
        for (int i = 0; i < NS; ++i)
            a[i] = (own && i < n) ? (float)(lsq[i] * o.G[(size_t)lidx[i] * nobs + ol] * sl) : 0.0f;
    } else if (Cp) {
        // C from the reduced-precision Gram pass.
#pragma unroll
        for (int i = 0; i < NS; ++i) a[i] = (lane < n && i < n) ? Cp[i * k + lane] : 0.0f;
    } else if (Cd) {
        // C from the FP64 Gram pass, rounded to binary32.
#pragma unroll
        for (int i = 0; i < NS; ++i) a[i] = (lane < n && i < n) ? (float)Cd[i * k + lane] : 0.0f;
    } else {
        // C = a I + Yh^T Yh in FP64; lane owns column `lane`.
#pragma unroll
        for (int i = 0; i < NS; ++i) a[i] = 0.0f;
        if (lane < n) {
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                if (i >= n) break;
                double s = (i == lane) ? aa : 0.0;
                for (int l = 0; l < p; ++l) {
                    const double* row = o.dY + (size_t)lidx[l] * k;
                    s += lsq[l] * lsq[l] * row[i] * row[lane];
                }
                a[i] = (float)s;
            }
        }
    }
    // Stop at 1e-6 ||A||_F: the FP64-class refinement takes the matrix
    // functions from there (its neglected terms are second order in the
    // remaining off-diagonal, ~1e-12 relative).
    const int sweeps = jacobi32_reg<NS>(a, u, lane, 1e-6f, kMaxSweeps, rs);
    if (sweeps < 0 && lane == 0) atomicOr(flags, FLAG_NOCONV);
    record_sweeps(o, sweeps, lane);
    if (lane < n) {
#pragma unroll
        for (int i = 0; i < NS; ++i)
            if (i < n) Xp[(size_t)i * NREG + lane] = u[i];
    }
}

// Kernel (A) for an ensemble-space point that follows another one in the
// same run of grid points: C (k x k, from the Gram pass) is solved from the
// previous point's basis U (lane c holds column c of U in up[]):
//   A' = U^T C U (column c: v = C u_c, then A'_ic = u_i . v), in binary32
//   through the warp's shared staging Cs / Us (row-major NS x NS);
//   the register Jacobi of A' gives J; the basis is U J, re-orthonormalised
//   to first order, U J (I - E/2) with E = (U J)^T (U J) - I, so that its
//   drift does not grow along the run. Neighbouring points differ by a
//   smooth change of the localisation weights, so A' is nearly diagonal and
//   the Jacobi needs fewer sweeps than from the identity. On return up[]
//   holds the new basis (for the next point) and X is stored as by
//   jacobi_point.
template <int NS>
__device__ void jacobi_point_warm(const ObsParams& o, int k, int n, int lane, float* __restrict__ Xp,
                                  int* flags, const float* __restrict__ Cp, const double* __restrict__ Cd,
                                  float (&up)[NREG], float* Cs, float* Us, float* rs) {
    // Every product below runs its outer index at run time and reads this
    // lane's own column back from shared memory, so that at most two
    // register columns are live (the register Jacobi needs the rest).
    float a[NS], u[NS];
    const bool own = lane < n;
    const int c = lane < NS ? lane : 0;  // lanes past NS compute a copy and store nothing
    __syncwarp();  // the previous point is done with Cs / Us
    if (lane < NS) {
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            float v = 0.0f;
            if (own && i < n) v = Cp ? Cp[i * k + lane] : (float)Cd[i * k + lane];
            Cs[i * NS + lane] = v;      // C symmetric: column lane
            Us[i * NS + lane] = up[i];  // column lane of U
        }
    }
    __syncwarp();
    // v = C u_c: v_i = sum_j C_ij U_jc (C_ij = C_ji = Cs row j).
#pragma unroll
    for (int i = 0; i < NS; ++i) u[i] = 0.0f;
#pragma unroll 2
    for (int j = 0; j < NS; ++j) {
        const float ujc = Us[j * NS + c];
#pragma unroll
        for (int i = 0; i < NS; ++i) u[i] = fmaf(Cs[j * NS + i], ujc, u[i]);
    }
    __syncwarp();  // Cs takes v
    if (lane < NS) {
#pragma unroll
        for (int i = 0; i < NS; ++i) Cs[i * NS + lane] = u[i];
    }
    __syncwarp();
    // A'_ic = sum_j U_ji v_j.
#pragma unroll
    for (int i = 0; i < NS; ++i) a[i] = 0.0f;
#pragma unroll 2
    for (int j = 0; j < NS; ++j) {
        const float vj = Cs[j * NS + c];
#pragma unroll
        for (int i = 0; i < NS; ++i) a[i] = fmaf(Us[j * NS + i], vj, a[i]);
    }
    if (lane >= NS) {
#pragma unroll
        for (int i = 0; i < NS; ++i) a[i] = 0.0f;
    }
    const int sweeps = jacobi32_reg<NS>(a, u, lane, 1e-6f, kMaxSweeps, rs);
    if (sweeps < 0 && lane == 0) atomicOr(flags, FLAG_NOCONV);
    record_sweeps(o, sweeps, lane);
    __syncwarp();  // Cs takes J
    if (lane < NS) {
#pragma unroll
        for (int i = 0; i < NS; ++i) Cs[i * NS + lane] = u[i];
    }
    __syncwarp();
    // W = U J, column c: W_ic = sum_j U_ij J_jc (into a).
#pragma unroll
    for (int i = 0; i < NS; ++i) a[i] = 0.0f;
#pragma unroll 2
    for (int j = 0; j < NS; ++j) {
        const float jjc = Cs[j * NS + c];
#pragma unroll
        for (int i = 0; i < NS; ++i) a[i] = fmaf(Us[i * NS + j], jjc, a[i]);
    }
    __syncwarp();  // Us takes W
    if (lane < NS) {
#pragma unroll
        for (int i = 0; i < NS; ++i) Us[i * NS + lane] = a[i];
    }
    __syncwarp();
    // E column c: E_jc = sum_i W_ij W_ic - delta_jc (into u).
#pragma unroll
    for (int j = 0; j < NS; ++j) u[j] = (j == lane) ? -1.0f : 0.0f;
#pragma unroll 2
    for (int i = 0; i < NS; ++i) {
        const float wic = Us[i * NS + c];
#pragma unroll
        for (int j = 0; j < NS; ++j) u[j] = fmaf(Us[i * NS + j], wic, u[j]);
    }
    __syncwarp();  // Cs takes E
    if (lane < NS) {
#pragma unroll
        for (int j = 0; j < NS; ++j) Cs[j * NS + lane] = u[j];
    }
    __syncwarp();
    // U_new = W (I - E/2), column c: W_ic - 1/2 sum_j W_ij E_jc.
#pragma unroll
    for (int i = 0; i < NS; ++i) u[i] = 0.0f;
#pragma unroll 2
    for (int j = 0; j < NS; ++j) {
        const float ejc = Cs[j * NS + c];
#pragma unroll
        for (int i = 0; i < NS; ++i) u[i] = fmaf(Us[i * NS + j], ejc, u[i]);
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) up[i] = lane < NS ? fmaf(-0.5f, u[i], a[i]) : 0.0f;
    if (lane < n) {
#pragma unroll
        for (int i = 0; i < NS; ++i)
            if (i < n) Xp[(size_t)i * NREG + lane] = up[i];
    }
}

// Per-chunk scratch shared by kernels (A) and (B).
struct MixScratch {
    float* X;      // [chunk][xr][xr] binary32 basis, row i at i * xr (xr = 32, 64 or 128)
    double* lsq;   // [chunk][nobs] sqrt(rho) of the local scalars
    int* lidx;     // [chunk][nobs] their observation indices
    int* pcount;   // [chunk] number of local scalars
    float* C32;    // [chunk][k][k] a I + Yh^T Yh from the reduced-precision Gram, or null
    float* b32;    // [chunk][k] Yh^T d-hat from the same pass, or null
    float* big;    // [chunk][4][nm][ld] kernel (B)'s A and A Y halves when nm > NMID, or null
    double* C64;   // [chunk][k][k] a I + Yh^T Yh from the FP64 Gram pass, or null
    double* b64;   // [chunk][k] Yh^T d-hat from the same pass, or null
    // Double-binary32 Gram pass: C as two binary32 planes in C64's space,
    // C32 = the high halves ([chunk][k][k], C rounded to binary32) and Clo
    // the low ones (C = C32 + Clo to FP64-class accuracy); b in b64.
    float* Clo;
};

// The double-binary32 pass's view of a scratch carved for 8-byte elements.
__host__ __device__ inline MixScratch mix_scratch_df2(MixScratch m, long long chunk, int kg) {
    if (m.C64) {
        m.C32 = reinterpret_cast<float*>(m.C64);
        m.Clo = m.C32 + (size_t)chunk * kg * kg;
        m.C64 = nullptr;
    }
    return m;
}

// Row stride of the basis scratch: 128-byte rows for the register Jacobi.
__host__ __device__ inline int mix_xr(int nm) { return nm <= NREG ? NREG : (nm <= NMID ? NMID : NMAX); }

// Row stride of the matrices of kernel (B): nm + 1 rounded to odd.
__host__ __device__ inline int mix_ld(int nm) { return (nm % 2 == 0) ? nm + 1 : nm; }

// Floats per grid point of kernel (B)'s matrices kept in global scratch
// (A and A Y, two binary32 halves each) when nm > NMID, else 0.
__host__ __device__ inline size_t mix_big_floats(int nm) {
    return nm > NMID ? 4 * (size_t)nm * mix_ld(nm) : 0;
}

// kg: members k when a Gram pass is used (its C and b per point), else 0;
// gsz: bytes of its elements (4 reduced precision, 8 FP64).
__host__ __device__ inline size_t mix_scratch_bytes_per_point(int nobs, int nm, int kg, int gsz) {
    const int xr = mix_xr(nm);
    return (size_t)xr * xr * sizeof(float) + (size_t)nobs * (sizeof(double) + sizeof(int)) +
           sizeof(int) + (size_t)kg * (kg + 1) * gsz + mix_big_floats(nm) * sizeof(float);
}

// Grid points per chunk: up to kChunkCells, with at most 384 MiB of scratch
// per buffer. Fewer, larger launches won over L2-resident chunks: at
// 256^2 x 64 (4.4 KB per point) the analysis took 10.6 / 10.3 / 10.0 / 9.9 ms
// with chunks of 8192 / 16384 / 32768 / 65536 points (11.9 ms at 4096),
// although the basis scratch then round-trips through HBM. Above NMID both
// kernels hold one grid point per SM; their chunks are at least four full
// waves of GB300's 152 SMs.
__host__ __device__ inline long long mix_chunk(long long cells, int nobs, int nm, int kg, int gsz) {
    long long c = (384ll << 20) / (long long)mix_scratch_bytes_per_point(nobs, nm, kg, gsz);
    if (c > kChunkCells) c = kChunkCells;
    const long long cmin = nm > NMID ? 4 * 152 : 256;
    if (c < cmin) c = cmin;
    return cells < c ? cells : c;
}

__host__ __device__ inline MixScratch mix_scratch_at(void* base, long long chunk, int nobs, int nm,
                                                    int kg, int gsz) {
    MixScratch m;
    unsigned char* p = reinterpret_cast<unsigned char*>(base);
    m.X = reinterpret_cast<float*>(p);
    p += (size_t)chunk * mix_xr(nm) * mix_xr(nm) * sizeof(float);
    m.lsq = reinterpret_cast<double*>(p);
    p += (size_t)chunk * nobs * sizeof(double);
    m.lidx = reinterpret_cast<int*>(p);
    p += (size_t)chunk * nobs * sizeof(int);
    m.pcount = reinterpret_cast<int*>(p);
    p += ((size_t)chunk * sizeof(int) + 15) / 16 * 16;
    m.C32 = (kg && gsz == 4) ? reinterpret_cast<float*>(p) : nullptr;
    m.C64 = (kg && gsz == 8) ? reinterpret_cast<double*>(p) : nullptr;
    p += (size_t)chunk * kg * kg * gsz;
    m.b32 = (kg && gsz == 4) ? reinterpret_cast<float*>(p) : nullptr;
    m.b64 = (kg && gsz == 8) ? reinterpret_cast<double*>(p) : nullptr;
    m.Clo = nullptr;
    p += (size_t)chunk * kg * gsz;
    m.big = nm > NMID ? reinterpret_cast<float*>(p) : nullptr;
    return m;
}

// Bytes of one scratch buffer, rounded up to 256 so that the second buffer of
// the pair starts as aligned as the first (its FP64 arrays need 8 bytes).
__host__ __device__ inline size_t mix_buf_bytes(long long chunk, int nobs, int nm, int kg, int gsz) {
    return ((size_t)chunk * mix_scratch_bytes_per_point(nobs, nm, kg, gsz) + 16 + 255) / 256 * 256;
}

// ---- Local Gram matrices in reduced precision (ensemble-space form) --------
// C = a I + Yh^T Yh and b = Yh^T d-hat for every grid point of a chunk, with
// Yh = diag(sqrt(rho)) dY_loc (Section 3.2), from the binary32 copy of dY:
// PROD_FP32 on the CUDA cores (local_gram_kernel), PROD_TF32 and PROD_BF16
// on the tcgen05 tensor cores (local_gram_tc_kernel), all accumulating in
// binary32. A block takes
// kGramPts consecutive grid points, one warp each; their local sets are
// merged into one list of observation points, whose rows are staged once per
// block in shared memory and weighted per point (rows outside a point's set
// get weight 0). The weights are the same FP64 Gaspari-Cohn values the local
// set uses, rounded to binary32.
constexpr int kGramPts = 8;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// sqrt(G(r / d_cut)) of observation point j seen from (x, y), 0 outside the
// support: the same FP64 operations as local_set.
__device__ __forceinline__ double local_weight(const ObsParams& o, int j, int x, int y, int nx,
                                               int ny, double d_cut, long long lim2) {
    const int dx = min_image(o.ix[j] - x, nx);
    const int dy = min_image(o.iy[j] - y, ny);
    if (dist2(dx, dy) > lim2) return 0.0;  // lim2 = support_lim2(d_cut)
    const double d2 = (double)dx * dx + (double)dy * dy;
    const double dist = sqrt(d2) / d_cut;
    if (!(dist < 2.0)) return 0.0;
    const double g = gaspari_cohn(dist);
    return g > 0.0 ? sqrt(g) : 0.0;
}

// Merged local sets of the kGramPts grid points cell0 + li0 + q (q < kGramPts,
// li0 + q < ncell), in increasing point order, into U; pcnt[q] counts the
// local points of grid point q. Returns the merged count. Block-cooperative
// (32 kGramPts threads).
__device__ int gram_merge(const ObsParams& o, int nx, int ny, double d_cut, int cell0, int li0, int ncell,
                          int* U, int* pcnt, int* wcount) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long lim2 = support_lim2(d_cut);
    if (threadIdx.x < kGramPts) pcnt[threadIdx.x] = 0;
    __syncthreads();
    int total = 0;
    for (int j0 = 0; j0 < o.npts; j0 += 32 * kGramPts) {
        const int j = j0 + threadIdx.x;
        unsigned bits = 0u;
        if (j < o.npts) {
            for (int q = 0; q < kGramPts; ++q) {
                if (li0 + q >= ncell) break;
                const int cell = cell0 + li0 + q;
                if (local_weight(o, j, cell % nx, cell / nx, nx, ny, d_cut, lim2) > 0.0) bits |= 1u << q;
            }
        }
        const bool in = bits != 0u;
#pragma unroll
        for (int q = 0; q < kGramPts; ++q) {
            const unsigned bq = __ballot_sync(kFull, (bits >> q) & 1u);
            if (lane == 0 && bq) atomicAdd(&pcnt[q], __popc(bq));
        }
        const unsigned bal = __ballot_sync(kFull, in);
        if (lane == 0) wcount[w] = __popc(bal);
        __syncthreads();
        int off = total, add = 0;
        for (int q = 0; q < kGramPts; ++q) {
            if (q < w) off += wcount[q];
            add += wcount[q];
        }
        if (in) U[off + __popc(bal & ((1u << lane) - 1u))] = j;
        total += add;
        __syncthreads();
    }

    return total;
}

// PROD_FP32: binary32 products and sums on the CUDA cores. Warp w is grid
// point w of the block; lane c owns output columns c (and c + 32 at 64
// members); at 128 members the columns go in passes of 32 so that the
// accumulators stay at 128 per lane.
template <int K>
__global__ void __launch_bounds__(32 * kGramPts, 1) local_gram_kernel(int nx, int ny, int k,
                                                                     ObsParams o, double d_cut,
                                                                     double aa, int cell0,
                                                                     int ncell, MixScratch sc) {
    constexpr int KC = 16;     // rows per stage
    constexpr int LD = K + 4;
    constexpr int KB = K > 64 ? 32 : K;       // output columns per pass over the rows
    constexpr int NCOL = KB > 32 ? 2 : 1;     // output columns per lane and pass
    constexpr int NBC = K > 32 ? K / 32 : 1;  // entries of b per lane
    __shared__ float Ys[KC][LD];
    __shared__ float Ws[kGramPts][KC];  // rho-tilde = (sqrt(G) / sigma)^2 per point and row
    __shared__ float Ds[KC];
    __shared__ int wcount[kGramPts];
    __shared__ int pcnt[kGramPts];  // local points of each grid point
    extern __shared__ int U[];  // [npts] merged observation points
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int li0 = blockIdx.x * kGramPts;
    const int nv = o.nvar;

    const int total = gram_merge(o, nx, ny, d_cut, cell0, li0, ncell, U, pcnt, wcount);
    const long long lim2 = support_lim2(d_cut);
    // Only grid points in the ensemble-space form (p >= k) read C and b.
    bool any_ens = false;
    for (int q = 0; q < kGramPts; ++q) any_ens |= pcnt[q] * nv >= k;
    if (!any_ens) return;
    const int rows = total * nv;
    const int li = li0 + w;
    float* C = sc.C32 + (size_t)li * k * k;
    const float fa = (float)aa;
    float accf[K][NCOL];
    float bacc[NBC];
#pragma unroll
    for (int c = 0; c < NBC; ++c) bacc[c] = 0.0f;
    for (int cb = 0; cb < K; cb += KB) {  // first column of this pass
#pragma unroll
        for (int m = 0; m < K; ++m)
#pragma unroll
            for (int c = 0; c < NCOL; ++c) accf[m][c] = 0.0f;
        for (int r0 = 0; r0 < rows; r0 += KC) {
            for (int e = threadIdx.x; e < KC * K; e += 32 * kGramPts) {
                const int rr = e / K, c = e % K, r = r0 + rr;
                float v = 0.0f;
                if (r < rows && c < k) v = o.dY32[(size_t)(nv * U[r / nv] + r % nv) * k + c];
                Ys[rr][c] = v;
            }
            if (threadIdx.x < KC * kGramPts) {
                const int q = threadIdx.x / KC, rr = threadIdx.x % KC, r = r0 + rr;
                float wv = 0.0f;
                if (r < rows && li0 + q < ncell) {
                    const int cell = cell0 + li0 + q;
                    const double sg = local_weight(o, U[r / nv], cell % nx, cell / nx, nx, ny, d_cut, lim2);
                    const int qv = r % nv;
                    const double l = sg / (qv == 0 ? o.sigma_u : (qv == 1 ? o.sigma_v : o.sigma_r));
                    wv = (float)(l * l);
                }
                Ws[q][rr] = wv;
            }
            if (threadIdx.x < KC) {
                const int r = r0 + threadIdx.x;
                Ds[threadIdx.x] = r < rows ? (float)o.d[nv * U[r / nv] + r % nv] : 0.0f;
            }
            __syncthreads();
            for (int rr = 0; rr < KC; ++rr) {
                const float wl = Ws[w][rr];
                if (wl == 0.0f) continue;
                float yc[NCOL];
#pragma unroll
                for (int c = 0; c < NCOL; ++c) yc[c] = (lane + 32 * c < KB) ? Ys[rr][cb + lane + 32 * c] : 0.0f;
                if (cb == 0) {
#pragma unroll
                    for (int c = 0; c < NBC; ++c)
                        bacc[c] += wl * Ds[rr] * ((lane + 32 * c < K) ? Ys[rr][lane + 32 * c] : 0.0f);
                }
#pragma unroll
                for (int m = 0; m < K; ++m) {
                    const float ym = wl * Ys[rr][m];
#pragma unroll
                    for (int c = 0; c < NCOL; ++c) accf[m][c] += ym * yc[c];
                }
            }
            __syncthreads();
        }
        if (li < ncell) {
#pragma unroll
            for (int m = 0; m < K; ++m)
#pragma unroll
                for (int c = 0; c < NCOL; ++c) {
                    const int n = cb + lane + 32 * c;
                    if (m < k && n < k && lane + 32 * c < KB) C[m * k + n] = accf[m][c] + (m == n ? fa : 0.0f);
                }
        }
    }  // passes over the output columns
    if (li >= ncell) return;
#pragma unroll
    for (int c = 0; c < NBC; ++c)
        if (lane + 32 * c < k) sc.b32[(size_t)li * k + lane + 32 * c] = bacc[c];
}

// ---- reduced-precision Gram on the tcgen05 tensor cores ------------------
// The same C = a I + sum_r rho_q(r) y_r y_r^T per grid point q of a block of
// kGramPts points (Section 3.2's Yh^T Yh in the ensemble-space form), with
// TF32 or BF16 products and FP32 accumulation in tensor memory. One
// tcgen05.mma computes D[128 x KP] += A[128 x Kmma] B[Kmma x KP] (K = the
// rows r of the block's merged local set):
//   B[n][r] = y_r[n]                 (n < k, zero up to KP)
//   A[p KP + m][r] = rho_q(r) y_r[m]  (the 128 / KP points q of one group
//                                      stacked along M; zero for m >= k)
// so D row p KP + m, column n is C_q[m][n] - a. Both operands are K-major
// in the no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix,
// LBO = 128 bytes between core matrices along K, SBO between 8-row groups).
// Per stage of 32 rows: TMA brings each row of the merged set (a one-row
// box of the binary32 copy of dY, gathered through the merged index list)
// into a 128-byte aligned row of shared memory; the block weights, rounds and lays out A and B; one
// thread issues the MMAs and commits them to an mbarrier; the next stage
// waits for them before rewriting the operands. The accumulators are read
// back with tcgen05.ld. b = Yh^T d-hat stays on the CUDA cores. Every wait
// is bounded: on a timeout the block records FLAG_TCWAIT, waits (bounded)
// for its MMAs in flight, frees its tensor memory and returns.
constexpr int kTcKC = 32;  // rows (K) per stage

template <bool TF32, int KP>
struct TcGram {
    static constexpr int ES = TF32 ? 4 : 2;                  // operand element bytes
    static constexpr int T = 16 / ES;                        // elements per 16-byte core-matrix row
    static constexpr int KCOL = kTcKC * ES / 16;             // core matrices along K per stage
    static constexpr int SBO = KCOL * 128;                   // bytes between 8-row groups
    static constexpr int PG = 128 / KP;                      // points per MMA group
    static constexpr int G = KP == 128 ? 4 : kGramPts / PG;  // groups per pass
    static constexpr int PASSES = KP == 128 ? 2 : 1;
    static constexpr int PPP = G * PG;                       // points per pass
    static constexpr int KMMA = TF32 ? 8 : 16;               // K of one MMA (32 bytes)
    static constexpr int NCOLS = G * KP < 32 ? 32 : G * KP;  // TMEM columns
    static constexpr int A_BYTES = 128 * kTcKC * ES;         // one group's A per stage
    static constexpr int B_BYTES = KP * kTcKC * ES;
    static constexpr int oA = 0;
    static constexpr int oB = oA + G * A_BYTES;
    static constexpr int SP = KP < 32 ? 32 : KP;             // staged row pitch (floats): 128-byte rows
    static constexpr int oS = oB + B_BYTES;                  // staged rows [KC][SP] binary32
    static constexpr int oW = oS + kTcKC * SP * 4;           // rho [kGramPts][KC]
    static constexpr int oD = oW + kGramPts * kTcKC * 4;     // innovations [KC]
    static constexpr int oBar = oD + kTcKC * 4;              // mbarriers: TMA, MMA
    static constexpr int oTm = oBar + 16;                    // TMEM base address
    static constexpr int oU = oTm + 16;                      // merged list [npts]
    static_assert(PPP * PASSES == kGramPts, "every point of the block in one pass");
    static_assert(NCOLS == 32 || NCOLS == 64 || NCOLS == 128 || NCOLS == 256 || NCOLS == 512,
                  "TMEM columns");
    static_assert(oS % 128 == 0 && (SP * 4) % 128 == 0 && (oU % 16) == 0, "TMA destinations on 128 bytes");
};

__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// One 16-byte core-matrix row from T binary32 values, rounded.
template <bool TF32>
__device__ __forceinline__ void store_core_row(unsigned char* dst, const float* v) {
    uint4 u;
    if constexpr (TF32) {
        u = make_uint4(tf32_bits(v[0]), tf32_bits(v[1]), tf32_bits(v[2]), tf32_bits(v[3]));
    } else {
        u = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    }
    *reinterpret_cast<uint4*>(dst) = u;
}

constexpr long long kTcWaitPolls = 1ll << 22;  // polls of ~50 ns: a few tenths of a second

template <bool TF32, int KP>
__global__ void __launch_bounds__(32 * kGramPts, 1)
    local_gram_tc_kernel(int nx, int ny, int k, ObsParams o, double d_cut, double aa, int cell0, int ncell,
                         MixScratch sc, const __grid_constant__ CUtensorMap ymap, int use_tma, int* flags) {
    using L = TcGram<TF32, KP>;
    extern __shared__ unsigned char tc_raw[];
    // 1024-byte aligned base (the launch adds the slack).
    unsigned char* tsm = tc_raw + ((1024u - (smem_u32(tc_raw) & 1023u)) & 1023u);
    unsigned char* Aop = tsm + L::oA;
    unsigned char* Bop = tsm + L::oB;
    float* Sg = reinterpret_cast<float*>(tsm + L::oS);
    float* Ws = reinterpret_cast<float*>(tsm + L::oW);
    float* Ds = reinterpret_cast<float*>(tsm + L::oD);
    uint64_t* bars = reinterpret_cast<uint64_t*>(tsm + L::oBar);
    uint32_t* tbase = reinterpret_cast<uint32_t*>(tsm + L::oTm);
    int* U = reinterpret_cast<int*>(tsm + L::oU);
    __shared__ int wcount[kGramPts];
    __shared__ int pcnt[kGramPts];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int li0 = blockIdx.x * kGramPts;
    const int nv = o.nvar;

    const int total = gram_merge(o, nx, ny, d_cut, cell0, li0, ncell, U, pcnt, wcount);
    const long long lim2 = support_lim2(d_cut);
    // Only grid points in the ensemble-space form (p >= k) read C and b.
    bool any_ens = false;
    for (int q = 0; q < kGramPts; ++q) any_ens |= pcnt[q] * nv >= k;
    if (!any_ens) return;
    const int rows = total * nv;
    const int nst = (rows + kTcKC - 1) / kTcKC;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    if (w == 0) {
        tmem_alloc(tbase, L::NCOLS);
        tmem_relinquish();
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = *tbase;
    constexpr uint32_t idesc = umma_idesc(TF32 ? 2u : 1u, 128, KP);
    constexpr int NBC = KP > 32 ? KP / 32 : 1;
    float bacc[NBC];
#pragma unroll
    for (int c = 0; c < NBC; ++c) bacc[c] = 0.0f;
    bool ok = true;
    uint32_t tphase = 0, mphase = 0;  // parity of the next phase to wait for
    bool mma_pending = false, tma_pending = false;
    for (int pass = 0; pass < L::PASSES && ok; ++pass) {
        const int q0 = pass * L::PPP;
        for (int s = 0; s < nst && ok; ++s) {
            const int r0 = s * kTcKC;
            const int nr = rows - r0 < kTcKC ? rows - r0 : kTcKC;
            // Stage rows r0 .. r0 + nr - 1 of the merged set.
            if (use_tma) {
                if (tid == 0) {
                    mbar_arrive_expect_tx(&bars[0], (uint32_t)(nr * k * 4));
                    for (int rr = 0; rr < nr; ++rr) {
                        const int r = r0 + rr;
                        tma_load_2d(Sg + rr * L::SP, &ymap, 0, nv * U[r / nv] + r % nv, &bars[0]);
                    }
                }
                tma_pending = true;
            } else {
                for (int e = tid; e < nr * k; e += 32 * kGramPts) {
                    const int rr = e / k, c = e - rr * k, r = r0 + rr;
                    Sg[rr * L::SP + c] = o.dY32[(size_t)(nv * U[r / nv] + r % nv) * k + c];
                }
            }
            // rho of every point for the stage's rows, and the innovations.
            if (tid < kTcKC * kGramPts) {
                const int q = tid / kTcKC, rr = tid % kTcKC, r = r0 + rr;
                float wv = 0.0f;
                if (rr < nr && li0 + q < ncell) {
                    const int cell = cell0 + li0 + q;
                    const double sg = local_weight(o, U[r / nv], cell % nx, cell / nx, nx, ny, d_cut, lim2);
                    const int qv = r % nv;
                    const double l = sg / (qv == 0 ? o.sigma_u : (qv == 1 ? o.sigma_v : o.sigma_r));
                    wv = (float)(l * l);
                }
                Ws[q * kTcKC + rr] = wv;
            }
            if (tid < kTcKC) {
                const int r = r0 + tid;
                Ds[tid] = tid < nr ? (float)o.d[nv * U[r / nv] + r % nv] : 0.0f;
            }
            if (tma_pending) {
                ok = mbar_wait(&bars[0], tphase, kTcWaitPolls);
                tphase ^= 1u;
                tma_pending = !ok;
            }
            // The previous stage's MMAs read the operands being rewritten.
            if (mma_pending && ok) {
                ok = mbar_wait(&bars[1], mphase, kTcWaitPolls);
                mphase ^= 1u;
                mma_pending = !ok;
            }
            ok = __syncthreads_and(ok) != 0;
            if (!ok) break;
            // B[n][rr] = y_rr[n]. Eight consecutive threads write the eight
            // 16-byte rows of one core matrix (128 contiguous bytes).
            for (int e = tid; e < KP * L::KCOL; e += 32 * kGramPts) {
                const int cm = e >> 3, kc = cm % L::KCOL;
                const int n = (cm / L::KCOL) * 8 + (e & 7);
                float v[L::T];
#pragma unroll
                for (int t = 0; t < L::T; ++t) {
                    const int rr = kc * L::T + t;
                    v[t] = (n < k && rr < nr) ? Sg[rr * L::SP + n] : 0.0f;
                }
                store_core_row<TF32>(Bop + (n >> 3) * L::SBO + kc * 128 + (n & 7) * 16, v);
            }
            // A_g[p KP + m][rr] = rho_q(rr) y_rr[m], q = q0 + g PG + p.
            for (int e = tid; e < L::G * 128 * L::KCOL; e += 32 * kGramPts) {
                const int g = e / (128 * L::KCOL);
                const int rem = e - g * 128 * L::KCOL;
                const int cm = rem >> 3, kc = cm % L::KCOL;
                const int R = (cm / L::KCOL) * 8 + (rem & 7);
                const int p = R / KP, m = R - p * KP, q = q0 + g * L::PG + p;
                float v[L::T];
#pragma unroll
                for (int t = 0; t < L::T; ++t) {
                    const int rr = kc * L::T + t;
                    v[t] = (m < k && rr < nr) ? Ws[q * kTcKC + rr] * Sg[rr * L::SP + m] : 0.0f;
                }
                store_core_row<TF32>(Aop + g * L::A_BYTES + (R >> 3) * L::SBO + kc * 128 + (R & 7) * 16, v);
            }
            // b = Yh^T d-hat on the CUDA cores (first pass; warp w is point w).
            if (pass == 0) {
                for (int rr = 0; rr < nr; ++rr) {
                    const float wd = Ws[w * kTcKC + rr] * Ds[rr];
#pragma unroll
                    for (int c = 0; c < NBC; ++c)
                        if (lane + 32 * c < k) bacc[c] += wd * Sg[rr * L::SP + lane + 32 * c];
                }
            }
            fence_async_smem();
            tc_fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after_sync();
                const uint32_t a0 = smem_u32(Aop), b0 = smem_u32(Bop);
#pragma unroll
                for (int j = 0; j < kTcKC / L::KMMA; ++j) {
                    const uint64_t bd = umma_smem_desc(b0 + j * 256, 128, L::SBO);
#pragma unroll
                    for (int g = 0; g < L::G; ++g) {
                        const uint64_t ad = umma_smem_desc(a0 + g * L::A_BYTES + j * 256, 128, L::SBO);
                        umma<TF32>(tmem + (uint32_t)(g * KP), ad, bd, idesc, (s > 0 || j > 0) ? 1u : 0u);
                    }
                }
                umma_commit(&bars[1]);
            }
            mma_pending = true;
        }
        if (!ok) break;
        ok = mbar_wait(&bars[1], mphase, kTcWaitPolls);
        mphase ^= 1u;
        mma_pending = !ok;
        ok = __syncthreads_and(ok) != 0;
        if (!ok) break;
        tc_fence_after_sync();
        // Epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of D)
        // of the groups g with g % 2 == w / 4.
        {
            const int quarter = w & 3;
            const int R = 32 * quarter + lane;
            const int p = R / KP, m = R - p * KP;
            for (int g = w >> 2; g < L::G; g += 2) {
                const int li = li0 + q0 + g * L::PG + p;
                for (int c0 = 0; c0 < KP; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(g * KP + c0), v);
                    if (li < ncell && m < k) {
                        float* C = sc.C32 + (size_t)li * k * k + (size_t)m * k;
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int n = c0 + i;
                            if (n < k) C[n] = v[i] + (m == n ? (float)aa : 0.0f);
                        }
                    }
                }
            }
        }
        tc_fence_before_sync();
        __syncthreads();  // the next pass overwrites the accumulators
        tc_fence_after_sync();
    }
    if (!ok) {
        // A wait ran out: record it, then let the copies and MMAs this block
        // issued finish (bounded) before its tensor memory is freed.
        if (tid == 0) atomicOr(flags, FLAG_TCWAIT);
        if (tma_pending) mbar_wait(&bars[0], tphase, kTcWaitPolls);
        if (mma_pending) mbar_wait(&bars[1], mphase, kTcWaitPolls);
    }
    tc_fence_before_sync();
    __syncthreads();
    if (w == 0) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, L::NCOLS);
    }
    if (!ok) return;
    const int li = li0 + w;
    if (li >= ncell) return;
#pragma unroll
    for (int c = 0; c < NBC; ++c)
        if (lane + 32 * c < k) sc.b32[(size_t)li * k + lane + 32 * c] = bacc[c];
}

template <bool TF32, int KP>
size_t tc_gram_smem(int npts) {
    return (size_t)TcGram<TF32, KP>::oU + (size_t)(npts > 0 ? npts : 1) * sizeof(int) + 1024;
}

// FP64 Gram (PROD_FP64): the same C and b in FP64 products and sums, from
// the FP64 dY, for the ensemble-space points of a mixed-precision analysis
// (kernel (A) starts its binary32 Jacobi from C rounded to binary32, kernel
// (B) refines against C itself). Each lane owns one output column and a
// range of K / RH rows, so a lane holds at most 64 FP64 accumulators; the
// output columns are covered in passes of KB.
template <int K>
__global__ void __launch_bounds__(32 * kGramPts, 1) local_gram_fp64_kernel(int nx, int ny, int k,
                                                                          ObsParams o, double d_cut,
                                                                          double aa, int cell0,
                                                                          int ncell, MixScratch sc) {
    constexpr int KC = 16;                          // rows per stage
    constexpr int RH = K > 64 ? 2 : 1;              // row ranges per column
    constexpr int KB = (K < 32 ? K : 32) / RH;      // output columns per pass
    constexpr int MR = K / RH;                      // rows per lane
    constexpr int NBC = K > 32 ? K / 32 : 1;        // entries of b per lane
    __shared__ double Ys[KC][K];
    __shared__ double Ws[kGramPts][KC];
    __shared__ double Ds[KC];
    __shared__ int wcount[kGramPts];
    __shared__ int pcnt[kGramPts];
    extern __shared__ int U[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int li0 = blockIdx.x * kGramPts;
    const int nv = o.nvar;
    const double sig[3] = {o.sigma_u, o.sigma_v, o.sigma_r};
    const int total = gram_merge(o, nx, ny, d_cut, cell0, li0, ncell, U, pcnt, wcount);
    const long long lim2 = support_lim2(d_cut);
    bool any_ens = false;
    for (int q = 0; q < kGramPts; ++q) any_ens |= pcnt[q] * nv >= k;
    if (!any_ens) return;
    const int rows = total * nv;
    const int li = li0 + w;
    const int col = lane % KB, rh = lane / KB;
    const bool act = rh < RH;  // K = 16: lanes 16..31 own no column
    double acc[MR];
    double bacc[NBC];
#pragma unroll
    for (int c = 0; c < NBC; ++c) bacc[c] = 0.0;
    for (int cb = 0; cb < K; cb += KB) {
#pragma unroll
        for (int m = 0; m < MR; ++m) acc[m] = 0.0;
        for (int r0 = 0; r0 < rows; r0 += KC) {
            for (int e = threadIdx.x; e < KC * K; e += 32 * kGramPts) {
                const int rr = e / K, c = e % K, r = r0 + rr;
                double v = 0.0;
                if (r < rows && c < k) v = o.dY[(size_t)(nv * U[r / nv] + r % nv) * k + c];
                Ys[rr][c] = v;
            }
            if (threadIdx.x < KC * kGramPts) {
                const int q = threadIdx.x / KC, rr = threadIdx.x % KC, r = r0 + rr;
                double wv = 0.0;
                if (r < rows && li0 + q < ncell) {
                    const int cell = cell0 + li0 + q;
                    const double sg = local_weight(o, U[r / nv], cell % nx, cell / nx, nx, ny, d_cut, lim2);
                    const double l = sg / sig[r % nv];
                    wv = l * l;
                }
                Ws[q][rr] = wv;
            }
            if (threadIdx.x < KC) {
                const int r = r0 + threadIdx.x;
                Ds[threadIdx.x] = r < rows ? o.d[nv * U[r / nv] + r % nv] : 0.0;
            }
            __syncthreads();
            for (int rr = 0; rr < KC; ++rr) {
                const double wl = Ws[w][rr];
                if (wl == 0.0) continue;
                if (cb == 0) {
#pragma unroll
                    for (int c = 0; c < NBC; ++c)
                        if (lane + 32 * c < K) bacc[c] += wl * Ds[rr] * Ys[rr][lane + 32 * c];
                }
                if (act) {
                    const double wy = wl * Ys[rr][cb + col];
#pragma unroll
                    for (int m = 0; m < MR; ++m) acc[m] += Ys[rr][rh * MR + m] * wy;
                }
            }
            __syncthreads();
        }
        if (li < ncell && act) {
            double* C = sc.C64 + (size_t)li * k * k;
            const int n = cb + col;
#pragma unroll
            for (int m = 0; m < MR; ++m) {
                const int row = rh * MR + m;
                if (row < k && n < k) C[(size_t)row * k + n] = acc[m] + (row == n ? aa : 0.0);
            }
        }
    }
    if (li >= ncell) return;
#pragma unroll
    for (int c = 0; c < NBC; ++c)
        if (lane + 32 * c < k) sc.b64[(size_t)li * k + lane + 32 * c] = bacc[c];
}

// A double-binary32 sum (s, c), plus (ah + al) when diag, renormalised into
// binary32 high and low halves (Fast2Sum: the compensated sum's s dominates).
__device__ __forceinline__ void df_pair_out(float s, float c, bool diag, float ah, float al, float& hi,
                                            float& lo) {
    if (diag) {
        float t, e;
        two_sum(s, ah, t, e);
        c = __fadd_rn(c, __fadd_rn(e, al));
        s = t;
    }
    const float h = __fadd_rn(s, c);
    hi = h;
    lo = __fsub_rn(c, __fsub_rn(h, s));
}

// Double-binary32 Gram (PROD_DF32, the default of a mixed-precision
// context): the C and b of the FP64 Gram pass to FP64-class accuracy on the
// binary32 units. The staged rows are split once into binary32 halves
// (y = yh + yl, exact to 2^-48), and so is each grid point's weight of a
// row (rho = rh + rl), when the row is staged. A lane's weighted column
// value wy = rho y_n is then formed in double-binary32: rh yh exactly (its
// rounding error recovered with one FMA) plus the cross terms rh yl and
// rl yh in binary32, rl yl dropped (relative ~3 2^-48 in all), renormalised
// into wyh + wyl. Every product (yh + yl)(wyh + wyl) enters a
// double-binary32 sum: yh wyh exactly (its error recovered with one FMA),
// the cross terms yh wyl and yl wyh in binary32 (relative 2^-48), yl wyl
// dropped (2^-48 of the product); the sum carries its error through TwoSum
// (Knuth; Dekker 1971; Ogita, Rump and Oishi 2005). Two rows per packed
// .f32x2 instruction, as in the refinement. b = sum rho d y stays FP64, with
// rho d formed once per grid point and row. GB300 issues FP64 at 1/64 of
// the binary32 rate, so no FP64 operation is left per lane and output
// entry. C goes out as renormalised binary32 pairs, high and low halves in
// two planes (MixScratch::C32, Clo), so that kernel (A) reads C rounded to
// binary32 and kernel (B) the pair without FP64 conversions; b stays FP64
// (b64).
template <int K>
__global__ void __launch_bounds__(32 * kGramPts, 1) local_gram_df_kernel(int nx, int ny, int k,
                                                                        ObsParams o, double d_cut,
                                                                        double aa, int cell0,
                                                                        int ncell, MixScratch sc) {
    constexpr int KC = 16;                      // rows per stage
    constexpr int RH = K > 64 ? 2 : 1;          // row ranges per column
    constexpr int KB = (K < 32 ? K : 32) / RH;  // output columns per pass
    constexpr int MR = K / RH;                  // rows per lane (even)
    constexpr int NBC = K > 32 ? K / 32 : 1;    // entries of b per lane
    static_assert(MR % 2 == 0, "row pairs");
    __shared__ double Ys[KC][K];
    __shared__ __align__(8) float Yh[KC][K];
    __shared__ __align__(8) float Yl[KC][K];
    __shared__ double WDs[kGramPts][KC];          // rho d of (point, row)
    __shared__ __align__(8) float Wh[kGramPts][KC];  // rho = Wh + Wl
    __shared__ __align__(8) float Wl[kGramPts][KC];
    __shared__ int wcount[kGramPts];
    __shared__ int pcnt[kGramPts];
    extern __shared__ int U[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int li0 = blockIdx.x * kGramPts;
    const int nv = o.nvar;
    const int total = gram_merge(o, nx, ny, d_cut, cell0, li0, ncell, U, pcnt, wcount);
    const long long lim2 = support_lim2(d_cut);
    const float aah = (float)aa, aal = (float)(aa - (double)aah);  // a = aah + aal
    bool any_ens = false;
    for (int q = 0; q < kGramPts; ++q) any_ens |= pcnt[q] * nv >= k;
    if (!any_ens) return;
    const int rows = total * nv;
    const int li = li0 + w;
    const int col = lane % KB, rh = lane / KB;
    const bool act = rh < RH;  // K = 16: lanes 16..31 own no column
    f2x S[MR / 2], Cc[MR / 2];
    double bacc[NBC];
#pragma unroll
    for (int c = 0; c < NBC; ++c) bacc[c] = 0.0;
    for (int cb = 0; cb < K; cb += KB) {
#pragma unroll
        for (int m = 0; m < MR / 2; ++m) S[m] = Cc[m] = 0ull;
        for (int r0 = 0; r0 < rows; r0 += KC) {
            for (int e = threadIdx.x; e < KC * K; e += 32 * kGramPts) {
                const int rr = e / K, c = e % K, r = r0 + rr;
                double v = 0.0;
                if (r < rows && c < k) v = o.dY[(size_t)(nv * U[r / nv] + r % nv) * k + c];
                const float h = (float)v;
                Ys[rr][c] = v;
                Yh[rr][c] = h;
                Yl[rr][c] = (float)(v - (double)h);
            }
            if (threadIdx.x < KC * kGramPts) {
                const int q = threadIdx.x / KC, rr = threadIdx.x % KC, r = r0 + rr;
                double wv = 0.0, dv = 0.0;
                if (r < rows && li0 + q < ncell) {
                    const int cell = cell0 + li0 + q;
                    const double sg = local_weight(o, U[r / nv], cell % nx, cell / nx, nx, ny, d_cut, lim2);
                    const int qv = r % nv;
                    const double l = sg / (qv == 0 ? o.sigma_u : (qv == 1 ? o.sigma_v : o.sigma_r));
                    wv = l * l;
                    dv = o.d[nv * U[r / nv] + qv];
                }
                const float h = (float)wv;
                Wh[q][rr] = h;
                Wl[q][rr] = (float)(wv - (double)h);
                WDs[q][rr] = wv * dv;
            }
            __syncthreads();
            for (int rr = 0; rr < KC; ++rr) {
                const float rhh = Wh[w][rr], rhl = Wl[w][rr];
                if (rhh == 0.0f) continue;  // rho = 0 (rh = 0 only then)
                if (cb == 0) {
                    const double wd = WDs[w][rr];
#pragma unroll
                    for (int c = 0; c < NBC; ++c)
                        if (lane + 32 * c < K) bacc[c] = fma(wd, Ys[rr][lane + 32 * c], bacc[c]);
                }
                if (act) {
                    // wy = rho y_n in double-binary32, renormalised (|e| << |p|).
                    const float yh = Yh[rr][cb + col], yl = Yl[rr][cb + col];
                    const float p = __fmul_rn(rhh, yh);
                    float e = __fmaf_rn(rhh, yh, -p);
                    e = __fmaf_rn(rhh, yl, __fmaf_rn(rhl, yh, e));
                    const float wh = __fadd_rn(p, e);
                    const float wlo = __fsub_rn(e, __fsub_rn(wh, p));
                    const f2x WH = f2pack(wh, wh), NWH = f2pack(-wh, -wh), WL = f2pack(wlo, wlo);
                    const f2x* yh2 = reinterpret_cast<const f2x*>(&Yh[rr][rh * MR]);
                    const f2x* yl2 = reinterpret_cast<const f2x*>(&Yl[rr][rh * MR]);
#pragma unroll
                    for (int m = 0; m < MR / 2; ++m) {
                        const f2x AH = yh2[m], AL = yl2[m];
                        df2_acc(S[m], Cc[m], AH, AL, WH, NWH);
                        Cc[m] = f2fma(AH, WL, Cc[m]);
                    }
                }
            }
            __syncthreads();
        }
        if (li < ncell && act) {
            // C = (s, c) + a I as renormalised binary32 pairs (high, low).
            float* Ch = sc.C32 + (size_t)li * k * k;
            float* Cl = sc.Clo + (size_t)li * k * k;
            const int n = cb + col;
#pragma unroll
            for (int m = 0; m < MR / 2; ++m) {
                float s0, s1, c0, c1;
                f2unpack(S[m], s0, s1);
                f2unpack(Cc[m], c0, c1);
                const int row0 = rh * MR + 2 * m;
                if (row0 < k && n < k) {
                    const size_t e0 = (size_t)row0 * k + n;
                    df_pair_out(s0, c0, row0 == n, aah, aal, Ch[e0], Cl[e0]);
                }
                if (row0 + 1 < k && n < k) {
                    const size_t e1 = (size_t)(row0 + 1) * k + n;
                    df_pair_out(s1, c1, row0 + 1 == n, aah, aal, Ch[e1], Cl[e1]);
                }
            }
        }
    }
    if (li >= ncell) return;
#pragma unroll
    for (int c = 0; c < NBC; ++c)
        if (lane + 32 * c < k) sc.b64[(size_t)li * k + lane + 32 * c] = bacc[c];
}

__global__ void __launch_bounds__(32 * kJacWarps, 5) mixed_jacobi_kernel(int nx, int ny, int k,
                                                                      ObsParams o, double d_cut,
                                                                      double beta, int cell0,
                                                                      int ncell, int nm,
                                                                      MixScratch sc,
                                                                      int* __restrict__ flags) {
    __shared__ __align__(16) float jrs[kJacWarps][2 * NREG];  // rotation slots per warp
    const int nobs = o.nvar * o.npts;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int li = blockIdx.x * kJacWarps + w;
    if (li >= ncell) return;
    const int cell = cell0 + li;
    const int x = cell % nx, y = cell / nx;
    const int cap = o.plmax > 0 ? o.plmax : nobs;
    double* lsq = sc.lsq + (size_t)li * cap;
    int* lidx = sc.lidx + (size_t)li * cap;
    const int p = local_set(o, x, y, nx, ny, d_cut, lane, lidx, lsq, cap);
    if (lane == 0) sc.pcount[li] = p;
    if (p == 0 || p > cap) return;  // p > cap: reported by kernel (B)
    const bool obs_space = p < k;
    const int n = obs_space ? p : k;
    if (n > nm || n > NREG) return;  // reported by kernel (B)
    const double aa = (k - 1) / beta;
    constexpr int xr = NREG;  // this kernel serves nm <= NREG
    float* Xp = sc.X + (size_t)li * xr * xr;
    const float* Cp = sc.C32 ? sc.C32 + (size_t)li * k * k : nullptr;
    const double* Cd = sc.C64 ? sc.C64 + (size_t)li * k * k : nullptr;
    if (n <= 8)
        jacobi_point<8>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, xr, flags, Cp, Cd, jrs[w]);
    else if (n <= 16)
        jacobi_point<16>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, xr, flags, Cp, Cd, jrs[w]);
    else if (n <= 24)
        jacobi_point<24>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, xr, flags, Cp, Cd, jrs[w]);
    else if (n <= 26)
        jacobi_point<26>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, xr, flags, Cp, Cd, jrs[w]);
    else if (n <= 28)
        jacobi_point<28>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, xr, flags, Cp, Cd, jrs[w]);
    else
        jacobi_point<32>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, xr, flags, Cp, Cd, jrs[w]);
}

// Observation-space points of the run kernel below, outside its register
// allocation.
template <int NS>
__device__ __noinline__ void jacobi_point_call(const ObsParams& o, int k, int n, int p, bool obs_space, double aa,
                                               const int* lidx, const double* lsq, int lane, float* Xp, int* flags,
                                               const float* Cp, const double* Cd, float* rs) {
    jacobi_point<NS>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, NREG, flags, Cp, Cd, rs);
}

// Kernel (A), one warp per run of `run` consecutive grid points of the
// chunk. Ensemble-space points (n = k, tile NE) start from the previous
// such point's basis (jacobi_point_warm; the first of a run from the
// identity through the same path); observation-space points are solved
// from the identity (jacobi_point).
template <int NE>
__global__ void __launch_bounds__(32 * kJacWarps, 4) mixed_jacobi_run_kernel(int nx, int ny, int k,
                                                                          ObsParams o, double d_cut,
                                                                          double beta, int cell0,
                                                                          int ncell, int nm, int run,
                                                                          MixScratch sc,
                                                                          int* __restrict__ flags) {
    extern __shared__ __align__(16) float jsm[];  // [kJacWarps][2][NE * NE]
    __shared__ __align__(16) float jrs[kJacWarps][2 * NREG];  // rotation slots per warp
    const int nobs = o.nvar * o.npts;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* Cs = jsm + (size_t)w * 2 * NE * NE;
    float* Us = Cs + NE * NE;
    float up[NREG];
#pragma unroll
    for (int i = 0; i < NREG; ++i) up[i] = (i == lane) ? 1.0f : 0.0f;
    for (int t = 0; t < run; ++t) {
        const long long lil = ((long long)blockIdx.x * kJacWarps + w) * run + t;
        if (lil >= ncell) return;
        const int li = (int)lil;
        const int cell = cell0 + li;
        const int x = cell % nx, y = cell / nx;
        const int cap = o.plmax > 0 ? o.plmax : nobs;
        double* lsq = sc.lsq + (size_t)li * cap;
        int* lidx = sc.lidx + (size_t)li * cap;
        const int p = local_set(o, x, y, nx, ny, d_cut, lane, lidx, lsq, cap);
        if (lane == 0) sc.pcount[li] = p;
        if (p == 0 || p > cap) continue;  // p > cap: reported by kernel (B)
        const bool obs_space = p < k;
        const int n = obs_space ? p : k;
        if (n > nm || n > NREG) continue;  // reported by kernel (B)
        const double aa = (k - 1) / beta;
        float* Xp = sc.X + (size_t)li * NREG * NREG;
        const float* Cp = sc.C32 ? sc.C32 + (size_t)li * k * k : nullptr;
        const double* Cd = sc.C64 ? sc.C64 + (size_t)li * k * k : nullptr;
        if (!obs_space && (Cp || Cd)) {
            jacobi_point_warm<NE>(o, k, n, lane, Xp, flags, Cp, Cd, up, Cs, Us, jrs[w]);
        } else if (n <= 8) {
            jacobi_point_call<8>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, flags, Cp, Cd, jrs[w]);
        } else if (n <= 16) {
            jacobi_point_call<16>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, flags, Cp, Cd, jrs[w]);
        } else if (n <= 24) {
            jacobi_point_call<24>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, flags, Cp, Cd, jrs[w]);
        } else if (n <= 28) {
            jacobi_point_call<28>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, flags, Cp, Cd, jrs[w]);
        } else {
            jacobi_point_call<32>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, flags, Cp, Cd, jrs[w]);
        }
    }
}

// Kernel (A) for local problems of 33..128: the binary32 Jacobi of
// jacobi_sym_block, kBlkThreads threads per grid point, same output.
constexpr int kBlkThreads = 256;
constexpr int kWideWarps = 4;  // warps per grid point of kernel (B) above NREG

__host__ __device__ inline size_t jacobi_block_smem_bytes(int nm) {
    return 2 * (size_t)nm * (nm + 1) * sizeof(float) + 64 * (2 * sizeof(float) + 2 * sizeof(int)) +
           4 * sizeof(unsigned) + (kBlkThreads / 32) * sizeof(float) + sizeof(int);
}

__global__ void __launch_bounds__(kBlkThreads) mixed_jacobi_block_kernel(int nx, int ny, int k, ObsParams o,
                                                                         double d_cut, double beta,
                                                                         int cell0, int nm, MixScratch sc,
                                                                         int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nobs = o.nvar * o.npts;
    const int ld = nm + 1;
    float* A = reinterpret_cast<float*>(smem_raw);
    float* U = A + (size_t)nm * ld;
    float* rc = U + (size_t)nm * ld;
    float* rs = rc + 64;
    int* rp = reinterpret_cast<int*>(rs + 64);
    int* rq = rp + 64;
    unsigned* mask = reinterpret_cast<unsigned*>(rq + 64);
    float* red = reinterpret_cast<float*>(mask + 4);
    int* pshare = reinterpret_cast<int*>(red + kBlkThreads / 32);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int li = blockIdx.x;
    const int cell = cell0 + li;
    const int x = cell % nx, y = cell / nx;
    const int cap = o.plmax > 0 ? o.plmax : nobs;
    double* lsq = sc.lsq + (size_t)li * cap;
    int* lidx = sc.lidx + (size_t)li * cap;
    if (w == 0) {
        const int p = local_set(o, x, y, nx, ny, d_cut, lane, lidx, lsq, cap);
        if (lane == 0) {
            sc.pcount[li] = p;
            *pshare = p;
        }
    }
    __syncthreads();
    const int p = *pshare;
    if (p == 0 || p > cap) return;  // p > cap: reported by kernel (B)
    const bool obs_space = p < k;
    const int n = obs_space ? p : k;
    if (n > nm) return;  // reported by kernel (B)
    const double aa = (k - 1) / beta;
    for (int e = tid; e < n * n; e += kBlkThreads) {
        const int i = e / n, c = e % n;
        float v;
        if (obs_space) {
            v = (float)(lsq[i] * o.G[(size_t)lidx[i] * nobs + lidx[c]] * lsq[c]);
        } else if (sc.C32) {
            v = sc.C32[(size_t)li * k * k + (size_t)i * k + c];
        } else if (sc.C64) {
            v = (float)sc.C64[(size_t)li * k * k + (size_t)i * k + c];
        } else {
            double s = (i == c) ? aa : 0.0;
            for (int l = 0; l < p; ++l) {
                const double* row = o.dY + (size_t)lidx[l] * k;
                s += lsq[l] * lsq[l] * row[i] * row[c];
            }
            v = (float)s;
        }
        A[i * ld + c] = v;
        U[i * ld + c] = (i == c) ? 1.0f : 0.0f;
    }
    __syncthreads();
    // Stop at 1e-6 ||A||_F: the refinement of kernel (B) is second order in
    // what remains.
    const int sweeps = jacobi_sym_block<kBlkThreads>(A, U, n, ld, rc, rs, rp, rq, mask, red, 1e-6f, kMaxSweeps);
    if (sweeps < 0 && tid == 0) atomicOr(flags, FLAG_NOCONV);
    if (w == 0) record_sweeps(o, sweeps, lane);
    const int xr = mix_xr(nm);
    float* Xp = sc.X + (size_t)li * xr * xr;
    for (int e = tid; e < n * n; e += kBlkThreads) {
        const int i = e / n, c = e % n;
        Xp[(size_t)i * xr + c] = U[i * ld + c];
    }
}

// Shared memory of kernel (B). The matrices are nm x ld with nm the largest
// local problem of this launch and ld = nm + 1 rounded to odd; vectors have
// nm entries.
struct MixSmem {
    // Six binary32 matrices, reused as the analysis proceeds:
    float* Ah;     // [nm][ld] A, high binary32 half; then S' off the diagonal
    float* Al;     // [nm][ld] A, low half; then Y f2(S) (ensemble space)
    float* Wh;     // [nm][ld] A Y, high half; then f(S) in binary32 (F32), then T
    float* Wl;     // [nm][ld] A Y, low half
    float* Y32;    // [nm][ld] the basis (binary32, exact)
    float* E32;    // [nm][ld] E = Y^T Y - I (non-orthogonality of the basis); up to
                   // NMID it shares Al's space (A's low half is dead once A Y is formed)
    double* lsq;   // [nl]
    double* ldh;   // [nl]
    double* vb;    // [nm]
    double* dS;    // [nm] diagonal of S' (FP64)
    float* vu;     // [nm] (binary32: only read as binary32 factors of f(S))
    float* vinv;   // [nm]
    float* dX;     // [9][k]
    float* xbar;   // [16]
    float* Z;      // [9][nm]
    float* B;      // [9][nm]
    float* zv;     // [16]
    float* vf;     // [nm]
    float* t1f;    // [nm]
    float* t2f;    // [nm]
    int* lidx;     // [nl]
};

// Up to NMID five matrices (E32 shares Al's space): at n = 28 and k = 64,
// 22.3 KB per grid point, ten points per SM. Above NMID, Ah, Al, Wh and Wl
// live in the global scratch (MixScratch::big) and shared memory holds Y32
// and E32.
__host__ __device__ inline size_t mix_smem_bytes(int k, int nl, int nm) {
    const int ld = mix_ld(nm);
    const size_t d = 2 * (size_t)nl + 2 * (size_t)nm;
    const size_t f = (nm > NMID ? 2 : 5) * (size_t)nm * ld + 9 * (size_t)k + 16 + 18 * (size_t)nm + 16 +
                     5 * (size_t)nm;
    return d * sizeof(double) + ((f * sizeof(float) + 7) / 8) * 8 + (size_t)nl * sizeof(int);
}

// big: this grid point's 4 nm ld floats of global scratch, or null.
__device__ inline MixSmem carve_mix(unsigned char* raw, int k, int nl, int nm, float* big) {
    const int ld = mix_ld(nm);
    MixSmem s;
    double* p = reinterpret_cast<double*>(raw);
    s.lsq = p;
    p += nl;
    s.ldh = p;
    p += nl;
    s.vb = p;
    p += nm;
    s.dS = p;
    p += nm;
    float* q = reinterpret_cast<float*>(p);
    float* m = big ? big : q;
    s.Ah = m;
    m += nm * ld;
    s.Al = m;
    m += nm * ld;
    s.Wh = m;
    m += nm * ld;
    s.Wl = m;
    m += nm * ld;
    if (!big) q = m;
    s.Y32 = q;
    q += nm * ld;
    if (big) {
        s.E32 = q;
        q += nm * ld;
    } else {
        s.E32 = s.Al;
    }
    s.dX = q;
    q += 9 * k;
    s.xbar = q;
    q += 16;
    s.Z = q;
    q += 9 * nm;
    s.B = q;
    q += 9 * nm;
    s.zv = q;
    q += 16;
    s.vf = q;
    q += nm;
    s.t1f = q;
    q += nm;
    s.t2f = q;
    q += nm;
    s.vu = q;
    q += nm;
    s.vinv = q;
    q += nm;
    const size_t fbytes = (size_t)(q - reinterpret_cast<float*>(p)) * sizeof(float);
    s.lidx = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(p) + ((fbytes + 7) / 8) * 8);
    return s;
}

// ---- Double-binary32 products (two_sum, df_acc: letkf_device.cuh) ---------

// C = P^T Q over the upper triangle (mirrored) in double-binary32: P binary32,
// Q = Qhi + Qlo (Qlo may be null). store(i, j, value) writes both halves.
// Thread t of NW warps takes entries t, t + 32 NW, ...
template <int NW = 1, typename Store>
__device__ void sym_product_df(const float* P, const float* Qhi, const float* Qlo, int n, int ld, int t,
                               Store&& store) {
    const int ne = n * (n + 1) / 2;
    for (int e0 = t; e0 < ne; e0 += 32 * NW) {
        int i = 0, j = e0;
        while (j >= n - i) {
            j -= n - i;
            ++i;
        }
        j += i;
        float s = 0.0f, c = 0.0f;
        for (int r = 0; r < n; ++r)
            df_acc(s, c, Qhi[r * ld + j], Qlo ? Qlo[r * ld + j] : 0.0f, P[r * ld + i]);
        store(i, j, df_value(s, c));
    }
}

// Rayleigh-Ritz refinement of the binary32 basis Y32 (exact) of the FP64
// matrix A = Ah + Al (two binary32 halves) without re-orthonormalising it.
// With E = Y^T Y - I (|E| ~ 1e-6), Y M^{-1/2} (M = I + E) is orthonormal
// and M^{-1/2} = I - E/2 + O(E^2), so
//   S' = M^{-1/2} (Y^T A Y) M^{-1/2} = S - (E S + S E)/2 + O(E^2)
// and, S being diagonal up to O(1e-6), (E S + S E)/2 = E o (d_i + d_j)/2 up
// to O(E |S_offdiag|): S' costs O(n^2) instead of a Cholesky factor and a
// triangular solve. The same first-order factor returns in the matrix
// functions (F - E o (f_i + f_j)/2, applied by the caller). The neglected
// terms are O(|E|^2) ~ 1e-11 relative. The products Y^T Y, A Y and
// Y^T (A Y) are double-binary32 (A Y goes to Wh + Wl). Leaves E in E32, the
// diagonal of S' in dS (FP64) and its off-diagonal in Soff (binary32: the
// entries are ~1e-6 of |A| and enter the matrix functions to first order).
// Soff may alias Ah and E32 may alias Al (A is not read after A Y).
template <bool WIDE, int NW = 1>
__device__ void refine_rr(const float* Ah, const float* Al, const float* Y32, float* Wh, float* Wl,
                          float* E32, float* Soff, double* dS, int n, int ld, int t) {
    // W = A Y, column col: four rows at a time, then the remainder.
    for_cols<WIDE, NW>(t, n, [&](int col) {
        int i0 = 0;
        for (; i0 + 3 < n; i0 += 4) {
            float s[4] = {0.0f, 0.0f, 0.0f, 0.0f}, c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int cc = 0; cc < n; ++cc) {
                const float y = Y32[cc * ld + col];
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    df_acc(s[r], c[r], Ah[(i0 + r) * ld + cc], Al[(i0 + r) * ld + cc], y);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) two_sum(s[r], c[r], Wh[(i0 + r) * ld + col], Wl[(i0 + r) * ld + col]);
        }
        for (; i0 < n; ++i0) {
            float s = 0.0f, c = 0.0f;
            for (int cc = 0; cc < n; ++cc) df_acc(s, c, Ah[i0 * ld + cc], Al[i0 * ld + cc], Y32[cc * ld + col]);
            two_sum(s, c, Wh[i0 * ld + col], Wl[i0 * ld + col]);
        }
    });
    point_sync<NW>();
    // E = Y^T Y - I.
    sym_product_df<NW>(Y32, Y32, nullptr, n, ld, t, [&](int i, int j, double v) {
        const float e = (float)(v - (i == j ? 1.0 : 0.0));
        E32[i * ld + j] = e;
        E32[j * ld + i] = e;
    });
    // S = Y^T (A Y), symmetric: diagonal to dS, off-diagonal to Soff.
    sym_product_df<NW>(Y32, Wh, Wl, n, ld, t, [&](int i, int j, double v) {
        if (i == j) {
            dS[i] = v;
        } else {
            Soff[i * ld + j] = (float)v;
            Soff[j * ld + i] = (float)v;
        }
    });
    point_sync<NW>();
    // S' = S - E o (d_i + d_j)/2 (the diagonal last, after every thread has
    // read the uncorrected one).
    for_cols<WIDE, NW>(t, n, [&](int c) {
        const double dc = dS[c];
        for (int i = 0; i < n; ++i)
            if (i != c)
                Soff[i * ld + c] = (float)((double)Soff[i * ld + c] - (double)E32[i * ld + c] * 0.5 * (dS[i] + dc));
    });
    point_sync<NW>();
    for_cols<WIDE, NW>(t, n, [&](int c) { dS[c] -= (double)E32[c * ld + c] * dS[c]; });
    point_sync<NW>();
}

// BIG (nm > NMID): A and A Y in global scratch (L2-resident), the rest as
// below. NW warps share a grid point (1 up to NREG).
template <bool WIDE, bool BIG, int NW>
__global__ void __launch_bounds__(32 * NW) analyze_mixed_kernel(float* __restrict__ f, int nx, int ny,
                                                           int k, ObsParams o, double d_cut,
                                                           double beta, int cell0, int nm,
                                                           MixScratch sc,
                                                           int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nobs = o.nvar * o.npts;
    const int cap = o.plmax > 0 ? o.plmax : nobs;
    const int li = blockIdx.x;
    MixSmem sm = carve_mix(smem_raw, k, cap, nm, BIG ? sc.big + (size_t)li * mix_big_floats(nm) : nullptr);
    const int ld = mix_ld(nm);
    constexpr int NTH = 32 * NW;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int cell = cell0 + li;
    const size_t plane = (size_t)nx * ny * k;
    float* fc = f + (size_t)cell * k;

    // Ensemble mean and perturbations in binary32.
    for (int a = wid; a < 9; a += NW) {  // one warp per component
        float s = 0.0f;
        for (int m = lane; m < k; m += 32) {
            const float xv = fc[a * plane + m];
            sm.dX[a * k + m] = xv;
            s += xv;
        }
        const float mean = warp_sum(s) / (float)k;
        for (int m = lane; m < k; m += 32) sm.dX[a * k + m] -= mean;
        if (lane == 0) sm.xbar[a] = mean;
    }

    // Local set from kernel (A).
    const int p = sc.pcount[li];
    if (p > cap) {
        if (tid == 0) atomicOr(flags, FLAG_TOOLARGE);
        return;
    }
    for (int i = tid; i < p; i += NTH) {
        const int oi = sc.lidx[(size_t)li * cap + i];
        const double si = sc.lsq[(size_t)li * cap + i];
        sm.lidx[i] = oi;
        sm.lsq[i] = si;
        sm.ldh[i] = si * o.d[oi];
    }
    point_sync<NW>();

    if (p == 0) {
        const float sb = (float)sqrt(beta);
        for (int a = 0; a < 9; ++a)
            for (int m = tid; m < k; m += NTH) fc[a * plane + m] = sm.xbar[a] + sb * sm.dX[a * k + m];
        return;
    }
    const bool obs_space = p < k;
    const int n = obs_space ? p : k;
    if (n > nm) {
        if (tid == 0) atomicOr(flags, FLAG_TOOLARGE);
        return;
    }
    const double aa = (k - 1) / beta;
    // A (FP64) goes to shared memory as two binary32 halves.
    auto put = [&](int i, int c, double v) {
        const float h = __double2float_rn(v);
        sm.Ah[i * ld + c] = h;
        sm.Al[i * ld + c] = __double2float_rn(v - (double)h);
    };

    // The symmetric matrix in FP64: A = Yh Yh^T (observation space) or
    // C = a I + Yh^T Yh with b = Yh^T d-hat (ensemble space); the basis X
    // from kernel (A).
    const int xr = WIDE ? mix_xr(nm) : NREG;
    const float* Xp = sc.X + (size_t)li * xr * xr;
    for_cols<WIDE, NW>(tid, n, [&](int c) {
        if (obs_space) {
            const int oc = sm.lidx[c];
            const double sl = sm.lsq[c];
            for (int i = 0; i < n; ++i)
                put(i, c, sm.lsq[i] * o.G[(size_t)sm.lidx[i] * nobs + oc] * sl);
        } else if (sc.Clo) {
            const float* Cp = sc.C32 + (size_t)li * k * k;
            const float* Cl = sc.Clo + (size_t)li * k * k;
            for (int i = 0; i < n; ++i) {
                sm.Ah[i * ld + c] = Cp[i * k + c];
                sm.Al[i * ld + c] = Cl[i * k + c];
            }
            sm.vb[c] = sc.b64[(size_t)li * k + c];
        } else if (sc.C32) {
            const float* Cp = sc.C32 + (size_t)li * k * k;
            for (int i = 0; i < n; ++i) {
                sm.Ah[i * ld + c] = Cp[i * k + c];
                sm.Al[i * ld + c] = 0.0f;
            }
            sm.vb[c] = (double)sc.b32[(size_t)li * k + c];
        } else if (sc.C64) {
            const double* Cd = sc.C64 + (size_t)li * k * k;
            for (int i = 0; i < n; ++i) put(i, c, Cd[i * k + c]);
            sm.vb[c] = sc.b64[(size_t)li * k + c];
        } else {
            double bj = 0.0;
            for (int i = 0; i < n; ++i) {
                double s = 0.0;
                for (int l = 0; l < p; ++l) {
                    const double* row = o.dY + (size_t)sm.lidx[l] * k;
                    s += sm.lsq[l] * sm.lsq[l] * row[i] * row[c];
                }
                put(i, c, s + (i == c ? aa : 0.0));
            }
            for (int l = 0; l < p; ++l) bj += sm.lsq[l] * o.dY[(size_t)sm.lidx[l] * k + c] * sm.ldh[l];
            sm.vb[c] = bj;
        }
        for (int i = 0; i < n; ++i) sm.Y32[i * ld + c] = Xp[(size_t)i * xr + c];
    });
    point_sync<NW>();
    refine_rr<WIDE, NW>(sm.Ah, sm.Al, sm.Y32, sm.Wh, sm.Wl, sm.E32, sm.Ah, sm.dS, n, ld, tid);
    const float* E32 = sm.E32;
    const float* Soff = sm.Ah;  // S' off the diagonal; its diagonal is dS
    float* Y32 = sm.Y32;
    float* F32 = sm.Wh;
    const float sk = (float)sqrt((double)(k - 1));

    if (obs_space) {
        // Functions of a + S: h = 1/(a+s) for the weights, g(s) = q[s, 0] with
        // q(s) = (a+s)^{-1/2} for the square root. u_i = sqrt(a + s_ii). The
        // scalars u_i, alpha_i and h_i enter binary32 products only, so they
        // are evaluated in binary32 (GB300's FP64 rate is 1/64 of it).
        const float af = (float)aa;
        const float rf = sqrtf(af);
        // d-hat in binary32, once (t2f is free until t2 is formed).
        for (int l = tid; l < n; l += NTH) sm.t2f[l] = (float)sm.ldh[l];
        point_sync<NW>();
        for_cols<WIDE, NW>(tid, n, [&](int c) {
            const float ap = af + (float)sm.dS[c];  // a + s_ii
            const float u = sqrtf(ap);
            sm.vu[c] = u;
            sm.vinv[c] = 1.0f / (u * (u + rf));  // alpha_i
            sm.vf[c] = 1.0f / ap;                // h_i = 1 / u_i^2 (vf is free until v)
            // t1 = Y^T d-hat (binary32 transform product).
            float t = 0.0f;
            for (int l = 0; l < n; ++l) t += Y32[l * ld + c] * sm.t2f[l];
            sm.t1f[c] = t;
        });
        point_sync<NW>();
        for_cols<WIDE, NW>(tid, n, [&](int c) {
            // t2 = h(S) t1 with h(S)_ii = h_i, h(S)_ij = -s_ij h_i h_j, and the
            // basis factor: minus E o (h_i + h_j)/2.
            const float hi = sm.vf[c];
            float t = 0.0f, te = 0.0f;
            for (int j = 0; j < n; ++j) {
                const float hj = sm.vf[j];
                if (j != c) t += Soff[c * ld + j] * (hj * sm.t1f[j]);
                te += E32[c * ld + j] * (0.5f * (hi + hj)) * sm.t1f[j];
            }
            sm.t2f[c] = hi * (sm.t1f[c] - t) - te;  // d-hat in t2f is read in the loop above only
            // g(S) in binary32: diagonal -alpha_i / r, off-diagonal
            // s_ij (u_i + u_j + r) alpha_i alpha_j / (r (u_i + u_j)).
            const float ai = sm.vinv[c];
            const float ui = sm.vu[c];
            const float gc = -ai / rf;
            for (int i = 0; i < n; ++i) {
                float v;
                const float aj = sm.vinv[i];
                if (i == c) {
                    v = gc;
                } else {
                    const float uj = (float)sm.vu[i];
                    v = Soff[i * ld + c] * (ui + uj + rf) * ai * aj / (rf * (ui + uj));
                }
                F32[i * ld + c] = v - E32[i * ld + c] * (0.5f * (gc - aj / rf));
            }
        });
        point_sync<NW>();
        for_cols<WIDE, NW>(tid, n, [&](int c) {
            float t = 0.0f;
            for (int l = 0; l < n; ++l) t += Y32[c * ld + l] * sm.t2f[l];
            sm.vf[c] = t;  // v = (a I + A)^{-1} d-hat
            // Z = dX Yh^T, column c: nine accumulators over members.
            const float* row = o.dY32 + (size_t)sm.lidx[c] * k;
            float acc[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] = 0.0f;
            for (int m = 0; m < k; ++m) {
                const float dy = row[m];
#pragma unroll
                for (int a = 0; a < 9; ++a) acc[a] += sm.dX[a * k + m] * dy;
            }
            const float sl = (float)sm.lsq[c];
#pragma unroll
            for (int a = 0; a < 9; ++a) sm.Z[a * nm + c] = sl * acc[a];
        });
        point_sync<NW>();
        if (tid < 9) {
            float s = 0.0f;
            for (int i = 0; i < n; ++i) s += sm.Z[tid * nm + i] * sm.vf[i];
            sm.zv[tid] = s;
        }
        for_cols<WIDE, NW>(tid, n, [&](int col) {
            float acc[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] = 0.0f;
            for (int c = 0; c < n; ++c) {
                const float yc = Y32[c * ld + col];
#pragma unroll
                for (int a = 0; a < 9; ++a) acc[a] += sm.Z[a * nm + c] * yc;
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) sm.B[a * nm + col] = acc[a];  // Z Y
        });
        point_sync<NW>();
        for_cols<WIDE, NW>(tid, n, [&](int col) {
            float acc[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] = 0.0f;
            for (int j = 0; j < n; ++j) {
                const float fj = F32[j * ld + col];
#pragma unroll
                for (int a = 0; a < 9; ++a) acc[a] += sm.B[a * nm + j] * fj;
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) sm.Z[a * nm + col] = acc[a];  // Z Y g(S)
        });
        point_sync<NW>();
        for_cols<WIDE, NW>(tid, n, [&](int col) {
            float acc[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] = 0.0f;
            for (int i = 0; i < n; ++i) {
                const float yi = Y32[col * ld + i];
#pragma unroll
                for (int a = 0; a < 9; ++a) acc[a] += sm.Z[a * nm + i] * yi;
            }
            const float sl = sk * (float)sm.lsq[col];
#pragma unroll
            for (int a = 0; a < 9; ++a) sm.B[a * nm + col] = sl * acc[a];  // sqrt(k-1) Z g(A) sqrt(rho)
        });
        point_sync<NW>();
        const float sb = (float)sqrt(beta);
        for (int m = tid; m < k; m += NTH) {
            float acc[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] = sm.xbar[a] + sm.zv[a] + sb * sm.dX[a * k + m];
            for (int i = 0; i < n; ++i) {
                const float dy = o.dY32[(size_t)sm.lidx[i] * k + m];
#pragma unroll
                for (int a = 0; a < 9; ++a) acc[a] += sm.B[a * nm + i] * dy;
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) fc[a * plane + m] = acc[a];
        }
    } else {
        // Functions of S directly: 1/lambda for P-tilde, lambda^{-1/2} for W,
        // evaluated in binary32 (they enter binary32 products only).
        for (int l = tid; l < n; l += NTH) sm.vf[l] = (float)sm.vb[l];  // b, once (vf is free until w-bar)
        point_sync<NW>();
        for_cols<WIDE, NW>(tid, n, [&](int c) {
            const float lam = (float)sm.dS[c];
            sm.vu[c] = sqrtf(lam);
            sm.vinv[c] = 1.0f / lam;
            float t = 0.0f;
            for (int l = 0; l < n; ++l) t += Y32[l * ld + c] * sm.vf[l];
            sm.t1f[c] = t;  // Y^T b
        });
        point_sync<NW>();
        for_cols<WIDE, NW>(tid, n, [&](int c) {
            // t2 = f1(S) t1, f1(S)_ii = 1/l_i, f1(S)_ij = -s_ij / (l_i l_j), and
            // the basis factor: minus E o (f1_i + f1_j)/2.
            const float fc1 = (float)sm.vinv[c];
            float t = 0.0f, te = 0.0f;
            for (int j = 0; j < n; ++j) {
                const float fj = (float)sm.vinv[j];
                if (j != c) t += Soff[c * ld + j] * (fj * sm.t1f[j]);
                te += E32[c * ld + j] * (0.5f * (fc1 + fj)) * sm.t1f[j];
            }
            sm.t2f[c] = fc1 * (sm.t1f[c] - t) - te;
            // f2(S) = S^{-1/2}: diagonal 1/sqrt(l_i), off-diagonal
            // -s_ij / (sqrt(l_i) sqrt(l_j) (sqrt(l_i) + sqrt(l_j))).
            const float si = (float)sm.vu[c];
            for (int i = 0; i < n; ++i) {
                float v;
                const float sj = (float)sm.vu[i];
                if (i == c) {
                    v = 1.0f / si;
                } else {
                    v = -Soff[i * ld + c] / (si * sj * (si + sj));
                }
                F32[i * ld + c] = v - E32[i * ld + c] * (0.5f * (1.0f / si + 1.0f / sj));
            }
        });
        point_sync<NW>();
        float* YF = sm.Al;  // A's low half is no longer needed
        for_cols<WIDE, NW>(tid, n, [&](int c) {
            float t = 0.0f;
            for (int l = 0; l < n; ++l) t += Y32[c * ld + l] * sm.t2f[l];
            sm.vf[c] = t;  // w-bar
        });
        point_sync<NW>();
        for_cols<WIDE, NW>(tid, n, [&](int c) {
            for (int i = 0; i < n; ++i) {
                float s = 0.0f;
                for (int l = 0; l < n; ++l) s += Y32[i * ld + l] * F32[l * ld + c];
                YF[i * ld + c] = s;
            }
    });
        point_sync<NW>();
        // T = sqrt(k-1) Y f2(S) Y^T + w-bar 1^T, over F32.
        for_cols<WIDE, NW>(tid, n, [&](int c) {
            for (int i = 0; i < n; ++i) {
                float s = 0.0f;
                for (int l = 0; l < n; ++l) s += YF[i * ld + l] * Y32[c * ld + l];
                F32[i * ld + c] = sk * s + sm.vf[i];
            }
    });
        point_sync<NW>();
        for (int m = tid; m < k; m += NTH) {
            for (int a = 0; a < 9; ++a) {
                float s = 0.0f;
                for (int j = 0; j < k; ++j) s += sm.dX[a * k + j] * F32[j * ld + m];
                fc[a * plane + m] = sm.xbar[a] + s;
            }
        }
    }
}

__global__ void to_f32_kernel(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)src[i];
}

}  // namespace

cudaError_t launch_run_fp64(double* f, int nx, int ny, int k, const ObsParams& o, double d_cut, double beta,
                            int run_len, int run0, int nruns, int ns, const float* Yg, const float* lamg,
                            const int* rinfo, int info_stride, int* flags, cudaStream_t s) {
    auto go = [&](auto kern, size_t sh) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)((size_t)nruns * run_len), 32, sh, s>>>(f, nx, ny, k, o, d_cut, beta, run_len, run0, Yg,
                                                                  lamg, rinfo, info_stride, flags);
        return cudaGetLastError();
    };
    switch (ns) {
        case 8: return go(run_fp64_kernel<8>, AnaSmem<8>::bytes(k, 8));
        case 16: return go(run_fp64_kernel<16>, AnaSmem<16>::bytes(k, 16));
        case 24: return go(run_fp64_kernel<24>, AnaSmem<24>::bytes(k, 24));
        case 28: return go(run_fp64_kernel<28>, AnaSmem<28>::bytes(k, 28));
        case 32: return go(run_fp64_kernel<32>, AnaSmem<32>::bytes(k, 32));
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_observe(const void* f, int fp32, int nx, int ny, int k, int npts, int nvar,
                           const int* ix, const int* iy, const double* yo, double* dY, double* d,
                           cudaStream_t s) {
    if (npts <= 0) return cudaSuccess;
    if (nvar != 2 && nvar != 3) return cudaErrorInvalidValue;
    const size_t sh = (3 * (size_t)k + 12) * sizeof(double);
    if (fp32)
        observe_kernel<float, true><<<npts, 128, sh, s>>>((const float*)f, nx, ny, k, nvar, ix, iy,
                                                          yo, dY, d);
    else
        observe_kernel<double, false><<<npts, 128, sh, s>>>((const double*)f, nx, ny, k, nvar, ix,
                                                            iy, yo, dY, d);
    return cudaGetLastError();
}

cudaError_t launch_obs_gram(const double* dY, int nobs, int k, double* G, cudaStream_t s) {
    if (nobs <= 0) return cudaSuccess;
    dim3 grid((nobs + 127) / 128, nobs);
    obs_gram_kernel<<<grid, 128, 0, s>>>(dY, nobs, k, G);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* src, float* dst, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    to_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

static int mixed_nm(int nmax) { return nmax < 2 ? 2 : (nmax > NMAX ? NMAX : nmax); }

// Members k when a Gram pass runs (mixed precision, some ensemble-space grid
// point, k <= 128), else 0; the bytes of its elements.
static int gram_k(int fp32, int k, int prod) {
    return (fp32 && prod != PROD_NONE && k <= NMAX) ? k : 0;
}
static int gram_sz(int prod) { return (prod == PROD_FP64 || prod == PROD_DF32) ? 8 : 4; }

template <int MODE>
static cudaError_t launch_gram_mode(int nx, int ny, int k, const ObsParams& o, double d_cut,
                                    double aa, int cell0, int nc, const MixScratch& sc,
                                    cudaStream_t s) {
    const size_t sh = (size_t)(o.npts > 0 ? o.npts : 1) * sizeof(int);
    const unsigned grid = (unsigned)((nc + kGramPts - 1) / kGramPts);
    auto go = [&](auto kern) {
        // The limit covers static plus dynamic shared memory above 48 KB.
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e != cudaSuccess) return e;
        kern<<<grid, 32 * kGramPts, sh, s>>>(nx, ny, k, o, d_cut, aa, cell0, nc, sc);
        return cudaGetLastError();
    };
    if constexpr (MODE == PROD_FP64) {
        if (k <= 16) return go(local_gram_fp64_kernel<16>);
        if (k <= 32) return go(local_gram_fp64_kernel<32>);
        if (k <= 64) return go(local_gram_fp64_kernel<64>);
        return go(local_gram_fp64_kernel<128>);
    } else if constexpr (MODE == PROD_DF32) {
        if (k <= 16) return go(local_gram_df_kernel<16>);
        if (k <= 32) return go(local_gram_df_kernel<32>);
        if (k <= 64) return go(local_gram_df_kernel<64>);
        return go(local_gram_df_kernel<128>);
    } else {
        if (k <= 16) return go(local_gram_kernel<16>);
        if (k <= 32) return go(local_gram_kernel<32>);
        if (k <= 64) return go(local_gram_kernel<64>);
        return go(local_gram_kernel<128>);
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library), or null.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tensor map of the binary32 dY [nobs][k] with boxes of one row (k values):
// TMA needs k * 4 bytes to be a multiple of 16 and a 16-byte aligned base.
static bool make_row_map(CUtensorMap* map, const float* dY32, int nobs, int k) {
    const auto enc = tensor_map_encoder();
    if (!enc || k % 4 != 0 || k > 256 || nobs < 1 || (reinterpret_cast<uintptr_t>(dY32) & 15u)) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)nobs};
    const cuuint64_t strides[1] = {(cuuint64_t)k * 4};
    const cuuint32_t box[2] = {(cuuint32_t)k, 1};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(dY32), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <bool TF32, int KP>
static cudaError_t launch_gram_tc_kp(int nx, int ny, int k, const ObsParams& o, double d_cut, double aa,
                                     int cell0, int nc, const MixScratch& sc, int* flags, cudaStream_t s) {
    CUtensorMap map;
    memset(&map, 0, sizeof map);
    const int use_tma = make_row_map(&map, o.dY32, o.nvar * o.npts, k) ? 1 : 0;
    const size_t sh = tc_gram_smem<TF32, KP>(o.npts);
    if (sh > 227 * 1024) return cudaErrorInvalidValue;  // merged list too long for shared memory
    const auto kern = local_gram_tc_kernel<TF32, KP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((nc + kGramPts - 1) / kGramPts);
    kern<<<grid, 32 * kGramPts, sh, s>>>(nx, ny, k, o, d_cut, aa, cell0, nc, sc, map, use_tma, flags);
    return cudaGetLastError();
}

template <bool TF32>
static cudaError_t launch_gram_tc(int nx, int ny, int k, const ObsParams& o, double d_cut, double aa, int cell0,
                                  int nc, const MixScratch& sc, int* flags, cudaStream_t s) {
    if (k <= 16) return launch_gram_tc_kp<TF32, 16>(nx, ny, k, o, d_cut, aa, cell0, nc, sc, flags, s);
    if (k <= 32) return launch_gram_tc_kp<TF32, 32>(nx, ny, k, o, d_cut, aa, cell0, nc, sc, flags, s);
    if (k <= 64) return launch_gram_tc_kp<TF32, 64>(nx, ny, k, o, d_cut, aa, cell0, nc, sc, flags, s);
    return launch_gram_tc_kp<TF32, 128>(nx, ny, k, o, d_cut, aa, cell0, nc, sc, flags, s);
}

static cudaError_t launch_gram(int prod, int nx, int ny, int k, const ObsParams& o, double d_cut,
                               double aa, int cell0, int nc, const MixScratch& sc, int* flags, cudaStream_t s) {
    if (prod == PROD_FP64) return launch_gram_mode<PROD_FP64>(nx, ny, k, o, d_cut, aa, cell0, nc, sc, s);
    if (prod == PROD_DF32) return launch_gram_mode<PROD_DF32>(nx, ny, k, o, d_cut, aa, cell0, nc, sc, s);
    if (prod == PROD_FP32) return launch_gram_mode<PROD_FP32>(nx, ny, k, o, d_cut, aa, cell0, nc, sc, s);
    if (prod == PROD_TF32) return launch_gram_tc<true>(nx, ny, k, o, d_cut, aa, cell0, nc, sc, flags, s);
    return launch_gram_tc<false>(nx, ny, k, o, d_cut, aa, cell0, nc, sc, flags, s);
}

size_t analyze_scratch_bytes(int nx, int ny, int fp32, int nl, int nmax, int k, int prod) {
    if (!fp32) return 0;
    const int nm = mixed_nm(nmax);
    const int kg = gram_k(fp32, k, prod), gsz = gram_sz(prod);
    const long long cells = (long long)nx * ny;
    const long long chunk = mix_chunk(cells, nl, nm, kg, gsz);
    return (chunk < cells ? 2 : 1) * mix_buf_bytes(chunk, nl, nm, kg, gsz);  // double-buffered
}

cudaError_t launch_analyze(void* f, int fp32, int nx, int ny, int k, const ObsParams& o,
                           double d_cut, double beta, int nmax, int prod, int warm_run, int* flags,
                           void* scratch, const AnalyzeAux* aux, cudaStream_t s) {
    const long long cells = (long long)nx * ny;
    if (cells > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    cudaError_t e;
    if (fp32) {
        if (!o.dY32 || !scratch || !aux) return cudaErrorInvalidValue;
        const int nobs = o.nvar * o.npts;
        const int nm = mixed_nm(nmax);
        const size_t nd = (size_t)nobs * k;
        to_f32_kernel<<<(unsigned)((nd + 255) / 256), 256, 0, s>>>(o.dY, o.dY32, nd);
        const int cap = o.plmax > 0 ? o.plmax : nobs;
        const size_t shB = mix_smem_bytes(k, cap, nm);
        const bool wide = nm > NREG, big = nm > NMID;
        const size_t shA = wide ? jacobi_block_smem_bytes(nm) : 0;
        // Above NREG a grid point has kWideWarps warps in kernel (B).
        auto kernB = big ? analyze_mixed_kernel<true, true, kWideWarps>
                         : (wide ? analyze_mixed_kernel<true, false, kWideWarps> : analyze_mixed_kernel<false, false, 1>);
        const int thB = wide ? 32 * kWideWarps : 32;
        e = cudaFuncSetAttribute(kernB, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shB);
        if (e != cudaSuccess) return e;
        if (wide) {
            e = cudaFuncSetAttribute(mixed_jacobi_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shA);
            if (e != cudaSuccess) return e;
        }
        const int kg = gram_k(fp32, k, prod), gsz = gram_sz(prod);
        // Runs of kernel (A): warm starts between ensemble-space points
        // (their C comes from the Gram pass).
        const int runA = (kg && warm_run > 1) ? warm_run : 1;
        const int ne = k <= 8 ? 8 : (k <= 16 ? 16 : (k <= 24 ? 24 : (k <= 28 ? 28 : 32)));
        const size_t shJ = runA > 1 ? (size_t)kJacWarps * 2 * ne * ne * sizeof(float) : 0;
        auto kernJ = ne == 8 ? mixed_jacobi_run_kernel<8>
                             : (ne == 16 ? mixed_jacobi_run_kernel<16>
                                         : (ne == 24 ? mixed_jacobi_run_kernel<24>
                                                     : (ne == 28 ? mixed_jacobi_run_kernel<28>
                                                                 : mixed_jacobi_run_kernel<32>)));
        if (runA > 1 && nm <= NREG) {
            e = cudaFuncSetAttribute(kernJ, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shJ);
            if (e != cudaSuccess) return e;
        }
        const long long chunk = mix_chunk(cells, cap, nm, kg, gsz);
        const size_t buf_bytes = mix_buf_bytes(chunk, cap, nm, kg, gsz);
        // Pipeline: (A) of chunk c on s2 overlaps (B) of chunk c-1 on s; the
        // scratch is double-buffered, (A) of chunk c waits for (B) of c-2.
        if ((e = cudaEventRecord(aux->start, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(aux->s2, aux->start, 0)) != cudaSuccess) return e;
        int c = 0;
        for (long long c0 = 0; c0 < cells; c0 += chunk, ++c) {
            const int nc = (int)((cells - c0) < chunk ? (cells - c0) : chunk);
            const int b = c & 1;
            MixScratch sc = mix_scratch_at((unsigned char*)scratch + b * buf_bytes, chunk, cap, nm, kg, gsz);
            if (prod == PROD_DF32) sc = mix_scratch_df2(sc, chunk, kg);
            if (c >= 2 && (e = cudaStreamWaitEvent(aux->s2, aux->ref_done[b], 0)) != cudaSuccess)
                return e;
            if (kg && (e = launch_gram(prod, nx, ny, k, o, d_cut, (k - 1) / beta, (int)c0, nc, sc, flags,
                                       aux->s2)) != cudaSuccess)
                return e;
            if (nm <= NREG && runA > 1)
                kernJ<<<(unsigned)((nc + kJacWarps * runA - 1) / (kJacWarps * runA)), 32 * kJacWarps, shJ,
                        aux->s2>>>(nx, ny, k, o, d_cut, beta, (int)c0, nc, nm, runA, sc, flags);
            else if (nm <= NREG)
                mixed_jacobi_kernel<<<(unsigned)((nc + kJacWarps - 1) / kJacWarps), 32 * kJacWarps, 0,
                                      aux->s2>>>(nx, ny, k, o, d_cut, beta, (int)c0, nc, nm, sc, flags);
            else
                mixed_jacobi_block_kernel<<<(unsigned)nc, kBlkThreads, shA, aux->s2>>>(nx, ny, k, o, d_cut, beta,
                                                                                       (int)c0, nm, sc, flags);
            if ((e = cudaEventRecord(aux->jac_done[b], aux->s2)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, aux->jac_done[b], 0)) != cudaSuccess) return e;
            kernB<<<(unsigned)nc, thB, shB, s>>>((float*)f, nx, ny, k, o, d_cut, beta, (int)c0, nm, sc, flags);
            if ((e = cudaEventRecord(aux->ref_done[b], s)) != cudaSuccess) return e;
        }
    } else {
        const int nobs = o.nvar * o.npts;
        if (nmax <= 32) {
            const size_t sh = AnaSmem<32>::bytes(k, o.plmax > 0 ? o.plmax : nobs);
            e = cudaFuncSetAttribute(analyze_fp64_kernel<32>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
            if (e != cudaSuccess) return e;
            analyze_fp64_kernel<32><<<(unsigned)cells, 32, sh, s>>>((double*)f, nx, ny, k, o, d_cut,
                                                                    beta, flags);
        } else {
            const size_t sh = AnaSmem<64>::bytes(k, o.plmax > 0 ? o.plmax : nobs);
            e = cudaFuncSetAttribute(analyze_fp64_kernel<64>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
            if (e != cudaSuccess) return e;
            analyze_fp64_kernel<64><<<(unsigned)cells, 32, sh, s>>>((double*)f, nx, ny, k, o, d_cut,
                                                                    beta, flags);
        }
    }
    return cudaGetLastError();
}

}  // namespace lbmgpu
