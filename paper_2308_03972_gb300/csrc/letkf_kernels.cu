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

#include "lbm_internal.cuh"

namespace lbmgpu {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int NMAX = 32;  // largest eigenproblem of the warp kernel
constexpr int LD = NMAX + 1;
constexpr int kMaxSweeps = 30;

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ int min_image(int d, int n) {
    if (d > n / 2) d -= n;
    if (d < -(n / 2)) d += n;
    return d;
}

// Gaspari-Cohn weight, both branches in nested (Horner) form.
__device__ __forceinline__ double gaspari_cohn(double d) {
    if (d <= 1.0) return 1.0 + d * d * (-5.0 / 3.0 + d * (0.625 + d * (0.5 - 0.25 * d)));
    if (d < 2.0)
        return d * d * (5.0 / 3.0 + d * (0.625 + d * (-0.5 + d * (1.0 / 12.0)))) - 5.0 * d + 4.0 -
               (2.0 / 3.0) / d;
    return 0.0;
}

// ------------------------------------------------------------------ K2
template <typename T, bool SHIFT>
__global__ void __launch_bounds__(128) observe_kernel(const T* __restrict__ f, int nx, int ny,
                                                      int k, const int* __restrict__ ix,
                                                      const int* __restrict__ iy,
                                                      const double* __restrict__ yo,
                                                      double* __restrict__ dY,
                                                      double* __restrict__ d) {
    extern __shared__ double sh[];  // yu[k], yv[k], red[2 * 4]
    double* yu = sh;
    double* yv = sh + k;
    double* red = sh + 2 * k;
    const int j = blockIdx.x;
    const size_t plane = (size_t)nx * ny * k;
    const size_t base = ((size_t)iy[j] * nx + ix[j]) * k;
    double su = 0.0, sv = 0.0;
    for (int m = threadIdx.x; m < k; m += blockDim.x) {
        double r = SHIFT ? 1.0 : 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const double g = (double)f[a * plane + base + m];
            r += g;
            jx += d2q9_cx(a) * g;
            jy += d2q9_cy(a) * g;
        }
        const double u = jx / r, v = jy / r;
        yu[m] = u;
        yv[m] = v;
        su += u;
        sv += v;
    }
    su = warp_sum(su);
    sv = warp_sum(sv);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[w] = su;
        red[4 + w] = sv;
    }
    __syncthreads();
    const double ubar = ((red[0] + red[1]) + (red[2] + red[3])) / k;
    const double vbar = ((red[4] + red[5]) + (red[6] + red[7])) / k;
    for (int m = threadIdx.x; m < k; m += blockDim.x) {
        dY[(size_t)(2 * j) * k + m] = yu[m] - ubar;
        dY[(size_t)(2 * j + 1) * k + m] = yv[m] - vbar;
    }
    if (threadIdx.x == 0) {
        d[2 * j] = yo[2 * j] - ubar;
        d[2 * j + 1] = yo[2 * j + 1] - vbar;
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

// ------------------------------------------------------------------ K3
// Cyclic Jacobi with round-robin ordering on the n x n symmetric matrix A
// (row-major, leading dimension LD, shared memory); U accumulates the
// rotations (U starts as I). One lane per column/row. A rotation is skipped
// when |a_pq| <= rel * ||A||_F; the solve stops after a sweep without
// rotations. Returns false if max_sweeps was reached. R is double or float.
template <typename R>
__device__ bool jacobi_warp(R* A, R* U, int n, int lane, R* rc, R* rs, int* rp, int* rq, R rel,
                            int max_sweeps) {
    const int np = n + (n & 1);
    const int half = np / 2;
    R fro = R(0);
    if (lane < n)
        for (int i = 0; i < n; ++i) fro += A[i * LD + lane] * A[i * LD + lane];
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
                R c = R(1), s = R(0);
                if (q < n) {
                    const R apq = A[p * LD + q];
                    if (fabs(apq) > thresh) {
                        // Symmetric 2 x 2 Schur decomposition.
                        const R app = A[p * LD + p], aqq = A[q * LD + q];
                        const R tau = (aqq - app) / (R(2) * apq);
                        const R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
                        c = R(1) / sqrt(R(1) + t * t);
                        s = t * c;
                        rot = true;
                    }
                }
                rp[lane] = p;
                rq[lane] = q;
                rc[lane] = c;
                rs[lane] = rot ? s : R(0);
            }
            const unsigned any = __ballot_sync(kFull, rot);
            __syncwarp();
            if (any == 0) continue;
            any_sweep = true;
            // A <- J^T A: rotate row pairs; lane owns column `lane`.
            if (lane < n) {
                for (int t = 0; t < half; ++t) {
                    if (!((any >> t) & 1u)) continue;
                    const int p = rp[t], q = rq[t];
                    const R c = rc[t], s = rs[t];
                    const R ap = A[p * LD + lane], aq = A[q * LD + lane];
                    A[p * LD + lane] = c * ap - s * aq;
                    A[q * LD + lane] = s * ap + c * aq;
                }
            }
            __syncwarp();
            // A <- A J and U <- U J: rotate column pairs; lane owns row `lane`.
            if (lane < n) {
                for (int t = 0; t < half; ++t) {
                    if (!((any >> t) & 1u)) continue;
                    const int p = rp[t], q = rq[t];
                    const R c = rc[t], s = rs[t];
                    const R ap = A[lane * LD + p], aq = A[lane * LD + q];
                    A[lane * LD + p] = c * ap - s * aq;
                    A[lane * LD + q] = s * ap + c * aq;
                    const R up = U[lane * LD + p], uq = U[lane * LD + q];
                    U[lane * LD + p] = c * up - s * uq;
                    U[lane * LD + q] = s * up + c * uq;
                }
            }
            __syncwarp();
            if (rot) {
                const int p = rp[lane], q = rq[lane];
                A[p * LD + q] = R(0);
                A[q * LD + p] = R(0);
            }
            __syncwarp();
        }
        if (!any_sweep) return true;
    }
    return false;
}

// FP64 cyclic Jacobi on the symmetric n x n matrix A (shared memory, row
// stride LD) with the same round-robin order, updating only what symmetry
// requires: each rotated pair's 2 x 2 diagonal block analytically
// (a_pp - t a_pq, a_qq + t a_pq, 0), the off-diagonal 2 x 2 blocks (P, Q),
// P < Q, as J_P^T X J_Q (mirrored), and the rows of U. A rotation is skipped
// when |a_pq| <= rel ||A||_F; the solve ends after a sweep without one.
// Returns false if max_sweeps was reached.
__device__ bool jacobi_sym_warp(double* A, double* U, int n, int lane, double* rc, double* rs,
                                double* rt, int* rp, int* rq, double rel, int max_sweeps) {
    const int np = n + (n & 1);
    const int half = np / 2;
    const int nb = half * (half - 1) / 2;
    double fro = 0.0;
    if (lane < n)
        for (int i = 0; i < n; ++i) fro += A[i * LD + lane] * A[i * LD + lane];
    fro = warp_sum(fro);
    const double thresh = rel * sqrt(fro);
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        bool any_sweep = false;
        for (int r = 0; r + 1 < np; ++r) {
            bool rot = false;
            if (lane < half) {
                const int pa = lane, pb = np - 1 - lane;
                const int P = pa == 0 ? 0 : 1 + (pa - 1 + r) % (np - 1);
                const int Q = 1 + (pb - 1 + r) % (np - 1);
                const int p = P < Q ? P : Q, q = P < Q ? Q : P;
                double c = 1.0, sn = 0.0, t = 0.0;
                if (q < n) {
                    const double apq = A[p * LD + q];
                    if (fabs(apq) > thresh) {
                        // t = phi / (theta + sgn(theta) sqrt(theta^2 + phi^2)),
                        // theta = a_qq - a_pp, phi = 2 a_pq: the smaller root of
                        // t^2 + 2 (theta / phi) t - 1 = 0.
                        const double app = A[p * LD + p], aqq = A[q * LD + q];
                        const double th = aqq - app, ph = 2.0 * apq;
                        const double rr = sqrt(th * th + ph * ph);
                        t = ph / (th >= 0.0 ? th + rr : th - rr);
                        c = rsqrt(1.0 + t * t);
                        sn = t * c;
                        rot = true;
                        // Diagonal block of the pair, analytically.
                        A[p * LD + p] = app - t * apq;
                        A[q * LD + q] = aqq + t * apq;
                        A[p * LD + q] = 0.0;
                        A[q * LD + p] = 0.0;
                    }
                }
                rp[lane] = p;
                rq[lane] = q;
                rc[lane] = c;
                rs[lane] = sn;
                rt[lane] = t;
            }
            const unsigned any = __ballot_sync(kFull, rot);
            __syncwarp();
            if (any == 0) continue;
            any_sweep = true;
            // Off-diagonal blocks (P, Q), P < Q, of the pairs of this round.
            for (int b = lane; b < nb; b += 32) {
                int P = 0, Q = b;
                while (Q >= half - 1 - P) { Q -= half - 1 - P; ++P; }
                Q += P + 1;
                const bool rP = (any >> P) & 1u, rQ = (any >> Q) & 1u;
                if (!rP && !rQ) continue;
                const int pP = rp[P], qP = rq[P], pQ = rp[Q], qQ = rq[Q];
                if (qP >= n || qQ >= n) continue;  // padding player
                const double cP = rc[P], sP = rs[P], cQ = rc[Q], sQ = rs[Q];
                const double x00 = A[pP * LD + pQ], x01 = A[pP * LD + qQ];
                const double x10 = A[qP * LD + pQ], x11 = A[qP * LD + qQ];
                // J_P^T X: rows p, q.
                const double y00 = cP * x00 - sP * x10, y01 = cP * x01 - sP * x11;
                const double y10 = sP * x00 + cP * x10, y11 = sP * x01 + cP * x11;
                // (J_P^T X) J_Q: columns p, q.
                const double z00 = cQ * y00 - sQ * y01, z01 = sQ * y00 + cQ * y01;
                const double z10 = cQ * y10 - sQ * y11, z11 = sQ * y10 + cQ * y11;
                A[pP * LD + pQ] = z00;
                A[pQ * LD + pP] = z00;
                A[pP * LD + qQ] = z01;
                A[qQ * LD + pP] = z01;
                A[qP * LD + pQ] = z10;
                A[pQ * LD + qP] = z10;
                A[qP * LD + qQ] = z11;
                A[qQ * LD + qP] = z11;
            }
            // U <- U J: rotate column pairs; lane owns row `lane`.
            if (lane < n) {
                for (int t = 0; t < half; ++t) {
                    if (!((any >> t) & 1u)) continue;
                    const int p = rp[t], q = rq[t];
                    const double c = rc[t], sn = rs[t];
                    const double up = U[lane * LD + p], uq = U[lane * LD + q];
                    U[lane * LD + p] = c * up - sn * uq;
                    U[lane * LD + q] = sn * up + c * uq;
                }
            }
            __syncwarp();
        }
        if (!any_sweep) return true;
    }
    return false;
}

struct AnaSmem {
    double* A;     // [NMAX][LD]
    double* U;     // [NMAX][LD]
    double* dX;    // [9][k]
    double* xbar;  // [16]
    double* lsq;   // [nl] sqrt of the localised inverse error variance
    double* ldh;   // [nl] sqrt(rho) * d
    double* v1;    // [NMAX]
    double* v2;    // [NMAX]
    double* v3;    // [NMAX]
    double* v4;    // [NMAX]
    double* v5;    // [NMAX]
    double* Z;     // [9][NMAX]
    double* B;     // [9][NMAX]
    double* zv;    // [16]
    double* rc;    // [NMAX / 2]
    double* rs;    // [NMAX / 2]
    double* rt;    // [NMAX / 2]
    int* rp;       // [NMAX / 2]
    int* rq;       // [NMAX / 2]
    int* lidx;     // [nl]
};

__host__ __device__ inline size_t ana_smem_bytes(int k, int nl) {
    size_t d = 2 * (size_t)NMAX * LD + 9 * (size_t)k + 16 + 2 * (size_t)nl + 5 * NMAX +
               18 * (size_t)NMAX + 16 + NMAX + NMAX / 2;
    return d * sizeof(double) + (size_t)(NMAX + nl) * sizeof(int);
}

__device__ inline AnaSmem carve(unsigned char* raw, int k, int nl) {
    AnaSmem s;
    double* p = reinterpret_cast<double*>(raw);
    s.A = p;
    p += NMAX * LD;
    s.U = p;
    p += NMAX * LD;
    s.dX = p;
    p += 9 * k;
    s.xbar = p;
    p += 16;
    s.lsq = p;
    p += nl;
    s.ldh = p;
    p += nl;
    s.v1 = p;
    p += NMAX;
    s.v2 = p;
    p += NMAX;
    s.v3 = p;
    p += NMAX;
    s.v4 = p;
    p += NMAX;
    s.v5 = p;
    p += NMAX;
    s.Z = p;
    p += 9 * NMAX;
    s.B = p;
    p += 9 * NMAX;
    s.zv = p;
    p += 16;
    s.rc = p;
    p += NMAX / 2;
    s.rs = p;
    p += NMAX / 2;
    s.rt = p;
    p += NMAX / 2;
    int* ip = reinterpret_cast<int*>(p);
    s.rp = ip;
    ip += NMAX / 2;
    s.rq = ip;
    ip += NMAX / 2;
    s.lidx = ip;
    return s;
}

template <typename T, bool SHIFT>
__global__ void __launch_bounds__(32) analyze_kernel(T* __restrict__ f, int nx, int ny, int k,
                                                     ObsParams o, double d_cut, double beta,
                                                     int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nobs = 2 * o.npts;
    AnaSmem sm = carve(smem_raw, k, nobs);
    const int lane = threadIdx.x;
    const int cell = blockIdx.x;
    const int x = cell % nx, y = cell / nx;
    const size_t plane = (size_t)nx * ny * k;
    T* fc = f + (size_t)cell * k;

    // Ensemble mean and perturbations of the nine components.
    for (int a = 0; a < 9; ++a) {
        double s = 0.0;
        for (int m = lane; m < k; m += 32) {
            const double xv = (double)fc[a * plane + m];
            sm.dX[a * k + m] = xv;
            s += xv;
        }
        const double mean = warp_sum(s) / k;
        for (int m = lane; m < k; m += 32) sm.dX[a * k + m] -= mean;
        if (lane == 0) sm.xbar[a] = mean;
    }

    // Local observation set: points with r / d_cut < 2 and G > 0, in
    // increasing point order, two scalars (u, v) per point.
    int count = 0;
    for (int j0 = 0; j0 < o.npts; j0 += 32) {
        const int j = j0 + lane;
        bool in = false;
        double g = 0.0;
        if (j < o.npts) {
            const int dx = min_image(o.ix[j] - x, nx);
            const int dy = min_image(o.iy[j] - y, ny);
            const double r = sqrt((double)dx * dx + (double)dy * dy);
            const double dist = r / d_cut;
            if (dist < 2.0) {
                g = gaspari_cohn(dist);
                in = g > 0.0;
            }
        }
        const unsigned bal = __ballot_sync(kFull, in);
        if (in) {
            const int pos = count + __popc(bal & ((1u << lane) - 1u));
            const double sg = sqrt(g);
            sm.lidx[2 * pos] = 2 * j;
            sm.lidx[2 * pos + 1] = 2 * j + 1;
            sm.lsq[2 * pos] = sg / o.sigma_u;
            sm.lsq[2 * pos + 1] = sg / o.sigma_v;
        }
        count += __popc(bal);
    }
    __syncwarp();
    const int p = 2 * count;
    for (int i = lane; i < p; i += 32) sm.ldh[i] = sm.lsq[i] * o.d[sm.lidx[i]];
    __syncwarp();

    if (p == 0) {
        // No observation in range: x^a_m = xbar + sqrt(beta) dx_m.
        const double sb = sqrt(beta);
        for (int a = 0; a < 9; ++a)
            for (int m = lane; m < k; m += 32)
                fc[a * plane + m] = (T)(sm.xbar[a] + sb * sm.dX[a * k + m]);
        return;
    }
    const bool obs_space = p < k;
    const int n = obs_space ? p : k;
    if (n > NMAX) {
        if (lane == 0) atomicOr(flags, FLAG_TOOLARGE);
        return;
    }
    const double aa = (k - 1) / beta;
    double* A = sm.A;
    double* U = sm.U;

    if (obs_space) {
        // A = Yh Yh^T gathered from the global Gram.
        if (lane < n) {
            const int ol = sm.lidx[lane];
            const double sl = sm.lsq[lane];
            for (int i = 0; i < n; ++i)
                A[i * LD + lane] = sm.lsq[i] * o.G[(size_t)sm.lidx[i] * nobs + ol] * sl;
        }
    } else {
        // C = a I + Yh^T Yh and b = Yh^T d-hat, column `lane`.
        if (lane < n) {
            double bj = 0.0;
            for (int i = 0; i < n; ++i) {
                double s = 0.0;
                for (int l = 0; l < p; ++l) {
                    const double* row = o.dY + (size_t)sm.lidx[l] * k;
                    const double w = sm.lsq[l] * sm.lsq[l];
                    s += w * row[i] * row[lane];
                }
                A[i * LD + lane] = s + (i == lane ? aa : 0.0);
            }
            for (int l = 0; l < p; ++l) bj += sm.lsq[l] * o.dY[(size_t)sm.lidx[l] * k + lane] * sm.ldh[l];
            sm.v3[lane] = bj;
        }
    }
    if (lane < n)
        for (int i = 0; i < n; ++i) U[i * LD + lane] = (i == lane) ? 1.0 : 0.0;
    __syncwarp();

    // Observation space: stop once the off-diagonal is below 1e-9 ||A||_F and
    // take the matrix functions to first order in it (Daleckii-Krein; the
    // neglected second-order term is below 1e-15 relative). Ensemble space
    // (small k) converges fully and uses the diagonal directly.
    if (!jacobi_sym_warp(A, U, n, lane, sm.rc, sm.rs, sm.rt, sm.rp, sm.rq,
                         obs_space ? 1e-9 : 1e-18, kMaxSweeps)) {
        if (lane == 0) atomicOr(flags, FLAG_NOCONV);
    }
    __syncwarp();

    if (obs_space) {
        // S = U^T A U (nearly diagonal, in A). With u_i = sqrt(a + s_ii),
        // h(s) = 1/(a+s) and g(s) = ((a+s)^{-1/2} - a^{-1/2}) / s:
        //   h(S)_ii = 1/u_i^2, h(S)_ij = -s_ij / (u_i^2 u_j^2),
        //   g(S)_ii = -alpha_i / r, g(S)_ij = s_ij (u_i+u_j+r) alpha_i alpha_j / (r (u_i+u_j)),
        // alpha_i = 1 / (u_i (u_i + r)), r = sqrt(a).
        const double rr = sqrt(aa);
        if (lane < n) {
            const double sii = A[lane * LD + lane];
            const double u = sqrt(aa + sii);
            sm.v3[lane] = u;
            sm.v4[lane] = 1.0 / (aa + sii);        // h_i
            sm.v5[lane] = 1.0 / (u * (u + rr));    // alpha_i
            double t = 0.0;
            for (int l = 0; l < n; ++l) t += U[l * LD + lane] * sm.ldh[l];
            sm.v1[lane] = t;  // t1 = U^T d-hat
        }
        __syncwarp();
        if (lane < n) {
            double t = 0.0;
            for (int j = 0; j < n; ++j)
                if (j != lane) t += A[lane * LD + j] * (sm.v4[j] * sm.v1[j]);
            sm.v2[lane] = sm.v4[lane] * (sm.v1[lane] - t);  // t2 = h(S) t1
        }
        __syncwarp();
        if (lane < n) {
            // g(S), column `lane`, over S (each lane reads and writes only its column).
            const double ui = sm.v3[lane];
            const double ai = sm.v5[lane];
            const double ir = 1.0 / rr;
            for (int j = 0; j < n; ++j) {
                const double uj = sm.v3[j];
                A[j * LD + lane] = (j == lane) ? -ai * ir
                                               : A[j * LD + lane] * (ui + uj + rr) * ai * sm.v5[j] * ir / (ui + uj);
            }
            double t = 0.0;
            for (int l = 0; l < n; ++l) t += U[lane * LD + l] * sm.v2[l];
            sm.v1[lane] = t;  // v = U t2 = (a I + A)^{-1} d-hat
            // Z = dX Yh^T, column `lane`.
            const double* row = o.dY + (size_t)sm.lidx[lane] * k;
            double acc[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] = 0.0;
            for (int m = 0; m < k; ++m) {
                const double dy = row[m];
#pragma unroll
                for (int a = 0; a < 9; ++a) acc[a] += sm.dX[a * k + m] * dy;
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) sm.Z[a * NMAX + lane] = sm.lsq[lane] * acc[a];
        }
        __syncwarp();
        // zv = Z v (= dX w-bar); B = Z U.
        if (lane < 9) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += sm.Z[lane * NMAX + i] * sm.v1[i];
            sm.zv[lane] = s;
        }
        if (lane < n)
            for (int a = 0; a < 9; ++a) {
                double s = 0.0;
                for (int l = 0; l < n; ++l) s += sm.Z[a * NMAX + l] * U[l * LD + lane];
                sm.B[a * NMAX + lane] = s;
            }
        __syncwarp();
        // Z <- (Z U) g(S).
        if (lane < n)
            for (int a = 0; a < 9; ++a) {
                double s = 0.0;
                for (int j = 0; j < n; ++j) s += sm.B[a * NMAX + j] * A[j * LD + lane];
                sm.Z[a * NMAX + lane] = s;
            }
        __syncwarp();
        // B <- sqrt(k-1) Z U^T diag(sqrt(rho)), ready to meet dY.
        const double sk = sqrt((double)(k - 1));
        if (lane < n)
            for (int a = 0; a < 9; ++a) {
                double s = 0.0;
                for (int l = 0; l < n; ++l) s += sm.Z[a * NMAX + l] * U[lane * LD + l];
                sm.B[a * NMAX + lane] = sk * sm.lsq[lane] * s;
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
                for (int a = 0; a < 9; ++a) acc[a] += sm.B[a * NMAX + i] * dy;
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) fc[a * plane + m] = (T)acc[a];
        }
    } else {
        // lam = diag; w-bar = U diag(1/lam) U^T b; T = W + w-bar 1^T with
        // W = sqrt(k-1) U diag(lam^{-1/2}) U^T, stored over A.
        if (lane < n) {
            const double lam = A[lane * LD + lane];
            double t = 0.0;
            for (int l = 0; l < n; ++l) t += U[l * LD + lane] * sm.v3[l];
            sm.v1[lane] = t / lam;
            sm.v2[lane] = sqrt((double)(k - 1) / lam);
        }
        __syncwarp();
        if (lane < n) {
            double t = 0.0;
            for (int l = 0; l < n; ++l) t += U[lane * LD + l] * sm.v1[l];
            sm.v3[lane] = t;  // w-bar
        }
        __syncwarp();
        if (lane < n)
            for (int i = 0; i < n; ++i) {
                double s = 0.0;
                for (int l = 0; l < n; ++l) s += U[i * LD + l] * sm.v2[l] * U[lane * LD + l];
                A[i * LD + lane] = s + sm.v3[i];
            }
        __syncwarp();
        if (lane < k) {
            const int m = lane;
            for (int a = 0; a < 9; ++a) {
                double s = 0.0;
                for (int j = 0; j < k; ++j) s += sm.dX[a * k + j] * A[j * LD + m];
                fc[a * plane + m] = (T)(sm.xbar[a] + s);
            }
        }
    }
}

// ------------------------------------------------------------------ K3, mixed precision
// The state is binary32 (g = f - w). The eigensolve is FP64-accurate at a
// fraction of the FP64 work, in two kernels over chunks of grid points:
//  (A) mixed_jacobi_kernel: the local set, the matrix in FP64 rounded to
//      binary32, and a binary32 cyclic Jacobi held in registers (no shared
//      memory, so many warps per SM hide its latency). The basis X goes to a
//      chunk-sized scratch that stays in L2.
//  (B) analyze_mixed_kernel: in FP64, re-orthonormalise X (Cholesky QR,
//      Y = X L^{-T} with X^T X = L L^T), form the Rayleigh-Ritz matrix
//      S = Y^T A Y, and evaluate f(A) = Y f(S) Y^T to first order in the
//      off-diagonal of S (Daleckii-Krein: f(S)_ii = f(s_ii),
//      f(S)_ij = s_ij f[s_ii, s_jj], divided differences in closed form).
//      The error is second order in the off-diagonal of S (relative ~1e-13
//      at these sizes). The transform products and the update run in
//      binary32 with binary32 accumulation.

constexpr int kChunkCells = 8192;   // grid points per (A)+(B) pass
constexpr int kJacWarps = 4;        // points per block in (A)
constexpr size_t kXStride = (size_t)NMAX * NMAX;  // floats of X per point

// Local observation set of grid point (x, y), in increasing point order:
// point j is in range when r / d_cut < 2 and G(r / d_cut) > 0; it gives the
// two scalars 2j (u) and 2j+1 (v) with sqrt(rho) = sqrt(G) / sigma.
// Returns the number of scalars p. Warp-cooperative.
__device__ int local_set(const ObsParams& o, int x, int y, int nx, int ny, double d_cut, int lane,
                         int* lidx, double* lsq) {
    int count = 0;
    for (int j0 = 0; j0 < o.npts; j0 += 32) {
        const int j = j0 + lane;
        bool in = false;
        double g = 0.0;
        if (j < o.npts) {
            const int dx = min_image(o.ix[j] - x, nx);
            const int dy = min_image(o.iy[j] - y, ny);
            const double r = sqrt((double)dx * dx + (double)dy * dy);
            const double dist = r / d_cut;
            if (dist < 2.0) {
                g = gaspari_cohn(dist);
                in = g > 0.0;
            }
        }
        const unsigned bal = __ballot_sync(kFull, in);
        if (in) {
            const int pos = count + __popc(bal & ((1u << lane) - 1u));
            const double sg = sqrt(g);
            lidx[2 * pos] = 2 * j;
            lidx[2 * pos + 1] = 2 * j + 1;
            lsq[2 * pos] = sg / o.sigma_u;
            lsq[2 * pos + 1] = sg / o.sigma_v;
        }
        count += __popc(bal);
    }
    __syncwarp();
    return 2 * count;
}

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
__device__ bool jacobi32_reg(float (&a)[NS], float (&u)[NS], int lane, float rel, int max_sweeps) {
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
                const float tau = (dp - dg) / (2.0f * off);
                t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
                c = 1.0f / sqrtf(1.0f + t * t);
                s = t * c;
                rot = true;
            }
            if (__ballot_sync(kFull, rot) != 0u) {
                any_sweep = true;
                // Row rotations: position t (row p) with position NS-1-t (row q).
#pragma unroll
                for (int tt = 0; tt < NS / 2; ++tt) {
                    const int pl = (tt == 0) ? 0 : 1 + ((tt - 1 + r) % m1);
                    const float ct = __shfl_sync(kFull, c, pl);
                    const float st = __shfl_sync(kFull, s, pl);
                    const float x0 = a[tt], x1 = a[NS - 1 - tt];
                    a[tt] = ct * x0 - st * x1;
                    a[NS - 1 - tt] = st * x0 + ct * x1;
                }
                // Column rotations with the partner lane; the diagonal moves
                // by -/+ t a_pq on the p/q side.
                const int pl_mine = pside ? lane : partner;
                const float cm = __shfl_sync(kFull, c, pl_mine & 31);
                const float sm_ = __shfl_sync(kFull, s, pl_mine & 31);
                const float tm = __shfl_sync(kFull, t, pl_mine & 31);
                const float om = __shfl_sync(kFull, off, pl_mine & 31);
                dg = pside ? dg - tm * om : dg + tm * om;
                const float sg = pside ? -sm_ : sm_;
#pragma unroll
                for (int i = 0; i < NS; ++i) {
                    const float th = __shfl_sync(kFull, a[i], partner & 31);
                    a[i] = cm * a[i] + sg * th;
                    const float tu = __shfl_sync(kFull, u[i], partner & 31);
                    u[i] = cm * u[i] + sg * tu;
                }
                // The rotated off-diagonal entry is zero by construction.
                if (sm_ != 0.0f) {
#pragma unroll
                    for (int i = 0; i < NS; ++i)
                        if (i == qp) a[i] = 0.0f;
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
        if (!any_sweep) return true;
    }
    return false;
}

// One point of kernel (A): build column `lane` of the matrix (FP64, rounded
// to binary32), run the Jacobi, store X = U (row i of X at Xp + i * NMAX).
template <int NS>
__device__ void jacobi_point(const ObsParams& o, int k, int n, int p, bool obs_space, double aa,
                             const int* lidx, const double* lsq, int lane, float* __restrict__ Xp,
                             int* flags) {
    const int nobs = 2 * o.npts;
    float a[NS], u[NS];
    if (obs_space) {
        const bool own = lane < n;
        const int ol = own ? lidx[lane] : 0;
        const double sl = own ? lsq[lane] : 0.0;
#pragma unroll
        for (int i = 0; i < NS; ++i)
            a[i] = (own && i < n) ? (float)(lsq[i] * o.G[(size_t)lidx[i] * nobs + ol] * sl) : 0.0f;
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
    if (!jacobi32_reg<NS>(a, u, lane, 3e-8f, kMaxSweeps)) {
        if (lane == 0) atomicOr(flags, FLAG_NOCONV);
    }
    if (lane < n) {
#pragma unroll
        for (int i = 0; i < NS; ++i)
            if (i < n) Xp[(size_t)i * NMAX + lane] = u[i];
    }
}

// Per-chunk scratch shared by kernels (A) and (B).
struct MixScratch {
    float* X;      // [chunk][NMAX][NMAX] binary32 basis, row i at i * NMAX
    double* lsq;   // [chunk][nobs] sqrt(rho) of the local scalars
    int* lidx;     // [chunk][nobs] their observation indices
    int* pcount;   // [chunk] number of local scalars
};

__host__ __device__ inline size_t mix_scratch_bytes_per_point(int nobs) {
    return kXStride * sizeof(float) + (size_t)nobs * (sizeof(double) + sizeof(int)) + sizeof(int);
}

__host__ __device__ inline MixScratch mix_scratch_at(void* base, int chunk, int nobs) {
    MixScratch m;
    unsigned char* p = reinterpret_cast<unsigned char*>(base);
    m.X = reinterpret_cast<float*>(p);
    p += (size_t)chunk * kXStride * sizeof(float);
    m.lsq = reinterpret_cast<double*>(p);
    p += (size_t)chunk * nobs * sizeof(double);
    m.lidx = reinterpret_cast<int*>(p);
    p += (size_t)chunk * nobs * sizeof(int);
    m.pcount = reinterpret_cast<int*>(p);
    return m;
}

__global__ void __launch_bounds__(32 * kJacWarps) mixed_jacobi_kernel(int nx, int ny, int k,
                                                                      ObsParams o, double d_cut,
                                                                      double beta, int cell0,
                                                                      int ncell, MixScratch sc,
                                                                      int* __restrict__ flags) {
    const int nobs = 2 * o.npts;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int li = blockIdx.x * kJacWarps + w;
    if (li >= ncell) return;
    const int cell = cell0 + li;
    const int x = cell % nx, y = cell / nx;
    double* lsq = sc.lsq + (size_t)li * nobs;
    int* lidx = sc.lidx + (size_t)li * nobs;
    const int p = local_set(o, x, y, nx, ny, d_cut, lane, lidx, lsq);
    if (lane == 0) sc.pcount[li] = p;
    if (p == 0) return;
    const bool obs_space = p < k;
    const int n = obs_space ? p : k;
    if (n > NMAX) return;  // reported by kernel (B)
    const double aa = (k - 1) / beta;
    float* Xp = sc.X + (size_t)li * kXStride;
    if (n <= 8)
        jacobi_point<8>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, flags);
    else if (n <= 16)
        jacobi_point<16>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, flags);
    else if (n <= 24)
        jacobi_point<24>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, flags);
    else if (n <= 26)
        jacobi_point<26>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, flags);
    else if (n <= 28)
        jacobi_point<28>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, flags);
    else
        jacobi_point<32>(o, k, n, p, obs_space, aa, lidx, lsq, lane, Xp, flags);
}

// Shared memory of kernel (B). The matrices are nm x ld with nm the largest
// local problem of this launch and ld = nm + 1 rounded to odd.
struct MixSmem {
    double* A;     // [nm][ld] matrix (FP64), then S = Y^T A Y
    double* Y;     // [nm][ld] FP64 basis
    double* W;     // [nm][ld] Y^T Y, its Cholesky factor, then A Y
    float* F32;    // [nm][ld] f(S) in binary32, then T (inside W)
    float* Y32;    // [nm][ld] Y in binary32
    double* lsq;   // [nl]
    double* ldh;   // [nl]
    double* vb;    // [NMAX]
    double* v1;    // [NMAX]
    double* vu;    // [NMAX]
    double* vinv;  // [NMAX]
    float* dX;     // [9][k]
    float* xbar;   // [16]
    float* Z;      // [9][NMAX]
    float* B;      // [9][NMAX]
    float* zv;     // [16]
    float* vf;     // [NMAX]
    float* t1f;    // [NMAX]
    float* t2f;    // [NMAX]
    int* lidx;     // [nl]
};

__host__ __device__ inline int mix_ld(int nm) { return (nm % 2 == 0) ? nm + 1 : nm; }

__host__ __device__ inline size_t mix_smem_bytes(int k, int nl, int nm) {
    const int ld = mix_ld(nm);
    const size_t d = 3 * (size_t)nm * ld + 2 * (size_t)nl + 4 * NMAX;
    const size_t f = (size_t)nm * ld + 9 * (size_t)k + 16 + 18 * NMAX + 16 + 3 * NMAX;
    return d * sizeof(double) + ((f * sizeof(float) + 7) / 8) * 8 + (size_t)nl * sizeof(int);
}

__device__ inline MixSmem carve_mix(unsigned char* raw, int k, int nl, int nm) {
    const int ld = mix_ld(nm);
    MixSmem s;
    double* p = reinterpret_cast<double*>(raw);
    s.A = p;
    p += nm * ld;
    s.Y = p;
    p += nm * ld;
    s.W = p;
    s.F32 = reinterpret_cast<float*>(p);
    p += nm * ld;
    s.lsq = p;
    p += nl;
    s.ldh = p;
    p += nl;
    s.vb = p;
    p += NMAX;
    s.v1 = p;
    p += NMAX;
    s.vu = p;
    p += NMAX;
    s.vinv = p;
    p += NMAX;
    float* q = reinterpret_cast<float*>(p);
    s.Y32 = q;
    q += nm * ld;
    s.dX = q;
    q += 9 * k;
    s.xbar = q;
    q += 16;
    s.Z = q;
    q += 9 * NMAX;
    s.B = q;
    q += 9 * NMAX;
    s.zv = q;
    q += 16;
    s.vf = q;
    q += NMAX;
    s.t1f = q;
    q += NMAX;
    s.t2f = q;
    q += NMAX;
    const size_t fbytes = (size_t)(q - reinterpret_cast<float*>(p)) * sizeof(float);
    s.lidx = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(p) + ((fbytes + 7) / 8) * 8);
    return s;
}

// Symmetric product C = P^T Q for P = Q (or P^T Q known to be symmetric):
// only the n(n+1)/2 entries i <= j are formed, spread over the lanes two at
// a time, and mirrored. P, Q, C are [n][ld] row-major in shared memory.
__device__ void sym_product(const double* P, const double* Q, double* C, int n, int ld, int lane) {
    const int ne = n * (n + 1) / 2;
    for (int e0 = lane; e0 < ne; e0 += 64) {
        const int e1 = e0 + 32;
        // Entry e -> (i, j), i <= j, row-major over the upper triangle.
        int i0 = 0, j0 = e0;
        while (j0 >= n - i0) { j0 -= n - i0; ++i0; }
        j0 += i0;
        const bool has1 = e1 < ne;
        int i1 = 0, j1 = has1 ? e1 : 0;
        if (has1) {
            while (j1 >= n - i1) { j1 -= n - i1; ++i1; }
            j1 += i1;
        }
        double s0 = 0.0, s1 = 0.0;
        for (int r = 0; r < n; ++r) {
            s0 += P[r * ld + i0] * Q[r * ld + j0];
            s1 += P[r * ld + i1] * Q[r * ld + j1];
        }
        C[i0 * ld + j0] = s0;
        C[j0 * ld + i0] = s0;
        if (has1) {
            C[i1 * ld + j1] = s1;
            C[j1 * ld + i1] = s1;
        }
    }
}

// FP64 refinement of the basis already in Y (columns = approximate
// eigenvectors of the symmetric matrix A): Y <- Y L^{-T} with Y^T Y = L L^T,
// then A <- S = Y^T A Y.
__device__ void refine_basis(double* A, double* Y, double* W, double* vinv, int n, int ld,
                             int lane) {
    sym_product(Y, Y, W, n, ld, lane);  // W = Y^T Y
    __syncwarp();
    // Cholesky factor of Y^T Y (close to I), lower triangle of W. Every lane
    // forms its row's candidate for column j in the same loop, so the warp
    // does not diverge; the diagonal comes from lane j by a shuffle.
    for (int j = 0; j < n; ++j) {
        double s0 = (lane < n) ? W[lane * ld + j] : 1.0, s1 = 0.0;
        if (lane < n) {
            int c = 0;
            for (; c + 1 < j; c += 2) {
                s0 -= W[lane * ld + c] * W[j * ld + c];
                s1 -= W[lane * ld + c + 1] * W[j * ld + c + 1];
            }
            if (c < j) s0 -= W[lane * ld + c] * W[j * ld + c];
        }
        const double s = s0 + s1;
        const double dj = __shfl_sync(kFull, s, j);
        // The basis is orthonormal to ~1e-5, so the pivot is 1 + e with tiny
        // e: the binomial series 1/sqrt(1+e) = 1 - e/2 + 3e^2/8 - 5e^3/16
        // truncates below 3e-17 for |e| < 1e-4; other pivots take rsqrt.
        const double ej = dj - 1.0;
        const double inv = (fabs(ej) < 1e-4) ? 1.0 + ej * (-0.5 + ej * (0.375 - 0.3125 * ej))
                                             : rsqrt(dj);
        __syncwarp();
        if (lane == j) {
            W[j * ld + j] = dj * inv;
            vinv[j] = inv;
        } else if (lane > j && lane < n) {
            W[lane * ld + j] = s * inv;
        }
        __syncwarp();
    }
    // Y <- Y L^{-T}, row `lane` by forward substitution.
    if (lane < n)
        for (int j = 0; j < n; ++j) {
            double z0 = Y[lane * ld + j], z1 = 0.0;
            int c = 0;
            for (; c + 1 < j; c += 2) {
                z0 -= Y[lane * ld + c] * W[j * ld + c];
                z1 -= Y[lane * ld + c + 1] * W[j * ld + c + 1];
            }
            if (c < j) z0 -= Y[lane * ld + c] * W[j * ld + c];
            Y[lane * ld + j] = (z0 + z1) * vinv[j];
        }
    __syncwarp();
    // W = A Y, column `lane`: four rows at a time, then the remainder.
    if (lane < n) {
        int i0 = 0;
        for (; i0 + 3 < n; i0 += 4) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            for (int c = 0; c < n; ++c) {
                const double yc = Y[c * ld + lane];
                s0 += A[i0 * ld + c] * yc;
                s1 += A[(i0 + 1) * ld + c] * yc;
                s2 += A[(i0 + 2) * ld + c] * yc;
                s3 += A[(i0 + 3) * ld + c] * yc;
            }
            W[i0 * ld + lane] = s0;
            W[(i0 + 1) * ld + lane] = s1;
            W[(i0 + 2) * ld + lane] = s2;
            W[(i0 + 3) * ld + lane] = s3;
        }
        for (; i0 < n; ++i0) {
            double s0 = 0.0;
            for (int c = 0; c < n; ++c) s0 += A[i0 * ld + c] * Y[c * ld + lane];
            W[i0 * ld + lane] = s0;
        }
    }
    __syncwarp();
    sym_product(Y, W, A, n, ld, lane);  // A <- S = Y^T (A Y), symmetric
    __syncwarp();
}

__global__ void __launch_bounds__(32) analyze_mixed_kernel(float* __restrict__ f, int nx, int ny,
                                                           int k, ObsParams o, double d_cut,
                                                           double beta, int cell0, int nm,
                                                           MixScratch sc,
                                                           int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nobs = 2 * o.npts;
    MixSmem sm = carve_mix(smem_raw, k, nobs, nm);
    const int ld = mix_ld(nm);
    const int lane = threadIdx.x;
    const int li = blockIdx.x;
    const int cell = cell0 + li;
    const size_t plane = (size_t)nx * ny * k;
    float* fc = f + (size_t)cell * k;

    // Ensemble mean and perturbations in binary32.
    for (int a = 0; a < 9; ++a) {
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
    for (int i = lane; i < p; i += 32) {
        const int oi = sc.lidx[(size_t)li * nobs + i];
        const double si = sc.lsq[(size_t)li * nobs + i];
        sm.lidx[i] = oi;
        sm.lsq[i] = si;
        sm.ldh[i] = si * o.d[oi];
    }
    __syncwarp();

    if (p == 0) {
        const float sb = (float)sqrt(beta);
        for (int a = 0; a < 9; ++a)
            for (int m = lane; m < k; m += 32) fc[a * plane + m] = sm.xbar[a] + sb * sm.dX[a * k + m];
        return;
    }
    const bool obs_space = p < k;
    const int n = obs_space ? p : k;
    if (n > nm) {
        if (lane == 0) atomicOr(flags, FLAG_TOOLARGE);
        return;
    }
    const double aa = (k - 1) / beta;
    double* A = sm.A;
    double* Y = sm.Y;

    // The symmetric matrix in FP64: A = Yh Yh^T (observation space) or
    // C = a I + Yh^T Yh with b = Yh^T d-hat (ensemble space); the basis X
    // from kernel (A).
    const float* Xp = sc.X + (size_t)li * kXStride;
    if (lane < n) {
        if (obs_space) {
            const int ol = sm.lidx[lane];
            const double sl = sm.lsq[lane];
            for (int i = 0; i < n; ++i)
                A[i * ld + lane] = sm.lsq[i] * o.G[(size_t)sm.lidx[i] * nobs + ol] * sl;
        } else {
            double bj = 0.0;
            for (int i = 0; i < n; ++i) {
                double s = 0.0;
                for (int l = 0; l < p; ++l) {
                    const double* row = o.dY + (size_t)sm.lidx[l] * k;
                    s += sm.lsq[l] * sm.lsq[l] * row[i] * row[lane];
                }
                A[i * ld + lane] = s + (i == lane ? aa : 0.0);
            }
            for (int l = 0; l < p; ++l) bj += sm.lsq[l] * o.dY[(size_t)sm.lidx[l] * k + lane] * sm.ldh[l];
            sm.vb[lane] = bj;
        }
        for (int i = 0; i < n; ++i) Y[i * ld + lane] = (double)Xp[(size_t)i * NMAX + lane];
    }
    __syncwarp();
    refine_basis(A, Y, sm.W, sm.vinv, n, ld, lane);
    // Y in binary32 for the transform products.
    if (lane < n)
        for (int c = 0; c < n; ++c) sm.Y32[lane * ld + c] = (float)Y[lane * ld + c];
    __syncwarp();
    float* Y32 = sm.Y32;
    float* F32 = sm.F32;
    const float sk = (float)sqrt((double)(k - 1));

    if (obs_space) {
        // Functions of a + S: h = 1/(a+s) for the weights, g(s) = q[s, 0] with
        // q(s) = (a+s)^{-1/2} for the square root. u_i = sqrt(a + s_ii).
        const double r = sqrt(aa);
        if (lane < n) {
            const double sii = A[lane * ld + lane];
            const double u = sqrt(aa + sii);
            sm.vu[lane] = u;
            sm.vinv[lane] = 1.0 / (u * (u + r));  // alpha_i
            sm.vb[lane] = 1.0 / (aa + sii);       // h_i = 1 / u_i^2
            // t1 = Y^T d-hat (binary32 transform product).
            float t = 0.0f;
            for (int c = 0; c < n; ++c) t += Y32[c * ld + lane] * (float)sm.ldh[c];
            sm.t1f[lane] = t;
        }
        __syncwarp();
        if (lane < n) {
            // t2 = h(S) t1 with h(S)_ii = h_i, h(S)_ij = -s_ij h_i h_j.
            const float hi = (float)sm.vb[lane];
            float t = 0.0f;
            for (int j = 0; j < n; ++j)
                if (j != lane) t += (float)A[lane * ld + j] * ((float)sm.vb[j] * sm.t1f[j]);
            sm.t2f[lane] = hi * (sm.t1f[lane] - t);
            // g(S) in binary32: diagonal -alpha_i / r, off-diagonal
            // s_ij (u_i + u_j + r) alpha_i alpha_j / (r (u_i + u_j)).
            const float ai = (float)sm.vinv[lane];
            const float ui = (float)sm.vu[lane];
            const float rf = (float)r;
            for (int i = 0; i < n; ++i) {
                float v;
                if (i == lane) {
                    v = (float)(-sm.vinv[lane] / r);
                } else {
                    const float uj = (float)sm.vu[i];
                    const float aj = (float)sm.vinv[i];
                    v = (float)A[i * ld + lane] * (ui + uj + rf) * ai * aj / (rf * (ui + uj));
                }
                F32[i * ld + lane] = v;
            }
        }
        __syncwarp();
        if (lane < n) {
            float t = 0.0f;
            for (int c = 0; c < n; ++c) t += Y32[lane * ld + c] * sm.t2f[c];
            sm.vf[lane] = t;  // v = (a I + A)^{-1} d-hat
            // Z = dX Yh^T, column `lane`: nine accumulators over members.
            const float* row = o.dY32 + (size_t)sm.lidx[lane] * k;
            float acc[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] = 0.0f;
            for (int m = 0; m < k; ++m) {
                const float dy = row[m];
#pragma unroll
                for (int a = 0; a < 9; ++a) acc[a] += sm.dX[a * k + m] * dy;
            }
            const float sl = (float)sm.lsq[lane];
#pragma unroll
            for (int a = 0; a < 9; ++a) sm.Z[a * NMAX + lane] = sl * acc[a];
        }
        __syncwarp();
        if (lane < 9) {
            float s = 0.0f;
            for (int i = 0; i < n; ++i) s += sm.Z[lane * NMAX + i] * sm.vf[i];
            sm.zv[lane] = s;
        }
        if (lane < n) {
            float acc[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] = 0.0f;
            for (int c = 0; c < n; ++c) {
                const float yc = Y32[c * ld + lane];
#pragma unroll
                for (int a = 0; a < 9; ++a) acc[a] += sm.Z[a * NMAX + c] * yc;
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) sm.B[a * NMAX + lane] = acc[a];  // Z Y
        }
        __syncwarp();
        if (lane < n) {
            float acc[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] = 0.0f;
            for (int j = 0; j < n; ++j) {
                const float fj = F32[j * ld + lane];
#pragma unroll
                for (int a = 0; a < 9; ++a) acc[a] += sm.B[a * NMAX + j] * fj;
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) sm.Z[a * NMAX + lane] = acc[a];  // Z Y g(S)
        }
        __syncwarp();
        if (lane < n) {
            float acc[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] = 0.0f;
            for (int i = 0; i < n; ++i) {
                const float yi = Y32[lane * ld + i];
#pragma unroll
                for (int a = 0; a < 9; ++a) acc[a] += sm.Z[a * NMAX + i] * yi;
            }
            const float sl = sk * (float)sm.lsq[lane];
#pragma unroll
            for (int a = 0; a < 9; ++a) sm.B[a * NMAX + lane] = sl * acc[a];  // sqrt(k-1) Z g(A) sqrt(rho)
        }
        __syncwarp();
        const float sb = (float)sqrt(beta);
        for (int m = lane; m < k; m += 32) {
            float acc[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] = sm.xbar[a] + sm.zv[a] + sb * sm.dX[a * k + m];
            for (int i = 0; i < n; ++i) {
                const float dy = o.dY32[(size_t)sm.lidx[i] * k + m];
#pragma unroll
                for (int a = 0; a < 9; ++a) acc[a] += sm.B[a * NMAX + i] * dy;
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) fc[a * plane + m] = acc[a];
        }
    } else {
        // Functions of S directly: 1/lambda for P-tilde, lambda^{-1/2} for W.
        if (lane < n) {
            const double lam = A[lane * ld + lane];
            sm.vu[lane] = sqrt(lam);
            sm.vinv[lane] = 1.0 / lam;
            float t = 0.0f;
            for (int c = 0; c < n; ++c) t += Y32[c * ld + lane] * (float)sm.vb[c];
            sm.t1f[lane] = t;  // Y^T b
        }
        __syncwarp();
        if (lane < n) {
            // t2 = f1(S) t1, f1(S)_ii = 1/l_i, f1(S)_ij = -s_ij / (l_i l_j).
            float t = 0.0f;
            for (int j = 0; j < n; ++j)
                if (j != lane) t += (float)A[lane * ld + j] * ((float)sm.vinv[j] * sm.t1f[j]);
            sm.t2f[lane] = (float)sm.vinv[lane] * (sm.t1f[lane] - t);
            // f2(S) = S^{-1/2}: diagonal 1/sqrt(l_i), off-diagonal
            // -s_ij / (sqrt(l_i) sqrt(l_j) (sqrt(l_i) + sqrt(l_j))).
            const float si = (float)sm.vu[lane];
            for (int i = 0; i < n; ++i) {
                float v;
                if (i == lane) {
                    v = (float)(1.0 / sm.vu[lane]);
                } else {
                    const float sj = (float)sm.vu[i];
                    v = -(float)A[i * ld + lane] / (si * sj * (si + sj));
                }
                F32[i * ld + lane] = v;
            }
        }
        __syncwarp();
        float* YF = reinterpret_cast<float*>(A);  // S is no longer needed after w-bar
        if (lane < n) {
            float t = 0.0f;
            for (int c = 0; c < n; ++c) t += Y32[lane * ld + c] * sm.t2f[c];
            sm.vf[lane] = t;  // w-bar
        }
        __syncwarp();
        if (lane < n)
            for (int i = 0; i < n; ++i) {
                float s = 0.0f;
                for (int l = 0; l < n; ++l) s += Y32[i * ld + l] * F32[l * ld + lane];
                YF[i * ld + lane] = s;
            }
        __syncwarp();
        // T = sqrt(k-1) Y f2(S) Y^T + w-bar 1^T, over F32.
        if (lane < n)
            for (int i = 0; i < n; ++i) {
                float s = 0.0f;
                for (int l = 0; l < n; ++l) s += YF[i * ld + l] * Y32[lane * ld + l];
                F32[i * ld + lane] = sk * s + sm.vf[i];
            }
        __syncwarp();
        if (lane < k) {
            const int m = lane;
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

cudaError_t launch_observe(const void* f, int fp32, int nx, int ny, int k, int npts, const int* ix,
                           const int* iy, const double* yo, double* dY, double* d,
                           cudaStream_t s) {
    if (npts <= 0) return cudaSuccess;
    const size_t sh = (2 * (size_t)k + 8) * sizeof(double);
    if (fp32)
        observe_kernel<float, true><<<npts, 128, sh, s>>>((const float*)f, nx, ny, k, ix, iy, yo, dY,
                                                          d);
    else
        observe_kernel<double, false><<<npts, 128, sh, s>>>((const double*)f, nx, ny, k, ix, iy, yo,
                                                            dY, d);
    return cudaGetLastError();
}

cudaError_t launch_obs_gram(const double* dY, int nobs, int k, double* G, cudaStream_t s) {
    if (nobs <= 0) return cudaSuccess;
    dim3 grid((nobs + 127) / 128, nobs);
    obs_gram_kernel<<<grid, 128, 0, s>>>(dY, nobs, k, G);
    return cudaGetLastError();
}

size_t analyze_scratch_bytes(int nx, int ny, int fp32, int npts) {
    if (!fp32) return 0;
    const long long cells = (long long)nx * ny;
    const long long chunk = cells < kChunkCells ? cells : kChunkCells;
    return 2 * (size_t)chunk * mix_scratch_bytes_per_point(2 * npts);  // double-buffered
}

cudaError_t launch_analyze(void* f, int fp32, int nx, int ny, int k, const ObsParams& o,
                           double d_cut, double beta, int nmax, int* flags, void* scratch,
                           const AnalyzeAux* aux, cudaStream_t s) {
    const long long cells = (long long)nx * ny;
    if (cells > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    cudaError_t e;
    if (fp32) {
        if (!o.dY32 || !scratch || !aux) return cudaErrorInvalidValue;
        const int nobs = 2 * o.npts;
        const int nm = nmax < 2 ? 2 : (nmax > NMAX ? NMAX : nmax);
        const size_t nd = (size_t)nobs * k;
        to_f32_kernel<<<(unsigned)((nd + 255) / 256), 256, 0, s>>>(o.dY, o.dY32, nd);
        const size_t shB = mix_smem_bytes(k, nobs, nm);
        e = cudaFuncSetAttribute(analyze_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)shB);
        if (e != cudaSuccess) return e;
        const long long chunk = cells < kChunkCells ? cells : kChunkCells;
        const size_t buf_bytes = (size_t)chunk * mix_scratch_bytes_per_point(nobs);
        // Pipeline: (A) of chunk c on s2 overlaps (B) of chunk c-1 on s; the
        // scratch is double-buffered, (A) of chunk c waits for (B) of c-2.
        if ((e = cudaEventRecord(aux->start, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(aux->s2, aux->start, 0)) != cudaSuccess) return e;
        int c = 0;
        for (long long c0 = 0; c0 < cells; c0 += chunk, ++c) {
            const int nc = (int)((cells - c0) < chunk ? (cells - c0) : chunk);
            const int b = c & 1;
            const MixScratch sc = mix_scratch_at((unsigned char*)scratch + b * buf_bytes, (int)chunk,
                                                 nobs);
            if (c >= 2 && (e = cudaStreamWaitEvent(aux->s2, aux->ref_done[b], 0)) != cudaSuccess)
                return e;
            mixed_jacobi_kernel<<<(unsigned)((nc + kJacWarps - 1) / kJacWarps), 32 * kJacWarps, 0,
                                  aux->s2>>>(nx, ny, k, o, d_cut, beta, (int)c0, nc, sc, flags);
            if ((e = cudaEventRecord(aux->jac_done[b], aux->s2)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, aux->jac_done[b], 0)) != cudaSuccess) return e;
            analyze_mixed_kernel<<<(unsigned)nc, 32, shB, s>>>((float*)f, nx, ny, k, o, d_cut, beta,
                                                               (int)c0, nm, sc, flags);
            if ((e = cudaEventRecord(aux->ref_done[b], s)) != cudaSuccess) return e;
        }
    } else {
        const size_t sh = ana_smem_bytes(k, 2 * o.npts);
        e = cudaFuncSetAttribute(analyze_kernel<double, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e != cudaSuccess) return e;
        analyze_kernel<double, false><<<(unsigned)cells, 32, sh, s>>>((double*)f, nx, ny, k, o,
                                                                      d_cut, beta, flags);
    }
    return cudaGetLastError();
}

}  // namespace lbmgpu
