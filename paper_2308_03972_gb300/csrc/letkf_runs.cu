// Mixed-precision LETKF analysis over runs of neighbouring grid points
// (arXiv 2308.03972, Section 3.2), observation-space form, unions of local
// sets of up to 32 scalars.
//
// A run is R consecutive grid points of one lattice row. Its observation
// scalars are the union of its points' local sets (Section 3.2.2: the
// observations with r / d_cut < 2); at a point, a scalar outside its
// support has weight zero, so the point's matrix A = Yh Yh^T
// (Yh = diag(sqrt(rho)) dY over the union) has a zero row and column there.
// Such a scalar adds nothing to the analysis: its entries of d-hat, of Yh
// and of the transform's right-hand factor diag(sqrt(rho)) are zero. With
// one index set for the whole run, the binary32 Jacobi of every point after
// the first starts from the previous point's basis U: the Gaspari-Cohn
// weights move by a few per cent from one grid point to the next, so
// A' = U^T A U is already nearly diagonal (about 4% off the diagonal at
// 256^2 with 8 x 8 observations) and the Jacobi needs about three sweeps
// instead of six.
//
// Two kernels per chunk of runs:
//  (J) run_jacobi_kernel, one warp per run, binary32: per point the weights
//      (FP64 support test, the same as the other analysis kernels), A from a
//      binary32 copy of the run's block of G = dY dY^T, the warm transform
//      U^T A U, the cyclic Jacobi, a first-order re-orthonormalisation of
//      the basis, U (I - E/2) with E = U^T U - I in binary32; the basis,
//      the Jacobi's eigenvalue estimates and the FP64 weights go to
//      scratch.
//  (F) run_refine_kernel, one warp per point: A again from J's weights, now
//      in double-binary32, and the refinement, first order in the basis'
//      non-orthogonality E = Y^T Y - I and in the off-diagonal of
//      S = Y^T A Y:
//        R = A Y - Y diag(l)   (double-binary32; l: the eigenvalue estimates,
//                               so R is small),
//        E                     (double-binary32),
//        T = Y^T R             (binary32: R is ~1e-6 of A),
//      so that S = (I + E) diag(l) + T exactly, and S' = M^{-1/2} S M^{-1/2}
//      (M = I + E; Y M^{-1/2} is orthonormal) is, to first order in E,
//        S'_ic = T_ic + E_ic (l_c - l_i) / 2   (i != c),
//        S'_cc = l_c + T_cc - E_cc T_cc - E_cc^2 l_c;
//      then the first-order (Daleckii-Krein) matrix functions
//      h(S') = (aI+S')^{-1} and g(S') = ((aI+S')^{-1/2} - a^{-1/2} I) S'^{-1}
//      with the same first-order basis factor (their scalars in binary32,
//      FP64 in the probe variant), the binary32 transform and the in-place
//      update of the nine f.
// A batch of experiments runs kernel J over all runs of a size class in one
// launch, then kernel F per experiment.
// With w-bar = Yh^T (aI+A)^{-1} d-hat and C^{-1/2} = a^{-1/2} I + Yh^T g(A) Yh
// (C = aI + Yh^T Yh, a = (k-1)/beta) the update is
//   x^a_m = xbar + Z v + sqrt(beta) dx_m + sqrt(k-1) Z g(A) yh_m,
//   Z = dX Yh^T, v = (aI+A)^{-1} d-hat.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "lbm_internal.cuh"
#include "letkf_device.cuh"

namespace lbmgpu {
namespace {

constexpr int kRunSweeps = 30;  // sweep cap of one Jacobi

struct RunArgs {
    float* f;           // binary32 state (null for a double-precision context)
    double* f64;        // FP64 state of a double-precision context, else null
    int nx, ny, k, R;
    ObsParams o;
    const float2* G2;   // [nobs][nobs] G = dY dY^T as binary32 (hi, lo)
    double d_cut, beta;
    long long lim2;     // support_lim2(d_cut)
    // Launch constants in binary32, rounded from FP64 on the host: a =
    // (k-1)/beta, sqrt(a), sqrt(beta), sqrt(k-1).
    float a_f, sqrt_a_f, sqrt_beta_f, sqrt_k1_f;
    int* flags;
    int run0, nruns;    // runs of this chunk
    float* Yg;          // [chunk cells][NS][NS] basis Y, row-major (Y_ic: component i of vector c)
    float* lamg;        // [chunk cells][NS] eigenvalue estimates
    double* wg;         // [chunk cells][NS] localisation weights w_c of the union's scalars (kernel J's)
    int* rinfo;         // [chunk runs][1 + 32] union size, then its scalars
    int* fp64_hist;     // sweep histogram of the FP64 Jacobi (double precision), or null
};

__host__ __device__ inline int run_cell_floats(int ns) { return ns * ns + ns; }
constexpr int kInfo = 33;

// ---- cp.async staging of one grid point's ensemble ------------------------
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// The nine rows f[a][cell][0..k) into dX[a][0..k).
__device__ __forceinline__ void stage_point(const RunArgs& ra, float* dX, size_t cell, int lane) {
    const size_t plane = (size_t)ra.nx * ra.ny * ra.k;
    const int k = ra.k;
    if ((k & 3) == 0) {
        const int kq = k >> 2;
        for (int e = lane; e < 9 * kq; e += 32) {
            const int a = e / kq, m4 = e - a * kq;
            cp_async16(dX + a * k + 4 * m4, ra.f + a * plane + cell * k + 4 * m4);
        }
    } else {
        for (int e = lane; e < 9 * k; e += 32) {
            const int a = e / k, m = e - a * k;
            cp_async4(dX + a * k + m, ra.f + a * plane + cell * k + m);
        }
    }
    cp_async_commit();
}

// a[idx] for a runtime idx in [0, NS), NS <= 32: five levels of selects on
// the bits of idx (depth 5 instead of a chain of NS).
template <int NS>
__device__ __forceinline__ float pick_reg(const float (&a)[NS], int idx) {
    static_assert(NS >= 2 && NS <= 32, "pick_reg");
    constexpr int N1 = (NS + 1) / 2, N2 = (N1 + 1) / 2, N3 = (N2 + 1) / 2, N4 = (N3 + 1) / 2;
    const bool b0 = idx & 1, b1 = idx & 2, b2 = idx & 4, b3 = idx & 8, b4 = idx & 16;
    float v1[N1], v2[N2], v3[N3], v4[N4];
#pragma unroll
    for (int i = 0; i < N1; ++i) v1[i] = (2 * i + 1 < NS && b0) ? a[2 * i + 1 < NS ? 2 * i + 1 : 2 * i] : a[2 * i];
#pragma unroll
    for (int i = 0; i < N2; ++i) v2[i] = (2 * i + 1 < N1 && b1) ? v1[2 * i + 1 < N1 ? 2 * i + 1 : 2 * i] : v1[2 * i];
#pragma unroll
    for (int i = 0; i < N3; ++i) v3[i] = (2 * i + 1 < N2 && b2) ? v2[2 * i + 1 < N2 ? 2 * i + 1 : 2 * i] : v2[2 * i];
#pragma unroll
    for (int i = 0; i < N4; ++i) v4[i] = (2 * i + 1 < N3 && b3) ? v3[2 * i + 1 < N3 ? 2 * i + 1 : 2 * i] : v3[2 * i];
    return (N4 > 1 && b4) ? v4[N4 > 1 ? 1 : 0] : v4[0];
}

// Weight sqrt(rho-tilde) of observation point j for scalar q at grid point
// (x, y): the local-set test of the other analysis kernels (FP64, the same
// operations), zero outside the support.
__device__ __forceinline__ double obs_weight(const RunArgs& ra, int j, int q, int x, int y) {
    const ObsParams& o = ra.o;
    const int dx = min_image(o.ix[j] - x, ra.nx);
    const int dy = min_image(o.iy[j] - y, ra.ny);
    if (dist2(dx, dy) > ra.lim2) return 0.0;
    const double d2 = (double)dx * dx + (double)dy * dy;
    const double dist = sqrt(d2) / ra.d_cut;
    if (!(dist < 2.0)) return 0.0;
    const double g = gaspari_cohn(dist);
    if (!(g > 0.0)) return 0.0;
    const double sig = q == 0 ? o.sigma_u : (q == 1 ? o.sigma_v : o.sigma_r);
    return sqrt(g) / sig;
}

// ---- per-run union of the local sets --------------------------------------
// Observation points with r / d_cut < 2 at some cell of [xa, xb) in row y,
// in increasing order, into pts; their scalars into gi. The test is the
// local-set test on the smallest squared distance over the cells (the test
// is monotone in it). Returns the number of scalars; above cap the lists
// are incomplete.
__device__ int run_union(const RunArgs& ra, int* pts, int* gi, int y, int xa, int xb, int cap, int lane) {
    const ObsParams& o = ra.o;
    const long long lim2 = ra.lim2;
    const int maxpts = cap / o.nvar;
    int count = 0;
    for (int j0 = 0; j0 < o.npts; j0 += 32) {
        const int j = j0 + lane;
        bool in = false;
        if (j < o.npts) {
            const int dy = min_image(o.iy[j] - y, ra.ny);
            int dxm = ra.nx;
            for (int x = xa; x < xb; ++x) {
                const int dx = abs(min_image(o.ix[j] - x, ra.nx));
                dxm = dx < dxm ? dx : dxm;
            }
            if (dist2(dxm, dy) <= lim2) in = sqrt((double)dxm * dxm + (double)dy * dy) / ra.d_cut < 2.0;
        }
        const unsigned bal = __ballot_sync(kFull, in);
        if (in) {
            const int pos = count + __popc(bal & ((1u << lane) - 1u));
            if (pos < maxpts) pts[pos] = j;
        }
        count += __popc(bal);
    }
    __syncwarp();
    const int nu = o.nvar * count;
    if (nu <= cap)
        for (int c = lane; c < nu; c += 32) gi[c] = o.nvar * pts[c / o.nvar] + c % o.nvar;
    __syncwarp();
    return nu;
}

// ---- binary32 Jacobi, warm or cold (kernel J) -----------------------------
// Cyclic Jacobi with the round-robin (tournament) ordering on NS players
// (NS even; players >= n are zero padding). Lane L owns column L of A, and
// row L of the accumulated rotations U. The rows of A and the columns of U
// are held in tournament-position order, so every round rotates the fixed
// register pairs (t, NS-1-t) of both: the row rotation of A (J^T A) and the
// column rotation of U (U J) combine the same two positions with the same
// (c, s), which every lane has anyway; only A's column rotation (A J) needs
// the partner lane's column. After a round, rows and columns move one
// position (q -> q-1 for q >= 2, 1 -> NS-1, 0 stays); the player at
// position q in round r is 0 for q = 0, else 1 + (q-1+r) mod (NS-1), and a
// sweep of NS-1 rounds returns every row to its place. The rotated entry is
// not reset to zero: what rounding leaves there is far below the
// threshold. A rotation is skipped when |a_pq| <= thresh, a_pq as held by
// the pair's p side (the lane at the lower position). The solve stops before
// a sweep in which no pair would rotate: pmask (p_side_mask) marks the
// players this lane meets as the p side, so the test reads exactly the
// entries the sweep would test (rounding leaves A slightly asymmetric, so
// the other side's copies do not decide). Returns the number of sweeps
// counting that last one, or -1 at the cap; lam: the lane's diagonal entry,
// tracked analytically.
template <int NS>
__device__ unsigned p_side_mask(int lane) {
    constexpr int m1 = NS - 1;
    unsigned mask = 0u;
    if (lane >= NS) return 0u;
    for (int r = 0; r < m1; ++r) {
        const int q = (lane == 0) ? 0 : 1 + ((lane - 1 - r + 2 * m1) % m1);
        const int qp = m1 - q;
        const int partner = (qp == 0) ? 0 : 1 + ((qp - 1 + r) % m1);
        if (q < NS / 2) mask |= 1u << partner;
    }
    return mask;
}

// Rounds of a sweep are taken in blocks of UB (UB divides NS - 1): within a
// block the rows stay where they are and round b of the block finds
// position t in register reg(t, b) = 1 + (t - 1 + b) mod (NS - 1) (t >= 1),
// so the registers move once per block, by UB positions.
template <int NS>
__host__ __device__ constexpr int jacobi_block() {
    return ((NS - 1) % 3 == 0) ? 3 : 1;
}

template <int NS>
__device__ int jacobi_rows(float (&a)[NS], float (&ur)[NS], int lane, unsigned pmask, float thresh, float& lam,
                           float* rs) {
    // rs: the warp's rotation slots, by pair (the p side's position): (c, s)
    // of pair t at rs[2t], (t, a_pq) at rs[NS + 2t]; 16-byte aligned.
    float2* const CS = reinterpret_cast<float2*>(rs);
    float2* const TO = reinterpret_cast<float2*>(rs + NS);
    constexpr int m1 = NS - 1;
    constexpr int UB = jacobi_block<NS>();
    static_assert(m1 % UB == 0, "block of rounds");
    float dg = pick_reg<NS>(a, lane < NS ? lane : 0);
    if (lane >= NS) dg = 0.0f;
    for (int sweep = 0; sweep < kRunSweeps; ++sweep) {
        float mx = 0.0f;
#pragma unroll
        for (int i = 0; i < NS; ++i) mx = ((pmask >> i) & 1u) ? fmaxf(mx, fabsf(a[i])) : mx;
        if (__all_sync(kFull, !(mx > thresh))) {
            lam = dg;
            return sweep + 1;
        }
        for (int r0 = 0; r0 < m1; r0 += UB) {
#pragma unroll
            for (int b = 0; b < UB; ++b) {
                const int r = r0 + b;
                const int q = (lane == 0) ? 0 : 1 + ((lane - 1 - r + 2 * m1) % m1);
                const int qp = m1 - q;
                const int partner = (qp == 0) ? 0 : 1 + ((qp - 1 + r) % m1);
                const bool pside = q < NS / 2;
                // Register of position qp in this block's frame.
                int rq = qp - 1 + b;
                rq = (qp == 0) ? 0 : 1 + (rq >= m1 ? rq - m1 : rq);
                const float off = pick_reg<NS>(a, rq < NS ? rq : 0);
                const float dp = __shfl_sync(kFull, dg, partner & 31);
                float c = 1.0f, s = 0.0f, t = 0.0f;
                bool rot = false;
                if (pside && lane < NS && fabsf(off) > thresh) {
                    // Angle from the approximate reciprocal and rsqrt (a few
                    // ulp, no special cases): the refinement takes the basis
                    // from here. sqrt(x) = x rsqrt(x) on [1, 1e30]; the clamp
                    // keeps tau^2 finite, where the rotation is negligible.
                    const float tau = __fdividef(dp - dg, 2.0f * off);
                    const float x = fminf(fmaf(tau, tau, 1.0f), 1e30f);
                    const float root = x * rsqrtf(x);
                    t = __fdividef(tau >= 0.0f ? 1.0f : -1.0f, fabsf(tau) + root);
                    c = rsqrtf(fmaf(t, t, 1.0f));
                    s = t * c;
                    rot = true;
                }
                if (__ballot_sync(kFull, rot) != 0u) {
                    // Every pair's rotation goes to its slot (the p side
                    // writes); all lanes read them back by position.
                    __syncwarp();  // the previous round's reads are done
                    if (pside && lane < NS) {
                        CS[q] = make_float2(c, s);
                        TO[q] = make_float2(t, off);
                    }
                    __syncwarp();
#pragma unroll
                    for (int tt = 0; tt < NS / 2; ++tt) {
                        // Pair tt's (c, s): two pairs per 16-byte load.
                        float ct, st;
                        if ((tt & 1) == 0) {
                            const float4 cs2 = reinterpret_cast<const float4*>(CS)[tt >> 1];
                            ct = cs2.x;
                            st = cs2.y;
                        } else {
                            const float4 cs2 = reinterpret_cast<const float4*>(CS)[tt >> 1];
                            ct = cs2.z;
                            st = cs2.w;
                        }
                        const int i0 = (tt == 0) ? 0 : 1 + ((tt - 1 + b) % m1);
                        const int i1 = 1 + ((NS - 2 - tt + b) % m1);
                        const float x0 = a[i0], x1 = a[i1];
                        a[i0] = fmaf(-st, x1, ct * x0);
                        a[i1] = fmaf(st, x0, ct * x1);
                        const float y0 = ur[i0], y1 = ur[i1];
                        ur[i0] = fmaf(-st, y1, ct * y0);
                        ur[i1] = fmaf(st, y0, ct * y1);
                    }
                    // This lane's own pair, from its slot.
                    const int pair = lane < NS ? (pside ? q : qp) : 0;
                    const float2 csm = CS[pair];
                    const float2 tom = TO[pair];
                    const float cm = csm.x, sm_ = csm.y, tm = tom.x, om = tom.y;
                    dg = pside ? dg - tm * om : dg + tm * om;
                    const float sg = pside ? -sm_ : sm_;
#pragma unroll
                    for (int i = 0; i < NS; ++i) {
                        const float th = __shfl_sync(kFull, a[i], partner & 31);
                        a[i] = fmaf(sg, th, cm * a[i]);
                    }
                }
            }
            // Rows move UB positions: position t takes register reg(t, UB).
            float ta[NS], tu[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                const int src = (i == 0) ? 0 : 1 + ((i - 1 + UB) % m1);
                ta[i] = a[src];
                tu[i] = ur[src];
            }
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                a[i] = ta[i];
                ur[i] = tu[i];
            }
        }
    }
    lam = dg;
    return -1;
}

// Shared memory of one warp of kernel J (floats): header pts[32], gi[32]
// (ints), weights w[NS], the run's block of G (GU, binary32), the basis rows
// Us (row i of U), a scratch matrix Vs and the Jacobi's rotation slots.
template <int NS>
struct JLayout {
    static constexpr int w = 64, GU = w + NS, Us = GU + NS * NS, Vs = Us + NS * NS;
    static constexpr int rs = Vs + NS * NS;  // rotation slots (2 NS floats)
    static constexpr int total = rs + 2 * NS;
    static_assert(rs % 4 == 0, "16-byte aligned rotation slots");
};

template <int NS>
__device__ __forceinline__ void run_jacobi_body(const RunArgs& ra, int blk) {
    extern __shared__ __align__(16) float smj[];
    using L = JLayout<NS>;
    int* const pts = reinterpret_cast<int*>(smj);
    int* const gi = pts + 32;
    float* const wv = smj + L::w;
    float* const GU = smj + L::GU;
    float* const Us = smj + L::Us;
    float* const Vs = smj + L::Vs;
    const int lane = threadIdx.x;
    const int rl = blk;  // run within the chunk
    const int run = ra.run0 + rl;
    const int runs_x = (ra.nx + ra.R - 1) / ra.R;
    const int y = run / runs_x;
    const int xa = (run - y * runs_x) * ra.R;
    const int xb = xa + ra.R < ra.nx ? xa + ra.R : ra.nx;
    const ObsParams& o = ra.o;
    const int nobs = o.nvar * o.npts;
    int* info = ra.rinfo + (size_t)rl * kInfo;
    const int nu = run_union(ra, pts, gi, y, xa, xb, NS, lane);
    if (nu > NS) {  // the host sizes NS for the largest union; not reached
        if (lane == 0) {
            atomicOr(ra.flags, FLAG_TOOLARGE);
            info[0] = -1;
        }
        return;
    }
    if (lane == 0) info[0] = nu;
    if (lane < nu) info[1 + lane] = gi[lane];
    const bool own = lane < NS, real = lane < nu;
    const int c = lane;
    const int gic = real ? gi[c] : 0;
    const int jc = real ? pts[c / o.nvar] : 0;
    const int qc = real ? c % o.nvar : 0;
    // The run's block of G, binary32 (column c by lane c).
    {
        float gcol[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) gcol[i] = (real && i < nu) ? ra.G2[(size_t)gi[i] * nobs + gic].x : 0.0f;
        if (own) {
#pragma unroll
            for (int i = 0; i < NS; ++i) GU[i * NS + c] = gcol[i];
        }
    }
    float ur[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) ur[i] = (i == c) ? 1.0f : 0.0f;
    const unsigned pmask = p_side_mask<NS>(lane);
    bool warm = false;
    for (int x = xa; x < xb; ++x) {
        const size_t lc = (size_t)(rl * ra.R + (x - xa));  // cell within the chunk
        const double w = real ? obs_weight(ra, jc, qc, x, y) : 0.0;
        const float wf = (float)w;
        const bool any = __ballot_sync(kFull, w > 0.0) != 0u;
        if (any && own) ra.wg[lc * NS + c] = w;  // for kernel F
        if (!any) {
            // No observation in range: nothing to solve (kernel F inflates).
            if (lane == 0) ra.lamg[lc * NS] = -1.0f;  // marker read by kernel F
            continue;
        }
        __syncwarp();  // the previous point is done with wv and Vs
        if (own) wv[c] = wf;
        __syncwarp();
        // Column c of A = w_i G_ic w_c (binary32).
        float a[NS];
#pragma unroll
        for (int i4 = 0; i4 < NS / 4; ++i4) {
            const float4 w4 = reinterpret_cast<const float4*>(wv)[i4];
            const float wi[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int r = 0; r < 4; ++r) a[4 * i4 + r] = own ? wi[r] * GU[(4 * i4 + r) * NS + c] * wf : 0.0f;
        }
        if (warm) {
            // V = A U (row c of V: sum_j A_cj U_j.), then X = U^T V (row c of
            // X: sum_i U_ic V_i.); X is symmetric, so row c is column c. G's
            // block is symmetric, so A_cj = w_c GU_cj w_j.
            float acc[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) acc[i] = 0.0f;
            for (int j = 0; j < NS; ++j) {
                const float acj = own ? wv[j] * GU[c * NS + j] * wf : 0.0f;
                const float4* u4 = reinterpret_cast<const float4*>(Us + j * NS);
#pragma unroll
                for (int i4 = 0; i4 < NS / 4; ++i4) {
                    const float4 uv = u4[i4];
                    acc[4 * i4] = fmaf(acj, uv.x, acc[4 * i4]);
                    acc[4 * i4 + 1] = fmaf(acj, uv.y, acc[4 * i4 + 1]);
                    acc[4 * i4 + 2] = fmaf(acj, uv.z, acc[4 * i4 + 2]);
                    acc[4 * i4 + 3] = fmaf(acj, uv.w, acc[4 * i4 + 3]);
                }
            }
            if (own) {
#pragma unroll
                for (int i4 = 0; i4 < NS / 4; ++i4)
                    reinterpret_cast<float4*>(Vs + c * NS)[i4] =
                        make_float4(acc[4 * i4], acc[4 * i4 + 1], acc[4 * i4 + 2], acc[4 * i4 + 3]);
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < NS; ++i) acc[i] = 0.0f;
            for (int i = 0; i < NS; ++i) {
                const float uic = own ? Us[i * NS + c] : 0.0f;
                const float4* v4 = reinterpret_cast<const float4*>(Vs + i * NS);
#pragma unroll
                for (int j4 = 0; j4 < NS / 4; ++j4) {
                    const float4 vv = v4[j4];
                    acc[4 * j4] = fmaf(uic, vv.x, acc[4 * j4]);
                    acc[4 * j4 + 1] = fmaf(uic, vv.y, acc[4 * j4 + 1]);
                    acc[4 * j4 + 2] = fmaf(uic, vv.z, acc[4 * j4 + 2]);
                    acc[4 * j4 + 3] = fmaf(uic, vv.w, acc[4 * j4 + 3]);
                }
            }
#pragma unroll
            for (int i = 0; i < NS; ++i) a[i] = acc[i];
            // The carried basis rows back from shared memory.
            if (own) {
#pragma unroll
                for (int i4 = 0; i4 < NS / 4; ++i4) {
                    const float4 u4 = reinterpret_cast<const float4*>(Us + c * NS)[i4];
                    ur[4 * i4] = u4.x;
                    ur[4 * i4 + 1] = u4.y;
                    ur[4 * i4 + 2] = u4.z;
                    ur[4 * i4 + 3] = u4.w;
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < NS; ++i) ur[i] = (i == c) ? 1.0f : 0.0f;
        }
        float fro = 0.0f;
#pragma unroll
        for (int i = 0; i < NS; ++i) fro = fmaf(a[i], a[i], fro);
        fro = warp_sum(fro);
        float lamc = 0.0f;
        // Stop at 1e-6 ||A||_F: the refinement is second order in the rest.
        const int sweeps = jacobi_rows<NS>(a, ur, lane, pmask, 1e-6f * sqrtf(fro), lamc, smj + L::rs);
        if (sweeps < 0 && lane == 0) atomicOr(ra.flags, FLAG_NOCONV);
        if (o.sweep_hist && lane == 0) atomicAdd(&o.sweep_hist[(sweeps < 0 || sweeps > 31) ? 31 : sweeps], 1);
        // Re-orthonormalise to first order: E = U^T U - I (binary32 is
        // enough here: the refinement recomputes E exactly for the basis it
        // receives), U <- U (I - E/2).
        __syncwarp();
        if (own) {
#pragma unroll
            for (int i4 = 0; i4 < NS / 4; ++i4)
                reinterpret_cast<float4*>(Us + c * NS)[i4] = make_float4(ur[4 * i4], ur[4 * i4 + 1], ur[4 * i4 + 2], ur[4 * i4 + 3]);
        }
        __syncwarp();
        {
            float acc[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) acc[i] = (i == c) ? -1.0f : 0.0f;
            for (int i = 0; i < NS; ++i) {
                const float uic = own ? Us[i * NS + c] : 0.0f;
                const float4* u4 = reinterpret_cast<const float4*>(Us + i * NS);
#pragma unroll
                for (int j4 = 0; j4 < NS / 4; ++j4) {
                    const float4 uv = u4[j4];
                    acc[4 * j4] = fmaf(uic, uv.x, acc[4 * j4]);
                    acc[4 * j4 + 1] = fmaf(uic, uv.y, acc[4 * j4 + 1]);
                    acc[4 * j4 + 2] = fmaf(uic, uv.z, acc[4 * j4 + 2]);
                    acc[4 * j4 + 3] = fmaf(uic, uv.w, acc[4 * j4 + 3]);
                }
            }
            // Row c of E (= column c) into Vs.
            if (own) {
#pragma unroll
                for (int i4 = 0; i4 < NS / 4; ++i4)
                    reinterpret_cast<float4*>(Vs + c * NS)[i4] =
                        make_float4(acc[4 * i4], acc[4 * i4 + 1], acc[4 * i4 + 2], acc[4 * i4 + 3]);
            }
        }
        __syncwarp();
        {
            // U <- U (I - E/2), row c: sum_j U_cj E_j. (U_cj from shared memory).
            float acc[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) acc[i] = 0.0f;
            for (int j = 0; j < NS; ++j) {
                const float ucj = own ? Us[c * NS + j] : 0.0f;
                const float4* e4 = reinterpret_cast<const float4*>(Vs + j * NS);
#pragma unroll
                for (int i4 = 0; i4 < NS / 4; ++i4) {
                    const float4 ev = e4[i4];
                    acc[4 * i4] = fmaf(ucj, ev.x, acc[4 * i4]);
                    acc[4 * i4 + 1] = fmaf(ucj, ev.y, acc[4 * i4 + 1]);
                    acc[4 * i4 + 2] = fmaf(ucj, ev.z, acc[4 * i4 + 2]);
                    acc[4 * i4 + 3] = fmaf(ucj, ev.w, acc[4 * i4 + 3]);
                }
            }
#pragma unroll
            for (int i = 0; i < NS; ++i) ur[i] = fmaf(-0.5f, acc[i], ur[i]);
        }
        __syncwarp();  // Us is rewritten below
        if (own) {
#pragma unroll
            for (int i4 = 0; i4 < NS / 4; ++i4)
                reinterpret_cast<float4*>(Us + c * NS)[i4] = make_float4(ur[4 * i4], ur[4 * i4 + 1], ur[4 * i4 + 2], ur[4 * i4 + 3]);
        }
        __syncwarp();
        // Out: row c of Y (= the re-orthonormalised U) and l_c.
        if (own) {
            float* yo = ra.Yg + lc * NS * NS + (size_t)c * NS;
#pragma unroll
            for (int i4 = 0; i4 < NS / 4; ++i4)
                reinterpret_cast<float4*>(yo)[i4] = make_float4(ur[4 * i4], ur[4 * i4 + 1], ur[4 * i4 + 2], ur[4 * i4 + 3]);
            ra.lamg[lc * NS + c] = lamc;
        }
        warm = true;
    }
}

// Shared memory of one warp of kernel F (floats), matrices of row stride NS:
//   Ah  [NS][NS]  A, high half; then E
//   Al  [NS][NS]  A, low half; then S' (off the diagonal), then g(S')
//   Ys  [NS][NS]  basis Y, row-major
//   Zb  [NS][NS]  scratch: R, then Z (rows 0..8) and Z Y (rows 9..17)
// Row groups of 8 or 16 read up to 8 floats past a matrix's last row; what
// follows each matrix in this layout is in bounds and the values are not
// used.
//   lsq [NS] (FP64) sqrt(rho-tilde); wh, wl its binary32 halves; dh d-hat;
//   lam eigenvalue estimates; vu sqrt(a + s_i); va 1/(u_i (u_i + sqrt a));
//   vh 1/(a + s_i); vt1 Y^T d-hat; vt2 h(S') vt1; vv Y vt2; xbar [32]
//   means (0..8) and Z v (9..17); gi [32] (ints); dX [9][k].
template <int NS>
struct FLayout {
    static constexpr int ZR = NS > 18 ? NS : 18;
    static constexpr int Ah = 0, Al = NS * NS, Yt = 2 * NS * NS, Zb = 3 * NS * NS;
    static constexpr int lsq = Zb + ZR * NS;
    static constexpr int wh = lsq + 2 * NS, wl = wh + NS, dh = wl + NS, lam = dh + NS;
    static constexpr int vu = lam + NS, va = vu + NS, vh = va + NS, vt1 = vh + NS, vt2 = vt1 + NS;
    static constexpr int vv = vt2 + NS, xbar = vv + NS, gi = xbar + 32, dX = gi + 32;
    static_assert(NS % 4 == 0, "rows of 16 bytes");
};

template <int NS>
__host__ __device__ inline size_t run_f_smem_bytes(int k) {
    return ((size_t)FLayout<NS>::dX + 9 * (size_t)k) * 4;
}

// Diagnostic output of the refinement kernel (PROBE = true): for listed
// grid points, the ensemble transform T = w-bar 1^T + W the refined
// representation gives, evaluated in FP64 (see probe_tail).
struct ProbeArgs {
    const int* cells;  // [npoints] grid points y * nx + x
    int npoints;
    double* T;         // [npoints][k][k]
    double* work;      // [npoints][probe_stride(NS, k)]
};

__host__ __device__ inline size_t probe_stride(int ns, int k) {
    return 8 * (size_t)ns + (size_t)ns * ns + 2 * (size_t)ns * k;
}

template <int NS>
__device__ void probe_tail(const RunArgs& ra, const ProbeArgs& pa, int pt, const float* Ys, const float* Ew,
                           const float* Sw, const double* lsq, const int* gi, int nu, double uu, double alpha,
                           double hh, int lane);

template <int NS, bool PROBE>
__device__ __forceinline__ void run_refine_body(const RunArgs& ra, const ProbeArgs& pa, int blk) {
    extern __shared__ __align__(16) float smf[];
    using L = FLayout<NS>;
    float* const Ah = smf + L::Ah;
    float* const Al = smf + L::Al;
    float* const Ys = smf + L::Yt;
    float* const Zb = smf + L::Zb;
    double* const lsq = reinterpret_cast<double*>(smf + L::lsq);
    float* const vwh = smf + L::wh;
    float* const vwl = smf + L::wl;
    float* const dh = smf + L::dh;
    float* const vlam = smf + L::lam;
    float* const vu = smf + L::vu;
    float* const va = smf + L::va;
    float* const vh = smf + L::vh;
    float* const vt1 = smf + L::vt1;
    float* const vt2 = smf + L::vt2;
    float* const vv = smf + L::vv;
    float* const xbar = smf + L::xbar;
    int* const gi = reinterpret_cast<int*>(smf + L::gi);
    float* const dX = smf + L::dX;
    const ObsParams& o = ra.o;
    const int k = ra.k;
    const int nobs = o.nvar * o.npts;
    const size_t plane = (size_t)ra.nx * ra.ny * k;
    const int lane = threadIdx.x;
    const int runs_x = (ra.nx + ra.R - 1) / ra.R;
    int lc, rl, x, y;
    if (PROBE) {
        // Block b takes listed point b if its run is in this chunk.
        const int cl = pa.cells[blk];
        y = cl / ra.nx;
        x = cl - y * ra.nx;
        const int run = y * runs_x + x / ra.R;
        if (run < ra.run0 || run >= ra.run0 + ra.nruns) return;
        rl = run - ra.run0;
        lc = rl * ra.R + (x - (x / ra.R) * ra.R);
    } else {
        lc = blk;  // cell within the chunk
        rl = lc / ra.R;
        const int run = ra.run0 + rl;
        y = run / runs_x;
        x = (run - y * runs_x) * ra.R + (lc - rl * ra.R);
        if (x >= ra.nx) return;  // past the end of a ragged last run
    }
    const size_t cell = (size_t)y * ra.nx + x;
    if (!PROBE) stage_point(ra, dX, cell, lane);
    const float sbeta = ra.sqrt_beta_f;
    const int* info = ra.rinfo + (size_t)rl * kInfo;
    const int nu = info[0];
    const float lam_mark = ra.lamg[(size_t)lc * NS];
    if (nu < 0) return;  // reported by kernel J
    if (PROBE && (nu == 0 || lam_mark == -1.0f)) {
        // No observation in range: T = sqrt(beta) I.
        double* Tp = pa.T + (size_t)blk * k * k;
        for (int e = lane; e < k * k; e += 32) Tp[e] = (e / k == e % k) ? sqrt(ra.beta) : 0.0;
        return;
    }
    if (nu == 0 || lam_mark == -1.0f) {
        // No observation in range: x^a = xbar + sqrt(beta) dx.
        cp_async_wait_all();
        __syncwarp();
        float* fc = ra.f + cell * k;
        for (int aq = 0; aq < 9; ++aq) {
            float s = 0.0f;
            for (int m = lane; m < k; m += 32) s += dX[aq * k + m];
            const float mean = warp_sum(s) / (float)k;
            for (int m = lane; m < k; m += 32) fc[aq * plane + m] = fmaf(sbeta, dX[aq * k + m] - mean, mean);
        }
        return;
    }
    const float rsf = ra.sqrt_a_f;
    const float sk = ra.sqrt_k1_f;
    const bool own = lane < NS;
    const bool real = lane < nu;
    const int c = lane;
    if (lane < nu) gi[lane] = info[1 + lane];
    // The basis (row-major) and eigenvalue estimates.
    {
        const float4* src = reinterpret_cast<const float4*>(ra.Yg + (size_t)lc * NS * NS);
        for (int e = lane; e < NS * NS / 4; e += 32) reinterpret_cast<float4*>(Ys)[e] = src[e];
        if (own) vlam[c] = ra.lamg[(size_t)lc * NS + c];
    }
    __syncwarp();
    const int gic = real ? gi[c] : 0;
    const double w = real ? ra.wg[(size_t)lc * NS + c] : 0.0;  // kernel J's weight of scalar c
    const float w_h = (float)w;
    const float w_l = (float)(w - (double)w_h);
    if (own) {
        lsq[c] = w;
        vwh[c] = w_h;
        vwl[c] = w_l;
        dh[c] = (float)(w * (real ? o.d[gic] : 0.0));
    }
    __syncwarp();
    // Column c of A = w_i G_ic w_c in double-binary32, as hi + lo.
    {
        float2 gv[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i)
            gv[i] = (real && i < nu) ? ra.G2[(size_t)gi[i] * nobs + gic] : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            // w_i w_c in double-binary32, formed the same way by lanes i and
            // c (so A is exactly symmetric), then times G_ic.
            const float wih = vwh[i], wil = vwl[i];
            const float p = wih * w_h;
            float e = fmaf(wih, w_h, -p);
            e += wih * w_l + wil * w_h;
            const float q = p * gv[i].x;
            float qe = fmaf(p, gv[i].x, -q);
            qe = fmaf(p, gv[i].y, fmaf(e, gv[i].x, qe));
            const float hv = q + qe;
            const float lv = qe - (hv - q);
            if (own) {
                Ah[i * NS + c] = hv;
                Al[i * NS + c] = lv;
            }
        }
    }
    float u[NS];  // column c of Y
#pragma unroll
    for (int j = 0; j < NS; ++j) u[j] = own ? Ys[j * NS + c] : 0.0f;
    const float lamc = own ? vlam[c] : 0.0f;
    __syncwarp();
    // R = A Y - Y diag(l), column c, double-binary32, into Zb. Rows in
    // groups of RG, two per packed register: A is symmetric, so rows
    // i..i+RG-1 of column j are entries i..i+RG-1 of row j. A group reads up
    // to RG - (NS mod RG) floats past a row's end; what follows each matrix
    // in this layout is in bounds and the extra rows are not stored.
    constexpr int RG = NS >= 16 ? 16 : 8;  // rows per group of E and T: RG / 2 independent sums
    constexpr int NQ = RG / 2;
    // R: all rows in one group (NS / 2 independent sums per lane; F is
    // stalled on fixed-latency dependences, and this fits the registers
    // of 3 warps per sub-partition). E and T in one group need more
    // registers and measured slower.
    constexpr int RG1 = NS, NQ1 = RG1 / 2;
    for (int i0 = 0; i0 < NS; i0 += RG1) {
        f2x S[NQ1], C[NQ1];
#pragma unroll
        for (int q = 0; q < NQ1; ++q) S[q] = C[q] = 0ull;
#pragma unroll 2
        for (int j = 0; j < NS; ++j) {
            const float uj = own ? Ys[j * NS + c] : 0.0f;  // Y_jc
            const f2x Y2 = f2pack(uj, uj), NY2 = f2pack(-uj, -uj);
#pragma unroll
            for (int g = 0; g < RG1 / 4; ++g) {
                const ulonglong2 h = *reinterpret_cast<const ulonglong2*>(Ah + j * NS + i0 + 4 * g);
                const ulonglong2 l = *reinterpret_cast<const ulonglong2*>(Al + j * NS + i0 + 4 * g);
                df2_acc(S[2 * g], C[2 * g], h.x, l.x, Y2, NY2);
                df2_acc(S[2 * g + 1], C[2 * g + 1], h.y, l.y, Y2, NY2);
            }
        }
#pragma unroll
        for (int q = 0; q < NQ1; ++q) {
            float s2[2], c2[2];
            f2unpack(S[q], s2[0], s2[1]);
            f2unpack(C[q], c2[0], c2[1]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = i0 + 2 * q + h;
                if (i < NS) {
                    const float yi = own ? Ys[i * NS + c] : 0.0f;
                    const float p = __fmul_rn(yi, lamc);
                    const float pe = __fmaf_rn(yi, lamc, -p);
                    if (own) Zb[i * NS + c] = __fadd_rn(__fsub_rn(s2[h], p), __fsub_rn(c2[h], pe));
                }
            }
        }
    }
    __syncwarp();  // A is no longer read: E and S' take its place
    // E = Y^T Y - I (double-binary32) and T = Y^T R (binary32); S'. Rows in
    // groups of RG: E_ic = sum_j Y_ji Y_jc, so rows i..i+RG-1 read entries
    // i..i+RG-1 of row j of Y.
    float ecc = 0.0f, tcc = 0.0f;
    // Unrolled: in the last group the sums of rows past NS are dead and go.
#pragma unroll
    for (int i0 = 0; i0 < NS; i0 += RG) {
        f2x ES[NQ], EC[NQ], TQ[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) ES[q] = EC[q] = TQ[q] = 0ull;
#pragma unroll 2
        for (int j = 0; j < NS; ++j) {
            const float uj = own ? Ys[j * NS + c] : 0.0f;  // Y_jc
            const float rj = own ? Zb[j * NS + c] : 0.0f;  // R_jc
            const f2x Y2 = f2pack(uj, uj), NY2 = f2pack(-uj, -uj), R2 = f2pack(rj, rj);
#pragma unroll
            for (int g = 0; g < RG / 4; ++g) {
                const ulonglong2 y = *reinterpret_cast<const ulonglong2*>(Ys + j * NS + i0 + 4 * g);
                df2_acc1(ES[2 * g], EC[2 * g], y.x, Y2, NY2);
                df2_acc1(ES[2 * g + 1], EC[2 * g + 1], y.y, Y2, NY2);
                TQ[2 * g] = f2fma(y.x, R2, TQ[2 * g]);
                TQ[2 * g + 1] = f2fma(y.y, R2, TQ[2 * g + 1]);
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float es2[2], ec2[2], tq2[2];
            f2unpack(ES[q], es2[0], es2[1]);
            f2unpack(EC[q], ec2[0], ec2[1]);
            f2unpack(TQ[q], tq2[0], tq2[1]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = i0 + 2 * q + h;
                if (i < NS) {
                    const float e = __fadd_rn(__fsub_rn(es2[h], i == c ? 1.0f : 0.0f), ec2[h]);
                    if (i == c) {
                        ecc = e;
                        tcc = tq2[h];
                    }
                    if (own) {
                        Ah[i * NS + c] = e;
                        Al[i * NS + c] = (i == c) ? 0.0f : fmaf(e, 0.5f * (lamc - vlam[i]), tq2[h]);
                    }
                }
            }
        }
    }
    // Matrix functions of S' (observation space): the diagonal entry s_c of
    // S' and u_c = sqrt(a + s_c), alpha_c = 1 / (u_c (u_c + sqrt a)),
    // h_c = 1 / (a + s_c). The probe evaluates them in FP64; the update
    // uses them in binary32 products, so it evaluates them in binary32.
    if constexpr (PROBE) {
        const double aa = (k - 1) / ra.beta;
        const double rs = sqrt(aa);
        const double dS = (double)lamc + (double)(tcc - ecc * tcc - ecc * ecc * lamc);
        const double uu = sqrt(aa + dS);
        const double alpha = 1.0 / (uu * (uu + rs));
        const double hh = 1.0 / (aa + dS);
        __syncwarp();
        probe_tail<NS>(ra, pa, blk, Ys, Ah, Al, lsq, gi, nu, uu, alpha, hh, lane);
        return;
    }
    float t1c = 0.0f;
#pragma unroll
    for (int l = 0; l < NS; ++l) t1c = fmaf(u[l], dh[l], t1c);  // (Y^T d-hat)_c
    const float ap = ra.a_f + (lamc + (tcc - ecc * tcc - ecc * ecc * lamc));  // a + s_c
    const float uc = sqrtf(ap);
    const float ac = 1.0f / (uc * (uc + rsf));
    const float hc = 1.0f / ap;
    if (own) {
        vu[c] = uc;
        va[c] = ac;
        vh[c] = hc;
        vt1[c] = t1c;
    }
    __syncwarp();
    {
        // t2 = h(S') t1: h_ii = h_i, h_ij = -S'_ij h_i h_j, and the basis
        // factor, minus E o (h_i + h_j)/2. g(S') column c over S'.
        float tt = 0.0f, te = 0.0f;
        const float gc = -ac / rsf;
        for (int j = 0; j < NS; ++j) {
            const float hj = vh[j], t1j = vt1[j];
            const float sv = own ? Al[j * NS + c] : 0.0f;  // S'_jc (zero at j = c)
            const float ev = own ? Ah[j * NS + c] : 0.0f;
            tt = fmaf(sv, hj * t1j, tt);
            te = fmaf(ev * (0.5f * (hc + hj)), t1j, te);
            // g(S')_jc: diagonal -alpha/sqrt(a); off the diagonal
            // S'_jc (u_j + u_c + sqrt a) alpha_j alpha_c / (sqrt(a) (u_j + u_c));
            // minus E_jc (g_j + g_c)/2.
            const float uj = vu[j], aj = va[j];
            float gv;
            if (j == c)
                gv = gc;
            else
                gv = sv * (uj + uc + rsf) * aj * ac / (rsf * (uj + uc));
            gv -= ev * (0.5f * (gc - aj / rsf));
            if (own) Al[j * NS + c] = gv;
        }
        if (own) vt2[c] = hc * (t1c - tt) - te;
    }
    __syncwarp();
    // v = Y t2 (lane c takes row c of Y).
    {
        float v0 = 0.0f, v1 = 0.0f;
#pragma unroll
        for (int l = 0; l < NS; l += 2) {
            v0 = fmaf(own ? Ys[c * NS + l] : 0.0f, vt2[l], v0);
            v1 = fmaf(own ? Ys[c * NS + l + 1] : 0.0f, vt2[l + 1], v1);
        }
        if (own) vv[c] = v0 + v1;
    }
    // Transform. The ensemble of this point has arrived in dX.
    cp_async_wait_all();
    __syncwarp();
    for (int aq = 0; aq < 9; ++aq) {
        float s = 0.0f;
        for (int m = lane; m < k; m += 32) s += dX[aq * k + m];
        s = warp_sum(s);
        const float mean = s / (float)k;
        for (int m = lane; m < k; m += 32) dX[aq * k + m] -= mean;
        if (lane == 0) xbar[aq] = mean;
    }
    __syncwarp();
    // Z = dX Yh^T, column c: sqrt(rho)_c dX dY32[gi_c]^T.
    float* const Z = Zb;            // [9][NS]
    float* const ZY = Zb + 9 * NS;  // [9][NS]
    {
        float acc[9];
#pragma unroll
        for (int aq = 0; aq < 9; ++aq) acc[aq] = 0.0f;
        if (real) {
            const float* row = o.dY32 + (size_t)gic * k;
            if ((k & 3) == 0) {
                const float4* row4 = reinterpret_cast<const float4*>(row);
#pragma unroll 4
                for (int m4 = 0; m4 < (k >> 2); ++m4) {
                    const float4 dy = row4[m4];
#pragma unroll
                    for (int aq = 0; aq < 9; ++aq) {
                        const float4 xv = reinterpret_cast<const float4*>(dX + aq * k)[m4];
                        acc[aq] = fmaf(xv.x, dy.x, acc[aq]);
                        acc[aq] = fmaf(xv.y, dy.y, acc[aq]);
                        acc[aq] = fmaf(xv.z, dy.z, acc[aq]);
                        acc[aq] = fmaf(xv.w, dy.w, acc[aq]);
                    }
                }
            } else {
                for (int m = 0; m < k; ++m) {
                    const float dy = row[m];
#pragma unroll
                    for (int aq = 0; aq < 9; ++aq) acc[aq] = fmaf(dX[aq * k + m], dy, acc[aq]);
                }
            }
        }
        if (own) {
#pragma unroll
            for (int aq = 0; aq < 9; ++aq) Z[aq * NS + c] = w_h * acc[aq];
        }
    }
    __syncwarp();
    // Z v, Z Y (column c).
    if (lane < 9) {
        float s = 0.0f;
        for (int i = 0; i < NS; ++i) s = fmaf(Z[lane * NS + i], vv[i], s);
        xbar[9 + lane] = s;
    }
    {
        float acc[9];
#pragma unroll
        for (int aq = 0; aq < 9; ++aq) acc[aq] = 0.0f;
#pragma unroll
        for (int l = 0; l < NS; ++l) {
#pragma unroll
            for (int aq = 0; aq < 9; ++aq) acc[aq] = fmaf(Z[aq * NS + l], u[l], acc[aq]);
        }
        if (own) {
#pragma unroll
            for (int aq = 0; aq < 9; ++aq) ZY[aq * NS + c] = acc[aq];
        }
    }
    __syncwarp();
    // (Z Y) g(S') (column c) into Z.
    {
        float acc[9];
#pragma unroll
        for (int aq = 0; aq < 9; ++aq) acc[aq] = 0.0f;
        for (int j = 0; j < NS; ++j) {
            const float gj = own ? Al[j * NS + c] : 0.0f;
#pragma unroll
            for (int aq = 0; aq < 9; ++aq) acc[aq] = fmaf(ZY[aq * NS + j], gj, acc[aq]);
        }
        __syncwarp();  // Z is read (Z v, Z Y) before it is overwritten
        if (own) {
#pragma unroll
            for (int aq = 0; aq < 9; ++aq) Z[aq * NS + c] = acc[aq];
        }
    }
    __syncwarp();
    // B = sqrt(k-1) (Z Y g) Y^T diag(sqrt rho), column c into ZY.
    {
        float acc[9];
#pragma unroll
        for (int aq = 0; aq < 9; ++aq) acc[aq] = 0.0f;
        for (int i = 0; i < NS; ++i) {
            const float yci = own ? Ys[c * NS + i] : 0.0f;  // Y[c][i]
#pragma unroll
            for (int aq = 0; aq < 9; ++aq) acc[aq] = fmaf(Z[aq * NS + i], yci, acc[aq]);
        }
        const float sl = sk * w_h;
        __syncwarp();
        if (own) {
#pragma unroll
            for (int aq = 0; aq < 9; ++aq) ZY[aq * NS + c] = sl * acc[aq];
        }
    }
    __syncwarp();
    // Update: x^a_m = xbar + Z v + sqrt(beta) dx_m + B yh_m.
    {
        float* fc = ra.f + cell * k;
        for (int m = lane; m < k; m += 32) {
            float acc[9];
#pragma unroll
            for (int aq = 0; aq < 9; ++aq) acc[aq] = fmaf(sbeta, dX[aq * k + m], xbar[aq] + xbar[9 + aq]);
#pragma unroll 4
            for (int i = 0; i < nu; ++i) {
                const float dy = o.dY32[(size_t)gi[i] * k + m];
#pragma unroll
                for (int aq = 0; aq < 9; ++aq) acc[aq] = fmaf(ZY[aq * NS + i], dy, acc[aq]);
            }
#pragma unroll
            for (int aq = 0; aq < 9; ++aq) fc[aq * plane + m] = acc[aq];
        }
    }
}

// FP64 evaluation of the ensemble transform from the refined representation
// of one grid point: basis Y (binary32, row-major in Ys), E = Y^T Y - I
// (column c of Ew), S' off the diagonal (column c of Sw) and, per lane c, the
// FP64 eigenvalue functions u_c = sqrt(a + s'_cc), alpha_c, h_c. With the
// same first-order formulas as the analysis (h(S') t1 and g(S')), but every
// product in FP64:
//   t1 = Y^T d-hat, t2 = h(S') t1, v = Y t2, F = g(S') (the basis factor
//   included), g(A) = Y F Y^T,
//   w-bar = Yh^T v, W = sqrt(beta) I + sqrt(k-1) Yh^T g(A) Yh,
//   T[j][m] = w-bar_j + W[j][m],
// the transform x^a_m = xbar + sum_j dx_j T[j][m] of Section 3.2.
template <int NS>
__device__ void probe_tail(const RunArgs& ra, const ProbeArgs& pa, int pt, const float* Ys, const float* Ew,
                           const float* Sw, const double* lsq, const int* gi, int nu, double uu, double alpha,
                           double hh, int lane) {
    const int k = ra.k;
    const bool own = lane < NS;
    const int c = lane;
    const ObsParams& o = ra.o;
    double* wk = pa.work + (size_t)pt * probe_stride(NS, k);
    double* U = wk;
    double* AL = U + NS;
    double* H = AL + NS;
    double* T1 = H + NS;
    double* T2 = T1 + NS;
    double* V = T2 + NS;
    double* LS = V + NS;
    double* DH = LS + NS;
    double* F = DH + NS;
    double* C1 = F + NS * NS;
    double* C2 = C1 + (size_t)NS * k;
    const double aa = (k - 1) / ra.beta;
    const double rs = sqrt(aa);
    if (own) {
        U[c] = uu;
        AL[c] = alpha;
        H[c] = hh;
        LS[c] = lsq[c];
        DH[c] = (c < nu) ? lsq[c] * o.d[gi[c]] : 0.0;
    }
    __syncwarp();
    if (own) {
        double t = 0.0;
        for (int l = 0; l < NS; ++l) t += (double)Ys[l * NS + c] * DH[l];
        T1[c] = t;
    }
    __syncwarp();
    if (own) {
        double tt = 0.0, te = 0.0;
        for (int j = 0; j < NS; ++j) {
            const double sv = (j == c) ? 0.0 : (double)Sw[j * NS + c];
            const double ev = (double)Ew[j * NS + c];
            tt += sv * H[j] * T1[j];
            te += ev * 0.5 * (hh + H[j]) * T1[j];
        }
        T2[c] = hh * (T1[c] - tt) - te;
        const double gc = -alpha / rs;
        for (int j = 0; j < NS; ++j) {
            const double ev = (double)Ew[j * NS + c];
            double g = gc;
            if (j != c) g = (double)Sw[j * NS + c] * (U[j] + uu + rs) * AL[j] * alpha / (rs * (U[j] + uu));
            F[j * NS + c] = g - ev * 0.5 * (gc - AL[j] / rs);
        }
    }
    __syncwarp();
    if (own) {
        double v = 0.0;
        for (int l = 0; l < NS; ++l) v += (double)Ys[c * NS + l] * T2[l];
        V[c] = v;
    }
    // C1 = Y^T Yh, Yh[l][m] = sqrt(rho)_l dY[gi_l][m].
    for (int m = lane; m < k; m += 32)
        for (int q = 0; q < NS; ++q) {
            double acc = 0.0;
            for (int l = 0; l < nu; ++l) acc += (double)Ys[l * NS + q] * LS[l] * o.dY[(size_t)gi[l] * k + m];
            C1[(size_t)q * k + m] = acc;
        }
    __syncwarp();
    // C2 = F C1, then B = Y C2 (into C1).
    for (int m = lane; m < k; m += 32)
        for (int p = 0; p < NS; ++p) {
            double acc = 0.0;
            for (int q = 0; q < NS; ++q) acc += F[p * NS + q] * C1[(size_t)q * k + m];
            C2[(size_t)p * k + m] = acc;
        }
    __syncwarp();
    for (int m = lane; m < k; m += 32)
        for (int i = 0; i < NS; ++i) {
            double acc = 0.0;
            for (int p = 0; p < NS; ++p) acc += (double)Ys[i * NS + p] * C2[(size_t)p * k + m];
            C1[(size_t)i * k + m] = acc;
        }
    __syncwarp();
    const double sq = sqrt((double)(k - 1)), sb = sqrt(ra.beta);
    double* Tp = pa.T + (size_t)pt * k * k;
    for (int m = lane; m < k; m += 32)
        for (int j = 0; j < k; ++j) {
            double wb = 0.0, s = 0.0;
            for (int i = 0; i < nu; ++i) {
                const double yh = LS[i] * o.dY[(size_t)gi[i] * k + j];
                wb += yh * V[i];
                s += yh * C1[(size_t)i * k + m];
            }
            Tp[(size_t)j * k + m] = wb + sq * s + (j == m ? sb : 0.0);
        }
}

// ---- kernels: one experiment, or a batch of experiments ------------------
// A batch launch of kernel J covers the runs of up to kRunBatch experiments
// of one size class (NS): block b belongs to the experiment e with
// jstart[e] <= b < jstart[e + 1]. The table travels as a kernel parameter.
// Kernel F is launched per experiment: its shared memory depends on the
// members k, and sizing it for a batch's largest k costs the others
// occupancy in this latency-bound kernel (a batched F was 12% slower than
// the per-experiment launches over the seven run-path experiments of the
// uneven batch, against 5% gained by batching J).
constexpr int kRunBatch = 16;

struct RunBatch {
    int n;
    int jstart[kRunBatch + 1];  // first run of each experiment
    RunArgs ex[kRunBatch];
};

__device__ __forceinline__ int batch_item(const int* start, int n, int blk) {
    int e = 0;
    while (e + 1 < n && blk >= start[e + 1]) ++e;
    return e;
}

template <int NS>
__global__ void __launch_bounds__(32, 16) run_jacobi_kernel(const __grid_constant__ RunArgs ra) {
    run_jacobi_body<NS>(ra, blockIdx.x);
}

template <int NS>
__global__ void __launch_bounds__(32, 16) run_jacobi_batch_kernel(const __grid_constant__ RunBatch tb) {
    const int e = batch_item(tb.jstart, tb.n, blockIdx.x);
    run_jacobi_body<NS>(tb.ex[e], blockIdx.x - tb.jstart[e]);
}

template <int NS, bool PROBE>
__global__ void __launch_bounds__(32, 12) run_refine_kernel(const __grid_constant__ RunArgs ra,
                                                            const __grid_constant__ ProbeArgs pa) {
    run_refine_body<NS, PROBE>(ra, pa, blockIdx.x);
}

// G = dY dY^T split into binary32 (hi, lo).
__global__ void split_gram_kernel(const double* __restrict__ G, float2* __restrict__ G2, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double v = G[i];
        const float h = (float)v;
        G2[i] = make_float2(h, (float)(v - (double)h));
    }
}

int run_ns(int maxunion) {
    if (maxunion <= 8) return 8;
    if (maxunion <= 16) return 16;
    if (maxunion <= 24) return 24;
    if (maxunion <= 28) return 28;
    return 32;
}

constexpr size_t kRunScratchBudget = 320ull << 20;  // basis scratch per chunk

long long run_chunk_runs(long long runs, int R, int ns) {
    const size_t per_run = (size_t)R * (run_cell_floats(ns) * 4 + ns * 8) + kInfo * 4;
    long long c = (long long)(kRunScratchBudget / per_run);
    if (c < 1) c = 1;
    return runs < c ? runs : c;
}

// Per chunk of runs: kernel J, then kernel F over the chunk's grid points,
// or (pa.npoints > 0) the probe variant of F over the listed points.
template <int NS>
cudaError_t launch_runs_ns(RunArgs ra, long long runs, long long chunk, const ProbeArgs& pa, cudaStream_t s) {
    const size_t shJ = (size_t)JLayout<NS>::total * 4;
    const size_t shF = run_f_smem_bytes<NS>(ra.k);
    const bool probe = pa.npoints > 0;
    cudaError_t e = cudaFuncSetAttribute(run_jacobi_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shJ);
    if (e != cudaSuccess) return e;
    if (!ra.f64)
        e = probe ? cudaFuncSetAttribute(run_refine_kernel<NS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shF)
              : cudaFuncSetAttribute(run_refine_kernel<NS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shF);
    if (e != cudaSuccess) return e;
    for (long long r0 = 0; r0 < runs; r0 += chunk) {
        const long long nr = runs - r0 < chunk ? runs - r0 : chunk;
        ra.run0 = (int)r0;
        ra.nruns = (int)nr;
        run_jacobi_kernel<NS><<<(unsigned)nr, 32, shJ, s>>>(ra);
        if (ra.f64) {
            // Double-precision context: the FP64 Jacobi from J's basis.
            ObsParams o = ra.o;
            o.sweep_hist = ra.fp64_hist;
            e = launch_run_fp64(ra.f64, ra.nx, ra.ny, ra.k, o, ra.d_cut, ra.beta, ra.R, ra.run0, ra.nruns, NS,
                                ra.Yg, ra.lamg, ra.rinfo, kInfo, ra.flags, s);
            if (e != cudaSuccess) return e;
        } else if (probe)
            run_refine_kernel<NS, true><<<(unsigned)pa.npoints, 32, shF, s>>>(ra, pa);
        else
            run_refine_kernel<NS, false><<<(unsigned)(nr * ra.R), 32, shF, s>>>(ra, pa);
    }
    return cudaGetLastError();
}

// Pipelined form of launch_runs_ns: chunks of `pipe` runs, kernel J of
// chunk c + 1 on the second stream while kernel F (or the FP64 kernel) of
// chunk c runs on s, so that the issue-bound Jacobi and the latency-bound
// (or FP64-pipe-bound) refinement share the SMs. A chunk of ~2,000 runs is
// under one wave of J, so F's blocks find room beside it. The basis scratch
// (sized for `cap` runs per pass, cap >= 2 pipe) holds two buffers of
// `pipe` runs; J of chunk c waits for F of chunk c - 2 before reusing one.
template <int NS>
cudaError_t launch_runs_pipe(RunArgs ra, long long runs, long long pipe, const AnalyzeAux& aux, cudaStream_t s) {
    const size_t shJ = (size_t)JLayout<NS>::total * 4;
    const size_t shF = run_f_smem_bytes<NS>(ra.k);
    cudaError_t e = cudaFuncSetAttribute(run_jacobi_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shJ);
    if (e != cudaSuccess) return e;
    if (!ra.f64) {
        e = cudaFuncSetAttribute(run_refine_kernel<NS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shF);
        if (e != cudaSuccess) return e;
    }
    float* Yb[2] = {ra.Yg, ra.Yg + (size_t)pipe * ra.R * NS * NS};
    float* Lb[2] = {ra.lamg, ra.lamg + (size_t)pipe * ra.R * NS};
    double* Wb[2] = {ra.wg, ra.wg + (size_t)pipe * ra.R * NS};
    int* Ib[2] = {ra.rinfo, ra.rinfo + (size_t)pipe * kInfo};
    if ((e = cudaEventRecord(aux.start, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(aux.s2, aux.start, 0)) != cudaSuccess) return e;
    int c = 0;
    for (long long r0 = 0; r0 < runs; r0 += pipe, ++c) {
        const int b = c & 1;
        const long long nr = runs - r0 < pipe ? runs - r0 : pipe;
        RunArgs rb = ra;
        rb.run0 = (int)r0;
        rb.nruns = (int)nr;
        rb.Yg = Yb[b];
        rb.lamg = Lb[b];
        rb.wg = Wb[b];
        rb.rinfo = Ib[b];
        if (c >= 2 && (e = cudaStreamWaitEvent(aux.s2, aux.ref_done[b], 0)) != cudaSuccess) return e;
        run_jacobi_kernel<NS><<<(unsigned)nr, 32, shJ, aux.s2>>>(rb);
        if ((e = cudaEventRecord(aux.jac_done[b], aux.s2)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, aux.jac_done[b], 0)) != cudaSuccess) return e;
        if (rb.f64) {
            ObsParams o = rb.o;
            o.sweep_hist = rb.fp64_hist;
            e = launch_run_fp64(rb.f64, rb.nx, rb.ny, rb.k, o, rb.d_cut, rb.beta, rb.R, rb.run0, rb.nruns, NS, rb.Yg,
                                rb.lamg, rb.rinfo, kInfo, rb.flags, s);
            if (e != cudaSuccess) return e;
        } else {
            const ProbeArgs none{nullptr, 0, nullptr, nullptr};
            run_refine_kernel<NS, false><<<(unsigned)(nr * rb.R), 32, shF, s>>>(rb, none);
        }
        if ((e = cudaEventRecord(aux.ref_done[b], s)) != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// Run arguments of one analysis: the scratch laid out for `chunk` runs per
// pass (G2, then the basis, eigenvalue estimates, weights and union lists
// of a chunk), and the preparation kernels queued (the binary32 copy of dY for a
// binary32 state, the split Gram).
cudaError_t run_setup(float* f, double* f64, int nx, int ny, int k, const ObsParams& o, double d_cut, double beta,
                      int run_len, int maxunion, int* flags, void* scratch, long long chunk, RunArgs& ra,
                      cudaStream_t s) {
    if (run_len < 1 || maxunion > kRunMaxUnion || !scratch || (f == nullptr) == (f64 == nullptr))
        return cudaErrorInvalidValue;
    if (f && !o.dY32) return cudaErrorInvalidValue;
    const int nobs = o.nvar * o.npts;
    const size_t ng = (size_t)nobs * nobs;
    const int ns = run_ns(maxunion);
    unsigned char* p = reinterpret_cast<unsigned char*>(scratch);
    float2* G2 = reinterpret_cast<float2*>(p);
    p += (ng * sizeof(float2) + 255) / 256 * 256;
    float* Yg = reinterpret_cast<float*>(p);
    p += ((size_t)chunk * run_len * ns * ns * 4 + 255) / 256 * 256;
    float* lamg = reinterpret_cast<float*>(p);
    p += ((size_t)chunk * run_len * ns * 4 + 255) / 256 * 256;
    double* wg = reinterpret_cast<double*>(p);
    p += ((size_t)chunk * run_len * ns * 8 + 255) / 256 * 256;
    int* rinfo = reinterpret_cast<int*>(p);
    // dY in binary32 for the transform (the same copy the chunked path makes).
    if (f) {
        const cudaError_t e = launch_to_f32(o.dY, o.dY32, (size_t)nobs * k, s);
        if (e != cudaSuccess) return e;
    }
    split_gram_kernel<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(o.G, G2, ng);
    ra.f = f;
    ra.f64 = f64;
    ra.nx = nx;
    ra.ny = ny;
    ra.k = k;
    ra.R = run_len;
    ra.o = o;
    ra.G2 = G2;
    ra.d_cut = d_cut;
    ra.beta = beta;
    ra.lim2 = support_lim2(d_cut);
    ra.a_f = (float)((k - 1) / beta);
    ra.sqrt_a_f = (float)std::sqrt((k - 1) / beta);
    ra.sqrt_beta_f = (float)std::sqrt(beta);
    ra.sqrt_k1_f = (float)std::sqrt((double)(k - 1));
    ra.flags = flags;
    ra.run0 = 0;
    ra.nruns = 0;
    ra.Yg = Yg;
    ra.lamg = lamg;
    ra.wg = wg;
    ra.rinfo = rinfo;
    ra.fp64_hist = nullptr;
    if (f64) {
        // The histogram records the FP64 solve, not the binary32 start.
        ra.fp64_hist = o.sweep_hist;
        ra.o.sweep_hist = nullptr;
    }
    return cudaGetLastError();
}

long long run_count(int nx, int ny, int run_len) { return (long long)ny * ((nx + run_len - 1) / run_len); }

cudaError_t launch_runs(float* f, double* f64, int nx, int ny, int k, const ObsParams& o, double d_cut,
                        double beta, int run_len, int maxunion, int* flags, void* scratch, const ProbeArgs& pa,
                        const AnalyzeAux* aux, int pipe_runs, cudaStream_t s) {
    if (f64 && pa.npoints > 0) return cudaErrorInvalidValue;
    if (run_len < 1) return cudaErrorInvalidValue;
    const int ns = run_ns(maxunion);
    const long long runs = run_count(nx, ny, run_len);
    if (runs > 0x7fffffffLL / run_len) return cudaErrorInvalidConfiguration;
    const long long chunk = run_chunk_runs(runs, run_len, ns);
    RunArgs ra;
    const cudaError_t e = run_setup(f, f64, nx, ny, k, o, d_cut, beta, run_len, maxunion, flags, scratch, chunk, ra, s);
    if (e != cudaSuccess) return e;
    // Pipelined when there is a second stream, more than one chunk of
    // pipe_runs, and room for two of them in the scratch.
    if (aux && pa.npoints == 0 && pipe_runs > 0 && runs > pipe_runs && 2 * (long long)pipe_runs <= chunk) {
        switch (ns) {
            case 8: return launch_runs_pipe<8>(ra, runs, pipe_runs, *aux, s);
            case 16: return launch_runs_pipe<16>(ra, runs, pipe_runs, *aux, s);
            case 24: return launch_runs_pipe<24>(ra, runs, pipe_runs, *aux, s);
            case 28: return launch_runs_pipe<28>(ra, runs, pipe_runs, *aux, s);
            default: return launch_runs_pipe<32>(ra, runs, pipe_runs, *aux, s);
        }
    }
    switch (ns) {
        case 8: return launch_runs_ns<8>(ra, runs, chunk, pa, s);
        case 16: return launch_runs_ns<16>(ra, runs, chunk, pa, s);
        case 24: return launch_runs_ns<24>(ra, runs, chunk, pa, s);
        case 28: return launch_runs_ns<28>(ra, runs, chunk, pa, s);
        default: return launch_runs_ns<32>(ra, runs, chunk, pa, s);
    }
}

// One size class of a batch: kernel J over every run of the experiments in
// launches of kRunBatch experiments, then per experiment kernel F over its
// grid points (binary32 states) or the FP64 kernel (FP64 states).
template <int NS>
cudaError_t launch_runs_batch_ns(const std::vector<RunArgs>& ex, cudaStream_t s) {
    const size_t shJ = (size_t)JLayout<NS>::total * 4;
    int kmax = 0;
    for (const RunArgs& ra : ex) kmax = ra.k > kmax ? ra.k : kmax;
    cudaError_t e = cudaFuncSetAttribute(run_jacobi_batch_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)shJ);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(run_refine_kernel<NS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)run_f_smem_bytes<NS>(kmax));
    if (e != cudaSuccess) return e;
    const ProbeArgs none{nullptr, 0, nullptr, nullptr};
    for (size_t i0 = 0; i0 < ex.size(); i0 += kRunBatch) {
        const int n = (int)std::min<size_t>(kRunBatch, ex.size() - i0);
        RunBatch tb{};
        tb.n = n;
        long long jt = 0;
        for (int i = 0; i < n; ++i) {
            tb.ex[i] = ex[i0 + i];
            tb.jstart[i] = (int)jt;
            jt += tb.ex[i].nruns;
            if (jt > 0x7fffffffLL || (long long)tb.ex[i].nruns * tb.ex[i].R > 0x7fffffffLL)
                return cudaErrorInvalidConfiguration;
        }
        tb.jstart[n] = (int)jt;
        run_jacobi_batch_kernel<NS><<<(unsigned)jt, 32, shJ, s>>>(tb);
        for (int i = 0; i < n; ++i) {
            const RunArgs& ra = tb.ex[i];
            if (ra.f64) {
                ObsParams o = ra.o;
                o.sweep_hist = ra.fp64_hist;
                e = launch_run_fp64(ra.f64, ra.nx, ra.ny, ra.k, o, ra.d_cut, ra.beta, ra.R, 0, ra.nruns, NS, ra.Yg,
                                    ra.lamg, ra.rinfo, kInfo, ra.flags, s);
                if (e != cudaSuccess) return e;
            } else {
                run_refine_kernel<NS, false>
                    <<<(unsigned)((long long)ra.nruns * ra.R), 32, run_f_smem_bytes<NS>(ra.k), s>>>(ra, none);
            }
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

size_t run_scratch_bytes(int nx, int ny, int nobs, int run_len, int maxunion, bool whole) {
    const int ns = run_ns(maxunion);
    const long long runs = run_count(nx, ny, run_len);
    const long long chunk = whole ? runs : run_chunk_runs(runs, run_len, ns);
    const size_t g2 = ((size_t)nobs * nobs * sizeof(float2) + 255) / 256 * 256;
    const size_t yb = ((size_t)chunk * run_len * ns * ns * 4 + 255) / 256 * 256;
    const size_t lb = ((size_t)chunk * run_len * ns * 4 + 255) / 256 * 256;
    const size_t wb = ((size_t)chunk * run_len * ns * 8 + 255) / 256 * 256;
    const size_t ib = (size_t)chunk * kInfo * 4;
    return g2 + yb + lb + wb + ib;
}

cudaError_t launch_analyze_runs(float* f, int nx, int ny, int k, const ObsParams& o, double d_cut,
                                double beta, int run_len, int maxunion, int* flags, void* scratch,
                                const AnalyzeAux* aux, int pipe_runs, cudaStream_t s) {
    const ProbeArgs none{nullptr, 0, nullptr, nullptr};
    return launch_runs(f, nullptr, nx, ny, k, o, d_cut, beta, run_len, maxunion, flags, scratch, none, aux,
                       pipe_runs, s);
}

cudaError_t launch_analyze_runs_fp64(double* f, int nx, int ny, int k, const ObsParams& o, double d_cut,
                                     double beta, int run_len, int maxunion, int* flags, void* scratch,
                                     const AnalyzeAux* aux, int pipe_runs, cudaStream_t s) {
    const ProbeArgs none{nullptr, 0, nullptr, nullptr};
    return launch_runs(nullptr, f, nx, ny, k, o, d_cut, beta, run_len, maxunion, flags, scratch, none, aux,
                       pipe_runs, s);
}

size_t probe_work_bytes(int npoints, int maxunion, int k) {
    return (size_t)npoints * probe_stride(run_ns(maxunion), k) * sizeof(double);
}

cudaError_t launch_probe_runs(float* f, int nx, int ny, int k, const ObsParams& o, double d_cut, double beta,
                              int run_len, int maxunion, int* flags, void* scratch, const int* cells,
                              int npoints, double* T, double* work, cudaStream_t s) {
    if (npoints < 1 || !cells || !T || !work) return cudaErrorInvalidValue;
    const ProbeArgs pa{cells, npoints, T, work};
    return launch_runs(f, nullptr, nx, ny, k, o, d_cut, beta, run_len, maxunion, flags, scratch, pa, nullptr, 0, s);
}

cudaError_t launch_analyze_runs_batch(const RunItem* items, int n, cudaStream_t s) {
    // Preparation per experiment (scratch for every run at once), then one
    // size class after another.
    std::vector<RunArgs> cls[5];
    const int sizes[5] = {8, 16, 24, 28, 32};
    for (int i = 0; i < n; ++i) {
        const RunItem& it = items[i];
        if (it.run_len < 1) return cudaErrorInvalidValue;
        const long long runs = run_count(it.nx, it.ny, it.run_len);
        if (runs > 0x7fffffffLL / it.run_len) return cudaErrorInvalidConfiguration;
        RunArgs ra;
        const cudaError_t e = run_setup(it.f, it.f64, it.nx, it.ny, it.k, it.o, it.d_cut, it.beta, it.run_len,
                                        it.maxunion, it.flags, it.scratch, runs, ra, s);
        if (e != cudaSuccess) return e;
        ra.nruns = (int)runs;
        const int ns = run_ns(it.maxunion);
        for (int c = 0; c < 5; ++c)
            if (ns == sizes[c]) cls[c].push_back(ra);
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess && !cls[0].empty()) e = launch_runs_batch_ns<8>(cls[0], s);
    if (e == cudaSuccess && !cls[1].empty()) e = launch_runs_batch_ns<16>(cls[1], s);
    if (e == cudaSuccess && !cls[2].empty()) e = launch_runs_batch_ns<24>(cls[2], s);
    if (e == cudaSuccess && !cls[3].empty()) e = launch_runs_batch_ns<28>(cls[3], s);
    if (e == cudaSuccess && !cls[4].empty()) e = launch_runs_batch_ns<32>(cls[4], s);
    return e;
}

}  // namespace lbmgpu
