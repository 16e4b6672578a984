// Device helpers shared by the LETKF translation units (sm_103a). Internal
// linkage: every translation unit that includes this header gets its own copy.
#pragma once
#include <cmath>
#include <cstdint>

namespace lbmgpu {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Periodic minimum-image displacement on a ring of n cells.
__device__ __forceinline__ int min_image(int d, int n) {
    if (d > n / 2) d -= n;
    if (d < -(n / 2)) d += n;
    return d;
}

// Support prefilter of the local-set test on integers: dx^2 + dy^2 is an
// exact integer, and for values below 2^53 (distances below 9.4e7 cells)
// d2 <= floor((2 d_cut + 1)^2) decides exactly as the FP64 comparison of
// d2 with (2 d_cut + 1)^2, on the integer units instead of GB300's
// 1/64-rate FP64 pipe.
__device__ __forceinline__ long long dist2(int dx, int dy) {
    return (long long)dx * dx + (long long)dy * dy;
}
__host__ __device__ __forceinline__ long long support_lim2(double d_cut) {
    const double l2 = (2.0 * d_cut + 1.0) * (2.0 * d_cut + 1.0);
    return l2 >= 9.0e18 ? 0x7fffffffffffffffLL : (long long)floor(l2);
}

// Gaspari-Cohn weight (Section 3.2.2), both branches in nested (Horner) form.
__device__ __forceinline__ double gaspari_cohn(double d) {
    if (d <= 1.0) return 1.0 + d * d * (-5.0 / 3.0 + d * (0.625 + d * (0.5 - 0.25 * d)));
    if (d < 2.0)
        return d * d * (5.0 / 3.0 + d * (0.625 + d * (-0.5 + d * (1.0 / 12.0)))) - 5.0 * d + 4.0 -
               (2.0 / 3.0) / d;
    return 0.0;
}

// ---- Double-binary32 arithmetic -------------------------------------------
// GB300 issues FP64 at 1/64 of the binary32 rate, so accurate products run
// in binary32 with error-free transformations and a second accumulator
// (Knuth's TwoSum; the product error from one FMA, as in Dekker's
// double-length products; accumulated as in Ogita, Rump and Oishi,
// "Accurate sum and dot product", 2005). A binary32 factor y is exact and an
// FP64 factor is split into hi + lo binary32 parts, so every term
// a y = ah y + al y enters with ah y exact and al y to 2^-48; the sums carry
// a relative error ~ n 2^-48 of sum |terms|. The _rn intrinsics keep the
// compiler from fusing or reordering these steps.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// (s, c) += (ah + al) y.
__device__ __forceinline__ void df_acc(float& s, float& c, float ah, float al, float y) {
    const float p = __fmul_rn(ah, y);
    const float e = __fmaf_rn(ah, y, -p);  // ah y - p, exactly
    float t;
    two_sum(s, p, s, t);
    c = __fadd_rn(c, __fadd_rn(t, __fmaf_rn(al, y, e)));
}

// (s, c) += a y for binary32 a and y (the product is exact as p + e).
__device__ __forceinline__ void df_acc1(float& s, float& c, float a, float y) {
    const float p = __fmul_rn(a, y);
    const float e = __fmaf_rn(a, y, -p);
    float t;
    two_sum(s, p, s, t);
    c = __fadd_rn(c, __fadd_rn(t, e));
}

__device__ __forceinline__ double df_value(float s, float c) { return (double)s + (double)c; }

// ---- Packed binary32 pairs (sm_100 family: add/sub/mul/fma .f32x2) --------
// Two independent binary32 values in one 64-bit register, low half first
// (the lower address when loaded from memory). Each packed operation rounds
// each half exactly as the scalar operation would.
typedef unsigned long long f2x;

__device__ __forceinline__ f2x f2pack(float lo, float hi) {
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2unpack(f2x v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2x f2add(f2x a, f2x b) {
    f2x d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x f2sub(f2x a, f2x b) {
    f2x d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x f2mul(f2x a, f2x b) {
    f2x d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x f2fma(f2x a, f2x b, f2x c) {
    f2x d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// df_acc on two independent accumulations at once: (S, C) += (AH + AL) Y,
// with NY = -Y. The steps, and so every rounding, are those of df_acc: the
// product's error is fma(ah, y, -p) with -p = ah (-y) exact, and TwoSum's
// b - z is taken as -(z + (-p)).
__device__ __forceinline__ void df2_acc(f2x& S, f2x& C, f2x AH, f2x AL, f2x Y, f2x NY) {
    const f2x NP = f2mul(AH, NY);    // -p
    const f2x E = f2fma(AH, Y, NP);  // ah y - p, exactly
    const f2x S1 = f2sub(S, NP);     // s + p
    const f2x Z = f2sub(S1, S);
    const f2x T2 = f2sub(S, f2sub(S1, Z));
    const f2x T3 = f2add(Z, NP);     // -(p - z)
    const f2x T = f2sub(T2, T3);
    C = f2add(C, f2add(T, f2fma(AL, Y, E)));
    S = S1;
}

// df_acc1 on two accumulations: (S, C) += A Y (A binary32).
__device__ __forceinline__ void df2_acc1(f2x& S, f2x& C, f2x A, f2x Y, f2x NY) {
    const f2x NP = f2mul(A, NY);
    const f2x E = f2fma(A, Y, NP);
    const f2x S1 = f2sub(S, NP);
    const f2x Z = f2sub(S1, S);
    const f2x T2 = f2sub(S, f2sub(S1, Z));
    const f2x T3 = f2add(Z, NP);
    const f2x T = f2sub(T2, T3);
    C = f2add(C, f2add(T, E));
    S = S1;
}

}  // namespace
}  // namespace lbmgpu
