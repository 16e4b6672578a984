// Vector loads and stores of V consecutive members (16-byte accesses for
// float4 / double2) shared by the lattice kernels. Internal header.
#pragma once
#include <cuda_runtime.h>

namespace lbmgpu {

template <typename T, int V>
struct Vec;
template <>
struct Vec<double, 1> {
    static __device__ __forceinline__ void ld(const double* p, double (&v)[1]) { v[0] = __ldg(p); }
    static __device__ __forceinline__ void st(double* p, const double (&v)[1]) { p[0] = v[0]; }
};
template <>
struct Vec<double, 2> {
    static __device__ __forceinline__ void ld(const double* p, double (&v)[2]) {
        double2 t = __ldg(reinterpret_cast<const double2*>(p));
        v[0] = t.x;
        v[1] = t.y;
    }
    static __device__ __forceinline__ void st(double* p, const double (&v)[2]) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    }
};
template <>
struct Vec<float, 1> {
    static __device__ __forceinline__ void ld(const float* p, float (&v)[1]) { v[0] = __ldg(p); }
    static __device__ __forceinline__ void st(float* p, const float (&v)[1]) { p[0] = v[0]; }
};
template <>
struct Vec<float, 2> {
    static __device__ __forceinline__ void ld(const float* p, float (&v)[2]) {
        float2 t = __ldg(reinterpret_cast<const float2*>(p));
        v[0] = t.x;
        v[1] = t.y;
    }
    static __device__ __forceinline__ void st(float* p, const float (&v)[2]) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    }
};
template <>
struct Vec<float, 4> {
    static __device__ __forceinline__ void ld(const float* p, float (&v)[4]) {
        float4 t = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    }
    static __device__ __forceinline__ void st(float* p, const float (&v)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};

// Work item t of a lattice kernel -> member group mv (of kv per cell), cell,
// and its coordinates (x, y). The divisions run in 32 bits while t fits
// (64-bit integer division is emulated and costs several times more).
__device__ __forceinline__ void split_item(long long t, int kv, int nx, int& mv, long long& cell, int& x,
                                           int& y) {
    if (t < 0x100000000LL) {
        const unsigned tt = (unsigned)t, ukv = (unsigned)kv, unx = (unsigned)nx;
        const unsigned c = tt / ukv;
        mv = (int)(tt - c * ukv);
        cell = c;
        const unsigned yy = c / unx;
        y = (int)yy;
        x = (int)(c - yy * unx);
    } else {
        mv = (int)(t % kv);
        cell = t / kv;
        x = (int)(cell % nx);
        y = (int)(cell / nx);
    }
}

}  // namespace lbmgpu
