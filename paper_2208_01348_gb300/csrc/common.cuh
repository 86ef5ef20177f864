// Shared device helpers: complex arithmetic on float2/double2, precision
// traits and launch-error plumbing.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };
template <typename R> using cx = typename Cx<R>::T;

template <typename C> __host__ __device__ __forceinline__ C mk(double re, double im) {
    C c; c.x = (decltype(c.x))re; c.y = (decltype(c.y))im; return c;
}
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator*(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a) { return make_float2(-a.x, -a.y); }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator*(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a) { return make_double2(-a.x, -a.y); }

template <typename C> __host__ __device__ __forceinline__ C conj_(C a) { a.y = -a.y; return a; }
template <typename C> __host__ __device__ __forceinline__ auto abs2_(C a) { return a.x * a.x + a.y * a.y; }
// multiply by +i (INV=false gives -i): used by radix butterflies
template <typename C> __host__ __device__ __forceinline__ C mul_i(C a) { C r; r.x = -a.y; r.y = a.x; return r; }
template <typename C> __host__ __device__ __forceinline__ C mul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }

__host__ __device__ __forceinline__ float2 to_f(double2 a) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }
template <typename C> __host__ __device__ __forceinline__ C cvt(double2 a);
template <> __host__ __device__ __forceinline__ double2 cvt<double2>(double2 a) { return a; }
template <> __host__ __device__ __forceinline__ float2 cvt<float2>(double2 a) { return to_f(a); }
template <typename C> __host__ __device__ __forceinline__ double2 widen(C a) { return make_double2(a.x, a.y); }

__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    // Smith's algorithm
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, den = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
    } else {
        double r = b.x / b.y, den = b.x * r + b.y;
        return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
    }
}
__host__ __device__ __forceinline__ double cabs_(double2 a) { return hypot(a.x, a.y); }

// Fixed-size per-system scalars of the solve (device resident).
#define EELS_MAX_MAT 8
