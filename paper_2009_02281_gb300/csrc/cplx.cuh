// Minimal complex helpers on float2 / double2 for device code.
#pragma once
#include <cuda_runtime.h>

#include "aimx_internal.h"

namespace aimx {

template <class T>
using cplx_t = typename Cplx<T>::type;

__host__ __device__ inline float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ inline double2 mk(double a, double b) { return make_double2(a, b); }

__host__ __device__ inline float2 operator+(float2 a, float2 b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 operator-(float2 a, float2 b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 operator*(float2 a, float2 b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 operator*(float s, float2 a) { return mk(s * a.x, s * a.y); }
__host__ __device__ inline float2 operator-(float2 a) { return mk(-a.x, -a.y); }
__host__ __device__ inline double2 operator+(double2 a, double2 b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 operator-(double2 a, double2 b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 operator*(double2 a, double2 b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 operator*(double s, double2 a) { return mk(s * a.x, s * a.y); }
__host__ __device__ inline double2 operator-(double2 a) { return mk(-a.x, -a.y); }
__host__ __device__ inline float2 conj(float2 a) { return mk(a.x, -a.y); }
__host__ __device__ inline double2 conj(double2 a) { return mk(a.x, -a.y); }

// a += b * c
__host__ __device__ inline void cfma(float2& a, float2 b, float2 c) {
    a.x = fmaf(b.x, c.x, a.x);
    a.x = fmaf(-b.y, c.y, a.x);
    a.y = fmaf(b.x, c.y, a.y);
    a.y = fmaf(b.y, c.x, a.y);
}
__host__ __device__ inline void cfma(double2& a, double2 b, double2 c) {
    a.x = fma(b.x, c.x, a.x);
    a.x = fma(-b.y, c.y, a.x);
    a.y = fma(b.x, c.y, a.y);
    a.y = fma(b.y, c.x, a.y);
}
// a += s * b (real s)
__host__ __device__ inline void rfma(float2& a, float s, float2 b) {
    a.x = fmaf(s, b.x, a.x);
    a.y = fmaf(s, b.y, a.y);
}
__host__ __device__ inline void rfma(double2& a, double s, double2 b) {
    a.x = fma(s, b.x, a.x);
    a.y = fma(s, b.y, a.y);
}

template <class T>
__host__ __device__ inline cplx_t<T> czero() {
    return mk(T(0), T(0));
}

}  // namespace aimx
