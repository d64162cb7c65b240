// Whole-line FFTs held in one thread's registers (lengths 8..64).
//
// Radix-2 decimation in time on a register array with compile-time indices:
// the bit-reversal is a renaming, twiddles W_L^k come from a constant-memory
// table read at warp-uniform addresses, and the trivial twiddles (1 and -i)
// are applied without multiplications.  Natural order in and out; INV gives
// the unnormalised inverse.
#pragma once

#include "cplx.cuh"

namespace aimx {

// e^{-2 pi i k / 4096}, k < 4096; include this header in one translation unit
// only, which fills the table once per device before the first launch
static __constant__ float2 c_tw4096[4096];

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }
__host__ __device__ constexpr int brevc(int v, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((v >> b) & 1) << (bits - 1 - b);
    return r;
}

// W_M^k (forward) or its conjugate (inverse) for a compile-time or uniform k
template <bool INV>
__device__ __forceinline__ float2 twc(int k, int M) {
    float2 w = c_tw4096[(k % M) * (4096 / M)];
    if (INV) w.y = -w.y;
    return w;
}

__host__ __device__ constexpr bool pow4c(int v) { return v == 1 || (v % 4 == 0 && pow4c(v / 4)); }
__host__ __device__ constexpr int drev4c(int v, int digits) {
    int r = 0;
    for (int d = 0; d < digits; ++d) {
        r = r * 4 + (v & 3);
        v >>= 2;
    }
    return r;
}

// x * W_M^k (or its conjugate) for compile-time k < M, without multiplications when the
// twiddle is 1, -1 or -i (+i for the inverse)
template <bool INV>
__device__ __forceinline__ float2 tw_mul(float2 x, int k, int M) {
    if (k == 0) return x;
    if (2 * k == M) return make_float2(-x.x, -x.y);
    if (4 * k == M) return INV ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
    return x * twc<INV>(k, M);
}

// Radix-4 decimation in time for L a power of four: base-4 digit reversal as a
// renaming, then log4 L stages of radix-4 butterflies with three twiddles each
// (fewer multiplications than the radix-2 form).  Natural order in and out.
template <int L, bool INV>
__device__ __forceinline__ void reg_fft4(float2 (&v)[L]) {
    constexpr int D = ilog2c(L) / 2;
#pragma unroll
    for (int i = 0; i < L; ++i) {
        const int j = drev4c(i, D);
        if (j > i) {
            float2 t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    }
#pragma unroll
    for (int q = 1; q < L; q *= 4) {
#pragma unroll
        for (int g = 0; g < L; g += 4 * q) {
#pragma unroll
            for (int j = 0; j < q; ++j) {
                const float2 a0 = v[g + j];
                const float2 a1 = tw_mul<INV>(v[g + j + q], j, 4 * q);
                const float2 a2 = tw_mul<INV>(v[g + j + 2 * q], 2 * j, 4 * q);
                const float2 a3 = tw_mul<INV>(v[g + j + 3 * q], 3 * j, 4 * q);
                const float2 t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3;
                const float2 d = a1 - a3;
                const float2 t3 = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);   // (-+i)(a1 - a3)
                v[g + j] = t0 + t2;
                v[g + j + q] = t1 + t3;
                v[g + j + 2 * q] = t0 - t2;
                v[g + j + 3 * q] = t1 - t3;
            }
        }
    }
}

template <int L, bool INV>
__device__ __forceinline__ void reg_fft(float2 (&v)[L]) {
    if constexpr (L >= 16 && pow4c(L)) {
        reg_fft4<L, INV>(v);
        return;
    }
    constexpr int LOG = ilog2c(L);
#pragma unroll
    for (int i = 0; i < L; ++i) {
        const int j = brevc(i, LOG);
        if (j > i) {
            float2 t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    }
#pragma unroll
    for (int half = 1; half < L; half <<= 1) {
#pragma unroll
        for (int start = 0; start < L; start += 2 * half) {
#pragma unroll
            for (int k = 0; k < half; ++k) {
                float2 a = v[start + k];
                float2 b = v[start + k + half];
                if (k == 0) {
                } else if (4 * k == 2 * half) {
                    b = INV ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
                } else {
                    b = b * twc<INV>(k, 2 * half);
                }
                v[start + k] = a + b;
                v[start + k + half] = a - b;
            }
        }
    }
}

}  // namespace aimx
