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

template <int L, bool INV>
__device__ __forceinline__ void reg_fft(float2 (&v)[L]) {
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
