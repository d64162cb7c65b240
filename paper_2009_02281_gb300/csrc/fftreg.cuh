// Block-cooperative in-place mixed-radix FFTs on lines held in shared memory.
//
// Radix sequence for length L (power of two): 8, 8, ..., then 4 or 2.
// Two in-place forms are provided, so no stage needs a second buffer and
// every butterfly group is independent (one barrier per stage):
//
//   fft_dit : decimation in time.  Input must sit at dit_pos(n) (mixed-radix
//             digit reversal); output is in natural order.
//   fft_dif : decimation in frequency.  Input in natural order; output
//             X[k] sits at dif_pos(k).
//
// Loads and stores apply the digit reversal in their addressing, so no
// separate permutation pass is needed.  Twiddles come from the shared table
// e^{-2 pi i k / 4096}; INV selects the conjugate (unnormalised inverse).
#pragma once

#include "aimx_internal.h"
#include "cplx.cuh"

namespace aimx {

template <bool INV>
__device__ inline float2 rot_mj(float2 a) {  // multiply by -i (forward) or +i (inverse)
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// in-register DFT of size R, natural order in and out
template <int R, bool INV>
__device__ inline void dft(float2* v);

template <>
__device__ inline void dft<2, false>(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
}
template <>
__device__ inline void dft<2, true>(float2* v) {
    dft<2, false>(v);
}

template <bool INV>
__device__ inline void dft4(float2* v) {
    float2 a0 = v[0] + v[2], a2 = v[0] - v[2];
    float2 a1 = v[1] + v[3], a3 = rot_mj<INV>(v[1] - v[3]);
    v[0] = a0 + a1;
    v[2] = a0 - a1;
    v[1] = a2 + a3;
    v[3] = a2 - a3;
}
template <>
__device__ inline void dft<4, false>(float2* v) {
    dft4<false>(v);
}
template <>
__device__ inline void dft<4, true>(float2* v) {
    dft4<true>(v);
}

template <bool INV>
__device__ inline void dft8(float2* v) {
    const float h = 0.70710678118654752440f;
    float2 a0 = v[0] + v[4], b0 = v[0] - v[4];
    float2 a1 = v[1] + v[5], b1 = v[1] - v[5];
    float2 a2 = v[2] + v[6], b2 = v[2] - v[6];
    float2 a3 = v[3] + v[7], b3 = v[3] - v[7];
    // b_j *= W8^j  (W8 = e^{-i pi/4} forward, e^{+i pi/4} inverse)
    b1 = INV ? make_float2(h * (b1.x - b1.y), h * (b1.x + b1.y)) : make_float2(h * (b1.x + b1.y), h * (b1.y - b1.x));
    b2 = rot_mj<INV>(b2);
    b3 = INV ? make_float2(-h * (b3.x + b3.y), h * (b3.x - b3.y)) : make_float2(h * (b3.y - b3.x), -h * (b3.x + b3.y));
    float2 c0 = a0 + a2, c2 = a0 - a2, c1 = a1 + a3, c3 = rot_mj<INV>(a1 - a3);
    float2 d0 = b0 + b2, d2 = b0 - b2, d1 = b1 + b3, d3 = rot_mj<INV>(b1 - b3);
    v[0] = c0 + c1;
    v[4] = c0 - c1;
    v[2] = c2 + c3;
    v[6] = c2 - c3;
    v[1] = d0 + d1;
    v[5] = d0 - d1;
    v[3] = d2 + d3;
    v[7] = d2 - d3;
}
template <>
__device__ inline void dft<8, false>(float2* v) {
    dft8<false>(v);
}
template <>
__device__ inline void dft<8, true>(float2* v) {
    dft8<true>(v);
}

// radix of stage s (0-based) for length L: 8 while at least 8 remain, then the rest
__host__ __device__ inline int stage_radix(int L, int s) {
    int rem = L;
    for (int k = 0; k < s; ++k) rem /= (rem >= 8 ? 8 : rem);
    return rem >= 8 ? 8 : rem;
}
__host__ __device__ inline int num_stages(int L) {
    int n = 0;
    for (int rem = L; rem > 1; rem /= (rem >= 8 ? 8 : rem)) ++n;
    return n;
}

// DIT input slot of natural index n: digits of n from the least significant
// (radix of the last stage) to the most significant (radix of the first
// stage) become the digits of the slot from the most to the least significant.
__device__ inline int dit_pos(int n, int L) {
    const int m = num_stages(L);
    int p = 0, rest = n;
    int G[8];
    G[0] = 1;
    for (int s = 1; s < m; ++s) G[s] = G[s - 1] * stage_radix(L, s - 1);
    for (int s = m - 1; s >= 0; --s) {
        int R = stage_radix(L, s);
        int d = rest % R;
        rest /= R;
        p += d * G[s];
    }
    return p;
}

// DIF output slot of frequency k: k = q1 + Q1 (q2 + Q2 (...)), slot = sum q_s T_s
// with T_s = L / (Q1 ... Qs).
__device__ inline int dif_pos(int k, int L) {
    const int m = num_stages(L);
    int p = 0, rest = k, T = L;
    for (int s = 0; s < m; ++s) {
        int R = stage_radix(L, s);
        T /= R;
        p += (rest % R) * T;
        rest /= R;
    }
    return p;
}

template <int R, bool INV>
__device__ inline void dit_stage(float2* buf, int nlines, int lstride, int es, int L, int Gp,
                                 const float2* __restrict__ tw) {
    const int Q = L / R;
    const int G = Gp * R;
    const int tstep = kTwiddleTab / G;
    for (int item = threadIdx.x; item < nlines * Q; item += blockDim.x) {
        int line = item % nlines, j = item / nlines;
        int g = j / Gp, k = j - g * Gp;
        float2* b = buf + line * lstride + (g * G + k) * es;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 x = b[r * Gp * es];
            if (r > 0 && k > 0) {
                float2 w = __ldg(tw + r * k * tstep);
                if (INV) w.y = -w.y;
                x = x * w;
            }
            v[r] = x;
        }
        dft<R, INV>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) b[r * Gp * es] = v[r];
    }
    __syncthreads();
}

template <int R, bool INV>
__device__ inline void dif_stage(float2* buf, int nlines, int lstride, int es, int L, int T,
                                 const float2* __restrict__ tw) {
    const int Tn = T / R;
    const int Q = L / R;
    const int tstep = kTwiddleTab / T;
    for (int item = threadIdx.x; item < nlines * Q; item += blockDim.x) {
        int line = item % nlines, j = item / nlines;
        int blk = j / Tn, k = j - blk * Tn;
        float2* b = buf + line * lstride + (blk * T + k) * es;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = b[r * Tn * es];
        dft<R, INV>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 x = v[r];
            if (r > 0 && k > 0) {
                float2 w = __ldg(tw + r * k * tstep);
                if (INV) w.y = -w.y;
                x = x * w;
            }
            b[r * Tn * es] = x;
        }
    }
    __syncthreads();
}

// All threads of the block must call these.  Consecutive threads take
// consecutive lines, so strided (es > 1) transforms of adjacent lines read
// adjacent words.
template <bool INV>
__device__ inline void fft_dit(float2* buf, int nlines, int lstride, int es, int L,
                               const float2* __restrict__ tw) {
    const int m = num_stages(L);
    int Gp = 1;
    for (int s = 0; s < m; ++s) {
        int R = stage_radix(L, s);
        if (R == 8)
            dit_stage<8, INV>(buf, nlines, lstride, es, L, Gp, tw);
        else if (R == 4)
            dit_stage<4, INV>(buf, nlines, lstride, es, L, Gp, tw);
        else
            dit_stage<2, INV>(buf, nlines, lstride, es, L, Gp, tw);
        Gp *= R;
    }
}

template <bool INV>
__device__ inline void fft_dif(float2* buf, int nlines, int lstride, int es, int L,
                               const float2* __restrict__ tw) {
    const int m = num_stages(L);
    int T = L;
    for (int s = 0; s < m; ++s) {
        int R = stage_radix(L, s);
        if (R == 8)
            dif_stage<8, INV>(buf, nlines, lstride, es, L, T, tw);
        else if (R == 4)
            dif_stage<4, INV>(buf, nlines, lstride, es, L, T, tw);
        else
            dif_stage<2, INV>(buf, nlines, lstride, es, L, T, tw);
        T /= R;
    }
}

}  // namespace aimx
