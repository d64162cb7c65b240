// Whole-line FFTs held in one thread's registers (lengths 8..64).
//
// Decimation in time on a register array with compile-time indices: radix 4
// for lengths that are powers of four (16, 64), radix 2 otherwise.  The digit
// reversal is a renaming, twiddles W_L^k are compile-time constants (instruction
// immediates), and the trivial twiddles (1, -1, -i) are applied without
// multiplications.  Natural order in and out; INV gives the
// unnormalised inverse.
#pragma once

#include "cplx.cuh"

namespace aimx {

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }
__host__ __device__ constexpr int brevc(int v, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((v >> b) & 1) << (bits - 1 - b);
    return r;
}

// Twiddles as compile-time constants.  Every line length here divides 384 = 3 * 128 (powers
// of two up to 128 and 3 * 2^k up to 384), so all twiddles are W_384^k = e^{-2 pi i k / 384}.
// The angle is reduced exactly with integers to [0, pi/4] (quadrant, then the complementary
// angle), where Taylor series of sin and cos summed in double precision are accurate to
// rounding; FP32 lines round the table to FP32.  Indices are compile-time constants after
// unrolling, so the values become instruction immediates instead of constant-memory loads.
constexpr int kTwTab = 384;
__host__ __device__ constexpr double taylor_sin(double x) {
    double x2 = x * x, term = x, sum = x;
    for (int n = 1; n < 12; ++n) {
        term *= -x2 / ((2.0 * n) * (2.0 * n + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int n = 1; n < 12; ++n) {
        term *= -x2 / ((2.0 * n - 1.0) * (2.0 * n));
        sum += term;
    }
    return sum;
}
struct TwTable {
    double re[kTwTab];
    double im[kTwTab];
};
__host__ __device__ constexpr TwTable make_tw_table() {
    TwTable t{};
    constexpr double two_pi = 6.283185307179586476925286766559;
    for (int k = 0; k < kTwTab; ++k) {
        const int q = k / (kTwTab / 4), r = k % (kTwTab / 4);   // angle = q pi/2 + 2 pi r / 384
        double c0 = 0.0, s0 = 0.0;
        if (r <= kTwTab / 8) {
            const double a = two_pi * r / kTwTab;
            c0 = taylor_cos(a);
            s0 = taylor_sin(a);
        } else {                                                // pi/2 - angle, also in [0, pi/4]
            const double a = two_pi * (kTwTab / 4 - r) / kTwTab;
            c0 = taylor_sin(a);
            s0 = taylor_cos(a);
        }
        const double c = q == 0 ? c0 : q == 1 ? -s0 : q == 2 ? -c0 : s0;
        const double sn = q == 0 ? s0 : q == 1 ? c0 : q == 2 ? -s0 : -c0;
        t.re[k] = c;
        t.im[k] = -sn;
    }
    return t;
}

// W_M^k (forward) or its conjugate (inverse) for k and M compile-time constants after
// unrolling, M dividing 384
template <bool INV>
__device__ __forceinline__ float2 twc(int k, int M) {
    constexpr TwTable tab = make_tw_table();
    const int i = (k % M) * (kTwTab / M);
    return make_float2((float)tab.re[i], INV ? -(float)tab.im[i] : (float)tab.im[i]);
}
template <bool INV>
__device__ __forceinline__ double2 twc_d(int k, int M) {
    constexpr TwTable tab = make_tw_table();
    const int i = (k % M) * (kTwTab / M);
    return make_double2(tab.re[i], INV ? -tab.im[i] : tab.im[i]);
}
template <class C, bool INV>
__device__ __forceinline__ C tw_any(int k, int M) {
    if constexpr (sizeof(C) == sizeof(float2))
        return twc<INV>(k, M);
    else
        return twc_d<INV>(k, M);
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

// Packed two-lane sums on FP32 pairs (one sm_100+ instruction for both lanes).  The
// difference is an FMA with -1, which rounds exactly like the scalar subtraction.
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// Two radix-4 butterflies of one stage (span q) at once, lanes j (even) and j + 1 of
// group g: each lane's twiddles are applied in scalar form, then the sixteen sums run on
// (lane j, lane j + 1) pairs of real parts and of imaginary parts.  Same operations and
// rounding as two scalar butterflies, half the add instructions.
template <bool INV>
__device__ __forceinline__ void bfly4_pair(float2* v, int g, int j, int q) {
    float2 R[4], I[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const float2 l0 = tw_mul<INV>(v[g + j + m * q], m * j, 4 * q);
        const float2 l1 = tw_mul<INV>(v[g + j + 1 + m * q], m * (j + 1), 4 * q);
        R[m] = make_float2(l0.x, l1.x);
        I[m] = make_float2(l0.y, l1.y);
    }
    const float2 t0r = padd(R[0], R[2]), t0i = padd(I[0], I[2]);
    const float2 t1r = psub(R[0], R[2]), t1i = psub(I[0], I[2]);
    const float2 t2r = padd(R[1], R[3]), t2i = padd(I[1], I[3]);
    const float2 dr = psub(R[1], R[3]), di = psub(I[1], I[3]);
    // t3 = (-+i) d: forward (di, -dr), inverse (-di, dr)
    float2 oR[4], oI[4];
    oR[0] = padd(t0r, t2r);
    oI[0] = padd(t0i, t2i);
    oR[2] = psub(t0r, t2r);
    oI[2] = psub(t0i, t2i);
    if (INV) {
        oR[1] = psub(t1r, di);
        oI[1] = padd(t1i, dr);
        oR[3] = padd(t1r, di);
        oI[3] = psub(t1i, dr);
    } else {
        oR[1] = padd(t1r, di);
        oI[1] = psub(t1i, dr);
        oR[3] = psub(t1r, di);
        oI[3] = padd(t1i, dr);
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        v[g + j + m * q] = make_float2(oR[m].x, oI[m].x);
        v[g + j + 1 + m * q] = make_float2(oR[m].y, oI[m].y);
    }
}

// Radix-4 decimation in time for L a power of four: base-4 digit reversal as a
// renaming, then log4 L stages of radix-4 butterflies with three twiddles each
// (fewer multiplications than the radix-2 form).  Natural order in and out.  The
// first stage (span 1, no twiddles) runs on complex values; later stages pair
// neighbouring butterflies and run their sums as packed FP32x2 instructions.
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
    for (int g = 0; g < L; g += 4) {
        const float2 a0 = v[g], a1 = v[g + 1], a2 = v[g + 2], a3 = v[g + 3];
        const float2 t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3;
        const float2 d = a1 - a3;
        const float2 t3 = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
        v[g] = t0 + t2;
        v[g + 1] = t1 + t3;
        v[g + 2] = t0 - t2;
        v[g + 3] = t1 - t3;
    }
#pragma unroll
    for (int q = 4; q < L; q *= 4) {
#pragma unroll
        for (int g = 0; g < L; g += 4 * q) {
#pragma unroll
            for (int j = 0; j < q; j += 2) bfly4_pair<INV>(v, g, j, q);
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

// Whole-line register FFT of any length L = 2^k (k >= 1) or 3 * 2^k dividing 384, on float2
// or double2.  Lengths 3 P: the decimated sequences x[3 n + r] are transformed (length P)
// and recombined by one radix-3 pass, X[k + m P] = sum_r W_L^{r k} W_3^{r m} Y_r[k], whose
// cube roots of unity are -1/2 and +-(sqrt 3 / 2) i.  FP32 powers of two take reg_fft
// (radix 4, packed sums); FP64 powers of two a radix-2 decimation in time.  Natural order
// in and out; INV gives the unnormalised inverse.
template <class C, int L, bool INV>
__device__ __forceinline__ void reg_fft_any(C (&v)[L]) {
    using R = decltype(C{}.x);
    if constexpr (L == 1) {
        return;
    } else if constexpr (L % 3 == 0) {
        constexpr int P = L / 3;
        C y[3][P];
#pragma unroll
        for (int n = 0; n < P; ++n) {
            y[0][n] = v[3 * n];
            y[1][n] = v[3 * n + 1];
            y[2][n] = v[3 * n + 2];
        }
        reg_fft_any<C, P, INV>(y[0]);
        reg_fft_any<C, P, INV>(y[1]);
        reg_fft_any<C, P, INV>(y[2]);
        const R hs = (R)0.86602540378443864676;   // sqrt(3) / 2
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const C a = y[0][k];
            const C b = k ? y[1][k] * tw_any<C, INV>(k, L) : y[1][k];
            const C c = k ? y[2][k] * tw_any<C, INV>(2 * k, L) : y[2][k];
            const C t = b + c, d = b - c;
            const C m = a - (R)0.5 * t;
            const C jd = INV ? mk(-hs * d.y, hs * d.x) : mk(hs * d.y, -hs * d.x);
            v[k] = a + t;
            v[k + P] = m + jd;
            v[k + 2 * P] = m - jd;
        }
    } else if constexpr (sizeof(C) == sizeof(float2)) {
        reg_fft<L, INV>(v);
    } else {
        constexpr int LOG = ilog2c(L);
#pragma unroll
        for (int i = 0; i < L; ++i) {
            const int j = brevc(i, LOG);
            if (j > i) {
                const C t = v[i];
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
                    const C a = v[start + k];
                    C b = v[start + k + half];
                    if (k == 0) {
                    } else if (4 * k == 2 * half) {
                        b = INV ? mk(-b.y, b.x) : mk(b.y, -b.x);
                    } else {
                        b = b * tw_any<C, INV>(k, 2 * half);
                    }
                    v[start + k] = a + b;
                    v[start + k + half] = a - b;
                }
            }
        }
    }
}

}  // namespace aimx
