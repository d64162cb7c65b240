// FP64 Krylov-vector kernels shared by the GMRES drivers (aimx_solve and the batched sweep).
// Right-hand sides are stored one after another (RHS-major); every kernel has internal linkage,
// so each translation unit that includes this header gets its own copy.
#pragma once

#include "aimx_internal.h"
#include "cplx.cuh"

namespace aimx {

// ------------------------------------------------------------------ vector kernels (FP64, RHS-major)

static __global__ void k_dots(const double2* __restrict__ V, const double2* __restrict__ w, double2* h, int nunk,
                       int64_t vstride, int ldh, int nvec) {
    // h[b * ldh + i] = sum_n conj(V[b][i][n]) w[b][n]; grid (nvec, nrhs)
    const int i = blockIdx.x, b = blockIdx.y;
    const double2* v = V + b * vstride + (int64_t)i * nunk;
    const double2* x = w + (int64_t)b * nunk;
    double re = 0.0, im = 0.0;
    for (int n = threadIdx.x; n < nunk; n += blockDim.x) {
        double2 a = v[n], c = x[n];
        re += a.x * c.x + a.y * c.y;
        im += a.x * c.y - a.y * c.x;
    }
    __shared__ double sr[32], si[32];
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sr[wid] = re;
        si[wid] = im;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        re = lane < nw ? sr[lane] : 0.0;
        im = lane < nw ? si[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_down_sync(0xffffffffu, re, o);
            im += __shfl_down_sync(0xffffffffu, im, o);
        }
        if (lane == 0) h[b * ldh + i] = make_double2(re, im);
    }
    (void)nvec;
}

// Segmented form of k_dots for the Arnoldi step: block (segment s, rhs b) holds
// its kDotSeg entries of w in registers (kDotSeg / 256 per thread) and streams
// the Krylov vectors four at a time, so w is read once per pass instead of once
// per vector; each warp writes its partial sums to
// part[((b * nseg + s) * 8 + warp) * ldp + i] (no block barriers; the final
// reduction runs in a fixed order, so the result is deterministic).
constexpr int kDotSeg = 2048;
constexpr int kDotPer = kDotSeg / 256;

static __global__ void __launch_bounds__(256) k_dots_seg(const double2* __restrict__ V, const double2* __restrict__ w,
                                                  double2* part, int nunk, int64_t vstride, int nvec, int nseg,
                                                  int ldp) {
    const int sg = blockIdx.x, b = blockIdx.y;
    const int n0 = sg * kDotSeg;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double2 xr[kDotPer];
#pragma unroll
    for (int k = 0; k < kDotPer; ++k) {
        const int n = n0 + threadIdx.x + 256 * k;
        xr[k] = n < nunk ? w[(int64_t)b * nunk + n] : make_double2(0.0, 0.0);
    }
    double2* pw = part + (((int64_t)b * nseg + sg) * 8 + wid) * ldp;
    for (int i0 = 0; i0 < nvec; i0 += 4) {
        double re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (i0 + t >= nvec) break;
            const double2* v = V + b * vstride + (int64_t)(i0 + t) * nunk;
#pragma unroll
            for (int k = 0; k < kDotPer; ++k) {
                const int n = n0 + threadIdx.x + 256 * k;
                if (n < nunk) {
                    const double2 a = v[n];
                    re[t] += a.x * xr[k].x + a.y * xr[k].y;
                    im[t] += a.x * xr[k].y - a.y * xr[k].x;
                }
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
            for (int o = 16; o > 0; o >>= 1) {
                re[t] += __shfl_down_sync(0xffffffffu, re[t], o);
                im[t] += __shfl_down_sync(0xffffffffu, im[t], o);
            }
        if (lane == 0)
            for (int t = 0; t < 4 && i0 + t < nvec; ++t) pw[i0 + t] = make_double2(re[t], im[t]);
    }
}

// h[b * ldh + i] = sum over segments and warps of part[((b * nseg + s) * 8 + warp) * ldp + i]
static __global__ void k_dots_fin(const double2* __restrict__ part, double2* h, int nvec, int nseg, int ldp, int ldh) {
    const int b = blockIdx.x;
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
        double2 t = make_double2(0.0, 0.0);
        for (int q = 0; q < nseg * 8; ++q) t = t + part[((int64_t)b * nseg * 8 + q) * ldp + i];
        h[b * ldh + i] = t;
    }
}

// w[b] -= sum_{i < nvec} h[b][i] V[b][i]
static __global__ void k_subtract(const double2* __restrict__ V, double2* w, const double2* __restrict__ h, int nunk,
                           int64_t vstride, int ldh, int nvec, int nrhs) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nunk * nrhs) return;
    const int b = (int)(t / nunk), n = (int)(t % nunk);
    // two independent accumulators (even / odd vectors) halve the dependent FP64 FMA chain
    double2 acc0 = w[t], acc1 = make_double2(0.0, 0.0);
    const double2* v = V + b * vstride + n;
    const double2* hb = h + b * ldh;
    int i = 0;
    for (; i + 1 < nvec; i += 2) {
        acc0 = acc0 - hb[i] * v[(int64_t)i * nunk];
        acc1 = acc1 - hb[i + 1] * v[(int64_t)(i + 1) * nunk];
    }
    if (i < nvec) acc0 = acc0 - hb[i] * v[(int64_t)i * nunk];
    w[t] = acc0 + acc1;
}

// y[b] = sum_{i < nvec} c[b][i] V[b][i]
static __global__ void k_combine(const double2* __restrict__ V, const double2* __restrict__ c, double2* y, int nunk,
                          int64_t vstride, int ldc, int nvec, int nrhs) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nunk * nrhs) return;
    const int b = (int)(t / nunk), n = (int)(t % nunk);
    double2 acc = make_double2(0, 0);
    const double2* v = V + b * vstride + n;
    for (int i = 0; i < nvec; ++i) acc = acc + c[b * ldc + i] * v[(int64_t)i * nunk];
    y[t] = acc;
}

static __global__ void k_norms(const double2* __restrict__ w, double* out, int nunk, int64_t stride) {
    const int b = blockIdx.x;
    const double2* x = w + b * stride;
    double s = 0.0;
    for (int n = threadIdx.x; n < nunk; n += blockDim.x) s += x[n].x * x[n].x + x[n].y * x[n].y;
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) out[b] = sqrt(s);
    }
}

// dst[b] = src[b] * scale[b] (scale[b] real); zero when scale[b] == 0
static __global__ void k_scale(const double2* __restrict__ src, double2* dst, const double* __restrict__ scale, int nunk,
                        int64_t sstride, int64_t dstride, int nrhs) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nunk * nrhs) return;
    const int b = (int)(t / nunk), n = (int)(t % nunk);
    dst[b * dstride + n] = scale[b] * src[b * sstride + n];
}

// r = b - y
static __global__ void k_residual(const double2* __restrict__ bv, const double2* __restrict__ y, double2* r, int64_t n) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) r[t] = bv[t] - y[t];
}

// x += d on active RHS
static __global__ void k_add_masked(double2* x, const double2* __restrict__ d, const int* __restrict__ active, int nunk,
                             int nrhs) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nunk * nrhs) return;
    if (active[t / nunk]) x[t] = x[t] + d[t];
}

// Preconditioner application z = M v (M: per-basis 1x1 or 2x2 inverse block), cast to FP32 or kept FP64.
template <class T>
static __global__ void k_precond(const double2* __restrict__ v, cplx_t<T>* z, const double2* __restrict__ minv0, int N,
                          int nunk, int nrhs, int form, int64_t vstride, const int* __restrict__ fidx = nullptr,
                          int64_t mstride = 0) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * nrhs) return;
    const int b = (int)(t / N), i = (int)(t % N);
    const double2* minv = fidx ? minv0 + fidx[b] * mstride : minv0;
    const double2* vb = v + (int64_t)b * vstride;
    cplx_t<T>* zb = z + (int64_t)b * nunk;
    if (form != AIMX_PMCHWT) {
        double2 r = minv[i] * vb[i];
        zb[i] = mk((T)r.x, (T)r.y);
    } else {
        const double2* m = minv + 4 * (int64_t)i;
        double2 a = vb[i], c = vb[N + i];
        double2 r0 = m[0] * a + m[1] * c, r1 = m[2] * a + m[3] * c;
        zb[i] = mk((T)r0.x, (T)r0.y);
        zb[N + i] = mk((T)r1.x, (T)r1.y);
    }
}

// in-place preconditioner on an FP64 vector (for the solution update)
static __global__ void k_precond_inplace(double2* v, const double2* __restrict__ minv0, int N, int nunk, int nrhs,
                                         int form, const int* __restrict__ fidx = nullptr, int64_t mstride = 0) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * nrhs) return;
    const int b = (int)(t / N), i = (int)(t % N);
    const double2* minv = fidx ? minv0 + fidx[b] * mstride : minv0;
    double2* vb = v + (int64_t)b * nunk;
    if (form != AIMX_PMCHWT) {
        vb[i] = minv[i] * vb[i];
    } else {
        const double2* m = minv + 4 * (int64_t)i;
        double2 a = vb[i], c = vb[N + i];
        vb[i] = m[0] * a + m[1] * c;
        vb[N + i] = m[2] * a + m[3] * c;
    }
}

static __global__ void k_f64_to_f32(const double2* __restrict__ a, float2* b, int64_t n) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) b[t] = make_float2((float)a[t].x, (float)a[t].y);
}

static __global__ void k_f32_to_f64(const float2* __restrict__ a, double2* b, int64_t n) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) b[t] = make_double2(a[t].x, a[t].y);
}

}  // namespace aimx
