// FP32 AIMx matvec, plane-fused path for grids padded to exactly twice their
// size (M_a = 2 N_a, N_a a power of two).
//
// The zero-padded transform of a field that is non-zero only on the first
// N_a nodes of each axis splits by output parity p_a (k_a = 2 k'_a + p_a)
// into N-point transforms of the field twisted by e^{-2 pi i p_a n_a / M_a};
// the inverse recombines the parity classes with the conjugate twist, and
// only the N_a outputs on the grid are formed.  Pass structure:
//
//   k_transpose_x : x[b][n] -> xT[i][b] (internal basis order, RHS fastest)
//   k_gather_tile : projection P, node-major gather (no atomics) -> G[b][f][z][y][x]
//   k_xy_fwd      : per z plane: 4 parity classes (px, py), 2-D N-point FFT
//                   -> S[b][f][z][q][ky'][kx']
//   k_zpass       : per (kx', ky', q) column tile: zero-padded M_z FFT along z,
//                   per-point kernel multiply (Eq. LAIMx / KAIMx grid term),
//                   inverse, z < N_z kept -> S in place
//   k_xy_inv      : per z plane and field group: inverse 2-D FFT of the four
//                   parity classes, untwist, sum -> output plane in shared
//                   memory -> interpolation W = P^T partial per basis and slot
//   k_final       : per 32 bases: sum partials + near correction (BSR-free CSR
//                   rows, RHS vectorised) -> y
//
// Every sum has a fixed order, so results are bitwise reproducible.

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "aimx_internal.h"
#include "cplx.cuh"
#include "fftreg.cuh"
#include "regfft.cuh"

namespace aimx {

static inline bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

constexpr int kThreads = 256;
constexpr int kTX = 8;     // kx' columns per z-pass block
constexpr int kRG = 8;     // RHS per z-pass block (kernel spectra reuse)
constexpr int kFinalRows = 32;
constexpr int kFinalB = 64;

static bool reg_shape(const aimx_ctx* ctx);

bool fused_supported(const aimx_ctx* ctx) {
    if (ctx->form == AIMX_CFIE) return false;   // the CFIE's K_g interpolation runs on the generic path
    for (int a = 0; a < 3; ++a) {
        if (!pow2(ctx->n[a]) || ctx->M[a] != 2 * ctx->n[a] || ctx->n[a] < 2) return false;
    }
    const int Nx = ctx->n[0], Ny = ctx->n[1], Nz = ctx->n[2];
    if ((size_t)Nx * Ny * sizeof(float2) > 40 * 1024) return false;
    if (Nx < kTX) return false;
    if (Nx > 4096 || Ny > 4096 || 2 * Nz > 4096) return false;
    if ((size_t)ctx->F * kTX * (2 * Nz + 1) * sizeof(float2) > 96 * 1024) return false;
    if (kTX * 2 * Nz > 4 * kThreads) return false;
    // the shared-memory inverse kernel (schedule variant 1, or shapes without register kernels)
    // keeps a plane's bases in shared memory
    int mpb = 0;
    for (int z = 0; z < Nz; ++z) mpb = std::max(mpb, ctx->plane_hi[z] - ctx->plane_lo[z]);
    if ((size_t)mpb * sizeof(float2) > 64 * 1024 && !(reg_shape(ctx) && ctx->sched_variant != 1)) return false;
    return true;
}

__device__ inline float2 twist(const float2* __restrict__ tw, int p, int n, int M) {
    if (!p) return make_float2(1.f, 0.f);
    return __ldg(tw + (size_t)n * (kTwiddleTab / M));
}

// ------------------------------------------------------------------ K0
__global__ void k_transpose_x(const float2* __restrict__ x, const int* __restrict__ perm, float2* xT,
                              int N, int nunk, int B) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nunk * B) return;
    int b = (int)(t % B);
    int r = (int)(t / B);
    int blk = r / N, i = r - blk * N;
    xT[t] = x[(int64_t)b * nunk + blk * N + perm[i]];
}

// ------------------------------------------------------------------ K1
// Projection gather, tiled: a block covers 16 consecutive grid nodes x 32
// right-hand sides; lane = right-hand side, so the x reads ([nunk][B] layout)
// are contiguous and each node's (basis, weight) list is read once per warp as
// broadcasts; a shared-memory transpose writes the projected grid node-fastest.
// Charge form (tnode_ptr given): the rho field(s) are gathered from the triangle charges qT
// ([t][b] of J, then, two-region, of M at qT + qt_m) with the pulse weights instead of from the
// RWG divergence weights.
template <int F>
__global__ void __launch_bounds__(256) k_gather_tile(const float4* __restrict__ w, const int* __restrict__ node_ptr,
                                                     const int* __restrict__ node_w, const float2* __restrict__ xT,
                                                     float2* G, int B, int N, int U, int64_t NG,
                                                     const int* __restrict__ tnode_ptr, const int* __restrict__ tnode_w,
                                                     const float* __restrict__ lp, const float2* __restrict__ qT,
                                                     int64_t qt_m) {
    constexpr int TG = 16;
    __shared__ float2 tile[F][32][TG + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t g0 = (int64_t)blockIdx.x * TG;
    const int b0 = blockIdx.y * 32;
    const int b = b0 + lane;
    const bool bok = b < B;
    const int bc = bok ? b : B - 1;   // lanes past the last RHS compute a copy and store nothing
    for (int gl = warp; gl < TG; gl += 8) {
        const int64_t g = g0 + gl;
        float2 acc[F];
#pragma unroll
        for (int f = 0; f < F; ++f) acc[f] = make_float2(0.f, 0.f);
        if (g < NG) {   // warp-uniform
            const int e1 = node_ptr[g + 1];
            // the node's entries 32 at a time: each lane loads one entry index and its weights
            // (coalesced), then the warp walks them with shuffles, so the x gathers of several
            // entries are in flight together instead of waiting on an index-then-weight chain
            for (int e0 = node_ptr[g]; e0 < e1; e0 += 32) {
                const int cnt = min(32, e1 - e0);
                const int lwi = lane < cnt ? node_w[e0 + lane] : 0;
                const float4 lw = lane < cnt ? __ldg(w + lwi) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
                for (int m = 0; m < cnt; ++m) {
                    const int wi = __shfl_sync(0xffffffffu, lwi, m);
                    const float4 wv = make_float4(__shfl_sync(0xffffffffu, lw.x, m), __shfl_sync(0xffffffffu, lw.y, m),
                                                  __shfl_sync(0xffffffffu, lw.z, m), __shfl_sync(0xffffffffu, lw.w, m));
                    const int i = wi / U;
                    const float2 xj = __ldg(xT + (int64_t)i * B + bc);
                    rfma(acc[0], wv.x, xj);
                    rfma(acc[1], wv.y, xj);
                    rfma(acc[2], wv.z, xj);
                    if (!tnode_ptr) rfma(acc[3], wv.w, xj);
                    if (F == 8) {
                        const float2 xm = __ldg(xT + (int64_t)(N + i) * B + bc);
                        rfma(acc[4], wv.x, xm);
                        rfma(acc[5], wv.y, xm);
                        rfma(acc[6], wv.z, xm);
                        if (!tnode_ptr) rfma(acc[7], wv.w, xm);
                    }
                }
            }
            if (tnode_ptr) {
                // triangle charges of J (and, two-region, of M: the second nt x B block of qT)
                const int t1 = tnode_ptr[g + 1];
                for (int e = tnode_ptr[g]; e < t1; ++e) {
                    const int wt = tnode_w[e];
                    const float l = __ldg(lp + wt);
                    const int64_t qi = (int64_t)(wt / U) * B + bc;
                    rfma(acc[3], l, __ldg(qT + qi));
                    if (F == 8) rfma(acc[7], l, __ldg(qT + qt_m + qi));
                }
            }
        }
#pragma unroll
        for (int f = 0; f < F; ++f) tile[f][lane][gl] = acc[f];
    }
    __syncthreads();
    // rows (f, b): TG consecutive nodes each; 16 lanes per row, two rows per warp instruction
    const int half = lane >> 4, gl = lane & 15;
    for (int r = 2 * warp + half; r < F * 32; r += 16) {
        const int f = r / 32, bl = r % 32;
        const int bb = b0 + bl;
        const int64_t g = g0 + gl;
        if (bb < B && g < NG) G[((int64_t)bb * F + f) * NG + g] = tile[f][bl][gl];
    }
}

// ------------------------------------------------------------------ K2
// Shared-memory planes use a row pitch of Nx + 1 complex so that transforms of
// adjacent rows touch different banks.
__global__ void __launch_bounds__(kThreads) k_xy_fwd(const float2* __restrict__ G, float2* S, int F, int Nx,
                                                     int Ny, int Nz, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    const int NP = Nx * Ny;
    const int pitch = Nx + 1;
    float2* P = sm;                 // natural plane, pitch Nx
    float2* W = sm + NP;            // work plane, pitch Nx + 1
    const int z = blockIdx.x, f = blockIdx.y, b = blockIdx.z;
    const int64_t plane = ((int64_t)(b * F + f) * Nz + z);
    const float2* src = G + plane * NP;
    for (int i = threadIdx.x; i < NP; i += blockDim.x) P[i] = src[i];
    __syncthreads();
    const int Mx = 2 * Nx, My = 2 * Ny;
    for (int q = 0; q < 4; ++q) {
        const int px = q & 1, py = q >> 1;
        // twisted input, digit-reversed along x for the DIT row transform
        for (int i = threadIdx.x; i < NP; i += blockDim.x) {
            int y = i / Nx, x = i - y * Nx;
            float2 v = P[i];
            if (px) v = v * twist(tw, 1, x, Mx);
            if (py) v = v * twist(tw, 1, y, My);
            W[y * pitch + dit_pos(x, Nx)] = v;
        }
        __syncthreads();
        fft_dit<false>(W, Ny, pitch, 1, Nx, tw);     // rows: natural kx' out
        fft_dif<false>(W, Nx, 1, pitch, Ny, tw);     // columns: ky' at dif_pos
        float2* dst = S + (plane * 4 + q) * NP;
        for (int i = threadIdx.x; i < NP; i += blockDim.x) {
            int ky = i / Nx, kx = i - ky * Nx;
            dst[i] = W[dif_pos(ky, Ny) * pitch + kx];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ K3
// spectra layout: [nspec][Oz][Oy][Ox] complex, octant 0..M/2; fold and odd signs applied here
__global__ void __launch_bounds__(kThreads) k_zpass(float2* S, const float2* __restrict__ spec, int F, int Nx,
                                                    int Ny, int Nz, int B, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    const int Mz = 2 * Nz, Mx = 2 * Nx, My = 2 * Ny;
    const int lp = Mz + 1;          // line pitch
    const int NP = Nx * Ny;
    const int kx0 = blockIdx.x * kTX;
    const int kyp = blockIdx.y;
    const int q = blockIdx.z & 3;
    const int b0 = (blockIdx.z >> 2) * kRG;
    const int px = q & 1, py = q >> 1;
    const int nlines = F * kTX;
    const int Ox = Mx / 2 + 1, Oy = My / 2 + 1, Oz = Mz / 2 + 1;
    const int64_t OT = (int64_t)Ox * Oy * Oz;
    const int ky = 2 * kyp + py;
    const int oy = ky <= My / 2 ? ky : My - ky;
    const float sy = ky > My / 2 ? -1.f : 1.f;
    // mix points owned by this thread: (c, kz), at most 4 per thread (kTX * Mz <= 4 * kThreads)
    constexpr int KP = 4;
    const int ns = F == 4 ? 2 : 7;
    float2 sp[KP][7];
    const int npts = kTX * Mz;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        int pt = threadIdx.x + k * blockDim.x;
        if (pt < npts) {
            int c = pt % kTX, kz = pt / kTX;
            int kx = 2 * (kx0 + c) + px;
            int ox = kx <= Mx / 2 ? kx : Mx - kx;
            int oz = kz <= Mz / 2 ? kz : Mz - kz;
            int64_t oi = ((int64_t)oz * Oy + oy) * Ox + ox;
#pragma unroll
            for (int s = 0; s < 7; ++s) sp[k][s] = s < ns ? __ldg(spec + s * OT + oi) : make_float2(0.f, 0.f);
            if (F == 8) {
                if (kx > Mx / 2) sp[k][4] = -sp[k][4];
                sp[k][5] = sy * sp[k][5];
                if (kz > Mz / 2) sp[k][6] = -sp[k][6];
            }
        }
    }
    for (int bb = 0; bb < kRG; ++bb) {
        const int b = b0 + bb;
        if (b >= B) break;
        // load z < Nz of F * kTX columns (digit-reversed slots), zero the padding
        for (int idx = threadIdx.x; idx < nlines * Mz; idx += blockDim.x) {
            int c = idx % kTX;
            int rest = idx / kTX;
            int z = rest % Mz;
            int f = rest / Mz;
            float2 v = make_float2(0.f, 0.f);
            if (z < Nz) v = S[((((int64_t)b * F + f) * Nz + z) * 4 + q) * NP + (int64_t)kyp * Nx + kx0 + c];
            sm[(f * kTX + c) * lp + dit_pos(z, Mz)] = v;
        }
        __syncthreads();
        fft_dit<false>(sm, nlines, lp, 1, Mz, tw);
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            int pt = threadIdx.x + k * blockDim.x;
            if (pt < npts) {
                int c = pt % kTX, kz = pt / kTX;
                float2* g = sm + c * lp + kz;
                const int fs = kTX * lp;  // field stride
                if (F == 4) {
                    g[0] = sp[k][0] * g[0];
                    g[fs] = sp[k][0] * g[fs];
                    g[2 * fs] = sp[k][0] * g[2 * fs];
                    g[3 * fs] = sp[k][1] * g[3 * fs];
                } else {
                    float2 jx = g[0], jy = g[fs], jz = g[2 * fs], rj = g[3 * fs];
                    float2 mx = g[4 * fs], my = g[5 * fs], mz = g[6 * fs], rm = g[7 * fs];
                    float2 s1 = sp[k][0], s2 = sp[k][1], s3 = sp[k][2], s4 = sp[k][3];
                    float2 vx = sp[k][4], vy = sp[k][5], vz = sp[k][6];
                    g[0] = s1 * jx + (vy * mz - vz * my);
                    g[fs] = s1 * jy + (vz * mx - vx * mz);
                    g[2 * fs] = s1 * jz + (vx * my - vy * mx);
                    g[3 * fs] = s2 * rj;
                    g[4 * fs] = s3 * mx - (vy * jz - vz * jy);
                    g[5 * fs] = s3 * my - (vz * jx - vx * jz);
                    g[6 * fs] = s3 * mz - (vx * jy - vy * jx);
                    g[7 * fs] = s4 * rm;
                }
            }
        }
        __syncthreads();
        fft_dif<true>(sm, nlines, lp, 1, Mz, tw);
        for (int idx = threadIdx.x; idx < nlines * Nz; idx += blockDim.x) {
            int c = idx % kTX;
            int rest = idx / kTX;
            int z = rest % Nz;
            int f = rest / Nz;
            S[((((int64_t)b * F + f) * Nz + z) * 4 + q) * NP + (int64_t)kyp * Nx + kx0 + c] =
                sm[(f * kTX + c) * lp + dif_pos(z, Mz)];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ K4
__global__ void __launch_bounds__(kThreads) k_xy_inv(const float2* __restrict__ S, const float* __restrict__ w,
                                                     const int* __restrict__ anc, const int* __restrict__ plane_lo,
                                                     const int* __restrict__ plane_hi, float2* part, int F, int Nx,
                                                     int Ny, int Nz, int N, int P, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    const int NP = Nx * Ny;
    const int pitch = Nx + 1;
    float2* O = sm;                     // output plane, pitch Nx
    float2* W = sm + NP;                // work plane, pitch Nx + 1
    float2* acc = sm + NP + Ny * pitch;
    const int z = blockIdx.x, grp = blockIdx.y, b = blockIdx.z;
    const int G = F / 4;
    const int lo = plane_lo[z], hi = plane_hi[z];
    const int nb = hi - lo;
    const int Mx = 2 * Nx, My = 2 * Ny;
    const int U = P * P * P;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) acc[k] = make_float2(0.f, 0.f);
    for (int fl = 0; fl < 4; ++fl) {
        const int f = grp * 4 + fl;
        const int64_t plane = ((int64_t)(b * F + f) * Nz + z);
        for (int q = 0; q < 4; ++q) {
            const int px = q & 1, py = q >> 1;
            const float2* src = S + (plane * 4 + q) * NP;
            for (int i = threadIdx.x; i < NP; i += blockDim.x) {
                int ky = i / Nx, kx = i - ky * Nx;
                W[ky * pitch + kx] = src[i];
            }
            __syncthreads();
            fft_dif<true>(W, Nx, 1, pitch, Ny, tw);   // columns: y at dif_pos
            fft_dif<true>(W, Ny, pitch, 1, Nx, tw);   // rows: x at dif_pos
            for (int i = threadIdx.x; i < NP; i += blockDim.x) {
                int y = i / Nx, x = i - y * Nx;
                float2 v = W[dif_pos(y, Ny) * pitch + dif_pos(x, Nx)];
                if (px) v = v * conj(twist(tw, 1, x, Mx));
                if (py) v = v * conj(twist(tw, 1, y, My));
                O[i] = q == 0 ? v : O[i] + v;
            }
            __syncthreads();
        }
        // interpolation partial of field f for the bases touching this plane
        for (int k = threadIdx.x; k < nb; k += blockDim.x) {
            int i = lo + k;
            int sx = anc[3 * i], sy = anc[3 * i + 1], sz = anc[3 * i + 2];
            int slot = z - sz;
            const float* wi = w + ((int64_t)i * U + slot * P * P) * 4 + fl;
            float2 s = make_float2(0.f, 0.f);
            for (int uy = 0; uy < P; ++uy)
                for (int ux = 0; ux < P; ++ux) rfma(s, __ldg(wi + (uy * P + ux) * 4), O[(sy + uy) * Nx + sx + ux]);
            acc[k] = acc[k] + s;
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        int i = lo + k;
        int slot = z - anc[3 * i + 2];
        part[(((int64_t)b * G + grp) * P + slot) * N + i] = acc[k];
    }
}

// ------------------------------------------------------------------ K5
struct NearC {
    float2 c[6];
    float2 lin[4];   // linear-term coefficients (J rows: A, Phi; M rows: A, Phi)
    float2 cphi;     // charge form: coefficient of the triangle near part (c[1] is then 0)
    float2 cphi2;    // two-region charge form: the same for the M rows (c[5] is then 0)
};

__global__ void __launch_bounds__(kThreads) k_final(const float2* __restrict__ part, const float2* __restrict__ xT,
                                                    const int* __restrict__ row_ptr, const int* __restrict__ cols,
                                                    const float* __restrict__ na, const float* __restrict__ np,
                                                    const float* __restrict__ nk, const int* __restrict__ perm,
                                                    const int* __restrict__ lin_ptr, const int* __restrict__ lin_cols,
                                                    const float* __restrict__ la, const float* __restrict__ lp,
                                                    const float2* __restrict__ zn, float2* y, NearC nc, int F, int N,
                                                    int nunk, int P, int B, const float2* __restrict__ phiT,
                                                    const int* __restrict__ btri_t, const double* __restrict__ blen,
                                                    int64_t pt_m) {
    __shared__ float2 accE[kFinalRows][kFinalB];
    __shared__ float2 accH[kFinalRows][kFinalB];
    const int G = F / 4;
    const int i0 = blockIdx.x * kFinalRows;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int bc = 0; bc < B; bc += kFinalB) {
        const int nbc = min(kFinalB, B - bc);
        // partial sums over slots
        for (int idx = threadIdx.x; idx < G * nbc * kFinalRows; idx += blockDim.x) {
            int r = idx % kFinalRows;
            int rest = idx / kFinalRows;
            int bl = rest % nbc;
            int g = rest / nbc;
            int i = i0 + r;
            float2 s = make_float2(0.f, 0.f);
            if (i < N)
                for (int sl = 0; sl < P; ++sl) s = s + part[(((int64_t)(bc + bl) * G + g) * P + sl) * N + i];
            if (g == 0)
                accE[r][bl] = s;
            else
                accH[r][bl] = s;
        }
        __syncthreads();
        for (int r = warp; r < kFinalRows; r += nwarps) {
            int i = i0 + r;
            if (i >= N) continue;
            if (lin_ptr) {
                // linear-term modification: a few overlapping pairs per row, added to this
                // lane's own partial sums before the near correction
                const int l1 = lin_ptr[i + 1];
                for (int e = lin_ptr[i]; e < l1; ++e) {
                    const int j = lin_cols[e];
                    const float va = __ldg(la + e), vp = __ldg(lp + e);
                    const float2 cJ = va * nc.lin[0] + vp * nc.lin[1];
                    const float2 cM = va * nc.lin[2] + vp * nc.lin[3];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        int bl = lane + 32 * h;
                        if (bl < nbc) {
                            accE[r][bl] = accE[r][bl] + cJ * __ldg(xT + (int64_t)j * B + bc + bl);
                            if (F == 8) accH[r][bl] = accH[r][bl] + cM * __ldg(xT + (int64_t)(N + j) * B + bc + bl);
                        }
                    }
                }
            }
            float2 aJ[2], pJ[2], kJ[2], aM[2], pM[2], kM[2];
            for (int h = 0; h < 2; ++h) aJ[h] = pJ[h] = kJ[h] = aM[h] = pM[h] = kM[h] = make_float2(0.f, 0.f);
            const int e1 = row_ptr[i + 1];
            if (zn) {
                // conventional-AIM mode (EFIE): complex per-frequency entries, coefficient folded in
                for (int e = row_ptr[i]; e < e1; ++e) {
                    const int j = cols[e];
                    const float2 z = __ldg(zn + e);
                    const float vk = nk ? __ldg(nk + e) : 0.f;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        int bl = lane + 32 * h;
                        if (bl < nbc) {
                            float2 xj = __ldg(xT + (int64_t)j * B + bc + bl);
                            cfma(aJ[h], z, xj);
                            if (nk) rfma(kJ[h], vk, xj);
                        }
                    }
                }
            } else
            for (int e = row_ptr[i]; e < e1; ++e) {
                int j = cols[e];
                float va = __ldg(na + e), vp = __ldg(np + e);
                float vk = nk ? __ldg(nk + e) : 0.f;   // N^K (two-region) or the Gram matrix (EFIE + SIBC)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    int bl = lane + 32 * h;
                    if (bl < nbc) {
                        float2 xj = __ldg(xT + (int64_t)j * B + bc + bl);
                        rfma(aJ[h], va, xj);
                        rfma(pJ[h], vp, xj);
                        if (F == 8) {
                            float2 xm = __ldg(xT + (int64_t)(N + j) * B + bc + bl);
                            rfma(kJ[h], vk, xj);
                            rfma(aM[h], va, xm);
                            rfma(pM[h], vp, xm);
                            rfma(kM[h], vk, xm);
                        } else if (nk) {
                            rfma(kJ[h], vk, xj);
                        }
                    }
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int bl = lane + 32 * h;
                if (bl < nbc) {
                    float2 e = accE[r][bl] + nc.c[0] * aJ[h] + nc.c[1] * pJ[h];
                    if (F == 4 && nk) e = e + nc.c[2] * kJ[h];
                    const int64_t tp = phiT ? (int64_t)btri_t[2 * i] * B + bc + bl : 0;
                    const int64_t tm = phiT ? (int64_t)btri_t[2 * i + 1] * B + bc + bl : 0;
                    if (phiT) e = e + (float)blen[i] * (__ldg(phiT + tp) - __ldg(phiT + tm));
                    if (F == 8) {
                        e = e + nc.c[2] * kM[h];
                        float2 hh = accH[r][bl] + nc.c[3] * kJ[h] + nc.c[4] * aM[h] + nc.c[5] * pM[h];
                        if (phiT) hh = hh + (float)blen[i] * (__ldg(phiT + pt_m + tp) - __ldg(phiT + pt_m + tm));
                        y[(int64_t)(bc + bl) * nunk + N + perm[i]] = hh;
                    }
                    y[(int64_t)(bc + bl) * nunk + perm[i]] = e;
                }
            }
        }
        __syncthreads();
    }
}

// K5, blocked form: the near correction of Eq. LAIMx (L_s,NR - L_s,P applied to x, Sec. III-A) for
// a block of <= 32 anchor-sorted rows whose near columns, taken together, form a union of at most
// a few hundred bases.  For each chunk of 32 right-hand sides (lane = RHS) and each unknown block
// (J, then M), the block stages x of every union column once in shared memory; each warp then
// walks its rows' CSR entries (one broadcast 16-byte load of local column and the three static
// values per entry) and reads x from shared memory instead of gathering it from L2 per entry.
// Sums run in CSR order per row, so results are bitwise reproducible.
constexpr int kNbRows = 32;        // rows per block at most
constexpr int kNbWarps = 16;
constexpr int kNbUmax = 448;       // target column union per block

template <int F, bool SPLIT>
__global__ void __launch_bounds__(kNbWarps * 32) k_near_blk(
    const float2* __restrict__ part, const float2* __restrict__ xT, const int* __restrict__ nb_rows,
    const int* __restrict__ nb_ustart, const int* __restrict__ nb_ucols, const float4* __restrict__ ent,
    const int* __restrict__ row_ptr, const int* __restrict__ perm, const int* __restrict__ lin_ptr,
    const int* __restrict__ lin_cols, const float* __restrict__ la, const float* __restrict__ lp, float2* y,
    NearC nc, int has_k, int N, int nunk, int P, int B, const float2* __restrict__ phiT,
    const int* __restrict__ btri_t, const double* __restrict__ blen, int64_t pt_m) {
    extern __shared__ float2 xs[];                         // [union][32]
    __shared__ float2 accE[kNbRows][32];
    __shared__ float2 accH[F == 8 ? kNbRows : 1][32];
    __shared__ float4 ebuf[kNbWarps][32];                  // per-warp entry staging
    constexpr int G = F / 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = nb_rows[blockIdx.x], nr = nb_rows[blockIdx.x + 1] - r0;
    const int u0 = nb_ustart[blockIdx.x], nu = nb_ustart[blockIdx.x + 1] - u0;
    for (int bc = 0; bc < B; bc += 32) {
        const int nbc = min(32, B - bc);
        // SPLIT (at most 16 RHS, instantiated separately so the wide form is unchanged): RB >= nbc
        // RHS lanes, and 32 / RB lane groups each take every (32 / RB)-th entry of a row, so the
        // warp applies several entries at once when the RHS fill only part of it
        int RB = 32;
        if (SPLIT)
            for (RB = 1; RB < nbc; RB <<= 1) {
            }
        const int ngrp = 32 / RB, gsub = lane / RB, rl = lane % RB;
        // interpolation partials summed over the stencil slots, rows fastest (coalesced)
        for (int idx = threadIdx.x; idx < G * 32 * kNbRows; idx += blockDim.x) {
            const int r = idx % kNbRows, rest = idx / kNbRows;
            const int bl = rest % 32, g = rest / 32;
            float2 s = make_float2(0.f, 0.f);
            if (r < nr && bl < nbc)
                for (int sl = 0; sl < P; ++sl) s = s + part[(((int64_t)(bc + bl) * G + g) * P + sl) * N + r0 + r];
            if (g == 0)
                accE[r][bl] = s;
            else if (F == 8)
                accH[r][bl] = s;
        }
        // accumulators per row slot: J block (A, Phi, K) then M block (A, Phi, K)
        float2 acc[2][6];
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int m = 0; m < 6; ++m) acc[k][m] = make_float2(0.f, 0.f);
#pragma unroll
        for (int ph = 0; ph < G; ++ph) {
            __syncthreads();                              // xs free (and accE / accH written)
            for (int u = warp; u < nu; u += kNbWarps)
                xs[u * 32 + lane] =
                    lane < nbc ? __ldg(xT + ((int64_t)ph * N + nb_ucols[u0 + u]) * B + bc + lane) : make_float2(0.f, 0.f);
            __syncthreads();
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int r = warp + k * kNbWarps;
                if (r >= nr) continue;   // warp-uniform
                const int eb = row_ptr[r0 + r], e1 = row_ptr[r0 + r + 1];
                float2 a = make_float2(0.f, 0.f), p = a, q = a;
                // entries 32 at a time: one coalesced load per lane into this warp's buffer, the
                // next 32 loaded while the current ones are applied
                float4 nxt = eb + lane < e1 ? __ldg(ent + eb + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
                for (int e0 = eb; e0 < e1; e0 += 32) {
                    __syncwarp();
                    ebuf[warp][lane] = nxt;
                    __syncwarp();
                    if (e0 + 32 + lane < e1) nxt = __ldg(ent + e0 + 32 + lane);
                    const int cnt = min(32, e1 - e0);
#pragma unroll 4
                    for (int m = gsub; m < cnt; m += ngrp) {
                        const float4 t = ebuf[warp][m];
                        const float2 xv = xs[__float_as_int(t.x) * 32 + rl];
                        rfma(a, t.y, xv);
                        rfma(p, t.z, xv);
                        rfma(q, t.w, xv);
                    }
                }
                // combine the entry groups (butterfly: every lane of a RHS ends with the same sum)
                for (int off = RB; off < 32; off <<= 1) {
                    a.x += __shfl_xor_sync(0xffffffffu, a.x, off);
                    a.y += __shfl_xor_sync(0xffffffffu, a.y, off);
                    p.x += __shfl_xor_sync(0xffffffffu, p.x, off);
                    p.y += __shfl_xor_sync(0xffffffffu, p.y, off);
                    q.x += __shfl_xor_sync(0xffffffffu, q.x, off);
                    q.y += __shfl_xor_sync(0xffffffffu, q.y, off);
                }
                acc[k][3 * ph] = a;
                acc[k][3 * ph + 1] = p;
                acc[k][3 * ph + 2] = q;
            }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int r = warp + k * kNbWarps;
            if (r >= nr || lane >= nbc) continue;
            const int i = r0 + r;
            float2 e = accE[r][lane] + nc.c[0] * acc[k][0] + nc.c[1] * acc[k][1];
            float2 h = make_float2(0.f, 0.f);
            if (F == 4 && has_k) e = e + nc.c[2] * acc[k][2];
            if (F == 8) {
                e = e + nc.c[2] * acc[k][5];
                h = accH[r][lane] + nc.c[3] * acc[k][2] + nc.c[4] * acc[k][3] + nc.c[5] * acc[k][4];
            }
            if (phiT) {
                // charge form: D^T phi, phi the triangle potentials (nc.c[1] = 0 drops N^Phi; two
                // regions: the M rows' potentials follow at phiT + nt B and nc.c[5] = 0)
                const int64_t tp = (int64_t)btri_t[2 * i] * B + bc + lane, tm = (int64_t)btri_t[2 * i + 1] * B + bc + lane;
                e = e + (float)blen[i] * (__ldg(phiT + tp) - __ldg(phiT + tm));
                if (F == 8) h = h + (float)blen[i] * (__ldg(phiT + pt_m + tp) - __ldg(phiT + pt_m + tm));
            }
            if (lin_ptr) {
                // linear-term modification: a few overlapping pairs per row
                const int l1 = lin_ptr[i + 1];
                for (int le = lin_ptr[i]; le < l1; ++le) {
                    const int j = lin_cols[le];
                    const float va = __ldg(la + le), vp = __ldg(lp + le);
                    e = e + (va * nc.lin[0] + vp * nc.lin[1]) * __ldg(xT + (int64_t)j * B + bc + lane);
                    if (F == 8) h = h + (va * nc.lin[2] + vp * nc.lin[3]) * __ldg(xT + (int64_t)(N + j) * B + bc + lane);
                }
            }
            y[(int64_t)(bc + lane) * nunk + perm[i]] = e;
            if (F == 8) y[(int64_t)(bc + lane) * nunk + N + perm[i]] = h;
        }
        __syncthreads();                                  // accE / accH reused by the next chunk
    }
}

// entries of the blocked near kernel: union-local column and the three static values
__global__ void k_pack_near_ent(const int* __restrict__ li, const float* __restrict__ na,
                                const float* __restrict__ np, const float* __restrict__ nk, int64_t nnz,
                                float4* ent) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    ent[e] = make_float4(__int_as_float(li[e]), na[e], np[e], nk ? nk[e] : 0.f);
}

// ------------------------------------------------------------------ register-FFT kernels
// Square planes Nx = Ny = N <= 64 and Nz <= 64: every line transform runs in
// one thread's registers; shared memory only carries the transposes.

// K2 (register form): thread (px, r) transforms row r for parity px, then
// column r for both y parities; output block q = px + 2 py.
template <int N>
__global__ void __launch_bounds__(2 * N) k_xy_fwd_reg(const float2* __restrict__ G, float2* S, int F, int Nz) {
    extern __shared__ float2 sm[];
    constexpr int PITCH = N + 1;
    const int z = blockIdx.x, f = blockIdx.y, b = blockIdx.z;
    const int px = threadIdx.x / N, r = threadIdx.x - px * N;
    float2* pl = sm + px * N * PITCH;
    const int64_t plane = ((int64_t)(b * F + f) * Nz + z);
    const float2* src = G + plane * N * N + (int64_t)r * N;
    float2 v[N];
#pragma unroll
    for (int x = 0; x < N; x += 2) {
        float4 t = __ldg(reinterpret_cast<const float4*>(src + x));
        v[x] = make_float2(t.x, t.y);
        v[x + 1] = make_float2(t.z, t.w);
    }
    if (px) {
#pragma unroll
        for (int x = 1; x < N; ++x) v[x] = v[x] * twc<false>(x, 2 * N);
    }
    reg_fft<N, false>(v);
#pragma unroll
    for (int k = 0; k < N; ++k) pl[r * PITCH + k] = v[k];
    __syncthreads();
#pragma unroll 1
    for (int py = 0; py < 2; ++py) {
#pragma unroll
        for (int y = 0; y < N; ++y) {
            float2 c = pl[y * PITCH + r];
            if (py && y) c = c * twc<false>(y, 2 * N);
            v[y] = c;
        }
        reg_fft<N, false>(v);
        float2* dst = S + (plane * 4 + (px + 2 * py)) * N * N + r;
#pragma unroll
        for (int ky = 0; ky < N; ++ky) dst[ky * N] = v[ky];
    }
}

// K3 (register form): thread pair (pz = 0, 1) per (field, column) computes the
// even / odd halves of the zero-padded 2 NZ transform, shared memory carries
// the per-point mix across fields and the final even + odd sum.
// One z-pass tile (TC columns of all F fields, both z parities) once each thread holds its
// column in v: forward transform, spectral multiply across the fields, inverse transform,
// and the even + odd sum written back to S.
template <int NZ, int F>
__device__ __forceinline__ void zpass_tile(float2 (&v)[NZ], float2* sm, float2* S, const float2* __restrict__ spec,
                                           int Nx, int Ny, int kx0, int kyp, int q, int c, int f, int pz,
                                           int64_t base, int64_t zs) {
    constexpr int TC = 8;
    constexpr int MZ = 2 * NZ;
    constexpr int LP = MZ + 2;       // line pitch: adjacent columns 2 banks apart
    constexpr int FS = TC * LP + 1;  // field stride: adjacent fields 1 bank apart
    const int Mx = 2 * Nx, My = 2 * Ny;
    const int px = q & 1, py = q >> 1;
    float2* line = sm + f * FS + c * LP;
    if (pz) {
#pragma unroll
        for (int z = 1; z < NZ; ++z) v[z] = v[z] * twc<false>(z, MZ);
    }
    reg_fft<NZ, false>(v);
#pragma unroll
    for (int k = 0; k < NZ; ++k) line[2 * k + pz] = v[k];     // spectral index kz = 2k + pz
    __syncthreads();
    // mix at (column, kz)
    const int Ox = Mx / 2 + 1, Oy = My / 2 + 1, Oz = MZ / 2 + 1;
    // spectra hold at most 8 arrays of 65^3 points and a column spans at most 64 planes of
    // 4 x 64 x 64 points: 32-bit offsets (fewer index instructions than 64-bit ones)
    const int OT = Ox * Oy * Oz;
    const int ky = 2 * kyp + py;
    const int oy = ky <= My / 2 ? ky : My - ky;
    // compile-time trip count (blockDim.x = 2 F TC divides TC MZ): the loop unrolls and every
    // point's spectrum loads issue together instead of one L2 round trip per point
    constexpr int NT = 2 * F * TC;
    static_assert((TC * MZ) % NT == 0, "mix points must split evenly over the block");
#pragma unroll
    for (int it = 0; it < TC * MZ / NT; ++it) {
        const int pt = threadIdx.x + it * NT;
        const int cc = pt % TC, kz = pt / TC;
        const int kx = 2 * (kx0 + cc) + px;
        const int ox = kx <= Mx / 2 ? kx : Mx - kx;
        const int oz = kz <= MZ / 2 ? kz : MZ - kz;
        const int oi = (oz * Oy + oy) * Ox + ox;
        float2* g = sm + cc * LP + kz;
        constexpr int fs = FS;
        if (F == 4) {
            const float2 s1 = __ldg(spec + oi), s2 = __ldg(spec + OT + oi);
            g[0] = s1 * g[0];
            g[fs] = s1 * g[fs];
            g[2 * fs] = s1 * g[2 * fs];
            g[3 * fs] = s2 * g[3 * fs];
        } else {
            const float2 s1 = __ldg(spec + oi), s2 = __ldg(spec + OT + oi), s3 = __ldg(spec + 2 * OT + oi),
                         s4 = __ldg(spec + 3 * OT + oi);
            float2 vx = __ldg(spec + 4 * OT + oi), vy = __ldg(spec + 5 * OT + oi), vz = __ldg(spec + 6 * OT + oi);
            if (kx > Mx / 2) vx = -vx;
            if (ky > My / 2) vy = -vy;
            if (kz > MZ / 2) vz = -vz;
            float2 jx = g[0], jy = g[fs], jz = g[2 * fs], rj = g[3 * fs];
            float2 mx = g[4 * fs], my = g[5 * fs], mz = g[6 * fs], rm = g[7 * fs];
            g[0] = s1 * jx + (vy * mz - vz * my);
            g[fs] = s1 * jy + (vz * mx - vx * mz);
            g[2 * fs] = s1 * jz + (vx * my - vy * mx);
            g[3 * fs] = s2 * rj;
            g[4 * fs] = s3 * mx - (vy * jz - vz * jy);
            g[5 * fs] = s3 * my - (vz * jx - vx * jz);
            g[6 * fs] = s3 * mz - (vx * jy - vy * jx);
            g[7 * fs] = s4 * rm;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NZ; ++k) v[k] = line[2 * k + pz];
    reg_fft<NZ, true>(v);
    if (pz) {
#pragma unroll
        for (int z = 1; z < NZ; ++z) v[z] = v[z] * twc<true>(z, MZ);
    }
    __syncthreads();
    if (pz) {
#pragma unroll
        for (int z = 0; z < NZ; ++z) line[z] = v[z];
    }
    __syncthreads();
    if (!pz) {
        float2* col = S + base;
        const int zs32 = (int)zs;
#pragma unroll
        for (int z = 0; z < NZ; ++z) col[z * zs32] = v[z] + line[z];
    }
}

template <int NZ, int F>
__global__ void __launch_bounds__(2 * F * 8) k_zpass_reg(float2* S, const float2* __restrict__ spec, int Nx,
                                                             int Ny, int B) {
    extern __shared__ float2 sm[];
    constexpr int TC = 8;
    const int NP = Nx * Ny;
    const int kx0 = blockIdx.x * TC, kyp = blockIdx.y;
    const int q = blockIdx.z & 3, b = blockIdx.z >> 2;
    const int c = threadIdx.x % TC;
    const int f = (threadIdx.x / TC) % F;
    const int pz = threadIdx.x / (TC * F);
    const int64_t zs = 4 * (int64_t)NP;
    const int64_t base = (((int64_t)b * F + f) * NZ * 4 + q) * NP + (int64_t)kyp * Nx + kx0 + c;
    float2 v[NZ];
    const float2* col = S + base;
    const int zs32 = (int)zs;   // (NZ - 1) zs <= 63 * 4 * 64 * 64 < 2^31
#pragma unroll
    for (int z = 0; z < NZ; ++z) v[z] = col[z * zs32];
    zpass_tile<NZ, F>(v, sm, S, spec, Nx, Ny, kx0, kyp, q, c, f, pz, base, zs);
}

// ------------------------------------------------------------------ K3, TMA-pipelined form
// A persistent form of the register z-pass: each block walks the tiles with a
// stride of the grid size, and while it transforms one tile the tensor-memory
// accelerator copies the next tile's columns (one [NZ][TC] box per field,
// cp.async.bulk.tensor) into shared memory, completing on an mbarrier.  Every
// wait is bounded: a block whose copy does not complete within about a second
// records the fault in `err`, waits (bounded) for its other copy and stops.

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// non-blocking probe of phase `parity`
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait on phase `parity`: false after `limit` cycles (~2e9: about a second).  try_wait
// may suspend the thread for a hardware-chosen time before it reports false, so a limit
// shortened below the default (the test hook) polls with the non-blocking test_wait instead.
constexpr long long kWaitLimit = 2000000000LL;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long limit = kWaitLimit) {
    const long long t0 = clock64();
    if (limit < kWaitLimit) {
        while (!mbar_test_wait(bar, parity))
            if (clock64() - t0 > limit) return false;
        return true;
    }
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// limit of the per-tile copy wait (aimx_set_wait_limit shortens it to make the wait run out in a
// test; the drain wait after a timeout always keeps the full bound)
__device__ long long g_tile_wait_limit = kWaitLimit;
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ int g_wait_timeouts = 0;   // bounded waits that ran out (read by aimx_wait_timeouts)

// tmap: S as float32 [B*F*NZ][4][Ny][2 Nx] (innermost last), box {2 TC, 1, 1, NZ}.
template <int NZ, int F>
__global__ void __launch_bounds__(2 * F * 8) k_zpass_tma(const __grid_constant__ CUtensorMap tmap, float2* S,
                                                             const float2* __restrict__ spec, int Nx, int Ny, int B) {
    extern __shared__ __align__(128) unsigned char smraw[];
    constexpr int TC = 8;
    constexpr unsigned COLB = NZ * TC * sizeof(float2);   // one field's box
    constexpr unsigned TILEB = F * COLB;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);
    unsigned char* buf = smraw + 128;
    float2* sm = reinterpret_cast<float2*>(smraw + 128 + TILEB);
    const int NP = Nx * Ny;
    const int tx = Nx / TC;
    const int64_t T = (int64_t)tx * Ny * 4 * B;
    const int c = threadIdx.x % TC;
    const int f = (threadIdx.x / TC) % F;
    const int pz = threadIdx.x / (TC * F);
    const int64_t zs = 4 * (int64_t)NP;
    auto issue = [&](int64_t t) {   // thread 0: copy tile t's columns into buf
        const int xb = (int)(t % tx);
        int64_t r = t / tx;
        const int kyp = (int)(r % Ny);
        r /= Ny;
        const int q = (int)(r & 3), b = (int)(r >> 2);
        fence_proxy_async();
        mbar_expect_tx(bar, TILEB);
        for (int ff = 0; ff < F; ++ff)
            tma_load_4d(buf + ff * COLB, &tmap, 2 * xb * TC, kyp, q, (b * F + ff) * NZ, bar);
    };
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    int64_t t = blockIdx.x;
    if (threadIdx.x == 0 && t < T) issue(t);
    unsigned parity = 0;
    bool failed = false;
    for (; t < T; t += gridDim.x) {
        const bool ok = mbar_wait_bounded(bar, parity, g_tile_wait_limit);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        parity ^= 1u;
        const int xb = (int)(t % tx);
        int64_t r = t / tx;
        const int kyp = (int)(r % Ny);
        r /= Ny;
        const int q = (int)(r & 3), b = (int)(r >> 2);
        const int kx0 = xb * TC;
        const float2* col = reinterpret_cast<const float2*>(buf + f * COLB) + c;   // rows z of TC columns
        float2 v[NZ];
#pragma unroll
        for (int z = 0; z < NZ; ++z) v[z] = col[z * TC];
        __syncthreads();                                   // every column is in registers: buf is free
        if (threadIdx.x == 0 && t + gridDim.x < T) issue(t + gridDim.x);
        const int64_t base = (((int64_t)b * F + f) * NZ * 4 + q) * NP + (int64_t)kyp * Nx + kx0 + c;
        zpass_tile<NZ, F>(v, sm, S, spec, Nx, Ny, kx0, kyp, q, c, f, pz, base, zs);
        __syncthreads();                                   // the line area is reused by the next tile
    }
    if (failed && threadIdx.x == 0) {
        atomicAdd(&g_wait_timeouts, 1);
        mbar_wait_bounded(bar, parity, kWaitLimit);        // the copy still in flight, full bound
    }
}

// K4 (register form): inverse of K2 plus the interpolation partials.
// Charge form (tpart given, EFIE): the rho field's output plane is interpolated with the pulse
// weights per triangle touching the plane (partials tpart[b][slot][t]) instead of per basis.
template <int N, bool CHG, bool BIG>
__global__ void __launch_bounds__(2 * N) k_xy_inv_reg(const float2* __restrict__ S, const float* __restrict__ w,
                                                      const int* __restrict__ anc, const int* __restrict__ plane_lo,
                                                      const int* __restrict__ plane_hi, float2* part, int F, int Nz,
                                                      int Ntot, int P, const int* __restrict__ tanc,
                                                      const int* __restrict__ tplane, const float* __restrict__ lps,
                                                      float2* tpart, int nt, int cap) {
    extern __shared__ float2 sm[];
    constexpr int PITCH = N + 1;
    float2* acc = sm + 2 * N * PITCH;
    const int z = blockIdx.x, grp = blockIdx.y, b = blockIdx.z;
    int2* meta = reinterpret_cast<int2*>(acc + (BIG ? min(plane_hi[z] - plane_lo[z], cap) : plane_hi[z] - plane_lo[z]));
    const int px = threadIdx.x / N, r = threadIdx.x - px * N;
    float2* pl = sm + px * N * PITCH;
    float2* O = sm;                       // parity-0 plane doubles as the output plane
    const int G = F / 4;
    const int lo = plane_lo[z], hi = plane_hi[z];
    const int nb = hi - lo;
    const int U = P * P * P;
    // per basis touching this plane: stencil corner (sx, sy) in the plane and the offset of its
    // weights for this plane's stencil slot, computed once and reused for the four fields.  A
    // plane with more bases than shared memory holds (cap) recomputes them per field and sums
    // the four fields' partials in the output array instead (same order, so the same sums).
    const bool gl = BIG && nb > cap;   // only instantiated for contexts with such planes
    auto meta_of = [&](int k) {
        const int i = lo + k;
        return make_int2(anc[3 * i + 1] * PITCH + anc[3 * i], (z - anc[3 * i + 2]) * P * P * Ntot + i);
    };
    auto part_at = [&](int k) -> float2& {
        const int i = lo + k;
        return part[(((int64_t)b * G + grp) * P + (z - anc[3 * i + 2])) * Ntot + i];
    };
    if (!gl) {
        for (int k = threadIdx.x; k < nb; k += blockDim.x) {
            const int i = lo + k;
            const int sx = anc[3 * i], sy = anc[3 * i + 1], slot = z - anc[3 * i + 2];
            acc[k] = make_float2(0.f, 0.f);
            meta[k] = make_int2(sy * PITCH + sx, slot * P * P * Ntot + i);
        }
    }
    float2 v[N];
#pragma unroll 1
    for (int fl = 0; fl < 4; ++fl) {
        const int f = grp * 4 + fl;
        const int64_t plane = ((int64_t)(b * F + f) * Nz + z);
        // columns kx' = r of both y parities -> plane px (sum over py)
#pragma unroll 1
        for (int py = 0; py < 2; ++py) {
            const float2* src = S + (plane * 4 + (px + 2 * py)) * N * N + r;
#pragma unroll
            for (int ky = 0; ky < N; ++ky) v[ky] = __ldg(src + ky * N);
            reg_fft<N, true>(v);
            if (py) {
#pragma unroll
                for (int y = 0; y < N; ++y) pl[y * PITCH + r] = pl[y * PITCH + r] + (y ? v[y] * twc<true>(y, 2 * N) : v[y]);
            } else {
#pragma unroll
                for (int y = 0; y < N; ++y) pl[y * PITCH + r] = v[y];
            }
        }
        __syncthreads();
        // rows y = r of plane px, untwisted in x; parity 1 is added into parity 0's row
#pragma unroll
        for (int x = 0; x < N; ++x) v[x] = pl[r * PITCH + x];
        reg_fft<N, true>(v);
        if (px) {
#pragma unroll
            for (int x = 1; x < N; ++x) v[x] = v[x] * twc<true>(x, 2 * N);
        } else {
#pragma unroll
            for (int x = 0; x < N; ++x) O[r * PITCH + x] = v[x];
        }
        __syncthreads();
        if (px) {
#pragma unroll
            for (int x = 0; x < N; ++x) O[r * PITCH + x] = O[r * PITCH + x] + v[x];
        }
        __syncthreads();
        if (CHG && (f & 3) == 3) {
            // charge form: triangle partials of the rho field (of J; f = 7: of M, the second
            // block of tpart), one per (triangle, stencil slot)
            const int tlo = tplane[z], thi = tplane[Nz + z];
            for (int k = tlo + threadIdx.x; k < thi; k += blockDim.x) {
                const int sx = tanc[3 * k], sy = tanc[3 * k + 1], slot = z - tanc[3 * k + 2];
                const float* lw = lps + (int64_t)slot * P * P * nt + k;
                float2 sk = make_float2(0.f, 0.f);
                for (int uy = 0; uy < P; ++uy)
                    for (int ux = 0; ux < P; ++ux)
                        rfma(sk, __ldg(lw + (int64_t)(uy * P + ux) * nt), O[(sy + uy) * PITCH + sx + ux]);
                tpart[((int64_t)(f >> 2) * gridDim.z * P + (int64_t)b * P + slot) * nt + k] = sk;
            }
        } else if (P == 3) {
            // four bases per iteration so that their 36 weight gathers are in flight together
            // (the transform's registers are free in this phase)
            const int bd = blockDim.x;
            for (int k = threadIdx.x; k < nb; k += 4 * bd) {
                int kk[4];
                int2 m[4];
                float a[4][9];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    kk[j] = k + j * bd;
                    m[j] = gl ? meta_of(kk[j] < nb ? kk[j] : k) : meta[kk[j] < nb ? kk[j] : k];
                    // field-major weights ws[fl][u][i]: neighbouring bases of one slot are adjacent
                    const float* wj = w + (int64_t)fl * U * Ntot + m[j].y;
#pragma unroll
                    for (int u = 0; u < 9; ++u) a[j][u] = __ldg(wj + (int64_t)u * Ntot);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float2 sj = make_float2(0.f, 0.f);
#pragma unroll
                    for (int uy = 0; uy < 3; ++uy)
#pragma unroll
                        for (int ux = 0; ux < 3; ++ux) rfma(sj, a[j][uy * 3 + ux], O[m[j].x + uy * PITCH + ux]);
                    if (kk[j] < nb) {
                        if (!gl)
                            acc[kk[j]] = acc[kk[j]] + sj;
                        else
                            part_at(kk[j]) = fl ? part_at(kk[j]) + sj : make_float2(0.f, 0.f) + sj;
                    }
                }
            }
        } else
        // two bases per iteration so that both weight gathers are in flight together
        for (int k = threadIdx.x; k < nb; k += 2 * blockDim.x) {
            const int k2 = k + blockDim.x;
            const bool two = k2 < nb;
            const int2 m0 = gl ? meta_of(k) : meta[k];
            const int2 m1 = two ? (gl ? meta_of(k2) : meta[k2]) : m0;
            const float* w0 = w + (int64_t)fl * U * Ntot + m0.y;
            const float* w1 = w + (int64_t)fl * U * Ntot + m1.y;
            {
                float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
                for (int uy = 0; uy < P; ++uy)
                    for (int ux = 0; ux < P; ++ux) {
                        rfma(s0, __ldg(w0 + (int64_t)(uy * P + ux) * Ntot), O[m0.x + uy * PITCH + ux]);
                        rfma(s1, __ldg(w1 + (int64_t)(uy * P + ux) * Ntot), O[m1.x + uy * PITCH + ux]);
                    }
                if (!gl) {
                    acc[k] = acc[k] + s0;
                    if (two) acc[k2] = acc[k2] + s1;
                } else {
                    part_at(k) = fl ? part_at(k) + s0 : make_float2(0.f, 0.f) + s0;
                    if (two) part_at(k2) = fl ? part_at(k2) + s1 : make_float2(0.f, 0.f) + s1;
                }
            }
        }
        __syncthreads();
    }
    if (!gl) {
        for (int k = threadIdx.x; k < nb; k += blockDim.x) {
            const int i = lo + k;
            const int slot = z - anc[3 * i + 2];
            part[(((int64_t)b * G + grp) * P + slot) * Ntot + i] = acc[k];
        }
    }
}

// ------------------------------------------------------------------ host driver

static bool reg_shape(const aimx_ctx* ctx) {
    const int N = ctx->n[0];
    if (ctx->n[1] != N) return false;
    if (N != 8 && N != 16 && N != 32 && N != 64) return false;
    const int Nz = ctx->n[2];
    if (Nz != 8 && Nz != 16 && Nz != 32 && Nz != 64) return false;
    return true;   // planes with more bases than shared memory holds sum in the output array
}

bool fused_reg_supported(const aimx_ctx* ctx) { return fused_supported(ctx) && reg_shape(ctx); }

// register kernels unless the schedule asks for the shared-memory ones
static bool reg_path(const aimx_ctx* ctx) { return ctx->sched_variant != 1 && reg_shape(ctx); }


template <class K>
static void set_smem(K kernel, size_t bytes) {
    // The limit is one value per kernel and device for the whole process, and the host threads
    // of a batch launch the same kernel for members of different sizes: it only ever grows, so a
    // launch never finds it lowered by another thread between setting it and launching.
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> granted;
    int dev = 0;
    AIMX_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t& g = granted[{dev, reinterpret_cast<const void*>(kernel)}];
    if (bytes > g) {
        AIMX_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        g = bytes;
    }
}

static int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        AIMX_CUDA_TRY(cudaGetDevice(&dev));
        AIMX_CUDA_TRY(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    }
    return n;
}

template <int N>
static void launch_xy_fwd_reg(const aimx_ctx* ctx, const float2* G, float2* S, int B, cudaStream_t s) {
    size_t sm = 2 * (size_t)N * (N + 1) * sizeof(float2);
    set_smem(k_xy_fwd_reg<N>, sm);
    k_xy_fwd_reg<N><<<dim3(ctx->n[2], ctx->F, B), 2 * N, sm, s>>>(G, S, ctx->F, ctx->n[2]);
}

template <int N>
static void launch_xy_inv_reg(const aimx_ctx* ctx, const float2* S, const int* plo, const int* phi, float2* part,
                              int B, cudaStream_t s) {
    // bases of a plane kept in shared memory (accumulator + metadata, 16 bytes each) up to 200 KB
    const int cap_fit = (int)std::min<size_t>(ctx->max_plane_bases,
                                          (200 * 1024 - 2 * (size_t)N * (N + 1) * sizeof(float2)) / 16);
    const int cap = ctx->plane_cap > 0 ? std::min(cap_fit, ctx->plane_cap) : cap_fit;
    size_t sm = (2 * (size_t)N * (N + 1) + 2 * (size_t)cap) * sizeof(float2);
    const dim3 grid(ctx->n[2], ctx->F / 4, B);
    auto go = [&](auto kern, bool chg) {
        set_smem(kern, sm);
        kern<<<grid, 2 * N, sm, s>>>(S, ctx->d_wsoa, ctx->d_anc, plo, phi, part, ctx->F, ctx->n[2], ctx->N, ctx->P,
                                     chg ? ctx->d_tanc : nullptr, chg ? ctx->d_tplane : nullptr,
                                     chg ? ctx->d_lp_soa : nullptr,
                                     chg ? reinterpret_cast<float2*>(ctx->d_tpart) : nullptr, ctx->nt, cap);
    };
    // the common case (every plane's bases in shared memory) keeps the kernel without the other form
    const bool big = ctx->max_plane_bases > cap;
    if (ctx->charge)
        big ? go(k_xy_inv_reg<N, true, true>, true) : go(k_xy_inv_reg<N, true, false>, true);
    else
        big ? go(k_xy_inv_reg<N, false, true>, false) : go(k_xy_inv_reg<N, false, false>, false);
}

template <int NZ, int F>
static void launch_zpass_reg(const aimx_ctx* ctx, float2* S, int B, cudaStream_t s) {
    constexpr int TC = 8, LP = 2 * NZ + 2, FS = TC * LP + 1;
    size_t sm = (size_t)F * FS * sizeof(float2);
    set_smem(k_zpass_reg<NZ, F>, sm);
    k_zpass_reg<NZ, F><<<dim3(ctx->n[0] / TC, ctx->n[1], 4 * B), 2 * F * TC, sm, s>>>(
        S, reinterpret_cast<const float2*>(ctx->f32.spec), ctx->n[0], ctx->n[1], B);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link-time driver dependency)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p) {
            cudaGetLastError();
            throw Error{AIMX_E_CUDA, "cuTensorMapEncodeTiled is not available"};
        }
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

template <int NZ, int F>
static void launch_zpass_tma(const aimx_ctx* ctx, float2* S, int B, cudaStream_t s) {
    constexpr int TC = 8, LP = 2 * NZ + 2, FS = TC * LP + 1;
    const int Nx = ctx->n[0], Ny = ctx->n[1];
    // S as float32 [B F NZ][4][Ny][2 Nx]; the box is TC complex columns (64 B, x a multiple of
    // 16 floats) by NZ planes of one field
    CUtensorMap map;
    const cuuint64_t dims[4] = {(cuuint64_t)2 * Nx, (cuuint64_t)Ny, 4, (cuuint64_t)B * F * NZ};
    const cuuint64_t strides[3] = {(cuuint64_t)Nx * sizeof(float2), (cuuint64_t)Nx * Ny * sizeof(float2),
                                   (cuuint64_t)4 * Nx * Ny * sizeof(float2)};
    const cuuint32_t box[4] = {2 * TC, 1, 1, NZ};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    if (reinterpret_cast<uintptr_t>(S) % 16 != 0) throw Error{AIMX_E_CUDA, "z-pass buffer not 16-byte aligned"};
    const CUresult r = tensor_map_encoder()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, S, dims, strides, box, estr,
                                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error{AIMX_E_CUDA, "cuTensorMapEncodeTiled failed for the z-pass"};
    const size_t sm = 128 + (size_t)F * NZ * TC * sizeof(float2) + (size_t)F * FS * sizeof(float2);
    set_smem(k_zpass_tma<NZ, F>, sm);
    const int64_t T = (int64_t)(Nx / TC) * Ny * 4 * B;
    const int grid = (int)std::min<int64_t>(T, 2 * (int64_t)num_sms());
    k_zpass_tma<NZ, F><<<grid, 2 * F * TC, sm, s>>>(map, S, reinterpret_cast<const float2*>(ctx->f32.spec), Nx, Ny, B);
}

struct FusedBufs {
    float2 *xT, *G, *S, *part;
};

// One plane-fused pass over B right-hand sides; `timed` wraps each stage in a
// profiling scope (off for the allocation-free entry point).
static void run_fused(aimx_ctx* ctx, const NearC& nc, int B, const float2* xb, float2* yb, cudaStream_t s,
                      const FusedBufs& fb, bool timed) {
    const int Nx = ctx->n[0], Ny = ctx->n[1], Nz = ctx->n[2];
    const int64_t NG = (int64_t)Nx * Ny * Nz;
    const int F = ctx->F, N = ctx->N, nunk = ctx->nunk, P = ctx->P, U = ctx->U;
    const int NP = Nx * Ny;
    const float2* tw = twiddles32();
    const int* plo = ctx->d_plane;
    const int* phi = plo + Nz;
    const bool reg = reg_path(ctx);
    auto scope = [&](int st) { return timed ? new StageScope(ctx, st, s) : nullptr; };
    StageScope* sc = scope(ST_TRANSPOSE);
    int64_t tot = (int64_t)nunk * B;
    k_transpose_x<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(xb, ctx->d_perm, fb.xT, N, nunk, B);
    AIMX_CUDA_TRY(cudaGetLastError());
    const bool chg = ctx->charge != 0;
    if (chg) charge_fused_q(ctx, fb.xT, B, s);
    delete sc;
    sc = scope(ST_GATHER);
    {
        const dim3 grid((unsigned)((NG + 15) / 16), (unsigned)((B + 31) / 32));
        const float4* w4 = reinterpret_cast<const float4*>(ctx->f32.w);
        const int64_t qt_m = (int64_t)ctx->nt * B;   // M charges after the J charges (two-region)
        if (F == 8)
            k_gather_tile<8><<<grid, 256, 0, s>>>(w4, ctx->d_node_ptr, ctx->d_node_w, fb.xT, fb.G, B, N, U, NG,
                                                  chg ? ctx->d_tnode_ptr : nullptr, ctx->d_tnode_w, ctx->f32.plw,
                                                  reinterpret_cast<const float2*>(ctx->d_qT), qt_m);
        else
            k_gather_tile<4><<<grid, 256, 0, s>>>(w4, ctx->d_node_ptr, ctx->d_node_w, fb.xT, fb.G, B, N, U, NG,
                                                  chg ? ctx->d_tnode_ptr : nullptr, ctx->d_tnode_w, ctx->f32.plw,
                                                  reinterpret_cast<const float2*>(ctx->d_qT), qt_m);
    }
    AIMX_CUDA_TRY(cudaGetLastError());
    delete sc;
    sc = scope(ST_XY_FWD);
    if (reg) {
        switch (Nx) {
            case 8: launch_xy_fwd_reg<8>(ctx, fb.G, fb.S, B, s); break;
            case 16: launch_xy_fwd_reg<16>(ctx, fb.G, fb.S, B, s); break;
            case 32: launch_xy_fwd_reg<32>(ctx, fb.G, fb.S, B, s); break;
            default: launch_xy_fwd_reg<64>(ctx, fb.G, fb.S, B, s); break;
        }
    } else {
        size_t sm = ((size_t)NP + (size_t)Ny * (Nx + 1)) * sizeof(float2);
        set_smem(k_xy_fwd, sm);
        k_xy_fwd<<<dim3(Nz, F, B), kThreads, sm, s>>>(fb.G, fb.S, F, Nx, Ny, Nz, tw);
    }
    AIMX_CUDA_TRY(cudaGetLastError());
    delete sc;
    sc = scope(ST_ZPASS);
    if (reg && ctx->sched_variant == 3) {
        if (F == 4) {
            switch (Nz) {
                case 8: launch_zpass_tma<8, 4>(ctx, fb.S, B, s); break;
                case 16: launch_zpass_tma<16, 4>(ctx, fb.S, B, s); break;
                case 32: launch_zpass_tma<32, 4>(ctx, fb.S, B, s); break;
                default: launch_zpass_tma<64, 4>(ctx, fb.S, B, s); break;
            }
        } else {
            switch (Nz) {
                case 8: launch_zpass_tma<8, 8>(ctx, fb.S, B, s); break;
                case 16: launch_zpass_tma<16, 8>(ctx, fb.S, B, s); break;
                case 32: launch_zpass_tma<32, 8>(ctx, fb.S, B, s); break;
                default: launch_zpass_tma<64, 8>(ctx, fb.S, B, s); break;
            }
        }
    } else if (reg) {
        if (F == 4) {
            switch (Nz) {
                case 8: launch_zpass_reg<8, 4>(ctx, fb.S, B, s); break;
                case 16: launch_zpass_reg<16, 4>(ctx, fb.S, B, s); break;
                case 32: launch_zpass_reg<32, 4>(ctx, fb.S, B, s); break;
                default: launch_zpass_reg<64, 4>(ctx, fb.S, B, s); break;
            }
        } else {
            switch (Nz) {
                case 8: launch_zpass_reg<8, 8>(ctx, fb.S, B, s); break;
                case 16: launch_zpass_reg<16, 8>(ctx, fb.S, B, s); break;
                case 32: launch_zpass_reg<32, 8>(ctx, fb.S, B, s); break;
                default: launch_zpass_reg<64, 8>(ctx, fb.S, B, s); break;
            }
        }
    } else {
        size_t sm = (size_t)F * kTX * (2 * Nz + 1) * sizeof(float2);
        set_smem(k_zpass, sm);
        k_zpass<<<dim3(Nx / kTX, Ny, 4 * ((B + kRG - 1) / kRG)), kThreads, sm, s>>>(
            fb.S, reinterpret_cast<const float2*>(ctx->f32.spec), F, Nx, Ny, Nz, B, tw);
    }
    AIMX_CUDA_TRY(cudaGetLastError());
    delete sc;
    sc = scope(ST_XY_INV);
    if (reg) {
        switch (Nx) {
            case 8: launch_xy_inv_reg<8>(ctx, fb.S, plo, phi, fb.part, B, s); break;
            case 16: launch_xy_inv_reg<16>(ctx, fb.S, plo, phi, fb.part, B, s); break;
            case 32: launch_xy_inv_reg<32>(ctx, fb.S, plo, phi, fb.part, B, s); break;
            default: launch_xy_inv_reg<64>(ctx, fb.S, plo, phi, fb.part, B, s); break;
        }
    } else {
        size_t sm = ((size_t)NP + (size_t)Ny * (Nx + 1) + ctx->max_plane_bases) * sizeof(float2);
        set_smem(k_xy_inv, sm);
        k_xy_inv<<<dim3(Nz, F / 4, B), kThreads, sm, s>>>(fb.S, ctx->f32.w, ctx->d_anc, plo, phi, fb.part, F, Nx, Ny,
                                                          Nz, N, P, tw);
    }
    AIMX_CUDA_TRY(cudaGetLastError());
    delete sc;
    sc = scope(ST_FINAL);
    if (chg) charge_fused_phi(ctx, B, nc.cphi, nc.cphi2, s);
    const float2* phiT = chg ? reinterpret_cast<const float2*>(ctx->d_phiT) : nullptr;
    if (!ctx->aim && ctx->nb_count > 0) {
        const size_t smem = (size_t)ctx->nb_umax * 32 * sizeof(float2);
        const int* lp_ = ctx->linterm ? ctx->d_lin_ptr : nullptr;
        const int has_k = F == 8 ? 1 : (ctx->f32.ng != nullptr);
        auto go = [&](auto kern) {
            set_smem(kern, smem);
            kern<<<ctx->nb_count, kNbWarps * 32, smem, s>>>(
                fb.part, fb.xT, ctx->d_nb_rows, ctx->d_nb_ustart, ctx->d_nb_ucols, ctx->d_nb_ent, ctx->d_row_ptr,
                ctx->d_perm, lp_, ctx->d_lin_cols, ctx->f32.la, ctx->f32.lp, yb, nc, has_k, N, nunk, P, B, phiT,
                ctx->d_btri_t, ctx->d_blen, (int64_t)ctx->nt * B);
        };
        // up to 16 RHS: each warp applies several entries at once
        const bool split = B <= 16;
        if (F == 8)
            split ? go(k_near_blk<8, true>) : go(k_near_blk<8, false>);
        else
            split ? go(k_near_blk<4, true>) : go(k_near_blk<4, false>);
    } else
    k_final<<<(N + kFinalRows - 1) / kFinalRows, kThreads, 0, s>>>(fb.part, fb.xT, ctx->d_row_ptr, ctx->d_cols,
                                                                   ctx->f32.na, ctx->f32.np,
                                                                   F == 8 ? ctx->f32.nk : ctx->f32.ng, ctx->d_perm,
                                                                   ctx->linterm && !ctx->aim ? ctx->d_lin_ptr : nullptr,
                                                                   ctx->d_lin_cols, ctx->f32.la, ctx->f32.lp,
                                                                   ctx->aim ? reinterpret_cast<const float2*>(ctx->f32.zn)
                                                                            : nullptr,
                                                                   yb, nc, F, N, nunk, P, B, phiT, ctx->d_btri_t,
                                                                   ctx->d_blen, (int64_t)ctx->nt * B);
    AIMX_CUDA_TRY(cudaGetLastError());
    delete sc;
}

static NearC near_c(const aimx_ctx* ctx, double freq) {
    Coefs cf = near_coefs(ctx, freq);
    NearC nc;
    for (int k = 0; k < 6; ++k) nc.c[k] = make_float2((float)cf.near[k].x, (float)cf.near[k].y);
    for (int k = 0; k < 4; ++k) nc.lin[k] = make_float2((float)cf.lin[k].x, (float)cf.lin[k].y);
    nc.cphi = nc.cphi2 = make_float2(0.f, 0.f);
    if (ctx->charge) {
        // charge form: the RWG N^Phi drops out; its coefficient scales the triangle near part
        // (two regions: of the J rows, c[1], and of the M rows, c[5])
        nc.cphi = nc.c[1];
        nc.c[1] = make_float2(0.f, 0.f);
        if (ctx->F == 8) {
            nc.cphi2 = nc.c[5];
            nc.c[5] = make_float2(0.f, 0.f);
        }
    }
    if (ctx->aim) {
        // the per-frequency entries carry j w mu and -j w mu / k^2 already; they are exact on the
        // near pairs, so the linear-term modification does not apply
        nc.c[0] = make_float2(1.f, 0.f);
        nc.c[1] = make_float2(0.f, 0.f);
        for (auto& v : nc.lin) v = make_float2(0.f, 0.f);
    }
    return nc;
}

static void ensure_fused_buffers(aimx_ctx* ctx, int B) {
    if (ctx->fused_cap >= B) return;
    const int64_t NG = (int64_t)ctx->n[0] * ctx->n[1] * ctx->n[2];
    const int F = ctx->F;
    if (ctx->d_xT) dev_free(ctx, ctx->d_xT);
    if (ctx->d_G) dev_free(ctx, ctx->d_G);
    if (ctx->d_S) dev_free(ctx, ctx->d_S);
    if (ctx->d_part) dev_free(ctx, ctx->d_part);
    ctx->d_xT = ctx->d_G = ctx->d_S = ctx->d_part = nullptr;
    ctx->fused_cap = 0;
    ctx->d_xT = (float*)dev_alloc(ctx, sizeof(float2) * (size_t)ctx->nunk * B);
    ctx->d_G = (float*)dev_alloc(ctx, sizeof(float2) * (size_t)B * F * NG);
    ctx->d_S = (float*)dev_alloc(ctx, sizeof(float2) * (size_t)B * F * NG * 4);
    ctx->d_part = (float*)dev_alloc(ctx, sizeof(float2) * (size_t)B * (F / 4) * ctx->P * ctx->N);
    ctx->fused_cap = B;
}

// plane ranges on the device (uploaded on the first fused call)
static void ensure_plane_table(aimx_ctx* ctx) {
    if (ctx->d_plane) return;
    std::vector<int> v(ctx->plane_lo);
    v.insert(v.end(), ctx->plane_hi.begin(), ctx->plane_hi.end());
    ctx->d_plane = (int*)dev_alloc(ctx, sizeof(int) * v.size());
    AIMX_CUDA_TRY(cudaMemcpy(ctx->d_plane, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice));
    int mpb = 0;
    for (size_t z = 0; z < ctx->plane_lo.size(); ++z) mpb = std::max(mpb, ctx->plane_hi[z] - ctx->plane_lo[z]);
    ctx->max_plane_bases = mpb;
}

// Row blocks of the near CSR for k_near_blk (built once per context, on the host from the
// internal-order pattern): consecutive rows are added to a block while it has fewer than
// kNbRows rows and the union of their columns stays within kNbUmax (a single row may exceed
// it).  If some block's union would not fit in shared memory the blocked kernel is not used.
static void ensure_near_blocks(aimx_ctx* ctx) {
    if (ctx->nb_count > 0 || ctx->nb_umax < 0) return;
    const int N = ctx->N;
    const std::vector<int>& rp = ctx->row_ptr;
    const std::vector<int>& cols = ctx->cols;
    std::vector<int> stamp(N, -1), pos(N, 0), rows{0}, ust{0}, ucols, li(ctx->nnz), tmp;
    int blk = 0, umax = 0;
    for (int i = 0; i < N;) {
        int j = i, u = 0;
        while (j < N && j - i < kNbRows) {
            int add = 0;
            for (int e = rp[j]; e < rp[j + 1]; ++e) add += stamp[cols[e]] != blk;
            if (j > i && u + add > kNbUmax) break;
            for (int e = rp[j]; e < rp[j + 1]; ++e) stamp[cols[e]] = blk;
            u += add;
            ++j;
        }
        tmp.clear();
        for (int e = rp[i]; e < rp[j]; ++e) {
            const int c = cols[e];
            if (stamp[c] == blk) {
                stamp[c] = -2 - blk;   // collected (never equal to a later block id)
                tmp.push_back(c);
            }
        }
        std::sort(tmp.begin(), tmp.end());
        for (size_t k = 0; k < tmp.size(); ++k) pos[tmp[k]] = (int)k;
        for (int e = rp[i]; e < rp[j]; ++e) li[e] = pos[cols[e]];
        ucols.insert(ucols.end(), tmp.begin(), tmp.end());
        rows.push_back(j);
        ust.push_back((int)ucols.size());
        umax = std::max(umax, (int)tmp.size());
        ++blk;
        i = j;
    }
    // shared memory: the staged union plus 24 KB of partial-sum tiles and entry buffers
    if ((size_t)umax * 32 * sizeof(float2) + 24 * 1024 > 200 * 1024) {
        ctx->nb_umax = -1;
        return;
    }
    ctx->d_nb_rows = (int*)dev_alloc(ctx, sizeof(int) * rows.size());
    ctx->d_nb_ustart = (int*)dev_alloc(ctx, sizeof(int) * ust.size());
    ctx->d_nb_ucols = (int*)dev_alloc(ctx, sizeof(int) * std::max<size_t>(1, ucols.size()));
    ctx->d_nb_ent = (float4*)dev_alloc(ctx, sizeof(float4) * std::max<int64_t>(1, ctx->nnz));
    AIMX_CUDA_TRY(cudaMemcpy(ctx->d_nb_rows, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice));
    AIMX_CUDA_TRY(cudaMemcpy(ctx->d_nb_ustart, ust.data(), sizeof(int) * ust.size(), cudaMemcpyHostToDevice));
    AIMX_CUDA_TRY(cudaMemcpy(ctx->d_nb_ucols, ucols.data(), sizeof(int) * ucols.size(), cudaMemcpyHostToDevice));
    if (ctx->nnz > 0) {
        int* d_li = (int*)dev_alloc(ctx, sizeof(int) * ctx->nnz);
        try {
            AIMX_CUDA_TRY(cudaMemcpy(d_li, li.data(), sizeof(int) * ctx->nnz, cudaMemcpyHostToDevice));
            const float* vk = ctx->F == 8 ? ctx->f32.nk : ctx->f32.ng;
            k_pack_near_ent<<<(unsigned)((ctx->nnz + 255) / 256), 256>>>(d_li, ctx->f32.na, ctx->f32.np, vk,
                                                                        ctx->nnz, ctx->d_nb_ent);
            AIMX_CUDA_TRY(cudaGetLastError());
            AIMX_CUDA_TRY(cudaDeviceSynchronize());
        } catch (...) {
            dev_free(ctx, d_li);
            throw;
        }
        dev_free(ctx, d_li);
        ctx->device_bytes -= (int64_t)sizeof(int) * ctx->nnz;
    }
    ctx->nb_umax = umax;
    ctx->nb_count = blk;
}

void matvec_fused(aimx_ctx* ctx, double freq, int nrhs, const float* x, float* y, cudaStream_t s) {
    {
        StageScope sc(ctx, ST_KERNELGEN, s);
        ensure_spectra<float>(ctx, freq, s);
    }
    ensure_aim_near(ctx, freq, s);
    ensure_plane_table(ctx);
    ensure_near_blocks(ctx);
    const NearC nc = near_c(ctx, freq);
    const int64_t NG = (int64_t)ctx->n[0] * ctx->n[1] * ctx->n[2];
    const int F = ctx->F;
    // RHS per pass bounded by an 8 GiB work-buffer budget
    const size_t per_rhs =
        sizeof(float2) * ((size_t)ctx->nunk + (size_t)F * NG * 5 + (size_t)(F / 4) * ctx->P * ctx->N);
    int cap = (int)std::max<size_t>(1, std::min<size_t>(nrhs, ((size_t)8 << 30) / per_rhs));
    if (ctx->sched_pass > 0) cap = std::min(cap, ctx->sched_pass);
    ensure_fused_buffers(ctx, cap);
    if (ctx->charge) ensure_charge_buffers(ctx, cap);
    FusedBufs fb{reinterpret_cast<float2*>(ctx->d_xT), reinterpret_cast<float2*>(ctx->d_G),
                 reinterpret_cast<float2*>(ctx->d_S), reinterpret_cast<float2*>(ctx->d_part)};
    for (int b0 = 0; b0 < nrhs; b0 += cap) {
        const int B = std::min(cap, nrhs - b0);
        run_fused(ctx, nc, B, reinterpret_cast<const float2*>(x) + (int64_t)b0 * ctx->nunk,
                  reinterpret_cast<float2*>(y) + (int64_t)b0 * ctx->nunk, s, fb, true);
    }
}

// Scratch bytes of one plane-fused pass over B right-hand sides when every
// work buffer starts on a 256-byte boundary.
size_t fused_scratch_bytes(const aimx_ctx* ctx, int B) {
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t NG = (size_t)ctx->n[0] * ctx->n[1] * ctx->n[2];
    const size_t F = ctx->F;
    return up(sizeof(float2) * (size_t)ctx->nunk * B) + up(sizeof(float2) * B * F * NG) +
           up(sizeof(float2) * B * F * NG * 4) + up(sizeof(float2) * (size_t)B * (F / 4) * ctx->P * ctx->N);
}

// The plane-fused FP32 product for all B right-hand sides at once, with the
// work buffers carved from caller-provided device memory `scratch` of at
// least fused_scratch_bytes(ctx, B) bytes.  Performs no allocation: the
// kernel spectra buffers, the plane table, the near row blocks and the device
// twiddle table must already exist (any earlier FP32 aimx_matvec on this
// context creates them).
void matvec_fused_into(aimx_ctx* ctx, double freq, int B, const float* x, float* y, cudaStream_t s,
                       unsigned char* scratch) {
    ensure_spectra<float>(ctx, freq, s);
    ensure_aim_near(ctx, freq, s);
    const NearC nc = near_c(ctx, freq);
    const size_t NG = (size_t)ctx->n[0] * ctx->n[1] * ctx->n[2];
    const size_t F = ctx->F;
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    FusedBufs fb;
    fb.xT = reinterpret_cast<float2*>(scratch);
    fb.G = reinterpret_cast<float2*>(scratch + up(sizeof(float2) * (size_t)ctx->nunk * B));
    fb.S = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(fb.G) + up(sizeof(float2) * B * F * NG));
    fb.part = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(fb.S) + up(sizeof(float2) * B * F * NG * 4));
    run_fused(ctx, nc, B, reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(y), s, fb, false);
}

}  // namespace aimx

extern "C" int aimx_set_plane_cap(aimx_ctx* ctx, int cap) {
    if (!ctx) return AIMX_E_ARG;
    ctx->plane_cap = cap > 0 ? cap : 0;
    return AIMX_OK;
}

extern "C" int aimx_set_wait_limit(int64_t cycles) {
    const long long v = cycles > 0 ? (long long)cycles : aimx::kWaitLimit;
    if (cudaMemcpyToSymbol(aimx::g_tile_wait_limit, &v, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return AIMX_E_CUDA;
    }
    return AIMX_OK;
}

extern "C" int aimx_wait_timeouts(int* count) {
    if (!count) return AIMX_E_ARG;
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, aimx::g_wait_timeouts, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return AIMX_E_CUDA;
    }
    const int zero = 0;
    if (cudaMemcpyToSymbol(aimx::g_wait_timeouts, &zero, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return AIMX_E_CUDA;
    }
    *count = v;
    return AIMX_OK;
}
