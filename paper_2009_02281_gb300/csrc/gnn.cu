// Learned near-field preconditioner (not in the paper; the paper preconditions
// with the diagonal of L_s and notes that off-diagonal entries may augment it,
// Sec. III-A-2).  The preconditioner is
//
//     M = D^{-1} (I + C),
//
// D the per-basis frequency-combined static self block (scalar EFIE, 2x2 for
// the two-region form) and C supported on the near graph and its diagonal.
// Reversing the orientation of RWG function n flips row and column n of the
// operator, and the ideal C transforms as C_mn -> s_m s_n C_mn.  The network
// respects this by construction: node states see only orientation-invariant
// inputs, and each edge entry is a learned combination of 8 signed bases
// b_c(m, n) (the normalised static near entries of Eq. LAIMx and their
// two-hop products on the near pattern):
//
//     h0   = relu(A0 x + a0)
//     q_mn = relu(B_l h_n + C_l e_mn + c_l)              (near edges n -> m, n != m)
//     h_l  = relu(D_l h_m + mean_n q_mn + d_l)            l = 1..L
//     u_mn = relu(Ua h_m + Ub h_n + Uc e_mn + u)
//     C_mn[k] = sum_c (E u_mn + f)[k, c] b_c(m, n),   C_mm = G h_m + g
//
// Training minimises the probe loss (1/P) sum_p |M y_p - z_p|^2 / |z_p|^2 with
// y_p = A z_p, which is quadratic in C, so the operator only enters through
// the probe pairs.  Forward, loss, backward and Adam run here; weights are
// BF16 (an FP32 master copy and FP32 Adam moments are kept), all activations
// and accumulations are FP32, and every weight-gradient reduction uses a fixed
// partition and a fixed summation order, so a training step is deterministic.
//
// Layouts (internal basis order, i.e. sorted by anchor):
//   node features x [N][8], edge features e [nnz][16] and bases b [nnz][8] in
//   near-CSR order, activations H [L+1][N][64], P [L][N][64], head hidden
//   U [nnz][64] (training only), outputs o [nnz][K], g [N][K] (K = 2: one
//   complex entry; K = 8: 2x2 complex block, (E,J),(E,M),(H,J),(H,M) real parts
//   then imaginary parts).  Probe vectors are caller order.

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "aimx_internal.h"
#include "cplx.cuh"

namespace aimx {

constexpr int kW = 64;               // hidden width
constexpr int kNin = 8;              // node features
constexpr int kNed = 16;             // edge features (orientation invariant)
constexpr int kNB = 8;               // signed bases
constexpr int kMaxLayers = 8;
constexpr int kPersistWarps = 2048;  // fixed warp count of the reducing per-node kernels
constexpr int kWgradBlocks = 304;    // fixed block count of the row-reduction kernels

static inline unsigned gb(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------ parameter layout

GnnLayout gnn_layout(int K, int L) {
    GnnLayout g;
    g.K = K;
    g.L = L;
    int64_t o = 0;
    g.A0 = o; o += kW * kNin;
    g.a0 = o; o += kW;
    for (int l = 0; l < L; ++l) {
        g.B[l] = o; o += kW * kW;
        g.C[l] = o; o += kW * kNed;
        g.c[l] = o; o += kW;
        g.D[l] = o; o += kW * kW;
        g.d[l] = o; o += kW;
    }
    g.Ua = o; o += kW * kW;
    g.Ub = o; o += kW * kW;
    g.Uc = o; o += kW * kNed;
    g.u = o; o += kW;
    g.E = o; o += K * kNB * kW;
    g.f = o; o += K * kNB;
    g.G = o; o += K * kW;
    g.g = o; o += K;
    g.total = o;
    return g;
}

// ------------------------------------------------------------------ features

__global__ void k_node_features(const double* __restrict__ xyz, const int* __restrict__ tri,
                                const double* __restrict__ area, const int* __restrict__ btri,
                                const double* __restrict__ blen, const int* __restrict__ anc, int N, double ox,
                                double oy, double oz, double hx, double hy, double hz, double hb, double half_order,
                                double khb, double contrast, float* __restrict__ x, double* __restrict__ center) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double c[3] = {0, 0, 0};
    for (int s = 0; s < 2; ++s) {
        const int* t = tri + 3 * btri[2 * i + s];
        for (int a = 0; a < 3; ++a) c[a] += (xyz[3 * t[0] + a] + xyz[3 * t[1] + a] + xyz[3 * t[2] + a]) / 3.0;
    }
    for (int a = 0; a < 3; ++a) c[a] *= 0.5;
    center[3 * i] = c[0];
    center[3 * i + 1] = c[1];
    center[3 * i + 2] = c[2];
    float* xi = x + (int64_t)i * kNin;
    xi[0] = (float)(blen[i] / hb);
    xi[1] = (float)(area[btri[2 * i]] / (hb * hb));
    xi[2] = (float)(area[btri[2 * i + 1]] / (hb * hb));
    xi[3] = (float)((c[0] - ox) / hx - anc[3 * i] - half_order);
    xi[4] = (float)((c[1] - oy) / hy - anc[3 * i + 1] - half_order);
    xi[5] = (float)((c[2] - oz) / hz - anc[3 * i + 2] - half_order);
    xi[6] = (float)khb;
    xi[7] = (float)contrast;
}

// normalised static near entries eta^A, eta^Phi, eta^K per stored pair
__global__ void k_edge_eta(const int* __restrict__ rows, const int* __restrict__ cols, const int* __restrict__ dpos,
                           const double* __restrict__ na, const double* __restrict__ np,
                           const double* __restrict__ nk, int64_t nnz, double hb, double* __restrict__ eta) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nnz) return;
    const int m = rows[t], n = cols[t];
    const double tiny = 1e-300;
    const double sA = sqrt(fmax(fabs(na[dpos[m]]) * fabs(na[dpos[n]]), tiny));
    const double sP = sqrt(fmax(fabs(np[dpos[m]]) * fabs(np[dpos[n]]), tiny));
    eta[3 * t] = na[t] / sA;
    eta[3 * t + 1] = np[t] / sP;
    eta[3 * t + 2] = hb * nk[t] / sA;
}

// bases [eta^A, eta^Phi, eta^K, AA, PP, AP, PA, KK]: two-hop products
// (XY)_mn = sum_j X_mj Y_jn / sqrt(deg_m deg_n) over j in row m and row n (sorted merge;
// (j, n) is the transpose of (n, j) in row n)
__global__ void k_two_hop(const int* __restrict__ row_ptr, const int* __restrict__ cols,
                          const int* __restrict__ rows, const int* __restrict__ trans,
                          const double* __restrict__ eta, int64_t nnz, float* __restrict__ basis) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nnz) return;
    const int m = rows[t], n = cols[t];
    int a = row_ptr[m], ae = row_ptr[m + 1], b = row_ptr[n], be = row_ptr[n + 1];
    double AA = 0, PP = 0, AP = 0, PA = 0, KK = 0;
    while (a < ae && b < be) {
        const int ja = cols[a], jb = cols[b];
        if (ja < jb) {
            ++a;
        } else if (jb < ja) {
            ++b;
        } else {
            const double* x = eta + 3 * (int64_t)a;              // (m, j)
            const double* y = eta + 3 * (int64_t)trans[b];       // (j, n)
            AA += x[0] * y[0];
            PP += x[1] * y[1];
            AP += x[0] * y[1];
            PA += x[1] * y[0];
            KK += x[2] * y[2];
            ++a;
            ++b;
        }
    }
    const double dm = (double)(row_ptr[m + 1] - row_ptr[m] - 1), dn = (double)(row_ptr[n + 1] - row_ptr[n] - 1);
    const double s = 1.0 / sqrt(fmax(dm, 1.0) * fmax(dn, 1.0));
    float* bt = basis + t * kNB;
    bt[0] = (float)eta[3 * t];
    bt[1] = (float)eta[3 * t + 1];
    bt[2] = (float)eta[3 * t + 2];
    bt[3] = (float)(AA * s);
    bt[4] = (float)(PP * s);
    bt[5] = (float)(AP * s);
    bt[6] = (float)(PA * s);
    bt[7] = (float)(KK * s);
}

// orientation-invariant edge features
__global__ void k_edge_features(const int* __restrict__ rows, const int* __restrict__ cols,
                                const double* __restrict__ center, const double* __restrict__ eta,
                                const float* __restrict__ basis, int64_t nnz, double hb, double khb,
                                float* __restrict__ e) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nnz) return;
    const int m = rows[t], n = cols[t];
    double d[3], r2 = 0;
    for (int a = 0; a < 3; ++a) {
        d[a] = (center[3 * n + a] - center[3 * m + a]) / hb;
        r2 += d[a] * d[a];
    }
    const double eA = eta[3 * t], eP = eta[3 * t + 1], eK = eta[3 * t + 2];
    const float* b = basis + t * kNB;
    float* et = e + t * kNed;
    et[0] = (float)d[0];
    et[1] = (float)d[1];
    et[2] = (float)d[2];
    et[3] = (float)sqrt(r2);
    et[4] = (float)fabs(eA);
    et[5] = (float)fabs(eP);
    et[6] = (float)(eA * eP);
    et[7] = (float)fabs(eK);
    for (int c = 0; c < 5; ++c) et[8 + c] = fabsf(b[3 + c]);
    et[13] = (float)(eA * (double)b[3]);
    et[14] = (float)(eP * (double)b[4]);
    et[15] = (float)khb;
}

// ------------------------------------------------------------------ forward kernels

__device__ __forceinline__ float bf(const __nv_bfloat16* w, int64_t i) { return __bfloat162float(w[i]); }

// H0 = relu(A0 x + a0); one thread per (node, channel)
__global__ void k_input_layer(const float* __restrict__ x, const __nv_bfloat16* __restrict__ w, int64_t oA,
                              int64_t oa, int N, float* __restrict__ H0) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * kW) return;
    const int i = (int)(t / kW), c = (int)(t % kW);
    float acc = bf(w, oa + c);
    for (int f = 0; f < kNin; ++f) acc = fmaf(bf(w, oA + c * kNin + f), x[(int64_t)i * kNin + f], acc);
    H0[t] = fmaxf(acc, 0.f);
}

// Y[n][o] (=|+=) act( sum_i X[n][i] W'[o][i] + bias[o] + add[n][o] ), 64 x 64 weights:
// W' = W (row-major [out][in]) or, with TRANS, W^T.  64 nodes per block of 256 threads.
template <bool TRANS>
__global__ void __launch_bounds__(256) k_node_gemm(const float* __restrict__ X, const __nv_bfloat16* __restrict__ W,
                                                   const __nv_bfloat16* __restrict__ bias,
                                                   const float* __restrict__ add, float* __restrict__ Y, int N,
                                                   int relu, int accumulate) {
    __shared__ float Ws[kW][kW + 1];
    __shared__ float Xs[64][kW + 1];
    const int t = threadIdx.x;
    const int n0 = blockIdx.x * 64;
    for (int k = t; k < kW * kW; k += 256) {
        int r = k / kW, c = k % kW;
        float v = __bfloat162float(W[k]);
        if (TRANS)
            Ws[c][r] = v;
        else
            Ws[r][c] = v;
    }
    for (int k = t; k < 64 * kW; k += 256) {
        int r = k / kW, c = k % kW;
        Xs[r][c] = (n0 + r < N) ? X[(int64_t)(n0 + r) * kW + c] : 0.f;
    }
    __syncthreads();
    const int o = t & 63, grp = t >> 6;
    float acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.f;
    for (int i = 0; i < kW; ++i) {
        const float wv = Ws[o][i];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = fmaf(Xs[grp * 16 + j][i], wv, acc[j]);
    }
    const float b = bias ? __bfloat162float(bias[o]) : 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int n = n0 + grp * 16 + j;
        if (n >= N) break;
        const int64_t idx = (int64_t)n * kW + o;
        float v = acc[j] + b + (add ? add[idx] : 0.f);
        if (relu) v = fmaxf(v, 0.f);
        Y[idx] = accumulate ? Y[idx] + v : v;
    }
}

template <int NF>
__device__ __forceinline__ void load_row(const float* __restrict__ a, int64_t t, float v[NF]) {
    const float4* p = reinterpret_cast<const float4*>(a + t * NF);
#pragma unroll
    for (int q = 0; q < NF / 4; ++q) {
        const float4 r = __ldg(p + q);
        v[4 * q] = r.x;
        v[4 * q + 1] = r.y;
        v[4 * q + 2] = r.z;
        v[4 * q + 3] = r.w;
    }
}

// S[m] = (1/deg_m) sum_{n != m} relu(P[n] + C e_mn + c); one warp per node, lane owns channels lane, lane+32
__global__ void k_edge_message(const float* __restrict__ P, const float* __restrict__ e,
                               const __nv_bfloat16* __restrict__ w, int64_t oC, int64_t oc,
                               const int* __restrict__ row_ptr, const int* __restrict__ cols,
                               const float* __restrict__ deginv, int N, float* __restrict__ S) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    float C0[kNed], C1[kNed];
    for (int f = 0; f < kNed; ++f) {
        C0[f] = bf(w, oC + lane * kNed + f);
        C1[f] = bf(w, oC + (lane + 32) * kNed + f);
    }
    const float cb0 = bf(w, oc + lane), cb1 = bf(w, oc + lane + 32);
    for (int m = warp; m < N; m += nwarp) {
        float s0 = 0.f, s1 = 0.f;
        auto edge = [&](int t) {
            const int n = cols[t];
            if (n == m) return;
            float ef[kNed];
            load_row<kNed>(e, t, ef);
            float w0 = P[(int64_t)n * kW + lane] + cb0, w1 = P[(int64_t)n * kW + lane + 32] + cb1;
#pragma unroll
            for (int f = 0; f < kNed; ++f) {
                w0 = fmaf(C0[f], ef[f], w0);
                w1 = fmaf(C1[f], ef[f], w1);
            }
            s0 += fmaxf(w0, 0.f);
            s1 += fmaxf(w1, 0.f);
        };
        // two edges per iteration keep two independent gathers in flight (four measured slower here)
        int t = row_ptr[m];
        const int te = row_ptr[m + 1];
        for (; t + 1 < te; t += 2) {
            edge(t);
            edge(t + 1);
        }
        if (t < te) edge(t);
        const float di = deginv[m];
        S[(int64_t)m * kW + lane] = s0 * di;
        S[(int64_t)m * kW + lane + 32] = s1 * di;
    }
}

// shared copy of the edge head: Uc [64][16], u [64], E [K*8][64], f [K*8]
template <int K>
struct HeadSmem {
    float Uc[kW][kNed];
    float u[kW];
    float E[K * kNB][kW];
    float f[K * kNB];
};

template <int K>
__device__ void load_head(HeadSmem<K>& sm, const __nv_bfloat16* __restrict__ w, int64_t oUc, int64_t ou,
                          int64_t oE, int64_t of) {
    for (int i = threadIdx.x; i < kW * kNed; i += blockDim.x) sm.Uc[i / kNed][i % kNed] = bf(w, oUc + i);
    for (int i = threadIdx.x; i < kW; i += blockDim.x) sm.u[i] = bf(w, ou + i);
    for (int i = threadIdx.x; i < K * kNB * kW; i += blockDim.x) sm.E[i / kW][i % kW] = bf(w, oE + i);
    for (int i = threadIdx.x; i < K * kNB; i += blockDim.x) sm.f[i] = bf(w, of + i);
}

// Edge head, one thread per stored pair t = (m, n):
//   u = relu(Pa[m] + Pb[n] + Uc e + u),  o[k] = sum_c b_c (E u + f)[k*8 + c]  (0 on the diagonal);
// U (optional) keeps u for the backward pass.
template <int K>
__global__ void __launch_bounds__(128) k_head_forward(const float* __restrict__ Pa, const float* __restrict__ Pb,
                                                      const float* __restrict__ e, const float* __restrict__ basis,
                                                      const __nv_bfloat16* __restrict__ w, int64_t oUc, int64_t ou,
                                                      int64_t oE, int64_t of, const int* __restrict__ rows,
                                                      const int* __restrict__ cols, int64_t nnz,
                                                      float* __restrict__ o, float* __restrict__ U) {
    __shared__ HeadSmem<K> sm;
    load_head<K>(sm, w, oUc, ou, oE, of);
    __syncthreads();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nnz) return;
    const int m = rows[t], n = cols[t];
    if (m == n) {
#pragma unroll
        for (int k = 0; k < K; ++k) o[t * K + k] = 0.f;
        if (U) {
            float4* Ur = reinterpret_cast<float4*>(U + t * kW);
            for (int q = 0; q < kW / 4; ++q) Ur[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return;
    }
    float ef[kNed], b[kNB];
    load_row<kNed>(e, t, ef);
    load_row<kNB>(basis, t, b);
    float acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float a = 0.f;
#pragma unroll
        for (int c = 0; c < kNB; ++c) a = fmaf(b[c], sm.f[k * kNB + c], a);
        acc[k] = a;
    }
    const float4* pa = reinterpret_cast<const float4*>(Pa + (int64_t)m * kW);
    const float4* pb = reinterpret_cast<const float4*>(Pb + (int64_t)n * kW);
    for (int q = 0; q < kW / 4; ++q) {
        const float4 A4 = __ldg(pa + q), B4 = __ldg(pb + q);
        const float za[4] = {A4.x + B4.x, A4.y + B4.y, A4.z + B4.z, A4.w + B4.w};
        float uq[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int j = 4 * q + r;
            float z = za[r] + sm.u[j];
#pragma unroll
            for (int f = 0; f < kNed; ++f) z = fmaf(sm.Uc[j][f], ef[f], z);
            const float uj = fmaxf(z, 0.f);
            uq[r] = uj;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float et = 0.f;
#pragma unroll
                for (int c = 0; c < kNB; ++c) et = fmaf(b[c], sm.E[k * kNB + c][j], et);
                acc[k] = fmaf(uj, et, acc[k]);
            }
        }
        if (U) reinterpret_cast<float4*>(U + t * kW)[q] = make_float4(uq[0], uq[1], uq[2], uq[3]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) o[t * K + k] = acc[k];
}

// diagonal head g_m = G h_m + g; one thread per (node, output)
__global__ void k_diag_head(const float* __restrict__ H, const __nv_bfloat16* __restrict__ w, int64_t oG,
                            int64_t og, int N, int K, float* __restrict__ g) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * K) return;
    const int m = (int)(t / K), k = (int)(t % K);
    float acc = bf(w, og + k);
    for (int c = 0; c < kW; ++c) acc = fmaf(bf(w, oG + k * kW + c), H[(int64_t)m * kW + c], acc);
    g[t] = acc;
}

// ------------------------------------------------------------------ probe loss

// lossw[p] = 1 / (P |z_p|^2)
__global__ void k_probe_weights(const float2* __restrict__ Z, int nunk, int P, double* __restrict__ lossw) {
    __shared__ double red[256];
    const int p = blockIdx.x;
    double acc = 0;
    for (int i = threadIdx.x; i < nunk; i += 256) {
        float2 v = Z[(int64_t)p * nunk + i];
        acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) lossw[p] = red[0] > 0 ? 1.0 / (P * red[0]) : 0.0;
}

__device__ __forceinline__ float2 warp_sum2(float2 v) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, s);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, s);
    }
    return v;
}

// Per probe p and row m (caller index mc): r = D^{-1} (y + g y + sum_n o_mn y_n) - z,
// RD_p[m] = (2 / (P|z_p|^2)) * (conj(r) D^{-1}) (row vector), lossn[m] = sum_p |r|^2 / (P |z_p|^2).
template <int K>
__global__ void k_probe_residual(const float* __restrict__ o, const float* __restrict__ g,
                                 const double2* __restrict__ minv, const int* __restrict__ row_ptr,
                                 const int* __restrict__ cols, const int* __restrict__ colc,
                                 const int* __restrict__ perm, const float2* __restrict__ Y,
                                 const float2* __restrict__ Z, const double* __restrict__ lossw, int N, int nunk,
                                 int P, float2* __restrict__ RD, double* __restrict__ lossn) {
    const int lane = threadIdx.x & 31;
    const int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (m >= N) return;
    const int mc = perm[m];
    double lsum = 0;
    for (int p = 0; p < P; ++p) {
        const float2* y = Y + (int64_t)p * nunk;
        if (K == 2) {
            float2 acc = mk(0.f, 0.f);
            for (int t = row_ptr[m] + lane; t < row_ptr[m + 1]; t += 32) {
                if (cols[t] == m) continue;
                cfma(acc, mk(o[2 * (int64_t)t], o[2 * (int64_t)t + 1]), y[colc[t]]);
            }
            acc = warp_sum2(acc);
            if (lane == 0) {
                const float2 ym = y[mc];
                float2 tv = ym + acc;
                cfma(tv, mk(g[2 * m], g[2 * m + 1]), ym);
                const double2 di = minv[mc];
                const double2 t2 = make_double2(tv.x, tv.y);
                const float2 zv = Z[(int64_t)p * nunk + mc];
                const double2 r = di * t2 - make_double2(zv.x, zv.y);
                lsum += lossw[p] * (r.x * r.x + r.y * r.y);
                const double2 rd = conj(r) * di;
                const double s = 2.0 * lossw[p];
                RD[(int64_t)p * nunk + mc] = mk((float)(s * rd.x), (float)(s * rd.y));
            }
        } else {
            float2 a0 = mk(0.f, 0.f), a1 = mk(0.f, 0.f);
            for (int t = row_ptr[m] + lane; t < row_ptr[m + 1]; t += 32) {
                if (cols[t] == m) continue;
                const float* ot = o + 8 * (int64_t)t;
                const int nc = colc[t];
                const float2 v0 = y[nc], v1 = y[N + nc];
                cfma(a0, mk(ot[0], ot[4]), v0);
                cfma(a0, mk(ot[1], ot[5]), v1);
                cfma(a1, mk(ot[2], ot[6]), v0);
                cfma(a1, mk(ot[3], ot[7]), v1);
            }
            a0 = warp_sum2(a0);
            a1 = warp_sum2(a1);
            if (lane == 0) {
                const float* gm = g + 8 * (int64_t)m;
                const float2 v0 = y[mc], v1 = y[N + mc];
                float2 t0 = v0 + a0, t1 = v1 + a1;
                cfma(t0, mk(gm[0], gm[4]), v0);
                cfma(t0, mk(gm[1], gm[5]), v1);
                cfma(t1, mk(gm[2], gm[6]), v0);
                cfma(t1, mk(gm[3], gm[7]), v1);
                const double2* d = minv + 4 * (int64_t)mc;
                const double2 T0 = make_double2(t0.x, t0.y), T1 = make_double2(t1.x, t1.y);
                const float2 z0 = Z[(int64_t)p * nunk + mc], z1 = Z[(int64_t)p * nunk + N + mc];
                const double2 r0 = d[0] * T0 + d[1] * T1 - make_double2(z0.x, z0.y);
                const double2 r1 = d[2] * T0 + d[3] * T1 - make_double2(z1.x, z1.y);
                lsum += lossw[p] * (r0.x * r0.x + r0.y * r0.y + r1.x * r1.x + r1.y * r1.y);
                // RD[a] = sum_g conj(r_g) D^{-1}[g][a]
                const double2 q0 = conj(r0) * d[0] + conj(r1) * d[2];
                const double2 q1 = conj(r0) * d[1] + conj(r1) * d[3];
                const double s = 2.0 * lossw[p];
                RD[(int64_t)p * nunk + mc] = mk((float)(s * q0.x), (float)(s * q0.y));
                RD[(int64_t)p * nunk + N + mc] = mk((float)(s * q1.x), (float)(s * q1.y));
            }
        }
    }
    if (lane == 0) lossn[m] = lsum;
}

// dL/do_mn and dL/dg_m: Ge[t][k], Gn[m][k] (real-part and imaginary-part derivatives)
template <int K>
__global__ void k_output_grads(const int* __restrict__ rows, const int* __restrict__ cols,
                               const int* __restrict__ colc, const int* __restrict__ perm,
                               const float2* __restrict__ RD, const float2* __restrict__ Y, int64_t nnz, int N,
                               int nunk, int P, float* __restrict__ Ge, float* __restrict__ Gn) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool node = t >= nnz;
    if (t >= nnz + N) return;
    int mc, nc;
    if (node) {
        const int m = (int)(t - nnz);
        mc = perm[m];
        nc = mc;
    } else {
        if (rows[t] == cols[t]) {
#pragma unroll
            for (int k = 0; k < K; ++k) Ge[t * K + k] = 0.f;
            return;
        }
        mc = perm[rows[t]];
        nc = colc[t];
    }
    float* out = node ? Gn + (t - nnz) * K : Ge + t * K;
    if (K == 2) {
        float2 acc = mk(0.f, 0.f);
        for (int p = 0; p < P; ++p) cfma(acc, RD[(int64_t)p * nunk + mc], Y[(int64_t)p * nunk + nc]);
        out[0] = acc.x;
        out[1] = -acc.y;
    } else {
        float2 acc[4] = {mk(0.f, 0.f), mk(0.f, 0.f), mk(0.f, 0.f), mk(0.f, 0.f)};
        for (int p = 0; p < P; ++p) {
            const float2 r0 = RD[(int64_t)p * nunk + mc], r1 = RD[(int64_t)p * nunk + N + mc];
            const float2 y0 = Y[(int64_t)p * nunk + nc], y1 = Y[(int64_t)p * nunk + N + nc];
            cfma(acc[0], r0, y0);
            cfma(acc[1], r0, y1);
            cfma(acc[2], r1, y0);
            cfma(acc[3], r1, y1);
        }
        for (int k = 0; k < 4; ++k) {
            out[k] = acc[k].x;
            out[4 + k] = -acc[k].y;
        }
    }
}

// ------------------------------------------------------------------ backward kernels

// Edge head backward, one thread per stored pair: dz_j = [u_j > 0] sum_k Ge[k] sum_c b_c E[k*8+c][j]
template <int K>
__global__ void __launch_bounds__(128) k_head_backward(const float* __restrict__ U, const float* __restrict__ Ge,
                                                       const float* __restrict__ basis,
                                                       const __nv_bfloat16* __restrict__ w, int64_t oUc,
                                                       int64_t ou, int64_t oE, int64_t of,
                                                       const int* __restrict__ rows, const int* __restrict__ cols,
                                                       int64_t nnz, float* __restrict__ DZ) {
    __shared__ HeadSmem<K> sm;
    load_head<K>(sm, w, oUc, ou, oE, of);
    __syncthreads();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nnz) return;
    float4* dz4 = reinterpret_cast<float4*>(DZ + t * kW);
    if (rows[t] == cols[t]) {
        for (int q = 0; q < kW / 4; ++q) dz4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    float b[kNB], ge[K];
    load_row<kNB>(basis, t, b);
#pragma unroll
    for (int k = 0; k < K; ++k) ge[k] = Ge[t * K + k];
    // fold the output gradient into one weight per (k, c): gb[k*8+c] = Ge[k] b_c
    const float4* u4 = reinterpret_cast<const float4*>(U + t * kW);
    for (int q = 0; q < kW / 4; ++q) {
        const float4 uu = __ldg(u4 + q);
        const float uv[4] = {uu.x, uu.y, uu.z, uu.w};
        float dz[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int j = 4 * q + r;
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float et = 0.f;
#pragma unroll
                for (int c = 0; c < kNB; ++c) et = fmaf(b[c], sm.E[k * kNB + c][j], et);
                s = fmaf(ge[k], et, s);
            }
            dz[r] = uv[r] > 0.f ? s : 0.f;
        }
        dz4[q] = make_float4(dz[0], dz[1], dz[2], dz[3]);
    }
}

// dza[m] = sum_{t in row m} DZ[t], dzb[m] = sum_{t in row m} DZ[trans t]; one warp per node
__global__ void k_head_node_back(const float* __restrict__ DZ, const int* __restrict__ row_ptr,
                                 const int* __restrict__ trans, int N, float* __restrict__ dza,
                                 float* __restrict__ dzb) {
    const int lane = threadIdx.x & 31;
    const int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (m >= N) return;
    float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
    for (int t = row_ptr[m]; t < row_ptr[m + 1]; ++t) {
        const int64_t tr = trans[t];
        a0 += DZ[(int64_t)t * kW + lane];
        a1 += DZ[(int64_t)t * kW + lane + 32];
        b0 += DZ[tr * kW + lane];
        b1 += DZ[tr * kW + lane + 32];
    }
    dza[(int64_t)m * kW + lane] = a0;
    dza[(int64_t)m * kW + lane + 32] = a1;
    dzb[(int64_t)m * kW + lane] = b0;
    dzb[(int64_t)m * kW + lane + 32] = b1;
}

// dH[m][c] += sum_k Gn[m][k] G[k][c]
__global__ void k_diag_head_back(const float* __restrict__ Gn, const __nv_bfloat16* __restrict__ w, int64_t oG,
                                 int N, int K, float* __restrict__ dH) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * kW) return;
    const int m = (int)(t / kW), c = (int)(t % kW);
    float acc = dH[t];
    for (int k = 0; k < K; ++k) acc = fmaf(Gn[(int64_t)m * K + k], bf(w, oG + k * kW + c), acc);
    dH[t] = acc;
}

// dU = dH * (H_l > 0); dS = dU / deg
__global__ void k_relu_back(const float* __restrict__ dH, const float* __restrict__ Hl,
                            const float* __restrict__ deginv, int N, float* __restrict__ dU, float* __restrict__ dS) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * kW) return;
    const float v = Hl[t] > 0.f ? dH[t] : 0.f;
    dU[t] = v;
    if (dS) dS[t] = v * deginv[t / kW];
}

// Message backward for layer l, one warp per node n over its row (near pattern symmetric):
//   dP[n] = sum_{m != n} dS[m] * [B h_n + C e_mn + c > 0],  per-warp partials of dC (64 x 16) and dc (64).
__global__ void k_edge_backward(const float* __restrict__ P, const float* __restrict__ e,
                                const __nv_bfloat16* __restrict__ w, int64_t oC, int64_t oc,
                                const int* __restrict__ row_ptr, const int* __restrict__ cols,
                                const int* __restrict__ trans, const float* __restrict__ dS, int N,
                                float* __restrict__ dP, float* __restrict__ part) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    float C0[kNed], C1[kNed], aC0[kNed], aC1[kNed];
    for (int f = 0; f < kNed; ++f) {
        C0[f] = bf(w, oC + lane * kNed + f);
        C1[f] = bf(w, oC + (lane + 32) * kNed + f);
        aC0[f] = aC1[f] = 0.f;
    }
    const float cb0 = bf(w, oc + lane), cb1 = bf(w, oc + lane + 32);
    float ac0 = 0.f, ac1 = 0.f;
    for (int n = warp; n < N; n += nwarp) {
        const float p0 = P[(int64_t)n * kW + lane] + cb0, p1 = P[(int64_t)n * kW + lane + 32] + cb1;
        float d0 = 0.f, d1 = 0.f;
        auto edge = [&](int t) {
            const int m = cols[t];
            const bool keep = m != n;   // the self pair contributes exact zeros (branch-free)
            const int tr = trans[t];  // edge (m, n) in row m
            float ef[kNed];
            load_row<kNed>(e, tr, ef);
            const float ds0 = dS[(int64_t)m * kW + lane], ds1 = dS[(int64_t)m * kW + lane + 32];
            float w0 = p0, w1 = p1;
#pragma unroll
            for (int f = 0; f < kNed; ++f) {
                w0 = fmaf(C0[f], ef[f], w0);
                w1 = fmaf(C1[f], ef[f], w1);
            }
            const float g0 = (keep && w0 > 0.f) ? ds0 : 0.f;
            const float g1 = (keep && w1 > 0.f) ? ds1 : 0.f;
            d0 += g0;
            d1 += g1;
#pragma unroll
            for (int f = 0; f < kNed; ++f) {
                aC0[f] = fmaf(g0, ef[f], aC0[f]);
                aC1[f] = fmaf(g1, ef[f], aC1[f]);
            }
        };
        int t = row_ptr[n];
        const int te = row_ptr[n + 1];
        for (; t + 3 < te; t += 4) {
            edge(t);
            edge(t + 1);
            edge(t + 2);
            edge(t + 3);
        }
        for (; t < te; ++t) edge(t);
        ac0 += d0;
        ac1 += d1;
        dP[(int64_t)n * kW + lane] = d0;
        dP[(int64_t)n * kW + lane + 32] = d1;
    }
    float* pw = part + (int64_t)warp * (kW * kNed + kW);
    for (int f = 0; f < kNed; ++f) {
        pw[lane * kNed + f] = aC0[f];
        pw[(lane + 32) * kNed + f] = aC1[f];
    }
    pw[kW * kNed + lane] = ac0;
    pw[kW * kNed + lane + 32] = ac1;
}

// Per-block partials of a row reduction over R rows in fixed chunks:
//   out[o][i] = sum_r A(r, o) B[r][i] (o < na <= 64, i < nb <= 64), then (bias) sum_r A(r, o).
// MODE 0: A(r, o) = A[r * na + o];  MODE 1: A(r, o) = Ge[r * K + o / 8] * basis[r * 8 + o % 8].
// Thread t owns the 4 x 4 output tile o in [4 (t / 16), +4), i in [4 (t % 16), +4): two 128-bit
// shared loads feed 16 FMAs per row.
template <int MODE>
__global__ void __launch_bounds__(256) k_rows_wgrad(const float* __restrict__ A, const float* __restrict__ Ge,
                                                    const float* __restrict__ basis, int K, int na,
                                                    const float* __restrict__ B, int nb, int bias, int64_t R,
                                                    int64_t chunk, float* __restrict__ part) {
    __shared__ __align__(16) float As[32][kW];
    __shared__ __align__(16) float Bs[32][kW];
    const int t = threadIdx.x;
    const int ot = t >> 4, it = t & 15;
    const bool active = 4 * ot < na && 4 * it < nb;
    const int64_t lo = blockIdx.x * chunk, hi = min(R, lo + chunk);
    float acc[4][4], accb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
    // the next 32-row chunk is loaded into registers while the current one is multiplied
    constexpr int PER = 32 * kW / 256;
    float ra[PER], rb[PER];
    auto load_chunk = [&](int64_t r0) {
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int k = t + 256 * i;
            const int r = k / kW, c = k % kW;
            float va = 0.f, vb = 0.f;
            if (r0 + r < hi) {
                if (c < na) {
                    if (MODE == 0)
                        va = A[(r0 + r) * na + c];
                    else
                        va = Ge[(r0 + r) * K + c / kNB] * basis[(r0 + r) * kNB + c % kNB];
                }
                if (c < nb) vb = B[(r0 + r) * nb + c];
            }
            ra[i] = va;
            rb[i] = vb;
        }
    };
    if (lo < hi) load_chunk(lo);
    for (int64_t r0 = lo; r0 < hi; r0 += 32) {
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int k = t + 256 * i;
            As[k / kW][k % kW] = ra[i];
            Bs[k / kW][k % kW] = rb[i];
        }
        __syncthreads();
        if (r0 + 32 < hi) load_chunk(r0 + 32);
        if (active) {
#pragma unroll 8
            for (int r = 0; r < 32; ++r) {
                const float4 a4 = *reinterpret_cast<const float4*>(&As[r][4 * ot]);
                const float4 b4 = *reinterpret_cast<const float4*>(&Bs[r][4 * it]);
                const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                for (int a = 0; a < 4; ++a) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(av[a], bv[c], acc[a][c]);
                    if (it == 0) accb[a] += av[a];
                }
            }
        }
        __syncthreads();
    }
    const int len = na * nb + (bias ? na : 0);
    float* pb = part + (int64_t)blockIdx.x * len;
    if (active) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int o = 4 * ot + a;
            if (o >= na) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int i = 4 * it + c;
                if (i < nb) pb[o * nb + i] = acc[a][c];
            }
            if (bias && it == 0) pb[na * nb + o] = accb[a];
        }
    }
}

// grad[j] = sum_b part[b][j]: one warp per output, lane-strided partial sums in FP64
// followed by a fixed shuffle tree (deterministic)
__global__ void k_reduce_parts(const float* __restrict__ part, int nparts, int len, float* __restrict__ grad) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (j >= len) return;
    double s = 0;
    for (int b = lane; b < nparts; b += 32) s += part[(int64_t)b * len + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) grad[j] = (float)s;
}

__global__ void k_reduce_loss(const double* __restrict__ lossn, int N, double* __restrict__ out) {
    __shared__ double red[256];
    double s = 0;
    // fixed per-thread strided order, then a fixed tree
    for (int i = threadIdx.x; i < N; i += 256) s += lossn[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) b[t] = __float2bfloat16_rn(a[t]);
}

// ------------------------------------------------------------------ learned preconditioner apply

// vT[u][b] = v[b * vstride + u]
template <class T>
__global__ void k_transpose_rhs(const double2* __restrict__ v, int64_t vstride, int nunk, int nrhs,
                                cplx_t<T>* __restrict__ vT) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nunk * nrhs) return;
    const int u = (int)(t / nrhs), b = (int)(t % nrhs);
    const double2 a = v[(int64_t)b * vstride + u];
    vT[t] = mk((T)a.x, (T)a.y);
}

// z[b][row] = D^{-1} (v + g v + sum_n o_mn v_n); one thread per (internal row, rhs)
template <class T, int K>
__global__ void k_learned_apply(const float* __restrict__ o, const float* __restrict__ g,
                                const double2* __restrict__ minv, const int* __restrict__ row_ptr,
                                const int* __restrict__ cols, const int* __restrict__ colc,
                                const int* __restrict__ perm, const cplx_t<T>* __restrict__ vT, int N, int nunk,
                                int nrhs, cplx_t<T>* __restrict__ z) {
    using C = cplx_t<T>;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * nrhs) return;
    const int m = (int)(t / nrhs), b = (int)(t % nrhs);
    const int mc = perm[m];
    if (K == 2) {
        const C vm = vT[(int64_t)mc * nrhs + b];
        C acc = vm;
        cfma(acc, mk((T)g[2 * m], (T)g[2 * m + 1]), vm);
        for (int e = row_ptr[m]; e < row_ptr[m + 1]; ++e) {
            if (cols[e] == m) continue;
            cfma(acc, mk((T)o[2 * (int64_t)e], (T)o[2 * (int64_t)e + 1]), vT[(int64_t)colc[e] * nrhs + b]);
        }
        const double2 r = minv[mc] * make_double2(acc.x, acc.y);
        z[(int64_t)b * nunk + mc] = mk((T)r.x, (T)r.y);
    } else {
        const C v0 = vT[(int64_t)mc * nrhs + b], v1 = vT[(int64_t)(N + mc) * nrhs + b];
        const float* gm = g + 8 * (int64_t)m;
        C a0 = v0, a1 = v1;
        cfma(a0, mk((T)gm[0], (T)gm[4]), v0);
        cfma(a0, mk((T)gm[1], (T)gm[5]), v1);
        cfma(a1, mk((T)gm[2], (T)gm[6]), v0);
        cfma(a1, mk((T)gm[3], (T)gm[7]), v1);
        for (int e = row_ptr[m]; e < row_ptr[m + 1]; ++e) {
            if (cols[e] == m) continue;
            const float* ot = o + 8 * (int64_t)e;
            const int nc = colc[e];
            const C w0 = vT[(int64_t)nc * nrhs + b], w1 = vT[(int64_t)(N + nc) * nrhs + b];
            cfma(a0, mk((T)ot[0], (T)ot[4]), w0);
            cfma(a0, mk((T)ot[1], (T)ot[5]), w1);
            cfma(a1, mk((T)ot[2], (T)ot[6]), w0);
            cfma(a1, mk((T)ot[3], (T)ot[7]), w1);
        }
        const double2* d = minv + 4 * (int64_t)mc;
        const double2 A0 = make_double2(a0.x, a0.y), A1 = make_double2(a1.x, a1.y);
        const double2 r0 = d[0] * A0 + d[1] * A1, r1 = d[2] * A0 + d[3] * A1;
        z[(int64_t)b * nunk + mc] = mk((T)r0.x, (T)r0.y);
        z[(int64_t)b * nunk + N + mc] = mk((T)r1.x, (T)r1.y);
    }
}

// ------------------------------------------------------------------ host side

template <class T>
static T* galloc(aimx_ctx* ctx, std::vector<void*>& own, size_t n) {
    T* p = (T*)dev_alloc(ctx, sizeof(T) * (n ? n : 1));
    own.push_back(p);
    return p;
}

// near-graph topology and the static (frequency-independent) bases, once per context
static void gnn_topology(aimx_ctx* ctx, cudaStream_t s) {
    if (ctx->form == AIMX_CFIE)
        throw Error{AIMX_E_STATE, "the learned preconditioner covers EFIE and PMCHWT contexts"};
    GnnGraph& G = ctx->gnn;
    if (G.d_rows) return;
    const int N = ctx->N;
    const int64_t nnz = ctx->nnz;
    std::vector<int> rows(nnz), trans(nnz), colc(nnz), dpos(N, -1);
    std::vector<float> deginv(N);
    for (int m = 0; m < N; ++m) {
        int deg = 0;
        for (int t = ctx->row_ptr[m]; t < ctx->row_ptr[m + 1]; ++t) {
            const int n = ctx->cols[t];
            rows[t] = m;
            colc[t] = ctx->perm[n];
            if (n == m)
                dpos[m] = t;
            else
                ++deg;
            const int* b = ctx->cols.data() + ctx->row_ptr[n];
            const int* e = ctx->cols.data() + ctx->row_ptr[n + 1];
            const int* f = std::lower_bound(b, e, m);
            if (f == e || *f != m) throw Error{AIMX_E_STATE, "near pattern is not symmetric"};
            trans[t] = (int)(f - ctx->cols.data());
        }
        if (dpos[m] < 0) throw Error{AIMX_E_STATE, "near pattern lacks a diagonal entry"};
        deginv[m] = 1.0f / (float)std::max(deg, 1);
    }
    auto up = [&](const auto& v) {
        using E = typename std::decay_t<decltype(v)>::value_type;
        E* p = galloc<E>(ctx, G.own, v.size());
        AIMX_CUDA_TRY(cudaMemcpy(p, v.data(), sizeof(E) * v.size(), cudaMemcpyHostToDevice));
        return p;
    };
    G.d_rows = up(rows);
    G.d_trans = up(trans);
    G.d_colc = up(colc);
    G.d_dpos = up(dpos);
    G.d_deginv = up(deginv);
    G.d_x = galloc<float>(ctx, G.own, (size_t)N * kNin);
    G.d_e = galloc<float>(ctx, G.own, (size_t)nnz * kNed);
    G.d_basis = galloc<float>(ctx, G.own, (size_t)nnz * kNB);
    G.d_eta = galloc<double>(ctx, G.own, (size_t)nnz * 3);
    G.d_center = galloc<double>(ctx, G.own, (size_t)N * 3);
    G.d_minv = galloc<double2>(ctx, G.own, (size_t)N * 4);
    G.d_lossn = galloc<double>(ctx, G.own, (size_t)N);
    const double hb = std::cbrt(ctx->h[0] * ctx->h[1] * ctx->h[2]);
    k_edge_eta<<<gb(nnz), 256, 0, s>>>(G.d_rows, ctx->d_cols, G.d_dpos, ctx->f64.na, ctx->f64.np, ctx->f64.nk, nnz,
                                       hb, G.d_eta);
    k_two_hop<<<gb(nnz), 256, 0, s>>>(ctx->d_row_ptr, ctx->d_cols, G.d_rows, G.d_trans, G.d_eta, nnz, G.d_basis);
    AIMX_CUDA_TRY(cudaGetLastError());
}

void gnn_features(aimx_ctx* ctx, double freq, cudaStream_t s) {
    gnn_topology(ctx, s);
    GnnGraph& G = ctx->gnn;
    if (G.feat_freq == freq) return;
    const int N = ctx->N;
    const double hb = std::cbrt(ctx->h[0] * ctx->h[1] * ctx->h[2]);
    const double k = 2.0 * kPi * freq * std::sqrt(ctx->eps_out * ctx->mu_out) / kC0;
    const double contrast =
        ctx->form == AIMX_EFIE ? 1.0 : std::sqrt(ctx->eps_in * ctx->mu_in / (ctx->eps_out * ctx->mu_out));
    k_node_features<<<gb(N), 256, 0, s>>>(ctx->d_xyz, ctx->d_tri, ctx->d_area, ctx->d_btri, ctx->d_blen,
                                          ctx->d_anc, N, ctx->origin[0], ctx->origin[1], ctx->origin[2], ctx->h[0],
                                          ctx->h[1], ctx->h[2], hb, 0.5 * ctx->order, k * hb, contrast, G.d_x,
                                          G.d_center);
    k_edge_features<<<gb(ctx->nnz), 256, 0, s>>>(G.d_rows, ctx->d_cols, G.d_center, G.d_eta, G.d_basis, ctx->nnz,
                                                  hb, k * hb, G.d_e);
    AIMX_CUDA_TRY(cudaGetLastError());
    G.feat_freq = freq;
}

static void ensure_activations(aimx_ctx* ctx, int K, int L) {
    GnnGraph& G = ctx->gnn;
    if (G.d_H && G.K == K && G.L >= L) return;
    if (G.d_H) throw Error{AIMX_E_STATE, "a network of another shape already used this context"};
    const int N = ctx->N;
    G.K = K;
    G.L = L;
    G.d_H = galloc<float>(ctx, G.own, (size_t)(L + 1) * N * kW);
    G.d_P = galloc<float>(ctx, G.own, (size_t)L * N * kW);
    G.d_S = galloc<float>(ctx, G.own, (size_t)N * kW);
    G.d_Pa = galloc<float>(ctx, G.own, (size_t)N * kW);
    G.d_Pb = galloc<float>(ctx, G.own, (size_t)N * kW);
    G.d_o = galloc<float>(ctx, G.own, (size_t)ctx->nnz * K);
    G.d_g = galloc<float>(ctx, G.own, (size_t)N * K);
}

// forward pass with BF16 weights w (layout gnn_layout(K, L)); fills H, P, Pa, Pb, o, g (and U if given)
static void gnn_forward(aimx_ctx* ctx, const __nv_bfloat16* w, int K, int L, float* U, cudaStream_t s) {
    ensure_activations(ctx, K, L);
    GnnGraph& G = ctx->gnn;
    const GnnLayout lay = gnn_layout(K, L);
    const int N = ctx->N;
    const int64_t nnz = ctx->nnz;
    const int64_t NW = (int64_t)N * kW;
    k_input_layer<<<gb(NW), 256, 0, s>>>(G.d_x, w, lay.A0, lay.a0, N, G.d_H);
    const unsigned nodeblk = (unsigned)((N + 63) / 64);
    const unsigned warpblk = (unsigned)std::min<int64_t>((N + 7) / 8, 4096);
    for (int l = 0; l < L; ++l) {
        const float* Hp = G.d_H + l * NW;
        float* Pl = G.d_P + l * NW;
        k_node_gemm<false><<<nodeblk, 256, 0, s>>>(Hp, w + lay.B[l], nullptr, nullptr, Pl, N, 0, 0);
        k_edge_message<<<warpblk, 256, 0, s>>>(Pl, G.d_e, w, lay.C[l], lay.c[l], ctx->d_row_ptr, ctx->d_cols,
                                               G.d_deginv, N, G.d_S);
        k_node_gemm<false><<<nodeblk, 256, 0, s>>>(Hp, w + lay.D[l], w + lay.d[l], G.d_S, G.d_H + (l + 1) * NW, N, 1,
                                                   0);
    }
    const float* HL = G.d_H + L * NW;
    k_node_gemm<false><<<nodeblk, 256, 0, s>>>(HL, w + lay.Ua, nullptr, nullptr, G.d_Pa, N, 0, 0);
    k_node_gemm<false><<<nodeblk, 256, 0, s>>>(HL, w + lay.Ub, nullptr, nullptr, G.d_Pb, N, 0, 0);
    if (K == 2)
        k_head_forward<2><<<gb(nnz, 128), 128, 0, s>>>(G.d_Pa, G.d_Pb, G.d_e, G.d_basis, w, lay.Uc, lay.u, lay.E,
                                                       lay.f, G.d_rows, ctx->d_cols, nnz, G.d_o, U);
    else
        k_head_forward<8><<<gb(nnz, 128), 128, 0, s>>>(G.d_Pa, G.d_Pb, G.d_e, G.d_basis, w, lay.Uc, lay.u, lay.E,
                                                       lay.f, G.d_rows, ctx->d_cols, nnz, G.d_o, U);
    k_diag_head<<<gb((int64_t)N * K), 256, 0, s>>>(HL, w, lay.G, lay.g, N, K, G.d_g);
    AIMX_CUDA_TRY(cudaGetLastError());
    G.out_w = w;
    G.out_freq = G.feat_freq;
}

// D^{-1} of the diagonal preconditioner at freq into G.d_minv (caller order)
static void gnn_diag_inverse(aimx_ctx* ctx, double freq, cudaStream_t s) {
    GnnGraph& G = ctx->gnn;
    if (G.minv_freq == freq) return;
    build_diag_inverse(ctx, freq, G.d_minv, s);
    G.minv_freq = freq;
}

static void reduce_into(const float* part, int nparts, int64_t len, float* grad, cudaStream_t s) {
    k_reduce_parts<<<gb(len * 32), 256, 0, s>>>(part, nparts, (int)len, grad);
}

// fixed-partition row reduction (see k_rows_wgrad) reduced into grad
template <int MODE>
static void rows_wgrad(const float* A, const float* Ge, const float* basis, int K, int na, const float* B, int nb,
                       int bias, int64_t R, float* part, float* grad, cudaStream_t s) {
    const int64_t chunk = std::max<int64_t>((R + kWgradBlocks - 1) / kWgradBlocks, 1);
    k_rows_wgrad<MODE><<<kWgradBlocks, 256, 0, s>>>(A, Ge, basis, K, na, B, nb, bias, R, chunk, part);
    reduce_into(part, kWgradBlocks, (int64_t)na * nb + (bias ? na : 0), grad, s);
}

}  // namespace aimx

// ------------------------------------------------------------------ network object

struct aimx_gnn {
    int K = 2, L = 4;
    aimx::GnnLayout lay;
    float* d_master = nullptr;    // FP32 master weights
    float* d_m1 = nullptr;        // Adam first moments
    float* d_m2 = nullptr;        // Adam second moments
    float* d_grad = nullptr;      // gradient of the last loss evaluation
    __nv_bfloat16* d_w = nullptr; // BF16 weights used by every kernel
    int64_t step = 0;
    // work buffers (grown on demand)
    float* d_part = nullptr;
    int64_t part_cap = 0;
    float2* d_RD = nullptr;
    int64_t rd_cap = 0;
    float* d_Ge = nullptr;
    int64_t ge_cap = 0;
    float* d_Gn = nullptr;
    int64_t gn_cap = 0;
    float* d_node = nullptr;      // 7 node buffers [N][64]: dH, dT, dU, dS, dP, dza, dzb
    int64_t node_cap = 0;
    float* d_U = nullptr;         // [nnz][64] head hidden state of the last forward
    int64_t u_cap = 0;
    float* d_DZ = nullptr;        // [nnz][64] its gradient
    int64_t dz_cap = 0;
    double* d_lossw = nullptr;
    int64_t lossw_cap = 0;
    double* d_scal = nullptr;     // [0] loss, [1] gradient scale
};

namespace aimx {

template <class T>
static void grow(T*& p, int64_t& cap, int64_t need) {
    if (p && cap >= need) return;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc((void**)&p, sizeof(T) * (size_t)std::max<int64_t>(need, 1));
    if (e != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        throw Error{AIMX_E_NOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e)};
    }
    cap = need;
}

static void free_net(aimx_gnn* n) {
    void* ptrs[] = {n->d_master, n->d_m1, n->d_m2,   n->d_grad,  n->d_w, n->d_part, n->d_RD,
                    n->d_Ge,     n->d_Gn, n->d_node, n->d_lossw, n->d_scal, n->d_U, n->d_DZ};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

// scale = min(1, clip / |grad|) (clip <= 0: 1), written to out[0]; fixed summation order
__global__ void k_grad_scale(const float* __restrict__ g, int64_t n, double clip, double* __restrict__ out) {
    __shared__ double red[256];
    double s = 0;
    for (int64_t i = threadIdx.x; i < n; i += 256) s += (double)g[i] * g[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double nrm = sqrt(red[0]);
        out[0] = (clip > 0 && nrm > clip) ? clip / nrm : 1.0;
        out[1] = nrm;
    }
}

__global__ void k_adam_step(float* __restrict__ master, float* __restrict__ m1, float* __restrict__ m2,
                            const float* __restrict__ grad, const double* __restrict__ scale,
                            __nv_bfloat16* __restrict__ wbf, int64_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float g = grad[t] * (float)scale[0];
    const float a = b1 * m1[t] + (1.f - b1) * g;
    const float b = b2 * m2[t] + (1.f - b2) * g * g;
    m1[t] = a;
    m2[t] = b;
    const float v = master[t] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    master[t] = v;
    wbf[t] = __float2bfloat16_rn(v);
}

// Probe loss for (ctx, freq) with the network's BF16 weights; with want_grad the
// gradient of every parameter is left in net->d_grad.  Returns the loss (synchronises s).
static double gnn_loss_grad(aimx_gnn* net, aimx_ctx* ctx, double freq, int P, const float2* Z, const float2* Y,
                            bool want_grad, cudaStream_t s) {
    const int K = net->K, L = net->L, N = ctx->N, nunk = ctx->nunk;
    const int64_t nnz = ctx->nnz;
    const int64_t NW = (int64_t)N * kW;
    gnn_features(ctx, freq, s);
    gnn_diag_inverse(ctx, freq, s);
    if (want_grad) grow(net->d_U, net->u_cap, nnz * kW);
    gnn_forward(ctx, net->d_w, K, L, want_grad ? net->d_U : nullptr, s);
    GnnGraph& G = ctx->gnn;
    const GnnLayout& lay = net->lay;
    grow(net->d_lossw, net->lossw_cap, P);
    grow(net->d_RD, net->rd_cap, (int64_t)P * nunk);
    k_probe_weights<<<P, 256, 0, s>>>(Z, nunk, P, net->d_lossw);
    const unsigned rowblk = gb((int64_t)N * 32);
    if (K == 2)
        k_probe_residual<2><<<rowblk, 256, 0, s>>>(G.d_o, G.d_g, G.d_minv, ctx->d_row_ptr, ctx->d_cols, G.d_colc,
                                                   ctx->d_perm, Y, Z, net->d_lossw, N, nunk, P, net->d_RD, G.d_lossn);
    else
        k_probe_residual<8><<<rowblk, 256, 0, s>>>(G.d_o, G.d_g, G.d_minv, ctx->d_row_ptr, ctx->d_cols, G.d_colc,
                                                   ctx->d_perm, Y, Z, net->d_lossw, N, nunk, P, net->d_RD, G.d_lossn);
    k_reduce_loss<<<1, 256, 0, s>>>(G.d_lossn, N, net->d_scal);
    AIMX_CUDA_TRY(cudaGetLastError());
    if (want_grad) {
        grow(net->d_Ge, net->ge_cap, nnz * K);
        grow(net->d_Gn, net->gn_cap, (int64_t)N * K);
        grow(net->d_node, net->node_cap, 7 * NW);
        grow(net->d_DZ, net->dz_cap, nnz * kW);
        grow(net->d_part, net->part_cap,
             std::max<int64_t>((int64_t)kPersistWarps * (kW * kNed + kW), (int64_t)kWgradBlocks * (kW * kW + kW)));
        float* dH = net->d_node;
        float* dT = dH + NW;
        float* dU = dT + NW;
        float* dS = dU + NW;
        float* dP = dS + NW;
        float* dza = dP + NW;
        float* dzb = dza + NW;
        const __nv_bfloat16* w = net->d_w;
        float* grad = net->d_grad;
        float* part = net->d_part;
        if (K == 2)
            k_output_grads<2><<<gb(nnz + N), 256, 0, s>>>(G.d_rows, ctx->d_cols, G.d_colc, ctx->d_perm, net->d_RD, Y,
                                                         nnz, N, nunk, P, net->d_Ge, net->d_Gn);
        else
            k_output_grads<8><<<gb(nnz + N), 256, 0, s>>>(G.d_rows, ctx->d_cols, G.d_colc, ctx->d_perm, net->d_RD, Y,
                                                         nnz, N, nunk, P, net->d_Ge, net->d_Gn);
        const float* HL = G.d_H + L * NW;
        // edge head: dE, df; dz; dUc, du; dza, dzb; dUa, dUb
        rows_wgrad<1>(nullptr, net->d_Ge, G.d_basis, K, K * kNB, net->d_U, kW, 1, nnz, part, grad + lay.E, s);
        if (K == 2)
            k_head_backward<2><<<gb(nnz, 128), 128, 0, s>>>(net->d_U, net->d_Ge, G.d_basis, w, lay.Uc, lay.u, lay.E,
                                                            lay.f, G.d_rows, ctx->d_cols, nnz, net->d_DZ);
        else
            k_head_backward<8><<<gb(nnz, 128), 128, 0, s>>>(net->d_U, net->d_Ge, G.d_basis, w, lay.Uc, lay.u, lay.E,
                                                            lay.f, G.d_rows, ctx->d_cols, nnz, net->d_DZ);
        rows_wgrad<0>(net->d_DZ, nullptr, nullptr, 0, kW, G.d_e, kNed, 1, nnz, part, grad + lay.Uc, s);
        k_head_node_back<<<gb((int64_t)N * 32), 256, 0, s>>>(net->d_DZ, ctx->d_row_ptr, G.d_trans, N, dza, dzb);
        rows_wgrad<0>(dza, nullptr, nullptr, 0, kW, HL, kW, 0, N, part, grad + lay.Ua, s);
        rows_wgrad<0>(dzb, nullptr, nullptr, 0, kW, HL, kW, 0, N, part, grad + lay.Ub, s);
        // diagonal head: dG, dg
        rows_wgrad<0>(net->d_Gn, nullptr, nullptr, 0, K, HL, kW, 1, N, part, grad + lay.G, s);
        // dH_L = dza Ua + dzb Ub + Gn G
        const unsigned nodeblk = (unsigned)((N + 63) / 64);
        k_node_gemm<true><<<nodeblk, 256, 0, s>>>(dza, w + lay.Ua, nullptr, nullptr, dH, N, 0, 0);
        k_node_gemm<true><<<nodeblk, 256, 0, s>>>(dzb, w + lay.Ub, nullptr, nullptr, dH, N, 0, 1);
        k_diag_head_back<<<gb(NW), 256, 0, s>>>(net->d_Gn, w, lay.G, N, K, dH);
        const unsigned pblk = kPersistWarps / 8;
        for (int l = L - 1; l >= 0; --l) {
            const float* Hl = G.d_H + (l + 1) * NW;
            const float* Hp = G.d_H + l * NW;
            const float* Pl = G.d_P + l * NW;
            k_relu_back<<<gb(NW), 256, 0, s>>>(dH, Hl, G.d_deginv, N, dU, dS);
            rows_wgrad<0>(dU, nullptr, nullptr, 0, kW, Hp, kW, 1, N, part, grad + lay.D[l], s);
            k_edge_backward<<<pblk, 256, 0, s>>>(Pl, G.d_e, w, lay.C[l], lay.c[l], ctx->d_row_ptr, ctx->d_cols,
                                                 G.d_trans, dS, N, dP, part);
            reduce_into(part, kPersistWarps, kW * kNed + kW, grad + lay.C[l], s);
            rows_wgrad<0>(dP, nullptr, nullptr, 0, kW, Hp, kW, 0, N, part, grad + lay.B[l], s);
            k_node_gemm<true><<<nodeblk, 256, 0, s>>>(dU, w + lay.D[l], nullptr, nullptr, dT, N, 0, 0);
            k_node_gemm<true><<<nodeblk, 256, 0, s>>>(dP, w + lay.B[l], nullptr, nullptr, dT, N, 0, 1);
            std::swap(dH, dT);
        }
        k_relu_back<<<gb(NW), 256, 0, s>>>(dH, G.d_H, G.d_deginv, N, dU, nullptr);
        rows_wgrad<0>(dU, nullptr, nullptr, 0, kW, G.d_x, kNin, 1, N, part, grad + lay.A0, s);
        AIMX_CUDA_TRY(cudaGetLastError());
    }
    double loss = 0;
    AIMX_CUDA_TRY(cudaMemcpyAsync(&loss, net->d_scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    AIMX_CUDA_TRY(cudaStreamSynchronize(s));
    return loss;
}

// ------------------------------------------------------------------ solver hooks

void learned_prepare(aimx_ctx* ctx, double freq, cudaStream_t s) {
    GnnGraph& G = ctx->gnn;
    if (!G.d_watt) throw Error{AIMX_E_STATE, "no learned preconditioner attached (aimx_gnn_attach)"};
    gnn_features(ctx, freq, s);
    gnn_diag_inverse(ctx, freq, s);
    if (G.out_w == G.d_watt && G.out_freq == freq) return;
    gnn_forward(ctx, G.d_watt, G.att_K, G.att_L, nullptr, s);
    G.out_w = G.d_watt;
    G.out_freq = freq;
}

template <class T>
void learned_apply(aimx_ctx* ctx, const double2* v, int64_t vstride, cplx_t<T>* z, int nrhs, cudaStream_t s) {
    GnnGraph& G = ctx->gnn;
    const int N = ctx->N, nunk = ctx->nunk;
    const size_t need = sizeof(cplx_t<T>) * (size_t)nunk * nrhs;
    if (G.vT_bytes < need) {
        if (G.d_vT) dev_free(ctx, G.d_vT);
        G.d_vT = nullptr;
        G.vT_bytes = 0;
        G.d_vT = dev_alloc(ctx, need);
        G.vT_bytes = need;
    }
    cplx_t<T>* vT = (cplx_t<T>*)G.d_vT;
    k_transpose_rhs<T><<<gb((int64_t)nunk * nrhs), 256, 0, s>>>(v, vstride, nunk, nrhs, vT);
    if (G.att_K == 2)
        k_learned_apply<T, 2><<<gb((int64_t)N * nrhs), 256, 0, s>>>(G.d_o, G.d_g, G.d_minv, ctx->d_row_ptr,
                                                                   ctx->d_cols, G.d_colc, ctx->d_perm, vT, N, nunk,
                                                                   nrhs, z);
    else
        k_learned_apply<T, 8><<<gb((int64_t)N * nrhs), 256, 0, s>>>(G.d_o, G.d_g, G.d_minv, ctx->d_row_ptr,
                                                                   ctx->d_cols, G.d_colc, ctx->d_perm, vT, N, nunk,
                                                                   nrhs, z);
    AIMX_CUDA_TRY(cudaGetLastError());
}

template void learned_apply<float>(aimx_ctx*, const double2*, int64_t, float2*, int, cudaStream_t);
template void learned_apply<double>(aimx_ctx*, const double2*, int64_t, double2*, int, cudaStream_t);

void gnn_free(aimx_ctx* ctx) {
    GnnGraph& G = ctx->gnn;
    for (void* p : G.own)
        if (p) cudaFree(p);
    G.own.clear();
    if (G.d_vT) cudaFree(G.d_vT);
    if (G.d_watt) cudaFree(G.d_watt);
    G = GnnGraph();
}

}  // namespace aimx

using namespace aimx;

static int gnn_fail(aimx_ctx* ctx, const Error& e) {
    if (ctx) ctx->last_error = e.msg;
    return e.code;
}

extern "C" {

int aimx_gnn_create(int formulation, int layers, aimx_gnn** out) {
    if (!out) return AIMX_E_ARG;
    *out = nullptr;
    if ((formulation != AIMX_EFIE && formulation != AIMX_PMCHWT) || layers < 1 || layers > kMaxLayers)
        return AIMX_E_ARG;
    aimx_gnn* n = new (std::nothrow) aimx_gnn();
    if (!n) return AIMX_E_NOMEM;
    n->K = formulation == AIMX_EFIE ? 2 : 8;
    n->L = layers;
    n->lay = gnn_layout(n->K, n->L);
    const int64_t np = n->lay.total;
    bool ok = cudaMalloc((void**)&n->d_master, sizeof(float) * np) == cudaSuccess &&
              cudaMalloc((void**)&n->d_m1, sizeof(float) * np) == cudaSuccess &&
              cudaMalloc((void**)&n->d_m2, sizeof(float) * np) == cudaSuccess &&
              cudaMalloc((void**)&n->d_grad, sizeof(float) * np) == cudaSuccess &&
              cudaMalloc((void**)&n->d_w, sizeof(__nv_bfloat16) * np) == cudaSuccess &&
              cudaMalloc((void**)&n->d_scal, sizeof(double) * 4) == cudaSuccess;
    if (ok)
        ok = cudaMemset(n->d_master, 0, sizeof(float) * np) == cudaSuccess &&
             cudaMemset(n->d_m1, 0, sizeof(float) * np) == cudaSuccess &&
             cudaMemset(n->d_m2, 0, sizeof(float) * np) == cudaSuccess &&
             cudaMemset(n->d_grad, 0, sizeof(float) * np) == cudaSuccess &&
             cudaMemset(n->d_w, 0, sizeof(__nv_bfloat16) * np) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_net(n);
        delete n;
        return AIMX_E_NOMEM;
    }
    *out = n;
    return AIMX_OK;
}

int aimx_gnn_destroy(aimx_gnn* net) {
    if (!net) return AIMX_OK;
    cudaDeviceSynchronize();
    free_net(net);
    delete net;
    return AIMX_OK;
}

int64_t aimx_gnn_num_params(const aimx_gnn* net) { return net ? net->lay.total : 0; }

int aimx_gnn_set_params(aimx_gnn* net, const float* host, int64_t n) {
    if (!net || !host || n != net->lay.total) return AIMX_E_ARG;
    if (cudaMemcpy(net->d_master, host, sizeof(float) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(net->d_m1, 0, sizeof(float) * n) != cudaSuccess ||
        cudaMemset(net->d_m2, 0, sizeof(float) * n) != cudaSuccess) {
        cudaGetLastError();
        return AIMX_E_CUDA;
    }
    k_to_bf16<<<gb(n), 256>>>(net->d_master, net->d_w, n);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return AIMX_E_CUDA;
    }
    net->step = 0;
    return AIMX_OK;
}

int aimx_gnn_get_params(const aimx_gnn* net, float* host, int64_t n) {
    if (!net || !host || n != net->lay.total) return AIMX_E_ARG;
    if (cudaMemcpy(host, net->d_master, sizeof(float) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return AIMX_E_CUDA;
    }
    return AIMX_OK;
}

static int check_pair(const aimx_gnn* net, const aimx_ctx* ctx) {
    if (!net || !ctx) return AIMX_E_ARG;
    if (ctx->form == AIMX_CFIE) return AIMX_E_STATE;   // the learned preconditioner covers EFIE and PMCHWT
    if ((ctx->form == AIMX_EFIE) != (net->K == 2)) return AIMX_E_ARG;
    return AIMX_OK;
}

int aimx_gnn_loss_grad(aimx_gnn* net, aimx_ctx* ctx, double freq, int nprobe, const void* Z, const void* Y,
                       double* loss, float* grad, void* stream) {
    int rc = check_pair(net, ctx);
    if (rc) return rc;
    if (nprobe <= 0 || !Z || !Y || !(freq > 0)) return gnn_fail(ctx, Error{AIMX_E_ARG, "aimx_gnn_loss_grad: bad argument"});
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    try {
        double L = gnn_loss_grad(net, ctx, freq, nprobe, (const float2*)Z, (const float2*)Y, grad != nullptr, s);
        if (loss) *loss = L;
        if (grad)
            AIMX_CUDA_TRY(cudaMemcpy(grad, net->d_grad, sizeof(float) * net->lay.total, cudaMemcpyDeviceToHost));
    } catch (const Error& e) {
        return gnn_fail(ctx, e);
    }
    return AIMX_OK;
}

int aimx_gnn_train_step(aimx_gnn* net, aimx_ctx* ctx, double freq, int nprobe, const void* Z, const void* Y,
                        const aimx_adam_opts* opt, double* loss, void* stream) {
    int rc = check_pair(net, ctx);
    if (rc) return rc;
    if (nprobe <= 0 || !Z || !Y || !(freq > 0) || !opt || !(opt->lr > 0))
        return gnn_fail(ctx, Error{AIMX_E_ARG, "aimx_gnn_train_step: bad argument"});
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    try {
        double L = gnn_loss_grad(net, ctx, freq, nprobe, (const float2*)Z, (const float2*)Y, true, s);
        if (loss) *loss = L;
        const double b1 = opt->beta1 > 0 ? opt->beta1 : 0.9, b2 = opt->beta2 > 0 ? opt->beta2 : 0.999;
        const double eps = opt->eps > 0 ? opt->eps : 1e-8;
        net->step += 1;
        const double c1 = 1.0 - std::pow(b1, (double)net->step), c2 = 1.0 - std::pow(b2, (double)net->step);
        const int64_t np = net->lay.total;
        k_grad_scale<<<1, 256, 0, s>>>(net->d_grad, np, opt->clip, net->d_scal + 2);
        k_adam_step<<<gb(np), 256, 0, s>>>(net->d_master, net->d_m1, net->d_m2, net->d_grad, net->d_scal + 2,
                                           net->d_w, np, (float)opt->lr, (float)b1, (float)b2, (float)eps, (float)c1,
                                           (float)c2);
        AIMX_CUDA_TRY(cudaGetLastError());
        AIMX_CUDA_TRY(cudaStreamSynchronize(s));
    } catch (const Error& e) {
        return gnn_fail(ctx, e);
    }
    return AIMX_OK;
}

int aimx_gnn_attach(aimx_ctx* ctx, const aimx_gnn* net) {
    if (!ctx) return AIMX_E_ARG;
    GnnGraph& G = ctx->gnn;
    try {
        if (!net) {
            if (G.d_watt) dev_free(ctx, G.d_watt);
            G.d_watt = nullptr;
            G.out_w = nullptr;
            return AIMX_OK;
        }
        int rc = check_pair(net, ctx);
        if (rc) return rc;
        const int64_t np = net->lay.total;
        if (G.d_watt && G.att_np != np) {
            dev_free(ctx, G.d_watt);
            G.d_watt = nullptr;
        }
        if (!G.d_watt) G.d_watt = (__nv_bfloat16*)dev_alloc(ctx, sizeof(__nv_bfloat16) * np);
        AIMX_CUDA_TRY(cudaMemcpy(G.d_watt, net->d_w, sizeof(__nv_bfloat16) * np, cudaMemcpyDeviceToDevice));
        G.att_np = np;
        G.att_K = net->K;
        G.att_L = net->L;
        G.out_w = nullptr;
    } catch (const Error& e) {
        return gnn_fail(ctx, e);
    }
    return AIMX_OK;
}

int aimx_gnn_features(aimx_ctx* ctx, double freq, float* node, float* edge, float* basis, int32_t* rows,
                      int32_t* cols) {
    if (!ctx || !(freq > 0)) return AIMX_E_ARG;
    try {
        gnn_features(ctx, freq, 0);
        GnnGraph& G = ctx->gnn;
        const int N = ctx->N;
        const int64_t nnz = ctx->nnz;
        if (node) {
            std::vector<float> x((size_t)N * kNin);
            AIMX_CUDA_TRY(cudaMemcpy(x.data(), G.d_x, sizeof(float) * x.size(), cudaMemcpyDeviceToHost));
            for (int i = 0; i < N; ++i)
                std::memcpy(node + (size_t)ctx->perm[i] * kNin, &x[(size_t)i * kNin], sizeof(float) * kNin);
        }
        if (edge) AIMX_CUDA_TRY(cudaMemcpy(edge, G.d_e, sizeof(float) * nnz * kNed, cudaMemcpyDeviceToHost));
        if (basis) AIMX_CUDA_TRY(cudaMemcpy(basis, G.d_basis, sizeof(float) * nnz * kNB, cudaMemcpyDeviceToHost));
        for (int m = 0; m < N; ++m)
            for (int t = ctx->row_ptr[m]; t < ctx->row_ptr[m + 1]; ++t) {
                if (rows) rows[t] = ctx->perm[m];
                if (cols) cols[t] = ctx->perm[ctx->cols[t]];
            }
    } catch (const Error& e) {
        return gnn_fail(ctx, e);
    }
    return AIMX_OK;
}

int aimx_gnn_outputs(aimx_ctx* ctx, const aimx_gnn* net, double freq, float* o, float* g) {
    int rc = check_pair(net, ctx);
    if (rc) return rc;
    if (!(freq > 0)) return AIMX_E_ARG;
    try {
        gnn_features(ctx, freq, 0);
        gnn_forward(ctx, net->d_w, net->K, net->L, nullptr, 0);
        GnnGraph& G = ctx->gnn;
        G.out_w = nullptr;
        const int N = ctx->N, K = net->K;
        if (o) AIMX_CUDA_TRY(cudaMemcpy(o, G.d_o, sizeof(float) * ctx->nnz * K, cudaMemcpyDeviceToHost));
        if (g) {
            std::vector<float> gv((size_t)N * K);
            AIMX_CUDA_TRY(cudaMemcpy(gv.data(), G.d_g, sizeof(float) * gv.size(), cudaMemcpyDeviceToHost));
            for (int i = 0; i < N; ++i)
                std::memcpy(g + (size_t)ctx->perm[i] * K, &gv[(size_t)i * K], sizeof(float) * K);
        }
    } catch (const Error& e) {
        return gnn_fail(ctx, e);
    }
    return AIMX_OK;
}

}  // extern "C"
