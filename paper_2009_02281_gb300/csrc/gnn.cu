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
// BF16 (an FP32 master copy and FP32 Adam moments are kept), activations and
// accumulations are FP32, and the 64-wide contractions (node GEMMs, the edge
// head and its backward, the weight-gradient row reductions) run on the tensor
// cores with BF16 operands (FP32 operands split into two BF16 terms) and FP32
// accumulation.  Every weight-gradient reduction uses a fixed partition and a
// fixed summation order, so a training step is deterministic.
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
constexpr int kPersistWarps = 1824;  // fixed warp count of the reducing per-node kernels (12 per SM)
constexpr int kWgradBlocks = 456;    // fixed block count of the row-reduction kernels (3 per SM)

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

// ------------------------------------------------------------------ tensor-core contractions
//
// The 64-wide contractions run on the tensor cores as mma.sync m16n8k16 with BF16 operands
// and FP32 accumulation.  Weights are BF16 numbers and enter exactly.  An FP32 activation or
// gradient x enters as the sum of two BF16 numbers, hi = bf16(x) and lo = bf16(x - hi), which
// together carry x to about 2^-17 of its magnitude: a product with an exact weight takes two
// MMAs (hi, lo) and a product of two split operands three (hi hi, hi lo, lo hi; lo lo lies
// below the FP32 rounding of the sum).  Each accumulator sees its MMAs in a fixed order, so
// results stay bitwise reproducible.
//
// Fragments of m16n8k16 (g = lane / 4, q = lane % 4; a 32-bit register holds two BF16 values,
// the lower column or row index in its low half):
//   A (16 x 16, row major)    a0 = (g, 2q..2q+1)  a1 = (g+8, 2q..)  a2 = (g, 2q+8..)  a3 = (g+8, 2q+8..)
//   B (16 x 8, column major)  b0 = (k = 2q..2q+1, n = g)  b1 = (k = 2q+8.., n = g)
//   C (16 x 8, FP32)          c0, c1 = (g, 2q..2q+1)  c2, c3 = (g+8, 2q..2q+1)

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 h) {
    uint32_t r;
    memcpy(&r, &h, sizeof(r));
    return r;
}

// (x0, x1) -> BF16 pairs hi and lo with x = hi + lo to about 2^-17 |x|
__device__ __forceinline__ void split_bf2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const float2 hf = __bfloat1622float2(h);
    hi = bf2_bits(h);
    lo = bf2_bits(__floats2bfloat162_rn(x0 - hf.x, x1 - hf.y));
}

// two consecutive BF16 values (even element offset) as one B-fragment register
__device__ __forceinline__ uint32_t ld_bf2(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ float2 ld_f2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// d += A B on the tensor cores (m16n8k16, BF16 in, FP32 accumulate)
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A fragment (hi, lo) of rows (ra, rb) of a row-major FP32 matrix, columns [c0, c0 + 16)
__device__ __forceinline__ void a_frag_rows(const float* ra, const float* rb, int c0, int q, uint32_t (&hi)[4],
                                            uint32_t (&lo)[4]) {
    const float2 x0 = ld_f2(ra + c0 + 2 * q), x1 = ld_f2(rb + c0 + 2 * q);
    const float2 x2 = ld_f2(ra + c0 + 2 * q + 8), x3 = ld_f2(rb + c0 + 2 * q + 8);
    split_bf2(x0.x, x0.y, hi[0], lo[0]);
    split_bf2(x1.x, x1.y, hi[1], lo[1]);
    split_bf2(x2.x, x2.y, hi[2], lo[2]);
    split_bf2(x3.x, x3.y, hi[3], lo[3]);
}

// Y[n][o] (=|+=) act( sum_i X[n][i] W'[o][i] + bias[o] + add[n][o] ), 64 x 64 BF16 weights:
// W' = W (row-major [out][in]) or, with TRANS, W^T.  W' is staged in shared memory as the B
// operand; each warp owns 16 nodes and all 64 outputs, a block of 4 warps 64 nodes.
template <bool TRANS>
__global__ void __launch_bounds__(128) k_node_gemm(const float* __restrict__ X, const __nv_bfloat16* __restrict__ W,
                                                   const __nv_bfloat16* __restrict__ bias,
                                                   const float* __restrict__ add, float* __restrict__ Y, int N,
                                                   int relu, int accumulate) {
    __shared__ __align__(16) __nv_bfloat16 Ws[kW][kW + 8];   // W'[o][i]; pitch 36 words: conflict-free fragments
    for (int k = threadIdx.x; k < kW * kW; k += blockDim.x) {
        const int r = k / kW, c = k % kW;
        if (TRANS)
            Ws[c][r] = W[k];
        else
            Ws[r][c] = W[k];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int n0 = blockIdx.x * 64 + (threadIdx.x >> 5) * 16;
    if (n0 >= N) return;
    const int na = min(n0 + g, N - 1), nb = min(n0 + g + 8, N - 1);
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[nt][i] = 0.f;
#pragma unroll
    for (int kt = 0; kt < kW / 16; ++kt) {
        uint32_t ah[4], al[4];
        a_frag_rows(X + (int64_t)na * kW, X + (int64_t)nb * kW, 16 * kt, q, ah, al);
        uint32_t b[8][2];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            b[nt][0] = ld_bf2(&Ws[nt * 8 + g][16 * kt + 2 * q]);
            b[nt][1] = ld_bf2(&Ws[nt * 8 + g][16 * kt + 2 * q + 8]);
        }
        // one pass per operand half over the eight independent accumulators, so that
        // consecutive MMAs never wait on each other
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) mma_bf16(acc[nt], ah, b[nt][0], b[nt][1]);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) mma_bf16(acc[nt], al, b[nt][0], b[nt][1]);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int n = n0 + g + 8 * h;
        if (n >= N) continue;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int o = nt * 8 + 2 * q;
            const int64_t idx = (int64_t)n * kW + o;
            float v0 = acc[nt][2 * h], v1 = acc[nt][2 * h + 1];
            if (bias) {
                v0 += __bfloat162float(bias[o]);
                v1 += __bfloat162float(bias[o + 1]);
            }
            if (add) {
                const float2 a2 = ld_f2(add + idx);
                v0 += a2.x;
                v1 += a2.y;
            }
            if (relu) {
                v0 = fmaxf(v0, 0.f);
                v1 = fmaxf(v1, 0.f);
            }
            if (accumulate) {
                const float2 y2 = ld_f2(Y + idx);
                v0 = y2.x + v0;
                v1 = y2.y + v1;
            }
            *reinterpret_cast<float2*>(Y + idx) = make_float2(v0, v1);
        }
    }
}

// S[m] = (1/deg_m) sum_{n != m} relu(P[n] + C e_mn + c) on the tensor cores: one warp per node m
// (warp-strided), its CSR row in tiles of 16 edges.  Per tile z = P[n] + c + e C^T
// (e [16 x 16] split hi/lo, C^T exact: 8 n-tiles), masked ReLU summed per lane; at the end of
// the row the 8 lanes of each column pair combine with a fixed shuffle tree.
__global__ void __launch_bounds__(256) k_edge_message(const float* __restrict__ P, const float* __restrict__ e,
                                                      const __nv_bfloat16* __restrict__ w, int64_t oC, int64_t oc,
                                                      const int* __restrict__ row_ptr, const int* __restrict__ cols,
                                                      const float* __restrict__ deginv, int N, float* __restrict__ S) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    uint32_t cb[8][2];   // B fragments of C^T: k = feature, n = channel
    float cv[8][2];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const __nv_bfloat16* cr = w + oC + (int64_t)(nt * 8 + g) * kNed + 2 * q;
        cb[nt][0] = ld_bf2(cr);
        cb[nt][1] = ld_bf2(cr + 8);
        cv[nt][0] = __bfloat162float(w[oc + nt * 8 + 2 * q]);
        cv[nt][1] = __bfloat162float(w[oc + nt * 8 + 2 * q + 1]);
    }
    for (int m = warp; m < N; m += nwarp) {
        const int ts = row_ptr[m], te = row_ptr[m + 1];
        float s[8][2];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) s[nt][0] = s[nt][1] = 0.f;
        for (int t0 = ts; t0 < te; t0 += 16) {
            const int ta = min(t0 + g, te - 1), tb = min(t0 + g + 8, te - 1);
            const int na = cols[ta], nb = cols[tb];
            const bool ka = t0 + g < te && na != m, kb = t0 + g + 8 < te && nb != m;
            float z[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int j = nt * 8 + 2 * q;
                const float2 pa = ld_f2(P + (int64_t)na * kW + j), pb = ld_f2(P + (int64_t)nb * kW + j);
                z[nt][0] = pa.x + cv[nt][0];
                z[nt][1] = pa.y + cv[nt][1];
                z[nt][2] = pb.x + cv[nt][0];
                z[nt][3] = pb.y + cv[nt][1];
            }
            uint32_t ah[4], al[4];
            a_frag_rows(e + (int64_t)ta * kNed, e + (int64_t)tb * kNed, 0, q, ah, al);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) mma_bf16(z[nt], ah, cb[nt][0], cb[nt][1]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) mma_bf16(z[nt], al, cb[nt][0], cb[nt][1]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                s[nt][0] += (ka ? fmaxf(z[nt][0], 0.f) : 0.f) + (kb ? fmaxf(z[nt][2], 0.f) : 0.f);
                s[nt][1] += (ka ? fmaxf(z[nt][1], 0.f) : 0.f) + (kb ? fmaxf(z[nt][3], 0.f) : 0.f);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                float v = s[nt][c];
                v += __shfl_xor_sync(0xffffffffu, v, 4);
                v += __shfl_xor_sync(0xffffffffu, v, 8);
                v += __shfl_xor_sync(0xffffffffu, v, 16);
                s[nt][c] = v;
            }
        // every lane of a column pair holds the sums; lane (g, q) stores n-tile g
        const float di = deginv[m];
        float2 out = make_float2(0.f, 0.f);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
            if (nt == g) out = make_float2(s[nt][0] * di, s[nt][1] * di);
        *reinterpret_cast<float2*>(S + (int64_t)m * kW + g * 8 + 2 * q) = out;
    }
}

// Edge head on the tensor cores, 16 stored pairs t = (m, n) per warp:
//   z = Pa[m] + Pb[n] + u + Uc e_t      (e [16] x Uc^T [16 x 64]: 8 n-tiles, hi and lo of e)
//   u_t = relu(z)                       (kept in U for the backward pass; 0 on the diagonal)
//   r = f + E u_t                       (u [64] x E^T [64 x K*8], the accumulators of z reused
//                                        as A fragments: n-tiles 2j, 2j+1 form k-tile j)
//   o[k] = sum_c b_c r[k*8 + c]         (each n-tile is one k; a quad shuffle sums over c)
template <int K>
__global__ void __launch_bounds__(128) k_head_forward(const float* __restrict__ Pa, const float* __restrict__ Pb,
                                                      const float* __restrict__ e, const float* __restrict__ basis,
                                                      const __nv_bfloat16* __restrict__ w, int64_t oUc, int64_t ou,
                                                      int64_t oE, int64_t of, const int* __restrict__ rows,
                                                      const int* __restrict__ cols, int64_t nnz,
                                                      float* __restrict__ o, float* __restrict__ U) {
    constexpr int NO = K * kNB;
    __shared__ __align__(16) __nv_bfloat16 Es[NO][kW + 8];   // E[n][j]: B operand of u E^T
    for (int k = threadIdx.x; k < NO * kW; k += blockDim.x) Es[k / kW][k % kW] = w[oE + k];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int64_t t0 = ((int64_t)blockIdx.x * 4 + (threadIdx.x >> 5)) * 16;
    if (t0 >= nnz) return;
    const int64_t ta = min(t0 + g, nnz - 1), tb = min(t0 + g + 8, nnz - 1);
    const bool va = t0 + g < nnz, vb = t0 + g + 8 < nnz;
    const int ma = rows[ta], na = cols[ta], mb = rows[tb], nb = cols[tb];
    float z[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int j = nt * 8 + 2 * q;
        const float u0 = __bfloat162float(w[ou + j]), u1 = __bfloat162float(w[ou + j + 1]);
        const float2 pa = ld_f2(Pa + (int64_t)ma * kW + j), pb = ld_f2(Pb + (int64_t)na * kW + j);
        const float2 qa = ld_f2(Pa + (int64_t)mb * kW + j), qb = ld_f2(Pb + (int64_t)nb * kW + j);
        z[nt][0] = pa.x + pb.x + u0;
        z[nt][1] = pa.y + pb.y + u1;
        z[nt][2] = qa.x + qb.x + u0;
        z[nt][3] = qa.y + qb.y + u1;
    }
    {
        uint32_t ah[4], al[4];
        a_frag_rows(e + ta * kNed, e + tb * kNed, 0, q, ah, al);
        uint32_t b[8][2];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const __nv_bfloat16* uc = w + oUc + (int64_t)(nt * 8 + g) * kNed + 2 * q;   // Uc[j][f]
            b[nt][0] = ld_bf2(uc);
            b[nt][1] = ld_bf2(uc + 8);
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) mma_bf16(z[nt], ah, b[nt][0], b[nt][1]);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) mma_bf16(z[nt], al, b[nt][0], b[nt][1]);
    }
    const bool ka = ma != na, kb = mb != nb;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        z[nt][0] = ka ? fmaxf(z[nt][0], 0.f) : 0.f;
        z[nt][1] = ka ? fmaxf(z[nt][1], 0.f) : 0.f;
        z[nt][2] = kb ? fmaxf(z[nt][2], 0.f) : 0.f;
        z[nt][3] = kb ? fmaxf(z[nt][3], 0.f) : 0.f;
    }
    if (U) {
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int j = nt * 8 + 2 * q;
            if (va) *reinterpret_cast<float2*>(U + ta * kW + j) = make_float2(z[nt][0], z[nt][1]);
            if (vb) *reinterpret_cast<float2*>(U + tb * kW + j) = make_float2(z[nt][2], z[nt][3]);
        }
    }
    float r[K][4];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float f0 = __bfloat162float(w[of + k * kNB + 2 * q]), f1 = __bfloat162float(w[of + k * kNB + 2 * q + 1]);
        r[k][0] = f0;
        r[k][1] = f1;
        r[k][2] = f0;
        r[k][3] = f1;
    }
#pragma unroll
    for (int kt = 0; kt < kW / 16; ++kt) {
        uint32_t ah[4], al[4];
        split_bf2(z[2 * kt][0], z[2 * kt][1], ah[0], al[0]);
        split_bf2(z[2 * kt][2], z[2 * kt][3], ah[1], al[1]);
        split_bf2(z[2 * kt + 1][0], z[2 * kt + 1][1], ah[2], al[2]);
        split_bf2(z[2 * kt + 1][2], z[2 * kt + 1][3], ah[3], al[3]);
        uint32_t b[K][2];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            b[k][0] = ld_bf2(&Es[k * kNB + g][16 * kt + 2 * q]);
            b[k][1] = ld_bf2(&Es[k * kNB + g][16 * kt + 2 * q + 8]);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) mma_bf16(r[k], ah, b[k][0], b[k][1]);
#pragma unroll
        for (int k = 0; k < K; ++k) mma_bf16(r[k], al, b[k][0], b[k][1]);
    }
    const float2 ba = ld_f2(basis + ta * kNB + 2 * q), bb = ld_f2(basis + tb * kNB + 2 * q);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float sa = fmaf(ba.y, r[k][1], ba.x * r[k][0]);
        float sb = fmaf(bb.y, r[k][3], bb.x * r[k][2]);
        // butterfly over the quad: every lane ends with the same sum (each add is commutative)
        sa += __shfl_xor_sync(0xffffffffu, sa, 1);
        sb += __shfl_xor_sync(0xffffffffu, sb, 1);
        sa += __shfl_xor_sync(0xffffffffu, sa, 2);
        sb += __shfl_xor_sync(0xffffffffu, sb, 2);
        if ((k & 3) == q) {
            if (va) o[ta * K + k] = ka ? sa : 0.f;
            if (vb) o[tb * K + k] = kb ? sb : 0.f;
        }
    }
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

// Edge head backward on the tensor cores, 16 stored pairs per warp:
//   dz_t[j] = [u_t[j] > 0] sum_n G'_t[n] E[n][j],  G'_t[k*8 + c] = Ge_t[k] b_c(t)
// (G' [K*8] x E [K*8 x 64]: A fragments formed from Ge and the bases, hi and lo; E^T staged in
// shared memory as the B operand).  u = 0 on the diagonal, so dz = 0 there.
template <int K>
__global__ void __launch_bounds__(128) k_head_backward(const float* __restrict__ U, const float* __restrict__ Ge,
                                                       const float* __restrict__ basis,
                                                       const __nv_bfloat16* __restrict__ w, int64_t oE,
                                                       int64_t nnz, float* __restrict__ DZ) {
    constexpr int NO = K * kNB;
    __shared__ __align__(16) __nv_bfloat16 Et[kW][NO + 8];   // E^T[j][n]
    for (int k = threadIdx.x; k < NO * kW; k += blockDim.x) Et[k % kW][k / kW] = w[oE + k];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int64_t t0 = ((int64_t)blockIdx.x * 4 + (threadIdx.x >> 5)) * 16;
    if (t0 >= nnz) return;
    const int64_t ta = min(t0 + g, nnz - 1), tb = min(t0 + g + 8, nnz - 1);
    const bool va = t0 + g < nnz, vb = t0 + g + 8 < nnz;
    const float2 ba = ld_f2(basis + ta * kNB + 2 * q), bb = ld_f2(basis + tb * kNB + 2 * q);
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[nt][i] = 0.f;
#pragma unroll
    for (int kt = 0; kt < NO / 16; ++kt) {
        // k-tile kt covers n = 16 kt + [0, 16): outputs k = 2 kt (columns 0..7) and 2 kt + 1 (8..15)
        const float ga0 = Ge[ta * K + 2 * kt], ga1 = Ge[ta * K + 2 * kt + 1];
        const float gb0 = Ge[tb * K + 2 * kt], gb1 = Ge[tb * K + 2 * kt + 1];
        uint32_t ah[4], al[4];
        split_bf2(ga0 * ba.x, ga0 * ba.y, ah[0], al[0]);
        split_bf2(gb0 * bb.x, gb0 * bb.y, ah[1], al[1]);
        split_bf2(ga1 * ba.x, ga1 * ba.y, ah[2], al[2]);
        split_bf2(gb1 * bb.x, gb1 * bb.y, ah[3], al[3]);
        uint32_t b[8][2];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            b[nt][0] = ld_bf2(&Et[nt * 8 + g][16 * kt + 2 * q]);
            b[nt][1] = ld_bf2(&Et[nt * 8 + g][16 * kt + 2 * q + 8]);
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) mma_bf16(acc[nt], ah, b[nt][0], b[nt][1]);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) mma_bf16(acc[nt], al, b[nt][0], b[nt][1]);
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int j = nt * 8 + 2 * q;
        if (va) {
            const float2 u = ld_f2(U + ta * kW + j);
            *reinterpret_cast<float2*>(DZ + ta * kW + j) =
                make_float2(u.x > 0.f ? acc[nt][0] : 0.f, u.y > 0.f ? acc[nt][1] : 0.f);
        }
        if (vb) {
            const float2 u = ld_f2(U + tb * kW + j);
            *reinterpret_cast<float2*>(DZ + tb * kW + j) =
                make_float2(u.x > 0.f ? acc[nt][2] : 0.f, u.y > 0.f ? acc[nt][3] : 0.f);
        }
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

// Message backward for layer l on the tensor cores, one warp per node n (warp-strided) over
// its CSR row in tiles of 16 edges (the near pattern is symmetric; edge (m, n) is trans[t]):
//   z^T = P[n] + c + C e_mn^T          (C exact as the A operand: 4 m-tiles of channels)
//   G^T = [z > 0, m != n] dS[m]        (per channel and edge, in the accumulator layout)
//   dP[n] = sum_m G^T,   dC^T += e^T G  (G's accumulators are the B fragments directly),
//   dc += sum_m G^T;  dC and dc as per-warp partials, combined by a fixed reduction.
__global__ void __launch_bounds__(128, 3) k_edge_backward(const float* __restrict__ P, const float* __restrict__ e,
                                                       const __nv_bfloat16* __restrict__ w, int64_t oC, int64_t oc,
                                                       const int* __restrict__ row_ptr, const int* __restrict__ cols,
                                                       const int* __restrict__ trans, const float* __restrict__ dS,
                                                       int N, float* __restrict__ dP, float* __restrict__ part) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    uint32_t ca[4][4];   // A fragments of C (64 x 16, row-major [channel][feature]), exact
    float cv[4][2];      // c at this lane's channels 16 mt + g (+8)
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
        const __nv_bfloat16* c0 = w + oC + (int64_t)(16 * mt + g) * kNed + 2 * q;
        ca[mt][0] = ld_bf2(c0);
        ca[mt][1] = ld_bf2(c0 + 8 * kNed);
        ca[mt][2] = ld_bf2(c0 + 8);
        ca[mt][3] = ld_bf2(c0 + 8 * kNed + 8);
        cv[mt][0] = __bfloat162float(w[oc + 16 * mt + g]);
        cv[mt][1] = __bfloat162float(w[oc + 16 * mt + g + 8]);
    }
    float dct[8][4];     // dC^T accumulators: features g (+8) x channels 8 j + 2 q (+1)
    float dcs[4][2];     // dc partial sums at this lane's channels
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) dct[j][i] = 0.f;
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) dcs[mt][0] = dcs[mt][1] = 0.f;
    for (int n = warp; n < N; n += nwarp) {
        const int ts = row_ptr[n], te = row_ptr[n + 1];
        float pv[4][2], d[4][2];
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            pv[mt][0] = P[(int64_t)n * kW + 16 * mt + g] + cv[mt][0];
            pv[mt][1] = P[(int64_t)n * kW + 16 * mt + g + 8] + cv[mt][1];
            d[mt][0] = d[mt][1] = 0.f;
        }
        for (int t0 = ts; t0 < te; t0 += 16) {
            // B operand e^T (k = feature, n = edge): edge g of each 8-edge n-tile
            int tr[2];
            bool kp[2][2];   // keep flags of edges 2q, 2q+1 (+8) owned in the accumulator layout
#pragma unroll
            for (int et = 0; et < 2; ++et) tr[et] = trans[min(t0 + 8 * et + g, te - 1)];
            int me[2][2];
#pragma unroll
            for (int et = 0; et < 2; ++et)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int t = t0 + 8 * et + 2 * q + c;
                    me[et][c] = cols[min(t, te - 1)];
                    kp[et][c] = t < te && me[et][c] != n;
                }
            float z[4][2][4];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int et = 0; et < 2; ++et) {
                    z[mt][et][0] = z[mt][et][1] = pv[mt][0];
                    z[mt][et][2] = z[mt][et][3] = pv[mt][1];
                }
            uint32_t ebh[2][2], ebl[2][2];
#pragma unroll
            for (int et = 0; et < 2; ++et) {
                const float* er = e + (int64_t)tr[et] * kNed + 2 * q;
                const float2 e0 = ld_f2(er), e1 = ld_f2(er + 8);
                split_bf2(e0.x, e0.y, ebh[et][0], ebl[et][0]);
                split_bf2(e1.x, e1.y, ebh[et][1], ebl[et][1]);
            }
            // hi pass, then lo pass, over the eight independent accumulators
#pragma unroll
            for (int et = 0; et < 2; ++et)
#pragma unroll
                for (int mt = 0; mt < 4; ++mt) mma_bf16(z[mt][et], ca[mt], ebh[et][0], ebh[et][1]);
#pragma unroll
            for (int et = 0; et < 2; ++et)
#pragma unroll
                for (int mt = 0; mt < 4; ++mt) mma_bf16(z[mt][et], ca[mt], ebl[et][0], ebl[et][1]);
            // gate: G^T(channel, edge) = [z > 0, keep] dS[m_edge][channel]
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int et = 0; et < 2; ++et)
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int c = i & 1, h = i >> 1;
                        const float ds = dS[(int64_t)me[et][c] * kW + 16 * mt + g + 8 * h];
                        const float gv = (kp[et][c] && z[mt][et][i] > 0.f) ? ds : 0.f;
                        z[mt][et][i] = gv;
                        d[mt][h] += gv;
                    }
            // dC^T += e^T G: A = e^T (m = feature g (+8), k = edges 2q.. (+8)), split hi/lo
            uint32_t ah[4], al[4];
            {
                float ev[4][2];
#pragma unroll
                for (int et = 0; et < 2; ++et)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int t = min(t0 + 8 * et + 2 * q + c, te - 1);
                        const int trc = trans[t];
                        ev[2 * et][c] = e[(int64_t)trc * kNed + g];         // feature g
                        ev[2 * et + 1][c] = e[(int64_t)trc * kNed + g + 8]; // feature g + 8
                    }
                // a0 = (g, edges 2q..), a1 = (g + 8, edges 2q..), a2 = (g, edges 8 + 2q..), a3 = (g + 8, ...)
                split_bf2(ev[0][0], ev[0][1], ah[0], al[0]);
                split_bf2(ev[1][0], ev[1][1], ah[1], al[1]);
                split_bf2(ev[2][0], ev[2][1], ah[2], al[2]);
                split_bf2(ev[3][0], ev[3][1], ah[3], al[3]);
            }
            // B fragments of G (k = edges, n = channels 8 j + g): rows (2q, 2q+1) of edge tiles 0, 1
            uint32_t gh[8][2], gl[8][2];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int mt = j >> 1, h = j & 1;
                split_bf2(z[mt][0][2 * h], z[mt][0][2 * h + 1], gh[j][0], gl[j][0]);
                split_bf2(z[mt][1][2 * h], z[mt][1][2 * h + 1], gh[j][1], gl[j][1]);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) mma_bf16(dct[j], ah, gh[j][0], gh[j][1]);
#pragma unroll
            for (int j = 0; j < 8; ++j) mma_bf16(dct[j], ah, gl[j][0], gl[j][1]);
#pragma unroll
            for (int j = 0; j < 8; ++j) mma_bf16(dct[j], al, gh[j][0], gh[j][1]);
        }
        // dP[n]: sum over the four lanes of each channel row (edges 2q, 2q + 1 of both tiles)
#pragma unroll
        for (int mt = 0; mt < 4; ++mt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float v = d[mt][h];
                dcs[mt][h] += v;
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                if (q == 0) dP[(int64_t)n * kW + 16 * mt + g + 8 * h] = v;
            }
    }
    float* pw = part + (int64_t)warp * (kW * kNed + kW);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int f = g + 8 * (i >> 1), ch = 8 * j + 2 * q + (i & 1);
            pw[ch * kNed + f] = dct[j][i];
        }
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v = dcs[mt][h];
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            if (q == 0) pw[kW * kNed + 16 * mt + g + 8 * h] = v;
        }
}

// Per-block partials of a row reduction over R rows in fixed chunks, on the tensor cores:
//   out[o][i] = sum_r A(r, o) B[r][i] (o < na <= 64, i < nb <= 64), then (bias) sum_r A(r, o).
// MODE 0: A(r, o) = A[r * na + o];  MODE 1: A(r, o) = Ge[r * K + o / 8] * basis[r * 8 + o % 8].
// Each 32-row stage is staged transposed in shared memory as split BF16 ([column][row], rows
// contiguous), so A^T is the MMA's A operand (m = o, k = r) and B its B operand (k = r,
// n = i), both read with ldmatrix; warp w owns outputs o in [16 w, 16 w + 16).  Stages are
// double-buffered (one barrier each) and the next one is loaded into registers while the
// current one is multiplied.  The bias sums run in FP32 on the staging threads (two per
// column, combined in a fixed order).
constexpr int kWgPitch = 40;   // BF16 per staged column: 32 rows + 8 (16-byte rows, conflict-free ldmatrix)

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const __nv_bfloat16* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

template <int MODE, int NP>
__global__ void __launch_bounds__(128) k_rows_wgrad(const float* __restrict__ A, const float* __restrict__ Ge,
                                                    const float* __restrict__ basis, int K, int na,
                                                    const float* __restrict__ B, int nb, int bias, int64_t R,
                                                    int64_t chunk, float* __restrict__ part) {
    // [buffer][hi, lo][column][row]
    __shared__ __align__(16) __nv_bfloat16 sA[2][2][kW][kWgPitch];
    __shared__ __align__(16) __nv_bfloat16 sB[2][2][kW][kWgPitch];
    __shared__ float sbias[4][kW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, q = lane & 3;
    // staging: item i of thread tid is column 8 (tid / 32 + 4 (i & 1)) + tid % 8 and row pair
    // 4 (i / 2) + (tid / 8) % 4, so that a warp's stores of one item cover 8 columns x 4 row
    // pairs (32 distinct banks) and its loads 4 rows x 8 consecutive columns
    const int scol = 8 * (tid >> 5) + (tid & 7), spair = (tid >> 3) & 3;
    const int64_t lo = blockIdx.x * chunk, hi = min(R, lo + chunk);
    // NP pairs of n-tiles (nb <= 16 NP).  With one pair the three products (hi hi, hi lo, lo hi)
    // keep separate accumulators, so that every MMA of a k-step is independent of the others.
    constexpr int SETS = NP == 1 ? 3 : 1;
    float acc[SETS][2 * NP][4];
#pragma unroll
    for (int st = 0; st < SETS; ++st)
#pragma unroll
        for (int nt = 0; nt < 2 * NP; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[st][nt][i] = 0.f;
    float accb[2] = {0.f, 0.f};
    constexpr int PP = 8;   // (column, row pair) items per thread and stage
    // next stage in registers: A (MODE 0) or its two factors Ge and basis (MODE 1, multiplied
    // at staging time, so that no instruction waits on these loads before the MMAs), and B
    float ra[2 * PP], rb[2 * PP], rc[MODE == 1 ? 2 * PP : 1];
    auto load_stage = [&](int64_t r0) {
#pragma unroll
        for (int p = 0; p < PP; ++p) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int col = scol + 32 * (p & 1);
                const int64_t r = r0 + 2 * (4 * (p >> 1) + spair) + s;
                float va = 0.f, vb = 0.f, vc = 0.f;
                if (r < hi) {
                    if (col < na) {
                        if (MODE == 0) {
                            va = A[r * na + col];
                        } else {
                            va = Ge[r * K + col / kNB];
                            vc = basis[r * kNB + col % kNB];
                        }
                    }
                    if (col < nb) vb = B[r * nb + col];
                }
                ra[2 * p + s] = va;
                rb[2 * p + s] = vb;
                if (MODE == 1) rc[2 * p + s] = vc;
            }
        }
    };
    // staged rows are 16-byte chunks of 8 BF16 values (every 8-row ldmatrix phase conflict-free)
    auto chunk_at = [](int x, int c) { return 8 * c; };
    const bool mts = warp * 16 < na;                // this warp's m-tile holds outputs
    // ldmatrix row addresses of this lane: A (16 x 16 per k-step), B (two n-tiles x 16 per k-step)
    const int arow = warp * 16 + (lane & 7) + 8 * ((lane >> 3) & 1), acol = 8 * (lane >> 4);
    const int brow = (lane & 7) + 8 * (lane >> 4), bcol = 8 * ((lane >> 3) & 1);
    if (lo < hi) load_stage(lo);
    int buf = 0;
    for (int64_t r0 = lo; r0 < hi; r0 += 32, buf ^= 1) {
#pragma unroll
        for (int p = 0; p < PP; ++p) {
            const int col = scol + 32 * (p & 1);
            const int pr = 4 * (p >> 1) + spair;          // row pair: rows 2 pr, 2 pr + 1
            const int at = chunk_at(col, pr >> 2) + 2 * (pr & 3);
            const float a0 = MODE == 1 ? ra[2 * p] * rc[2 * p] : ra[2 * p];
            const float a1 = MODE == 1 ? ra[2 * p + 1] * rc[2 * p + 1] : ra[2 * p + 1];
            uint32_t h, l;
            split_bf2(a0, a1, h, l);
            *reinterpret_cast<uint32_t*>(&sA[buf][0][col][at]) = h;
            *reinterpret_cast<uint32_t*>(&sA[buf][1][col][at]) = l;
            split_bf2(rb[2 * p], rb[2 * p + 1], h, l);
            *reinterpret_cast<uint32_t*>(&sB[buf][0][col][at]) = h;
            *reinterpret_cast<uint32_t*>(&sB[buf][1][col][at]) = l;
            accb[p & 1] += a0;
            accb[p & 1] += a1;
        }
        __syncthreads();
        if (r0 + 32 < hi) load_stage(r0 + 32);
        if (mts) {
#pragma unroll
            for (int kt = 0; kt < 2; ++kt) {
                uint32_t ah[4], al[4];
                const int ac = chunk_at(arow, 2 * kt + acol / 8);
                ldsm_x4(ah, &sA[buf][0][arow][ac]);
                ldsm_x4(al, &sA[buf][1][arow][ac]);
                uint32_t bh[NP][4], bl[NP][4];   // n-tiles 2 np (regs 0, 1) and 2 np + 1 (regs 2, 3)
#pragma unroll
                for (int np = 0; np < NP; ++np) {
                    const int bc = chunk_at(16 * np + brow, 2 * kt + bcol / 8);
                    ldsm_x4(bh[np], &sB[buf][0][16 * np + brow][bc]);
                    ldsm_x4(bl[np], &sB[buf][1][16 * np + brow][bc]);
                }
#pragma unroll
                for (int nt = 0; nt < 2 * NP; ++nt)
                    mma_bf16(acc[0][nt], ah, bh[nt >> 1][2 * (nt & 1)], bh[nt >> 1][2 * (nt & 1) + 1]);
#pragma unroll
                for (int nt = 0; nt < 2 * NP; ++nt)
                    mma_bf16(acc[1 % SETS][nt], ah, bl[nt >> 1][2 * (nt & 1)], bl[nt >> 1][2 * (nt & 1) + 1]);
#pragma unroll
                for (int nt = 0; nt < 2 * NP; ++nt)
                    mma_bf16(acc[2 % SETS][nt], al, bh[nt >> 1][2 * (nt & 1)], bh[nt >> 1][2 * (nt & 1) + 1]);
            }
        }
    }
    const int len = na * nb + (bias ? na : 0);
    float* pb = part + (int64_t)blockIdx.x * len;
    if (mts) {
#pragma unroll
        for (int nt = 0; nt < 2 * NP; ++nt) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int o = warp * 16 + g + 8 * h;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int i = nt * 8 + 2 * q + c;
                    float v = acc[0][nt][2 * h + c];
#pragma unroll
                    for (int st = 1; st < SETS; ++st) v += acc[st][nt][2 * h + c];
                    if (o < na && i < nb) pb[o * nb + i] = v;
                }
            }
        }
    }
    if (bias) {
        sbias[spair][scol] = accb[0];
        sbias[spair][scol + 32] = accb[1];
        __syncthreads();
        if (tid < na) pb[na * nb + tid] = (sbias[0][tid] + sbias[1][tid]) + (sbias[2][tid] + sbias[3][tid]);
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
        k_node_gemm<false><<<nodeblk, 128, 0, s>>>(Hp, w + lay.B[l], nullptr, nullptr, Pl, N, 0, 0);
        k_edge_message<<<warpblk, 256, 0, s>>>(Pl, G.d_e, w, lay.C[l], lay.c[l], ctx->d_row_ptr, ctx->d_cols,
                                               G.d_deginv, N, G.d_S);
        k_node_gemm<false><<<nodeblk, 128, 0, s>>>(Hp, w + lay.D[l], w + lay.d[l], G.d_S, G.d_H + (l + 1) * NW, N, 1,
                                                   0);
    }
    const float* HL = G.d_H + L * NW;
    k_node_gemm<false><<<nodeblk, 128, 0, s>>>(HL, w + lay.Ua, nullptr, nullptr, G.d_Pa, N, 0, 0);
    k_node_gemm<false><<<nodeblk, 128, 0, s>>>(HL, w + lay.Ub, nullptr, nullptr, G.d_Pb, N, 0, 0);
    if (K == 2)
        k_head_forward<2><<<gb(nnz, 64), 128, 0, s>>>(G.d_Pa, G.d_Pb, G.d_e, G.d_basis, w, lay.Uc, lay.u, lay.E,
                                                       lay.f, G.d_rows, ctx->d_cols, nnz, G.d_o, U);
    else
        k_head_forward<8><<<gb(nnz, 64), 128, 0, s>>>(G.d_Pa, G.d_Pb, G.d_e, G.d_basis, w, lay.Uc, lay.u, lay.E,
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
    if constexpr (MODE == 0) {
        if (nb <= 16) {
            k_rows_wgrad<0, 1><<<kWgradBlocks, 128, 0, s>>>(A, Ge, basis, K, na, B, nb, bias, R, chunk, part);
            reduce_into(part, kWgradBlocks, (int64_t)na * nb + (bias ? na : 0), grad, s);
            return;
        }
    }
    k_rows_wgrad<MODE, 4><<<kWgradBlocks, 128, 0, s>>>(A, Ge, basis, K, na, B, nb, bias, R, chunk, part);
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
            k_head_backward<2><<<gb(nnz, 64), 128, 0, s>>>(net->d_U, net->d_Ge, G.d_basis, w, lay.E, nnz, net->d_DZ);
        else
            k_head_backward<8><<<gb(nnz, 64), 128, 0, s>>>(net->d_U, net->d_Ge, G.d_basis, w, lay.E, nnz, net->d_DZ);
        rows_wgrad<0>(net->d_DZ, nullptr, nullptr, 0, kW, G.d_e, kNed, 1, nnz, part, grad + lay.Uc, s);
        k_head_node_back<<<gb((int64_t)N * 32), 256, 0, s>>>(net->d_DZ, ctx->d_row_ptr, G.d_trans, N, dza, dzb);
        rows_wgrad<0>(dza, nullptr, nullptr, 0, kW, HL, kW, 0, N, part, grad + lay.Ua, s);
        rows_wgrad<0>(dzb, nullptr, nullptr, 0, kW, HL, kW, 0, N, part, grad + lay.Ub, s);
        // diagonal head: dG, dg
        rows_wgrad<0>(net->d_Gn, nullptr, nullptr, 0, K, HL, kW, 1, N, part, grad + lay.G, s);
        // dH_L = dza Ua + dzb Ub + Gn G
        const unsigned nodeblk = (unsigned)((N + 63) / 64);
        k_node_gemm<true><<<nodeblk, 128, 0, s>>>(dza, w + lay.Ua, nullptr, nullptr, dH, N, 0, 0);
        k_node_gemm<true><<<nodeblk, 128, 0, s>>>(dzb, w + lay.Ub, nullptr, nullptr, dH, N, 0, 1);
        k_diag_head_back<<<gb(NW), 256, 0, s>>>(net->d_Gn, w, lay.G, N, K, dH);
        const unsigned pblk = kPersistWarps / 4;
        for (int l = L - 1; l >= 0; --l) {
            const float* Hl = G.d_H + (l + 1) * NW;
            const float* Hp = G.d_H + l * NW;
            const float* Pl = G.d_P + l * NW;
            k_relu_back<<<gb(NW), 256, 0, s>>>(dH, Hl, G.d_deginv, N, dU, dS);
            rows_wgrad<0>(dU, nullptr, nullptr, 0, kW, Hp, kW, 1, N, part, grad + lay.D[l], s);
            k_edge_backward<<<pblk, 128, 0, s>>>(Pl, G.d_e, w, lay.C[l], lay.c[l], ctx->d_row_ptr, ctx->d_cols,
                                                 G.d_trans, dS, N, dP, part);
            reduce_into(part, kPersistWarps, kW * kNed + kW, grad + lay.C[l], s);
            rows_wgrad<0>(dP, nullptr, nullptr, 0, kW, Hp, kW, 0, N, part, grad + lay.B[l], s);
            k_node_gemm<true><<<nodeblk, 128, 0, s>>>(dU, w + lay.D[l], nullptr, nullptr, dT, N, 0, 0);
            k_node_gemm<true><<<nodeblk, 128, 0, s>>>(dP, w + lay.B[l], nullptr, nullptr, dT, N, 0, 1);
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
