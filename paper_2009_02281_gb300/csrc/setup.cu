// One-time setup of an AIMx context (Sec. II-B and Sec. III-A of the paper).
//
// Host (C++): mesh validation, RWG functions, grid, integer stencil anchors,
// near-region pair list and the node-major gather lists; these are integer
// or exactly specified floating-point steps.
// Device (FP64 CUDA): moment-matching projection weights, the static near
// integrals L^A_s, L^Phi_s, K_s with closed-form inner potentials, and the
// static grid precorrection on the same pairs (Eq. aimLPs).
//
// Host floating-point code in this file is compiled with -ffp-contract=off
// so that the anchor arithmetic rounds identically on every host CPU.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "aimx_internal.h"
#include "geom.cuh"

namespace aimx {

// ------------------------------------------------------------------ quadrature

// Gauss-Legendre nodes/weights on [0, 1] by Newton iteration on the
// three-term Legendre recurrence; returned in ascending node order.
static void gauss_legendre01(int q, std::vector<double>& x, std::vector<double>& w) {
    x.assign(q, 0.0);
    w.assign(q, 0.0);
    for (int i = 0; i < q; ++i) {
        double t = std::cos(kPi * (i + 0.75) / (q + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int j = 2; j <= q; ++j) {
                double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            double pq = (q == 1) ? t : p1;
            double pqm1 = (q == 1) ? 1.0 : p0;
            dp = q * (t * pq - pqm1) / (t * t - 1.0);
            double dt = pq / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        // recompute derivative at the converged node for the weight
        double p0 = 1.0, p1 = t;
        for (int j = 2; j <= q; ++j) {
            double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        double pq = (q == 1) ? t : p1, pqm1 = (q == 1) ? 1.0 : p0;
        dp = q * (t * pq - pqm1) / (t * t - 1.0);
        x[q - 1 - i] = 0.5 * (t + 1.0);
        w[q - 1 - i] = 0.5 * 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

// Collapsed (Duffy) product rule: barycentric (u, (1-u)v, (1-u)(1-v)) with
// normalised weight 2 w_u w_v (1-u); exact to total degree 2q-2.
void triangle_rule(int q, std::vector<double>& out /* [Q][4] l1 l2 l3 w */) {
    std::vector<double> x, w;
    gauss_legendre01(q, x, w);
    out.clear();
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
            out.push_back(x[i]);
            out.push_back((1.0 - x[i]) * x[j]);
            out.push_back((1.0 - x[i]) * (1.0 - x[j]));
            out.push_back(2.0 * w[i] * w[j] * (1.0 - x[i]));
        }
}

__constant__ double c_qproj[kMaxQuad * 4];
__constant__ double c_qnear[kMaxQuad * 4];

// ------------------------------------------------------------------ device setup kernels

// Lambda_f[u, i] = int f_i,f l_u dS (f = x, y, z) and int div f_i l_u dS, one thread per (i, u).
__global__ void k_weights(GeomView g, const int* anc, int N, int P, int nq, double ox, double oy,
                          double oz, double hx, double hy, double hz, double* w) {
    int U = P * P * P;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * U) return;
    int i = t / U, u = t % U;
    int ui = u % P, uj = (u / P) % P, uk = u / (P * P);
    double acc[4] = {0, 0, 0, 0};
    for (int side = 0; side < 2; ++side) {
        int tr = g.btri[2 * i + side];
        double sg = side == 0 ? 1.0 : -1.0;
        double A = g.area[tr];
        double c = g.blen[i] / (2.0 * A);
        V3 p = load3(g.xyz + 3 * g.bfree[2 * i + side]);
        V3 a = vtx(g, tr, 0), b = vtx(g, tr, 1), cc = vtx(g, tr, 2);
        for (int q = 0; q < nq; ++q) {
            V3 r = c_qproj[4 * q] * a + c_qproj[4 * q + 1] * b + c_qproj[4 * q + 2] * cc;
            double W = c_qproj[4 * q + 3] * A;
            double xi[3] = {(r.x - ox) / hx - anc[3 * i], (r.y - oy) / hy - anc[3 * i + 1],
                            (r.z - oz) / hz - anc[3 * i + 2]};
            int sel[3] = {ui, uj, uk};
            double ell = 1.0;
            for (int ax = 0; ax < 3; ++ax) {
                for (int m = 0; m < P; ++m)
                    if (m != sel[ax]) ell *= (xi[ax] - m) / double(sel[ax] - m);
            }
            V3 f = (sg * c) * (r - p);
            acc[0] += W * f.x * ell;
            acc[1] += W * f.y * ell;
            acc[2] += W * f.z * ell;
            acc[3] += W * (sg * 2.0 * c) * ell;
        }
    }
    for (int k = 0; k < 4; ++k) w[(size_t)t * 4 + k] = acc[k];
}

// CFIE testing moments Lambda_g[u, i] = int (n x f_i) l_u dS (n the triangle's unit normal), one
// thread per (i, u), the rule of the projection weights.
__global__ void k_weights_g(GeomView g, const int* anc, int N, int P, int nq, double ox, double oy, double oz,
                            double hx, double hy, double hz, double* wg) {
    int U = P * P * P;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * U) return;
    int i = t / U, u = t % U;
    int sel[3] = {u % P, (u / P) % P, u / (P * P)};
    double acc[3] = {0, 0, 0};
    for (int side = 0; side < 2; ++side) {
        int tr = g.btri[2 * i + side];
        double sg = side == 0 ? 1.0 : -1.0;
        double A = g.area[tr];
        double c = g.blen[i] / (2.0 * A);
        V3 p = load3(g.xyz + 3 * g.bfree[2 * i + side]);
        V3 a = vtx(g, tr, 0), b = vtx(g, tr, 1), cc = vtx(g, tr, 2);
        const V3 ncr = cross(b - a, cc - a);
        const V3 n = (1.0 / norm3(ncr)) * ncr;
        for (int q = 0; q < nq; ++q) {
            V3 r = c_qproj[4 * q] * a + c_qproj[4 * q + 1] * b + c_qproj[4 * q + 2] * cc;
            double W = c_qproj[4 * q + 3] * A;
            double xi[3] = {(r.x - ox) / hx - anc[3 * i], (r.y - oy) / hy - anc[3 * i + 1],
                            (r.z - oz) / hz - anc[3 * i + 2]};
            double ell = 1.0;
            for (int ax = 0; ax < 3; ++ax)
                for (int m = 0; m < P; ++m)
                    if (m != sel[ax]) ell *= (xi[ax] - m) / double(sel[ax] - m);
            V3 gf = cross(n, (sg * c) * (r - p));
            acc[0] += W * gf.x * ell;
            acc[1] += W * gf.y * ell;
            acc[2] += W * gf.z * ell;
        }
    }
    for (int k = 0; k < 3; ++k) wg[(size_t)t * 3 + k] = acc[k];
}

// Static near integrals for every stored pair (row i, column j), one thread per pair.
// rot = 1 (CFIE): the K integral is tested with n x f_i (n the testing triangle's normal).
__global__ void k_near_static(GeomView g, const int* row_of, const int* cols, int64_t nnz, int nq, int rot,
                              double* LA, double* LP, double* KK) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    int i = row_of[e], j = cols[e];
    double la = 0.0, lp = 0.0, kk = 0.0;
    for (int ss = 0; ss < 2; ++ss) {
        int ts = g.btri[2 * j + ss];
        double sgs = ss == 0 ? 1.0 : -1.0;
        double cs = g.blen[j] / (2.0 * g.area[ts]);
        V3 ps = load3(g.xyz + 3 * g.bfree[2 * j + ss]);
        TriFrame T;
        make_frame(T, vtx(g, ts, 0), vtx(g, ts, 1), vtx(g, ts, 2));
        for (int so = 0; so < 2; ++so) {
            int to = g.btri[2 * i + so];
            double sgo = so == 0 ? 1.0 : -1.0;
            double Ao = g.area[to];
            double co = g.blen[i] / (2.0 * Ao);
            V3 po = load3(g.xyz + 3 * g.bfree[2 * i + so]);
            V3 a = vtx(g, to, 0), b = vtx(g, to, 1), c = vtx(g, to, 2);
            const V3 ncr = cross(b - a, c - a);
            const V3 no = (1.0 / norm3(ncr)) * ncr;
            for (int q = 0; q < nq; ++q) {
                V3 r = c_qnear[4 * q] * a + c_qnear[4 * q + 1] * b + c_qnear[4 * q + 2] * c;
                double W = c_qnear[4 * q + 3] * Ao;
                double I1;
                V3 J, G, rho;
                tri_potentials(T, r, I1, J, G, rho);
                V3 fo = (sgo * co) * (r - po);
                V3 vp = (sgs * cs) * (J + I1 * (rho - ps));
                la += W * dot(fo, vp);
                lp += W * (sgo * 2.0 * co) * (sgs * 2.0 * cs) * I1;
                V3 kv = (sgs * cs) * cross(G, r - ps);
                kk += W * dot(rot ? cross(no, fo) : fo, kv);
            }
        }
    }
    const double inv4pi = 1.0 / (4.0 * kPi);
    LA[e] = la * inv4pi;
    LP[e] = lp * inv4pi;
    KK[e] = kk * inv4pi;
}

// Precorrection with the static grid kernel between the two stencils, then
// N = direct - precorrection; FP64 and FP32 copies.
// wg (CFIE, else null): the K precorrection takes the testing side's moments of n x f.
__global__ void k_precorrect(const double* w, const double* wg, const int* anc, const int* row_of, const int* cols,
                             int64_t nnz, int P, int span, const double* hs_tab, const double* hg_tab,
                             const double* LA, const double* LP, const double* KK, double* NA,
                             double* NP, double* NK, float* NA32, float* NP32, float* NK32) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    int U = P * P * P;
    int i = row_of[e], j = cols[e];
    int D = 2 * span + 1;
    int dx0 = anc[3 * i] - anc[3 * j], dy0 = anc[3 * i + 1] - anc[3 * j + 1],
        dz0 = anc[3 * i + 2] - anc[3 * j + 2];
    const double* wi = w + (size_t)i * U * 4;
    const double* wj = w + (size_t)j * U * 4;
    double pa = 0.0, pp = 0.0, pk = 0.0;
    for (int u = 0; u < U; ++u) {
        int ux = u % P, uy = (u / P) % P, uz = u / (P * P);
        double a0 = wi[4 * u], a1 = wi[4 * u + 1], a2 = wi[4 * u + 2], a3 = wi[4 * u + 3];
        double k0 = a0, k1 = a1, k2 = a2;
        if (wg) {
            const double* gi = wg + ((size_t)i * U + u) * 3;
            k0 = gi[0];
            k1 = gi[1];
            k2 = gi[2];
        }
        for (int v = 0; v < U; ++v) {
            int vx = v % P, vy = (v / P) % P, vz = v / (P * P);
            int ix = dx0 + ux - vx + span, iy = dy0 + uy - vy + span, iz = dz0 + uz - vz + span;
            int t = (iz * D + iy) * D + ix;
            double hs = hs_tab[t];
            double gx = hg_tab[3 * t], gy = hg_tab[3 * t + 1], gz = hg_tab[3 * t + 2];
            double b0 = wj[4 * v], b1 = wj[4 * v + 1], b2 = wj[4 * v + 2], b3 = wj[4 * v + 3];
            pa += hs * (a0 * b0 + a1 * b1 + a2 * b2);
            pp += hs * a3 * b3;
            // a . (g x b), a the testing moments (of f, or of n x f for the CFIE)
            pk += k0 * (gy * b2 - gz * b1) + k1 * (gz * b0 - gx * b2) + k2 * (gx * b1 - gy * b0);
        }
    }
    double na = LA[e] - pa, np_ = LP[e] - pp, nk = KK[e] - pk;
    NA[e] = na;
    NP[e] = np_;
    NK[e] = nk;
    NA32[e] = (float)na;
    NP32[e] = (float)np_;
    NK32[e] = (float)nk;
}

// Linear-term modification (Sec. III-A-3, Eq. Lmatdecomplin), one thread per
// overlapping pair (row i, column j): the direct integrals of the kernel
// G_lin = -R / (8 pi) (closed-form inner potentials, 5 x 5 outer rule) minus
// their precorrection with the sampled kernel H_lin[d] = -|d h| / (8 pi)
// between the two stencils.  FP64 and FP32 copies.
__global__ void k_linterm(GeomView g, const int* __restrict__ row_of, const int* __restrict__ cols, int64_t nlin,
                          int nq, const double* __restrict__ w, const int* __restrict__ anc, int P, double hx,
                          double hy, double hz, double* NA, double* NP, float* NA32, float* NP32) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nlin) return;
    const int i = row_of[e], j = cols[e];
    double la = 0.0, lp = 0.0;
    for (int ss = 0; ss < 2; ++ss) {
        int ts = g.btri[2 * j + ss];
        double sgs = ss == 0 ? 1.0 : -1.0;
        double cs = g.blen[j] / (2.0 * g.area[ts]);
        V3 ps = load3(g.xyz + 3 * g.bfree[2 * j + ss]);
        TriFrame T;
        make_frame(T, vtx(g, ts, 0), vtx(g, ts, 1), vtx(g, ts, 2));
        for (int so = 0; so < 2; ++so) {
            int to = g.btri[2 * i + so];
            double sgo = so == 0 ? 1.0 : -1.0;
            double Ao = g.area[to];
            double co = g.blen[i] / (2.0 * Ao);
            V3 po = load3(g.xyz + 3 * g.bfree[2 * i + so]);
            V3 a = vtx(g, to, 0), b = vtx(g, to, 1), c = vtx(g, to, 2);
            for (int q = 0; q < nq; ++q) {
                V3 r = c_qnear[4 * q] * a + c_qnear[4 * q + 1] * b + c_qnear[4 * q + 2] * c;
                double W = c_qnear[4 * q + 3] * Ao;
                double IR;
                V3 JR, rho;
                tri_r_potentials(T, r, IR, JR, rho);
                V3 fo = (sgo * co) * (r - po);
                V3 vp = (sgs * cs) * (JR + IR * (rho - ps));
                la += W * dot(fo, vp);
                lp += W * (sgo * 2.0 * co) * (sgs * 2.0 * cs) * IR;
            }
        }
    }
    const double inv8pi = 1.0 / (8.0 * kPi);
    la *= -inv8pi;
    lp *= -inv8pi;
    const int U = P * P * P;
    const int dx0 = anc[3 * i] - anc[3 * j], dy0 = anc[3 * i + 1] - anc[3 * j + 1],
              dz0 = anc[3 * i + 2] - anc[3 * j + 2];
    const double* wi = w + (size_t)i * U * 4;
    const double* wj = w + (size_t)j * U * 4;
    double pa = 0.0, pp = 0.0;
    for (int u = 0; u < U; ++u) {
        int ux = u % P, uy = (u / P) % P, uz = u / (P * P);
        double a0 = wi[4 * u], a1 = wi[4 * u + 1], a2 = wi[4 * u + 2], a3 = wi[4 * u + 3];
        for (int v = 0; v < U; ++v) {
            int vx = v % P, vy = (v / P) % P, vz = v / (P * P);
            double rx = (dx0 + ux - vx) * hx, ry = (dy0 + uy - vy) * hy, rz = (dz0 + uz - vz) * hz;
            double hl = -sqrt(rx * rx + ry * ry + rz * rz) * inv8pi;
            const double* b = wj + 4 * v;
            pa += hl * (a0 * b[0] + a1 * b[1] + a2 * b[2]);
            pp += hl * a3 * b[3];
        }
    }
    NA[e] = la - pa;
    NP[e] = lp - pp;
    NA32[e] = (float)(la - pa);
    NP32[e] = (float)(lp - pp);
}

// Surface-impedance Gram matrix on the near pattern: G_mn = int f_m . f_n dS over
// the triangles m and n share (a degree-2 integrand; the 5 x 5 collapsed rule
// q5 is exact).  Internal order; also the self terms into gdiag.
__global__ void k_gram(GeomView g, const int* __restrict__ row_of, const int* __restrict__ cols, int64_t nnz,
                       const double* __restrict__ q5, double* __restrict__ ng, double* __restrict__ gdiag) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const int m = row_of[e], n = cols[e];
    double acc = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int t = g.btri[2 * m + a];
            if (t != g.btri[2 * n + b]) continue;
            const double sm = a ? -1.0 : 1.0, sn = b ? -1.0 : 1.0;
            const double cm = g.blen[m] / (2.0 * g.area[t]), cn = g.blen[n] / (2.0 * g.area[t]);
            const double* pm = g.xyz + 3 * g.bfree[2 * m + a];
            const double* pn = g.xyz + 3 * g.bfree[2 * n + b];
            const int* tv = g.tri + 3 * t;
            const double* v0 = g.xyz + 3 * tv[0];
            const double* v1 = g.xyz + 3 * tv[1];
            const double* v2 = g.xyz + 3 * tv[2];
            double s = 0.0;
            for (int k = 0; k < 25; ++k) {
                const double l1 = q5[4 * k], l2 = q5[4 * k + 1], l3 = q5[4 * k + 2], wq = q5[4 * k + 3];
                double d = 0.0;
                for (int c = 0; c < 3; ++c) {
                    const double r = l1 * v0[c] + l2 * v1[c] + l3 * v2[c];
                    d += (r - pm[c]) * (r - pn[c]);
                }
                s += wq * d;
            }
            acc += sm * sn * cm * cn * g.area[t] * s;
        }
    ng[e] = acc;
    if (m == n) gdiag[m] = acc;
}

// field-major FP32 copy of the weights, ws[f][u][i] = w[i][u][f] (coalesced per-plane interpolation)
__global__ void k_weights_soa(const double* __restrict__ w, float* __restrict__ ws, int N, int U) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * U * 4) return;
    const int i = (int)(t % N);
    const int64_t r = t / N;
    const int u = (int)(r % U), f = (int)(r / U);
    ws[t] = (float)w[((int64_t)i * U + u) * 4 + f];
}

__global__ void k_to_float(const double* a, float* b, size_t n) {
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t < n) b[t] = (float)a[t];
}

__global__ void k_diag(const int* row_ptr, const int* cols, const double* LA, const double* LP,
                       const double* KK, int N, double* diag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
        if (cols[e] == i) {
            diag[3 * i] = LA[e];
            diag[3 * i + 1] = LP[e];
            diag[3 * i + 2] = KK[e];
        }
}

// ------------------------------------------------------------------ host setup

template <class T>
static T* upload(aimx_ctx* ctx, const std::vector<T>& v) {
    T* p = (T*)dev_alloc(ctx, std::max<size_t>(1, v.size()) * sizeof(T));
    if (!v.empty()) AIMX_CUDA_TRY(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}

static int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// smallest FFT length >= v of the form 2^k or 3 * 2^k
static int next_fft_len(int v) {
    int p3 = 3;
    while (p3 < v) p3 <<= 1;
    return std::min(next_pow2(v), p3);
}

static bool fft_len_ok(int L) {
    int P = (L % 3 == 0) ? L / 3 : L;
    return P >= 1 && (P & (P - 1)) == 0;
}

// Gram values on the near pattern (FP64 and FP32) and their self terms, when a surface impedance is set
static void build_gram(aimx_ctx* ctx, const GeomView& gv, const int* d_row_of) {
    if (!(ctx->sigma > 0) && ctx->form != AIMX_CFIE) return;
    const int64_t nnz = ctx->nnz;
    ctx->f64.ng = (double*)dev_alloc(ctx, sizeof(double) * nnz);
    ctx->f32.ng = (float*)dev_alloc(ctx, sizeof(float) * nnz);
    ctx->d_gdiag = (double*)dev_alloc(ctx, sizeof(double) * ctx->N);
    k_gram<<<(unsigned)((nnz + 127) / 128), 128>>>(gv, d_row_of, ctx->d_cols, nnz, ctx->d_q5, ctx->f64.ng,
                                                   ctx->d_gdiag);
    k_to_float<<<(unsigned)((nnz + 255) / 256), 256>>>(ctx->f64.ng, ctx->f32.ng, (size_t)nnz);
    AIMX_CUDA_TRY(cudaGetLastError());
}

void build_linterm(aimx_ctx* ctx) {
    if (ctx->nlin) return;
    const int N = ctx->N;
    // bases on each triangle (internal ids); pairs that share one overlap
    std::vector<std::vector<int>> on_tri(ctx->nt);
    for (int i = 0; i < N; ++i) {
        const int o = ctx->perm[i];
        on_tri[ctx->h_tp[o]].push_back(i);
        on_tri[ctx->h_tm[o]].push_back(i);
    }
    std::vector<int> ptr(N + 1, 0), cols, row_of;
    std::vector<int> nb;
    for (int i = 0; i < N; ++i) {
        const int o = ctx->perm[i];
        nb.clear();
        for (int t : {ctx->h_tp[o], ctx->h_tm[o]}) nb.insert(nb.end(), on_tri[t].begin(), on_tri[t].end());
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        cols.insert(cols.end(), nb.begin(), nb.end());
        row_of.insert(row_of.end(), nb.size(), i);
        ptr[i + 1] = (int)cols.size();
    }
    const int64_t nl = (int64_t)cols.size();
    int* d_row_of = upload(ctx, row_of);
    ctx->d_lin_ptr = upload(ctx, ptr);
    ctx->d_lin_cols = upload(ctx, cols);
    ctx->f64.la = (double*)dev_alloc(ctx, sizeof(double) * nl);
    ctx->f64.lp = (double*)dev_alloc(ctx, sizeof(double) * nl);
    ctx->f32.la = (float*)dev_alloc(ctx, sizeof(float) * nl);
    ctx->f32.lp = (float*)dev_alloc(ctx, sizeof(float) * nl);
    GeomView gv{ctx->d_xyz, ctx->d_tri, ctx->d_area, ctx->d_btri, ctx->d_bfree, ctx->d_blen};
    k_linterm<<<(unsigned)((nl + 127) / 128), 128>>>(gv, d_row_of, ctx->d_lin_cols, nl, 25, ctx->f64.w, ctx->d_anc,
                                                     ctx->P, ctx->h[0], ctx->h[1], ctx->h[2], ctx->f64.la,
                                                     ctx->f64.lp, ctx->f32.la, ctx->f32.lp);
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaDeviceSynchronize();
    dev_free(ctx, d_row_of);
    AIMX_CUDA_TRY(e1);
    AIMX_CUDA_TRY(e2);
    ctx->lin_ptr = ptr;
    ctx->lin_cols = cols;
    ctx->nlin = nl;
}

void setup_context(aimx_ctx* ctx, const aimx_mesh* mesh, const aimx_material* mat,
                   const aimx_grid* grid, int order, const StaticData* pre) {
    if (!mesh || !mat || !grid || !mesh->xyz || !mesh->tri || mesh->nv < 3 || mesh->nt < 1)
        throw Error{AIMX_E_ARG, "null or empty mesh/material/grid"};
    if (order < 1 || order > 3) throw Error{AIMX_E_ARG, "order must be 1..3"};
    if (mat->formulation != AIMX_EFIE && mat->formulation != AIMX_PMCHWT && mat->formulation != AIMX_CFIE)
        throw Error{AIMX_E_ARG, "unknown formulation"};
    if (mat->formulation == AIMX_CFIE && !(mat->cfie_alpha >= 0.0 && mat->cfie_alpha <= 1.0))
        throw Error{AIMX_E_ARG, "cfie_alpha must lie in (0, 1] (0 selects 1/2)"};
    for (int a = 0; a < 3; ++a)
        if (grid->n[a] < order + 2) throw Error{AIMX_E_ARG, "grid has too few nodes"};
    ctx->form = mat->formulation;
    ctx->eps_out = mat->eps_out > 0 ? mat->eps_out : 1.0;
    ctx->mu_out = mat->mu_out > 0 ? mat->mu_out : 1.0;
    ctx->eps_in = mat->eps_in > 0 ? mat->eps_in : 1.0;
    ctx->mu_in = mat->mu_in > 0 ? mat->mu_in : 1.0;
    ctx->sigma = (mat->formulation != AIMX_PMCHWT && mat->sigma > 0) ? mat->sigma : 0.0;
    ctx->cfie_alpha = mat->formulation == AIMX_CFIE && mat->cfie_alpha > 0 ? mat->cfie_alpha : 0.5;
    ctx->order = order;
    ctx->P = order + 1;
    ctx->U = ctx->P * ctx->P * ctx->P;
    ctx->radius = grid->near_radius > 0 ? grid->near_radius : 3;
    // grid fields per RHS: EFIE (J, rho); PMCHWT (J, rho, M, rho_M); CFIE (J, rho, K[J], unused)
    ctx->F = ctx->form == AIMX_EFIE ? 4 : 8;
    ctx->nspec = ctx->form == AIMX_EFIE ? 2 : (ctx->form == AIMX_CFIE ? 5 : 7);

    const int nv = mesh->nv, nt = mesh->nt;
    ctx->nv = nv;
    ctx->nt = nt;
    std::vector<double> xyz(mesh->xyz, mesh->xyz + 3 * (size_t)nv);
    std::vector<int> tri(mesh->tri, mesh->tri + 3 * (size_t)nt);
    for (int v : tri)
        if (v < 0 || v >= nv) throw Error{AIMX_E_MESH, "vertex id out of range"};

    // triangle geometry: area, centroid ((v0 + v1) + v2) / 3
    std::vector<double> area(nt), cen(3 * (size_t)nt);
    for (int t = 0; t < nt; ++t) {
        const double* a = &xyz[3 * tri[3 * t]];
        const double* b = &xyz[3 * tri[3 * t + 1]];
        const double* c = &xyz[3 * tri[3 * t + 2]];
        double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                        e1[0] * e2[1] - e1[1] * e2[0]};
        double n2 = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        if (!(n2 > 0.0)) throw Error{AIMX_E_MESH, "degenerate triangle"};
        area[t] = 0.5 * n2;
        for (int k = 0; k < 3; ++k) cen[3 * t + k] = ((a[k] + b[k]) + c[k]) / 3.0;
    }

    // RWG functions: one per edge shared by two oppositely oriented triangles
    struct HalfEdge {
        int a, b, t;
        bool fwd;
    };
    std::vector<HalfEdge> he;
    he.reserve(3 * (size_t)nt);
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) {
            int u = tri[3 * t + k], v = tri[3 * t + (k + 1) % 3];
            he.push_back(HalfEdge{std::min(u, v), std::max(u, v), t, u < v});
        }
    std::stable_sort(he.begin(), he.end(), [](const HalfEdge& x, const HalfEdge& y) {
        return x.a != y.a ? x.a < y.a : x.b < y.b;
    });
    std::vector<int> tp, tm, pp, pm, ea, eb;
    std::vector<double> blen;
    for (size_t s = 0; s < he.size();) {
        size_t e = s;
        while (e < he.size() && he[e].a == he[s].a && he[e].b == he[s].b) ++e;
        size_t cnt = e - s;
        if (cnt > 2) throw Error{AIMX_E_MESH, "edge shared by more than two triangles"};
        if (cnt == 2) {
            if (he[s].fwd == he[s + 1].fwd) throw Error{AIMX_E_MESH, "inconsistent triangle orientation"};
            int tplus = he[s].fwd ? he[s].t : he[s + 1].t;
            int tminus = he[s].fwd ? he[s + 1].t : he[s].t;
            auto freev = [&](int t) {
                for (int k = 0; k < 3; ++k) {
                    int v = tri[3 * t + k];
                    if (v != he[s].a && v != he[s].b) return v;
                }
                return -1;
            };
            tp.push_back(tplus);
            tm.push_back(tminus);
            ea.push_back(he[s].a);
            eb.push_back(he[s].b);
            pp.push_back(freev(tplus));
            pm.push_back(freev(tminus));
            const double* A = &xyz[3 * he[s].a];
            const double* B = &xyz[3 * he[s].b];
            double d[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
            blen.push_back(std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
        }
        s = e;
    }
    const int N = (int)tp.size();
    if (N == 0) throw Error{AIMX_E_MESH, "mesh has no interior edge"};
    ctx->N = N;
    ctx->h_xyz = xyz;
    ctx->h_ea = ea;
    ctx->h_eb = eb;
    ctx->h_tp = tp;
    ctx->h_tm = tm;
    ctx->h_cen = cen;
    ctx->nunk = two_blocks(ctx->form) ? 2 * N : N;

    // grid
    const int m = (order + 1) / 2;
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = hi[a] = xyz[a];
        for (int v = 1; v < nv; ++v) {
            lo[a] = std::min(lo[a], xyz[3 * v + a]);
            hi[a] = std::max(hi[a], xyz[3 * v + a]);
        }
    }
    bool auto_h = grid->h[0] == 0.0 && grid->h[1] == 0.0 && grid->h[2] == 0.0;
    for (int a = 0; a < 3; ++a) {
        ctx->n[a] = grid->n[a];
        if (auto_h) {
            double denom = (double)(grid->n[a] - 1 - 2 * m);
            if (!(denom > 0)) throw Error{AIMX_E_GRID, "grid too small for the stencil margin"};
            ctx->h[a] = (hi[a] - lo[a]) / denom;
            ctx->origin[a] = lo[a] - m * ctx->h[a];
        } else {
            ctx->h[a] = grid->h[a];
            ctx->origin[a] = grid->origin[a];
        }
        int pmin = 2 * grid->n[a] - 1;
        int pad = grid->pad[a] > 0 ? grid->pad[a] : next_fft_len(pmin);
        if (pad < pmin || !fft_len_ok(pad) || pad > kTwiddleLen)
            throw Error{AIMX_E_ARG, "pad must be 2^k or 3 * 2^k, >= 2n-1 and <= 4096"};
        ctx->M[a] = pad;
    }

    if (auto_h) {
        // an axis along which the mesh is flat takes the largest spacing of the others
        const double hmax = std::max(ctx->h[0], std::max(ctx->h[1], ctx->h[2]));
        for (int a = 0; a < 3; ++a)
            if (!(hi[a] - lo[a] > 0) && hmax > 0) {
                ctx->h[a] = hmax;
                ctx->origin[a] = lo[a] - m * hmax;
            }
    }
    for (int a = 0; a < 3; ++a)
        if (!(ctx->h[a] > 0)) throw Error{AIMX_E_GRID, "non-positive grid spacing"};

    // anchors s_a = floor((c_a - o_a) / h_a - (n - 1) / 2), caller order
    std::vector<int> anc0(3 * (size_t)N);
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) {
            double c = (cen[3 * tp[i] + a] + cen[3 * tm[i] + a]) * 0.5;
            double t = (c - ctx->origin[a]) / ctx->h[a] - (order - 1) / 2.0;
            double f = std::floor(t);
            if (!(f >= 0.0) || f + order > ctx->n[a] - 1)
                throw Error{AIMX_E_GRID, "stencil outside the grid"};
            anc0[3 * i + a] = (int)f;
        }

    // internal order: sorted by anchor (z, y, x), ties by caller index
    std::vector<int> perm(N);
    std::iota(perm.begin(), perm.end(), 0);
    auto key = [&](int i) {
        return ((int64_t)anc0[3 * i + 2] * ctx->n[1] + anc0[3 * i + 1]) * ctx->n[0] + anc0[3 * i];
    };
    std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return key(x) < key(y); });
    std::vector<int> iperm(N);
    for (int i = 0; i < N; ++i) iperm[perm[i]] = i;
    ctx->perm = perm;
    ctx->iperm = iperm;
    ctx->anc.resize(3 * (size_t)N);
    std::vector<int64_t> keys(N);
    for (int i = 0; i < N; ++i) {
        for (int a = 0; a < 3; ++a) ctx->anc[3 * i + a] = anc0[3 * perm[i] + a];
        keys[i] = key(perm[i]);
    }

    // near pairs: anchors within Chebyshev distance R; rows internal, columns ascending
    const int R = ctx->radius;
    std::vector<int> row_ptr(N + 1, 0);
    std::vector<int> cols;
    cols.reserve((size_t)N * 64);
    for (int i = 0; i < N; ++i) {
        const int* s = &ctx->anc[3 * i];
        size_t start = cols.size();
        for (int dz = -R; dz <= R; ++dz) {
            int z = s[2] + dz;
            if (z < 0 || z >= ctx->n[2]) continue;
            for (int dy = -R; dy <= R; ++dy) {
                int y = s[1] + dy;
                if (y < 0 || y >= ctx->n[1]) continue;
                int x0 = std::max(0, s[0] - R), x1 = std::min(ctx->n[0] - 1, s[0] + R);
                int64_t k0 = ((int64_t)z * ctx->n[1] + y) * ctx->n[0] + x0;
                int64_t k1 = ((int64_t)z * ctx->n[1] + y) * ctx->n[0] + x1;
                auto b = std::lower_bound(keys.begin(), keys.end(), k0);
                auto e = std::upper_bound(keys.begin(), keys.end(), k1);
                for (auto it = b; it != e; ++it) cols.push_back((int)(it - keys.begin()));
            }
        }
        std::sort(cols.begin() + start, cols.end());
        if (cols.size() > (size_t)INT32_MAX) throw Error{AIMX_E_NOMEM, "near list too large"};
        row_ptr[i + 1] = (int)cols.size();
    }
    ctx->row_ptr = row_ptr;
    ctx->cols = cols;
    ctx->nnz = (int64_t)cols.size();
    std::vector<int> row_of(cols.size());
    for (int i = 0; i < N; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) row_of[e] = i;

    // node-major gather lists: for each grid node, the (basis, stencil node) entries touching it
    const int P = ctx->P, U = ctx->U;
    const int64_t NG = (int64_t)ctx->n[0] * ctx->n[1] * ctx->n[2];
    std::vector<int> node_ptr(NG + 1, 0);
    for (int i = 0; i < N; ++i)
        for (int u = 0; u < U; ++u) {
            int x = ctx->anc[3 * i] + u % P, y = ctx->anc[3 * i + 1] + (u / P) % P,
                z = ctx->anc[3 * i + 2] + u / (P * P);
            node_ptr[((int64_t)z * ctx->n[1] + y) * ctx->n[0] + x + 1]++;
        }
    for (int64_t g = 0; g < NG; ++g) node_ptr[g + 1] += node_ptr[g];
    std::vector<int> fill(node_ptr.begin(), node_ptr.end() - 1);
    std::vector<int> node_w((size_t)N * U), node_x((size_t)N * U);
    for (int i = 0; i < N; ++i)
        for (int u = 0; u < U; ++u) {
            int x = ctx->anc[3 * i] + u % P, y = ctx->anc[3 * i + 1] + (u / P) % P,
                z = ctx->anc[3 * i + 2] + u / (P * P);
            int64_t g = ((int64_t)z * ctx->n[1] + y) * ctx->n[0] + x;
            int slot = fill[g]++;
            node_w[slot] = i * U + u;
            node_x[slot] = perm[i];
        }

    // bases touching each z plane (contiguous in internal order)
    ctx->plane_lo.assign(ctx->n[2], 0);
    ctx->plane_hi.assign(ctx->n[2], 0);
    for (int z = 0; z < ctx->n[2]; ++z) {
        int lo_i = 0, hi_i = 0;
        while (lo_i < N && ctx->anc[3 * lo_i + 2] < z - order) ++lo_i;
        hi_i = lo_i;
        while (hi_i < N && ctx->anc[3 * hi_i + 2] <= z) ++hi_i;
        ctx->plane_lo[z] = lo_i;
        ctx->plane_hi[z] = hi_i;
    }

    // per-basis geometry in internal order
    std::vector<int> btri(2 * (size_t)N), bfree(2 * (size_t)N);
    std::vector<double> blen_i(N);
    for (int i = 0; i < N; ++i) {
        int o = perm[i];
        btri[2 * i] = tp[o];
        btri[2 * i + 1] = tm[o];
        bfree[2 * i] = pp[o];
        bfree[2 * i + 1] = pm[o];
        blen_i[i] = blen[o];
    }

    // ---------------- device upload
    ctx->d_xyz = upload(ctx, xyz);
    ctx->d_tri = upload(ctx, tri);
    ctx->d_area = upload(ctx, area);
    ctx->d_btri = upload(ctx, btri);
    ctx->d_bfree = upload(ctx, bfree);
    ctx->d_blen = upload(ctx, blen_i);
    ctx->d_anc = upload(ctx, ctx->anc);
    ctx->d_perm = upload(ctx, perm);
    ctx->d_row_ptr = upload(ctx, row_ptr);
    ctx->d_cols = upload(ctx, cols);
    ctx->d_node_ptr = upload(ctx, node_ptr);
    ctx->d_node_w = upload(ctx, node_w);
    ctx->d_node_x = upload(ctx, node_x);
    int* d_row_of = upload(ctx, row_of);

    // quadrature tables
    std::vector<double> qp, qn;
    triangle_rule((3 * order + 4) / 2, qp);
    triangle_rule(5, qn);
    AIMX_CUDA_TRY(cudaMemcpyToSymbol(c_qproj, qp.data(), qp.size() * sizeof(double)));
    AIMX_CUDA_TRY(cudaMemcpyToSymbol(c_qnear, qn.data(), qn.size() * sizeof(double)));
    ctx->d_q5 = upload(ctx, qn);
    const int nq_proj = (int)qp.size() / 4, nq_near = (int)qn.size() / 4;

    GeomView gv{ctx->d_xyz, ctx->d_tri, ctx->d_area, ctx->d_btri, ctx->d_bfree, ctx->d_blen};

    // projection weights
    ctx->f64.w = (double*)dev_alloc(ctx, sizeof(double) * (size_t)N * U * 4);
    ctx->f32.w = (float*)dev_alloc(ctx, sizeof(float) * (size_t)N * U * 4);
    if (pre && (pre->w.size() != (size_t)N * U * 4 || pre->na.size() != (size_t)ctx->nnz ||
                pre->np.size() != (size_t)ctx->nnz || pre->nk.size() != (size_t)ctx->nnz ||
                pre->diag.size() != 3 * (size_t)N))
        throw Error{AIMX_E_IO, "static data does not match the mesh and grid"};
    {
        int threads = 128;
        int64_t tot = (int64_t)N * U;
        if (pre)
            AIMX_CUDA_TRY(cudaMemcpy(ctx->f64.w, pre->w.data(), sizeof(double) * pre->w.size(),
                                     cudaMemcpyHostToDevice));
        else
            k_weights<<<(unsigned)((tot + threads - 1) / threads), threads>>>(
                gv, ctx->d_anc, N, P, nq_proj, ctx->origin[0], ctx->origin[1], ctx->origin[2], ctx->h[0],
                ctx->h[1], ctx->h[2], ctx->f64.w);
        AIMX_CUDA_TRY(cudaGetLastError());
        size_t n4 = (size_t)N * U * 4;
        k_to_float<<<(unsigned)((n4 + 255) / 256), 256>>>(ctx->f64.w, ctx->f32.w, n4);
        ctx->d_wsoa = (float*)dev_alloc(ctx, sizeof(float) * n4);
        k_weights_soa<<<(unsigned)((n4 + 255) / 256), 256>>>(ctx->f64.w, ctx->d_wsoa, N, U);
        AIMX_CUDA_TRY(cudaGetLastError());
        if (ctx->form == AIMX_CFIE) {
            const size_t n3 = (size_t)N * U * 3;
            ctx->f64.wg = (double*)dev_alloc(ctx, sizeof(double) * n3);
            ctx->f32.wg = (float*)dev_alloc(ctx, sizeof(float) * n3);
            k_weights_g<<<(unsigned)((tot + threads - 1) / threads), threads>>>(
                gv, ctx->d_anc, N, P, nq_proj, ctx->origin[0], ctx->origin[1], ctx->origin[2], ctx->h[0],
                ctx->h[1], ctx->h[2], ctx->f64.wg);
            k_to_float<<<(unsigned)((n3 + 255) / 256), 256>>>(ctx->f64.wg, ctx->f32.wg, n3);
            AIMX_CUDA_TRY(cudaGetLastError());
        }
    }

    // static near integrals + precorrection
    const int64_t nnz = ctx->nnz;
    if (pre) {
        auto put = [&](const std::vector<double>& h, double*& d64, float*& d32) {
            d64 = (double*)dev_alloc(ctx, sizeof(double) * h.size());
            d32 = (float*)dev_alloc(ctx, sizeof(float) * h.size());
            AIMX_CUDA_TRY(cudaMemcpy(d64, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice));
            k_to_float<<<(unsigned)((h.size() + 255) / 256), 256>>>(d64, d32, h.size());
            AIMX_CUDA_TRY(cudaGetLastError());
        };
        put(pre->na, ctx->f64.na, ctx->f32.na);
        put(pre->np, ctx->f64.np, ctx->f32.np);
        put(pre->nk, ctx->f64.nk, ctx->f32.nk);
        ctx->d_diag = upload(ctx, pre->diag);
        build_gram(ctx, gv, d_row_of);
        AIMX_CUDA_TRY(cudaDeviceSynchronize());
        dev_free(ctx, d_row_of);
        return;
    }
    double* d_LA = (double*)dev_alloc(ctx, sizeof(double) * nnz);
    double* d_LP = (double*)dev_alloc(ctx, sizeof(double) * nnz);
    double* d_KK = (double*)dev_alloc(ctx, sizeof(double) * nnz);
    ctx->f64.na = (double*)dev_alloc(ctx, sizeof(double) * nnz);
    ctx->f64.np = (double*)dev_alloc(ctx, sizeof(double) * nnz);
    ctx->f64.nk = (double*)dev_alloc(ctx, sizeof(double) * nnz);
    ctx->f32.na = (float*)dev_alloc(ctx, sizeof(float) * nnz);
    ctx->f32.np = (float*)dev_alloc(ctx, sizeof(float) * nnz);
    ctx->f32.nk = (float*)dev_alloc(ctx, sizeof(float) * nnz);
    {
        int threads = 128;
        k_near_static<<<(unsigned)((nnz + threads - 1) / threads), threads>>>(
            gv, d_row_of, ctx->d_cols, nnz, nq_near, ctx->form == AIMX_CFIE ? 1 : 0, d_LA, d_LP, d_KK);
        AIMX_CUDA_TRY(cudaGetLastError());
    }
    // static grid kernel tables over offsets [-span, span]^3
    const int span = R + order;
    const int D = 2 * span + 1;
    std::vector<double> hs((size_t)D * D * D), hg(3 * (size_t)D * D * D);
    for (int iz = 0; iz < D; ++iz)
        for (int iy = 0; iy < D; ++iy)
            for (int ix = 0; ix < D; ++ix) {
                size_t t = ((size_t)iz * D + iy) * D + ix;
                double rx = (ix - span) * ctx->h[0], ry = (iy - span) * ctx->h[1],
                       rz = (iz - span) * ctx->h[2];
                double r = std::sqrt(rx * rx + ry * ry + rz * rz);
                if (ix == span && iy == span && iz == span) {
                    hs[t] = 0.0;
                    hg[3 * t] = hg[3 * t + 1] = hg[3 * t + 2] = 0.0;
                } else {
                    hs[t] = 1.0 / (4.0 * kPi * r);
                    double c = -1.0 / (4.0 * kPi * r * r * r);
                    hg[3 * t] = c * rx;
                    hg[3 * t + 1] = c * ry;
                    hg[3 * t + 2] = c * rz;
                }
            }
    double* d_hs = upload(ctx, hs);
    double* d_hg = upload(ctx, hg);
    {
        int threads = 128;
        k_precorrect<<<(unsigned)((nnz + threads - 1) / threads), threads>>>(
            ctx->f64.w, ctx->f64.wg, ctx->d_anc, d_row_of, ctx->d_cols, nnz, P, span, d_hs, d_hg, d_LA, d_LP, d_KK,
            ctx->f64.na, ctx->f64.np, ctx->f64.nk, ctx->f32.na, ctx->f32.np, ctx->f32.nk);
        AIMX_CUDA_TRY(cudaGetLastError());
    }
    ctx->d_diag = (double*)dev_alloc(ctx, sizeof(double) * 3 * (size_t)N);
    k_diag<<<(N + 127) / 128, 128>>>(ctx->d_row_ptr, ctx->d_cols, d_LA, d_LP, d_KK, N, ctx->d_diag);
    AIMX_CUDA_TRY(cudaGetLastError());
    build_gram(ctx, gv, d_row_of);
    AIMX_CUDA_TRY(cudaDeviceSynchronize());
    dev_free(ctx, d_LA);
    dev_free(ctx, d_LP);
    dev_free(ctx, d_KK);
    dev_free(ctx, d_hs);
    dev_free(ctx, d_hg);
    dev_free(ctx, d_row_of);
}

}  // namespace aimx
