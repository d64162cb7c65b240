// Conventional-AIM comparison mode for the EFIE (Sec. II-B): at every new
// frequency the near-region entries are integrated directly with the full
// Green's function and precorrected with the grid kernel H(k),
//
//     Z_near(k) = j w mu [ N^A(k) - k^-2 N^Phi(k) ],
//     N(k) = L_NR(k) - L_P(k),   L_P(k) = sum_{u,v} Lambda[u,m] H(k)[s_m+u-s_n-v] Lambda[v,n],
//
// where AIMx keeps one static, real near matrix per operator.  L_NR(k) splits
// G = G_s + G_d(k): the G_s part with the closed-form inner potentials and the
// 5 x 5 outer rule (as in setup), the smooth G_d part with the 5 x 5 product
// rule on both triangles.  Nothing is cached across frequencies: this is the
// per-frequency matrix fill the paper's method removes.

#include <cmath>
#include <vector>

#include "aimx_internal.h"
#include "cplx.cuh"
#include "geom.cuh"

namespace aimx {

// G_d(k, R) = (e^{-jkR} - 1) / (4 pi R); the real part as -2 sin^2(kR/2) / (4 pi R)
// (no cancellation at small kR), sin(kR) = 2 sin(kR/2) cos(kR/2); -jk / (4 pi) at R = 0.
__device__ inline double2 green_d(double k, double R) {
    if (R > 0.0) {
        double s, c;
        sincos(0.5 * k * R, &s, &c);
        const double inv = 1.0 / (4.0 * kPi * R);
        return make_double2(-2.0 * s * s * inv, -2.0 * s * c * inv);
    }
    return make_double2(0.0, -k / (4.0 * kPi));
}

// One thread per near pair (row i, column j), internal order.  q5: [25][4]
// collapsed Gauss rule (l1, l2, l3, w); htab: H(k) on offsets [-span, span]^3.
__global__ void __launch_bounds__(128) k_aim_near(GeomView g, const int* __restrict__ row_of,
                                                  const int* __restrict__ cols, int64_t nnz,
                                                  const double* __restrict__ q5, double k,
                                                  const double* __restrict__ w, const int* __restrict__ anc, int P,
                                                  int span, const double2* __restrict__ htab, double2 cA,
                                                  double2 cP, double2* zn64, float2* zn32) {
    __shared__ double sq[25 * 4];
    for (int t = threadIdx.x; t < 100; t += blockDim.x) sq[t] = q5[t];
    __syncthreads();
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const int i = row_of[e], j = cols[e];
    double2 la = make_double2(0, 0), lp = make_double2(0, 0);
    const double inv4pi = 1.0 / (4.0 * kPi);
    for (int ss = 0; ss < 2; ++ss) {
        const int ts = g.btri[2 * j + ss];
        const double sgs = ss == 0 ? 1.0 : -1.0;
        const double As = g.area[ts];
        const double cs = g.blen[j] / (2.0 * As);
        const V3 ps = load3(g.xyz + 3 * g.bfree[2 * j + ss]);
        TriFrame T;
        make_frame(T, vtx(g, ts, 0), vtx(g, ts, 1), vtx(g, ts, 2));
        const double dvs = sgs * 2.0 * cs;
        for (int so = 0; so < 2; ++so) {
            const int to = g.btri[2 * i + so];
            const double sgo = so == 0 ? 1.0 : -1.0;
            const double Ao = g.area[to];
            const double co = g.blen[i] / (2.0 * Ao);
            const V3 po = load3(g.xyz + 3 * g.bfree[2 * i + so]);
            const V3 a = vtx(g, to, 0), b = vtx(g, to, 1), c = vtx(g, to, 2);
            const double dvo = sgo * 2.0 * co;
            for (int q = 0; q < 25; ++q) {
                const V3 r = sq[4 * q] * a + sq[4 * q + 1] * b + sq[4 * q + 2] * c;
                const double W = sq[4 * q + 3] * Ao;
                const V3 fo = (sgo * co) * (r - po);
                // G_s: closed-form inner potentials
                double I1;
                V3 J, G, rho;
                tri_potentials(T, r, I1, J, G, rho);
                const V3 vp = (sgs * cs) * (J + I1 * (rho - ps));
                la.x += W * dot(fo, vp) * inv4pi;
                lp.x += W * dvo * dvs * I1 * inv4pi;
                // G_d(k): product rule over the source triangle
                double2 ga = make_double2(0, 0), gp = make_double2(0, 0);
                for (int q2 = 0; q2 < 25; ++q2) {
                    const V3 rs = sq[4 * q2] * T.v[0] + sq[4 * q2 + 1] * T.v[1] + sq[4 * q2 + 2] * T.v[2];
                    const double Ws = sq[4 * q2 + 3] * As;
                    const double2 gd = Ws * green_d(k, norm3(r - rs));
                    const double ff = dot(fo, (sgs * cs) * (rs - ps));
                    ga = ga + ff * gd;
                    gp = gp + gd;
                }
                la = la + W * ga;
                lp = lp + (W * dvo * dvs) * gp;
            }
        }
    }
    // precorrection with the grid kernel between the two stencils
    const int U = P * P * P;
    const int D = 2 * span + 1;
    const int dx0 = anc[3 * i] - anc[3 * j] + span, dy0 = anc[3 * i + 1] - anc[3 * j + 1] + span,
              dz0 = anc[3 * i + 2] - anc[3 * j + 2] + span;
    const double* wi = w + (size_t)i * U * 4;
    const double* wj = w + (size_t)j * U * 4;
    double2 pa = make_double2(0, 0), pp = make_double2(0, 0);
    for (int u = 0; u < U; ++u) {
        const int ux = u % P, uy = (u / P) % P, uz = u / (P * P);
        const double a0 = wi[4 * u], a1 = wi[4 * u + 1], a2 = wi[4 * u + 2], a3 = wi[4 * u + 3];
        for (int v = 0; v < U; ++v) {
            const int vx = v % P, vy = (v / P) % P, vz = v / (P * P);
            const double2 hk = __ldg(htab + ((dz0 + uz - vz) * D + (dy0 + uy - vy)) * D + (dx0 + ux - vx));
            const double* bv = wj + 4 * v;
            pa = pa + (a0 * bv[0] + a1 * bv[1] + a2 * bv[2]) * hk;
            pp = pp + (a3 * bv[3]) * hk;
        }
    }
    const double2 z = cA * (la - pa) + cP * (lp - pp);
    zn64[e] = z;
    zn32[e] = make_float2((float)z.x, (float)z.y);
}

void aim_enable(aimx_ctx* ctx) {
    if (ctx->form != AIMX_EFIE) throw Error{AIMX_E_STATE, "the conventional-AIM mode is defined for EFIE contexts"};
    const int64_t nnz = ctx->nnz;
    if (!ctx->d_aim_row_of) {
        std::vector<int> row_of(nnz);
        for (int i = 0; i < ctx->N; ++i)
            for (int e = ctx->row_ptr[i]; e < ctx->row_ptr[i + 1]; ++e) row_of[e] = i;
        ctx->d_aim_row_of = (int*)dev_alloc(ctx, sizeof(int) * nnz);
        AIMX_CUDA_TRY(cudaMemcpy(ctx->d_aim_row_of, row_of.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice));
        ctx->f64.zn = (double*)dev_alloc(ctx, sizeof(double2) * nnz);
        ctx->f32.zn = (float*)dev_alloc(ctx, sizeof(float2) * nnz);
        const int span = ctx->radius + ctx->order;
        const int D = 2 * span + 1;
        ctx->d_aim_htab = (double*)dev_alloc(ctx, sizeof(double2) * (size_t)D * D * D);
    }
    ctx->aim_freq = -1.0;
}

void ensure_aim_near(aimx_ctx* ctx, double freq, cudaStream_t s) {
    if (!ctx->aim || ctx->aim_freq == freq) return;
    if (!(freq > 0.0)) throw Error{AIMX_E_ARG, "frequency must be positive"};
    StageScope sc(ctx, ST_AIM_FILL, s);
    const Coefs cf = near_coefs(ctx, freq);
    const double k = 2.0 * kPi * freq * std::sqrt(kMu0 * ctx->mu_out * kEps0 * ctx->eps_out);
    const int span = ctx->radius + ctx->order;
    const int D = 2 * span + 1;
    std::vector<double2>& ht = ctx->h_aim_htab;
    ht.resize((size_t)D * D * D);
    for (int iz = 0; iz < D; ++iz)
        for (int iy = 0; iy < D; ++iy)
            for (int ix = 0; ix < D; ++ix) {
                const double rx = (ix - span) * ctx->h[0], ry = (iy - span) * ctx->h[1],
                             rz = (iz - span) * ctx->h[2];
                const double r = std::sqrt(rx * rx + ry * ry + rz * rz);
                double2 v;
                if (r > 0.0)
                    v = make_double2(std::cos(k * r) / (4.0 * kPi * r), -std::sin(k * r) / (4.0 * kPi * r));
                else
                    v = make_double2(0.0, -k / (4.0 * kPi));   // AIMx self-term, as in the grid kernel
                ht[((size_t)iz * D + iy) * D + ix] = v;
            }
    AIMX_CUDA_TRY(cudaMemcpyAsync(ctx->d_aim_htab, ht.data(), sizeof(double2) * ht.size(), cudaMemcpyHostToDevice, s));
    GeomView gv{ctx->d_xyz, ctx->d_tri, ctx->d_area, ctx->d_btri, ctx->d_bfree, ctx->d_blen};
    const int64_t nnz = ctx->nnz;
    k_aim_near<<<(unsigned)((nnz + 127) / 128), 128, 0, s>>>(
        gv, ctx->d_aim_row_of, ctx->d_cols, nnz, ctx->d_q5, k, ctx->f64.w, ctx->d_anc, ctx->P, span,
        reinterpret_cast<const double2*>(ctx->d_aim_htab), cf.near[0], cf.near[1],
        reinterpret_cast<double2*>(ctx->f64.zn), reinterpret_cast<float2*>(ctx->f32.zn));
    AIMX_CUDA_TRY(cudaGetLastError());
    // the host table must outlive the copy
    AIMX_CUDA_TRY(cudaStreamSynchronize(s));
    ctx->aim_freq = freq;
}

}  // namespace aimx
