// Frequency-dependent preconditioners built from the AIMx operator's entries.
//
// AIMX_PRECOND_DIAG: inverse of the per-basis static self block (the diagonal
// of L_s, Sec. III-A-2): a scalar for the EFIE, a 2x2 (J, M) block for the
// two-region form.
//
// AIMX_PRECOND_BLOCK: block Jacobi over groups of bases whose anchors share a
// 2 x 2 x 2 cell (at most kBlockMax bases per group).  Every pair in a group
// is a near pair, so each block entry is the full AIMx matrix entry
//
//     Z(m, n) = coefficients x ( N(m, n) + sum_{u,v} Lambda[u,m] H(k)[s_m+u-s_n-v] Lambda[v,n] )
//
// i.e. the static near matrix augmented with the grid-generated
// frequency-dependent part on the selected entries (Sec. III-A-2: off-diagonal
// preconditioner entries generated with the FFT operator instead of direct
// integration).  Blocks are assembled and inverted (Gauss-Jordan, partial
// pivoting) in FP64 on the device once per frequency; the inverse is applied
// in FP32.

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "aimx_internal.h"
#include "cplx.cuh"

namespace aimx {

constexpr int kBlockMax = 32;   // bases per block (unknowns: 32 EFIE, 64 two-region)

static inline unsigned nb_(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------ partition (host, once per context)

static void build_partition(aimx_ctx* ctx) {
    if (ctx->pc.nblk > 0) return;
    const int N = ctx->N;
    const int cx = (ctx->n[0] + 1) / 2, cy = (ctx->n[1] + 1) / 2;
    std::vector<std::pair<int64_t, int>> keyed(N);
    for (int i = 0; i < N; ++i) {
        const int* s = &ctx->anc[3 * i];
        int64_t key = ((int64_t)(s[2] >> 1) * cy + (s[1] >> 1)) * cx + (s[0] >> 1);
        keyed[i] = {key, i};
    }
    std::stable_sort(keyed.begin(), keyed.end());
    std::vector<int> ptr{0}, idx;
    idx.reserve(N);
    for (size_t a = 0; a < keyed.size();) {
        size_t b = a;
        while (b < keyed.size() && keyed[b].first == keyed[a].first) ++b;
        for (size_t c = a; c < b; c += kBlockMax) {
            for (size_t d = c; d < std::min(b, c + kBlockMax); ++d) idx.push_back(keyed[d].second);
            ptr.push_back((int)idx.size());
        }
        a = b;
    }
    int mx = 0;
    for (size_t k = 0; k + 1 < ptr.size(); ++k) mx = std::max(mx, ptr[k + 1] - ptr[k]);
    ctx->pc.nblk = (int)ptr.size() - 1;
    ctx->pc.maxnb = mx;
    ctx->pc.D = ctx->form == AIMX_EFIE ? mx : 2 * mx;
    ctx->pc.d_ptr = (int*)dev_alloc(ctx, sizeof(int) * ptr.size());
    ctx->pc.d_idx = (int*)dev_alloc(ctx, sizeof(int) * idx.size());
    AIMX_CUDA_TRY(cudaMemcpy(ctx->pc.d_ptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice));
    AIMX_CUDA_TRY(cudaMemcpy(ctx->pc.d_idx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice));
}

// ------------------------------------------------------------------ block assembly

struct RegionTables {
    int nreg;
    int span;            // offsets in [-span, span]^3
    double2 cA[2], cP[2];  // per region: multiplier of (N^A + G^A) and of (N^Phi + G^Phi) in the E (or EFIE) rows
    double2 dA[2], dP[2];  // the same in the H rows (two-region form)
    double cK;             // eta0 (K blocks: E-M gets +cK * sum_regions, H-J gets -cK * sum_regions)
    double2 zs;            // surface impedance multiplying the Gram matrix (EFIE), 0 without
};

__device__ inline double near_value(const int* row_ptr, const int* cols, const double* vals, int m, int n) {
    int lo = row_ptr[m], hi = row_ptr[m + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int c = cols[mid];
        if (c == n) return vals[mid];
        if (c < n) lo = mid + 1; else hi = mid - 1;
    }
    return 0.0;
}

// One thread per (block, basis pair): full AIMx entries of the block into work[blk][D][D].
__global__ void k_block_assemble(const int* __restrict__ bptr, const int* __restrict__ bidx, int nblk, int D,
                                 const int* __restrict__ anc, const double* __restrict__ w, int P,
                                 const int* __restrict__ row_ptr, const int* __restrict__ cols,
                                 const double* __restrict__ na, const double* __restrict__ np,
                                 const double* __restrict__ nk, const double2* __restrict__ H,
                                 const double2* __restrict__ Hg, RegionTables rt, int form, double2* work) {
    const int blk = blockIdx.x;
    const int b0 = bptr[blk], nb = bptr[blk + 1] - b0;
    const int U = P * P * P;
    const int S = 2 * rt.span + 1;
    const int64_t ST = (int64_t)S * S * S;
    double2* Z = work + (int64_t)blk * D * D;
    const int Deff = form == AIMX_EFIE ? nb : 2 * nb;
    for (int t = threadIdx.x; t < D * D; t += blockDim.x) {
        int l = t / D, c = t % D;
        if (l >= Deff || c >= Deff) Z[t] = make_double2(l == c ? 1.0 : 0.0, 0.0);
    }
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int lm = t / nb, ln = t % nb;
        const int m = bidx[b0 + lm], n = bidx[b0 + ln];
        const double vA = near_value(row_ptr, cols, na, m, n);
        const double vP = near_value(row_ptr, cols, np, m, n);
        const double vK = form == AIMX_EFIE ? 0.0 : near_value(row_ptr, cols, nk, m, n);
        double2 GA[2] = {make_double2(0, 0), make_double2(0, 0)}, GP[2] = {make_double2(0, 0), make_double2(0, 0)},
                GK[2] = {make_double2(0, 0), make_double2(0, 0)};
        const double* wm = w + (int64_t)m * U * 4;
        const double* wn = w + (int64_t)n * U * 4;
        const int dx0 = anc[3 * m] - anc[3 * n], dy0 = anc[3 * m + 1] - anc[3 * n + 1],
                  dz0 = anc[3 * m + 2] - anc[3 * n + 2];
        for (int u = 0; u < U; ++u) {
            const int ux = u % P, uy = (u / P) % P, uz = u / (P * P);
            const double a0 = wm[4 * u], a1 = wm[4 * u + 1], a2 = wm[4 * u + 2], a3 = wm[4 * u + 3];
            for (int v = 0; v < U; ++v) {
                const int vx = v % P, vy = (v / P) % P, vz = v / (P * P);
                const int64_t ti = ((int64_t)(dz0 + uz - vz + rt.span) * S + (dy0 + uy - vy + rt.span)) * S +
                                   (dx0 + ux - vx + rt.span);
                const double b0v = wn[4 * v], b1 = wn[4 * v + 1], b2 = wn[4 * v + 2], b3 = wn[4 * v + 3];
                const double sA = a0 * b0v + a1 * b1 + a2 * b2, sP = a3 * b3;
                // a . (e_x x b) etc.: cross-product weights for the three gradient components
                const double kx = a1 * b2 - a2 * b1, ky = a2 * b0v - a0 * b2, kz = a0 * b1 - a1 * b0v;
                for (int g = 0; g < rt.nreg; ++g) {
                    const double2 h = H[g * ST + ti];
                    GA[g] = GA[g] + sA * h;
                    GP[g] = GP[g] + sP * h;
                    if (form != AIMX_EFIE) {
                        const double2* hg = Hg + (int64_t)g * 3 * ST;
                        // a . (hg x b) = hg . (b x a) = -(hg . (a x b))
                        GK[g] = GK[g] - (kx * hg[ti] + ky * hg[ST + ti] + kz * hg[2 * ST + ti]);
                    }
                }
            }
        }
        if (form == AIMX_EFIE) {
            double2 z = rt.cA[0] * (make_double2(vA, 0) + GA[0]) + rt.cP[0] * (make_double2(vP, 0) + GP[0]);
            if (nk) z = z + near_value(row_ptr, cols, nk, m, n) * rt.zs;   // nk carries the Gram matrix here
            Z[lm * D + ln] = z;
        } else {
            double2 eJ = make_double2(0, 0), hM = make_double2(0, 0), k = make_double2(0, 0);
            for (int g = 0; g < rt.nreg; ++g) {
                const double2 LA = make_double2(vA, 0) + GA[g], LP = make_double2(vP, 0) + GP[g];
                eJ = eJ + rt.cA[g] * LA + rt.cP[g] * LP;
                hM = hM + rt.dA[g] * LA + rt.dP[g] * LP;
                k = k + (make_double2(vK, 0) + GK[g]);
            }
            Z[lm * D + ln] = eJ;
            Z[lm * D + nb + ln] = rt.cK * k;
            Z[(nb + lm) * D + ln] = -rt.cK * k;
            Z[(nb + lm) * D + nb + ln] = hM;
        }
    }
}

// One thread per block: Gauss-Jordan inverse with partial pivoting (FP64, in
// place in work), written as FP32 to inv.
__global__ void k_block_invert(double2* work, float2* inv, int nblk, int D) {
    const int blk = blockIdx.x * blockDim.x + threadIdx.x;
    if (blk >= nblk) return;
    double2* A = work + (int64_t)blk * D * D;
    // augment implicitly: track the inverse in place using the standard
    // in-place Gauss-Jordan with a column permutation record
    int piv[64];
    for (int k = 0; k < D; ++k) {
        int p = k;
        double best = A[k * D + k].x * A[k * D + k].x + A[k * D + k].y * A[k * D + k].y;
        for (int r = k + 1; r < D; ++r) {
            double mag = A[r * D + k].x * A[r * D + k].x + A[r * D + k].y * A[r * D + k].y;
            if (mag > best) {
                best = mag;
                p = r;
            }
        }
        piv[k] = p;
        if (p != k)
            for (int c = 0; c < D; ++c) {
                double2 t = A[k * D + c];
                A[k * D + c] = A[p * D + c];
                A[p * D + c] = t;
            }
        double2 d = A[k * D + k];
        double den = d.x * d.x + d.y * d.y;
        double2 di = den > 0 ? make_double2(d.x / den, -d.y / den) : make_double2(0.0, 0.0);
        A[k * D + k] = make_double2(1.0, 0.0);
        for (int c = 0; c < D; ++c) A[k * D + c] = A[k * D + c] * di;
        for (int r = 0; r < D; ++r) {
            if (r == k) continue;
            double2 f = A[r * D + k];
            if (f.x == 0.0 && f.y == 0.0) continue;
            A[r * D + k] = make_double2(0.0, 0.0);
            for (int c = 0; c < D; ++c) A[r * D + c] = A[r * D + c] - f * A[k * D + c];
        }
    }
    // undo the row interchanges as column interchanges of the inverse
    for (int k = D - 1; k >= 0; --k) {
        int p = piv[k];
        if (p != k)
            for (int r = 0; r < D; ++r) {
                double2 t = A[r * D + k];
                A[r * D + k] = A[r * D + p];
                A[r * D + p] = t;
            }
    }
    float2* out = inv + (int64_t)blk * D * D;
    for (int t = 0; t < D * D; ++t) out[t] = make_float2((float)A[t].x, (float)A[t].y);
}

// z = M v per block: v FP64 with per-RHS stride vstride, z of type T with stride nunk.
template <class T>
__global__ void k_block_apply(const float2* __restrict__ inv, const int* __restrict__ bptr,
                              const int* __restrict__ bidx, const int* __restrict__ perm, int D, int N, int form,
                              const double2* __restrict__ v, int64_t vstride, cplx_t<T>* z, int nunk, int nrhs) {
    extern __shared__ float2 smv[];   // [D][8]
    const int blk = blockIdx.x;
    const int r0 = blockIdx.y * 8;
    const int nr = min(8, nrhs - r0);
    const int b0 = bptr[blk], nb = bptr[blk + 1] - b0;
    const int Deff = form == AIMX_EFIE ? nb : 2 * nb;
    auto gidx = [&](int l) {
        return l < nb ? perm[bidx[b0 + l]] : N + perm[bidx[b0 + l - nb]];
    };
    for (int t = threadIdx.x; t < Deff * nr; t += blockDim.x) {
        const int l = t % Deff, r = t / Deff;
        const double2 x = v[(int64_t)(r0 + r) * vstride + gidx(l)];
        smv[l * 8 + r] = make_float2((float)x.x, (float)x.y);
    }
    __syncthreads();
    const float2* M = inv + (int64_t)blk * D * D;
    for (int t = threadIdx.x; t < Deff * nr; t += blockDim.x) {
        const int l = t % Deff, r = t / Deff;
        float2 acc = make_float2(0.f, 0.f);
        for (int c = 0; c < Deff; ++c) cfma(acc, M[l * D + c], smv[c * 8 + r]);
        z[(int64_t)(r0 + r) * nunk + gidx(l)] = mk((T)acc.x, (T)acc.y);
    }
}

// ------------------------------------------------------------------ host driver

static void region_tables(const aimx_ctx* ctx, double freq, int span, std::vector<double2>& H,
                          std::vector<double2>& Hg, RegionTables& rt) {
    const double w = 2.0 * kPi * freq;
    const int nreg = ctx->form == AIMX_EFIE ? 1 : 2;
    double mu[2] = {kMu0 * ctx->mu_out, kMu0 * ctx->mu_in};
    double eps[2] = {kEps0 * ctx->eps_out, kEps0 * ctx->eps_in};
    const int S = 2 * span + 1;
    const size_t ST = (size_t)S * S * S;
    H.assign(nreg * ST, make_double2(0, 0));
    Hg.assign(nreg * 3 * ST, make_double2(0, 0));
    rt.nreg = nreg;
    rt.span = span;
    rt.cK = kEta0;
    rt.zs = near_coefs(ctx, freq).near[2];
    if (ctx->form != AIMX_EFIE) rt.zs = make_double2(0.0, 0.0);
    for (int g = 0; g < nreg; ++g) {
        const double k = w * std::sqrt(mu[g] * eps[g]);
        for (int iz = 0; iz < S; ++iz)
            for (int iy = 0; iy < S; ++iy)
                for (int ix = 0; ix < S; ++ix) {
                    const size_t t = ((size_t)iz * S + iy) * S + ix;
                    const double rx = (ix - span) * ctx->h[0], ry = (iy - span) * ctx->h[1], rz = (iz - span) * ctx->h[2];
                    const double r = std::sqrt(rx * rx + ry * ry + rz * rz);
                    if (ix == span && iy == span && iz == span) {
                        H[g * ST + t] = make_double2(0.0, -k / (4.0 * kPi));
                    } else {
                        const std::complex<double> e = std::exp(std::complex<double>(0.0, -k * r));
                        const std::complex<double> G = e / (4.0 * kPi * r);
                        H[g * ST + t] = make_double2(G.real(), G.imag());
                        const std::complex<double> f = -(1.0 + std::complex<double>(0.0, k * r)) * e / (4.0 * kPi * r * r * r);
                        const double comp[3] = {rx, ry, rz};
                        for (int a = 0; a < 3; ++a) {
                            std::complex<double> v = f * comp[a];
                            Hg[(g * 3 + a) * ST + t] = make_double2(v.real(), v.imag());
                        }
                    }
                }
        if (ctx->form == AIMX_EFIE) {
            rt.cA[g] = make_double2(0.0, w * mu[g]);
            rt.cP[g] = make_double2(0.0, -w * mu[g] / (k * k));
        } else {
            rt.cA[g] = make_double2(0.0, w * mu[g]);
            rt.cP[g] = make_double2(0.0, -w * mu[g] / (k * k));
            rt.dA[g] = make_double2(0.0, kEta0 * kEta0 * w * eps[g]);
            rt.dP[g] = make_double2(0.0, -kEta0 * kEta0 * w * eps[g] / (k * k));
        }
    }
}

void precond_block_prepare(aimx_ctx* ctx, double freq, cudaStream_t s) {
    if (ctx->form == AIMX_CFIE)
        throw Error{AIMX_E_STATE, "the block preconditioner covers EFIE and PMCHWT contexts"};
    build_partition(ctx);
    if (ctx->pc.freq == freq && ctx->pc.d_inv) return;
    const int D = ctx->pc.D, nblk = ctx->pc.nblk;
    if (!ctx->pc.d_work) ctx->pc.d_work = (double2*)dev_alloc(ctx, sizeof(double2) * (size_t)nblk * D * D);
    if (!ctx->pc.d_inv) ctx->pc.d_inv = (float2*)dev_alloc(ctx, sizeof(float2) * (size_t)nblk * D * D);
    const int span = 1 + ctx->order;   // anchors in one 2x2x2 cell differ by at most 1 per axis
    std::vector<double2> H, Hg;
    RegionTables rt;
    region_tables(ctx, freq, span, H, Hg, rt);
    double2* dH = (double2*)dev_alloc(ctx, sizeof(double2) * H.size());
    double2* dHg = (double2*)dev_alloc(ctx, sizeof(double2) * Hg.size());
    AIMX_CUDA_TRY(cudaMemcpyAsync(dH, H.data(), sizeof(double2) * H.size(), cudaMemcpyHostToDevice, s));
    AIMX_CUDA_TRY(cudaMemcpyAsync(dHg, Hg.data(), sizeof(double2) * Hg.size(), cudaMemcpyHostToDevice, s));
    k_block_assemble<<<nblk, 128, 0, s>>>(ctx->pc.d_ptr, ctx->pc.d_idx, nblk, D, ctx->d_anc, ctx->f64.w, ctx->P,
                                          ctx->d_row_ptr, ctx->d_cols, ctx->f64.na, ctx->f64.np,
                                          ctx->form == AIMX_EFIE ? ctx->f64.ng : ctx->f64.nk, dH, dHg,
                                          rt, ctx->form, ctx->pc.d_work);
    AIMX_CUDA_TRY(cudaGetLastError());
    k_block_invert<<<nb_(nblk, 64), 64, 0, s>>>(ctx->pc.d_work, ctx->pc.d_inv, nblk, D);
    AIMX_CUDA_TRY(cudaGetLastError());
    AIMX_CUDA_TRY(cudaStreamSynchronize(s));
    dev_free(ctx, dH);
    dev_free(ctx, dHg);
    ctx->pc.freq = freq;
}

template <class T>
void precond_block_apply(aimx_ctx* ctx, const double2* v, int64_t vstride, cplx_t<T>* z, int nrhs, cudaStream_t s) {
    dim3 grid(ctx->pc.nblk, (nrhs + 7) / 8);
    size_t sm = sizeof(float2) * (size_t)ctx->pc.D * 8;
    k_block_apply<T><<<grid, 128, sm, s>>>(ctx->pc.d_inv, ctx->pc.d_ptr, ctx->pc.d_idx, ctx->d_perm, ctx->pc.D,
                                           ctx->N, ctx->form, v, vstride, z, ctx->nunk, nrhs);
    AIMX_CUDA_TRY(cudaGetLastError());
}

template void precond_block_apply<float>(aimx_ctx*, const double2*, int64_t, float2*, int, cudaStream_t);
template void precond_block_apply<double>(aimx_ctx*, const double2*, int64_t, double2*, int, cudaStream_t);

}  // namespace aimx
