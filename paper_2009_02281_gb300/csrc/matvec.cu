// AIMx matrix-vector product, generic path (any precision, any power-of-two pad).
//
//   y = N x + W H(k) P x                                   (Eq. LAIMx / Eq. KAIMx)
//
// 1. projection P: each grid node gathers the weighted coefficients of the
//    bases whose stencil contains it (node-major lists, no atomics);
// 2. zero-padded 3-D FFT, per-point multiply with the kernel spectra
//    (scalar L parts; cross product with the gradient spectra for K),
//    inverse FFT;
// 3. interpolation W = P^T and the sparse near correction, written once.

#include <cufft.h>

#include "aimx_internal.h"
#include "cplx.cuh"

namespace aimx {


// Fields per RHS: EFIE (Jx, Jy, Jz, rho); PMCHWT adds (Mx, My, Mz, rho_M).
// Field f uses weight component f % 4 and unknown block f / 4.  F fields are
// projected into grids of Fg fields per RHS (CFIE: 4 of 8; the rest stay zero).
template <class T>
__global__ void k_project(const T* __restrict__ w, const int* __restrict__ node_ptr,
                          const int* __restrict__ node_w, const int* __restrict__ node_x,
                          const cplx_t<T>* __restrict__ x, cplx_t<T>* grid, int nrhs, int F, int Fg, int N,
                          int nunk, int nx, int ny, int nz, int Mx, int My, int Mz) {
    using C = cplx_t<T>;
    int64_t NG = (int64_t)nx * ny * nz;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= NG * nrhs) return;
    int64_t g = t % NG;
    int b = (int)(t / NG);
    int gx = (int)(g % nx), gy = (int)((g / nx) % ny), gz = (int)(g / ((int64_t)nx * ny));
    C acc[8];
    for (int f = 0; f < 8; ++f) acc[f] = czero<T>();
    const C* xb = x + (int64_t)b * nunk;
    for (int e = node_ptr[g]; e < node_ptr[g + 1]; ++e) {
        const T* we = w + (int64_t)node_w[e] * 4;
        int xi = node_x[e];
        C xj = xb[xi];
        for (int f = 0; f < 4; ++f) rfma(acc[f], we[f], xj);
        if (F == 8) {
            C xm = xb[N + xi];
            for (int f = 0; f < 4; ++f) rfma(acc[4 + f], we[f], xm);
        }
    }
    int64_t SB = (int64_t)Mx * My * Mz;
    C* gb = grid + (int64_t)b * Fg * SB + ((int64_t)gz * My + gy) * Mx + gx;
    for (int f = 0; f < F; ++f) gb[f * SB] = acc[f];
}


// The kernel multiply at one spectral point for one RHS (g: that RHS's first field at the point,
// fields MT apart).  sp: the point's spectra, odd signs of the gradient components applied.
// EFIE (A, Phi): S1 J, S2 rho; PMCHWT: E rows S1 J + V x M, S2 rho_J; H rows S3 M - V x J,
// S4 rho_M; CFIE: (A, Phi) of J and the K part V x J (V = (1 - alpha) eta grad G).
template <class T>
__device__ inline void mix_rhs(cplx_t<T>* g, int64_t MT, const cplx_t<T>* sp, int F, int cfie) {
    using C = cplx_t<T>;
    if (cfie) {
        const C s1 = sp[0], s2 = sp[1], vx = sp[2], vy = sp[3], vz = sp[4];
        C jx = g[0], jy = g[MT], jz = g[2 * MT];
        g[0] = s1 * jx;
        g[MT] = s1 * jy;
        g[2 * MT] = s1 * jz;
        g[3 * MT] = s2 * g[3 * MT];
        g[4 * MT] = vy * jz - vz * jy;
        g[5 * MT] = vz * jx - vx * jz;
        g[6 * MT] = vx * jy - vy * jx;
        g[7 * MT] = czero<T>();
    } else if (F == 4) {
        g[0] = sp[0] * g[0];
        g[MT] = sp[0] * g[MT];
        g[2 * MT] = sp[0] * g[2 * MT];
        g[3 * MT] = sp[1] * g[3 * MT];
    } else {
        const C s1 = sp[0], s2 = sp[1], s3 = sp[2], s4 = sp[3], vx = sp[4], vy = sp[5], vz = sp[6];
        C jx = g[0], jy = g[MT], jz = g[2 * MT], rj = g[3 * MT];
        C mx = g[4 * MT], my = g[5 * MT], mz = g[6 * MT], rm = g[7 * MT];
        g[0] = s1 * jx + (vy * mz - vz * my);
        g[MT] = s1 * jy + (vz * mx - vx * mz);
        g[2 * MT] = s1 * jz + (vx * my - vy * mx);
        g[3 * MT] = s2 * rj;
        g[4 * MT] = s3 * mx - (vy * jz - vz * jy);
        g[5 * MT] = s3 * my - (vz * jx - vx * jz);
        g[6 * MT] = s3 * mz - (vx * jy - vy * jx);
        g[7 * MT] = s4 * rm;
    }
}

// the octant spectra of point t (index oi), with the odd components' signs applied
template <class T>
__device__ inline int load_point_spectra(const cplx_t<T>* spec, int64_t t, int F, int cfie, int Mx, int My, int Mz,
                                         cplx_t<T>* sp) {
    const int kx = (int)(t % Mx), ky = (int)((t / Mx) % My), kz = (int)(t / ((int64_t)Mx * My));
    const int ox = kx <= Mx / 2 ? kx : Mx - kx;
    const int oy = ky <= My / 2 ? ky : My - ky;
    const int oz = kz <= Mz / 2 ? kz : Mz - kz;
    const int64_t OT = (int64_t)(Mx / 2 + 1) * (My / 2 + 1) * (Mz / 2 + 1);
    const int64_t oi = ((int64_t)oz * (My / 2 + 1) + oy) * (Mx / 2 + 1) + ox;
    const int ns = cfie ? 5 : (F == 4 ? 2 : 7);
    const int g0 = cfie ? 2 : 4;                 // first gradient component
    for (int k = 0; k < ns; ++k) sp[k] = spec[k * OT + oi];
    if (cfie || F == 8) {
        if (kx > Mx / 2) sp[g0] = -sp[g0];
        if (ky > My / 2) sp[g0 + 1] = -sp[g0 + 1];
        if (kz > Mz / 2) sp[g0 + 2] = -sp[g0 + 2];
    }
    return ns;
}

// Per spectral point: out = mix(in) with the octant spectra, all RHS of the pass (one frequency)
template <class T>
__global__ void k_mix(cplx_t<T>* grid, const cplx_t<T>* __restrict__ spec, int nrhs, int F, int cfie, int Mx,
                      int My, int Mz) {
    using C = cplx_t<T>;
    const int64_t MT = (int64_t)Mx * My * Mz;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= MT) return;
    C sp[7];
    load_point_spectra<T>(spec, t, F, cfie, Mx, My, Mz, sp);
    const int Fg = cfie ? 8 : F;
    for (int b = 0; b < nrhs; ++b) mix_rhs<T>(grid + (int64_t)b * Fg * MT + t, MT, sp, F, cfie);
}

// The same with a frequency per RHS: RHS b takes the spectra of frequency fidx[b] (fstride
// complex apart); one thread per (point, RHS)
template <class T>
__global__ void k_mix_multi(cplx_t<T>* grid, const cplx_t<T>* __restrict__ spec, const int* __restrict__ fidx,
                            int64_t fstride, int nrhs, int F, int cfie, int Mx, int My, int Mz) {
    using C = cplx_t<T>;
    const int64_t MT = (int64_t)Mx * My * Mz;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= MT * nrhs) return;
    const int b = (int)(t / MT);
    const int64_t p = t % MT;
    C sp[7];
    load_point_spectra<T>(spec + fidx[b] * fstride, p, F, cfie, Mx, My, Mz, sp);
    const int Fg = cfie ? 8 : F;
    mix_rhs<T>(grid + (int64_t)b * Fg * MT + p, MT, sp, F, cfie);
}

// y[b][perm i] (and y[b][N + perm i]) = W-gather of the output fields + near correction.
// Output fields: EFIE (A, Phi) with Lambda; PMCHWT E rows (fields 0-3) and H rows
// (4-7) with Lambda; CFIE (A, Phi) with Lambda and K[J] (fields 4-6) with the
// moments of n x f (wg).  Near part: N^A, N^Phi, and nk = N^K (PMCHWT) or N^{K_g}
// (CFIE); ng = the Gram matrix (surface impedance, CFIE residue term) or null.
template <class T>
__global__ void k_interp_near(const T* __restrict__ w, const T* __restrict__ wg, const int* __restrict__ anc,
                              const int* __restrict__ perm, const int* __restrict__ row_ptr,
                              const int* __restrict__ cols, const T* __restrict__ na,
                              const T* __restrict__ np, const T* __restrict__ nk, const T* __restrict__ ng,
                              const int* __restrict__ lin_ptr, const int* __restrict__ lin_cols,
                              const T* __restrict__ la, const T* __restrict__ lp,
                              const cplx_t<T>* __restrict__ zn,
                              const cplx_t<T>* __restrict__ grid, const cplx_t<T>* __restrict__ x,
                              const cplx_t<T>* __restrict__ phi, const cplx_t<T>* __restrict__ phim,
                              const int* __restrict__ btri_t, const double* __restrict__ blen, int nt,
                              cplx_t<T>* y, NearCoefs nc0, const NearCoefs* __restrict__ ncs,
                              const int* __restrict__ fidx, int nrhs, int F, int two, int N, int nunk, int P,
                              int Mx, int My, int Mz) {
    using C = cplx_t<T>;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * nrhs) return;
    int i = (int)(t % N);
    int b = (int)(t / N);
    // near coefficients of this RHS's frequency (one frequency per pass unless ncs is given)
    const NearCoefs& nc = ncs ? ncs[fidx[b]] : nc0;
    int U = P * P * P;
    int64_t MT = (int64_t)Mx * My * Mz;
    const C* gb = grid + (int64_t)b * F * MT;
    const T* wi = w + (int64_t)i * U * 4;
    const T* wgi = wg ? wg + (int64_t)i * U * 3 : nullptr;
    C aE = czero<T>(), aH = czero<T>();
    int sx = anc[3 * i], sy = anc[3 * i + 1], sz = anc[3 * i + 2];
    // charge form (phi given): the rho field belongs to the triangles, not to the RWG weights
    const int nfe = phi ? 3 : 4;
    for (int u = 0; u < U; ++u) {
        int64_t node = ((int64_t)(sz + u / (P * P)) * My + (sy + (u / P) % P)) * Mx + (sx + u % P);
        for (int f = 0; f < nfe; ++f) rfma(aE, wi[4 * u + f], gb[f * MT + node]);
        if (wgi)
            for (int c = 0; c < 3; ++c) rfma(aE, wgi[3 * u + c], gb[(4 + c) * MT + node]);
        else if (two)
            for (int f = 0; f < nfe; ++f) rfma(aH, wi[4 * u + f], gb[(4 + f) * MT + node]);
    }
    const C* xb = x + (int64_t)b * nunk;
    if (lin_ptr) {
        // linear-term modification on the overlapping pairs
        const C lA = mk((T)nc.lin[0].x, (T)nc.lin[0].y), lP = mk((T)nc.lin[1].x, (T)nc.lin[1].y);
        const C mA = mk((T)nc.lin[2].x, (T)nc.lin[2].y), mP = mk((T)nc.lin[3].x, (T)nc.lin[3].y);
        C sA = czero<T>(), sP = czero<T>(), tA = czero<T>(), tP = czero<T>();
        for (int e = lin_ptr[i]; e < lin_ptr[i + 1]; ++e) {
            const int j = perm[lin_cols[e]];
            rfma(sA, la[e], xb[j]);
            rfma(sP, lp[e], xb[j]);
            if (two) {
                rfma(tA, la[e], xb[N + j]);
                rfma(tP, lp[e], xb[N + j]);
            }
        }
        aE = aE + lA * sA + lP * sP;
        if (two) aH = aH + mA * tA + mP * tP;
    }
    C cA = mk((T)nc.c[0].x, (T)nc.c[0].y), cP = mk((T)nc.c[1].x, (T)nc.c[1].y);
    if (!two) {
        C sA = czero<T>(), sP = czero<T>(), sK = czero<T>(), sG = czero<T>();
        if (zn) {
            // conventional-AIM mode: complex per-frequency entries, coefficient folded in (cA = 1, cP = 0)
            for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                C xj = xb[perm[cols[e]]];
                cfma(sA, zn[e], xj);
                if (ng) rfma(sG, ng[e], xj);
            }
        } else {
            for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                C xj = xb[perm[cols[e]]];
                rfma(sA, na[e], xj);
                rfma(sP, np[e], xj);
                if (nk) rfma(sK, nk[e], xj);
                if (ng) rfma(sG, ng[e], xj);
            }
        }
        if (phi) {
            // charge form: D^T phi in place of the RWG scalar potential's near part
            const C* pb = phi + (int64_t)b * nt;
            aE = aE + cA * sA + (T)blen[i] * (pb[btri_t[2 * i]] - pb[btri_t[2 * i + 1]]);
        } else {
            aE = aE + cA * sA + cP * sP;
        }
        if (nk) aE = aE + mk((T)nc.c[2].x, (T)nc.c[2].y) * sK;            // CFIE: K_g
        if (ng) {
            const int g = nk ? 3 : 2;                                      // Gram: c[3] (CFIE), c[2] (EFIE)
            aE = aE + mk((T)nc.c[g].x, (T)nc.c[g].y) * sG;
        }
        y[(int64_t)b * nunk + perm[i]] = aE;
    } else {
        C cK = mk((T)nc.c[2].x, (T)nc.c[2].y), dK = mk((T)nc.c[3].x, (T)nc.c[3].y);
        C dA = mk((T)nc.c[4].x, (T)nc.c[4].y), dP = mk((T)nc.c[5].x, (T)nc.c[5].y);
        C aJ = czero<T>(), pJ = czero<T>(), kJ = czero<T>(), aM = czero<T>(), pM = czero<T>(),
          kM = czero<T>();
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int j = perm[cols[e]];
            C xj = xb[j], xm = xb[N + j];
            rfma(aJ, na[e], xj);
            rfma(pJ, np[e], xj);
            rfma(kJ, nk[e], xj);
            rfma(aM, na[e], xm);
            rfma(pM, np[e], xm);
            rfma(kM, nk[e], xm);
        }
        if (phi) {
            // two-region charge form: D^T phi of J in the E rows, of M (phim) in the H rows
            const C* pb = phi + (int64_t)b * nt;
            const C* qb = phim + (int64_t)b * nt;
            const int tp = btri_t[2 * i], tm = btri_t[2 * i + 1];
            aE = aE + cA * aJ + (T)blen[i] * (pb[tp] - pb[tm]) + cK * kM;
            aH = aH + dK * kJ + dA * aM + (T)blen[i] * (qb[tp] - qb[tm]);
        } else {
            aE = aE + cA * aJ + cP * pJ + cK * kM;
            aH = aH + dK * kJ + dA * aM + dP * pM;
        }
        y[(int64_t)b * nunk + perm[i]] = aE;
        y[(int64_t)b * nunk + N + perm[i]] = aH;
    }
}

// Comparison path: the full (unpruned) 3-D transforms of the padded grids by cuFFT
// (Z2Z / C2C, unnormalised, the same sign convention as fft3d_padded; the 1/M of
// the round trip is folded into the kernel spectra).  Plans are cached per
// precision and batch size.
template <class T>
static void cufft_padded(aimx_ctx* ctx, cplx_t<T>* grid, int batch, int dir, cudaStream_t s) {
    constexpr int pi = sizeof(T) == 8 ? 1 : 0;
    cufftHandle& plan = reinterpret_cast<cufftHandle&>(ctx->cufft_plan[pi]);
    if (plan && ctx->cufft_batch[pi] != batch) {
        cufftDestroy(plan);
        plan = 0;
    }
    if (!plan) {
        int n[3] = {ctx->M[2], ctx->M[1], ctx->M[0]};
        if (cufftPlanMany(&plan, 3, n, nullptr, 1, 0, nullptr, 1, 0, pi ? CUFFT_Z2Z : CUFFT_C2C, batch) !=
            CUFFT_SUCCESS) {
            plan = 0;
            throw Error{AIMX_E_CUDA, "cufftPlanMany failed"};
        }
        ctx->cufft_batch[pi] = batch;
    }
    if (cufftSetStream(plan, s) != CUFFT_SUCCESS) throw Error{AIMX_E_CUDA, "cufftSetStream failed"};
    cufftResult r;
    if (pi)
        r = cufftExecZ2Z(plan, reinterpret_cast<cufftDoubleComplex*>(grid), reinterpret_cast<cufftDoubleComplex*>(grid),
                         dir);
    else
        r = cufftExecC2C(plan, reinterpret_cast<cufftComplex*>(grid), reinterpret_cast<cufftComplex*>(grid), dir);
    if (r != CUFFT_SUCCESS) throw Error{AIMX_E_CUDA, "cufftExec failed"};
}

void cufft_release(aimx_ctx* ctx) {
    for (int k = 0; k < 2; ++k)
        if (ctx->cufft_plan[k]) {
            cufftDestroy((cufftHandle)ctx->cufft_plan[k]);
            ctx->cufft_plan[k] = 0;
        }
}

// The generic product for one frequency (mf == nullptr) or for a batch whose RHS b takes
// frequency mf->d_fidx[b] (spectra, near coefficients and charge-form coefficient of that
// frequency from the tables in mf).
template <class T>
static void generic_product(aimx_ctx* ctx, double freq, const MultiFreq* mf, int nrhs, const T* x, T* y,
                            cudaStream_t s) {
    using C = cplx_t<T>;
    PrecData<T>& pd = prec<T>(ctx);
    NearCoefs nc;
    if (!mf) {
        ensure_spectra<T>(ctx, freq, s);
        Coefs cf = near_coefs(ctx, freq);
        for (int k = 0; k < 6; ++k) nc.c[k] = cf.near[k];
        for (int k = 0; k < 4; ++k) nc.lin[k] = cf.lin[k];
        ensure_aim_near(ctx, freq, s);
        if (ctx->aim) {
            nc.c[0] = make_double2(1.0, 0.0);
            nc.c[1] = make_double2(0.0, 0.0);
            for (auto& v : nc.lin) v = make_double2(0.0, 0.0);
        }
    } else {
        if (ctx->aim) throw Error{AIMX_E_STATE, "the conventional-AIM mode has no multi-frequency product"};
        for (auto& v : nc.c) v = make_double2(0.0, 0.0);
        for (auto& v : nc.lin) v = make_double2(0.0, 0.0);
    }
    const int F = ctx->F;
    const bool two = two_blocks(ctx->form);
    const int64_t MT = (int64_t)ctx->M[0] * ctx->M[1] * ctx->M[2];
    const size_t per_rhs = (size_t)F * MT;
    const size_t budget = (size_t)4 << 30;  // bytes of padded-grid work buffer
    int chunk = (int)std::max<size_t>(1, std::min<size_t>(nrhs, budget / (per_rhs * sizeof(C))));
    if (ctx->sched_pass > 0) chunk = std::min(chunk, ctx->sched_pass);
    if (pd.grid_elems < per_rhs * chunk) {
        if (pd.grid) dev_free(ctx, pd.grid);
        pd.grid = (T*)dev_alloc(ctx, sizeof(C) * per_rhs * chunk);
        pd.grid_elems = per_rhs * chunk;
    }
    C* grid = reinterpret_cast<C*>(pd.grid);
    const bool chg = ctx->charge != 0;
    C *cq = nullptr, *cphi = nullptr, *cqm = nullptr, *cphim = nullptr;
    if (chg && mf && two)
        throw Error{AIMX_E_STATE, "the two-region charge form has no multi-frequency product"};
    if (chg) {
        const size_t need = (two ? 4 : 2) * (size_t)ctx->nt * chunk;
        if (pd.cwork_elems < need) {
            if (pd.cwork) dev_free(ctx, pd.cwork);
            pd.cwork = (T*)dev_alloc(ctx, sizeof(C) * need);
            pd.cwork_elems = need;
        }
        cq = reinterpret_cast<C*>(pd.cwork);
        cphi = cq + (size_t)ctx->nt * chunk;
        if (two) {   // M charges and potentials (two-region form)
            cqm = cphi + (size_t)ctx->nt * chunk;
            cphim = cqm + (size_t)ctx->nt * chunk;
        }
    }
    const C* xc = reinterpret_cast<const C*>(x);
    C* yc = reinterpret_cast<C*>(y);
    const int act[3] = {ctx->n[0], ctx->n[1], ctx->n[2]};
    const int64_t NG = (int64_t)ctx->n[0] * ctx->n[1] * ctx->n[2];
    for (int b0 = 0; b0 < nrhs; b0 += chunk) {
        int nb = std::min(chunk, nrhs - b0);
        StageScope sc0(ctx, ST_G_PROJECT, s);
        // the register-line forward transform reads only the projected nodes; the others need zeros
        if (ctx->path == 2 || !fft3d_reads_active_only<T>(ctx->M, nb * F))
            AIMX_CUDA_TRY(cudaMemsetAsync(grid, 0, sizeof(C) * per_rhs * nb, s));
        int64_t tot = NG * nb;
        k_project<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
            pd.w, ctx->d_node_ptr, ctx->d_node_w, ctx->d_node_x, xc + (int64_t)b0 * ctx->nunk, grid, nb,
            two ? 8 : 4, F, ctx->N, ctx->nunk, ctx->n[0], ctx->n[1], ctx->n[2], ctx->M[0], ctx->M[1], ctx->M[2]);
        AIMX_CUDA_TRY(cudaGetLastError());
        if (chg) {
            charge_project<T>(ctx, xc + (int64_t)b0 * ctx->nunk, nb, cq, grid, F, 3, s);
            if (two) charge_project<T>(ctx, xc + (int64_t)b0 * ctx->nunk + ctx->N, nb, cqm, grid, F, 7, s);
        }
        if (ctx->path == 2)
            cufft_padded<T>(ctx, grid, nb * F, CUFFT_FORWARD, s);
        else
            fft3d_padded<T>(reinterpret_cast<T*>(grid), nb * F, ctx->M, act, false, s);
        if (mf)
            k_mix_multi<T><<<(unsigned)((MT * nb + 255) / 256), 256, 0, s>>>(
                grid, reinterpret_cast<const C*>(mf->spec), mf->d_fidx + b0, mf->fstride, nb, F,
                ctx->form == AIMX_CFIE ? 1 : 0, ctx->M[0], ctx->M[1], ctx->M[2]);
        else
            k_mix<T><<<(unsigned)((MT + 255) / 256), 256, 0, s>>>(
                grid, reinterpret_cast<const C*>(pd.spec), nb, F, ctx->form == AIMX_CFIE ? 1 : 0, ctx->M[0],
                ctx->M[1], ctx->M[2]);
        AIMX_CUDA_TRY(cudaGetLastError());
        if (ctx->path == 2)
            cufft_padded<T>(ctx, grid, nb * F, CUFFT_INVERSE, s);
        else
            fft3d_padded<T>(reinterpret_cast<T*>(grid), nb * F, ctx->M, act, true, s);
        if (chg) {
            charge_potential<T>(ctx, grid, F, 3, nb, cq, cphi, nc.c[1], s, mf ? mf->d_cphi : nullptr,
                                mf ? mf->d_fidx + b0 : nullptr);
            // two-region: the M rows' potentials, with the M block's scalar-potential coefficient
            if (two) charge_potential<T>(ctx, grid, F, 7, nb, cqm, cphim, nc.c[5], s, nullptr, nullptr);
        }
        int64_t tn = (int64_t)ctx->N * nb;
        k_interp_near<T><<<(unsigned)((tn + 127) / 128), 128, 0, s>>>(
            pd.w, ctx->form == AIMX_CFIE ? pd.wg : nullptr, ctx->d_anc, ctx->d_perm, ctx->d_row_ptr, ctx->d_cols,
            pd.na, pd.np, ctx->form == AIMX_EFIE ? nullptr : pd.nk, two ? nullptr : pd.ng,
            ctx->linterm && !ctx->aim ? ctx->d_lin_ptr : nullptr, ctx->d_lin_cols, pd.la, pd.lp,
            ctx->aim ? reinterpret_cast<const C*>(pd.zn) : nullptr, grid,
            xc + (int64_t)b0 * ctx->nunk, chg ? cphi : nullptr, chg ? cphim : nullptr, ctx->d_btri_t, ctx->d_blen,
            ctx->nt,
            yc + (int64_t)b0 * ctx->nunk, nc, mf ? mf->d_ncs : nullptr, mf ? mf->d_fidx + b0 : nullptr, nb, F,
            two ? 1 : 0, ctx->N, ctx->nunk, ctx->P, ctx->M[0], ctx->M[1], ctx->M[2]);
        AIMX_CUDA_TRY(cudaGetLastError());
    }
}

template <class T>
void matvec_generic(aimx_ctx* ctx, double freq, int nrhs, const T* x, T* y, cudaStream_t s) {
    generic_product<T>(ctx, freq, nullptr, nrhs, x, y, s);
}

template <class T>
void matvec_generic_multi(aimx_ctx* ctx, const MultiFreq& mf, int nrhs, const T* x, T* y, cudaStream_t s) {
    generic_product<T>(ctx, 0.0, &mf, nrhs, x, y, s);
}

template void matvec_generic<float>(aimx_ctx*, double, int, const float*, float*, cudaStream_t);
template void matvec_generic<double>(aimx_ctx*, double, int, const double*, double*, cudaStream_t);
template void matvec_generic_multi<float>(aimx_ctx*, const MultiFreq&, int, const float*, float*, cudaStream_t);
template void matvec_generic_multi<double>(aimx_ctx*, const MultiFreq&, int, const double*, double*, cudaStream_t);

}  // namespace aimx
