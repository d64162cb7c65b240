// Charge-form scalar potential of the EFIE (the discretisation of the augmented EFIE, which the
// paper uses for its on-chip examples, Sec. V-C to V-E), accelerated by AIMx like every other
// operator (Eq. LAIMx).
//
// The RWG scalar-potential operator L^Phi_mn = int int div f_m div' f_n G is written through the
// charges the currents carry.  With the charge of triangle t a pulse of density q_t / A_t and the
// incidence D_tn = int_{T_t} div f_n dS = +-l_n (T+ / T-),
//
//     L^Phi = D^T Pt D,     Pt_ij = (A_i A_j)^-1 int_{T_i} int_{T_j} G dS' dS,
//     Pt    = (Pt_s,NR - Pt_s,P) + Lp^T H(k) Lp,
//
// with pulse projection weights Lp[u, t] = A_t^-1 int_{T_t} l_u dS on each triangle's own
// stencil (moment matching, Sec. II-B), triangle near pairs by anchor distance, the static
// kernel 1/(4 pi R) for the near part (closed-form inner integral, the 5 x 5 collapsed outer
// rule) and its grid samples for the precorrection.  A divergence-free current (D x = 0) then
// gets exactly zero scalar potential, whatever the accuracy of the grid part.
//
// Setup (once, on the first aimx_set_charge_form): host integer steps (anchors, internal
// triangle order, near pattern, node-major lists, incidence), FP64 device kernels for the
// weights, the static integrals and the precorrection.  Product steps: q = D x; the rho field of
// the grid projected from q; after the convolution, phi = Lp^T (rho field) + c_Phi N_Pt q per
// triangle; y += D^T phi in the final kernel of each path.

#include <algorithm>
#include <cmath>
#include <numeric>

#include "aimx_internal.h"
#include "cplx.cuh"
#include "geom.cuh"

namespace aimx {

// ------------------------------------------------------------------ setup kernels

// Lp[t, u] = sum_q w_q l_u(r_q) over triangle t (the normalised rule already carries 1 / A_t),
// one thread per (internal triangle, stencil node).
__global__ void k_pulse_weights(const double* __restrict__ xyz, const int* __restrict__ tri,
                                const int* __restrict__ tperm, const int* __restrict__ tanc,
                                const double* __restrict__ rule, int nq, int nt, int P, double ox, double oy,
                                double oz, double hx, double hy, double hz, double* lp) {
    const int U = P * P * P;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt * U) return;
    const int ti = t / U, u = t % U;
    const int tr = tperm[ti];
    const int sel[3] = {u % P, (u / P) % P, u / (P * P)};
    const V3 a = load3(xyz + 3 * tri[3 * tr]), b = load3(xyz + 3 * tri[3 * tr + 1]),
             c = load3(xyz + 3 * tri[3 * tr + 2]);
    double acc = 0.0;
    for (int q = 0; q < nq; ++q) {
        const V3 r = rule[4 * q] * a + rule[4 * q + 1] * b + rule[4 * q + 2] * c;
        const double xi[3] = {(r.x - ox) / hx - tanc[3 * ti], (r.y - oy) / hy - tanc[3 * ti + 1],
                              (r.z - oz) / hz - tanc[3 * ti + 2]};
        double ell = 1.0;
        for (int ax = 0; ax < 3; ++ax)
            for (int m = 0; m < P; ++m)
                if (m != sel[ax]) ell *= (xi[ax] - m) / double(sel[ax] - m);
        acc += rule[4 * q + 3] * ell;
    }
    lp[t] = acc;
}

// Pt_s(i, j) = (A_i A_j)^-1 int_{T_i} int_{T_j} 1/(4 pi R): closed-form inner integral over T_j at
// the outer rule's points of T_i; then minus the precorrection sum_{u,v} Lp[i,u] H_s[d] Lp[j,v]
// with the static grid kernel between the two stencils.  FP64 and FP32 copies.
__global__ void k_pulse_near(const double* __restrict__ xyz, const int* __restrict__ tri,
                             const double* __restrict__ area, const int* __restrict__ tperm,
                             const int* __restrict__ tanc, const int* __restrict__ row_of,
                             const int* __restrict__ cols, int64_t nnz, const double* __restrict__ rule, int nq,
                             const double* __restrict__ lp, int P, int span, const double* __restrict__ hs_tab,
                             double* npt64, float* npt32) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const int i = row_of[e], j = cols[e];
    const int ti = tperm[i], tj = tperm[j];
    TriFrame T;
    make_frame(T, load3(xyz + 3 * tri[3 * tj]), load3(xyz + 3 * tri[3 * tj + 1]), load3(xyz + 3 * tri[3 * tj + 2]));
    const V3 a = load3(xyz + 3 * tri[3 * ti]), b = load3(xyz + 3 * tri[3 * ti + 1]), c = load3(xyz + 3 * tri[3 * ti + 2]);
    double s = 0.0;
    for (int q = 0; q < nq; ++q) {
        const V3 r = rule[4 * q] * a + rule[4 * q + 1] * b + rule[4 * q + 2] * c;
        double I1;
        V3 J, G, rho;
        tri_potentials(T, r, I1, J, G, rho);
        s += rule[4 * q + 3] * I1;
    }
    const double direct = s / (4.0 * kPi * area[tj]);
    const int U = P * P * P, D = 2 * span + 1;
    const int dx0 = tanc[3 * i] - tanc[3 * j], dy0 = tanc[3 * i + 1] - tanc[3 * j + 1],
              dz0 = tanc[3 * i + 2] - tanc[3 * j + 2];
    const double* li = lp + (size_t)i * U;
    const double* lj = lp + (size_t)j * U;
    double pc = 0.0;
    for (int u = 0; u < U; ++u) {
        const int ux = u % P, uy = (u / P) % P, uz = u / (P * P);
        double row = 0.0;
        for (int v = 0; v < U; ++v) {
            const int vx = v % P, vy = (v / P) % P, vz = v / (P * P);
            const int ix = dx0 + ux - vx + span, iy = dy0 + uy - vy + span, iz = dz0 + uz - vz + span;
            row += hs_tab[(iz * D + iy) * D + ix] * lj[v];
        }
        pc += li[u] * row;
    }
    const double v = direct - pc;
    npt64[e] = v;
    npt32[e] = (float)v;
}

__global__ void k_lp_soa(const double* __restrict__ lp, float* __restrict__ lp32, float* __restrict__ soa, int nt,
                         int U) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nt * U) return;
    const int ti = (int)(t / U), u = (int)(t % U);
    lp32[t] = (float)lp[t];
    soa[(int64_t)u * nt + ti] = (float)lp[t];
}

// ------------------------------------------------------------------ host setup

template <class T>
static T* upload_vec(aimx_ctx* ctx, const std::vector<T>& v) {
    T* p = (T*)dev_alloc(ctx, std::max<size_t>(1, v.size()) * sizeof(T));
    if (!v.empty()) AIMX_CUDA_TRY(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}

void build_charge(aimx_ctx* ctx) {
    if (ctx->charge_built) return;
    if (ctx->form != AIMX_EFIE && ctx->form != AIMX_PMCHWT)
        throw Error{AIMX_E_STATE, "the charge form is available for the EFIE and the PMCHWT"};
    const int nt = ctx->nt, N = ctx->N, P = ctx->P, U = ctx->U, order = ctx->order;
    const int nx = ctx->n[0], ny = ctx->n[1], nz = ctx->n[2];

    // anchors from the centroids ((v0 + v1) + v2) / 3, exactly as the basis anchors
    std::vector<int> a0(3 * (size_t)nt);
    for (int t = 0; t < nt; ++t)
        for (int a = 0; a < 3; ++a) {
            const double tt = (ctx->h_cen[3 * t + a] - ctx->origin[a]) / ctx->h[a] - (order - 1) / 2.0;
            const double f = std::floor(tt);
            if (!(f >= 0.0) || f + order > ctx->n[a] - 1)
                throw Error{AIMX_E_GRID, "a triangle stencil falls outside the grid"};
            a0[3 * t + a] = (int)f;
        }
    // internal triangle order: by anchor (z, y, x), ties by caller index
    auto key = [&](int t) { return ((int64_t)a0[3 * t + 2] * ny + a0[3 * t + 1]) * nx + a0[3 * t]; };
    std::vector<int> tperm(nt), tiperm(nt);
    std::iota(tperm.begin(), tperm.end(), 0);
    std::stable_sort(tperm.begin(), tperm.end(), [&](int x, int y) { return key(x) < key(y); });
    for (int i = 0; i < nt; ++i) tiperm[tperm[i]] = i;
    std::vector<int> tanc(3 * (size_t)nt);
    std::vector<int64_t> keys(nt);
    for (int i = 0; i < nt; ++i) {
        for (int a = 0; a < 3; ++a) tanc[3 * i + a] = a0[3 * tperm[i] + a];
        keys[i] = key(tperm[i]);
    }
    // near pairs: anchors within Chebyshev distance R; columns ascending
    const int R = ctx->radius;
    std::vector<int> trow_ptr(nt + 1, 0), tcols;
    tcols.reserve((size_t)nt * 64);
    for (int i = 0; i < nt; ++i) {
        const int* s = &tanc[3 * i];
        const size_t start = tcols.size();
        for (int dz = -R; dz <= R; ++dz) {
            const int z = s[2] + dz;
            if (z < 0 || z >= nz) continue;
            for (int dy = -R; dy <= R; ++dy) {
                const int y = s[1] + dy;
                if (y < 0 || y >= ny) continue;
                const int x0 = std::max(0, s[0] - R), x1 = std::min(nx - 1, s[0] + R);
                const int64_t k0 = ((int64_t)z * ny + y) * nx + x0, k1 = ((int64_t)z * ny + y) * nx + x1;
                auto b = std::lower_bound(keys.begin(), keys.end(), k0);
                auto e = std::upper_bound(keys.begin(), keys.end(), k1);
                for (auto it = b; it != e; ++it) tcols.push_back((int)(it - keys.begin()));
            }
        }
        std::sort(tcols.begin() + start, tcols.end());
        if (tcols.size() > (size_t)INT32_MAX) throw Error{AIMX_E_NOMEM, "triangle near list too large"};
        trow_ptr[i + 1] = (int)tcols.size();
    }
    const int64_t tnnz = (int64_t)tcols.size();
    std::vector<int> row_of(tcols.size());
    for (int i = 0; i < nt; ++i)
        for (int e = trow_ptr[i]; e < trow_ptr[i + 1]; ++e) row_of[e] = i;
    // node-major triangle lists
    const int64_t NG = (int64_t)nx * ny * nz;
    std::vector<int> node_ptr(NG + 1, 0);
    auto node_of = [&](int i, int u) {
        return ((int64_t)(tanc[3 * i + 2] + u / (P * P)) * ny + tanc[3 * i + 1] + (u / P) % P) * nx + tanc[3 * i] +
               u % P;
    };
    for (int i = 0; i < nt; ++i)
        for (int u = 0; u < U; ++u) node_ptr[node_of(i, u) + 1]++;
    for (int64_t g = 0; g < NG; ++g) node_ptr[g + 1] += node_ptr[g];
    std::vector<int> fill(node_ptr.begin(), node_ptr.end() - 1), node_w((size_t)nt * U);
    for (int i = 0; i < nt; ++i)
        for (int u = 0; u < U; ++u) node_w[fill[node_of(i, u)]++] = i * U + u;
    // triangles touching each z plane (contiguous in internal order)
    std::vector<int> plo(nz), phi(nz);
    int mpt = 0;
    for (int z = 0, lo = 0; z < nz; ++z) {
        while (lo < nt && tanc[3 * lo + 2] < z - order) ++lo;
        int hi = lo;
        while (hi < nt && tanc[3 * hi + 2] <= z) ++hi;
        plo[z] = lo;
        phi[z] = hi;
        mpt = std::max(mpt, hi - lo);
    }
    // incidence: the (at most three) RWG edges of each triangle with +l (T+) or -l (T-), and the
    // two triangles of each basis
    std::vector<int> tinc(3 * (size_t)nt, -1), btri_t(2 * (size_t)N);
    std::vector<double> tl(3 * (size_t)nt, 0.0);
    std::vector<int> deg(nt, 0);
    for (int i = 0; i < N; ++i) {
        const int o = ctx->perm[i];
        const double* A = &ctx->h_xyz[3 * ctx->h_ea[o]];
        const double* B = &ctx->h_xyz[3 * ctx->h_eb[o]];
        const double d[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        const double len = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const int tp = tiperm[ctx->h_tp[o]], tm = tiperm[ctx->h_tm[o]];
        btri_t[2 * i] = tp;
        btri_t[2 * i + 1] = tm;
        for (int side = 0; side < 2; ++side) {
            const int t = side ? tm : tp;
            if (deg[t] >= 3) throw Error{AIMX_E_MESH, "triangle with more than three RWG edges"};
            tinc[3 * t + deg[t]] = i;
            tl[3 * t + deg[t]] = side ? -len : len;
            ++deg[t];
        }
    }

    // device data
    ctx->d_tanc = upload_vec(ctx, tanc);
    ctx->d_trow_ptr = upload_vec(ctx, trow_ptr);
    ctx->d_tcols = upload_vec(ctx, tcols);
    ctx->d_tnode_ptr = upload_vec(ctx, node_ptr);
    ctx->d_tnode_w = upload_vec(ctx, node_w);
    ctx->d_tinc = upload_vec(ctx, tinc);
    ctx->d_btri_t = upload_vec(ctx, btri_t);
    std::vector<int> planes(plo);
    planes.insert(planes.end(), phi.begin(), phi.end());
    ctx->d_tplane = upload_vec(ctx, planes);
    ctx->f64.tl = upload_vec(ctx, tl);
    std::vector<float> tl32(tl.begin(), tl.end());
    ctx->f32.tl = upload_vec(ctx, tl32);
    int* d_tperm = upload_vec(ctx, tperm);
    int* d_row_of = upload_vec(ctx, row_of);
    // rules: projection (exact for the stencil polynomials) and the 5 x 5 outer rule of the near part
    std::vector<double> qp;
    triangle_rule((3 * order + 4) / 2, qp);
    double* d_qp = upload_vec(ctx, qp);
    const int span = R + order, D = 2 * span + 1;
    std::vector<double> hs((size_t)D * D * D);
    for (int iz = 0; iz < D; ++iz)
        for (int iy = 0; iy < D; ++iy)
            for (int ix = 0; ix < D; ++ix) {
                const double rx = (ix - span) * ctx->h[0], ry = (iy - span) * ctx->h[1], rz = (iz - span) * ctx->h[2];
                const double r = std::sqrt(rx * rx + ry * ry + rz * rz);
                hs[((size_t)iz * D + iy) * D + ix] = (ix == span && iy == span && iz == span) ? 0.0 : 1.0 / (4.0 * kPi * r);
            }
    double* d_hs = upload_vec(ctx, hs);
    ctx->f64.plw = (double*)dev_alloc(ctx, sizeof(double) * (size_t)nt * U);
    ctx->f32.plw = (float*)dev_alloc(ctx, sizeof(float) * (size_t)nt * U);
    ctx->d_lp_soa = (float*)dev_alloc(ctx, sizeof(float) * (size_t)nt * U);
    ctx->f64.npt = (double*)dev_alloc(ctx, sizeof(double) * std::max<int64_t>(1, tnnz));
    ctx->f32.npt = (float*)dev_alloc(ctx, sizeof(float) * std::max<int64_t>(1, tnnz));
    cudaError_t err = cudaSuccess;
    {
        const int64_t tot = (int64_t)nt * U;
        k_pulse_weights<<<(unsigned)((tot + 127) / 128), 128>>>(ctx->d_xyz, ctx->d_tri, d_tperm, ctx->d_tanc, d_qp,
                                                                (int)qp.size() / 4, nt, P, ctx->origin[0],
                                                                ctx->origin[1], ctx->origin[2], ctx->h[0], ctx->h[1],
                                                                ctx->h[2], ctx->f64.plw);
        k_lp_soa<<<(unsigned)((tot + 255) / 256), 256>>>(ctx->f64.plw, ctx->f32.plw, ctx->d_lp_soa, nt, U);
        if (tnnz > 0)
            k_pulse_near<<<(unsigned)((tnnz + 127) / 128), 128>>>(ctx->d_xyz, ctx->d_tri, ctx->d_area, d_tperm,
                                                                  ctx->d_tanc, d_row_of, ctx->d_tcols, tnnz, ctx->d_q5,
                                                                  25, ctx->f64.plw, P, span, d_hs, ctx->f64.npt,
                                                                  ctx->f32.npt);
        err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaDeviceSynchronize();
    }
    dev_free(ctx, d_tperm);
    dev_free(ctx, d_row_of);
    dev_free(ctx, d_qp);
    dev_free(ctx, d_hs);
    AIMX_CUDA_TRY(err);
    ctx->tperm = tperm;
    ctx->tanc = tanc;
    ctx->trow_ptr = trow_ptr;
    ctx->tcols = tcols;
    ctx->tplane_lo = plo;
    ctx->tplane_hi = phi;
    ctx->max_plane_tris = mpt;
    ctx->tnnz = tnnz;
    ctx->charge_built = 1;
}

// ------------------------------------------------------------------ generic path

// q[b][t] = (D x)_t = sum over the triangle's edges of +-l_n x_n (caller-order x)
template <class T>
__global__ void k_charge_q(const T* __restrict__ tl, const int* __restrict__ tinc, const int* __restrict__ perm,
                           const cplx_t<T>* __restrict__ x, int nb, int nunk, int nt, cplx_t<T>* q) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nt * nb) return;
    const int ti = (int)(t % nt), b = (int)(t / nt);
    cplx_t<T> acc = czero<T>();
    for (int k = 0; k < 3; ++k) {
        const int i = tinc[3 * ti + k];
        if (i >= 0) rfma(acc, tl[3 * ti + k], x[(int64_t)b * nunk + perm[i]]);
    }
    q[t] = acc;
}

// rho field of the padded grid from the triangle charges: node-major gather (no atomics)
template <class T>
__global__ void k_project_rho(const T* __restrict__ lp, const int* __restrict__ node_ptr,
                              const int* __restrict__ node_w, const cplx_t<T>* __restrict__ q, cplx_t<T>* grid,
                              int nb, int Fg, int rho_field, int U, int nt, int nx, int ny, int nz, int Mx, int My,
                              int Mz) {
    const int64_t NG = (int64_t)nx * ny * nz;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= NG * nb) return;
    const int64_t g = t % NG;
    const int b = (int)(t / NG);
    const int gx = (int)(g % nx), gy = (int)((g / nx) % ny), gz = (int)(g / ((int64_t)nx * ny));
    cplx_t<T> acc = czero<T>();
    for (int e = node_ptr[g]; e < node_ptr[g + 1]; ++e) {
        const int w = node_w[e];
        rfma(acc, lp[w], q[(int64_t)b * nt + w / U]);
    }
    const int64_t SB = (int64_t)Mx * My * Mz;
    grid[((int64_t)b * Fg + rho_field) * SB + ((int64_t)gz * My + gy) * Mx + gx] = acc;
}

// phi[b][t] = sum_u Lp[t, u] rho_out[s_t + u] + cP sum_j N_Pt(t, j) q[b][j]
template <class T>
__global__ void k_potential(const T* __restrict__ lp, const int* __restrict__ tanc, const int* __restrict__ row_ptr,
                            const int* __restrict__ cols, const T* __restrict__ npt,
                            const cplx_t<T>* __restrict__ grid, int Fg, int rho_field, const cplx_t<T>* __restrict__ q,
                            cplx_t<T>* phi, double2 cP0, const double2* __restrict__ cps, const int* __restrict__ fidx,
                            int nb, int nt, int P, int Mx, int My, int Mz) {
    using C = cplx_t<T>;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nt * nb) return;
    const int ti = (int)(t % nt), b = (int)(t / nt);
    const double2 cP = cps ? cps[fidx[b]] : cP0;   // per-RHS frequency in batched products
    const int U = P * P * P;
    const int64_t SB = (int64_t)Mx * My * Mz;
    const C* gr = grid + ((int64_t)b * Fg + rho_field) * SB;
    const int sx = tanc[3 * ti], sy = tanc[3 * ti + 1], sz = tanc[3 * ti + 2];
    C s = czero<T>();
    for (int u = 0; u < U; ++u) {
        const int64_t node = ((int64_t)(sz + u / (P * P)) * My + (sy + (u / P) % P)) * Mx + (sx + u % P);
        rfma(s, lp[(int64_t)ti * U + u], gr[node]);
    }
    C nr = czero<T>();
    const C* qb = q + (int64_t)b * nt;
    for (int e = row_ptr[ti]; e < row_ptr[ti + 1]; ++e) rfma(nr, npt[e], qb[cols[e]]);
    phi[t] = s + mk((T)cP.x, (T)cP.y) * nr;
}

template <class T>
void charge_project(aimx_ctx* ctx, const cplx_t<T>* x, int nb, cplx_t<T>* q, cplx_t<T>* grid, int Fg, int rho_field,
                    cudaStream_t s) {
    PrecData<T>& pd = prec<T>(ctx);
    const int nt = ctx->nt;
    const int64_t tq = (int64_t)nt * nb;
    k_charge_q<T><<<(unsigned)((tq + 255) / 256), 256, 0, s>>>(pd.tl, ctx->d_tinc, ctx->d_perm, x, nb, ctx->nunk, nt,
                                                                q);
    const int64_t NG = (int64_t)ctx->n[0] * ctx->n[1] * ctx->n[2];
    k_project_rho<T><<<(unsigned)((NG * nb + 255) / 256), 256, 0, s>>>(
        pd.plw, ctx->d_tnode_ptr, ctx->d_tnode_w, q, grid, nb, Fg, rho_field, ctx->U, nt, ctx->n[0], ctx->n[1],
        ctx->n[2], ctx->M[0], ctx->M[1], ctx->M[2]);
    AIMX_CUDA_TRY(cudaGetLastError());
}

template <class T>
void charge_potential(aimx_ctx* ctx, const cplx_t<T>* grid, int Fg, int rho_field, int nb, const cplx_t<T>* q,
                      cplx_t<T>* phi, double2 cP, cudaStream_t s, const double2* cps, const int* fidx) {
    PrecData<T>& pd = prec<T>(ctx);
    const int nt = ctx->nt;
    const int64_t tq = (int64_t)nt * nb;
    k_potential<T><<<(unsigned)((tq + 127) / 128), 128, 0, s>>>(pd.plw, ctx->d_tanc, ctx->d_trow_ptr, ctx->d_tcols,
                                                                 pd.npt, grid, Fg, rho_field, q, phi, cP, cps, fidx, nb, nt,
                                                                 ctx->P, ctx->M[0], ctx->M[1], ctx->M[2]);
    AIMX_CUDA_TRY(cudaGetLastError());
}

template void charge_project<float>(aimx_ctx*, const float2*, int, float2*, float2*, int, int, cudaStream_t);
template void charge_project<double>(aimx_ctx*, const double2*, int, double2*, double2*, int, int, cudaStream_t);
template void charge_potential<float>(aimx_ctx*, const float2*, int, int, int, const float2*, float2*, double2,
                                      cudaStream_t, const double2*, const int*);
template void charge_potential<double>(aimx_ctx*, const double2*, int, int, int, const double2*, double2*, double2,
                                       cudaStream_t, const double2*, const int*);

// ------------------------------------------------------------------ plane-fused path

// qT[t][b] = sum over the triangle's edges of +-l_n xT[n][b] (internal order, RHS fastest)
__global__ void k_charge_qT(const float* __restrict__ tl, const int* __restrict__ tinc,
                            const float2* __restrict__ xT, int nt, int B, float2* qT) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nt * B) return;
    const int ti = (int)(t / B), b = (int)(t % B);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int i = tinc[3 * ti + k];
        if (i >= 0) rfma(acc, tl[3 * ti + k], xT[(int64_t)i * B + b]);
    }
    qT[t] = acc;
}

// phiT[t][b] = sum over the triangle's stencil planes of the interpolation partials
// + cP sum_j N_Pt(t, j) qT[j][b]
__global__ void k_phi_fused(const float2* __restrict__ tpart, const int* __restrict__ row_ptr,
                            const int* __restrict__ cols, const float* __restrict__ npt,
                            const float2* __restrict__ qT, float2 cP, int nt, int B, int P, float2* phiT) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nt * B) return;
    const int ti = (int)(t / B), b = (int)(t % B);
    float2 s = make_float2(0.f, 0.f);
    for (int sl = 0; sl < P; ++sl) s = s + tpart[((int64_t)b * P + sl) * nt + ti];
    float2 nr = make_float2(0.f, 0.f);
    for (int e = row_ptr[ti]; e < row_ptr[ti + 1]; ++e) rfma(nr, __ldg(npt + e), __ldg(qT + (int64_t)cols[e] * B + b));
    phiT[t] = s + cP * nr;
}

// Two-region forms (F = 8) keep the M charges, potentials and partials in a second block after
// those of J: qT and phiT [2][nt][B], tpart [2][B][P][nt].
void ensure_charge_buffers(aimx_ctx* ctx, int B) {
    if (ctx->charge_cap >= B) return;
    if (ctx->d_qT) dev_free(ctx, ctx->d_qT);
    if (ctx->d_phiT) dev_free(ctx, ctx->d_phiT);
    if (ctx->d_tpart) dev_free(ctx, ctx->d_tpart);
    ctx->d_qT = ctx->d_phiT = ctx->d_tpart = nullptr;
    ctx->charge_cap = 0;
    const size_t nt = (size_t)ctx->nt * (ctx->F / 4);
    ctx->d_qT = (float*)dev_alloc(ctx, sizeof(float2) * nt * B);
    ctx->d_phiT = (float*)dev_alloc(ctx, sizeof(float2) * nt * B);
    ctx->d_tpart = (float*)dev_alloc(ctx, sizeof(float2) * nt * B * ctx->P);
    ctx->charge_cap = B;
}

void charge_fused_q(aimx_ctx* ctx, const float2* xT, int B, cudaStream_t s) {
    const int64_t tot = (int64_t)ctx->nt * B;
    for (int g = 0; g < ctx->F / 4; ++g)   // J; two-region: M (rows N.. of xT)
        k_charge_qT<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
            ctx->f32.tl, ctx->d_tinc, xT + (int64_t)g * ctx->N * B, ctx->nt, B,
            reinterpret_cast<float2*>(ctx->d_qT) + g * tot);
    AIMX_CUDA_TRY(cudaGetLastError());
}

void charge_fused_phi(aimx_ctx* ctx, int B, float2 cP, float2 cP2, cudaStream_t s) {
    const int64_t tot = (int64_t)ctx->nt * B;
    for (int g = 0; g < ctx->F / 4; ++g)
        k_phi_fused<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
            reinterpret_cast<const float2*>(ctx->d_tpart) + g * tot * ctx->P, ctx->d_trow_ptr, ctx->d_tcols,
            ctx->f32.npt, reinterpret_cast<const float2*>(ctx->d_qT) + g * tot, g ? cP2 : cP, ctx->nt, B, ctx->P,
            reinterpret_cast<float2*>(ctx->d_phiT) + g * tot);
    AIMX_CUDA_TRY(cudaGetLastError());
}

}  // namespace aimx
