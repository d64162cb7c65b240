// Batched frequency sweep (the paper's Discussion: a sweep costs T = T_s + N T_d, one static
// setup and N frequency-dependent solves): all nf x nrhs systems A(k_f) x = b are solved together.
//
// * One product carries a frequency index per batch member: the member reads that frequency's
//   kernel spectra, near coefficients and preconditioner (matvec_generic_multi).
// * GMRES(m) with right preconditioning runs in lockstep over the systems held in S slots.  The
//   Arnoldi steps, the classical Gram-Schmidt passes (always two), the Givens rotations, the
//   convergence test and the back substitution are device kernels, so a cycle of m steps has no
//   host round trip; it is captured once into a CUDA graph and replayed for every cycle with the
//   same slot count.
// * Between cycles the host reads one residual per slot (one synchronisation per cycle), retires
//   converged systems, moves pending ones into free slots and halves the slot count (a new
//   graph) when fewer than three quarters of the slots are busy.
// * Every cycle starts from the true residual b - A x of its systems (iterative refinement, as in
//   aimx_solve); with FP32 inner products and tol >= 1e-5 those residuals use the FP32 product and
//   convergence is confirmed with the FP64 product before a system is reported.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "aimx_internal.h"
#include "cplx.cuh"
#include "krylov.cuh"

namespace aimx {

__device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ inline double cabsd(double2 a) { return hypot(a.x, a.y); }
__device__ inline double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// Cycle start per slot: g = (|r|, 0, ...), the inner target |r - A d| <= eta |r| (a fraction of
// what the outer tolerance needs, floored at what the inner precision delivers), the done flag
// (nothing to do for a zero residual or an empty slot) and 1 / |r|.
__global__ void k_cycle_init(int S, int m, const double* __restrict__ rnorm, const double* __restrict__ bnorm,
                             double tol, double eta_floor, double2* g, double* thresh, int* done, double* scale,
                             int* kused) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const double r = rnorm[s];
    for (int i = 0; i <= m; ++i) g[(int64_t)s * (m + 1) + i] = make_double2(0.0, 0.0);
    g[(int64_t)s * (m + 1)] = make_double2(r, 0.0);
    const double eta = fmax(0.3 * tol * bnorm[s] / fmax(r, 1e-300), eta_floor);
    thresh[s] = eta * r;
    const int d = !(r > 0.0) || !isfinite(r);
    done[s] = d;
    scale[s] = d ? 0.0 : 1.0 / r;
    kused[s] = 0;
}

// Column j of the Hessenberg matrix of every slot from the two Gram-Schmidt passes (h1 + h2)
// and |w|; the previous rotations are applied, a new one zeroes the subdiagonal, the residual
// estimate |g[j+1]| is compared with the slot's target.  One thread per slot; the slot's
// Hessenberg columns are H[s][j][0..m] (column-major), rotations cs, sn [s][m].
__global__ void k_givens(int S, int j, int m, const double2* __restrict__ h1, const double2* __restrict__ h2,
                         const double* __restrict__ hn, double2* H, double2* cs, double2* sn, double2* g,
                         const double* __restrict__ thresh, const double* __restrict__ rnorm, int* done,
                         double* scale, int* kused) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    if (done[s]) {
        scale[s] = 0.0;
        return;
    }
    double2* col = H + ((int64_t)s * m + j) * (m + 1);
    const double2* a1 = h1 + (int64_t)s * (m + 1);
    const double2* a2 = h2 + (int64_t)s * (m + 1);
    for (int i = 0; i <= j; ++i) col[i] = a1[i] + a2[i];
    col[j + 1] = make_double2(hn[s], 0.0);
    double2* c = cs + (int64_t)s * m;
    double2* n = sn + (int64_t)s * m;
    for (int i = 0; i < j; ++i) {
        const double2 t = cconj(c[i]) * col[i] + cconj(n[i]) * col[i + 1];
        col[i + 1] = -(n[i] * col[i]) + c[i] * col[i + 1];
        col[i] = t;
    }
    const double r = hypot(cabsd(col[j]), cabsd(col[j + 1]));
    if (r == 0.0) {
        c[j] = make_double2(1.0, 0.0);
        n[j] = make_double2(0.0, 0.0);
    } else {
        c[j] = (1.0 / r) * col[j];
        n[j] = (1.0 / r) * col[j + 1];
    }
    col[j] = make_double2(r, 0.0);
    col[j + 1] = make_double2(0.0, 0.0);
    double2* gs = g + (int64_t)s * (m + 1);
    const double2 gj = gs[j];
    gs[j] = cconj(c[j]) * gj;
    gs[j + 1] = -(n[j] * gj);
    const double est = cabsd(gs[j + 1]);
    kused[s] = j + 1;
    const int d = est <= thresh[s] || hn[s] <= 1e-14 * rnorm[s] || !isfinite(est);
    done[s] = d;
    scale[s] = (!d && hn[s] > 0.0) ? 1.0 / hn[s] : 0.0;
}

// y = R^-1 g over the slot's kused columns (zero beyond), the coefficients of the correction
__global__ void k_backsolve(int S, int m, const double2* __restrict__ H, const double2* __restrict__ g,
                            const int* __restrict__ kused, double2* y) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int k = kused[s];
    double2* ys = y + (int64_t)s * (m + 1);
    for (int i = 0; i <= m; ++i) ys[i] = make_double2(0.0, 0.0);
    const double2* gs = g + (int64_t)s * (m + 1);
    for (int i = k - 1; i >= 0; --i) {
        double2 sum = gs[i];
        for (int l = i + 1; l < k; ++l) sum = sum - H[((int64_t)s * m + l) * (m + 1) + i] * ys[l];
        ys[i] = cdiv(sum, H[((int64_t)s * m + i) * (m + 1) + i]);
    }
}

// slot vectors from system vectors (map[s] < 0: an empty slot, zero)
__global__ void k_gather_sys(const double2* __restrict__ src, double2* dst, const int* __restrict__ map, int nunk,
                             int S) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nunk * S) return;
    const int s = (int)(t / nunk), n = (int)(t % nunk);
    dst[t] = map[s] >= 0 ? src[(int64_t)map[s] * nunk + n] : make_double2(0.0, 0.0);
}

__global__ void k_scatter_sys(const double2* __restrict__ src, double2* dst, const int* __restrict__ map, int nunk,
                              int S) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nunk * S) return;
    const int s = (int)(t / nunk), n = (int)(t % nunk);
    if (map[s] >= 0) dst[(int64_t)map[s] * nunk + n] = src[t];
}

__global__ void k_add_vec(double2* x, const double2* __restrict__ d, int64_t n) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) x[t] = x[t] + d[t];
}

// relative residual per slot (0 for an empty slot)
__global__ void k_relres(int S, const double* __restrict__ rn, const double* __restrict__ bn, double* rel) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) rel[s] = bn[s] > 0.0 ? rn[s] / bn[s] : 0.0;
}

}  // namespace aimx

namespace aimx {

static inline unsigned nb256(int64_t n) { return (unsigned)((n + 255) / 256); }

// Per-frequency tables of a sweep and the slot arrays of the lockstep solver.
struct BatchSweep {
    aimx_ctx* ctx = nullptr;
    cudaStream_t s = nullptr;
    int nf = 0, S = 0, m = 0, nunk = 0, N = 0, nseg = 0, sms = 0;
    int inner = AIMX_F32, precond = AIMX_PRECOND_DIAG;
    double tol = 1e-6;
    std::vector<void*> own;
    // per frequency
    double2* spec64 = nullptr;
    float2* spec32 = nullptr;
    int64_t fstride = 0;
    NearCoefs* ncs = nullptr;
    double2* cphi = nullptr;
    double2* minv = nullptr;      // [nf][4N]
    // per slot
    double2 *V = nullptr, *w = nullptr, *r = nullptr, *d = nullptr, *XS = nullptr, *BS = nullptr;
    void *z = nullptr, *az = nullptr;
    double2 *h1 = nullptr, *h2 = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
    double2* dpart = nullptr;
    double *rnorm = nullptr, *bnorm = nullptr, *hn = nullptr, *thresh = nullptr, *scale = nullptr, *rel = nullptr;
    int *done = nullptr, *kused = nullptr, *map = nullptr, *fidx = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_S = 0, graph_low = -1;
    int64_t products = 0, graphs = 0, cycles = 0;

    void* alloc(size_t bytes) {
        void* p = dev_alloc(ctx, bytes);
        own.push_back(p);
        return p;
    }
    ~BatchSweep() {
        if (exec) cudaGraphExecDestroy(exec);
        for (void* p : own) dev_free(ctx, p);
    }

    MultiFreq multi(int prec) const {
        MultiFreq mf;
        mf.d_fidx = fidx;
        mf.spec = prec == AIMX_F32 ? (const void*)spec32 : (const void*)spec64;
        mf.fstride = fstride;
        mf.d_ncs = ncs;
        mf.d_cphi = cphi;
        return mf;
    }
    // y = A(k_fidx) x over all slots
    void product(const void* x, void* yv, int prec) {
        if (prec == AIMX_F32)
            matvec_generic_multi<float>(ctx, multi(prec), S, (const float*)x, (float*)yv, s);
        else
            matvec_generic_multi<double>(ctx, multi(prec), S, (const double*)x, (double*)yv, s);
    }
    // r = BS - A XS and |r| per slot
    void residual(bool low) {
        const int64_t nv = (int64_t)nunk * S;
        if (low) {
            k_f64_to_f32<<<nb256(nv), 256, 0, s>>>(XS, (float2*)z, nv);
            product(z, az, AIMX_F32);
            k_f32_to_f64<<<nb256(nv), 256, 0, s>>>((const float2*)az, w, nv);
        } else {
            product(XS, w, AIMX_F64);
        }
        k_residual<<<nb256(nv), 256, 0, s>>>(BS, w, r, nv);
        k_norms<<<S, 256, 0, s>>>(r, rnorm, nunk, nunk);
        AIMX_CUDA_TRY(cudaGetLastError());
    }
    void dots(int nvec, double2* hout) {
        const int64_t vstride = (int64_t)(m + 1) * nunk;
        if ((int64_t)nseg * S >= 2 * sms) {
            k_dots_seg<<<dim3(nseg, S), 256, 0, s>>>(V, w, dpart, nunk, vstride, nvec, nseg, m + 1);
            k_dots_fin<<<S, 128, 0, s>>>(dpart, hout, nvec, nseg, m + 1, m + 1);
        } else {
            k_dots<<<dim3(nvec, S), 256, 0, s>>>(V, w, hout, nunk, vstride, m + 1, nvec);
        }
    }
    // One GMRES(m) cycle of every slot from the residual in r: Arnoldi with two classical
    // Gram-Schmidt passes, device Givens rotations, back substitution, x += M V y, and the slot
    // solutions scattered back to the systems' X.
    void cycle_body(double2* X) {
        const int64_t nv = (int64_t)nunk * S;
        const int64_t vstride = (int64_t)(m + 1) * nunk;
        const unsigned tb = (unsigned)((S + 127) / 128);
        const double eta_floor = inner == AIMX_F32 ? 3e-6 : 1e-13;
        k_cycle_init<<<tb, 128, 0, s>>>(S, m, rnorm, bnorm, tol, eta_floor, g, thresh, done, scale, kused);
        k_scale<<<nb256(nv), 256, 0, s>>>(r, V, scale, nunk, nunk, vstride, S);
        for (int j = 0; j < m; ++j) {
            // w = A M v_j, M the slot frequency's inverse blocks (identity without a preconditioner)
            const double2* vj = V + (int64_t)j * nunk;
            if (inner == AIMX_F32) {
                k_precond<float><<<nb256((int64_t)N * S), 256, 0, s>>>(vj, (float2*)z, minv, N, nunk, S, ctx->form,
                                                                      vstride, fidx, 4 * (int64_t)N);
                product(z, az, AIMX_F32);
                k_f32_to_f64<<<nb256(nv), 256, 0, s>>>((const float2*)az, w, nv);
            } else {
                k_precond<double><<<nb256((int64_t)N * S), 256, 0, s>>>(vj, (double2*)z, minv, N, nunk, S, ctx->form,
                                                                        vstride, fidx, 4 * (int64_t)N);
                product(z, w, AIMX_F64);
            }
            dots(j + 1, h1);
            k_subtract<<<nb256(nv), 256, 0, s>>>(V, w, h1, nunk, vstride, m + 1, j + 1, S);
            dots(j + 1, h2);
            k_subtract<<<nb256(nv), 256, 0, s>>>(V, w, h2, nunk, vstride, m + 1, j + 1, S);
            k_norms<<<S, 256, 0, s>>>(w, hn, nunk, nunk);
            k_givens<<<tb, 128, 0, s>>>(S, j, m, h1, h2, hn, H, cs, sn, g, thresh, rnorm, done, scale, kused);
            k_scale<<<nb256(nv), 256, 0, s>>>(w, V + (int64_t)(j + 1) * nunk, scale, nunk, nunk, vstride, S);
        }
        k_backsolve<<<tb, 128, 0, s>>>(S, m, H, g, kused, y);
        k_combine<<<nb256(nv), 256, 0, s>>>(V, y, d, nunk, vstride, m + 1, m, S);
        k_precond_inplace<<<nb256((int64_t)N * S), 256, 0, s>>>(d, minv, N, nunk, S, ctx->form, fidx, 4 * (int64_t)N);
        k_add_vec<<<nb256(nv), 256, 0, s>>>(XS, d, nv);
        k_scatter_sys<<<nb256(nv), 256, 0, s>>>(XS, X, map, nunk, S);
        AIMX_CUDA_TRY(cudaGetLastError());
    }
};

}  // namespace aimx

using namespace aimx;

extern "C" int aimx_sweep_batched(aimx_ctx* ctx, int nf, const double* freqs, int nrhs, const void* Bdev, void* Xdev,
                                  const aimx_solve_opts* opts_in, int max_batch, int warm_start,
                                  aimx_solve_stats* stats, int64_t* counters, void* stream) {
    if (!ctx) return AIMX_E_ARG;
    if (nf <= 0 || !freqs || nrhs <= 0 || !Bdev || !Xdev || max_batch < 0) {
        ctx->last_error = "aimx_sweep_batched: bad argument";
        return AIMX_E_ARG;
    }
    for (int f = 0; f < nf; ++f)
        if (!(freqs[f] > 0)) {
            ctx->last_error = "aimx_sweep_batched: frequencies must be positive";
            return AIMX_E_ARG;
        }
    aimx_solve_opts o;
    if (opts_in)
        o = *opts_in;
    else
        std::memset(&o, 0, sizeof(o));
    if (!(o.tol > 0)) o.tol = 1e-6;
    if (o.restart <= 0) o.restart = 50;
    if (o.max_iter <= 0) o.max_iter = 1000;
    if (o.max_refine <= 0) o.max_refine = o.max_iter / o.restart + 10;
    if (o.inner_precision != AIMX_F64) o.inner_precision = AIMX_F32;
    if (o.precond != AIMX_PRECOND_DIAG && o.precond != AIMX_PRECOND_NONE) {
        ctx->last_error = "aimx_sweep_batched: only the diagonal preconditioner or none";
        return AIMX_E_STATE;
    }
    if (ctx->aim) {
        ctx->last_error = "aimx_sweep_batched: not available in the conventional-AIM mode";
        return AIMX_E_STATE;
    }
    cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
    cudaStream_t ps = nullptr;
    cudaEvent_t ev = nullptr;
    const bool prof_on = ctx->prof.on;
    int rc = AIMX_OK;
    try {
        AIMX_CUDA_TRY(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking));
        AIMX_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        AIMX_CUDA_TRY(cudaEventRecord(ev, caller));
        AIMX_CUDA_TRY(cudaStreamWaitEvent(ps, ev, 0));
        BatchSweep bs;
        bs.ctx = ctx;
        bs.s = ps;
        bs.nf = nf;
        bs.m = o.restart;
        bs.nunk = ctx->nunk;
        bs.N = ctx->N;
        bs.inner = o.inner_precision;
        bs.precond = o.precond;
        bs.tol = o.tol;
        int dev = 0;
        AIMX_CUDA_TRY(cudaGetDevice(&dev));
        AIMX_CUDA_TRY(cudaDeviceGetAttribute(&bs.sms, cudaDevAttrMultiProcessorCount, dev));
        const int N = ctx->N, nunk = ctx->nunk, m = o.restart;
        const int nsys = nf * nrhs;
        // ---- per-frequency tables: spectra, near coefficients, preconditioner blocks
        const int64_t OT = (int64_t)(ctx->M[0] / 2 + 1) * (ctx->M[1] / 2 + 1) * (ctx->M[2] / 2 + 1);
        bs.fstride = (int64_t)ctx->nspec * OT;
        bs.spec64 = (double2*)bs.alloc(sizeof(double2) * nf * bs.fstride);
        bs.spec32 = (float2*)bs.alloc(sizeof(float2) * nf * bs.fstride);
        bs.ncs = (NearCoefs*)bs.alloc(sizeof(NearCoefs) * nf);
        bs.cphi = (double2*)bs.alloc(sizeof(double2) * nf);
        bs.minv = (double2*)bs.alloc(sizeof(double2) * 4 * (size_t)N * nf);
        std::vector<NearCoefs> hnc(nf);
        std::vector<double2> hcp(nf);
        for (int f = 0; f < nf; ++f) {
            ensure_spectra<double>(ctx, freqs[f], ps);   // fills the FP64 and FP32 octant spectra
            AIMX_CUDA_TRY(cudaMemcpyAsync(bs.spec64 + f * bs.fstride, ctx->f64.spec, sizeof(double2) * bs.fstride,
                                          cudaMemcpyDeviceToDevice, ps));
            AIMX_CUDA_TRY(cudaMemcpyAsync(bs.spec32 + f * bs.fstride, ctx->f32.spec, sizeof(float2) * bs.fstride,
                                          cudaMemcpyDeviceToDevice, ps));
            const Coefs cf = near_coefs(ctx, freqs[f]);
            for (int k = 0; k < 6; ++k) hnc[f].c[k] = cf.near[k];
            for (int k = 0; k < 4; ++k) hnc[f].lin[k] = cf.lin[k];
            hcp[f] = cf.near[1];
            if (o.precond == AIMX_PRECOND_DIAG) build_diag_inverse(ctx, freqs[f], bs.minv + 4 * (size_t)N * f, ps);
        }
        if (o.precond == AIMX_PRECOND_NONE) {
            std::vector<double2> one(4 * (size_t)N * nf, make_double2(0, 0));
            for (int f = 0; f < nf; ++f)
                for (int i = 0; i < N; ++i) {
                    double2* blk = one.data() + 4 * (size_t)N * f;
                    if (ctx->form != AIMX_PMCHWT) {
                        blk[i] = make_double2(1, 0);
                    } else {
                        blk[4 * i] = make_double2(1, 0);
                        blk[4 * i + 3] = make_double2(1, 0);
                    }
                }
            AIMX_CUDA_TRY(cudaMemcpyAsync(bs.minv, one.data(), sizeof(double2) * one.size(), cudaMemcpyHostToDevice, ps));
            AIMX_CUDA_TRY(cudaStreamSynchronize(ps));
        }
        AIMX_CUDA_TRY(cudaMemcpyAsync(bs.ncs, hnc.data(), sizeof(NearCoefs) * nf, cudaMemcpyHostToDevice, ps));
        AIMX_CUDA_TRY(cudaMemcpyAsync(bs.cphi, hcp.data(), sizeof(double2) * nf, cudaMemcpyHostToDevice, ps));
        // ---- slots: as many systems as fit about 8 GiB of Krylov vectors (or max_batch)
        const size_t per_slot = sizeof(double2) * (size_t)nunk * (m + 8);
        int Smax = (int)std::max<size_t>(1, std::min<size_t>(nsys, ((size_t)8 << 30) / per_slot));
        if (max_batch > 0) Smax = std::min(Smax, max_batch);
        const int S0 = Smax;
        bs.nseg = (nunk + kDotSeg - 1) / kDotSeg;
        const int64_t nv0 = (int64_t)nunk * S0;
        bs.V = (double2*)bs.alloc(sizeof(double2) * (size_t)S0 * (m + 1) * nunk);
        bs.w = (double2*)bs.alloc(sizeof(double2) * nv0);
        bs.r = (double2*)bs.alloc(sizeof(double2) * nv0);
        bs.d = (double2*)bs.alloc(sizeof(double2) * nv0);
        bs.XS = (double2*)bs.alloc(sizeof(double2) * nv0);
        bs.BS = (double2*)bs.alloc(sizeof(double2) * nv0);
        bs.z = bs.alloc(sizeof(double2) * nv0);
        bs.az = bs.alloc(sizeof(double2) * nv0);
        bs.h1 = (double2*)bs.alloc(sizeof(double2) * (size_t)S0 * (m + 1));
        bs.h2 = (double2*)bs.alloc(sizeof(double2) * (size_t)S0 * (m + 1));
        bs.g = (double2*)bs.alloc(sizeof(double2) * (size_t)S0 * (m + 1));
        bs.y = (double2*)bs.alloc(sizeof(double2) * (size_t)S0 * (m + 1));
        bs.H = (double2*)bs.alloc(sizeof(double2) * (size_t)S0 * m * (m + 1));
        bs.cs = (double2*)bs.alloc(sizeof(double2) * (size_t)S0 * m);
        bs.sn = (double2*)bs.alloc(sizeof(double2) * (size_t)S0 * m);
        bs.dpart = (double2*)bs.alloc(sizeof(double2) * (size_t)S0 * bs.nseg * 8 * (m + 1));
        for (double** p : {&bs.rnorm, &bs.bnorm, &bs.hn, &bs.thresh, &bs.scale, &bs.rel})
            *p = (double*)bs.alloc(sizeof(double) * S0);
        for (int** p : {&bs.done, &bs.kused, &bs.map, &bs.fidx}) *p = (int*)bs.alloc(sizeof(int) * S0);
        const double2* B = (const double2*)Bdev;
        double2* X = (double2*)Xdev;
        if (!o.use_x0) AIMX_CUDA_TRY(cudaMemsetAsync(X, 0, sizeof(double2) * (size_t)nsys * nunk, ps));
        // ---- host state per system
        enum { PENDING = 0, ACTIVE = 1, DONE32 = 2, DONE = 3, FAILED = 4 };
        std::vector<int> state(nsys, PENDING), iters(nsys, 0), refs(nsys, 0);
        std::vector<double> relres(nsys, 1.0);
        bool low = o.inner_precision == AIMX_F32 && o.tol >= 1e-5;
        int S = S0, next = 0;
        // admission order: frequency-major; with warm starts even frequency indices first, so that
        // the odd ones enter next to converged neighbours whose solutions start them
        std::vector<int> order;
        order.reserve(nsys);
        for (int par = 0; par < (warm_start ? 2 : 1); ++par)
            for (int f = warm_start ? par : 0; f < nf; f += warm_start ? 2 : 1)
                for (int wv = 0; wv < nrhs; ++wv) order.push_back(f * nrhs + wv);
        auto warm = [&](int q) {
            // the converged system of the same right-hand side at the nearest frequency
            const int f = q / nrhs, wv = q % nrhs;
            int best = -1;
            for (int d = 1; d < nf && best < 0; ++d)
                for (int f2 : {f - d, f + d})
                    if (f2 >= 0 && f2 < nf && best < 0 &&
                        (state[f2 * nrhs + wv] == DONE || state[f2 * nrhs + wv] == DONE32))
                        best = f2 * nrhs + wv;
            if (best >= 0)
                AIMX_CUDA_TRY(cudaMemcpyAsync(X + (size_t)q * nunk, X + (size_t)best * nunk, sizeof(double2) * nunk,
                                              cudaMemcpyDeviceToDevice, ps));
        };
        std::vector<int> slot_sys(S0, -1), hmap(S0), hfidx(S0), hk(S0);
        std::vector<double> hrel(S0);
        bool changed = true;
        auto upload_slots = [&]() {
            for (int sl = 0; sl < S; ++sl) {
                hmap[sl] = slot_sys[sl];
                hfidx[sl] = slot_sys[sl] >= 0 ? slot_sys[sl] / nrhs : 0;
            }
            AIMX_CUDA_TRY(cudaMemcpyAsync(bs.map, hmap.data(), sizeof(int) * S, cudaMemcpyHostToDevice, ps));
            AIMX_CUDA_TRY(cudaMemcpyAsync(bs.fidx, hfidx.data(), sizeof(int) * S, cudaMemcpyHostToDevice, ps));
            const int64_t nv = (int64_t)nunk * S;
            k_gather_sys<<<nb256(nv), 256, 0, ps>>>(X, bs.XS, bs.map, nunk, S);
            k_gather_sys<<<nb256(nv), 256, 0, ps>>>(B, bs.BS, bs.map, nunk, S);
            k_norms<<<S, 256, 0, ps>>>(bs.BS, bs.bnorm, nunk, nunk);
            AIMX_CUDA_TRY(cudaGetLastError());
        };
        for (int pass = 0; pass < 2; ++pass) {
            for (;;) {
                // retire finished systems, fill free slots with pending ones
                int busy = 0;
                for (int sl = 0; sl < S; ++sl) {
                    const int q = slot_sys[sl];
                    if (q >= 0 && state[q] != ACTIVE) {
                        slot_sys[sl] = -1;
                        changed = true;
                    }
                    if (slot_sys[sl] < 0) {
                        while (next < nsys && state[order[next]] != PENDING) ++next;
                        if (next < nsys) {
                            const int q = order[next++];
                            if (warm_start && !o.use_x0 && pass == 0) warm(q);
                            slot_sys[sl] = q;
                            state[q] = ACTIVE;
                            changed = true;
                        }
                    }
                    busy += slot_sys[sl] >= 0;
                }
                if (busy == 0) break;
                if (busy < (3 * S) / 4) {
                    // compact onto fewer slots (a new graph for the new count)
                    std::vector<int> keep;
                    for (int sl = 0; sl < S; ++sl)
                        if (slot_sys[sl] >= 0) keep.push_back(slot_sys[sl]);
                    S = busy;
                    for (int sl = 0; sl < S0; ++sl) slot_sys[sl] = sl < S ? keep[sl] : -1;
                    changed = true;
                }
                bs.S = S;
                if (changed) {
                    upload_slots();
                    bs.residual(low);
                    ++bs.products;
                    changed = false;
                }
                if (!bs.exec || bs.graph_S != S || bs.graph_low != (int)low) {
                    // every buffer the products use exists at this slot count before capture
                    bs.product(bs.z, bs.az, o.inner_precision);
                    bs.product(bs.z, bs.az, low ? AIMX_F32 : AIMX_F64);
                    AIMX_CUDA_TRY(cudaStreamSynchronize(ps));
                    if (bs.exec) {
                        cudaGraphExecDestroy(bs.exec);
                        bs.exec = nullptr;
                    }
                    ctx->prof.on = false;
                    cudaGraph_t graph = nullptr;
                    AIMX_CUDA_TRY(cudaStreamBeginCapture(ps, cudaStreamCaptureModeThreadLocal));
                    try {
                        bs.cycle_body(X);
                        bs.residual(low);
                        k_relres<<<(unsigned)((S + 127) / 128), 128, 0, ps>>>(S, bs.rnorm, bs.bnorm, bs.rel);
                    } catch (...) {
                        cudaStreamEndCapture(ps, &graph);
                        if (graph) cudaGraphDestroy(graph);
                        throw;
                    }
                    AIMX_CUDA_TRY(cudaStreamEndCapture(ps, &graph));
                    const cudaError_t ie = cudaGraphInstantiate(&bs.exec, graph, 0);
                    cudaGraphDestroy(graph);
                    AIMX_CUDA_TRY(ie);
                    ctx->prof.on = prof_on;
                    bs.graph_S = S;
                    bs.graph_low = (int)low;
                    ++bs.graphs;
                }
                AIMX_CUDA_TRY(cudaGraphLaunch(bs.exec, ps));
                ++bs.cycles;
                bs.products += m + 1;          // m Arnoldi products and the closing residual
                AIMX_CUDA_TRY(cudaMemcpyAsync(hrel.data(), bs.rel, sizeof(double) * S, cudaMemcpyDeviceToHost, ps));
                AIMX_CUDA_TRY(cudaMemcpyAsync(hk.data(), bs.kused, sizeof(int) * S, cudaMemcpyDeviceToHost, ps));
                AIMX_CUDA_TRY(cudaStreamSynchronize(ps));
                for (int sl = 0; sl < S; ++sl) {
                    const int q = slot_sys[sl];
                    if (q < 0) continue;
                    iters[q] += hk[sl];
                    refs[q] += 1;
                    relres[q] = hrel[sl];
                    if (relres[q] <= o.tol)
                        state[q] = low ? DONE32 : DONE;
                    else if (!std::isfinite(relres[q]) || iters[q] >= o.max_iter || refs[q] >= o.max_refine)
                        state[q] = FAILED;
                }
            }
            // reported residuals from the FP64 product, for every system, in batches of slots
            bool reopen = false;
            S = S0;
            bs.S = S;
            for (int q0 = 0; q0 < nsys; q0 += S) {
                for (int sl = 0; sl < S; ++sl) slot_sys[sl] = q0 + sl < nsys ? q0 + sl : -1;
                upload_slots();
                bs.residual(false);
                ++bs.products;
                k_relres<<<(unsigned)((S + 127) / 128), 128, 0, ps>>>(S, bs.rnorm, bs.bnorm, bs.rel);
                AIMX_CUDA_TRY(cudaMemcpyAsync(hrel.data(), bs.rel, sizeof(double) * S, cudaMemcpyDeviceToHost, ps));
                AIMX_CUDA_TRY(cudaStreamSynchronize(ps));
                for (int sl = 0; sl < S; ++sl) {
                    const int q = slot_sys[sl];
                    if (q < 0) continue;
                    relres[q] = hrel[sl];
                    if (state[q] == DONE32) {
                        if (relres[q] <= o.tol) {
                            state[q] = DONE;
                        } else if (pass == 0 && iters[q] < o.max_iter && refs[q] < o.max_refine) {
                            state[q] = PENDING;   // not confirmed: more cycles with FP64 residuals
                            reopen = true;
                        } else {
                            state[q] = FAILED;
                        }
                    }
                }
            }
            for (int sl = 0; sl < S0; ++sl) slot_sys[sl] = -1;
            changed = true;
            if (!reopen) break;
            low = false;
            next = 0;
        }
        bool allok = true;
        for (int q = 0; q < nsys; ++q) {
            const bool ok = state[q] == DONE && relres[q] <= o.tol;
            allok = allok && ok;
            if (stats) {
                stats[q].iterations = iters[q];
                stats[q].refinements = refs[q];
                stats[q].rel_residual = relres[q];
                stats[q].status = ok ? AIMX_OK : AIMX_E_NOCONV;
                stats[q].precond_used = o.precond;
            }
        }
        if (counters) {
            counters[0] = bs.cycles;
            counters[1] = bs.graphs;
            counters[2] = bs.products;
        }
        if (!allok) rc = AIMX_E_NOCONV;
        AIMX_CUDA_TRY(cudaEventRecord(ev, ps));
        AIMX_CUDA_TRY(cudaStreamWaitEvent(caller, ev, 0));
        AIMX_CUDA_TRY(cudaStreamSynchronize(ps));
    } catch (const Error& e) {
        ctx->last_error = e.msg;
        rc = e.code;
        if (ps) cudaStreamSynchronize(ps);
    }
    ctx->prof.on = prof_on;
    if (ev) cudaEventDestroy(ev);
    if (ps) cudaStreamDestroy(ps);
    return rc;
}
