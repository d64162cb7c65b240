// C ABI entry points of libaimx (declared in include/aimx.h).  Every entry
// point catches internal errors and returns a status code; nothing throws
// across the ABI.

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>

#include "aimx_internal.h"

namespace aimx {

void* dev_alloc(aimx_ctx* ctx, size_t bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes ? bytes : 1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{AIMX_E_NOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e)};
    }
    ctx->device_bytes += (int64_t)bytes;
    return p;
}

void dev_free(aimx_ctx* ctx, void* p) {
    (void)ctx;
    if (p) cudaFree(p);
}

static int fail(aimx_ctx* ctx, const Error& e) {
    if (ctx) ctx->last_error = e.msg;
    return e.code;
}

static void free_all(aimx_ctx* c) {
    void* ptrs[] = {c->d_xyz,     c->d_tri,     c->d_area,     c->d_btri,   c->d_bfree,  c->d_blen,
                    c->d_anc,     c->d_perm,    c->d_row_ptr,  c->d_cols,   c->d_node_ptr,
                    c->d_node_w,  c->d_node_x,  c->d_diag,     c->f32.w,    c->f32.na,   c->f32.np,
                    c->f32.nk,    c->f32.spec,  c->f32.grid,   c->f64.w,    c->f64.na,   c->f64.np,
                    c->f64.nk,    c->f64.spec,  c->f64.grid,   c->d_kgen,   c->d_stage,
                    c->d_xT,      c->d_G,       c->d_S,        c->d_part,   c->d_plane,  c->d_q5,
                    c->pc.d_ptr,  c->pc.d_idx,  c->pc.d_work,  c->pc.d_inv, c->d_wsoa,   c->f32.ng,
                    c->f64.ng,    c->d_gdiag,   c->d_lin_ptr,  c->d_lin_cols, c->f64.la, c->f64.lp,
                    c->f32.la,    c->f32.lp,    c->f64.zn,     c->f32.zn,     c->d_aim_row_of, c->d_aim_htab,
                    c->d_nb_rows, c->d_nb_ustart, c->d_nb_ucols, c->d_nb_ent,
                    c->d_tanc, c->d_trow_ptr, c->d_tcols, c->d_tnode_ptr, c->d_tnode_w, c->d_tinc,
                    c->d_btri_t, c->d_tplane, c->d_lp_soa, c->d_qT, c->d_phiT, c->d_tpart,
                    c->f64.plw, c->f32.plw, c->f64.npt, c->f32.npt, c->f64.tl, c->f32.tl,
                    c->f64.cwork, c->f32.cwork};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& r : c->prof.recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->prof.pool) cudaEventDestroy(e);
    gnn_free(c);
    cufft_release(c);
    c->prof.recs.clear();
    c->prof.pool.clear();
}

static cudaEvent_t pool_event(aimx_ctx* ctx) {
    if (!ctx->prof.pool.empty()) {
        cudaEvent_t e = ctx->prof.pool.back();
        ctx->prof.pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    AIMX_CUDA_TRY(cudaEventCreate(&e));
    return e;
}

StageScope::StageScope(aimx_ctx* c, int st, cudaStream_t str) : ctx(c), stage(st), s(str) {
    if (!ctx->prof.on) return;
    a = pool_event(ctx);
    b = pool_event(ctx);
    AIMX_CUDA_TRY(cudaEventRecord(a, s));
}

StageScope::~StageScope() {
    if (!a) return;
    if (cudaEventRecord(b, s) == cudaSuccess) ctx->prof.recs.push_back(ProfRec{stage, a, b});
}

static const char* kStageNames[ST_COUNT] = {
    "kernel_spectra", "transpose_x", "gather_projection", "xy_fft_forward", "z_fft_mix_inverse",
    "xy_fft_inverse_interp", "near_final", "generic_projection", "generic_fft", "generic_mix",
    "generic_interp_near", "solver_vector_ops", "solver_true_residual", "solver_precond",
    "solver_reorthogonalization", "aim_near_fill"};

}  // namespace aimx

using namespace aimx;

extern "C" {

const char* aimx_status_string(int status) {
    switch (status) {
        case AIMX_OK: return "ok";
        case AIMX_E_ARG: return "invalid argument";
        case AIMX_E_MESH: return "invalid mesh";
        case AIMX_E_GRID: return "stencil outside the grid";
        case AIMX_E_NOMEM: return "out of memory";
        case AIMX_E_CUDA: return "CUDA error";
        case AIMX_E_TIMEOUT: return "bounded device wait expired";
        case AIMX_E_STATE: return "call not valid for this context";
        case AIMX_E_IO: return "static-data file error";
        case AIMX_E_NOCONV: return "solver did not reach the tolerance";
        default: return "unknown status";
    }
}

const char* aimx_last_error(const aimx_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int aimx_setup(const aimx_mesh* mesh, const aimx_material* mat, const aimx_grid* grid, int order,
               aimx_ctx** out) {
    if (!out) return AIMX_E_ARG;
    *out = nullptr;
    aimx_ctx* ctx = new (std::nothrow) aimx_ctx();
    if (!ctx) return AIMX_E_NOMEM;
    try {
        setup_context(ctx, mesh, mat, grid, order);
    } catch (const Error& e) {
        cudaDeviceSynchronize();
        cudaGetLastError();
        free_all(ctx);
        int code = e.code;
        delete ctx;
        return code;
    } catch (const std::bad_alloc&) {
        free_all(ctx);
        delete ctx;
        return AIMX_E_NOMEM;
    }
    *out = ctx;
    return AIMX_OK;
}

int aimx_destroy(aimx_ctx* ctx) {
    if (!ctx) return AIMX_OK;
    cudaDeviceSynchronize();
    free_all(ctx);
    delete ctx;
    return AIMX_OK;
}

int aimx_info(const aimx_ctx* ctx, aimx_info_t* out) {
    if (!ctx || !out) return AIMX_E_ARG;
    std::memset(out, 0, sizeof(*out));
    out->n_basis = ctx->N;
    out->n_unknowns = ctx->nunk;
    out->near_nnz = ctx->nnz;
    for (int a = 0; a < 3; ++a) {
        out->grid_n[a] = ctx->n[a];
        out->pad[a] = ctx->M[a];
        out->grid_h[a] = ctx->h[a];
        out->grid_origin[a] = ctx->origin[a];
    }
    out->order = ctx->order;
    out->formulation = ctx->form;
    out->device_bytes = ctx->device_bytes;
    return AIMX_OK;
}

int aimx_matvec(aimx_ctx* ctx, double freq, int nrhs, const void* x, void* y, int precision,
                void* stream) {
    if (!ctx || !x || !y || nrhs <= 0 || !(freq > 0)) return ctx ? fail(ctx, Error{AIMX_E_ARG, "bad argument"}) : AIMX_E_ARG;
    if (precision != AIMX_F32 && precision != AIMX_F64) return fail(ctx, Error{AIMX_E_ARG, "bad precision"});
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    try {
        if (precision == AIMX_F32 && use_fused(ctx))
            matvec_fused(ctx, freq, nrhs, (const float*)x, (float*)y, s);
        else if (precision == AIMX_F32)
            matvec_generic<float>(ctx, freq, nrhs, (const float*)x, (float*)y, s);
        else
            matvec_generic<double>(ctx, freq, nrhs, (const double*)x, (double*)y, s);
    } catch (const Error& e) {
        return fail(ctx, e);
    }
    return AIMX_OK;
}

int aimx_matvec_host(aimx_ctx* ctx, double freq, int nrhs, const void* x, void* y, int precision,
                     void* stream) {
    if (!ctx || !x || !y || nrhs <= 0) return ctx ? fail(ctx, Error{AIMX_E_ARG, "bad argument"}) : AIMX_E_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    size_t es = precision == AIMX_F64 ? 2 * sizeof(double) : 2 * sizeof(float);
    size_t bytes = es * (size_t)nrhs * ctx->nunk;
    try {
        if (ctx->stage_bytes < 2 * bytes) {
            if (ctx->d_stage) dev_free(ctx, ctx->d_stage);
            ctx->d_stage = dev_alloc(ctx, 2 * bytes);
            ctx->stage_bytes = 2 * bytes;
        }
        char* dx = (char*)ctx->d_stage;
        char* dy = dx + bytes;
        AIMX_CUDA_TRY(cudaMemcpyAsync(dx, x, bytes, cudaMemcpyHostToDevice, s));
        int rc = aimx_matvec(ctx, freq, nrhs, dx, dy, precision, stream);
        if (rc != AIMX_OK) return rc;
        AIMX_CUDA_TRY(cudaMemcpyAsync(y, dy, bytes, cudaMemcpyDeviceToHost, s));
        AIMX_CUDA_TRY(cudaStreamSynchronize(s));
    } catch (const Error& e) {
        return fail(ctx, e);
    }
    return AIMX_OK;
}

int aimx_set_path(aimx_ctx* ctx, int path) {
    if (!ctx || path < 0 || path > 2) return AIMX_E_ARG;
    if (ctx->path != path) ctx->config_gen++;
    ctx->path = path;
    return AIMX_OK;
}

int aimx_set_linear_term(aimx_ctx* ctx, int enable) {
    if (!ctx || enable < 0 || enable > 1) return AIMX_E_ARG;
    if (enable && ctx->charge)
        return fail(ctx, Error{AIMX_E_STATE, "the linear term is not combined with the charge form"});
    try {
        if (enable) build_linterm(ctx);
        if (ctx->linterm != enable) ctx->config_gen++;
        ctx->linterm = enable;
    } catch (const Error& e) {
        return fail(ctx, e);
    }
    return AIMX_OK;
}

int aimx_set_conventional_aim(aimx_ctx* ctx, int enable) {
    if (!ctx || enable < 0 || enable > 1) return AIMX_E_ARG;
    if (enable && ctx->charge)
        return fail(ctx, Error{AIMX_E_STATE, "the conventional-AIM mode is not combined with the charge form"});
    try {
        if (enable) aim_enable(ctx);
        if (ctx->aim != enable) ctx->config_gen++;
        ctx->aim = enable;
    } catch (const Error& e) {
        return fail(ctx, e);
    }
    return AIMX_OK;
}

int aimx_set_charge_form(aimx_ctx* ctx, int enable) {
    if (!ctx || enable < 0 || enable > 1) return AIMX_E_ARG;
    if (enable && ctx->form != AIMX_EFIE && ctx->form != AIMX_PMCHWT)
        return fail(ctx, Error{AIMX_E_STATE, "the charge form is available for the EFIE and the PMCHWT"});
    if (enable && (ctx->linterm || ctx->aim))
        return fail(ctx, Error{AIMX_E_STATE,
                               "the charge form is not combined with the linear term or the conventional-AIM mode"});
    try {
        if (enable) build_charge(ctx);
        if (ctx->charge != enable) ctx->config_gen++;
        ctx->charge = enable;
    } catch (const Error& e) {
        return fail(ctx, e);
    }
    return AIMX_OK;
}

int aimx_export_charge(aimx_ctx* ctx, int32_t* nt_out, int64_t* tnnz, int32_t* tanc, int32_t* rows, int32_t* cols,
                       double* npt, double* lp) {
    if (!ctx) return AIMX_E_ARG;
    if (!ctx->charge_built) {
        ctx->last_error = "the charge form has not been enabled on this context";
        return AIMX_E_STATE;
    }
    try {
        const int nt = ctx->nt, U = ctx->U;
        const int64_t nn = ctx->tnnz;
        if (nt_out) *nt_out = nt;
        if (tnnz) *tnnz = nn;
        if (tanc)
            for (int i = 0; i < nt; ++i)
                for (int a = 0; a < 3; ++a) tanc[3 * (size_t)ctx->tperm[i] + a] = ctx->tanc[3 * (size_t)i + a];
        if (rows || cols)
            for (int i = 0; i < nt; ++i)
                for (int e = ctx->trow_ptr[i]; e < ctx->trow_ptr[i + 1]; ++e) {
                    if (rows) rows[e] = ctx->tperm[i];
                    if (cols) cols[e] = ctx->tperm[ctx->tcols[e]];
                }
        if (npt && nn) AIMX_CUDA_TRY(cudaMemcpy(npt, ctx->f64.npt, nn * sizeof(double), cudaMemcpyDeviceToHost));
        if (lp) {
            std::vector<double> v((size_t)nt * U);
            AIMX_CUDA_TRY(cudaMemcpy(v.data(), ctx->f64.plw, v.size() * sizeof(double), cudaMemcpyDeviceToHost));
            for (int i = 0; i < nt; ++i)
                std::memcpy(lp + (size_t)ctx->tperm[i] * U, v.data() + (size_t)i * U, sizeof(double) * U);
        }
    } catch (const Error& e) {
        ctx->last_error = e.msg;
        return e.code;
    }
    return AIMX_OK;
}

int aimx_export_aim_near(aimx_ctx* ctx, double freq, double* z) {
    if (!ctx || !z) return AIMX_E_ARG;
    if (!ctx->aim) {
        ctx->last_error = "the conventional-AIM mode is not enabled on this context";
        return AIMX_E_STATE;
    }
    try {
        ensure_aim_near(ctx, freq, 0);
        std::vector<double2> v(ctx->nnz);
        AIMX_CUDA_TRY(cudaMemcpy(v.data(), ctx->f64.zn, ctx->nnz * sizeof(double2), cudaMemcpyDeviceToHost));
        const int N = ctx->N;
        std::vector<int64_t> rp(N + 1, 0);
        for (int i = 0; i < N; ++i) rp[ctx->perm[i] + 1] = ctx->row_ptr[i + 1] - ctx->row_ptr[i];
        for (int i = 0; i < N; ++i) rp[i + 1] += rp[i];
        std::vector<std::pair<int, int>> tmp;
        for (int i = 0; i < N; ++i) {
            tmp.clear();
            for (int e = ctx->row_ptr[i]; e < ctx->row_ptr[i + 1]; ++e) tmp.push_back({ctx->perm[ctx->cols[e]], e});
            std::sort(tmp.begin(), tmp.end());
            const int64_t base = rp[ctx->perm[i]];
            for (size_t k = 0; k < tmp.size(); ++k) {
                z[2 * (base + k)] = v[tmp[k].second].x;
                z[2 * (base + k) + 1] = v[tmp[k].second].y;
            }
        }
    } catch (const Error& e) {
        return fail(ctx, e);
    }
    return AIMX_OK;
}

int aimx_export_linear_term(const aimx_ctx* ctx, int64_t* nlin, int64_t* row_ptr, int32_t* cols, double* na,
                            double* nphi) {
    if (!ctx) return AIMX_E_ARG;
    aimx_ctx* c = const_cast<aimx_ctx*>(ctx);
    if (!ctx->nlin) {
        c->last_error = "the linear term has not been enabled on this context";
        return AIMX_E_STATE;
    }
    try {
        const int N = ctx->N;
        const int64_t nl = ctx->nlin;
        if (nlin) *nlin = nl;
        if (row_ptr || cols || na || nphi) {
            std::vector<double> va(nl), vp(nl);
            AIMX_CUDA_TRY(cudaMemcpy(va.data(), ctx->f64.la, nl * sizeof(double), cudaMemcpyDeviceToHost));
            AIMX_CUDA_TRY(cudaMemcpy(vp.data(), ctx->f64.lp, nl * sizeof(double), cudaMemcpyDeviceToHost));
            std::vector<int64_t> rp(N + 1, 0);
            for (int i = 0; i < N; ++i) rp[ctx->perm[i] + 1] = ctx->lin_ptr[i + 1] - ctx->lin_ptr[i];
            for (int i = 0; i < N; ++i) rp[i + 1] += rp[i];
            if (row_ptr) std::memcpy(row_ptr, rp.data(), sizeof(int64_t) * (N + 1));
            std::vector<std::pair<int, int>> tmp;
            for (int i = 0; i < N; ++i) {
                tmp.clear();
                for (int e = ctx->lin_ptr[i]; e < ctx->lin_ptr[i + 1]; ++e)
                    tmp.push_back({ctx->perm[ctx->lin_cols[e]], e});
                std::sort(tmp.begin(), tmp.end());
                const int64_t base = rp[ctx->perm[i]];
                for (size_t k = 0; k < tmp.size(); ++k) {
                    if (cols) cols[base + k] = tmp[k].first;
                    if (na) na[base + k] = va[tmp[k].second];
                    if (nphi) nphi[base + k] = vp[tmp[k].second];
                }
            }
        }
    } catch (const Error& e) {
        return fail(c, e);
    }
    return AIMX_OK;
}

int aimx_matvec_path(const aimx_ctx* ctx, int precision) {
    if (!ctx) return AIMX_E_ARG;
    if (precision == AIMX_F32 && use_fused(ctx)) return 0;
    return ctx->path == 2 ? 2 : 1;
}

int aimx_profile(aimx_ctx* ctx, int enable) {
    if (!ctx) return AIMX_E_ARG;
    ctx->prof.on = enable != 0;
    return AIMX_OK;
}

const char* aimx_profile_stage_name(int stage) {
    return (stage >= 0 && stage < ST_COUNT) ? kStageNames[stage] : "";
}

int aimx_profile_read(aimx_ctx* ctx, double* ms, int64_t* launches, int max_stages) {
    if (!ctx || max_stages < 0) return AIMX_E_ARG;
    try {
        for (auto& r : ctx->prof.recs) {
            AIMX_CUDA_TRY(cudaEventSynchronize(r.b));
            float t = 0.f;
            AIMX_CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
            ctx->prof.ms[r.stage] += t;
            ctx->prof.count[r.stage] += 1;
            ctx->prof.pool.push_back(r.a);
            ctx->prof.pool.push_back(r.b);
        }
        ctx->prof.recs.clear();
        for (int k = 0; k < max_stages && k < ST_COUNT; ++k) {
            if (ms) ms[k] = ctx->prof.ms[k];
            if (launches) launches[k] = ctx->prof.count[k];
            ctx->prof.ms[k] = 0.0;
            ctx->prof.count[k] = 0;
        }
    } catch (const Error& e) {
        return fail(ctx, e);
    }
    return ST_COUNT;
}

int aimx_export_setup(const aimx_ctx* ctx, int32_t* anchors, double* weights, int64_t* row_ptr,
                      int32_t* cols, double* na, double* nphi, double* nk) {
    if (!ctx) return AIMX_E_ARG;
    aimx_ctx* c = const_cast<aimx_ctx*>(ctx);
    try {
        const int N = ctx->N, U = ctx->U;
        if (anchors)
            for (int i = 0; i < N; ++i)
                for (int a = 0; a < 3; ++a) anchors[3 * ctx->perm[i] + a] = ctx->anc[3 * i + a];
        if (weights) {
            std::vector<double> w((size_t)N * U * 4);
            AIMX_CUDA_TRY(cudaMemcpy(w.data(), ctx->f64.w, w.size() * sizeof(double), cudaMemcpyDeviceToHost));
            for (int i = 0; i < N; ++i)
                std::memcpy(weights + (size_t)ctx->perm[i] * U * 4, &w[(size_t)i * U * 4], sizeof(double) * U * 4);
        }
        // near pairs re-indexed to caller numbering, columns ascending
        if (row_ptr || cols || na || nphi || nk) {
            std::vector<double> va(ctx->nnz), vp(ctx->nnz), vk(ctx->nnz);
            AIMX_CUDA_TRY(cudaMemcpy(va.data(), ctx->f64.na, ctx->nnz * sizeof(double), cudaMemcpyDeviceToHost));
            AIMX_CUDA_TRY(cudaMemcpy(vp.data(), ctx->f64.np, ctx->nnz * sizeof(double), cudaMemcpyDeviceToHost));
            AIMX_CUDA_TRY(cudaMemcpy(vk.data(), ctx->f64.nk, ctx->nnz * sizeof(double), cudaMemcpyDeviceToHost));
            std::vector<int64_t> rp(N + 1, 0);
            for (int i = 0; i < N; ++i) rp[ctx->perm[i] + 1] = ctx->row_ptr[i + 1] - ctx->row_ptr[i];
            for (int i = 0; i < N; ++i) rp[i + 1] += rp[i];
            if (row_ptr) std::memcpy(row_ptr, rp.data(), sizeof(int64_t) * (N + 1));
            std::vector<std::pair<int, int>> tmp;
            for (int i = 0; i < N; ++i) {
                int o = ctx->perm[i];
                tmp.clear();
                for (int e = ctx->row_ptr[i]; e < ctx->row_ptr[i + 1]; ++e) tmp.push_back({ctx->perm[ctx->cols[e]], e});
                std::sort(tmp.begin(), tmp.end());
                int64_t base = rp[o];
                for (size_t k = 0; k < tmp.size(); ++k) {
                    if (cols) cols[base + k] = tmp[k].first;
                    if (na) na[base + k] = va[tmp[k].second];
                    if (nphi) nphi[base + k] = vp[tmp[k].second];
                    if (nk) nk[base + k] = vk[tmp[k].second];
                }
            }
        }
    } catch (const Error& e) {
        return fail(c, e);
    }
    return AIMX_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ static data files

namespace {

constexpr char kMagic[8] = {'A', 'I', 'M', 'X', 'S', 'T', 'A', 'T'};
constexpr int32_t kStaticVersion = 2;   // 2 adds the CFIE weight after sigma

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= c[i];
            h *= 1099511628211ull;
        }
    }
};

struct Writer {
    FILE* f;
    Fnv fnv;
    bool ok = true;
    void put(const void* p, size_t n) {
        if (n && std::fwrite(p, 1, n, f) != n) ok = false;
        fnv.add(p, n);
    }
    template <class T>
    void val(const T& v) { put(&v, sizeof(T)); }
    template <class T>
    void vec(const std::vector<T>& v) { put(v.data(), sizeof(T) * v.size()); }
};

struct Reader {
    FILE* f;
    Fnv fnv;
    bool ok = true;
    void get(void* p, size_t n) {
        if (n && std::fread(p, 1, n, f) != n) ok = false;
        fnv.add(p, n);
    }
    template <class T>
    T val() {
        T v{};
        get(&v, sizeof(T));
        return v;
    }
    template <class T>
    void vec(std::vector<T>& v, size_t n) {
        if (!ok || n > (size_t(1) << 36) / sizeof(T)) {
            ok = false;
            return;
        }
        v.resize(n);
        get(v.data(), sizeof(T) * n);
    }
};

template <class T>
std::vector<T> from_device(const T* d, size_t n) {
    std::vector<T> h(n);
    AIMX_CUDA_TRY(cudaMemcpy(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost));
    return h;
}

}  // namespace

extern "C" {

int aimx_save_static(const aimx_ctx* ctx, const char* path) {
    if (!ctx || !path) return AIMX_E_ARG;
    aimx_ctx* c = const_cast<aimx_ctx*>(ctx);
    try {
        const int N = ctx->N;
        const size_t nw = (size_t)N * ctx->U * 4;
        std::vector<double> xyz = from_device(ctx->d_xyz, 3 * (size_t)ctx->nv);
        std::vector<int> tri = from_device(ctx->d_tri, 3 * (size_t)ctx->nt);
        std::vector<double> w = from_device(ctx->f64.w, nw);
        std::vector<double> na = from_device(ctx->f64.na, (size_t)ctx->nnz);
        std::vector<double> np = from_device(ctx->f64.np, (size_t)ctx->nnz);
        std::vector<double> nk = from_device(ctx->f64.nk, (size_t)ctx->nnz);
        std::vector<double> diag = from_device(ctx->d_diag, 3 * (size_t)N);
        FILE* f = std::fopen(path, "wb");
        if (!f) throw Error{AIMX_E_IO, std::string("cannot open ") + path + " for writing"};
        Writer wr{f};
        wr.put(kMagic, sizeof(kMagic));
        wr.fnv = Fnv();
        wr.val(kStaticVersion);
        wr.val<int32_t>(ctx->nv);
        wr.val<int32_t>(ctx->nt);
        wr.val<int32_t>(ctx->form);
        wr.val<int32_t>(ctx->order);
        for (int a = 0; a < 3; ++a) wr.val<int32_t>(ctx->n[a]);
        wr.val<int32_t>(ctx->radius);
        wr.val<int32_t>(N);
        wr.val<int64_t>(ctx->nnz);
        wr.val(ctx->eps_out);
        wr.val(ctx->mu_out);
        wr.val(ctx->eps_in);
        wr.val(ctx->mu_in);
        wr.val(ctx->sigma);
        wr.val(ctx->cfie_alpha);
        for (int a = 0; a < 3; ++a) wr.val(ctx->h[a]);
        for (int a = 0; a < 3; ++a) wr.val(ctx->origin[a]);
        wr.vec(xyz);
        wr.vec(tri);
        wr.vec(w);
        wr.vec(na);
        wr.vec(np);
        wr.vec(nk);
        wr.vec(diag);
        const uint64_t sum = wr.fnv.h;
        if (std::fwrite(&sum, 1, sizeof(sum), f) != sizeof(sum)) wr.ok = false;
        if (std::fclose(f) != 0) wr.ok = false;
        if (!wr.ok) throw Error{AIMX_E_IO, std::string("write to ") + path + " failed"};
    } catch (const Error& e) {
        return fail(c, e);
    }
    return AIMX_OK;
}

int aimx_load_static(const char* path, aimx_ctx** out) {
    if (!path || !out) return AIMX_E_ARG;
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return AIMX_E_IO;
    Reader rd{f};
    char magic[8];
    if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kMagic, 8) != 0) {
        std::fclose(f);
        return AIMX_E_IO;
    }
    const int32_t version = rd.val<int32_t>();
    const int32_t nv = rd.val<int32_t>(), nt = rd.val<int32_t>(), form = rd.val<int32_t>(),
                  order = rd.val<int32_t>();
    aimx_grid grid{};
    for (int a = 0; a < 3; ++a) grid.n[a] = rd.val<int32_t>();
    grid.near_radius = rd.val<int32_t>();
    const int32_t N = rd.val<int32_t>();
    const int64_t nnz = rd.val<int64_t>();
    aimx_material mat{};
    mat.formulation = form;
    mat.eps_out = rd.val<double>();
    mat.mu_out = rd.val<double>();
    mat.eps_in = rd.val<double>();
    mat.mu_in = rd.val<double>();
    mat.sigma = rd.val<double>();
    if (version >= 2) mat.cfie_alpha = rd.val<double>();
    for (int a = 0; a < 3; ++a) grid.h[a] = rd.val<double>();
    for (int a = 0; a < 3; ++a) grid.origin[a] = rd.val<double>();
    std::vector<double> xyz;
    std::vector<int> tri;
    StaticData st;
    const int U = (order + 1) * (order + 1) * (order + 1);
    const bool sane = rd.ok && (version == 1 || version == kStaticVersion) && nv > 0 && nt > 0 && N > 0 && nnz > 0 && order >= 1 &&
                      order <= 3;
    if (sane) {
        rd.vec(xyz, 3 * (size_t)nv);
        rd.vec(tri, 3 * (size_t)nt);
        rd.vec(st.w, (size_t)N * U * 4);
        rd.vec(st.na, (size_t)nnz);
        rd.vec(st.np, (size_t)nnz);
        rd.vec(st.nk, (size_t)nnz);
        rd.vec(st.diag, 3 * (size_t)N);
    }
    uint64_t sum = 0;
    const bool got_sum = std::fread(&sum, 1, sizeof(sum), f) == sizeof(sum);
    std::fclose(f);
    if (!sane || !rd.ok || !got_sum || sum != rd.fnv.h) return AIMX_E_IO;
    aimx_mesh mesh{nv, nt, xyz.data(), tri.data()};
    aimx_ctx* ctx = new (std::nothrow) aimx_ctx();
    if (!ctx) return AIMX_E_NOMEM;
    try {
        setup_context(ctx, &mesh, &mat, &grid, order, &st);
        if (ctx->N != N || ctx->nnz != nnz) throw Error{AIMX_E_IO, "static data does not match the mesh"};
    } catch (const Error& e) {
        cudaDeviceSynchronize();
        cudaGetLastError();
        free_all(ctx);
        int code = e.code;
        delete ctx;
        return code;
    } catch (const std::bad_alloc&) {
        free_all(ctx);
        delete ctx;
        return AIMX_E_NOMEM;
    }
    *out = ctx;
    return AIMX_OK;
}

}  // extern "C"
