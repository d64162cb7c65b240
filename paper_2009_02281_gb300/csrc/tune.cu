// Product-schedule autotuner: times the FP32 product of a context under each
// candidate schedule (kernel variant x right-hand sides per pass) with CUDA
// events on the caller's stream, keeps the fastest, and caches the choice in
// a text file keyed by device and problem shape so that later contexts of the
// same shape reuse it without timing.
//
// Cache line: "<key>\t<variant> <pass> <ms>", key = device name, SM count,
// grid nodes, padded sizes, fields, bases, near pairs, order, formulation and
// right-hand-side count.  Unreadable or foreign lines are skipped.

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "aimx_internal.h"

using namespace aimx;

namespace {

std::string tune_key(const aimx_ctx* ctx, int nrhs) {
    int dev = 0;
    cudaDeviceProp p{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
        cudaGetLastError();
        std::strcpy(p.name, "unknown");
    }
    std::string name(p.name);
    for (char& c : name)
        if (c == ' ' || c == '\t') c = '_';
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s sm%d n%dx%dx%d m%dx%dx%d F%d N%d nnz%lld o%d f%d b%d", name.c_str(),
                  p.multiProcessorCount, ctx->n[0], ctx->n[1], ctx->n[2], ctx->M[0], ctx->M[1], ctx->M[2], ctx->F,
                  ctx->N, (long long)ctx->nnz, ctx->order, ctx->form, nrhs);
    return buf;
}

bool cache_lookup(const char* path, const std::string& key, aimx_schedule* out) {
    if (!path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        char* tab = std::strchr(line, '\t');
        if (!tab) continue;
        *tab = 0;
        if (key != line) continue;
        aimx_schedule s{};
        if (std::sscanf(tab + 1, "%d %d %lf", &s.variant, &s.pass, &s.ms) == 3) {
            *out = s;   // the last matching line wins
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void cache_store(const char* path, const std::string& key, const aimx_schedule& s) {
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) throw Error{AIMX_E_IO, std::string("cannot append to ") + path};
    std::fprintf(f, "%s\t%d %d %.6f\n", key.c_str(), s.variant, s.pass, s.ms);
    if (std::fclose(f) != 0) throw Error{AIMX_E_IO, std::string("write to ") + path + " failed"};
}

bool schedule_valid(const aimx_ctx* ctx, const aimx_schedule& s) {
    if (s.pass < 0) return false;
    if (s.variant == 2) return true;
    if (s.variant == 1) return fused_supported(ctx);
    if (s.variant == 3) return fused_reg_supported(ctx);
    if (s.variant == 0) return true;   // register kernels where they apply, else the fused or generic default
    return false;
}

}  // namespace

extern "C" {

int aimx_set_schedule(aimx_ctx* ctx, const aimx_schedule* s) {
    if (!ctx || !s) return AIMX_E_ARG;
    if (!schedule_valid(ctx, *s)) {
        ctx->last_error = "schedule not available for this context";
        return AIMX_E_ARG;
    }
    if (ctx->sched_variant != s->variant || ctx->sched_pass != s->pass) ctx->config_gen++;
    ctx->sched_variant = s->variant;
    ctx->sched_pass = s->pass;
    return AIMX_OK;
}

int aimx_get_schedule(const aimx_ctx* ctx, aimx_schedule* s) {
    if (!ctx || !s) return AIMX_E_ARG;
    s->variant = ctx->sched_variant;
    s->pass = ctx->sched_pass;
    s->ms = 0.0;
    return AIMX_OK;
}

int aimx_autotune(aimx_ctx* ctx, double freq, int nrhs, const char* cache_path, aimx_schedule* best,
                  aimx_schedule* tried, int max_tried, int* ntried, void* stream) {
    if (!ctx || nrhs <= 0 || !(freq > 0) || (max_tried > 0 && !tried)) return AIMX_E_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (ntried) *ntried = 0;
    const std::string key = tune_key(ctx, nrhs);
    aimx_schedule pick{};
    if (cache_lookup(cache_path, key, &pick) && schedule_valid(ctx, pick)) {
        ctx->sched_variant = pick.variant;
        ctx->sched_pass = pick.pass;
        ctx->config_gen++;
        if (best) *best = pick;
        return AIMX_OK;
    }
    // candidates: kernel variants the grid allows x passes {all, 1/2, 1/4 of the RHS (>= 4)}
    std::vector<int> variants;
    if (fused_reg_supported(ctx)) variants.push_back(0);
    if (fused_reg_supported(ctx)) variants.push_back(3);
    if (fused_supported(ctx)) variants.push_back(1);
    variants.push_back(2);
    std::vector<int> passes{0};
    for (int d = 2; d <= 4; d *= 2)
        if (nrhs / d >= 4) passes.push_back(nrhs / d);
    const int keep_v = ctx->sched_variant, keep_p = ctx->sched_pass, keep_path = ctx->path;
    const bool keep_prof = ctx->prof.on;
    float2* x = nullptr;
    float2* y = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = AIMX_OK;
    try {
        const size_t bytes = sizeof(float2) * (size_t)nrhs * ctx->nunk;
        x = (float2*)dev_alloc(ctx, bytes);
        y = (float2*)dev_alloc(ctx, bytes);
        // timing is data-independent: any finite input will do (0x3c3c3c3c ~ 0.0115)
        AIMX_CUDA_TRY(cudaMemsetAsync(x, 0x3c, bytes, s));
        AIMX_CUDA_TRY(cudaEventCreate(&e0));
        AIMX_CUDA_TRY(cudaEventCreate(&e1));
        ctx->path = 0;
        ctx->prof.on = false;   // no profiling events for the trial products
        double best_ms = 1e300, default_ms = 1e300;
        int n = 0;
        for (int v : variants)
            for (int p : passes) {
                ctx->sched_variant = v;
                ctx->sched_pass = p;
                auto run = [&]() {
                    if (use_fused(ctx))
                        matvec_fused(ctx, freq, nrhs, (const float*)x, (float*)y, s);
                    else
                        matvec_generic<float>(ctx, freq, nrhs, (const float*)x, (float*)y, s);
                };
                run();   // first call: buffers, tables and spectra
                run();
                constexpr int reps = 3;
                AIMX_CUDA_TRY(cudaEventRecord(e0, s));
                for (int r = 0; r < reps; ++r) run();
                AIMX_CUDA_TRY(cudaEventRecord(e1, s));
                AIMX_CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.f;
                AIMX_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                aimx_schedule c{v, p, ms / reps};
                if (v == variants[0] && p == 0) default_ms = c.ms;
                if (n < max_tried) tried[n] = c;
                ++n;
                if (c.ms < best_ms) {
                    best_ms = c.ms;
                    pick = c;
                }
            }
        // keep the default schedule (first variant, all RHS per pass) unless another candidate
        // is more than 5% faster: the timings of near-equal candidates are within noise
        if (n > 0 && (pick.variant != variants[0] || pick.pass != 0) && pick.ms > 0.95 * default_ms) {
            pick.variant = variants[0];
            pick.pass = 0;
            pick.ms = default_ms;
        }
        if (ntried) *ntried = n;
        cache_store(cache_path, key, pick);
    } catch (const Error& e) {
        ctx->last_error = e.msg;
        rc = e.code;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (x) dev_free(ctx, x);
    if (y) dev_free(ctx, y);
    ctx->path = keep_path;
    ctx->prof.on = keep_prof;
    if (rc != AIMX_OK) {
        ctx->sched_variant = keep_v;
        ctx->sched_pass = keep_p;
        return rc;
    }
    ctx->sched_variant = pick.variant;
    ctx->sched_pass = pick.pass;
    ctx->config_gen++;
    if (best) *best = pick;
    return AIMX_OK;
}

}  // extern "C"
