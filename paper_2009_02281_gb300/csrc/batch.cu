// Batches of uneven meshes: one call applies the FP32 AIMx product of every
// member context (each its own mesh, grid, formulation, frequency and RHS
// count).  Members run concurrently on a small set of internal streams, and
// the whole batch is captured once into a CUDA graph that is replayed while
// the members' frequencies, RHS counts and buffer pointers stay the same, so a
// batch of small meshes costs one graph launch instead of ~7 kernel launches
// and host round trips per mesh.

#include <algorithm>
#include <thread>
#include <vector>

#include "aimx_internal.h"

using namespace aimx;

struct aimx_batch {
    std::vector<aimx_ctx*> ctx;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;   // one per internal stream
    cudaStream_t cap = nullptr;      // capture origin (the caller's stream may be the legacy default stream)
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // signature of the captured graph
    std::vector<double> freq;
    std::vector<int> nrhs;
    std::vector<const void*> x;
    std::vector<void*> y;
    std::vector<int> gen;            // members' config_gen at capture
    size_t nodes = 0;
    std::string last_error;
};

namespace {

void member_matvec(aimx_ctx* c, double freq, int nrhs, const void* x, void* y, cudaStream_t s) {
    if (use_fused(c))
        matvec_fused(c, freq, nrhs, static_cast<const float*>(x), static_cast<float*>(y), s);
    else
        matvec_generic<float>(c, freq, nrhs, static_cast<const float*>(x), static_cast<float*>(y), s);
}

void release_graph(aimx_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->nodes = 0;
}

bool same_signature(const aimx_batch* b, const double* freqs, const int* nrhs, const void* const* x,
                    void* const* y) {
    if (!b->exec) return false;
    for (size_t i = 0; i < b->ctx.size(); ++i)
        if (b->freq[i] != freqs[i] || b->nrhs[i] != nrhs[i] || b->x[i] != x[i] || b->y[i] != y[i] ||
            b->gen[i] != b->ctx[i]->config_gen)
            return false;
    return true;
}

// Run every member once outside any capture (creates spectra and work buffers),
// then capture all members into one graph from the batch's own capture stream.
void capture(aimx_batch* b, const double* freqs, const int* nrhs, const void* const* x, void* const* y,
             cudaStream_t caller) {
    release_graph(b);
    const size_t n = b->ctx.size();
    for (size_t i = 0; i < n; ++i) member_matvec(b->ctx[i], freqs[i], nrhs[i], x[i], y[i], caller);
    AIMX_CUDA_TRY(cudaStreamSynchronize(caller));
    cudaStream_t s = b->cap;
    std::vector<bool> prof(n);
    for (size_t i = 0; i < n; ++i) {
        prof[i] = b->ctx[i]->prof.on;
        b->ctx[i]->prof.on = false;   // no profiling events inside the graph
    }
    cudaGraph_t g = nullptr;
    cudaError_t err = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
    if (err == cudaSuccess) {
        try {
            AIMX_CUDA_TRY(cudaEventRecord(b->fork, s));
            for (cudaStream_t t : b->streams) AIMX_CUDA_TRY(cudaStreamWaitEvent(t, b->fork, 0));
            for (size_t i = 0; i < n; ++i)
                member_matvec(b->ctx[i], freqs[i], nrhs[i], x[i], y[i], b->streams[i % b->streams.size()]);
            for (size_t k = 0; k < b->streams.size(); ++k) {
                AIMX_CUDA_TRY(cudaEventRecord(b->done[k], b->streams[k]));
                AIMX_CUDA_TRY(cudaStreamWaitEvent(s, b->done[k], 0));
            }
        } catch (const Error&) {
            cudaStreamEndCapture(s, &g);
            if (g) cudaGraphDestroy(g);
            for (size_t i = 0; i < n; ++i) b->ctx[i]->prof.on = prof[i];
            cudaGetLastError();
            throw;
        }
        err = cudaStreamEndCapture(s, &g);
    }
    for (size_t i = 0; i < n; ++i) b->ctx[i]->prof.on = prof[i];
    if (err != cudaSuccess || !g) {
        cudaGetLastError();
        throw Error{AIMX_E_CUDA, std::string("batch graph capture failed: ") + cudaGetErrorString(err)};
    }
    b->graph = g;
    AIMX_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &b->nodes));
    AIMX_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
    b->freq.assign(freqs, freqs + n);
    b->nrhs.assign(nrhs, nrhs + n);
    b->x.assign(x, x + n);
    b->y.assign(y, y + n);
    b->gen.resize(n);
    for (size_t i = 0; i < n; ++i) b->gen[i] = b->ctx[i]->config_gen;
}

}  // namespace

extern "C" {

int aimx_batch_create(int n, aimx_ctx* const* ctxs, int nstreams, aimx_batch** out) {
    if (!out) return AIMX_E_ARG;
    *out = nullptr;
    if (n <= 0 || !ctxs) return AIMX_E_ARG;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return AIMX_E_ARG;
    aimx_batch* b = new (std::nothrow) aimx_batch();
    if (!b) return AIMX_E_NOMEM;
    b->ctx.assign(ctxs, ctxs + n);
    const int k = std::max(1, std::min(nstreams > 0 ? nstreams : 8, n));
    bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; ok && i < k; ++i) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (s) b->streams.push_back(s);
        if (e) b->done.push_back(e);
    }
    if (!ok) {
        cudaGetLastError();
        for (auto s : b->streams) cudaStreamDestroy(s);
        for (auto e : b->done) cudaEventDestroy(e);
        if (b->fork) cudaEventDestroy(b->fork);
        if (b->cap) cudaStreamDestroy(b->cap);
        delete b;
        return AIMX_E_CUDA;
    }
    *out = b;
    return AIMX_OK;
}

int aimx_batch_destroy(aimx_batch* b) {
    if (!b) return AIMX_OK;
    for (auto s : b->streams) cudaStreamSynchronize(s);
    release_graph(b);
    for (auto s : b->streams) cudaStreamDestroy(s);
    for (auto e : b->done) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) {
        cudaStreamSynchronize(b->cap);
        cudaStreamDestroy(b->cap);
    }
    delete b;
    return AIMX_OK;
}

int aimx_batch_matvec(aimx_batch* b, const double* freqs, const int* nrhs, const void* const* x, void* const* y,
                      void* stream) {
    if (!b || !freqs || !nrhs || !x || !y) return AIMX_E_ARG;
    for (size_t i = 0; i < b->ctx.size(); ++i)
        if (!(freqs[i] > 0) || nrhs[i] <= 0 || !x[i] || !y[i]) {
            b->last_error = "aimx_batch_matvec: bad member argument " + std::to_string(i);
            return AIMX_E_ARG;
        }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    try {
        if (!same_signature(b, freqs, nrhs, x, y)) capture(b, freqs, nrhs, x, y, s);
        AIMX_CUDA_TRY(cudaGraphLaunch(b->exec, s));
    } catch (const Error& e) {
        b->last_error = e.msg;
        return e.code;
    }
    return AIMX_OK;
}

// Solve every member's systems: member i on internal stream i % k, driven by host thread i % k
// (aimx_solve synchronises its stream at every Arnoldi step, so one thread per stream lets the
// members' GPU work overlap).  The work is ordered after `stream`, and `stream` after it.
int aimx_batch_solve(aimx_batch* b, const double* freqs, const int* nrhs, const void* const* B, void* const* X,
                     const aimx_solve_opts* opts, aimx_solve_stats* const* stats, void* stream) {
    if (!b || !freqs || !nrhs || !B || !X) return AIMX_E_ARG;
    const int n = (int)b->ctx.size();
    for (int i = 0; i < n; ++i)
        if (!(freqs[i] > 0) || nrhs[i] <= 0 || !B[i] || !X[i]) {
            b->last_error = "aimx_batch_solve: bad member argument " + std::to_string(i);
            return AIMX_E_ARG;
        }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaEventRecord(b->fork, s) != cudaSuccess) {
        cudaGetLastError();
        b->last_error = "aimx_batch_solve: could not order the batch after the caller's stream";
        return AIMX_E_CUDA;
    }
    const int k = (int)b->streams.size();
    for (int t = 0; t < k; ++t) cudaStreamWaitEvent(b->streams[t], b->fork, 0);
    std::vector<int> rc(n, AIMX_OK);
    auto work = [&](int t) {
        cudaSetDevice(dev);
        for (int i = t; i < n; i += k)
            rc[i] = aimx_solve(b->ctx[i], freqs[i], nrhs[i], B[i], X[i], opts, stats ? stats[i] : nullptr,
                               b->streams[t]);
    };
    std::vector<std::thread> th;
    for (int t = 1; t < k; ++t) th.emplace_back(work, t);
    work(0);
    for (auto& x : th) x.join();
    int worst = AIMX_OK;
    for (int i = 0; i < n; ++i) {
        if (rc[i] < 0 && worst >= 0) {
            worst = rc[i];
            b->last_error = "member " + std::to_string(i) + ": " + aimx_last_error(b->ctx[i]);
        } else if (rc[i] > 0 && worst == AIMX_OK) {
            worst = rc[i];
        }
    }
    for (int t = 0; t < k; ++t) {
        cudaEventRecord(b->done[t], b->streams[t]);
        cudaStreamWaitEvent(s, b->done[t], 0);
    }
    return worst;
}

int64_t aimx_batch_graph_nodes(const aimx_batch* b) { return b ? (int64_t)b->nodes : 0; }

const char* aimx_batch_last_error(const aimx_batch* b) { return b ? b->last_error.c_str() : ""; }

}  // extern "C"
