// Delta-gap ports and Y-parameter sweeps (ports are cited in Sec. VI; the
// reading: a 1 V gap across the plane of the port excites <f_m, E> = l_m s_m on
// the gap edges, and the port current of coefficients x is the flux across the
// same edges, sum_m x_m l_m s_m, with s_m the sign of the RWG function's
// direction (T+ -> T-) along the port normal).

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "aimx_internal.h"
#include "cplx.cuh"

namespace aimx {

struct PortList {
    std::vector<int> ptr{0};      // [nport + 1]
    std::vector<int> id;          // caller basis ids of the gap edges
    std::vector<double> val;      // l_m s_m
};

static PortList gap_edges(const aimx_ctx* ctx, int nport, const aimx_port* ports) {
    if (ctx->form != AIMX_EFIE) throw Error{AIMX_E_STATE, "ports are defined for EFIE (conductor) contexts"};
    if (nport <= 0 || !ports) throw Error{AIMX_E_ARG, "no ports"};
    const int N = ctx->N;
    const double* xyz = ctx->h_xyz.data();
    double scale = 0.0;
    std::vector<double> len(N);
    for (int m = 0; m < N; ++m) {
        const double* a = xyz + 3 * ctx->h_ea[m];
        const double* b = xyz + 3 * ctx->h_eb[m];
        len[m] = std::sqrt((b[0] - a[0]) * (b[0] - a[0]) + (b[1] - a[1]) * (b[1] - a[1]) + (b[2] - a[2]) * (b[2] - a[2]));
        scale = std::max(scale, len[m]);
    }
    const double tol = 1e-9 * scale;
    PortList pl;
    for (int p = 0; p < nport; ++p) {
        const aimx_port& P = ports[p];
        double n[3] = {P.normal[0], P.normal[1], P.normal[2]};
        const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(nn > 0)) throw Error{AIMX_E_ARG, "port normal is zero"};
        for (double& v : n) v /= nn;
        for (int m = 0; m < N; ++m) {
            const double* a = xyz + 3 * ctx->h_ea[m];
            const double* b = xyz + 3 * ctx->h_eb[m];
            double da = 0, db = 0;
            bool inside = true;
            for (int c = 0; c < 3; ++c) {
                da += (a[c] - P.point[c]) * n[c];
                db += (b[c] - P.point[c]) * n[c];
                const double mid = 0.5 * (a[c] + b[c]);
                inside = inside && mid >= P.box_lo[c] - tol && mid <= P.box_hi[c] + tol;
            }
            if (!inside || std::fabs(da) > tol || std::fabs(db) > tol) continue;
            const double* cp = ctx->h_cen.data() + 3 * ctx->h_tp[m];
            const double* cm = ctx->h_cen.data() + 3 * ctx->h_tm[m];
            double d = 0;
            for (int c = 0; c < 3; ++c) d += (cm[c] - cp[c]) * n[c];
            const double sgn = d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0);
            pl.id.push_back(m);
            pl.val.push_back(len[m] * sgn);
        }
        if ((int)pl.id.size() == pl.ptr.back()) throw Error{AIMX_E_ARG, "port " + std::to_string(p) + " has no gap edge"};
        pl.ptr.push_back((int)pl.id.size());
    }
    return pl;
}

// b[p][id] = val (b zeroed first); one thread per gap edge
__global__ void k_port_rhs(const int* __restrict__ ptr, const int* __restrict__ id, const double* __restrict__ val,
                           int nport, int nunk, double2* b) {
    const int p = blockIdx.x;
    for (int k = ptr[p] + threadIdx.x; k < ptr[p + 1]; k += blockDim.x)
        b[(int64_t)p * nunk + id[k]] = make_double2(val[k], 0.0);
}

// I[r][p] = sum_k val_k x[r][id_k]; one block per (r, p), fixed reduction order
__global__ void k_port_currents(const int* __restrict__ ptr, const int* __restrict__ id,
                                const double* __restrict__ val, int nport, int nunk, const double2* __restrict__ x,
                                double2* I) {
    __shared__ double2 red[128];
    const int p = blockIdx.x, r = blockIdx.y;
    double2 acc = make_double2(0, 0);
    for (int k = ptr[p] + threadIdx.x; k < ptr[p + 1]; k += blockDim.x)
        acc = acc + val[k] * x[(int64_t)r * nunk + id[k]];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 64; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) I[(int64_t)r * nport + p] = red[0];
}

struct DevPorts {
    int* ptr = nullptr;
    int* id = nullptr;
    double* val = nullptr;
    aimx_ctx* ctx;
    explicit DevPorts(aimx_ctx* c, const PortList& pl) : ctx(c) {
        ptr = (int*)dev_alloc(ctx, sizeof(int) * pl.ptr.size());
        id = (int*)dev_alloc(ctx, sizeof(int) * pl.id.size());
        val = (double*)dev_alloc(ctx, sizeof(double) * pl.val.size());
        AIMX_CUDA_TRY(cudaMemcpy(ptr, pl.ptr.data(), sizeof(int) * pl.ptr.size(), cudaMemcpyHostToDevice));
        AIMX_CUDA_TRY(cudaMemcpy(id, pl.id.data(), sizeof(int) * pl.id.size(), cudaMemcpyHostToDevice));
        AIMX_CUDA_TRY(cudaMemcpy(val, pl.val.data(), sizeof(double) * pl.val.size(), cudaMemcpyHostToDevice));
    }
    ~DevPorts() {
        dev_free(ctx, ptr);
        dev_free(ctx, id);
        dev_free(ctx, val);
    }
};

static void port_rhs(aimx_ctx* ctx, const DevPorts& dp, int nport, double2* b, cudaStream_t s) {
    AIMX_CUDA_TRY(cudaMemsetAsync(b, 0, sizeof(double2) * (size_t)nport * ctx->nunk, s));
    k_port_rhs<<<nport, 128, 0, s>>>(dp.ptr, dp.id, dp.val, nport, ctx->nunk, b);
    AIMX_CUDA_TRY(cudaGetLastError());
}

}  // namespace aimx

using namespace aimx;

extern "C" {

int aimx_port_vectors(aimx_ctx* ctx, int nport, const aimx_port* ports, double* c, int32_t* nedges) {
    if (!ctx) return AIMX_E_ARG;
    try {
        PortList pl = gap_edges(ctx, nport, ports);
        if (c) std::memset(c, 0, sizeof(double) * (size_t)nport * ctx->N);
        for (int p = 0; p < nport; ++p) {
            if (nedges) nedges[p] = pl.ptr[p + 1] - pl.ptr[p];
            if (c)
                for (int k = pl.ptr[p]; k < pl.ptr[p + 1]; ++k) c[(size_t)p * ctx->N + pl.id[k]] = pl.val[k];
        }
    } catch (const Error& e) {
        ctx->last_error = e.msg;
        return e.code;
    }
    return AIMX_OK;
}

int aimx_rhs_ports(aimx_ctx* ctx, int nport, const aimx_port* ports, void* b, void* stream) {
    if (!ctx || !b) return AIMX_E_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    try {
        PortList pl = gap_edges(ctx, nport, ports);
        DevPorts dp(ctx, pl);
        port_rhs(ctx, dp, nport, (double2*)b, s);
        AIMX_CUDA_TRY(cudaStreamSynchronize(s));
    } catch (const Error& e) {
        ctx->last_error = e.msg;
        return e.code;
    }
    return AIMX_OK;
}

int aimx_port_currents(aimx_ctx* ctx, int nport, const aimx_port* ports, int nrhs, const void* x, void* I,
                       void* stream) {
    if (!ctx || !x || !I || nrhs <= 0) return AIMX_E_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    try {
        PortList pl = gap_edges(ctx, nport, ports);
        DevPorts dp(ctx, pl);
        double2* dI = (double2*)dev_alloc(ctx, sizeof(double2) * (size_t)nrhs * nport);
        k_port_currents<<<dim3(nport, nrhs), 128, 0, s>>>(dp.ptr, dp.id, dp.val, nport, ctx->nunk,
                                                          (const double2*)x, dI);
        cudaError_t e1 = cudaGetLastError();
        cudaError_t e2 = cudaMemcpyAsync(I, dI, sizeof(double2) * (size_t)nrhs * nport, cudaMemcpyDeviceToHost, s);
        cudaError_t e3 = cudaStreamSynchronize(s);
        dev_free(ctx, dI);
        AIMX_CUDA_TRY(e1);
        AIMX_CUDA_TRY(e2);
        AIMX_CUDA_TRY(e3);
    } catch (const Error& e) {
        ctx->last_error = e.msg;
        return e.code;
    }
    return AIMX_OK;
}

int aimx_sweep_ports(aimx_ctx* ctx, int nf, const double* freqs, int nport, const aimx_port* ports, void* Y,
                     const aimx_solve_opts* opts, aimx_solve_stats* stats, void* stream) {
    if (!ctx || nf <= 0 || !freqs || !Y) return AIMX_E_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int rc = AIMX_OK;
    double2* b = nullptr;
    double2* X = nullptr;
    double2* dI = nullptr;
    try {
        PortList pl = gap_edges(ctx, nport, ports);
        DevPorts dp(ctx, pl);
        const size_t nv = (size_t)nport * ctx->nunk;
        b = (double2*)dev_alloc(ctx, sizeof(double2) * nv);
        X = (double2*)dev_alloc(ctx, sizeof(double2) * nv);
        dI = (double2*)dev_alloc(ctx, sizeof(double2) * (size_t)nport * nport);
        port_rhs(ctx, dp, nport, b, s);
        aimx_solve_opts o;
        if (opts)
            o = *opts;
        else
            std::memset(&o, 0, sizeof(o));
        std::vector<double2> I((size_t)nport * nport);
        double2* Yh = static_cast<double2*>(Y);
        for (int f = 0; f < nf; ++f) {
            o.use_x0 = f > 0 ? 1 : 0;   // warm start from the previous frequency
            const int r = aimx_solve(ctx, freqs[f], nport, b, X, &o, stats ? stats + (size_t)f * nport : nullptr, stream);
            if (r < 0) throw Error{r, ctx->last_error};
            if (r > 0) rc = r;
            k_port_currents<<<dim3(nport, nport), 128, 0, s>>>(dp.ptr, dp.id, dp.val, nport, ctx->nunk, X, dI);
            AIMX_CUDA_TRY(cudaGetLastError());
            AIMX_CUDA_TRY(cudaMemcpyAsync(I.data(), dI, sizeof(double2) * I.size(), cudaMemcpyDeviceToHost, s));
            AIMX_CUDA_TRY(cudaStreamSynchronize(s));
            // I[j][i]: current at port i for 1 V at port j  ->  Y[f][i][j]
            for (int i = 0; i < nport; ++i)
                for (int j = 0; j < nport; ++j) Yh[((size_t)f * nport + i) * nport + j] = I[(size_t)j * nport + i];
        }
    } catch (const Error& e) {
        ctx->last_error = e.msg;
        rc = e.code;
    }
    if (b) dev_free(ctx, b);
    if (X) dev_free(ctx, X);
    if (dI) dev_free(ctx, dI);
    return rc;
}

}  // extern "C"
