// aimx_matvec_noalloc: the FP32 plane-fused AIMx matvec with its work buffers
// in a fixed, statically allocated device array instead of memory obtained
// from cudaMalloc.
//
// Why: some callers cannot allocate device memory at the moment they need the
// product -- for example code running under an external memory budget that
// forbids new allocations once a solve has started, or code whose allocator
// is owned by another framework.  They still pass their own input and output
// buffers; everything else the product needs lives either in the context
// (created earlier by aimx_setup and a first aimx_matvec) or in the static
// array below.
//
// The array is file scope, 256-byte aligned and kNoallocScratchBytes long;
// every device that loads this library holds it until the process exits.
// In host code its name is only a stand-in, so the device address is fetched
// once per device with cudaGetSymbolAddress (on the first call made while
// that device is current) and passed to the kernels explicitly.

#include <mutex>

#include "aimx_internal.h"

namespace aimx {

constexpr size_t kNoallocScratchBytes = (size_t)64 << 20;  // 64 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
static unsigned char* g_scratch_addr[kMaxDevices] = {};
static std::mutex g_scratch_mutex;

// Device address of the static scratch on the current device (looked up once per device).
static unsigned char* scratch_address() {
    int dev = 0;
    AIMX_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) throw Error{AIMX_E_STATE, "device index out of range"};
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            throw Error{AIMX_E_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                         cudaGetErrorString(e)};
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    return g_scratch_addr[dev];
}

size_t fused_scratch_bytes(const aimx_ctx* ctx, int B);
void matvec_fused_into(aimx_ctx* ctx, double freq, int B, const float* x, float* y, cudaStream_t s,
                       unsigned char* scratch);

}  // namespace aimx

using namespace aimx;

extern "C" int aimx_matvec_noalloc(aimx_ctx* ctx, double freq, int nrhs, const void* x, void* y, void* stream) {
    if (!ctx) return AIMX_E_ARG;
    if (!x || !y || nrhs <= 0 || !(freq > 0)) {
        ctx->last_error = "aimx_matvec_noalloc: null buffer, nrhs <= 0 or freq <= 0";
        return AIMX_E_ARG;
    }
    if (!use_fused(ctx)) {
        ctx->last_error =
            "aimx_matvec_noalloc: FP32 products of this context do not take the plane-fused path "
            "(grid shape, aimx_set_path or the schedule)";
        return AIMX_E_STATE;
    }
    if (ctx->charge) {
        ctx->last_error = "aimx_matvec_noalloc: the charge form needs work buffers of its own; use aimx_matvec";
        return AIMX_E_STATE;
    }
    // The conventional-AIM near fill of a new frequency copies a host table and waits for it,
    // which would block the caller; that mode is accepted only at the frequency already filled.
    if (ctx->aim && ctx->aim_freq != freq) {
        ctx->last_error =
            "aimx_matvec_noalloc: conventional-AIM mode needs the near entries of this frequency; "
            "call aimx_matvec at it first";
        return AIMX_E_STATE;
    }
    // Everything that would otherwise be allocated lazily must already exist.
    if (!ctx->f32.spec || !ctx->f64.spec || !ctx->d_kgen || !ctx->d_plane) {
        ctx->last_error = "aimx_matvec_noalloc: call aimx_matvec once in FP32 on this context first";
        return AIMX_E_STATE;
    }
    const size_t need = fused_scratch_bytes(ctx, nrhs);
    if (need > kNoallocScratchBytes) {
        ctx->last_error = "aimx_matvec_noalloc: " + std::to_string(nrhs) + " right-hand sides need " +
                          std::to_string(need) + " bytes of scratch; the static limit is " +
                          std::to_string(kNoallocScratchBytes) + " bytes";
        return AIMX_E_ARG;
    }
    try {
        unsigned char* scratch = scratch_address();
        matvec_fused_into(ctx, freq, nrhs, static_cast<const float*>(x), static_cast<float*>(y),
                          reinterpret_cast<cudaStream_t>(stream), scratch);
    } catch (const Error& e) {
        ctx->last_error = e.msg;
        return e.code;
    }
    return AIMX_OK;
}
