// Generic power-of-two 3-D FFT on padded grids (radix-2, shared-memory tiles)
// and the per-frequency generation of the grid-kernel spectra.
//
// The convolution matrix H(k) is 3-level Toeplitz (Eq. Hmn, Sec. III-A-1);
// its first row, sampled at the grid offsets d with the AIMx self term
// H(0) = -jk/(4 pi) (Eq. Hmm), is embedded in a circulant of the padded size
// M >= 2n - 1 per axis (offset d -> index d mod M, unused slots zero) and
// transformed once per frequency in FP64.  Only the octant 0..M/2 of each
// spectrum is stored: the scalar kernel is even in every axis, the gradient
// component along axis a is odd in that axis and even in the others.

#include <cmath>
#include <mutex>

#include "aimx_internal.h"
#include "cplx.cuh"
#include "regfft.cuh"

namespace aimx {

// ------------------------------------------------------------------ twiddles

// one table pair per device: a context on another device must not be handed
// this device's pointers
constexpr int kTwMaxDevices = 64;
static double2* g_tw64[kTwMaxDevices] = {};
static float2* g_tw32[kTwMaxDevices] = {};
static std::mutex g_tw_mutex;

static int tw_device() {
    int dev = 0;
    AIMX_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kTwMaxDevices) throw Error{AIMX_E_STATE, "device index out of range"};
    return dev;
}

static void init_twiddles(int dev) {
    std::lock_guard<std::mutex> lock(g_tw_mutex);
    if (g_tw64[dev]) return;
    const int H = kTwiddleTab;   // full circle: e^{-2 pi i k / 12288}, k < 12288
    std::vector<double2> t64(H);
    std::vector<float2> t32(H);
    for (int k = 0; k < H; ++k) {
        double a = -2.0 * kPi * (double)k / (double)kTwiddleTab;
        t64[k] = make_double2(std::cos(a), std::sin(a));
        t32[k] = make_float2((float)t64[k].x, (float)t64[k].y);
    }
    double2* d64;
    float2* d32;
    AIMX_CUDA_TRY(cudaMalloc(&d64, H * sizeof(double2)));
    AIMX_CUDA_TRY(cudaMalloc(&d32, H * sizeof(float2)));
    AIMX_CUDA_TRY(cudaMemcpy(d64, t64.data(), H * sizeof(double2), cudaMemcpyHostToDevice));
    AIMX_CUDA_TRY(cudaMemcpy(d32, t32.data(), H * sizeof(float2), cudaMemcpyHostToDevice));
    g_tw32[dev] = d32;
    g_tw64[dev] = d64;
}

const double2* twiddles64() {
    const int dev = tw_device();
    if (!g_tw64[dev]) init_twiddles(dev);
    return g_tw64[dev];
}
const float2* twiddles32() {
    const int dev = tw_device();
    if (!g_tw64[dev]) init_twiddles(dev);
    return g_tw32[dev];
}

template <class T>
static const cplx_t<T>* twiddles();
template <>
const float2* twiddles<float>() {
    return twiddles32();
}
template <>
const double2* twiddles<double>() {
    return twiddles64();
}

// ------------------------------------------------------------------ FFT on smem lines, lengths 2^k and 3 * 2^k

__device__ inline int bitrev(int v, int bits) { return (int)(__brev((unsigned)v) >> (32 - bits)); }

// Slot of input p in a shared-memory line before the in-place passes.  Length 2^k: bit-reversed
// (decimation in time).  Length L = 3 P: the three decimated sequences x[3 n + r] are placed in
// blocks r of P, each bit-reversed within its block.
__device__ inline int fft_load_pos(int p, int L, int logP, int r3) {
    if (!r3) return bitrev(p, logP);
    return (p % 3) * (L / 3) + bitrev(p / 3, logP);
}

// In-place FFT of nl lines (pitch elements apart) loaded by fft_load_pos: radix-2
// decimation-in-time passes over each block of P = 2^logP, then for L = 3 P one radix-3 pass
// X[k + m P] = sum_r W_L^{r k} W_3^{r m} Y_r[k].  inv selects e^{+j..} twiddles.  tw: the
// kTwiddleTab-point table e^{-2 pi i k / kTwiddleTab}.
template <class C>
__device__ void smem_fft_lines(C* s, int nl, int pitch, int L, int logP, int r3, bool inv, const C* tw) {
    const int P = r3 ? L / 3 : L, nsub = r3 ? 3 : 1;
    const int halfP = P >> 1;
    for (int st = 1; st <= logP; ++st) {
        const int half = 1 << (st - 1);
        const int tstep = kTwiddleTab / (2 * half);
        for (int idx = threadIdx.x; idx < nl * nsub * halfP; idx += blockDim.x) {
            const int l = idx / (nsub * halfP), rem = idx - l * (nsub * halfP);
            const int r = rem / halfP, j = rem - r * halfP;
            const int pos = j & (half - 1);
            const int i0 = ((j >> (st - 1)) << st) + pos;
            const int i1 = i0 + half;
            C w = tw[pos * tstep];
            if (inv) w = conj(w);
            C* line = s + l * pitch + r * P;
            C b = w * line[i1];
            C a = line[i0];
            line[i0] = a + b;
            line[i1] = a - b;
        }
        __syncthreads();
    }
    if (r3) {
        using R = decltype(C{}.x);
        const R hs = (R)0.86602540378443864676;   // sqrt(3) / 2
        const int step = kTwiddleTab / L;
        for (int idx = threadIdx.x; idx < nl * P; idx += blockDim.x) {
            const int l = idx / P, k = idx - l * P;
            C* line = s + l * pitch;
            C w1 = tw[k * step], w2 = tw[2 * k * step];
            if (inv) {
                w1 = conj(w1);
                w2 = conj(w2);
            }
            const C a = line[k], b = w1 * line[k + P], c = w2 * line[k + 2 * P];
            const C t = b + c, d = b - c;
            const C m = a - (R)0.5 * t;
            // forward: X1 = m - i hs d, X2 = m + i hs d (omega = e^{-2 pi i / 3}); inverse: conjugate
            const C jd = inv ? mk(-hs * d.y, hs * d.x) : mk(hs * d.y, -hs * d.x);
            line[k] = a + t;
            line[k + P] = m + jd;
            line[k + 2 * P] = m - jd;
        }
        __syncthreads();
    }
}

// Lines that are contiguous rows: row r at base + a*S1 + b*S2 + c*S3 with
// r = (a*D1 + b)*D2 + c.  RPB rows per block.
template <class T>
__global__ void k_fft_rows(cplx_t<T>* base, int64_t nrows, int D1, int D2, int64_t S1, int64_t S2,
                           int64_t S3, int L, int logP, int r3, int RPB, int inv, const cplx_t<T>* tw) {
    using C = cplx_t<T>;
    extern __shared__ unsigned char smraw[];
    C* s = reinterpret_cast<C*>(smraw);
    const int pitch = L + 1;
    int64_t r0 = (int64_t)blockIdx.x * RPB;
    int64_t rem = nrows - r0;
    int nl = rem < RPB ? (int)rem : RPB;
    for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
        int rr = idx / L, p = idx - rr * L;
        int64_t r = r0 + rr;
        int64_t c = r % D2, b = (r / D2) % D1, a = r / ((int64_t)D1 * D2);
        s[rr * pitch + fft_load_pos(p, L, logP, r3)] = base[a * S1 + b * S2 + c * S3 + p];
    }
    __syncthreads();
    smem_fft_lines<C>(s, nl, pitch, L, logP, r3, inv != 0, tw);
    for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
        int rr = idx / L, p = idx - rr * L;
        int64_t r = r0 + rr;
        int64_t c = r % D2, b = (r / D2) % D1, a = r / ((int64_t)D1 * D2);
        base[a * S1 + b * S2 + c * S3 + p] = s[rr * pitch + p];
    }
}

// Strided lines: line (o, x) starts at base + (o / D1)*S1 + (o % D1)*S2 + x and
// its points are S apart; each block takes TC consecutive x of one o.
template <class T>
__global__ void k_fft_cols(cplx_t<T>* base, int64_t nouter, int D1, int64_t S1, int64_t S2, int64_t S,
                           int Mx, int L, int logP, int r3, int TC, int inv, const cplx_t<T>* tw) {
    using C = cplx_t<T>;
    extern __shared__ unsigned char smraw[];
    C* s = reinterpret_cast<C*>(smraw);
    const int pitch = L + 1;
    int ntiles = (Mx + TC - 1) / TC;
    int64_t o = blockIdx.x / ntiles;
    int x0 = (blockIdx.x % ntiles) * TC;
    int nl = min(TC, Mx - x0);
    C* lb = base + (o / D1) * S1 + (o % D1) * S2 + x0;
    for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
        int p = idx / nl, c = idx - p * nl;
        s[c * pitch + fft_load_pos(p, L, logP, r3)] = lb[(int64_t)p * S + c];
    }
    __syncthreads();
    smem_fft_lines<C>(s, nl, pitch, L, logP, r3, inv != 0, tw);
    for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
        int p = idx / nl, c = idx - p * nl;
        lb[(int64_t)p * S + c] = s[c * pitch + p];
    }
}

// ------------------------------------------------------------------ register-line FFTs
//
// One thread holds one whole line of compile-time length L in registers (reg_fft_any:
// radix 4/2 and one radix-3 pass, twiddles as instruction immediates).  Only the first nin
// inputs are read (the rest is the zero padding) and only the first nout outputs are written
// (the pruned inverse).  Lengths without a register kernel take the shared-memory kernels
// above, which read and write whole lines.

// Strided lines as in k_fft_cols; consecutive threads take consecutive x (coalesced).
template <class C, int L, bool INV>
__global__ void __launch_bounds__(128) k_fft_cols_reg(C* base, int64_t nlines, int D1, int64_t S1, int64_t S2,
                                                      int64_t S, int Mx, int nin, int nout) {
    using R = decltype(C{}.x);
    const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    const int64_t o = line / Mx;
    const int x = (int)(line - o * Mx);
    C* lb = base + (o / D1) * S1 + (o % D1) * S2 + x;
    // L <= 64 and padded sides <= 4096, so a line spans L S < 2^31 elements: 32-bit point offsets
    const int s32 = (int)S;
    C v[L];
#pragma unroll
    for (int p = 0; p < L; ++p) v[p] = p < nin ? lb[p * s32] : mk(R(0), R(0));
    reg_fft_any<C, L, INV>(v);
#pragma unroll
    for (int p = 0; p < L; ++p)
        if (p < nout) lb[p * s32] = v[p];
}

// Contiguous rows as in k_fft_rows, kRowsReg rows per block staged through shared memory
// (coalesced row loads and stores), one row per thread in registers.
constexpr int kRowsReg = 64;

template <class C, int L, bool INV>
__global__ void __launch_bounds__(kRowsReg) k_fft_rows_reg(C* base, int64_t nrows, int D1, int D2, int64_t S1,
                                                           int64_t S2, int64_t S3, int nin, int nout) {
    using R = decltype(C{}.x);
    constexpr int PITCH = L + 1;
    extern __shared__ unsigned char smraw[];
    __shared__ C* rowp[kRowsReg];
    C* t = reinterpret_cast<C*>(smraw);
    const int64_t r0 = (int64_t)blockIdx.x * kRowsReg;
    const int nl = (int)min((int64_t)kRowsReg, nrows - r0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = kRowsReg / 32;
    if ((int)threadIdx.x < nl) {   // row start of row threadIdx.x (64-bit index arithmetic once per row)
        const int64_t r = r0 + threadIdx.x;
        const int64_t c = r % D2, b = (r / D2) % D1, a = r / ((int64_t)D1 * D2);
        rowp[threadIdx.x] = base + a * S1 + b * S2 + c * S3;
    }
    __syncthreads();
    // each warp copies whole rows, its lanes on consecutive points
    for (int rr = warp; rr < nl; rr += NW) {
        const C* src = rowp[rr];
        for (int p = lane; p < nin; p += 32) t[rr * PITCH + p] = src[p];
    }
    __syncthreads();
    if ((int)threadIdx.x < nl) {
        C v[L];
#pragma unroll
        for (int p = 0; p < L; ++p) v[p] = p < nin ? t[threadIdx.x * PITCH + p] : mk(R(0), R(0));
        reg_fft_any<C, L, INV>(v);
#pragma unroll
        for (int p = 0; p < L; ++p)
            if (p < nout) t[threadIdx.x * PITCH + p] = v[p];
    }
    __syncthreads();
    for (int rr = warp; rr < nl; rr += NW) {
        C* dst = rowp[rr];
        for (int p = lane; p < nout; p += 32) dst[p] = t[rr * PITCH + p];
    }
}

template <class C, int L, bool INV>
static void launch_cols_reg(C* g, int64_t nouter, int D1, int64_t S1, int64_t S2, int64_t S, int Mx, int nin,
                            int nout, cudaStream_t s) {
    const int64_t nlines = nouter * Mx;
    k_fft_cols_reg<C, L, INV><<<(unsigned)((nlines + 127) / 128), 128, 0, s>>>(g, nlines, D1, S1, S2, S, Mx, nin,
                                                                               nout);
}

template <class C, int L, bool INV>
static void launch_rows_reg(C* g, int64_t nrows, int D1, int D2, int64_t S1, int64_t S2, int64_t S3, int nin,
                            int nout, cudaStream_t s) {
    const size_t sm = (size_t)kRowsReg * (L + 1) * sizeof(C);
    static bool attr[64] = {};   // per device: the dynamic shared-memory opt-in of this instantiation
    int dev = 0;
    AIMX_CUDA_TRY(cudaGetDevice(&dev));
    if (sm > 48 * 1024 && dev < 64 && !attr[dev]) {
        AIMX_CUDA_TRY(cudaFuncSetAttribute(k_fft_rows_reg<C, L, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sm));
        attr[dev] = true;
    }
    k_fft_rows_reg<C, L, INV><<<(unsigned)((nrows + kRowsReg - 1) / kRowsReg), kRowsReg, sm, s>>>(
        g, nrows, D1, D2, S1, S2, S3, nin, nout);
}

// launch arguments of the register-line kernels, dispatched on the compile-time length
template <class C>
struct RowsRun {
    C* g;
    int64_t nrows;
    int D1, D2;
    int64_t S1, S2, S3;
    int nin, nout;
    bool inv;
    cudaStream_t s;
    template <int LL>
    void run() {
        if (inv)
            launch_rows_reg<C, LL, true>(g, nrows, D1, D2, S1, S2, S3, nin, nout, s);
        else
            launch_rows_reg<C, LL, false>(g, nrows, D1, D2, S1, S2, S3, nin, nout, s);
    }
};
template <class C>
struct ColsRun {
    C* g;
    int64_t nouter;
    int D1;
    int64_t S1, S2, S;
    int Mx, nin, nout;
    bool inv;
    cudaStream_t s;
    template <int LL>
    void run() {
        if (inv)
            launch_cols_reg<C, LL, true>(g, nouter, D1, S1, S2, S, Mx, nin, nout, s);
        else
            launch_cols_reg<C, LL, false>(g, nouter, D1, S1, S2, S, Mx, nin, nout, s);
    }
};

// Calls f.template run<L>() for the register-line lengths of this precision; false if L has none.
template <class C, class F>
static bool reg_length_dispatch(int L, F&& f) {
    // FP32 lines up to 64 points, FP64 lines up to 48 (a line's values take at most 192 of the
    // 255 registers a thread can hold)
    constexpr bool sp = sizeof(C) == sizeof(float2);
    switch (L) {
        case 16: f.template run<16>(); return true;
        case 24: f.template run<24>(); return true;
        case 32: f.template run<32>(); return true;
        case 48: f.template run<48>(); return true;
        case 64:
            if (!sp) return false;
            f.template run<sp ? 64 : 16>();
            return true;
        default: return false;
    }
}

// (log2 P, 1) for L = 3 * 2^logP, (log2 L, 0) for L = 2^logP
static void fft_factors(int L, int& logP, int& r3) {
    r3 = (L % 3 == 0) ? 1 : 0;
    int P = r3 ? L / 3 : L;
    logP = 0;
    while ((1 << logP) < P) ++logP;
    if ((1 << logP) != P) throw Error{AIMX_E_ARG, "FFT length must be 2^k or 3 * 2^k"};
}

template <class T>
static void fft_rows(cplx_t<T>* g, int64_t nrows, int D1, int D2, int64_t S1, int64_t S2, int64_t S3,
                     int L, bool inv, cudaStream_t s, int nin = -1, int nout = -1, bool reg = false) {
    if (nrows <= 0) return;
    using C = cplx_t<T>;
    nin = nin < 0 ? L : nin;
    nout = nout < 0 ? L : nout;
    RowsRun<C> run{g, nrows, D1, D2, S1, S2, S3, nin, nout, inv, s};
    if (reg && reg_length_dispatch<C>(L, run)) {
        AIMX_CUDA_TRY(cudaGetLastError());
        return;
    }
    int RPB = std::max(1, 8192 / L);
    size_t sm = (size_t)RPB * (L + 1) * sizeof(cplx_t<T>);
    if (sm > 48 * 1024) {
        RPB = std::max(1, (int)((48 * 1024) / ((L + 1) * sizeof(cplx_t<T>))));
        sm = (size_t)RPB * (L + 1) * sizeof(cplx_t<T>);
    }
    unsigned nb = (unsigned)((nrows + RPB - 1) / RPB);
    int logP, r3;
    fft_factors(L, logP, r3);
    k_fft_rows<T><<<nb, 256, sm, s>>>(g, nrows, D1, D2, S1, S2, S3, L, logP, r3, RPB, inv ? 1 : 0,
                                      twiddles<T>());
    AIMX_CUDA_TRY(cudaGetLastError());
}

template <class T>
static void fft_cols(cplx_t<T>* g, int64_t nouter, int D1, int64_t S1, int64_t S2, int64_t S, int Mx,
                     int L, bool inv, cudaStream_t s, int nin = -1, int nout = -1, bool reg = false) {
    if (nouter <= 0) return;
    using C = cplx_t<T>;
    nin = nin < 0 ? L : nin;
    nout = nout < 0 ? L : nout;
    ColsRun<C> run{g, nouter, D1, S1, S2, S, Mx, nin, nout, inv, s};
    if (reg && reg_length_dispatch<C>(L, run)) {
        AIMX_CUDA_TRY(cudaGetLastError());
        return;
    }
    int TC = sizeof(T) == 4 ? 32 : 16;
    TC = std::min(TC, Mx);
    while ((size_t)TC * (L + 1) * sizeof(cplx_t<T>) > 48 * 1024 && TC > 1) TC >>= 1;
    size_t sm = (size_t)TC * (L + 1) * sizeof(cplx_t<T>);
    int ntiles = (Mx + TC - 1) / TC;
    unsigned nb = (unsigned)(nouter * ntiles);
    int logP, r3;
    fft_factors(L, logP, r3);
    k_fft_cols<T><<<nb, 256, sm, s>>>(g, nouter, D1, S1, S2, S, Mx, L, logP, r3, TC, inv ? 1 : 0,
                                      twiddles<T>());
    AIMX_CUDA_TRY(cudaGetLastError());
}

// 3-D transform of `batch` padded grids [batch][Mz][My][Mx] whose non-zero
// input (forward) or needed output (inverse) lies in z < act[2], y < act[1]:
// forward = x rows (y < act1, z < act2), y columns (z < act2), z columns (all);
// inverse runs the same passes in reverse order.
template <class T>
void fft3d_padded(T* grid, int batch, const int M[3], const int act[3], bool inverse, cudaStream_t s) {
    using C = cplx_t<T>;
    C* g = reinterpret_cast<C*>(grid);
    const int64_t Mx = M[0], My = M[1], Mz = M[2];
    const int64_t SB = Mx * My * Mz;
    // forward passes read only the non-zero inputs (first act), inverse passes write only the
    // outputs later passes and the interpolation read (first act); register-line kernels use this
    auto in = [&](int a) { return inverse ? M[a] : act[a]; };
    auto out = [&](int a) { return inverse ? act[a] : M[a]; };
    const bool reg = fft3d_reads_active_only<T>(M, batch);   // all passes on register lines, or none
    auto xpass = [&]() {
        fft_rows<T>(g, (int64_t)batch * act[2] * act[1], act[2], act[1], SB, My * Mx, Mx, M[0], inverse, s, in(0),
                    out(0), reg);
    };
    auto ypass = [&]() {
        fft_cols<T>(g, (int64_t)batch * act[2], act[2], SB, My * Mx, Mx, M[0], M[1], inverse, s, in(1), out(1),
                    reg);
    };
    auto zpass = [&]() {
        fft_cols<T>(g, (int64_t)batch * My, (int)My, SB, Mx, My * Mx, M[0], M[2], inverse, s, in(2), out(2), reg);
    };
    if (!inverse) {
        xpass();
        ypass();
        zpass();
    } else {
        zpass();
        ypass();
        xpass();
    }
}

template <class T>
void fft3d_full(T* grid, int batch, const int M[3], bool inverse, cudaStream_t s) {
    int act[3] = {M[0], M[1], M[2]};
    fft3d_padded<T>(grid, batch, M, act, inverse, s);
}

// True when every pass of fft3d_padded runs on register lines for this precision: the forward
// transform then reads only the active input region, so the padding needs no zeroing.
struct LenProbe {
    template <int LL>
    void run() {}
};
// Every pass of a batch of `batch` grids on register lines: all three lengths have register
// kernels and, in FP64 (up to 222 registers a thread), the z pass has lines enough to fill the
// GPU at two blocks per SM; smaller FP64 batches keep the shared-memory kernels.
constexpr int64_t kMinRegLinesF64 = 32768;
template <class T>
bool fft3d_reads_active_only(const int M[3], int batch) {
    LenProbe probe;
    for (int a = 0; a < 3; ++a)
        if (!reg_length_dispatch<cplx_t<T>>(M[a], probe)) return false;
    return sizeof(T) == sizeof(float) || (int64_t)batch * M[0] * M[1] >= kMinRegLinesF64;
}
template bool fft3d_reads_active_only<float>(const int*, int);
template bool fft3d_reads_active_only<double>(const int*, int);

template void fft3d_padded<float>(float*, int, const int*, const int*, bool, cudaStream_t);
template void fft3d_padded<double>(double*, int, const int*, const int*, bool, cudaStream_t);
template void fft3d_full<float>(float*, int, const int*, bool, cudaStream_t);
template void fft3d_full<double>(double*, int, const int*, bool, cudaStream_t);

// ------------------------------------------------------------------ kernel generation

struct Region {
    double k;       // wavenumber
    double gscale;  // multiplier of this region's gradient samples in V (eta0 for PMCHWT)
};

// Circulant samples: scalar G per region (arrays 0..nreg-1) and, for the
// K operator, V_a = sum_reg eta0 * d_a G_reg (arrays nreg..nreg+2).
__global__ void k_sample(double2* out, int nreg, int want_grad, Region r0, Region r1, int Mx, int My,
                         int Mz, int nx, int ny, int nz, double hx, double hy, double hz) {
    int64_t MT = (int64_t)Mx * My * Mz;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= MT) return;
    int ix = (int)(t % Mx), iy = (int)((t / Mx) % My), iz = (int)(t / ((int64_t)Mx * My));
    auto off = [](int i, int M, int n, bool& gap) {
        if (i <= n - 1) return i;
        if (i >= M - n + 1) return i - M;
        gap = true;
        return 0;
    };
    bool gap = false;
    int dx = off(ix, Mx, nx, gap), dy = off(iy, My, ny, gap), dz = off(iz, Mz, nz, gap);
    int nout = nreg + (want_grad ? 3 : 0);
    if (gap) {
        for (int a = 0; a < nout; ++a) out[a * MT + t] = make_double2(0.0, 0.0);
        return;
    }
    double rx = dx * hx, ry = dy * hy, rz = dz * hz;
    double r = sqrt(rx * rx + ry * ry + rz * rz);
    bool self = (dx == 0 && dy == 0 && dz == 0);
    double2 V[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    for (int g = 0; g < nreg; ++g) {
        Region R = g == 0 ? r0 : r1;
        double2 H;
        if (self) {
            H = make_double2(0.0, -R.k / (4.0 * kPi));   // Eq. Hmm
        } else {
            double s_, c_;
            sincos(R.k * r, &s_, &c_);
            double inv = 1.0 / (4.0 * kPi * r);
            H = make_double2(c_ * inv, -s_ * inv);        // e^{-jkr} / (4 pi r)
            if (want_grad) {
                // grad G = -(1 + jkr) e^{-jkr} / (4 pi r^3) * r_vec
                double inv3 = -1.0 / (4.0 * kPi * r * r * r);
                double2 f = make_double2((c_ + R.k * r * s_) * inv3, (R.k * r * c_ - s_) * inv3);
                V[0] = V[0] + (R.gscale * rx) * f;
                V[1] = V[1] + (R.gscale * ry) * f;
                V[2] = V[2] + (R.gscale * rz) * f;
            }
        }
        out[g * MT + t] = H;
    }
    if (want_grad)
        for (int a = 0; a < 3; ++a) out[(nreg + a) * MT + t] = V[a];
}

struct SpecCoef {
    double2 c[4][2];  // scalar spectrum s = sum_reg c[s][reg] * Htilde_reg
};

// Octant spectra: spec[s][kz][ky][kx] for 0 <= k <= M/2, divided by M (the
// 1/M of the inverse transform).
__global__ void k_octant(const double2* full, int nreg, int nscal, int want_grad, SpecCoef cf, int Mx,
                         int My, int Mz, double invM, double2* spec64, float2* spec32) {
    int Ox = Mx / 2 + 1, Oy = My / 2 + 1, Oz = Mz / 2 + 1;
    int64_t OT = (int64_t)Ox * Oy * Oz;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= OT) return;
    int ox = (int)(t % Ox), oy = (int)((t / Ox) % Oy), oz = (int)(t / ((int64_t)Ox * Oy));
    int64_t MT = (int64_t)Mx * My * Mz;
    int64_t src = ((int64_t)oz * My + oy) * Mx + ox;
    for (int s = 0; s < nscal; ++s) {
        double2 acc = make_double2(0, 0);
        for (int g = 0; g < nreg; ++g) acc = acc + cf.c[s][g] * full[g * MT + src];
        acc = invM * acc;
        spec64[s * OT + t] = acc;
        spec32[s * OT + t] = make_float2((float)acc.x, (float)acc.y);
    }
    if (want_grad)
        for (int a = 0; a < 3; ++a) {
            double2 v = invM * full[(nreg + a) * MT + src];
            spec64[(nscal + a) * OT + t] = v;
            spec32[(nscal + a) * OT + t] = make_float2((float)v.x, (float)v.y);
        }
}

struct Mats {
    int nreg;
    double w;
    double mu[2], eps[2], k[2];
};

static Mats materials(const aimx_ctx* ctx, double freq) {
    Mats m;
    m.w = 2.0 * kPi * freq;
    m.nreg = two_blocks(ctx->form) ? 2 : 1;
    m.mu[0] = kMu0 * ctx->mu_out;
    m.eps[0] = kEps0 * ctx->eps_out;
    m.mu[1] = kMu0 * ctx->mu_in;
    m.eps[1] = kEps0 * ctx->eps_in;
    for (int g = 0; g < 2; ++g) m.k[g] = m.w * std::sqrt(m.mu[g] * m.eps[g]);
    return m;
}

// j*a as a complex number
static double2 jmul(double a) { return make_double2(0.0, a); }

Coefs near_coefs(const aimx_ctx* ctx, double freq) {
    Mats m = materials(ctx, freq);
    Coefs c;
    for (auto& v : c.near) v = make_double2(0, 0);
    for (auto& v : c.lin) v = make_double2(0, 0);
    // EFIE weight of the CFIE (1 for the other formulations)
    const double ea = ctx->form == AIMX_CFIE ? ctx->cfie_alpha : 1.0;
    if (ctx->linterm) {
        // L = L^A - k^-2 L^Phi gains k^2 (N^A_lin - k^-2 N^Phi_lin) = k^2 N^A_lin - N^Phi_lin,
        // scaled like L in each region's rows
        for (int g = 0; g < m.nreg; ++g) {
            const double k2 = m.k[g] * m.k[g];
            c.lin[0] = c.lin[0] + jmul(ea * m.w * m.mu[g] * k2);
            c.lin[1] = c.lin[1] + jmul(-ea * m.w * m.mu[g]);
            if (ctx->form == AIMX_PMCHWT) {
                c.lin[2] = c.lin[2] + jmul(kEta0 * kEta0 * m.w * m.eps[g] * k2);
                c.lin[3] = c.lin[3] + jmul(-kEta0 * kEta0 * m.w * m.eps[g]);
            }
        }
    }
    if (ctx->form == AIMX_EFIE || ctx->form == AIMX_CFIE) {
        c.near[0] = jmul(ea * m.w * m.mu[0]);
        c.near[1] = jmul(-ea * m.w * m.mu[0] / (m.k[0] * m.k[0]));
        double2 zs = make_double2(0, 0);
        if (ctx->sigma > 0) {
            // surface impedance Z_s = (1 + j) / (sigma delta), delta = sqrt(2 / (w mu0 sigma))
            const double delta = std::sqrt(2.0 / (m.w * kMu0 * ctx->sigma));
            zs = make_double2(1.0 / (ctx->sigma * delta), 1.0 / (ctx->sigma * delta));
        }
        if (ctx->form == AIMX_EFIE) {
            c.near[2] = zs;
        } else {
            // CFIE: (1 - alpha) eta (G / 2 + K_g) with eta = w mu / k the background impedance
            const double eta = m.w * m.mu[0] / m.k[0];
            c.near[2] = make_double2((1.0 - ea) * eta, 0.0);
            c.near[3] = make_double2((1.0 - ea) * eta * 0.5, 0.0) + ea * zs;
        }
    } else {
        for (int g = 0; g < 2; ++g) {
            c.near[0] = c.near[0] + jmul(m.w * m.mu[g]);
            c.near[1] = c.near[1] + jmul(-m.w * m.mu[g] / (m.k[g] * m.k[g]));
            c.near[4] = c.near[4] + jmul(kEta0 * kEta0 * m.w * m.eps[g]);
            c.near[5] = c.near[5] + jmul(-kEta0 * kEta0 * m.w * m.eps[g] / (m.k[g] * m.k[g]));
        }
        c.near[2] = make_double2(2.0 * kEta0, 0.0);
        c.near[3] = make_double2(-2.0 * kEta0, 0.0);
    }
    return c;
}

template <class T>
void ensure_spectra(aimx_ctx* ctx, double freq, cudaStream_t s) {
    if (prec<T>(ctx).spec_freq == freq && prec<T>(ctx).spec) return;
    if (!(freq > 0.0)) throw Error{AIMX_E_ARG, "frequency must be positive"};
    Mats m = materials(ctx, freq);
    const int want_grad = ctx->form != AIMX_EFIE;
    const int nreg = m.nreg;
    const int narr = nreg + (want_grad ? 3 : 0);
    const int64_t MT = (int64_t)ctx->M[0] * ctx->M[1] * ctx->M[2];
    const int Ox = ctx->M[0] / 2 + 1, Oy = ctx->M[1] / 2 + 1, Oz = ctx->M[2] / 2 + 1;
    const int64_t OT = (int64_t)Ox * Oy * Oz;
    if (ctx->kgen_elems < (size_t)(narr * MT)) {
        if (ctx->d_kgen) dev_free(ctx, ctx->d_kgen);
        ctx->d_kgen = (double*)dev_alloc(ctx, sizeof(double2) * narr * MT);
        ctx->kgen_elems = narr * MT;
    }
    if (!ctx->f64.spec) ctx->f64.spec = (double*)dev_alloc(ctx, sizeof(double2) * ctx->nspec * OT);
    if (!ctx->f32.spec) ctx->f32.spec = (float*)dev_alloc(ctx, sizeof(float2) * ctx->nspec * OT);
    // gradient samples: eta0 for PMCHWT; (1 - alpha) eta for the K_g part of the CFIE
    double gs = 0.0;
    if (ctx->form == AIMX_PMCHWT) gs = kEta0;
    if (ctx->form == AIMX_CFIE) gs = (1.0 - ctx->cfie_alpha) * m.w * m.mu[0] / m.k[0];
    Region r0{m.k[0], gs}, r1{m.k[1], gs};
    double2* full = reinterpret_cast<double2*>(ctx->d_kgen);
    k_sample<<<(unsigned)((MT + 255) / 256), 256, 0, s>>>(full, nreg, want_grad, r0, r1, ctx->M[0],
                                                          ctx->M[1], ctx->M[2], ctx->n[0], ctx->n[1],
                                                          ctx->n[2], ctx->h[0], ctx->h[1], ctx->h[2]);
    AIMX_CUDA_TRY(cudaGetLastError());
    fft3d_full<double>(ctx->d_kgen, narr, ctx->M, false, s);
    SpecCoef cf;
    for (auto& row : cf.c)
        for (auto& v : row) v = make_double2(0, 0);
    int nscal;
    if (!two_blocks(ctx->form)) {
        const double ea = ctx->form == AIMX_CFIE ? ctx->cfie_alpha : 1.0;
        nscal = 2;
        cf.c[0][0] = jmul(ea * m.w * m.mu[0]);
        cf.c[1][0] = jmul(-ea * m.w * m.mu[0] / (m.k[0] * m.k[0]));
    } else {
        nscal = 4;
        for (int g = 0; g < 2; ++g) {
            cf.c[0][g] = jmul(m.w * m.mu[g]);
            cf.c[1][g] = jmul(-m.w * m.mu[g] / (m.k[g] * m.k[g]));
            cf.c[2][g] = jmul(kEta0 * kEta0 * m.w * m.eps[g]);
            cf.c[3][g] = jmul(-kEta0 * kEta0 * m.w * m.eps[g] / (m.k[g] * m.k[g]));
        }
    }
    k_octant<<<(unsigned)((OT + 255) / 256), 256, 0, s>>>(
        full, nreg, nscal, want_grad, cf, ctx->M[0], ctx->M[1], ctx->M[2], 1.0 / (double)MT,
        reinterpret_cast<double2*>(ctx->f64.spec), reinterpret_cast<float2*>(ctx->f32.spec));
    AIMX_CUDA_TRY(cudaGetLastError());
    ctx->f64.spec_freq = freq;
    ctx->f32.spec_freq = freq;
}

template void ensure_spectra<float>(aimx_ctx*, double, cudaStream_t);
template void ensure_spectra<double>(aimx_ctx*, double, cudaStream_t);

}  // namespace aimx
