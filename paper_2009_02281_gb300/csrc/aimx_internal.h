// Internal declarations shared by the translation units of libaimx.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/aimx.h"

namespace aimx {

constexpr double kPi = 3.14159265358979323846;
constexpr double kMu0 = 4.0e-7 * kPi;
constexpr double kC0 = 299792458.0;
constexpr double kEps0 = 1.0 / (kMu0 * kC0 * kC0);
constexpr double kEta0 = kMu0 * kC0;

constexpr int kMaxQuad = 64;        // points of the largest triangle rule kept on the device
constexpr int kTwiddleLen = 4096;   // largest FFT length supported (2^k or 3 * 2^k)
constexpr int kTwiddleTab = 3 * kTwiddleLen;   // device twiddle table length: every supported length divides it

template <class T>
struct Cplx;
template <>
struct Cplx<float> {
    using type = float2;
};
template <>
struct Cplx<double> {
    using type = double2;
};

// Status carrier used inside the library (never crosses the ABI).
struct Error {
    int code;
    std::string msg;
};

#define AIMX_CUDA_TRY(expr)                                                        \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess)                                                     \
            throw ::aimx::Error{AIMX_E_CUDA, std::string(#expr) + ": " +           \
                                                 cudaGetErrorString(e_)};          \
    } while (0)

// Typed device allocation owned by a context.
template <class T>
struct DArray {
    T* p = nullptr;
    size_t n = 0;
};

// Per-precision device data of a context.
template <class T>
struct PrecData {
    T* w = nullptr;        // projection weights [N][U][4] (internal order)
    T* wg = nullptr;       // CFIE: moments of n x f, [N][U][3] (internal order)
    T* na = nullptr;       // near N^A  [nnz]
    T* np = nullptr;       // near N^Phi[nnz]
    T* nk = nullptr;       // near N^K  [nnz]
    T* ng = nullptr;       // near Gram matrix [nnz] (surface impedance, EFIE with sigma > 0)
    T* la = nullptr;       // linear-term N^A_lin on the overlap pattern [nlin] (when enabled)
    T* lp = nullptr;       // linear-term N^Phi_lin on the overlap pattern [nlin]
    T* zn = nullptr;       // conventional-AIM near entries j w mu (N^A(k) - k^-2 N^Phi(k)) [nnz] complex
    T* plw = nullptr;      // charge form: pulse weights [nt][U] (internal triangle order)
    T* npt = nullptr;      // charge form: static pulse near values Pt_s,NR - Pt_s,P [tnnz]
    T* tl = nullptr;       // charge form: incidence [nt][3] signed edge lengths (0 = no edge)
    T* cwork = nullptr;    // charge form, generic path: q and phi [2][chunk][nt] complex
    size_t cwork_elems = 0;
    T* spec = nullptr;     // octant spectra [nspec][Oz][Oy][Ox] complex (2 T each)
    double spec_freq = -1.0;
    // work buffers of the generic FFT path
    T* grid = nullptr;     // [chunk][F][Mz][My][Mx] complex
    size_t grid_elems = 0; // complex elements allocated
};

// Per-stage CUDA-event timing (enabled by aimx_profile).
enum Stage {
    ST_KERNELGEN = 0,
    ST_TRANSPOSE,
    ST_GATHER,
    ST_XY_FWD,
    ST_ZPASS,
    ST_XY_INV,
    ST_FINAL,
    ST_G_PROJECT,
    ST_G_FFT,
    ST_G_MIX,
    ST_G_INTERP,
    ST_SOLVE_BLAS,
    ST_SOLVE_RESIDUAL,
    ST_SOLVE_PRECOND,
    ST_SOLVE_REORTH,
    ST_AIM_FILL,
    ST_COUNT
};

struct ProfRec {
    int stage;
    cudaEvent_t a, b;
};

struct Profiler {
    bool on = false;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    double ms[ST_COUNT] = {};
    int64_t count[ST_COUNT] = {};
};

// block-Jacobi preconditioner state (precond.cu)
struct PrecondBlocks {
    int nblk = 0, maxnb = 0, D = 0;   // blocks, bases per block (max), matrix order
    int* d_ptr = nullptr;            // [nblk+1]
    int* d_idx = nullptr;            // [N] internal basis ids grouped by block
    double2* d_work = nullptr;       // [nblk][D][D] FP64 assembly / factorisation
    float2* d_inv = nullptr;         // [nblk][D][D] FP32 inverse
    double freq = -1.0;
};

// parameter offsets of the learned-preconditioner network (gnn.cu)
struct GnnLayout {
    int K = 2, L = 4;
    int64_t A0 = 0, a0 = 0, B[8] = {}, C[8] = {}, c[8] = {}, D[8] = {}, d[8] = {};
    int64_t Ua = 0, Ub = 0, Uc = 0, u = 0, E = 0, f = 0, G = 0, g = 0, total = 0;
};

// per-context state of the learned preconditioner (gnn.cu)
struct GnnGraph {
    std::vector<void*> own;        // allocations below (freed together)
    int* d_rows = nullptr;         // [nnz] internal row of each near entry
    int* d_trans = nullptr;        // [nnz] position of (n, m) for entry (m, n)
    int* d_colc = nullptr;         // [nnz] caller index of the column
    int* d_dpos = nullptr;         // [N] position of the diagonal entry in each row
    float* d_deginv = nullptr;     // [N] 1 / off-diagonal degree
    float* d_x = nullptr;          // [N][8] node features
    float* d_e = nullptr;          // [nnz][16] orientation-invariant edge features
    float* d_basis = nullptr;      // [nnz][8] signed bases (static)
    double* d_eta = nullptr;       // [nnz][3] normalised static near entries (static)
    double* d_center = nullptr;    // [N][3] basis centres
    double2* d_minv = nullptr;     // [N] or [N][2][2] D^{-1}, caller order
    double* d_lossn = nullptr;     // [N] per-row loss terms
    double feat_freq = -1.0, minv_freq = -1.0;
    int K = 0, L = 0;              // shape the activation buffers were sized for
    float* d_H = nullptr;          // [L+1][N][64]
    float* d_P = nullptr;          // [L][N][64]
    float* d_S = nullptr;          // [N][64]
    float* d_Pa = nullptr;         // [N][64] Ua h_L
    float* d_Pb = nullptr;         // [N][64] Ub h_L
    float* d_o = nullptr;          // [nnz][K]
    float* d_g = nullptr;          // [N][K]
    const __nv_bfloat16* out_w = nullptr;  // weights that produced d_o / d_g
    double out_freq = -1.0;
    __nv_bfloat16* d_watt = nullptr;       // attached weights (aimx_gnn_attach)
    int64_t att_np = 0;
    int att_K = 0, att_L = 0;
    void* d_vT = nullptr;          // transposed right-hand sides for the apply
    size_t vT_bytes = 0;
};

}  // namespace aimx

struct aimx_ctx {
    // problem description
    int form = AIMX_EFIE;
    int order = 2;
    int P = 3;             // stencil nodes per axis
    int U = 27;            // stencil nodes per basis
    int N = 0;             // RWG functions
    int nunk = 0;          // unknowns (N or 2N)
    int n[3] = {0, 0, 0};  // grid nodes
    int M[3] = {0, 0, 0};  // padded FFT lengths
    double h[3] = {0, 0, 0};
    double origin[3] = {0, 0, 0};
    int radius = 3;
    double eps_out = 1, mu_out = 1, eps_in = 1, mu_in = 1;
    double sigma = 0;      // conductivity for the surface impedance (EFIE, CFIE), 0 = PEC
    double cfie_alpha = 0.5;  // EFIE weight of the CFIE
    int F = 4;             // grid fields per RHS (4 EFIE, 8 PMCHWT)
    int nspec = 2;         // spectra per frequency (2 EFIE, 7 PMCHWT)
    int64_t nnz = 0;

    // host-side products (internal order = bases sorted by anchor z, y, x)
    std::vector<int> perm;         // internal -> caller index
    std::vector<int> iperm;        // caller index -> internal
    std::vector<int> anc;          // [N][3] internal order
    std::vector<int> row_ptr;      // near CSR, internal order [N+1]
    std::vector<int> cols;         // [nnz] internal column ids, ascending
    std::vector<int> plane_lo, plane_hi;   // per z plane: internal bases touching it

    // device geometry / topology
    int nt = 0, nv = 0;
    double* d_xyz = nullptr;       // [nv][3]
    int* d_tri = nullptr;          // [nt][3]
    double* d_area = nullptr;      // [nt]
    int* d_btri = nullptr;         // [N][2] triangle of T+ / T- (internal order)
    int* d_bfree = nullptr;        // [N][2] free vertex id
    double* d_blen = nullptr;      // [N] edge length
    int* d_anc = nullptr;          // [N][3]
    int* d_perm = nullptr;         // [N]
    int* d_row_ptr = nullptr;      // [N+1]
    int* d_cols = nullptr;         // [nnz]
    int* d_node_ptr = nullptr;     // [Nz*Ny*Nx + 1]
    int* d_node_w = nullptr;       // [N*U] weight row index i*U+u
    int* d_node_x = nullptr;       // [N*U] caller basis index of that entry
    double* d_diag = nullptr;      // [N][3] static self terms L^A_s, L^Phi_s, K_s
    double* d_gdiag = nullptr;     // [N] Gram self terms (surface impedance only)
    // linear-term modification (Sec. III-A-3): pairs of bases that share a triangle
    int linterm = 0;               // 1 = products add k^2 (L_lin,direct - L_lin,P) on those pairs
    int64_t nlin = 0;              // overlapping pairs (0 until first enabled)
    std::vector<int> lin_ptr;      // overlap CSR, internal order [N+1]
    std::vector<int> lin_cols;     // [nlin] internal column ids, ascending
    int* d_lin_ptr = nullptr;
    int* d_lin_cols = nullptr;
    int config_gen = 0;            // bumped when a setting that changes the product's kernels changes
    // conventional-AIM comparison mode (Sec. II-B): per-frequency near fill
    int aim = 0;                   // 1 = products use the per-frequency near entries f32/f64.zn
    double aim_freq = -1.0;        // frequency the zn arrays were filled for
    int* d_aim_row_of = nullptr;   // [nnz] row of each near entry
    double* d_aim_htab = nullptr;  // H(k) on offsets [-span, span]^3, complex
    std::vector<double2> h_aim_htab;
    // host copies for port definitions (caller order)
    std::vector<double> h_xyz;     // [nv][3]
    std::vector<int> h_ea, h_eb, h_tp, h_tm;   // [N] edge vertices, T+ / T-
    std::vector<double> h_cen;     // [nt][3] triangle centroids
    double* d_q5 = nullptr;        // [25][4] 5 x 5 collapsed Gauss-Legendre rule (l1, l2, l3, w)

    aimx::PrecData<float> f32;
    aimx::PrecData<double> f64;
    float* d_wsoa = nullptr;       // FP32 weights, field-major [4][U][N] (internal order)

    // kernel-generation scratch (FP64 full grids)
    double* d_kgen = nullptr;
    size_t kgen_elems = 0;

    // matvec host-buffer staging
    void* d_stage = nullptr;
    size_t stage_bytes = 0;

    // fused FP32 path work buffers
    float* d_xT = nullptr;         // [nunk][B] complex, internal order
    float* d_G = nullptr;          // [B][F][Nz][Ny][Nx] complex (projected grid)
    float* d_S = nullptr;          // [B][F][Nz][4][Ny][Nx] complex (xy spectra, parity blocks)
    float* d_part = nullptr;       // [B][F/4][P][N] complex (per-plane interpolation partials)
    int fused_cap = 0;             // RHS capacity of the buffers above
    // charge-form scalar potential (EFIE): L^Phi = D^T Pt D with the pulse matrix Pt in AIMx form
    int charge = 0;                // 1 = products use the charge form (aimx_set_charge_form)
    int charge_built = 0;
    int64_t tnnz = 0;              // triangle near pairs
    std::vector<int> tperm;        // internal triangle -> caller triangle (sorted by anchor z, y, x)
    std::vector<int> tanc;         // [nt][3] triangle anchors, internal order
    std::vector<int> trow_ptr, tcols;       // triangle near CSR, internal order, columns ascending
    std::vector<int> tplane_lo, tplane_hi;  // per z plane: internal triangles touching it
    int max_plane_tris = 0;
    int* d_tanc = nullptr;         // [nt][3]
    int* d_trow_ptr = nullptr;     // [nt+1]
    int* d_tcols = nullptr;        // [tnnz]
    int* d_tnode_ptr = nullptr;    // [Nz*Ny*Nx + 1] node-major triangle lists
    int* d_tnode_w = nullptr;      // [nt*U] entry t*U+u
    int* d_tinc = nullptr;         // [nt][3] internal basis id of each edge (-1 = boundary edge)
    int* d_btri_t = nullptr;       // [N][2] internal triangle ids of T+ / T- (internal basis order)
    int* d_tplane = nullptr;       // [2][Nz] tplane_lo then tplane_hi
    float* d_lp_soa = nullptr;     // FP32 pulse weights field-major [U][nt]
    float* d_qT = nullptr;         // fused path: triangle charges [nt][B] complex
    float* d_phiT = nullptr;       // fused path: triangle potentials [nt][B] complex
    float* d_tpart = nullptr;      // fused path: per-plane triangle partials [B][P][nt] complex
    int charge_cap = 0;            // RHS capacity of the three buffers above
    // near rows grouped into blocks for the final kernel of the plane-fused path: each block
    // is <= 32 consecutive internal rows whose near columns, taken together, are staged once
    int nb_count = 0;              // row blocks (0 = not built, or a row too wide: CSR kernel)
    int nb_umax = 0;               // largest column union of a block
    int* d_nb_rows = nullptr;      // [nb_count+1] first internal row of each block
    int* d_nb_ustart = nullptr;    // [nb_count+1] offset of each block's union in d_nb_ucols
    int* d_nb_ucols = nullptr;     // [sum of unions] internal column ids, ascending per block
    float4* d_nb_ent = nullptr;    // [nnz] CSR order: (union-local column as int bits, N^A, N^Phi, N^K or Gram)
    int max_plane_bases = 0;
    int plane_cap = 0;                  // test hook: bases per plane kept in shared memory (0: all that fit)
    int* d_plane = nullptr;        // [2][Nz] plane_lo then plane_hi
    int path = 0;                  // 0 = automatic, 1 = generic FFT path, 2 = generic with cuFFT (comparison)
    int cufft_plan[2] = {0, 0};    // cached cuFFT plans (FP32, FP64) of the comparison path
    int cufft_batch[2] = {0, 0};   // batch each plan was made for

    // product schedule (autotuner): variant 0 = plane-fused with register-resident lines
    // where the grid allows, 1 = plane-fused with shared-memory lines, 2 = generic path,
    // 3 = as 0 with the TMA-pipelined persistent z-pass;
    // pass = right-hand sides per pass (0 = all that fit the work-buffer budget)
    int sched_variant = 0;
    int sched_pass = 0;

    aimx::Profiler prof;
    aimx::PrecondBlocks pc;
    aimx::GnnGraph gnn;

    int64_t device_bytes = 0;
    std::string last_error;
};

namespace aimx {

// memory helpers (throw Error on failure, book-keep ctx->device_bytes)
void* dev_alloc(aimx_ctx* ctx, size_t bytes);
void dev_free(aimx_ctx* ctx, void* p);

// setup.cu
// Precomputed setup products (internal basis order) restored by aimx_load_static.
struct StaticData {
    std::vector<double> w;     // [N][U][4] projection weights
    std::vector<double> na, np, nk;  // [nnz] near matrices N^A, N^Phi, N^K
    std::vector<double> diag;  // [N][3] static self terms
};
// collapsed Gauss-Legendre product rule on a triangle, q x q points: [Q][4] = (l1, l2, l3, w),
// weights normalised to sum to one; exact to total degree 2q - 2
void triangle_rule(int q, std::vector<double>& out);
// formulations with one unknown block (EFIE, CFIE) vs two (PMCHWT)
inline bool two_blocks(int form) { return form == AIMX_PMCHWT; }

// overlap pattern and N^A_lin, N^Phi_lin (direct - precorrection), built once on demand
void build_linterm(aimx_ctx* ctx);
// aim.cu: conventional-AIM mode buffers, and the near fill for a frequency (no-op when current)
void aim_enable(aimx_ctx* ctx);
void ensure_aim_near(aimx_ctx* ctx, double freq, cudaStream_t s);
void setup_context(aimx_ctx* ctx, const aimx_mesh* mesh, const aimx_material* mat,
                   const aimx_grid* grid, int order, const StaticData* pre = nullptr);

// fft.cu
const double2* twiddles64();
const float2* twiddles32();
template <class T>
void fft3d_padded(T* grid, int batch, const int M[3], const int act[3], bool inverse,
                  cudaStream_t s);
template <class T>
void fft3d_full(T* grid, int batch, const int M[3], bool inverse, cudaStream_t s);
// fft3d_padded of `batch` grids reads only the active input region of a forward transform (its
// passes run on register lines, so no zero padding is needed)
template <class T>
bool fft3d_reads_active_only(const int M[3], int batch);

// kernelgen.cu
template <class T>
void ensure_spectra(aimx_ctx* ctx, double freq, cudaStream_t s);
struct Coefs {
    // near-matrix coefficients; EFIE: aA, aPhi, Z_s (Gram, 0 without a surface
    // impedance); PMCHWT: aA, aPhi, aK, bK, bA, bPhi; CFIE: aA, aPhi, aKg (of K_g),
    // aG (of the Gram matrix: the residue term plus the surface impedance)
    double2 near[6];
    // linear-term coefficients of N^A_lin and N^Phi_lin x, J rows then M rows
    // (zero while the modification is off)
    double2 lin[4];
};
Coefs near_coefs(const aimx_ctx* ctx, double freq);

template <class T>
inline PrecData<T>& prec(aimx_ctx* ctx);
template <>
inline PrecData<float>& prec<float>(aimx_ctx* ctx) {
    return ctx->f32;
}
template <>
inline PrecData<double>& prec<double>(aimx_ctx* ctx) {
    return ctx->f64;
}

// profiling scope: records CUDA events around a stage on stream s when enabled
struct StageScope {
    aimx_ctx* ctx;
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    StageScope(aimx_ctx* c, int st, cudaStream_t str);
    ~StageScope();
};

// fused.cu
bool fused_supported(const aimx_ctx* ctx);
// the plane-fused kernels with register-resident lines apply to this grid
bool fused_reg_supported(const aimx_ctx* ctx);
// FP32 products of this context take the plane-fused path (path setting and schedule); the
// charge form is carried by the register-line kernels only
inline bool use_fused(const aimx_ctx* ctx) {
    if (ctx->charge && (ctx->sched_variant == 1 || !fused_reg_supported(ctx))) return false;
    return ctx->path == 0 && ctx->sched_variant != 2 && fused_supported(ctx);
}

// charge.cu: the charge-form scalar potential (setup on the first enable; product steps)
void build_charge(aimx_ctx* ctx);
// generic path: q = D x for nb right-hand sides ([nb][nt], caller-order x), and the rho field
// of the padded grid (field rho_field of Fg per RHS) projected from q with the pulse weights
template <class T>
void charge_project(aimx_ctx* ctx, const typename Cplx<T>::type* x, int nb, typename Cplx<T>::type* q,
                    typename Cplx<T>::type* grid, int Fg, int rho_field, cudaStream_t s);
// generic path: phi = Lp^T (convolved rho field) + cP N_Pt q per triangle ([nb][nt])
template <class T>
void charge_potential(aimx_ctx* ctx, const typename Cplx<T>::type* grid, int Fg, int rho_field, int nb,
                      const typename Cplx<T>::type* q, typename Cplx<T>::type* phi, double2 cP, cudaStream_t s,
                      const double2* cps = nullptr, const int* fidx = nullptr);
// plane-fused path: qT = D x from xT ([nt][B]); phiT = sum of plane partials + cP N_Pt qT
void charge_fused_q(aimx_ctx* ctx, const float2* xT, int B, cudaStream_t s);
void charge_fused_phi(aimx_ctx* ctx, int B, float2 cP, float2 cP2, cudaStream_t s);
void ensure_charge_buffers(aimx_ctx* ctx, int B);
void matvec_fused(aimx_ctx* ctx, double freq, int nrhs, const float* x, float* y, cudaStream_t s);

// precond.cu
void precond_block_prepare(aimx_ctx* ctx, double freq, cudaStream_t s);
template <class T>
void precond_block_apply(aimx_ctx* ctx, const double2* v, int64_t vstride, typename Cplx<T>::type* z, int nrhs,
                         cudaStream_t s);

// gnn.cu (learned preconditioner)
GnnLayout gnn_layout(int K, int L);
void gnn_features(aimx_ctx* ctx, double freq, cudaStream_t s);
void learned_prepare(aimx_ctx* ctx, double freq, cudaStream_t s);
template <class T>
void learned_apply(aimx_ctx* ctx, const double2* v, int64_t vstride, typename Cplx<T>::type* z, int nrhs,
                   cudaStream_t s);
void gnn_free(aimx_ctx* ctx);

// solve.cu: inverse of the frequency-combined static self blocks (caller order)
void build_diag_inverse(aimx_ctx* ctx, double freq, double2* minv, cudaStream_t s);

// near coefficients of a product (the generic path's form of Coefs)
struct NearCoefs {
    double2 c[6];
    double2 lin[4];   // linear-term coefficients (J rows: A, Phi; M rows: A, Phi)
};
// Frequencies of a batched product: RHS b of the pass takes frequency d_fidx[b]
struct MultiFreq {
    const int* d_fidx = nullptr;       // [nrhs] frequency index per RHS (device)
    const void* spec = nullptr;        // [nf][nspec][Oz][Oy][Ox] complex of the product's precision
    int64_t fstride = 0;               // complex elements per frequency in spec
    const NearCoefs* d_ncs = nullptr;  // [nf] near coefficients (device)
    const double2* d_cphi = nullptr;   // [nf] charge-form near coefficient (device)
};

// matvec.cu
void cufft_release(aimx_ctx* ctx);
template <class T>
void matvec_generic_multi(aimx_ctx* ctx, const MultiFreq& mf, int nrhs, const T* x, T* y, cudaStream_t s);
template <class T>
void matvec_generic(aimx_ctx* ctx, double freq, int nrhs, const T* x, T* y, cudaStream_t s);

}  // namespace aimx
