/*
 * aimx.h -- C ABI of the GB300 AIMx library.
 *
 * AIMx (Sharma & Triverio, "AIMx: An Extended Adaptive Integral Method for the
 * Fast Electromagnetic Modeling of Complex Structures", arXiv 2009.02281)
 * writes every surface-integral operator as
 *
 *     A(k) = (L_s,NR - L_s,P) + W H(k) P                      (Eq. LAIMx, Eq. KAIMx)
 *
 * with a frequency-independent sparse near part built once (Sec. III-A) and a
 * frequency-dependent part evaluated on a regular auxiliary grid by a
 * zero-padded FFT convolution (Sec. II-B, Eq. aimLFR) whose kernel carries
 * the modified self term H(0) = -jk / (4 pi) (Eq. Hmm).
 *
 * Conventions shared by every entry point
 *   - Time dependence e^{j w t}.  Complex numbers are interleaved (re, im).
 *   - Unknown vectors are RHS-major: element (b, n) of an [nrhs][nunk] array
 *     sits at index b * nunk + n.  nunk = N (EFIE) or 2N (PMCHWT: [J ; M/eta0])
 *     where N is the number of RWG functions (one per interior mesh edge,
 *     ordered by (smaller vertex id, larger vertex id)).
 *   - Pointers documented as "device" must be CUDA device memory of the
 *     current device; "host" pointers are ordinary host memory.  The caller
 *     keeps ownership of everything it passes in; the context owns all memory
 *     it allocates and frees it in aimx_destroy.
 *   - stream is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Calls that take a stream are asynchronous with respect to the
 *     host unless stated otherwise.
 *   - Every call returns an int status: AIMX_OK (0), a negative error, or a
 *     positive warning.  No call aborts the process or throws; the message of
 *     the last failure is available from aimx_last_error.
 */
#ifndef AIMX_H
#define AIMX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define AIMX_OK          0
#define AIMX_E_ARG      -1   /* invalid argument (null pointer, size <= 0, bad enum)  */
#define AIMX_E_MESH     -2   /* degenerate triangle, edge shared by > 2 triangles,
                                inconsistent orientation                               */
#define AIMX_E_GRID     -3   /* a basis stencil falls outside the grid                 */
#define AIMX_E_NOMEM    -4   /* device or host allocation failed                       */
#define AIMX_E_CUDA     -5   /* a CUDA runtime call failed                             */
#define AIMX_E_TIMEOUT  -6   /* a bounded device wait expired                          */
#define AIMX_E_STATE    -7   /* call not valid for this context (e.g. wrong formulation) */
#define AIMX_E_IO       -8   /* file not readable / writable, or not a matching static-data file */
#define AIMX_E_NOCONV    1   /* warning: at least one RHS missed the solver tolerance  */

/* ------------------------------------------------------------------ inputs */

/* Closed (or open) triangle mesh.  xyz: host [nv][3] float64 coordinates in
 * metres; tri: host [nt][3] int32 vertex ids, counter-clockwise when seen from
 * the side the normal points to (outward for a closed body).  Copied by
 * aimx_setup.  Sec. II-A: RWG functions on pairs of adjacent triangles. */
typedef struct {
    int32_t nv;
    int32_t nt;
    const double* xyz;
    const int32_t* tri;
} aimx_mesh;

#define AIMX_EFIE    0   /* PEC body in a homogeneous background (Eq. EFIEAIMx)          */
#define AIMX_PMCHWT  1   /* penetrable body, two regions, unknowns [J ; M/eta0]            */
#define AIMX_CFIE    2   /* closed PEC body, combined field (Sec. III-B), unknowns J       */

/* Materials.  Relative permittivity / permeability of the background (region
 * 1) and, for AIMX_PMCHWT, of the body (region 2); lossless values.  sigma:
 * conductivity (S/m) of an AIMX_EFIE body for the surface impedance boundary
 * condition (skin effect, cited in Sec. VI): the system becomes Z + Z_s(w) G
 * with Z_s = (1 + j)/(sigma delta), delta = sqrt(2/(w mu0 sigma)) and G the
 * RWG Gram matrix, a static near-region matrix like N^A.  0 = perfect
 * conductor.  Ignored for AIMX_PMCHWT.
 *
 * AIMX_CFIE (Eqs. CFIEout, CFIEAIMx): a closed PEC surface whose triangles are
 * ordered counter-clockwise about the outward normal.  The system is
 *   Z_C = alpha Z_E + (1 - alpha) eta Z_M,  Z_M = G / 2 + K_g,
 * with Z_E the EFIE matrix (including the surface impedance when sigma > 0),
 * G the RWG Gram matrix (the residue term), (K_g)_mn = <n x f_m, PV K[f_n]>
 * and K[X] = int grad G x X dS' (the MFIE J/2 - n x PV K[J] = n x H_inc
 * tested with f_m); eta the background wave impedance.  cfie_alpha in (0, 1],
 * 0 selects 1/2.  Right-hand sides: alpha <f, E_inc> + (1 - alpha) eta
 * <f, n x H_inc>.  Products run on the generic path (aimx_matvec_path
 * returns 1 or 2). */
typedef struct {
    int32_t formulation;
    double eps_out, mu_out;
    double eps_in, mu_in;
    double sigma;
    double cfie_alpha;
} aimx_material;

/* Auxiliary grid (Sec. II-B).  n: nodes per axis (required).  h: spacing per
 * axis; all zero = derived from the vertex bounding box as
 * h_a = (hi_a - lo_a) / (n_a - 1 - 2m), origin_a = lo_a - m h_a with margin
 * m = floor((order + 1) / 2); an axis along which the mesh is flat takes the
 * largest spacing of the other axes.  When h is given, origin must be given too.
 * near_radius: near-region radius in cells (Chebyshev distance of stencil
 * anchors), 0 = 3.  pad: zero-padded FFT length per axis, of the form 2^k or
 * 3 * 2^k, >= 2 n_a - 1 and <= 4096; 0 = the smallest such length (any valid
 * value gives the same product). */
typedef struct {
    int32_t n[3];
    double h[3];
    double origin[3];
    int32_t near_radius;
    int32_t pad[3];
} aimx_grid;

typedef struct aimx_ctx aimx_ctx;

/* Sizes of a context (filled by aimx_info). */
typedef struct {
    int32_t n_basis;       /* N, RWG functions                       */
    int32_t n_unknowns;    /* N (EFIE) or 2N (PMCHWT)                */
    int64_t near_nnz;      /* stored near pairs (m, n), m = n included */
    int32_t grid_n[3];
    int32_t pad[3];
    double grid_h[3];
    double grid_origin[3];
    int32_t order;
    int32_t formulation;
    int64_t device_bytes;  /* device memory held by the context      */
} aimx_info_t;

/* ------------------------------------------------------------------ lifecycle */

/* Build a context: RWG functions, grid, stencil anchors (Sec. II-B),
 * moment-matching projection weights P (W = P^T), the near-region pair list
 * and the frequency-independent near matrices N = L_s,NR - L_s,P for the
 * vector potential, scalar potential and K operator (Eqs. Lmatdecomp2,
 * aimLPs, KAIMx), all in FP64 on the current device.  order: stencil order n
 * (n + 1 nodes per axis), 1..3.  Errors: AIMX_E_ARG, AIMX_E_MESH, AIMX_E_GRID,
 * AIMX_E_NOMEM, AIMX_E_CUDA.  Synchronous. */
int aimx_setup(const aimx_mesh* mesh, const aimx_material* mat, const aimx_grid* grid,
               int order, aimx_ctx** out);

/* Free every resource of ctx (NULL is accepted).  Synchronises the device. */
int aimx_destroy(aimx_ctx* ctx);

int aimx_info(const aimx_ctx* ctx, aimx_info_t* out);

/* Human-readable text for a status code (static storage). */
const char* aimx_status_string(int status);

/* Message of the last failure on ctx (static per context; "" when none). */
const char* aimx_last_error(const aimx_ctx* ctx);

/* ------------------------------------------------------------------ hot path */

#define AIMX_F32 0
#define AIMX_F64 1

/* y = A(k) x for nrhs vectors (Eq. EFIEAIMx for AIMX_EFIE; the two-region form
 * for AIMX_PMCHWT), at frequency freq in Hz:
 *   projection P onto the grid, zero-padded 3-D FFT convolution with the grid
 *   kernels H(k) (and grad H(k) for the K operator), interpolation W = P^T,
 *   and the sparse near correction.
 * x, y: device [nrhs][nunk] complex (float2 for AIMX_F32, double2 for
 * AIMX_F64), x and y must not overlap.  The grid kernels for freq are
 * generated on the first call at that frequency and cached.  Work buffers are
 * grown on demand (the first call at a new nrhs may allocate).  Asynchronous
 * on stream; errors of queued work surface at the next synchronising call. */
int aimx_matvec(aimx_ctx* ctx, double freq, int nrhs, const void* x, void* y,
                int precision, void* stream);

/* Same product with host arrays x, y ([nrhs][nunk] complex, same precision
 * rules); copies in, runs aimx_matvec, copies out and synchronises stream. */
int aimx_matvec_host(aimx_ctx* ctx, double freq, int nrhs, const void* x, void* y,
                     int precision, void* stream);

/* ------------------------------------------------------------------ solve and sweep */

#define AIMX_PRECOND_DIAG 0   /* inverse of the static self block per basis (diagonal of L_s, Sec. III-A-2) */
#define AIMX_PRECOND_NONE 1
#define AIMX_PRECOND_BLOCK 2  /* block Jacobi: bases grouped by 2x2x2 anchor cells (<= 32 per block); each block
                                 is the full AIMx matrix block, static near part plus the grid-generated
                                 frequency-dependent part (Sec. III-A-2), inverted in FP64, applied in FP32 */
#define AIMX_PRECOND_LEARNED 3 /* M = D^{-1} (I + C): D as for AIMX_PRECOND_DIAG, C on the near graph predicted
                                  by the network attached with aimx_gnn_attach (not in the paper; the learned
                                  analogue of augmenting the diagonal of L_s with off-diagonal entries,
                                  Sec. III-A-2).  Linear in the vector, so GMRES stays valid. */
/* AIMX_CFIE contexts take AIMX_PRECOND_DIAG (static self terms of all three
 * operators and the residue) or AIMX_PRECOND_NONE; _BLOCK and _LEARNED return
 * AIMX_E_STATE. */

typedef struct {
    double tol;               /* target relative true residual |b - A x| / |b| (0 = 1e-6)            */
    int32_t restart;          /* Krylov vectors per cycle (0 = 50)                                    */
    int32_t max_iter;         /* total inner iterations per right-hand side (0 = 1000)                */
    int32_t max_refine;       /* FP64 refinement cycles (0 = max_iter / restart + 10)                 */
    int32_t inner_precision;  /* AIMX_F32 (default) or AIMX_F64 products inside a cycle              */
    int32_t precond;          /* AIMX_PRECOND_DIAG (default), _NONE, _BLOCK or _LEARNED              */
    int32_t use_x0;           /* 1: x holds an initial guess on entry                                 */
    int32_t learned_trial;    /* AIMX_PRECOND_LEARNED only: Krylov steps of the trial that compares it
                                 with the diagonal preconditioner (0 = 10, < 0 = no trial)            */
} aimx_solve_opts;

typedef struct {
    int32_t iterations;       /* inner GMRES iterations used                                          */
    int32_t refinements;      /* FP64 refinement cycles used                                          */
    double rel_residual;      /* final |b - A x| / |b| from the FP64 product                         */
    int32_t status;           /* AIMX_OK or AIMX_E_NOCONV                                             */
    int32_t precond_used;     /* the preconditioner that finished the solve (differs from the one
                                 requested when the learned one lost its trial)                       */
} aimx_solve_stats;

/* Solve A(k) x = b for nrhs right-hand sides in lockstep (the iterative GMRES
 * solve of Sec. V): cycles of right-preconditioned GMRES(restart) with FP64
 * Krylov vectors (classical Gram-Schmidt applied twice) and FP32 (or FP64)
 * AIMx products, each cycle started from the true residual b - A x
 * (iterative refinement).  With FP32 inner products and tol >= 1e-5 the
 * intermediate true residuals use the FP32 product (its ~1e-6 relative error
 * is far below the target); convergence is always confirmed, and
 * stats.rel_residual always computed, with the FP64 product.  b, x: device
 * [nrhs][nunk] complex128 (double2), caller-owned; stats: host array [nrhs] or
 * NULL.  Returns AIMX_E_NOCONV (> 0) when any right-hand side misses tol.
 * With AIMX_PRECOND_LEARNED the diagonal preconditioner is its fallback and
 * the true residual judges it: the solve first runs one short cycle
 * (learned_trial Krylov steps) with each of the two from the same start, and
 * continues from the learned one's iterate unless its true residual is more
 * than twice the diagonal one's for the median right-hand side, in which case
 * it continues from the diagonal one's iterate with the diagonal
 * preconditioner; both trials count in stats.iterations and
 * stats.precond_used names the winner.  The trial catches networks that are
 * bad from the start, not ones that only fall behind after many steps.
 * Electrically small conductors (EFIE with k h below about 1e-3, h the mesh
 * edge) can stall with AIMX_F32 inner products: the vector-potential term is
 * O((k h)^2) of the scalar-potential term and falls below FP32 rounding, so the
 * refinement stops short of tol (AIMX_E_NOCONV); use AIMX_F64 there.
 * Synchronises stream. */
int aimx_solve(aimx_ctx* ctx, double freq, int nrhs, const void* b, void* x, const aimx_solve_opts* opts,
               aimx_solve_stats* stats, void* stream);

/* z = M v for the preconditioner `precond` (AIMX_PRECOND_*) at freq; v, z:
 * device [nrhs][nunk] complex128, not overlapping.  The block preconditioner
 * is assembled and inverted on the first call at a frequency and cached.
 * Synchronises stream. */
int aimx_precond_apply(aimx_ctx* ctx, double freq, int precond, int nrhs, const void* v, void* z, void* stream);

/* Plane-wave right-hand sides (Eq. EFIEdis / CFIEdis excitation): for wave w
 * with unit propagation direction dirs[w] and polarisation pols[w] (host
 * [nwave][3] doubles, E0 = 1 V/m, background medium), b[w] = <f_m, E_inc>,
 * and for AIMX_PMCHWT additionally eta0 <f_m, H_inc> in the second half; for
 * AIMX_CFIE b[w] = alpha <f_m, E_inc> + (1 - alpha) eta <f_m, n x H_inc>.
 * b: device [nwave][nunk] complex128.  Synchronises stream. */
int aimx_rhs_planewave(aimx_ctx* ctx, double freq, int nwave, const double* dirs, const double* pols, void* b,
                       void* stream);

/* Far-zone electric field r e^{jkr} E(rhat) of the solved surface currents in
 * the background medium for ndir unit directions (host [ndir][3]); x: device
 * [nrhs][nunk] complex128; E: host [nrhs][ndir][3] complex128 (interleaved).
 * RCS = 4 pi |E|^2 / |E0|^2.  Synchronises stream. */
int aimx_farfield(aimx_ctx* ctx, double freq, int nrhs, const void* x, int ndir, const double* dirs, double* E,
                  void* stream);

/* Frequency sweep (Sec. V-A, Discussion: T = T_s + N T_d): for every
 * frequency, plane-wave right-hand sides, then aimx_solve, reusing the
 * frequency-independent near matrices built once by aimx_setup; only the grid
 * kernel spectra and the preconditioner coefficients change per frequency.
 * X: device [nf][nwave][nunk] complex128; stats: host [nf][nwave] or NULL.
 * warm_start = 1 starts each frequency from the previous solution.  Returns
 * AIMX_E_NOCONV if any system missed tol.  Synchronises stream. */
int aimx_sweep(aimx_ctx* ctx, int nf, const double* freqs, int nwave, const double* dirs, const double* pols, void* X,
               const aimx_solve_opts* opts, int warm_start, aimx_solve_stats* stats, void* stream);

/* Batched frequency sweep (the cost model of the Discussion, T = T_s + N T_d):
 * the nf x nrhs systems A(k_f) x_{f,w} = b_{f,w} are solved together instead of
 * one frequency after another.
 *   - B: device [nf][nrhs][nunk] complex128 right-hand sides (plane waves,
 *     ports or any other); X: device [nf][nrhs][nunk] complex128 solutions
 *     (an initial guess when opts->use_x0).  Caller-owned, not overlapping.
 *   - Right-preconditioned GMRES(restart) in lockstep over up to max_batch
 *     systems at a time (0 = as many as fit about 8 GiB of Krylov vectors).
 *     Each product of the batch carries one frequency per system: that
 *     frequency's kernel spectra (Eq. Hmm), near coefficients and diagonal
 *     preconditioner, built once per call for all frequencies, while the
 *     static near matrices and weights are shared (Sec. III-A).
 *   - The Arnoldi steps (classical Gram-Schmidt twice, FP64), the Givens
 *     rotations, the convergence test and the back substitution run on the
 *     device; one cycle of restart steps is captured into a CUDA graph and
 *     replayed while the batch size stays the same.  The host synchronises
 *     once per cycle to retire converged systems and admit pending ones; the
 *     batch shrinks (a new graph) when fewer than 3/4 of it is busy.
 *   - Every cycle starts from the true residual; with AIMX_F32 inner products
 *     and tol >= 1e-5 cycle residuals use the FP32 product, and every reported
 *     residual (stats[f][w].rel_residual, host array or NULL) is recomputed with
 *     the FP64 product; systems that fail that check run more cycles with FP64
 *     residuals.
 *   - Products use the generic path (the plane-fused kernels take one
 *     frequency per pass).  opts->precond: AIMX_PRECOND_DIAG or _NONE, others
 *     AIMX_E_STATE; AIMX_E_STATE in the conventional-AIM mode.  The linear term
 *     and the charge form apply.
 *   - warm_start = 1: systems are admitted with even frequency indices first,
 *     and each later system starts from the converged solution of the same
 *     right-hand side at the nearest frequency (with max_batch below nf x nrhs
 *     the odd frequencies then start next to converged neighbours); ignored
 *     with opts->use_x0 (the caller's guesses are kept).
 *   - counters (host int64 [3] or NULL): cycles, graphs captured, batched
 *     products.  Returns AIMX_E_NOCONV if any system missed tol.  Runs on a
 *     private stream ordered after `stream`; synchronous on return. */
int aimx_sweep_batched(aimx_ctx* ctx, int nf, const double* freqs, int nrhs, const void* B, void* X,
                       const aimx_solve_opts* opts, int max_batch, int warm_start, aimx_solve_stats* stats,
                       int64_t* counters, void* stream);

/* Select the matvec implementation: 0 = automatic (FP32: the plane-fused
 * path whenever the grid is padded to exactly twice a power-of-two size per
 * axis, else the generic path), 1 = always the generic path, 2 = the generic
 * path with its 3-D FFTs done by cuFFT (full, unpruned transforms; the plain
 * comparison path, FP32 and FP64).  All compute the same product; FP64 uses
 * the generic path (with cuFFT under 2).  aimx_matvec_path returns 0
 * (plane-fused), 1 (generic) or 2 (generic with cuFFT). */
int aimx_set_path(aimx_ctx* ctx, int path);

/* 0 if aimx_matvec at this precision runs the plane-fused path, 1 if generic. */
int aimx_matvec_path(const aimx_ctx* ctx, int precision);

/* ------------------------------------------------------------------ linear-term modification
 * Sec. III-A-3, Eqs. linterm and Lmatdecomplin.  The term k^2 G_lin,
 * G_lin = -r / (8 pi), of the Green's function's Taylor series is not smooth
 * at r = 0, so the grid represents it poorly where a basis and a testing
 * function overlap (share a triangle).  With enable = 1 every product of this
 * context (aimx_matvec in both precisions and paths, aimx_solve, aimx_sweep,
 * batches) adds, on those pairs, k^2 (L_lin,direct - L_lin,P): the direct
 * integrals of G_lin minus their precorrection with the sampled kernel
 * -|d h| / (8 pi) (0 at d = 0).  In the L operator this is
 * k^2 N^A_lin - N^Phi_lin, scaled as L is in each region's rows (EFIE; both
 * regions of PMCHWT).  The K operator is unchanged.
 *   - The first enable builds the overlap pattern and its values (FP64 direct
 *     integrals: closed-form inner integrals of |r - r'|, the 5 x 5 collapsed
 *     Gauss rule outside) and keeps them until aimx_destroy; synchronous.
 *   - Preconditioners (diagonal, block, learned) keep the unmodified near
 *     matrices.  Static data files do not hold these values.
 *   - enable = 0 turns the term off again; other values are AIMX_E_ARG.
 * Off by default, as in the paper's numerical results. */
int aimx_set_linear_term(aimx_ctx* ctx, int enable);

/* ------------------------------------------------------------------ conventional-AIM comparison mode
 * Sec. II-B: the method AIMx is compared against.  With enable = 1 the
 * products of this EFIE context (aimx_matvec in both precisions and paths,
 * aimx_solve, aimx_sweep, batches, aimx_matvec_noalloc) use, on the near
 * pairs, entries recomputed at every new frequency:
 *     j w mu [N^A(k) - k^-2 N^Phi(k)],   N(k) = L_NR(k) - L_P(k),
 * L_NR(k) the full-wave direct integrals (static part: closed-form inner
 * potentials and the 5 x 5 outer rule; smooth part G_d(k) = (e^{-jkR} - 1) /
 * (4 pi R): the 5 x 5 product rule on both triangles) and L_P(k) their
 * precorrection with the grid kernel H(k).  The far part is the unchanged grid
 * product, so near entries equal the full-wave Galerkin entries and far ones
 * the AIMx ones.
 *   - The fill runs on the product's stream when the frequency changes (stage
 *     "aim_near_fill" of aimx_profile); it synchronises that stream once.
 *   - Preconditioners keep the static self terms; the linear-term
 *     modification is ignored while this mode is on (the near pairs are exact).
 *   - AIMX_E_STATE for AIMX_PMCHWT contexts.  enable = 0 returns to AIMx.
 * Off by default. */
int aimx_set_conventional_aim(aimx_ctx* ctx, int enable);

/* ------------------------------------------------------------------ charge-form scalar potential
 * The discretisation of the augmented EFIE that the paper uses for its on-chip
 * examples (Sec. V-C to V-E), kept on the RWG unknowns.  With enable = 1 the
 * scalar-potential operator of this EFIE context (or, for AIMX_PMCHWT, of each
 * region in both the J and the M blocks) is written through the triangle
 * charges q = D x (D_tn = +l_n on T+, -l_n on T-):
 *     L^Phi = D^T Pt D,   Pt = (Pt_s,NR - Pt_s,P) + Lp^T H(k) Lp,
 * Pt_ij = (A_i A_j)^-1 int_{T_i} int_{T_j} G the pulse-pulse potential, Lp the
 * pulse projection weights (moment matching of a unit charge on each
 * triangle's own stencil), triangle anchors and near pairs as for the bases
 * (same anchor formula on the centroids, same Chebyshev radius), the static
 * near values Pt_s,NR from the closed-form inner potential of 1/(4 pi R) and
 * the 5 x 5 outer rule, and Pt_s,P their precorrection with the static grid
 * kernel.  The product replaces the RWG terms N^Phi x + P_rho^T H P_rho x;
 * the vector potential is unchanged.  A divergence-free current then gets
 * exactly zero scalar potential (no residue of the grid approximation).
 *   - The first enable builds the triangle data (host integer steps, FP64
 *     device kernels) and synchronises the device.  Later toggles are cheap.
 *   - Applies to aimx_matvec (both precisions, generic and plane-fused paths),
 *     aimx_solve, aimx_sweep, ports and batches.  Preconditioners keep the RWG
 *     static self terms.  aimx_matvec_noalloc returns AIMX_E_STATE while on.
 *   - AIMX_PMCHWT: each region r contributes -k_r^-2 D^T Pt(k_r) D, with the
 *     region's coefficient, to the J block (E rows) and the M block (H rows);
 *     aimx_sweep_batched then returns AIMX_E_STATE (no multi-frequency
 *     two-region charge product).
 *   - AIMX_E_STATE for CFIE contexts, or with the linear term or the
 *     conventional-AIM mode on; AIMX_E_GRID if a triangle stencil leaves the
 *     grid.  enable = 0 returns to the RWG form.
 * Off by default. */
int aimx_set_charge_form(aimx_ctx* ctx, int enable);

/* Copy the charge-form setup to host arrays in caller triangle numbering (any
 * output may be NULL): nt = triangles; tnnz = triangle near pairs; tanc int32 [nt][3]
 * anchors; rows, cols int32 [tnnz] the pairs (internal order of rows, so
 * compare as sets); npt double [tnnz] = Pt_s,NR - Pt_s,P on them (same
 * order); lp double [nt][(order+1)^3] pulse weights (stencil node u = ux +
 * (order+1) (uy + (order+1) uz)).  AIMX_E_STATE before the first enable.
 * Synchronous. */
int aimx_export_charge(aimx_ctx* ctx, int32_t* nt, int64_t* tnnz, int32_t* tanc, int32_t* rows, int32_t* cols,
                       double* npt, double* lp);

/* The conventional-AIM near entries at freq as complex float64 pairs z [nnz][2],
 * in the near pattern of aimx_export_setup (caller numbering, columns
 * ascending).  AIMX_E_STATE unless the mode is on.  Synchronous. */
int aimx_export_aim_near(aimx_ctx* ctx, double freq, double* z);

/* Copy the linear-term values to host arrays in caller numbering (any output
 * pointer may be NULL): nlin = number of overlapping pairs; row_ptr int64
 * [N+1]; cols int32 [nlin] (ascending per row); na, nphi double [nlin] =
 * N^A_lin, N^Phi_lin.  AIMX_E_STATE before the first aimx_set_linear_term(ctx, 1).
 * Synchronous. */
int aimx_export_linear_term(const aimx_ctx* ctx, int64_t* nlin, int64_t* row_ptr, int32_t* cols,
                            double* na, double* nphi);

/* ------------------------------------------------------------------ product schedule and autotuner
 * How FP32 products of a context are scheduled (not part of the method; the
 * same product in every case, to rounding):
 *   variant 0  plane-fused kernels, lines held in registers where the grid
 *              allows (square 8..64 planes, 8..64 z nodes), else in shared memory
 *   variant 1  plane-fused kernels with lines in shared memory
 *   variant 2  generic path (projection, radix-2 3-D FFT, interpolation)
 *   variant 3  as variant 0, with the z transforms in a persistent kernel whose
 *              tiles are copied into shared memory by the tensor-memory
 *              accelerator (cp.async.bulk.tensor) while the previous tile is
 *              transformed; needs the register-line grids of variant 0
 *   pass       right-hand sides per pass through the work buffers (0 = as many
 *              as the work-buffer budget allows); also bounds the generic
 *              path's chunk and the FP64 products' chunk.
 * The schedule applies when aimx_set_path is 0; variant 1 needs a grid the
 * plane-fused path supports (aimx_matvec_path 0), else AIMX_E_ARG.  Default
 * {0, 0}.  Changing it makes batches recapture their graphs. */
typedef struct {
    int32_t variant;
    int32_t pass;
    double ms;      /* autotune: measured milliseconds per product (0 elsewhere) */
} aimx_schedule;
int aimx_set_schedule(aimx_ctx* ctx, const aimx_schedule* s);
int aimx_get_schedule(const aimx_ctx* ctx, aimx_schedule* s);

/* Number of bounded device waits (copy-completion barriers of the variant-3
 * z-pass) that ran out since the last call, and reset it.  A wait that runs
 * out leaves that product's output incomplete; 0 is the normal answer.
 * Synchronous. */
int aimx_wait_timeouts(int* count);

/* Test hook: the limit, in SM clock cycles, of the per-tile copy wait of the
 * variant-3 z-pass (default about 2e9, a second); cycles <= 0 restores the
 * default.  A short limit makes that wait run out, so a test can check the
 * timeout path (aimx_wait_timeouts > 0, the product's output incomplete, the
 * context still usable).  The wait that drains the copy still in flight after
 * a timeout always keeps the full bound, so no block exits with a bulk copy
 * outstanding.  Process-wide on the current device.  Synchronous. */
int aimx_set_wait_limit(int64_t cycles);

/* Test hook: at most `cap` bases of one grid plane are kept in shared memory by
 * the register inverse-xy kernel of the plane-fused FP32 product (the default,
 * cap <= 0, is whatever fits in 200 KB).  A plane with more bases (a dense mesh
 * on a coarse grid) sums its four fields' interpolation partials in the output
 * array instead; both forms add in the same order, so the product is bitwise
 * the same.  A small cap lets a test run that form on a small mesh.  Host-side
 * setting of ctx, effective from the next product.  Errors: AIMX_E_ARG (null ctx). */
int aimx_set_plane_cap(aimx_ctx* ctx, int cap);

/* Time the FP32 product of nrhs right-hand sides at freq under every candidate
 * schedule (the variants the grid allows x passes {all, nrhs/2, nrhs/4 with at
 * least 4}), two untimed and three timed products each with CUDA events on
 * `stream`, and keep the fastest on the context (the default variant with all
 * RHS in one pass stays unless another is more than 5% faster).  cache_path (may be NULL): a
 * text file of earlier choices keyed by device, grid, padded sizes, fields,
 * bases, near pairs, order, formulation and nrhs; a matching line is applied
 * without timing, and a new choice is appended.  best: the chosen schedule;
 * tried: up to max_tried timed candidates, their count in *ntried (0 on a
 * cache hit).  Allocates two [nrhs][n_unknowns] FP32 work vectors for the
 * duration of the call.  Synchronous.  Errors: AIMX_E_ARG, AIMX_E_IO (cache
 * not writable), AIMX_E_NOMEM, AIMX_E_CUDA; the schedule is unchanged on error. */
int aimx_autotune(aimx_ctx* ctx, double freq, int nrhs, const char* cache_path, aimx_schedule* best,
                  aimx_schedule* tried, int max_tried, int* ntried, void* stream);

/* ------------------------------------------------------------------ profiling
 * Per-stage timing with CUDA events recorded on the stream each stage is
 * launched on (the paper's per-phase accounting, Table II, at kernel level).
 * aimx_profile_read synchronises on the recorded events, writes the summed
 * milliseconds and launch counts of up to max_stages stages, resets them and
 * returns the number of stages the library defines. */
int aimx_profile(aimx_ctx* ctx, int enable);
int aimx_profile_read(aimx_ctx* ctx, double* ms, int64_t* launches, int max_stages);
const char* aimx_profile_stage_name(int stage);

/* ------------------------------------------------------------------ device peak
 * FP32 arithmetic rate of the current device for the ALU roofline of the FFT
 * passes (the paper has no counterpart; a measurement utility).  variant 0:
 * chains of scalar FMAs, 1: packed two-lane FMAs (the form of the register
 * FFTs' butterfly sums).  Runs 8 blocks of 256 threads per SM, 16 independent
 * chains per thread, best of 5 timed launches with CUDA events on the legacy
 * default stream; *tflops = FLOP/s / 1e12 with an FMA counted as 2 FLOPs (a
 * packed FMA as 4).  Synchronous; allocates and frees 16 bytes.  Errors:
 * AIMX_E_ARG (null pointer, unknown variant), AIMX_E_NOMEM, AIMX_E_CUDA. */
int aimx_measure_fp32_peak(int variant, double* tflops);

/* ------------------------------------------------------------------ allocation-free product
 * aimx_matvec_noalloc: the FP32 product y = A(k) x of aimx_matvec (plane-fused
 * path), for callers that must not allocate device memory when they need it,
 * e.g. code working under a fixed memory budget or inside a framework that
 * owns the allocator.  The paper has no counterpart; this is a property of the
 * library, not of the method.
 *   - Allocates nothing: no cudaMalloc / cudaFree / allocating library call.
 *     Its work buffers live in one file-scope static device array of 64 MiB
 *     that every device loading the library holds until the process exits.
 *   - Preconditions: FP32 products of this context take the plane-fused path
 *     (aimx_matvec_path(ctx, AIMX_F32) == 0, i.e. the grid allows it and
 *     neither aimx_set_path nor the schedule selects the generic path) and
 *     aimx_matvec has run once in FP32 on this context (it creates the
 *     kernel-spectra buffers and plane tables that are reused here; a new
 *     frequency then regenerates spectra in place, on the stream).  In
 *     conventional-AIM mode the frequency must be the one whose near entries
 *     were last filled (a new fill would block the host).  Otherwise
 *     AIMX_E_STATE.
 *   - x, y: device [nrhs][nunk] float2, caller-owned, not overlapping.
 *     nrhs is limited by the 64 MiB array; larger requests return AIMX_E_ARG
 *     with the required byte count in aimx_last_error.
 *   - The first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress (once per device, with that device current); make
 *     that first call before any stream capture.
 *   - All calls share the one array and it keeps the previous call's contents
 *     (every kernel writes its whole work region before reading it, so nothing
 *     needs clearing).  Calls whose execution overlaps on the GPU (different
 *     streams, contexts or host threads without ordering) race on the array.
 *   - Asynchronous on stream, like aimx_matvec. */
int aimx_matvec_noalloc(aimx_ctx* ctx, double freq, int nrhs, const void* x, void* y, void* stream);

/* ------------------------------------------------------------------ export (tests) */

/* Copy setup products to host arrays (any pointer may be NULL to skip it).
 * Order and layout follow the caller's RWG numbering:
 *   anchors  int32 [N][3]           stencil start node (x, y, z)
 *   weights  double [N][(n+1)^3][4] projection weights (x, y, z, rho)
 *   row_ptr  int64 [N+1], cols int32 [nnz]  near pairs, columns ascending
 *   na, nphi, nk double [nnz]       near matrices N^A, N^Phi, N^K
 * Synchronous. */
int aimx_export_setup(const aimx_ctx* ctx, int32_t* anchors, double* weights,
                      int64_t* row_ptr, int32_t* cols, double* na, double* nphi, double* nk);

/* ------------------------------------------------------------------ delta-gap ports */

/* A delta-gap port (cited in Sec. VI): the plane through `point` with unit
 * `normal`, restricted to the axis-aligned box [box_lo, box_hi] (one conductor's
 * cut).  Its gap edges are the RWG edges lying in the plane (to 1e-9 of the
 * longest edge) with midpoints inside the box.  The port vector is
 * c_m = l_m s_m on the gap edges, s_m = sign((centroid(T-) - centroid(T+)) . normal):
 * a 1 V gap excites b = c, and the port current of coefficients x is c . x.
 * AIMX_EFIE contexts only (AIMX_E_STATE otherwise); a port with no gap edge is
 * AIMX_E_ARG. */
typedef struct {
    double point[3];
    double normal[3];
    double box_lo[3];
    double box_hi[3];
} aimx_port;

/* Host port vectors c [nport][N] (caller basis order, float64) and gap-edge
 * counts nedges [nport] (either may be NULL).  Synchronous. */
int aimx_port_vectors(aimx_ctx* ctx, int nport, const aimx_port* ports, double* c, int32_t* nedges);
/* b: device complex128 [nport][n_unknowns] = the unit-voltage excitations. */
int aimx_rhs_ports(aimx_ctx* ctx, int nport, const aimx_port* ports, void* b, void* stream);
/* I: host complex128 [nrhs][nport] port currents of device complex128 x [nrhs][n_unknowns].  Synchronous. */
int aimx_port_currents(aimx_ctx* ctx, int nport, const aimx_port* ports, int nrhs, const void* x, void* I,
                       void* stream);
/* Y-parameter sweep: for each frequency solve the nport unit-voltage systems
 * (lockstep GMRES, opts as aimx_solve, warm start from the previous frequency)
 * and write Y [nf][nport][nport] (host complex128, Y[f][i][j] = current at port
 * i for 1 V at port j).  stats: host [nf][nport] or NULL.  Static data and the
 * kernel-generation buffers are reused across the sweep (Sec. III-A).  Returns
 * AIMX_E_NOCONV (> 0) if any system missed the tolerance (Y still written). */
int aimx_sweep_ports(aimx_ctx* ctx, int nf, const double* freqs, int nport, const aimx_port* ports, void* Y,
                     const aimx_solve_opts* opts, aimx_solve_stats* stats, void* stream);

/* ------------------------------------------------------------------ static data (lifecycle) */

/* The frequency-independent setup products of a context (mesh, material,
 * resolved grid, order, FP64 projection weights, precorrected near matrices
 * N^A, N^Phi, N^K and static self terms: the static part that AIMx computes
 * once for all frequencies, Sec. III-A) written to / read from a binary file
 * (native byte order, FNV-1a checksum; version 2 stores the CFIE weight,
 * version 1 files still load).  aimx_load_static rebuilds the
 * topology from the stored mesh and restores the stored arrays instead of
 * recomputing the near integrals; the new context computes the same products
 * bit for bit.  Errors: AIMX_E_ARG (null arguments), AIMX_E_IO (I/O failure,
 * bad magic or version, checksum mismatch, arrays that do not match the
 * mesh), plus the aimx_setup errors on load.  Synchronous. */
int aimx_save_static(const aimx_ctx* ctx, const char* path);
int aimx_load_static(const char* path, aimx_ctx** out);

/* ------------------------------------------------------------------ batches of uneven meshes */

/* A batch of n contexts (different meshes, grids, formulations) whose FP32
 * products are applied together: members run concurrently on `nstreams`
 * internal streams (0 = min(8, n)) and the whole batch is captured into one
 * CUDA graph on the first call, replayed by later calls with the same
 * per-member frequencies, RHS counts and buffer pointers (any change
 * recaptures).  The paper treats one problem at a time; batching many small
 * problems is how a GPU stays busy on them.  The member contexts are borrowed
 * (the caller keeps them alive and does not use them concurrently with the
 * batch); profiling is off inside the graph.
 *   freqs [n] Hz, nrhs [n], x[i] / y[i]: device complex64 [nrhs[i]][n_unknowns_i]
 *   of member i, caller-owned.  Asynchronous on `stream` after the first call
 *   (the first call runs each member once and synchronises to build the graph).
 * Errors: AIMX_E_ARG, AIMX_E_CUDA (capture failed), AIMX_E_NOMEM. */
typedef struct aimx_batch aimx_batch;
int aimx_batch_create(int n, aimx_ctx* const* ctxs, int nstreams, aimx_batch** out);
int aimx_batch_destroy(aimx_batch* b);
int aimx_batch_matvec(aimx_batch* b, const double* freqs, const int* nrhs, const void* const* x, void* const* y,
                      void* stream);
/* Solve A_i(k_i) x_i = b_i for every member i (the members' own aimx_solve with
 * the shared opts): member i runs on internal stream i % nstreams, driven by
 * one host thread per internal stream, so the members' solves overlap on the
 * GPU.  freqs [n], nrhs [n]; B[i], X[i]: device complex128 [nrhs[i]][nunk_i]
 * of member i (X[i] an initial guess when opts->use_x0); stats: host array of
 * n pointers, each to [nrhs[i]] aimx_solve_stats (or NULL), or NULL.  Ordered
 * after `stream`, which is ordered after the batch; synchronous on return.
 * Returns the first member error (aimx_batch_last_error names the member),
 * else AIMX_E_NOCONV if any member missed tol, else AIMX_OK. */
int aimx_batch_solve(aimx_batch* b, const double* freqs, const int* nrhs, const void* const* B, void* const* X,
                     const aimx_solve_opts* opts, aimx_solve_stats* const* stats, void* stream);
int64_t aimx_batch_graph_nodes(const aimx_batch* b);      /* nodes of the captured graph (0 before the first call) */
const char* aimx_batch_last_error(const aimx_batch* b);

/* ------------------------------------------------------------------------
 * Learned near-field preconditioner (no counterpart in the paper, whose
 * preconditioner is the diagonal of L_s, Sec. III-A-2).
 *
 * M = D^{-1} (I + C): D as for AIMX_PRECOND_DIAG, C on the near graph and its
 * diagonal, predicted by a message-passing network of width 64 with `layers`
 * layers.  Reversing an RWG function's orientation flips row and column n of
 * the operator and C_mn -> s_m s_n C_mn; the network respects this exactly:
 * its inputs are orientation invariant and each edge entry is a learned
 * combination of 8 signed bases.  With h the geometric-mean grid spacing, k
 * the exterior wavenumber and N the precorrected static near matrices
 * (Eq. LAIMx):
 *   bases b(m, n): eta^A = N^A_mn / sqrt|N^A_mm N^A_nn|, eta^Phi (same with N^Phi),
 *           eta^K = h N^K_mn / sqrt|N^A_mm N^A_nn|, and the two-hop products
 *           (XY)_mn = sum_j X_mj Y_jn / sqrt(deg_m deg_n) over the near pattern
 *           for XY = AA, PP, AP, PA, KK (deg: off-diagonal near count, >= 1);
 *   node features x_m: l/h, A+/h^2, A-/h^2, basis-centre offset from the
 *           stencil centre in cells (3), k h, refractive contrast (1 for EFIE);
 *   edge features e_mn: (c_n - c_m)/h (3), |c_n - c_m|/h, |eta^A|, |eta^Phi|,
 *           eta^A eta^Phi, |eta^K|, |AA|, |PP|, |AP|, |PA|, |KK|, eta^A AA,
 *           eta^Phi PP, k h.
 * Network:
 *   h0 = relu(A0 x + a0);  h_l = relu(D_l h_m + mean_{n != m} relu(B_l h_n + C_l e_mn + c_l) + d_l);
 *   u_mn = relu(Ua h_m + Ub h_n + Uc e_mn + u);
 *   C_mn[k] = sum_c (E u_mn + f)[8k + c] b_c(m, n) (n != m);  C_mm[k] = G h_m + g,
 * K = 2 outputs (one complex entry, EFIE) or 8 (2x2 complex block, rows
 * (E, H) x columns (J, M), real parts then imaginary parts; two-region form).
 * Parameters are one FP32 vector in the order A0[64][8], a0[64], then per
 * layer B[64][64], C[64][16], c[64], D[64][64], d[64], then Ua[64][64],
 * Ub[64][64], Uc[64][16], u[64], E[8K][64], f[8K], G[K][64], g[K] (matrices
 * row-major [out][in]).  The kernels use the parameters rounded to BF16 and
 * accumulate in FP32.
 *
 * Training minimises the probe loss (1/P) sum_p |M y_p - z_p|^2 / |z_p|^2 over
 * pairs y_p = A z_p supplied by the caller (e.g. from aimx_matvec), P = nprobe.
 * ------------------------------------------------------------------------ */
typedef struct aimx_gnn aimx_gnn;

typedef struct {
    double lr;      /* Adam step size (> 0)                              */
    double beta1;   /* 0 = 0.9                                           */
    double beta2;   /* 0 = 0.999                                         */
    double eps;     /* 0 = 1e-8                                          */
    double clip;    /* global gradient-norm clip (<= 0: none)            */
} aimx_adam_opts;

/* New network for `formulation` (AIMX_EFIE: K = 2, AIMX_PMCHWT: K = 8) with
 * 1..8 layers; parameters start at zero.  The caller destroys it. */
int aimx_gnn_create(int formulation, int layers, aimx_gnn** out);
int aimx_gnn_destroy(aimx_gnn* net);
int64_t aimx_gnn_num_params(const aimx_gnn* net);
/* Host FP32 parameter vector (n = aimx_gnn_num_params) in / out.  Setting
 * parameters resets the Adam state.  Synchronous. */
int aimx_gnn_set_params(aimx_gnn* net, const float* host, int64_t n);
int aimx_gnn_get_params(const aimx_gnn* net, float* host, int64_t n);
/* Probe loss for the context at freq; Z, Y: device complex64 [nprobe][n_unknowns]
 * (caller order), Y = A Z.  grad (host FP32 [num_params], may be NULL) receives
 * the gradient.  Synchronous on `stream`.  AIMX_E_ARG if the network's K does
 * not match the context's formulation. */
int aimx_gnn_loss_grad(aimx_gnn* net, aimx_ctx* ctx, double freq, int nprobe, const void* Z, const void* Y,
                       double* loss, float* grad, void* stream);
/* One Adam step on the probe loss (loss before the step returned). */
int aimx_gnn_train_step(aimx_gnn* net, aimx_ctx* ctx, double freq, int nprobe, const void* Z, const void* Y,
                        const aimx_adam_opts* opt, double* loss, void* stream);
/* Copy the network's current BF16 parameters into the context for
 * AIMX_PRECOND_LEARNED (the network may be destroyed afterwards); NULL detaches.
 * Solving with AIMX_PRECOND_LEARNED and nothing attached returns AIMX_E_STATE. */
int aimx_gnn_attach(aimx_ctx* ctx, const aimx_gnn* net);
/* Inspection (host outputs, any may be NULL): node features [N][8] by caller
 * basis index; edge features [nnz][16], bases [nnz][8], rows[nnz], cols[nnz]
 * (caller indices) in the context's internal near order; network outputs with
 * `net`'s parameters at freq: o [nnz][K] in the same edge order (0 on the
 * diagonal), g [N][K] by caller basis index. */
int aimx_gnn_features(aimx_ctx* ctx, double freq, float* node, float* edge, float* basis, int32_t* rows,
                      int32_t* cols);
int aimx_gnn_outputs(aimx_ctx* ctx, const aimx_gnn* net, double freq, float* o, float* g);

#ifdef __cplusplus
}
#endif
#endif /* AIMX_H */
