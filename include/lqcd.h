/*
 * lqcd.h -- C ABI of the GB300 lattice-QCD fermion library.
 *
 * The library applies the Wilson-Dirac operator and its five-dimensional
 * domain-wall variant (the operators the Grid paper, arXiv:1512.03487,
 * benchmarks in Sec. 3 and lists in Sec. 4), solves M^dag M x = b by
 * even-odd preconditioned conjugate gradient in FP64 or in mixed precision
 * with FP64 reliable updates, and computes the pseudofermion force.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns an int status: LQCD_OK (0) or a negative LQCD_ERR_*
 *    code. lqcd_last_error() gives a thread-local message for the last error.
 *  - Pointers named *_dev are device pointers (cudaMalloc / torch memory)
 *    borrowed for the duration of the call; the caller owns them. Host
 *    pointers (named *_host) are read or written before the call returns
 *    when the call synchronises, otherwise they must stay valid until the
 *    stream reaches the copy. Nothing is allocated on the device by the
 *    library except where a call says so; scratch space is passed in as a
 *    workspace of the size a *_workspace_bytes() query returns.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream. Calls enqueue work on it and return without synchronising
 *    unless stated (the solvers synchronise; they return iteration counts).
 *  - Gamma matrices (chiral basis): gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]
 *    for k = x, y, z, gamma_t = [[0, 1], [1, 0]], gamma_5 = diag(1, 1, -1, -1).
 *
 * Layouts
 * -------
 *  Host ("user") layout, complex FP64 as interleaved (re, im) doubles:
 *    gauge   U[t][z][y][x][mu][row][col]                       (mu = x, y, z, t)
 *    spinor  psi[i5][t][z][y][x][spin][colour]                  (subset LQCD_FULL)
 *            psi[i5][t][z][y][x/2][spin][colour]                (LQCD_EVEN / LQCD_ODD:
 *                                                                sites of one parity in
 *                                                                lexicographic order)
 *    i5 runs over the inner extent n5 (L_s of a domain-wall field, or the
 *    right-hand sides of a multi-RHS field).
 *  Device layout (opaque to callers; produced by the pack calls): one
 *    checkerboard (parity) at a time, structure-of-arrays, site fastest so
 *    that consecutive threads touch consecutive addresses:
 *      spinor  chunk c of site j at chunk_base + c * stride + j, site
 *              j = cb * n5 + i5 (i5 fastest), stride = n_sites rounded up to 32.
 *              FP64: 12 chunks of double2; FP32: 6 chunks of float4;
 *              FP16: 3 chunks of 8 halves followed by one float norm per site
 *              (value = half * norm, norm = max |component| of the site).
 *              A LQCD_FULL field is the even checkerboard followed by the odd.
 *      gauge   [parity][mu][chunk][cb]; 18-real links store the full 3x3
 *              matrix, 12-real links store rows 0 and 1 and rebuild
 *              row 2 = conj(row0 x row1) (exact for SU(3)).
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define LQCD_OK                 0
#define LQCD_ERR_ARG           -1  /* invalid argument (size, alignment, enum) */
#define LQCD_ERR_CUDA          -2  /* a CUDA runtime call failed */
#define LQCD_ERR_NOT_CONVERGED -3  /* solver hit maxiter above the tolerance */
#define LQCD_ERR_NAN           -4  /* a reduction produced NaN / Inf / a non-positive p^dag A p */
#define LQCD_ERR_TIMEOUT       -5  /* solver exceeded its wall-clock limit */
#define LQCD_ERR_UNSUPPORTED   -6  /* valid but not implemented combination */
#define LQCD_ERR_WORKSPACE     -7  /* workspace too small */

/* ---------------------------------------------------------------- enums */
#define LQCD_F64 0   /* storage precision: FP64, FP64 arithmetic */
#define LQCD_F32 1   /* FP32 storage, FP32 arithmetic */
#define LQCD_F16 2   /* FP16 storage (+ FP32 norm per spinor site), FP32 arithmetic */
#define LQCD_F64_DF 3  /* FP64 storage (the LQCD_F64 layout) with double-float arithmetic: each
                          real a pair of FP32 numbers (about 48 bits; results within a few 1e-15
                          of the FP64 arithmetic), for GPUs whose FP64 units are few. An operator
                          precision only (op->prec: lqcd_dslash, lqcd_M, lqcd_MdagM, and for Wilson
                          lqcd_eo_prepare, lqcd_eo_reconstruct); Wilson without G-parity, or domain
                          wall on 18-real links with L_s dividing 32 (LQCD_ERR_UNSUPPORTED
                          otherwise); fields are LQCD_F64 */

#define LQCD_EVEN 0  /* field subset: even checkerboard */
#define LQCD_ODD  1  /* odd checkerboard */
#define LQCD_FULL 2  /* both checkerboards */

#define LQCD_WILSON 0
#define LQCD_DWF    1

#define LQCD_FORCE_TA   0  /* traceless Hermitian F, dS = eps tr(T F) for U -> exp(i eps T) U */
#define LQCD_FORCE_GRAD 1  /* conjugate-Wirtinger gradient G, dS = Re sum conj(dU) G */

/* ---------------------------------------------------------------- structs */

/* Lattice geometry (Grid paper, Sec. 2.4: a Grid object describes a 4D or 5D,
 * possibly single-checkerboard, Cartesian lattice). */
typedef struct {
    int dims[4];     /* Lx, Ly, Lz, Lt; every extent even and >= 2 (checkerboarding:
                        a hop wrapping around an odd extent keeps its parity) */
    int n5;          /* inner extent: L_s (domain wall) or number of RHS; >= 1 */
    double bc[4];    /* boundary phase per direction, +1 (periodic) or -1 */
} lqcd_lattice;

/* Operator parameters. Wilson: D_W = (4 + mass) - H/2. Domain wall (Shamir):
 * D_DW = (5 - M5) - P_- S_up - P_+ S_down - H/2 with mf corners.
 * G-parity (the paper lists G-parity boundary conditions, Sec. 4): with
 * gparity != 0 (Wilson only, n5 = 2 flavours, LQCD_F64 or LQCD_F32) the field
 * holds Psi = (Psi_0, Psi_1) as i5 = 0, 1; flavour 1 couples to the conjugate
 * links U*, and a hop across the boundary of a direction in the mask maps
 * Psi_0 -> +Psi_1, Psi_1 -> -Psi_0 in place of that direction's phase; the
 * forward link belongs to the site, the backward link to its neighbour (whose
 * flavour decides the conjugation). The solvers treat the two flavours as
 * one system. */
typedef struct {
    int kind;        /* LQCD_WILSON or LQCD_DWF */
    double mass;     /* Wilson bare mass m */
    double M5;       /* domain-wall height */
    double mf;       /* domain-wall quark mass */
    int prec;        /* storage precision of the gauge field and spinors */
    int recon;       /* 18 or 12 reals per stored link */
    int gparity;     /* bit mask of G-parity directions: 1 x, 2 y, 4 z, 8 t; 0 = none */
} lqcd_operator;

typedef struct {
    double tol;            /* target true relative residual ||b - A x|| / ||b|| (per RHS) */
    int maxiter;           /* iteration cap (>= 1) */
    int sloppy_prec;       /* LQCD_F64: plain FP64 CG; LQCD_F32 / LQCD_F16: mixed precision */
    int sloppy_recon;      /* 18 or 12: link format of gauge_sloppy */
    double delta;          /* reliable-update threshold on ||r|| / max ||r|| (e.g. 0.1) */
    int check_interval;    /* iterations per captured chunk between host checks (0 = 16) */
    int use_graph;         /* 1: replay chunks as a captured CUDA graph; 0: plain launches */
    double timeout_ms;     /* wall-clock limit; 0 = none */
    double delta_mid;      /* lqcd_cg_solve with sloppy_prec LQCD_F16 only (0 = off): threshold of the
                              intermediate FP32-arithmetic residual replacement (e.g. 0.003); see below */
    int update_prec;       /* mixed solves: arithmetic of the FP64-field operator of the reliable
                              updates (and of lqcd_eo_solve's Wilson source preparation), LQCD_F64 (0,
                              the default) or LQCD_F64_DF (double-float: the true residual b - A x within
                              a few 1e-15 |b| of the FP64 one, about 1.8x faster on GB300). Applies to
                              Wilson operators without G-parity and to domain wall on 18-real links with
                              L_s dividing 32; other operators keep FP64 updates */
    int reserved;          /* 0 */
} lqcd_solver_params;

typedef struct {
    int iterations;           /* inner iterations executed */
    int reliable_updates;     /* FP64 residual recomputations (including the final check) */
    double true_rel_residual; /* max over RHS of ||b - A x|| / ||b|| in FP64 at exit */
    double time_ms;           /* wall time of the solve */
    int status;               /* same as the return value */
    int residual_replacements; /* intermediate FP32-arithmetic replacements (delta_mid) */
} lqcd_solve_info;

/* ---------------------------------------------------------------- library */

/* Version string of the library. */
const char* lqcd_version(void);
/* Message describing the last error on this host thread ("" if none). */
const char* lqcd_last_error(void);
/* Number of kernel launches issued by this library in this process (graph
 * replays count every kernel node they run). */
uint64_t lqcd_launch_count(void);
/* Destroy the CUDA graphs the solver caches across calls (one per distinct
 * set of buffers and parameters, at most 16, least recently used evicted).
 * Call before freeing solver buffers whose addresses may be reused with
 * other meanings, or at shutdown. */
void lqcd_release_caches(void);

/* ---------------------------------------------------------------- sizes */

/* Bytes of a device spinor field (Sec. 2.4 layout transformation: SoA,
 * site fastest). subset: LQCD_EVEN / LQCD_ODD / LQCD_FULL. 0 on bad input. */
size_t lqcd_spinor_bytes(const lqcd_lattice* lat, int prec, int subset);
/* Bytes of a device gauge field (4 directions, both parities). */
size_t lqcd_gauge_bytes(const lqcd_lattice* lat, int prec, int recon);

/* ---------------------------------------------------------------- layout */

/* Convert a spinor in the host layout (already in device memory, src_dev,
 * complex FP64) into the device layout dst_dev of precision prec. FP16
 * rounds each site to the nearest half after scaling by the site norm. */
int lqcd_spinor_pack(void* dst_dev, int prec, int subset, const double* src_dev,
                     const lqcd_lattice* lat, void* stream);
/* Inverse of lqcd_spinor_pack (widening to FP64). */
int lqcd_spinor_unpack(double* dst_dev, const void* src_dev, int prec, int subset,
                       const lqcd_lattice* lat, void* stream);
/* Convert a host-layout FP64 gauge field in device memory to the device
 * layout with prec and recon (12: rows 0, 1 only). */
int lqcd_gauge_pack(void* dst_dev, int prec, int recon, const double* src_dev,
                    const lqcd_lattice* lat, void* stream);
/* Inverse of lqcd_gauge_pack (12-real links are rebuilt). */
int lqcd_gauge_unpack(double* dst_dev, const void* src_dev, int prec, int recon,
                      const lqcd_lattice* lat, void* stream);
/* Host-pointer variants: copy src_host into the device staging buffer
 * staging_dev (at least the host-layout size: 24 doubles per spinor site,
 * 72 per gauge site) with cudaMemcpyAsync, then pack. Unpack variants pack
 * into staging_dev and copy back to dst_host; they synchronise the stream. */
int lqcd_spinor_upload(void* dst_dev, int prec, int subset, const double* src_host,
                       double* staging_dev, const lqcd_lattice* lat, void* stream);
int lqcd_spinor_download(double* dst_host, const void* src_dev, int prec, int subset,
                         double* staging_dev, const lqcd_lattice* lat, void* stream);
int lqcd_gauge_upload(void* dst_dev, int prec, int recon, const double* src_host,
                      double* staging_dev, const lqcd_lattice* lat, void* stream);

/* ---------------------------------------------------------------- operators */

/* Hopping term (Grid paper Sec. 2.6 stencil: spin-project, SU(3) x
 * half-spinor, reconstruct, accumulate; Sec. 3 "Wilson kernel"):
 *   out(x) = sum_mu (1 - gamma_mu) U_mu(x) in(x+mu) + (1 + gamma_mu) U_mu(x-mu)^dag in(x-mu)
 * (dagger = 1 swaps 1 -+ gamma). out_subset LQCD_EVEN / LQCD_ODD: out lives
 * on that checkerboard and in on the other; LQCD_FULL: both are full fields.
 * With n5 > 1 the same links act on every i5 (the "L_s replicated Wilson
 * dslash" of Sec. 3, Table 4; also multi-RHS). gauge_dev and the spinors
 * share op->prec; op->recon selects the link format. out and in must not
 * alias. */
int lqcd_dslash(void* out_dev, const void* in_dev, const void* gauge_dev,
                const lqcd_lattice* lat, const lqcd_operator* op,
                int out_subset, int dagger, void* stream);

/* Dirac operator: the Wilson fermion operator and the five-dimensional chiral
 * (domain-wall) operator the paper lists among its actions (Sec. 4, "Wilson
 * Fermion Action", "Five dimensional chiral fermions") and benchmarks as
 * "Wilson and Domain Wall fermion operators" (Sec. 3). The paper writes
 * neither down; these are the textbook forms. subset LQCD_FULL: out = D in
 *   Wilson  D_W  = (4 + m) - H / 2
 *   DWF     D_DW = M5op - H / 2 (H replicated over L_s, M5op the fifth-
 *           dimension hopping with the mf-twisted wrap).
 * subset LQCD_EVEN: out = M_hat in, the even-odd Schur complement on the
 * paper's single-checkerboard grids (Sec. 2.4):
 *   Wilson  M_hat = (4 + m) - H_eo H_oe / (4 (4 + m))
 *   DWF     M_hat = M5op - H_eo M5op^-1 H_oe / 4
 * with dagger giving the adjoint. tmp_dev: workspace of
 * lqcd_operator_workspace_bytes() bytes. */
int lqcd_M(void* out_dev, const void* in_dev, const void* gauge_dev,
           const lqcd_lattice* lat, const lqcd_operator* op, int subset, int dagger,
           void* tmp_dev, void* stream);
/* out = M^dag M in (subset FULL) or M_hat^dag M_hat in (subset EVEN): the
 * Hermitian positive operator the paper's conjugate gradient (Sec. 4) solves
 * with. */
int lqcd_MdagM(void* out_dev, const void* in_dev, const void* gauge_dev,
               const lqcd_lattice* lat, const lqcd_operator* op, int subset,
               void* tmp_dev, void* stream);
size_t lqcd_operator_workspace_bytes(const lqcd_lattice* lat, const lqcd_operator* op, int subset);

/* Even-odd helpers around a solve on the single-checkerboard grid (Sec. 2.4:
 * the paper's grids may hold one checkerboard; the Schur-complement reduction
 * itself is textbook). FP64 fields; op->prec LQCD_F64 (or LQCD_F64_DF for
 * Wilson; the domain-wall helpers' separate M5op^-1 has no double-float form):
 *   b_hat_e = b_e + H_eo A_oo^-1 b_o / 2            (prepare)
 *   x_o     = A_oo^-1 (b_o + H_oe x_e / 2)          (reconstruct, writes the
 *                                                    odd half of x_full)
 * with A_oo = 4 + m (Wilson) or M5op (DWF). b_full / x_full are LQCD_FULL. */
int lqcd_eo_prepare(void* bhat_even_dev, const void* b_full_dev, const void* gauge_dev,
                    const lqcd_lattice* lat, const lqcd_operator* op, void* tmp_dev, void* stream);
int lqcd_eo_reconstruct(void* x_full_dev, const void* b_full_dev, const void* gauge_dev,
                        const lqcd_lattice* lat, const lqcd_operator* op, void* tmp_dev, void* stream);

/* ---------------------------------------------------------------- solvers */

/* Conjugate gradient (Grid paper Sec. 4 lists CG) for A x = b with
 * A = M^dag M (subset LQCD_FULL) or M_hat^dag M_hat (subset LQCD_EVEN), x0 = 0.
 * x_dev, b_dev: FP64 fields (op->prec == LQCD_F64) of that subset.
 * gauge_dev: FP64 gauge in op->recon. gauge_sloppy_dev: gauge in
 * (params->sloppy_prec, params->sloppy_recon), used by the inner iteration.
 * When sloppy_prec is LQCD_F64 it is ignored (may be NULL): the inner
 * iteration then runs on gauge_dev in op->recon, whatever sloppy_recon says. With a Wilson operator
 * and n5 > 1 every i5 is an independent system (multi-RHS, own scalars,
 * shared link loads); with a domain-wall operator n5 = L_s is one system.
 * Mixed precision: the iteration runs in the sloppy format; x accumulates
 * in FP64; whenever ||r|| falls below delta times its maximum since the last
 * update, or below tol, r = b - A x is recomputed in FP64. Exit only when
 * every system's FP64 true residual is <= tol. Synchronises the stream.
 * Three levels (sloppy_prec LQCD_F16, delta_mid > 0): FP16 storage needs a
 * fresh residual every few decades, so between FP64 updates the iterated
 * residual is replaced by r - A x_s whenever it falls below delta_mid times
 * its maximum since the last replacement, with r the residual of the last
 * FP64 update, x_s the sloppy solution since then, and A applied with FP32
 * arithmetic on an FP32 / 12-real copy of gauge_dev that the solve makes in
 * its workspace; FP64 updates then follow delta,
 * which this allows down to about 1e-5. The solve's result and exit test are
 * unchanged (FP64 true residual); only the update schedule differs. Ignored
 * by the block and batched solvers.
 * workspace_dev: lqcd_cg_workspace_bytes() bytes, 256-byte aligned. */
size_t lqcd_cg_workspace_bytes(const lqcd_lattice* lat, const lqcd_operator* op,
                               const lqcd_solver_params* params, int subset);
int lqcd_cg_solve(void* x_dev, const void* b_dev, const void* gauge_dev,
                  const void* gauge_sloppy_dev, const lqcd_lattice* lat,
                  const lqcd_operator* op, const lqcd_solver_params* params, int subset,
                  lqcd_solve_info* info, void* workspace_dev, size_t workspace_bytes,
                  void* stream);

/* CGNR (CG on the normal equations; the Grid paper lists CG, Sec. 4, for the
 * Wilson and domain-wall operators of Sec. 3): solves M x = b (subset
 * LQCD_FULL) or M_hat x = b (LQCD_EVEN, b = b_hat of lqcd_eo_prepare) by CG on
 * M^dag M x = M^dag b. Every
 * reliable update recomputes the residual of the system itself, s = b - M x,
 * and its norm in FP64 (two FP64 hops for M_hat), and the exit test is on it:
 * ||b - M x|| / ||b|| <= tol, reported as true_rel_residual (CG on M^dag M
 * minimises exactly this norm of the error over its Krylov space). The
 * normal-equation residual M^dag s, which only restarts the iterated
 * recurrence, and the start M^dag b are applied in the inner iteration's
 * arithmetic: FP32 on the workspace's FP32 / 12-real copy of gauge_dev for a
 * mixed solve, FP64 for a plain
 * one. M^dag b is never formed in FP64. Arguments, workspace
 * (lqcd_cg_workspace_bytes), delta, delta_mid and the rest as lqcd_cg_solve. */
int lqcd_cgnr_solve(void* x_dev, const void* b_dev, const void* gauge_dev, const void* gauge_sloppy_dev,
                    const lqcd_lattice* lat, const lqcd_operator* op, const lqcd_solver_params* params,
                    int subset, lqcd_solve_info* info, void* workspace_dev, size_t workspace_bytes,
                    void* stream);

/* Even-odd solve of the full system D x = b (Wilson D_W or domain wall D_DW,
 * the mass-form operators of lqcd_M; single-checkerboard fields as the paper's
 * grids allow them, Sec. 2.4, with CG, Sec. 4): b_hat = b_e - D_eo D_oo^-1 b_o (as
 * lqcd_eo_prepare), CGNR on M_hat x_e = b_hat (lqcd_cgnr_solve), then
 * x_o = D_oo^-1 (b_o - D_oe x_e). Once the odd half is in place the full
 * system's residual b - D x is b_hat - M_hat x_e on the even sites and zero
 * (up to rounding) on the odd ones, so the exit test is ||b_hat - M_hat x_e||
 * <= tol ||b|| with the FP64 b_hat - M_hat x_e of a reliable update and ||b||
 * of the full source: tol applies to the full system, and true_rel_residual
 * reports ||b - D x|| / ||b||. For the Wilson operator the odd half takes
 * H_oe x_e from the last reliable update (the first hop of its M_hat x_e), so
 * it needs no hop of its own. x_dev, b_dev: FP64
 * full fields (x is overwritten, b is not). workspace_dev:
 * lqcd_eo_solve_workspace_bytes() bytes, 256-byte aligned. Returns the solver's
 * status; on LQCD_ERR_NOT_CONVERGED or LQCD_ERR_TIMEOUT x is still the full
 * solution of the last FP64 update. Synchronises the stream. */
size_t lqcd_eo_solve_workspace_bytes(const lqcd_lattice* lat, const lqcd_operator* op,
                                     const lqcd_solver_params* params);
int lqcd_eo_solve(void* x_dev, const void* b_dev, const void* gauge_dev, const void* gauge_sloppy_dev,
                  const lqcd_lattice* lat, const lqcd_operator* op, const lqcd_solver_params* params,
                  lqcd_solve_info* info, void* workspace_dev, size_t workspace_bytes, void* stream);

/* Block CG (O'Leary 1980) for the n5 <= 16 right-hand sides of a Wilson
 * multi-RHS field (subset LQCD_EVEN: M_hat^dag M_hat X = B): one block Krylov
 * space shared by all columns, N x N Gram matrices accumulated in FP64,
 * alpha and beta from Cholesky factorisations on the device, the same
 * sloppy-operator / FP64-reliable-update scheme as lqcd_cg_solve. Converged
 * columns are frozen; a breakdown falls back to per-column steps. Exit when
 * every column's FP64 true residual is <= tol. Arguments as lqcd_cg_solve
 * (no subset argument). */
size_t lqcd_block_cg_workspace_bytes(const lqcd_lattice* lat, const lqcd_operator* op,
                                     const lqcd_solver_params* params);
int lqcd_block_cg_solve(void* x_dev, const void* b_dev, const void* gauge_dev, const void* gauge_sloppy_dev,
                        const lqcd_lattice* lat, const lqcd_operator* op, const lqcd_solver_params* params,
                        lqcd_solve_info* info, void* workspace_dev, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------- batched solves */

/* One lattice of a batched solve: independent Wilson systems of different
 * sizes solved together (the paper's Grid objects of different geometry
 * active at once, Sec. 2.4, with CG of Sec. 4 on each). */
typedef struct {
    lqcd_lattice lat;          /* this instance's geometry; n5 must be 1 */
    double mass;               /* this instance's Wilson bare mass m */
    const void* gauge;         /* FP64 links, device layout, recon as passed to the call */
    const void* gauge_sloppy;  /* links in (sloppy_prec, sloppy_recon); ignored if sloppy_prec is LQCD_F64 */
    void* x;                   /* FP64 even-checkerboard solution (written) */
    const void* b;             /* FP64 even-checkerboard source */
} lqcd_batch_item;

/* Solves M_hat_i^dag M_hat_i x_i = b_i (Wilson, even-odd) for n <= 64
 * instances at once with the CG of lqcd_cg_solve (FP64 or mixed precision,
 * per-instance alpha, beta, reliable updates and convergence). Every phase of
 * an iteration is one persistent launch over a work list of (instance, tile)
 * pairs; the tile size (64, 128 or 256 sites) and the number of resident
 * blocks per SM are chosen together by timing candidates on the first solve
 * of each batch shape (see lqcd_tune_save). infos: n
 * entries (iterations and reliable updates are shared, true residuals are per
 * instance). Synchronises the stream. workspace: lqcd_batch_cg_workspace_bytes()
 * bytes, 256-byte aligned. */
size_t lqcd_batch_cg_workspace_bytes(int n, const lqcd_batch_item* items, int recon,
                                     const lqcd_solver_params* params);
int lqcd_batch_cg_solve(int n, const lqcd_batch_item* items, int recon, const lqcd_solver_params* params,
                        lqcd_solve_info* infos, void* workspace_dev, size_t workspace_bytes, void* stream);

/* The autotuner (the paper tunes its layout to the SIMD width at compile time,
 * Sec. 2.4 "Nsimd"; here launch parameters are timed on the GPU at run time).
 * Its table maps a text key to the integer choice made for it:
 *  - "batch_hop sms=... prec=... recon=... : <dims of every instance>" ->
 *    resident blocks per SM of the persistent batch launch, and "batch_tile"
 *    with the same tail -> its tile size (0: 64, 1: 128, 2: 256 sites and
 *    threads per block), timed together on the first lqcd_batch_cg_solve of
 *    each batch shape;
 *  - "hop prec=P recon=R dagger=D epi=E red=Q full=F lat=XxYxZxT n5=N" ->
 *    launch-shape index of an FP32 / FP16 hop kernel (one site per thread
 *    with 0: 128 threads per block, registers as the compiler chooses; 1: 128
 *    threads and at least 7 resident blocks per SM; 2: as 6 with at least 7
 *    blocks per SM; 3: 128 threads and at least 5 blocks per SM; 4: 128 threads, two sites per
 *    thread in packed FP32x2 arithmetic, 3 blocks per SM; 5: 128 threads,
 *    one site per thread, at least 6 blocks per SM, the eight links of each 4D
 *    site loaded once into shared memory for its n5 threads when n5 >= 4;
 *    6: 128 threads, one site per thread, the two spin components of each
 *    half spinor paired in packed FP32x2 arithmetic; 7 / 8: as 1 / 2 with
 *    each direction's neighbour spinor and link copied asynchronously into a
 *    per-thread ring in shared memory while an earlier direction is computed,
 *    29-37 KB of shared memory per block). All shapes give
 *    bit-identical hop results. A hop key is
 *    timed (a warm-up of every shape, then three interleaved rounds of two
 *    back-to-back launches each on the caller's stream, which is
 *    synchronised; shape 0 is kept unless another is at least 3 % faster
 *    in its fastest round) on its first launch outside
 *    a stream capture when running it again cannot change what it leaves
 *    behind (no reduction, output not aliasing an input); the solvers time
 *    their in-iteration hops (which reduce and are captured in graphs) once
 *    per configuration in a tuning pass on their own workspace before the
 *    first iteration. Untimed keys use shape 0.
 * lqcd_tune_save writes the table to a text file (one "value<TAB>key" line
 * per entry); lqcd_tune_load reads one back (its entries replace current
 * ones; loaded hop keys are never re-timed); lqcd_tune_entries counts the
 * entries; lqcd_tune_get returns the value stored for key, or -1;
 * lqcd_tune_clear forgets every entry (hops are timed again on next use);
 * lqcd_tune_set_enabled(0) stops all timing (untimed keys then keep their
 * default), 1 (the default) allows it. */
int lqcd_tune_save(const char* path);
int lqcd_tune_load(const char* path);
int lqcd_tune_entries(void);
int lqcd_tune_get(const char* key);
void lqcd_tune_clear(void);
void lqcd_tune_set_enabled(int on);

/* ---------------------------------------------------------------- no-allocation operator */

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: code running inside a host callback
 * (cudaLaunchHostFunc), where CUDA calls that allocate are not allowed; code
 * on a latency-critical path, where cudaMalloc's implicit device
 * synchronisation is unacceptable; or a plugin whose host framework owns the
 * whole device memory pool.
 *
 * lqcd_M_noalloc computes exactly what lqcd_M computes (same kernels, same
 * arguments minus tmp_dev): the caller still passes in_dev and out_dev, but
 * the operator's odd-checkerboard temporaries live in one fixed device array
 * of LQCD_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU
 * that loads the library holds until the process exits. The call allocates
 * nothing (no cudaMalloc, cudaFree or allocating library routine).
 *  - Limit: the temporaries (one odd checkerboard field, two for domain wall,
 *    none for subset LQCD_FULL) must fit in the array, e.g. a 24^3 x 48
 *    FP32 or FP16 Wilson Schur operator fits, its FP64 form does not;
 *    larger requests return LQCD_ERR_ARG with a message saying so.
 *  - Set-up: the first call on each device, made with that device current,
 *    looks up the array's device address (cudaGetSymbolAddress) once; make
 *    that first call before any stream capture. After a device reset, call
 *    lqcd_release_caches() before the next call: the array may have moved.
 *  - No timing: this call never runs the launch-shape autotuner (which would
 *    synchronise the stream); it uses the table's shapes or the defaults.
 *  - Sharing: every call on a device uses the same array and the array keeps
 *    the last call's contents. The operator writes its temporaries before
 *    reading them, so nothing has to start at zero, but calls whose work
 *    overlaps on the GPU (different streams, or host threads without
 *    ordering) race on the array: order them on one stream. */
#define LQCD_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
int lqcd_M_noalloc(void* out_dev, const void* in_dev, const void* gauge_dev,
                   const lqcd_lattice* lat, const lqcd_operator* op, int subset, int dagger,
                   void* stream);

/* ---------------------------------------------------------------- colour-matrix fields */

/* Fields of 3x3 complex matrices, one per site (the paper's
 * LatticeColourMatrix), and their site-by-site product z = x * y, the first
 * kernel of the paper's performance section (Sec. 5: SU(3) x SU(3) product of
 * fields, performance against memory footprint).
 *  Sites: every site of the lattice times n5 (no checkerboarding).
 *  Host layout: M[i5][t][z][y][x][row][col], complex FP64 interleaved.
 *  Device layout (produced by lqcd_colour_matrix_pack): structure of arrays,
 *    site fastest, stride = sites rounded up to 32; FP64 9 chunks of double2
 *    (entries row-major); FP32 4 chunks of float4 (entries 0-7) then one
 *    chunk of float2 (entry 8). prec: LQCD_F64 or LQCD_F32 (else
 *    LQCD_ERR_ARG). Pointers must be 16-byte aligned. */
size_t lqcd_colour_matrix_bytes(const lqcd_lattice* lat, int prec);
int lqcd_colour_matrix_pack(void* dst_dev, int prec, const double* src_dev, const lqcd_lattice* lat,
                            void* stream);
int lqcd_colour_matrix_unpack(double* dst_dev, const void* src_dev, int prec, const lqcd_lattice* lat,
                              void* stream);
/* z(s) = x(s) y(s) at every site s (z_ik = sum_j x_ij y_jk), computed in the
 * field precision. z may be x or y (each site is read before it is written).
 * Asynchronous on stream. 198 flop per site. */
int lqcd_su3_mul(void* z_dev, const void* x_dev, const void* y_dev, const lqcd_lattice* lat, int prec,
                 void* stream);

/* ---------------------------------------------------------------- gauge action and HMC */

/* Wilson gauge action, its force and hybrid Monte Carlo (the paper lists HMC,
 * the Wilson gauge action and the leapfrog and minimum-norm integrators among
 * its algorithms, Sec. 4; the formulas are the textbook ones):
 *   S_g = beta sum_{x, mu<nu} (1 - Re tr U_munu(x) / 3), periodic in every direction;
 *   F_g = (beta / 3) traceless[(W - W^dag) / (2 i)], W = U_mu(x) times its staple sum,
 *   so that dS_g = eps tr(T F_g) under U -> exp(i eps T) U (the convention of lqcd_force).
 * Gauge and momentum fields are FP64 in the device layout with recon 18
 * (lqcd_gauge_pack / _unpack); a momentum field holds one traceless Hermitian
 * matrix per link. Calls that return a number reduce through a workspace of
 * lqcd_reduce_workspace_bytes() bytes (256-byte aligned) and synchronise. */
size_t lqcd_reduce_workspace_bytes(const lqcd_lattice* lat);
/* Mean plaquette: the average of Re tr U_munu(x) / 3 over sites and the six planes. */
int lqcd_plaquette(double* plaquette_host, const void* gauge_dev, const lqcd_lattice* lat,
                   void* workspace_dev, size_t workspace_bytes, void* stream);
/* Re <a, b> = Re sum_x a(x)^dag b(x) of two FP64 full spinor fields (n5 = 1),
 * summed in FP64 in a fixed order (deterministic): the pseudofermion action
 * S = phi^dag (M^dag M)^-1 phi = Re <phi, X> of the force's forward pass (HMC,
 * Sec. 4 of the paper; the action of FermionAction). */
int lqcd_spinor_dot_re(double* result_host, const void* a_dev, const void* b_dev, const lqcd_lattice* lat,
                       void* workspace_dev, size_t workspace_bytes, void* stream);
/* Kinetic energy sum over links of tr(P^2) / 2. */
int lqcd_momentum_kinetic(double* kinetic_host, const void* mom_dev, const lqcd_lattice* lat,
                          void* workspace_dev, size_t workspace_bytes, void* stream);
/* out_dev = F_g (must not alias gauge_dev). Asynchronous. */
int lqcd_gauge_force(void* out_dev, const void* gauge_dev, const lqcd_lattice* lat, double beta, void* stream);
/* U <- exp(i eps P) U for every link (FP64 Taylor series with scaling and squaring). Asynchronous. */
int lqcd_gauge_exp_update(void* gauge_dev, const void* mom_dev, double eps, const lqcd_lattice* lat,
                          void* stream);

#define LQCD_LEAPFROG 0  /* P(eps/2) U(eps) P(eps) ... U(eps) P(eps/2) */
#define LQCD_MINNORM2 1  /* per step P(l eps) U(eps/2) P((1-2l) eps) U(eps/2) P(l eps), l = 0.1931833 */

typedef struct {
    double beta;     /* Wilson gauge coupling */
    double tau;      /* trajectory length; eps = tau / nsteps */
    int nsteps;      /* molecular-dynamics steps (>= 1) */
    int integrator;  /* LQCD_LEAPFROG or LQCD_MINNORM2 */
    int fermion;     /* 1: add one Wilson pseudofermion S_f = phi^dag (M^dag M)^-1 phi */
} lqcd_hmc_params;

typedef struct {
    double H0, H1;              /* Hamiltonian K + S_g + S_f before and after the trajectory */
    double kinetic0, kinetic1;
    double gauge0, gauge1;
    double fermion0, fermion1;
    int force_evaluations;      /* momentum steps: nsteps + 1 (leapfrog), 2 nsteps + 1 (min. norm) */
    int cg_iterations;          /* summed over every solve of the trajectory */
    int status;
} lqcd_hmc_info;

/* One molecular-dynamics trajectory of hybrid Monte Carlo: integrates
 * dU/dt = i P U, dP/dt = -(F_g + F_f) over tau, updating gauge_dev and
 * mom_dev in place, and reports H before and after. The caller draws the
 * momenta (density exp(-tr P^2 / 2) on traceless Hermitian matrices) and the
 * pseudofermion phi = M^dag eta (eta of density exp(-eta^dag eta)), and makes
 * the accept / reject decision with exp(H0 - H1), keeping a copy of the gauge
 * field to restore on rejection. op: Wilson, LQCD_F64, recon 18, n5 = 1;
 * phi_dev: FP64 LQCD_FULL spinor (ignored without fermion). Every fermion
 * force solves M^dag M X = phi on the full lattice with lqcd_cg_solve and
 * params (sloppy_prec LQCD_F64 or LQCD_F32; the sloppy links are repacked
 * from the updated field before each solve). Synchronises. */
size_t lqcd_hmc_workspace_bytes(const lqcd_lattice* lat, const lqcd_operator* op,
                                const lqcd_solver_params* params);
int lqcd_hmc_trajectory(void* gauge_dev, void* mom_dev, const void* phi_dev, const lqcd_lattice* lat,
                        const lqcd_operator* op, const lqcd_hmc_params* hmc,
                        const lqcd_solver_params* params, lqcd_hmc_info* info,
                        void* workspace_dev, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------- multigrid */

/* Two-level adaptive multigrid for the Wilson operator (the paper shows the
 * coarse-grid operator of an adaptive multigrid inverter as its stencil
 * example, Sec. 2, and lists multigrid-preconditioned solvers, Sec. 4).
 * Aggregates are blocks of block^4 fine sites (block 2 or 4, dividing every
 * extent) split by chirality (spins 0, 1 / 2, 3); a coarse site carries
 * Nc = 2 nvec complex components ordered (chirality, k). Fine vector sets:
 * nvec full-lattice spinors (n5 = 1) in the device layout at consecutive
 * field offsets. Coarse vectors: [coarse site][Nc] complex (FP64 double2 or
 * FP32 float2), coarse sites lexicographic with x fastest. Coarse operator:
 * [9][coarse site][Nc][Nc], d = 0 self, 1 + 2 mu the +mu and 2 + 2 mu the -mu
 * neighbour, with (D_c c)(X) = sum_d Y_d(X) c(X + d). All calls asynchronous
 * except lqcd_mg_solve. */
typedef struct {
    int block;         /* aggregate extent in every direction: 2 or 4 */
    int nvec;          /* near-null vectors, 1..32 */
    int setup_iters;   /* CG iterations on M^dag M v = random, per vector */
    int pre_smooth;    /* MR steps before the coarse correction */
    int post_smooth;   /* MR steps after it */
    int coarse_iters;  /* fixed CGNR iterations of the coarse solve */
    int restart;       /* flexible-GCR restart length (>= 4) */
} lqcd_mg_params;

size_t lqcd_mg_coarse_bytes(const lqcd_lattice* lat, int nvec, int block, int prec);
size_t lqcd_mg_coarse_op_bytes(const lqcd_lattice* lat, int nvec, int block, int prec);
/* In place: per aggregate and chirality, modified Gram-Schmidt of the nvec FP64 vectors. */
int lqcd_mg_block_orthonormalize(void* vecs_dev, int nvec, int block, const lqcd_lattice* lat, void* stream);
/* coarse = P^dag fine and fine = P coarse, with P = vecs (orthonormalised); prec F64 or F32 for all three. */
int lqcd_mg_restrict(void* coarse_dev, const void* fine_dev, const void* vecs_dev, int nvec, int block, int prec,
                     const lqcd_lattice* lat, void* stream);
int lqcd_mg_prolong(void* fine_dev, const void* coarse_dev, const void* vecs_dev, int nvec, int block, int prec,
                    const lqcd_lattice* lat, void* stream);
/* Y = the Galerkin coarse operator P^dag D_W P (FP64) from the FP64 gauge field
 * (op: Wilson, LQCD_F64, recon 18; boundary phases from lat) and FP64 vecs. */
int lqcd_mg_coarse_build(void* Y_dev, const void* gauge_dev, const void* vecs_dev, int nvec, int block,
                         const lqcd_lattice* lat, const lqcd_operator* op, void* stream);
/* out = D_c in (dagger 0) or D_c^dag in (dagger 1), in the precision prec of Y, in and out (out != in). */
int lqcd_mg_coarse_apply(void* out_dev, const void* in_dev, const void* Y_dev, int nvec, int block, int prec,
                         int dagger, const lqcd_lattice* lat, void* stream);
/* Solver: lqcd_mg_setup computes nvec near-null vectors from the caller's
 * random FP64 full-lattice fields (setup_iters CG iterations on M^dag M each),
 * orthonormalises them and builds the coarse operator, all inside the
 * workspace; lqcd_mg_solve then solves D_W x = b (FP64 full-lattice fields) by
 * refinement cycles: r = b - D x in FP64, then flexible GCR in FP32 on D c = r
 * (up to `restart` vectors, until |r| drops 1e-5-fold or below tol),
 * preconditioned by an FP32 V-cycle (MR smoothing, restriction, coarse_iters
 * CGNR iterations on D_c, prolongation, MR smoothing) replayed as one CUDA
 * graph, and x += c in FP64; it returns when the FP64 true residual
 * |b - D x| / |b| <= params->tol.
 * gauge64: FP64 18-real; gauge32: FP32 12-real of the same field. The
 * workspace (lqcd_mg_workspace_bytes, 256-byte aligned) must have gone
 * through lqcd_mg_setup with the same lattice, operator and parameters.
 * info->iterations counts preconditioned GCR iterations. Synchronises. */
size_t lqcd_mg_workspace_bytes(const lqcd_lattice* lat, const lqcd_operator* op, const lqcd_mg_params* mg);
int lqcd_mg_setup(const void* gauge64_dev, const void* gauge32_dev, const double* random_vectors_dev,
                  const lqcd_lattice* lat, const lqcd_operator* op, const lqcd_mg_params* mg,
                  void* workspace_dev, size_t workspace_bytes, void* stream);
int lqcd_mg_solve(void* x_dev, const void* b_dev, const void* gauge64_dev, const void* gauge32_dev,
                  const lqcd_lattice* lat, const lqcd_operator* op, const lqcd_mg_params* mg,
                  const lqcd_solver_params* params, lqcd_solve_info* info, void* workspace_dev,
                  size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------- force */

/* Pseudofermion force for S = phi^dag (M^dag M)^-1 phi with M = D_W (Grid
 * paper Sec. 4 lists HMC; formula is the textbook derivative):
 *   X = (M^dag M)^-1 phi, Y = M X (FP64 LQCD_FULL fields, n5 == 1),
 *   A = sum_spin X(x+mu) ((1 - gamma_mu) Y(x))^dag,
 *   B = sum_spin ((1 + gamma_mu) X(x)) Y(x+mu)^dag,  both times the link's boundary phase,
 *   kind LQCD_FORCE_GRAD: out = A^dag + B               (dS = Re sum conj(dU) out)
 *   kind LQCD_FORCE_TA:   out = TA[i (U A - B U^dag - h.c.) / 2]  (traceless Hermitian)
 * out_dev: FP64 gauge field in the device layout with recon 18 (unpack it
 * with lqcd_gauge_unpack). gauge_dev: FP64, op->recon. */
int lqcd_force(void* out_dev, const void* gauge_dev, const void* X_dev, const void* Y_dev,
               const lqcd_lattice* lat, const lqcd_operator* op, int kind, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LQCD_H */
