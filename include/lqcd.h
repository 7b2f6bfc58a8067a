/*
 * lqcd.h - C ABI of the B300 (sm_103a) distillation solver for the domain-decomposition
 * subtraction estimator of quark-line disconnected correlators ("Subtraction method for
 * disconnected diagrams in full QCD", Barca, Crawford, Finkenrath, Schaefer, Urrea-Nino).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice: extents L[4] = {Lx, Ly, Lz, Lt}, all even, Lt <= 256; volume V = Lx Ly Lz Lt;
 *   lexicographic site s = x + Lx (y + Ly (z + Lz t)); directions mu = 0..3 = x, y, z, t.
 * Complex numbers are interleaved (re, im) doubles.
 * Gauge links:  links[s][mu][a][b]                (V * 4 * 9 complex)
 * Spinors:      psi[r][s][spin][colour]            (nrhs * V * 12 complex)
 * Colour vecs:  V[k][i][s3][colour], s3 = x + Lx (y + Ly z)   (k indexes the timeslices passed)
 * Dirac basis: Euclidean chiral, gamma_k = [[0,-i sigma_k],[i sigma_k,0]], gamma_t = [[0,1],[1,0]],
 *   gamma_5 = gamma_x gamma_y gamma_z gamma_t = diag(1,1,-1,-1).  The paper's gamma_0 is gamma_t.
 * Operator (Sec. 2.1 and Sec. 3 of the paper: Wilson-clover; normalisation fixed here):
 *   D = A - kappa H,
 *   (H psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu),
 *   A = 1 + i kappa c_sw sum_{mu<nu} sigma_{mu nu} Fhat_{mu nu},  sigma = (i/2)[gamma_mu, gamma_nu],
 *   Fhat = (Q - Q^dag)/8 with Q the four-leaf clover; fermion boundary phase on the t-hop
 *   between t = Lt-1 and 0 (LQCD_BC_*), spatially periodic.
 * Domain operator D_Lambda (Sec. 2.1, Dirichlet restriction): the time axis is tiled from t = 0
 *   by consecutive domains (lqcd_set_domains); D_Lambda is D with every t-hop between two
 *   different domains removed, the clover term unchanged; it is block diagonal over domains.
 *
 * Memory: the caller owns every buffer it passes.  `where` says whether the data pointers of a
 * call are host (LQCD_HOST) or device (LQCD_DEVICE, e.g. torch.Tensor.data_ptr()) memory;
 * device pointers must belong to the context's device.  Calls are ordered on the stream given
 * to lqcd_create / lqcd_set_stream; host-pointer calls return after their results are in host
 * memory, device-pointer calls return after the work is queued on that stream.
 * Errors: every function returns LQCD_OK (0) or an LQCD_ERR_* code and leaves a message for
 * lqcd_last_error; on LQCD_ERR_INVALID_ARG nothing was done.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lqcd_ctx lqcd_ctx;

enum {
  LQCD_OK = 0,
  LQCD_ERR_INVALID_ARG = 1,
  LQCD_ERR_NOT_CONVERGED = 2,
  LQCD_ERR_CUDA = 3,
  LQCD_ERR_OOM = 4,
  LQCD_ERR_TIMEOUT = 5,
  LQCD_ERR_NAN = 6,
  LQCD_ERR_STATE = 7
};

enum { LQCD_BC_PERIODIC = 0, LQCD_BC_ANTIPERIODIC = 1, LQCD_BC_OPEN = 2 };
enum { LQCD_HOST = 0, LQCD_DEVICE = 1 };
enum { LQCD_MODE_FULL = 0, LQCD_MODE_DOMAIN = 1 };
enum { LQCD_SINKS_DIAG = 0, LQCD_SINKS_ALL = 1, LQCD_SINKS_DIAG_SRCV = 2 };

/* Krylov solvers.  All are judged by the true residual ||b - D x|| / ||b|| of the
 * unpreconditioned operator computed from the FP64 fields (per right-hand side, and per domain for
 * domain solves; the residual's arithmetic is lqcd_solve_params.residual):
 *   LQCD_SOLVER_BICGSTAB64: even-odd preconditioned BiCGStab entirely in FP64 (the plain solver);
 *   LQCD_SOLVER_MIXED:      FP64 defect correction around an FP32 even-odd BiCGStab
 *                           (inner_prec = LQCD_PREC_F32) or an FP32 flexible GCR preconditioned
 *                           by FP16-storage BiCGStab sweeps (inner_prec = LQCD_PREC_F16);
 *   LQCD_SOLVER_FGCR_NN:    FP64 defect correction around FP32 flexible GCR preconditioned by the
 *                           loaded gauge-covariant network (lqcd_nn_load); falls back to MIXED
 *                           when no network is loaded or it fails to reduce the residual.
 * With use_graph = 1 a batch's whole solve (defect-correction cycles and inner iterations) is one
 * CUDA graph whose loops run on the device (conditional WHILE nodes): no host round trip until the
 * batch ends.  Where the driver refuses such a graph, the library drives the cycles from the host,
 * replaying captured chunks of check_every inner iterations. */
enum {
  LQCD_SOLVER_BICGSTAB64 = 0,
  LQCD_SOLVER_MIXED = 1,
  LQCD_SOLVER_FGCR_NN = 2
};
/* LQCD_PREC_DF: FP64 fields with double-float arithmetic; used by the true-residual kernel only
 * (lqcd_tune_dslash / lqcd_set_dslash_variant tune and set that kernel's launch variant). */
enum { LQCD_PREC_F64 = 0, LQCD_PREC_F32 = 1, LQCD_PREC_F16 = 2, LQCD_PREC_DF = 3 };

typedef struct {
  double tol;        /* target true relative residual per RHS (and per domain); 0 -> 1e-10 */
  int max_iter;      /* cap on inner Krylov iterations summed over restarts; 0 -> 20000 */
  int solver;        /* LQCD_SOLVER_* */
  int inner_prec;    /* LQCD_PREC_F32 or LQCD_PREC_F16 (MIXED / FGCR_NN) */
  int rhs_block;     /* right-hand sides per batched launch; 0 -> chosen by the library */
  int use_graph;     /* 1: replay Krylov iterations from a captured CUDA graph */
  double inner_tol;  /* residual reduction per defect-correction cycle; 0 -> default */
  int max_outer;     /* cap on defect-correction cycles; 0 -> 20 */
  int check_every;   /* Krylov iterations between convergence checks; 0 -> 1 for batches of at
                        least 2^22 (site, RHS) pairs per parity, up to 8 for smaller ones */
  int gcr_nkrylov;   /* flexible GCR restart length; 0 -> 8 */
  int precond_iters; /* FP16 MR preconditioner sweeps per application; 0 -> 6; < 0: no preconditioner
                        (plain FP32 GCR inside the defect correction, for comparisons) */
  int pipeline;      /* right-hand-side batches in flight at once: 1 or 2; 0 -> 1.  With 2, a call
                        of several batches keeps two sets of work vectors (twice the solver memory)
                        on two streams, so one batch's FP64 true residual runs beside the next
                        batch's FP32 iterations; results are the same as with 1 */
  int projection;    /* perambulator projection V^dag X: 0 double-float arithmetic (pairs of floats,
                        48-bit significands, FP64 accumulation every 512 terms) on the FP32 pipe;
                        1 native FP64.  Both agree to about 1e-13 relative */
  int residual;      /* arithmetic of the defect correction's true residual b - D x (read from and
                        written to the FP64 fields): 0 double-float (pairs of floats, 48-bit
                        significands) on the FP32 pipe; 1 native FP64.  The double-float residual
                        errs by about 1e-13 of ||b|| + ||D|| ||x||, far below any tolerance >= 1e-12,
                        for entries of magnitude 2^-74 (5e-23) to 2^127; use 1 for fields outside
                        that range */
} lqcd_solve_params;

typedef struct {
  /* caller-provided output arrays (either may be NULL) */
  int* iters;               /* [nrhs] inner Krylov iterations, summed over cycles */
  double* true_resid;       /* [nrhs * n_seg] final FP64 true relative residual, seg fastest */
  /* filled by the library (accumulated over the batches of one call) */
  int n_seg;                /* 1 for full solves, number of domains for domain solves */
  int outer_cycles;         /* largest number of defect-correction cycles of a batch */
  long long total_iters;    /* inner iterations summed over batches */
  long long dslash_calls;   /* half-lattice hopping-term launches */
  double max_true_resid;    /* largest final true relative residual */
  double seconds;           /* wall time of the call */
  int fallback;             /* 1 if FGCR_NN fell back to MIXED */
  int device_loops;         /* batches that ran as one graph with device-side loops (the rest were
                               driven from the host) */
} lqcd_solve_stats;

/* Fill *p with the defaults (tol 1e-10, BiCGStab64, graphs on). */
void lqcd_default_params(lqcd_solve_params* p);

/* Create a context for extents L[4] on the current CUDA device; bc_t = LQCD_BC_*; stream is a
 * cudaStream_t (NULL = legacy default stream).  *out receives the context or NULL.
 * Errors: INVALID_ARG (odd or non-positive extent, Lt > 256), CUDA. */
int lqcd_create(lqcd_ctx** out, const int L[4], int bc_t, void* stream);
int lqcd_destroy(lqcd_ctx* ctx);
int lqcd_set_stream(lqcd_ctx* ctx, void* stream);
/* Free the device work buffers the context keeps between calls (solver vectors, scratch) and the
 * CUDA graphs captured on them, after waiting for the context's queued work.  The next call that
 * needs them allocates them again.  For callers that make large allocations of their own between
 * library calls.  The gauge field, clover and network weights stay.  Errors: INVALID_ARG (NULL). */
int lqcd_release_workspace(lqcd_ctx* ctx);
/* Message of the last error on this context; with ctx = NULL, of the last failed call that takes
 * no context (lqcd_create, lqcd_disc_correlator_noalloc). */
const char* lqcd_last_error(const lqcd_ctx* ctx);

/* Upload gauge links and set kappa, c_sw (Sec. 3: Wilson-clover).  Builds the clover term A and
 * A^{-1} in FP64 on the GPU and the FP32 / FP16 link and clover copies used by the mixed solvers.
 * links: [V][4][3][3] complex, host or device per `where`.  A new kappa drops the context's
 * captured solver graphs (they hold kappa by value).  Errors: INVALID_ARG (NULL, non-finite
 * kappa or c_sw), NAN (a clover block with no inverse, e.g. a NaN or Inf link; the context then
 * holds no usable gauge field). */
int lqcd_gauge_upload(lqcd_ctx* ctx, const double* links, int where, double kappa, double c_sw);

/* Tile the time axis by n_dom domains of the given extents, starting at t = 0 (Sec. 2.1; the
 * paper's regions Lambda_0, Lambda_1 of width Delta).  Errors: INVALID_ARG if an extent < 1 or
 * they do not sum to Lt (nothing changed). */
int lqcd_set_domains(lqcd_ctx* ctx, const int* extents, int n_dom);

/* The same tiling shifted to start at timeslice t_start: domain d covers
 * t_start + (e_0 + ... + e_{d-1}) + [0, e_d) modulo Lt, so the last domain may wrap around the
 * time boundary.  Shifted tilings place the regions Lambda_0, Lambda_1 of width Delta around the
 * chosen x0, y0 (Sec. 2.1, Fig. 1; Sec. 4 chooses Delta per separation).  The Dirichlet cuts sit
 * between consecutive domains, the antiperiodic (or open) boundary phase stays on the t-hop
 * from Lt-1 to 0, and every domain-mode call (solves, perambulators, correlator validity) uses the
 * shifted domains.  lqcd_set_domains(ctx, e, n) = lqcd_set_domains_at(ctx, 0, e, n).  Errors:
 * INVALID_ARG (as lqcd_set_domains, or t_start outside [0, Lt); nothing changed). */
int lqcd_set_domains_at(lqcd_ctx* ctx, int t_start, const int* extents, int n_dom);

/* out = D in (domain_restricted = 0) or out = D_Lambda in (1), FP64, nrhs spinors. */
int lqcd_dirac_apply(lqcd_ctx* ctx, const double* in, double* out, int nrhs, int domain_restricted,
                     int where);

/* The even-odd preconditioned operator the solvers iterate on, in the storage precision prec
 * (LQCD_PREC_F64 / F32 / F16; the dslash launch variant tuned for prec and nrhs):
 *   out_e = M in_e,  M = 1 - kappa^2 A_ee^{-1} H_eo A_oo^{-1} H_oe   (D = A - kappa H, Sec. 3),
 * with the domain cuts of D_Lambda when domain_restricted = 1.  in / out: [nrhs][V][4][3] complex
 * (lexicographic, as lqcd_dirac_apply); the odd sites of in are ignored and those of out are set
 * to zero.  FP32 / FP16 round in to the storage precision and compute in FP32.  Not an operation
 * of the paper's method itself: the Schur complement is the solvers' internal operator, exposed
 * for verification of the reduced-precision kernels.  Errors: INVALID_ARG (NULL, nrhs < 1, bad
 * prec), STATE (no gauge field), OOM, TIMEOUT (staged launch variant). */
int lqcd_schur_apply(lqcd_ctx* ctx, int prec, const double* in, double* out, int nrhs, int domain_restricted,
                     int where);

/* Solve D x = b (full) or D_Lambda x = b (domain; every domain of every RHS converged to tol
 * relative to its own source norm) for nrhs right-hand sides; x is overwritten.  Returns
 * NOT_CONVERGED (x holds the last iterate, stats filled) if tol is not reached, and NAN if a
 * right-hand side (or one domain of it) has a non-finite residual, e.g. a NaN or Inf in its
 * source: its true_resid entry is NaN, and every other right-hand side is still solved to tol
 * and written to x (the systems are independent).  NAN outranks NOT_CONVERGED. */
int lqcd_solve_full(lqcd_ctx* ctx, const double* b, double* x, int nrhs, int where,
                    const lqcd_solve_params* p, lqcd_solve_stats* st);
int lqcd_solve_domain(lqcd_ctx* ctx, const double* b, double* x, int nrhs, int where,
                      const lqcd_solve_params* p, lqcd_solve_stats* st);

/* Distillation perambulators (Sec. 3.1): for each source timeslice t in t_src and each
 * (j, beta), solve with the source delta_{x0,t} e_beta (x) v_j(t) and project the solution on
 * the sink timeslice(s): tau(t',t)^{ij}_{alpha beta} = sum_{xvec,a} v_i(t')^* X(t',xvec,alpha,a).
 * mode FULL uses D, mode DOMAIN uses D_Lambda with one source timeslice per domain solved at
 * once (multi-site sources, Sec. 4).  sinks DIAG: t' = t only; ALL: every t' (FULL mode).
 *   Vt:  [Lt][n_ev][Lx Ly Lz][3] complex colour vectors of every timeslice;
 *   tau: DIAG -> [n_tsrc][n_ev][4][n_ev][4]; ALL -> [n_tsrc][Lt][n_ev][4][n_ev][4] complex,
 *        index order (sink vector i, sink spin alpha, source vector j, source spin beta).
 *   sinks DIAG_SRCV: as DIAG, but Vt holds only the colour vectors of the source timeslices,
 *        [n_tsrc][n_ev][Lx Ly Lz][3] in t_src order (no timeslice may repeat); the diagonal
 *        perambulators need no other timeslice, and at large Lt the full array would not fit.
 * st (may be NULL): only the aggregate fields are filled; st->iters and st->true_resid are
 * not written.
 * Errors: INVALID_ARG (n_ev < 1 or > 3 Lx Ly Lz, t out of range, ALL with DOMAIN, a repeated
 * timeslice with DIAG_SRCV).  NAN: a non-finite residual (NaN or Inf in the inputs); every
 * other right-hand side is still solved and written. */
int lqcd_perambulator(lqcd_ctx* ctx, const double* Vt, int n_ev, const int* t_src, int n_tsrc,
                      int mode, int sinks, int where, double* tau, const lqcd_solve_params* p,
                      lqcd_solve_stats* st);

/* lqcd_perambulator restricted to the source vectors j in [j0, j0 + nj), all four source spins
 * each (4 nj right-hand sides per source group): the columns (j, beta) of tau with j in that range
 * are written and every other entry of tau is left as it was (host tau is read back first).
 * Serves callers that spread the N_ev x 4 right-hand sides of a timeslice over several calls
 * (checkpointing, sharding, bounded work per call).  Same layouts and errors as
 * lqcd_perambulator, plus INVALID_ARG when j0 < 0, nj < 1 or j0 + nj > n_ev. */
int lqcd_perambulator_cols(lqcd_ctx* ctx, const double* Vt, int n_ev, const int* t_src, int n_tsrc,
                           int mode, int sinks, int j0, int nj, int where, double* tau,
                           const lqcd_solve_params* p, lqcd_solve_stats* st);

/* Quark loops from diagonal perambulators (Sec. 2 loop definition with the elementals of
 * Sec. 3.2): L_G(t) = sum_i w_i sum_{alpha beta} G_{alpha beta} tau^{ii}_{beta alpha}(t,t) and the
 * same with G~ = gamma_t G^dag gamma_t.  gamma_ids[n_gamma] index the Clifford table
 *   0: 1, 1-4: gamma_x,y,z,t, 5: gamma_5, 6-9: gamma_mu gamma_5, 10-15: sigma_{xy,xz,xt,yz,yt,zt}.
 * weights: [n_t][n_ev] real (NULL = 1).  L, Lt: [n_gamma][n_t] complex. */
int lqcd_loops(lqcd_ctx* ctx, const double* tau, int n_ev, int n_t, const int* gamma_ids,
               int n_gamma, const double* weights, double* L, double* Lt, int where);

/* Disconnected correlators over n_cfg configurations (Eqs. Cdisc, correlator_factorised,
 * subtracted_correlator, corr1-corr4):
 *   C[g][x0][y0]  = <L(x0) Lt(y0)> - <L(x0)><Lt(y0)>   (vev = 1; vev = 0 drops the product term)
 *   Cdd           = same with the domain loops (completely factorised term)
 *   dC            = C - Cdd;  valid[x0][y0] = dom(x0) != dom(y0)
 *   C_avg[g][dt]  = mean over y0 of C((y0+dt) mod Lt, y0); dC_avg over valid y0 only
 *   terms (optional, may be NULL): [4][n_gamma][Lt][Lt] the four pieces of Eqs. corr1-corr4.
 * Inputs L, Lt, Ld, Ltd: [n_cfg][n_gamma][Lt] complex; uses the context's domain tiling.
 * Errors: INVALID_ARG (n_cfg < 1, vev = 1 with n_cfg = 1). */
int lqcd_disc_correlator(lqcd_ctx* ctx, const double* L, const double* Lt, const double* Ld,
                         const double* Ltd, int n_cfg, int n_gamma, int vev, double* C, double* Cdd,
                         double* dC, double* C_avg, double* dC_avg, int* valid, int* n_valid,
                         double* terms, int where);

/* Averages over source positions restricted to a bulk window, as the paper does on its
 * open-boundary ensemble (Sec. 3: x0 and y0 both in the bulk, 24a..71a of 96 in Sec. 4):
 *   C_avg[g][dt]  = mean over y0 with t_lo <= y0 and y0 + dt <= t_hi of C[g][y0 + dt][y0]
 *                   (no wrap-around: dt = x0 - y0 >= 0 inside the window),
 *   dC_avg[g][dt] = the same mean over the pairs with valid[y0 + dt][y0] != 0 only,
 *   n_pairs[dt], n_valid[dt]: the number of pairs in each mean (0 where none; the mean is 0 then).
 * C, dC: [n_gamma][Lt][Lt] complex indexed [g][x0][y0] and valid [Lt][Lt] as lqcd_disc_correlator
 * writes them; C_avg, dC_avg: [n_gamma][Lt] complex; n_pairs, n_valid: [Lt] int.
 * Errors: INVALID_ARG (NULL, n_gamma < 1, not 0 <= t_lo <= t_hi < Lt). */
int lqcd_window_average(lqcd_ctx* ctx, const double* C, const double* dC, const int* valid, int n_gamma,
                        int t_lo, int t_hi, double* C_avg, double* dC_avg, int* n_pairs, int* n_valid,
                        int where);

/* Quark-line connected correlator of Eq. Cfull with distilled quark lines, from all-sink
 * perambulators (lqcd_perambulator with LQCD_SINKS_ALL, full mode):
 *   C[g][x0][k] = - Tr[ Gamma tau(x0, y0) Gamma~ tau(y0, x0) ],  y0 = t_src[k],
 * trace over eigenvector and spin, Gamma~ = gamma_t Gamma^dag gamma_t, tau(y0, x0) =
 * gamma_5 tau(x0, y0)^dag gamma_5 (gamma_5-hermiticity of D), and the minus sign of the fermion
 * loop; C_avg[g][dt] = mean over k of C[g][(t_src[k] + dt) mod Lt][k] (may be NULL).
 * tau_all: [n_t][Lt][n_ev][4][n_ev][4] complex (sink t', sink eigvec, sink spin, source eigvec,
 * source spin), C: [n_gamma][Lt][n_t], C_avg: [n_gamma][Lt].  gamma_ids index the 16 Clifford
 * elements as in lqcd_loops.  Errors: INVALID_ARG (sizes, t_src or gamma ids out of range), OOM. */
int lqcd_conn_correlator(lqcd_ctx* ctx, const double* tau_all, int n_ev, const int* t_src, int n_t,
                         const int* gamma_ids, int n_gamma, double* C, double* C_avg, int where);

/* Noise-reduced estimator (Sec. 4): the full correlator of Eq. Cfull with the disconnected part
 * replaced by the subtracted one of the block size Delta chosen for each separation,
 *   C_nr[g][dt] = C_conn_avg[g][dt] + dC_avg[d][g][dt],   d = delta_of_dt[dt] >= 0,
 *               = C_conn_avg[g][dt] + C_disc_avg[g][dt],  d = -1 (standard estimator).
 * C_conn_avg, C_disc_avg, C_nr: [n_gamma][Lt]; dC_avg: [n_delta][n_gamma][Lt], the dC_avg outputs
 * of lqcd_disc_correlator for n_delta tilings (NULL if n_delta = 0); delta_of_dt: [Lt] host array.
 * Errors: INVALID_ARG (an index outside [-1, n_delta)). */
int lqcd_nr_estimator(lqcd_ctx* ctx, const double* C_conn_avg, const double* C_disc_avg, const double* dC_avg,
                      int n_delta, int n_gamma, const int* delta_of_dt, double* C_nr, int where);

/* APE smearing of the spatial links for the distillation vectors (Sec. 3.1 computes them on
 * APE-smeared links; the paper gives no parameters, so they are inputs).  n_iter steps of
 *   X_k(x) = (1 - alpha) U_k(x) + (alpha/4) sum_{j != k spatial} [U_j(x) U_k(x+j) U_j(x+k)^dag
 *                                                + U_j(x-j)^dag U_k(x-j) U_j(x-j+k)],
 *   U'_k(x) = X W-projected onto SU(3): W = X (X^dag X)^(-1/2) divided by det(W)^(1/3)
 * (principal root), k = x, y, z, in FP64, starting from the uploaded links each call.  The
 * smeared field is kept in the context and used by lqcd_laplace_eigs until the next
 * lqcd_gauge_upload or a call with n_iter = 0.  The Dirac operator never uses it.  Errors:
 * INVALID_ARG (n_iter < 0, alpha outside [0, 1]), STATE (no gauge field), NAN (a staple sum with
 * no polar factor). */
int lqcd_ape_smear(lqcd_ctx* ctx, double alpha, int n_iter);

/* The smeared spatial links: out [V][3 (k = x, y, z)][3][3] complex, site order of the links.
 * Errors: STATE (no smeared field). */
int lqcd_smeared_links(lqcd_ctx* ctx, double* out, int where);

/* Distillation vectors (Sec. 3.1, 3.2): the n_ev lowest eigenpairs of the gauge-covariant 3D
 * Laplacian  (-Lap phi)(x) = sum_k [2 phi(x) - U_k(x) phi(x+k) - U_k(x-k)^dag phi(x-k)]  on every
 * timeslice of the uploaded gauge field (of its APE-smeared spatial links after lqcd_ape_smear),
 * to residual ||(-Lap) v - lambda v|| <= tol (0 -> 1e-10).
 *   V:      [Lt][n_ev][Lx Ly Lz][3] complex, unit norm, largest-modulus component (first on ties)
 *           made real positive;   lambda: [Lt][n_ev] real, ascending per timeslice.
 *   iters (may be NULL): filter iterations of the slowest timeslice chunk.
 * Errors: INVALID_ARG (n_ev < 1 or > 3 Lx Ly Lz), STATE (no gauge field), NOT_CONVERGED. */
int lqcd_laplace_eigs(lqcd_ctx* ctx, int n_ev, double* V, double* lambda, int where, double tol, int* iters);

/* Time the even-odd hopping kernel with the fused inverse-clover epilogue,
 * out_o = A_oo^{-1} H_oe in_e (one half of the Schur operator of Sec. 2.1's block form), on
 * nrhs right-hand sides in precision prec (LQCD_PREC_*), over n_iter launches on the context's
 * work stream with CUDA events.  flush_l2 = 1 writes a 256 MB buffer between launches so every
 * launch reads its operands from HBM (the flush is outside the timed intervals).
 *   ms_per_launch:        average kernel duration [ms]
 *   algo_bytes_per_launch: Vh * (8 links + clover + 2 * nrhs spinors) in the stored formats
 *                          (ideal reuse: every input read once, output written once).
 * With prec = LQCD_PREC_DF it times the defect correction's true-residual kernel instead,
 * out = z - (A y - kappa H x) with x = y = z = the input, in double-float arithmetic on the FP64
 * fields: algo_bytes_per_launch = Vh * (8 links + clover + 4 * nrhs FP64 spinors).
 * Fills the input with deterministic non-zero data.  Needs a gauge field.  Errors: INVALID_ARG. */
int lqcd_dslash_bench(lqcd_ctx* ctx, int prec, int nrhs, int n_iter, int flush_l2, double* ms_per_launch,
                      double* algo_bytes_per_launch);

/* lqcd_disc_correlator without any GPU memory allocation, for callers that cannot allocate:
 * hosts that reserve all device memory up front and forbid later allocations, or loops where an
 * allocation would synchronise the device.  (The paper has no counterpart; this is an
 * interface for such callers.)  Same results as lqcd_disc_correlator for the same inputs.
 *   All array arguments are DEVICE pointers on the current device, owned by the caller, with
 *   the layouts of lqcd_disc_correlator; T = Lt; dom_of_t: [T] int domain index of each
 *   timeslice (the tiling of lqcd_set_domains); stream: cudaStream_t the work is queued on
 *   (the call returns once it is queued).
 *   Scratch: the differences L - Ld and Lt - Ltd needed for `terms` live in a fixed 2 MiB
 *   device array compiled into the library (held on every GPU that loads the library until the
 *   process exits), so n_cfg * n_gamma * T must not exceed 65536 when terms != NULL
 *   (INVALID_ARG otherwise, with a message for lqcd_last_error(NULL)).  Every call shares that
 *   array: calls whose GPU work overlaps (different streams, or threads) race on it; each call
 *   writes all the scratch it reads, so nothing needs clearing between calls.
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 *   make that first call before any stream capture.
 * Errors: INVALID_ARG (NULL, sizes, vev with n_cfg = 1, T > 256), CUDA. */
int lqcd_disc_correlator_noalloc(const double* L, const double* Lt, const double* Ld, const double* Ltd, int n_cfg,
                                 int n_gamma, int T, const int* dom_of_t, int vev, double* C, double* Cdd, double* dC,
                                 double* C_avg, double* dC_avg, int* valid, int* n_valid, double* terms,
                                 void* stream);

/* ---- Learned preconditioner (not in the paper: an accelerator of the solves of Sec. 4, whose
 * results it cannot change because the FP64 true residual still decides convergence).
 * A gauge-covariant network of four linear parallel-transport layers, channel widths
 * 4 -> 8 -> 8 -> 8 -> 4 (colour-vector channels; the four spin components of a spinor in and out):
 *   out_o(x) = sum_{p=0..8} sum_c W[p][o][c] (T_p h_c)(x),  T_0 = 1,
 *   T_{1+mu} h(x) = U_mu(x) h(x+mu),  T_{5+mu} h(x) = U_mu(x-mu)^dag h(x-mu),
 * on the fermion links (boundary phase; Dirichlet cuts when domain = 1).  Weights: complex, stored
 * per layer as [9][C_out][C_in], layers one after the other, as (re, im) float pairs; inference
 * reads a BF16 copy and accumulates in FP32, training updates FP32 master weights with Adam.
 * Fields for lqcd_nn_apply / lqcd_nn_loss_grad: [n][V][4][3] complex64 (FP32 re, im), full lattice. */
int lqcd_nn_num_weights(void); /* number of complex weights */
int lqcd_nn_set_weights(lqcd_ctx* ctx, const float* w);  /* host, 2 * lqcd_nn_num_weights() floats */
int lqcd_nn_get_weights(lqcd_ctx* ctx, float* w);
/* out = network(in) with the FP32 master weights. */
int lqcd_nn_apply(lqcd_ctx* ctx, const float* in, float* out, int nsamp, int domain, int where);
/* out = network(in) on the inference path the FGCR preconditioner uses: the BF16 weight copy and
 * BF16-rounded activations, channel mixing on the tensor cores (tcgen05, FP32 accumulation in
 * tensor memory), transports on the CUDA cores in FP32.  Same layouts as lqcd_nn_apply.  Errors as
 * lqcd_nn_apply, plus TIMEOUT (a tensor-core completion wait ran out of its iteration limit). */
int lqcd_nn_apply_tc(lqcd_ctx* ctx, const float* in, float* out, int nsamp, int domain, int where);
/* Loss sum |N(in) - target|^2 / sum |target|^2 over all sites (even_only = 1: even sites) and its
 * gradient dL/dconj(W) (host, 2 * lqcd_nn_num_weights() floats; may be NULL). */
int lqcd_nn_loss_grad(lqcd_ctx* ctx, const float* in, const float* target, int nsamp, int domain, int even_only,
                      int where, double* loss, float* grad);
/* The same loss and gradient computed by the BF16 training kernels that lqcd_nn_train runs:
 * forward and backward-data layers on the tensor cores (BF16 weights and activations, FP32
 * accumulation), transported activations stored in BF16 for the weight gradient (FP32
 * accumulation).  Agrees with lqcd_nn_loss_grad to BF16 rounding. */
int lqcd_nn_loss_grad_bf16(lqcd_ctx* ctx, const float* in, const float* target, int nsamp, int domain,
                           int even_only, int where, double* loss, float* grad);
/* Train on n_pairs (r, e) pairs of the even-odd Schur system M e = r generated from random r
 * (seeded) by the solver without the network (FP64 defect correction around FP32 BiCGStab, true
 * residual 1e-8): pools of pairs that fit a quarter of the free device memory are generated in
 * turn, and each pool gets `epochs` passes of Adam (learning rate lr) over batches of `batch`
 * pairs, loss over even sites; loss_hist[epochs] (may be NULL) receives the mean loss per epoch
 * (averaged over the pools).
 * Starts from the weights set before (lqcd_nn_set_weights).  Afterwards LQCD_SOLVER_FGCR_NN uses
 * the network.  Errors: STATE (no weights or no gauge field), OOM. */
int lqcd_nn_train(lqcd_ctx* ctx, int n_pairs, int epochs, int batch, double lr, int domain, unsigned seed,
                  double* loss_hist);

/* Autotuning of the dslash launch: time the hopping kernel of precision prec on nrhs right-hand
 * sides in its compiled variants and keep the fastest for this context; every later dslash launch
 * of that precision and RHS count uses it.  Variants 0 / 1 / 2: direct loads with register caps
 * of 128 / 80 / 64 per thread (4 / 6 / 8 resident 128-thread blocks per SM); 3: links rebuilt and
 * clover copied once per site into shared memory, 32-bit indexing, register cap 80 (FP32 and
 * FP16, nrhs a power of two in [8, 128]); 4: the neighbour spinors staged in shared memory by
 * bulk asynchronous copies 3 hops ahead (FP32 and FP16, nrhs a multiple of 32); 5: as 3 with the
 * hopping arithmetic on paired FP32 instructions (two lanes per fused multiply-add); 6: as 3 with
 * each thread's neighbour spinors copied asynchronously one hop ahead into shared memory; 7: two
 * right-hand sides per thread on paired FP32 instructions (6 and 7: FP32 only, 7: nrhs >= 16).
 * Where a variant does
 * not apply it runs as variant 0.  FP64 has variants 0 / 1 / 2 with register caps 128 / 255 / 168;
 * LQCD_PREC_DF (the true-residual kernel, timed as such) variants 0 / 1 / 2 with caps 255 / 168 /
 * 128.  All variants compute the same arithmetic (variant 5 may order the two products of an
 * imaginary part differently; so may 7).  lqcd_set_dslash_variant
 * installs a known choice (e.g. from a cache) without timing.  Errors: INVALID_ARG (variant
 * outside 0..7), STATE (no gauge), TIMEOUT (a staged copy did not complete within its wait
 * limit; the solvers report the same). */
int lqcd_tune_dslash(lqcd_ctx* ctx, int prec, int nrhs, int* best_variant, double* best_ms);
int lqcd_set_dslash_variant(lqcd_ctx* ctx, int prec, int nrhs, int variant);

/* Per-phase GPU time of this context's calls (prepare, inner Krylov, reconstruct, FP64 true
 * residual, sources, projection, ...) as a JSON object {"phase": milliseconds, ...} written to
 * buf (len bytes); reset = 1 clears the totals.  Timing is recorded only when the environment
 * variable LQCD_PHASE_TIMING=1 was set when the context was created (it adds CUDA events around
 * phases outside captured graphs).  Errors: INVALID_ARG (buffer too small). */
int lqcd_phase_times(lqcd_ctx* ctx, char* buf, int len, int reset);

/* Number of CUDA kernels this library has put on GPU queues in this process (all contexts):
 * direct launches plus the kernel nodes of every replayed CUDA graph.  For accounting only. */
long long lqcd_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif
