// Krylov solver driver for the full operator D and the Dirichlet domain operator D_Lambda
// (Sec. 2.1; the paper's "inversions", Sec. 4).
//
// Every solve is an FP64 defect-correction loop judged by the FP64 true residual of the
// unpreconditioned operator, per system (one right-hand side, or one domain of one right-hand
// side: because D_Lambda is block diagonal over domains, a multi-site source with one source
// timeslice per domain is as many independent systems, each with its own Krylov scalars):
//
//   x = 0, r = b
//   repeat while some system has ||r|| > tol ||b||:
//     rhat_e = A_ee^-1 (r_e + kappa H_eo A_oo^-1 r_o)          (even-odd Schur right-hand side)
//     solve  M e_e = rhat_e,  M = 1 - kappa^2 A_ee^-1 H_eo A_oo^-1 H_oe,  to relative residual delta
//     e_o = A_oo^-1 (r_o + kappa H_oe e_e);  x += e;  r = b - D x  (FP64)
//
// The inner solve is BiCGStab run in lockstep over all systems of the batch, in FP64 (the plain
// solver), FP32, or FP16 storage with FP32 arithmetic; its right-hand side is rescaled to unit
// norm per system.  The prepare / reconstruct steps run in the inner precision (their errors are
// relative to the correction, not to x); only r = b - D x needs FP64.  One BiCGStab iteration is
// 10 launches with all scalars on the device: the two dot products of each Schur apply are
// fused into its second dslash.  Chunks of iterations are captured once into a CUDA graph and
// replayed, with a host convergence check (one 4-byte read) between chunks.
#include <chrono>
#include <cmath>
#include <cstring>

#include "lqcd_blas.h"
#include "lqcd_distill.h"

namespace lqcd {

size_t spinor_bytes(const Geom& g, int prec, int nrhs) {
  return (size_t)g.Vh * nrhs * 12 * (prec == P64 ? 16 : (prec == P32 ? 8 : 4));
}
size_t clover_bytes(const Geom& g, int prec) {
  return (size_t)g.Vh * 2 * (prec == P64 ? 18 * 16 : (prec == P32 ? 9 * 16 : 9 * 8));
}
size_t link_bytes(const Geom& g, int prec) {
  return (size_t)g.Vh * 8 * (prec == P64 ? 9 * 16 : (prec == P32 ? 3 * 16 : 3 * 8));
}

static inline void* off(void* base, size_t b, int p) { return reinterpret_cast<char*>(base) + b * p; }
static inline const void* off(const void* base, size_t b, int p) {
  return reinterpret_cast<const char*>(base) + b * p;
}

static DslashCall call(lqcd_ctx* c, int prec, int epi, const void* in, const void* y, const void* z, void* out,
                       const void* U, const void* C, int out_par, int nrhs, double a, double b,
                       const signed char* tc) {
  DslashCall k{prec, epi, 0, in, y, z, out, U, C, out_par, nrhs, a, b, tc};
  k.coord = coord_of(c, out_par);
  return k;
}

void apply_D(lqcd_ctx* c, const double2* in, double2* out, int nrhs, int domain, cudaStream_t st) {
  const size_t sb = spinor_bytes(c->g, P64, nrhs), cbb = clover_bytes(c->g, P64);
  for (int p = 0; p < 2; p++) {
    DslashCall k = call(c, P64, EPI_CY_H, off(in, sb, 1 - p), off(in, sb, p), nullptr, off(out, sb, p), c->U64,
                        off(c->A64, cbb, p), p, nrhs, 1.0, -c->kappa, domain ? c->d_tc_dom : c->d_tc_full);
    launch_dslash(c->g, k, st);
  }
}

// dst = M src; the second dslash also forms the partial sums `red` (RED_DOT_Z with zred, or
// RED_DOT_Y_NORM with y = src) for the following BiCGStab scalar.
static void schur(lqcd_ctx* c, const Inner& in, const void* src, void* dst, int red, const void* zred,
                  cudaStream_t st) {
  DslashCall k1 = call(c, in.prec, EPI_CH, src, nullptr, nullptr, in.tmp, in.U, in.Ainv_o, 1, in.nrhs, 0.0, 1.0,
                       in.tc);
  launch_dslash(c->g, k1, st, in.variant);
  DslashCall k2 = call(c, in.prec, EPI_Y_CH, in.tmp, src, nullptr, dst, in.U, in.Ainv_e, 0, in.nrhs, 1.0,
                       -in.kappa * in.kappa, in.tc);
  k2.red = red;
  k2.zred = zred;
  k2.partial = in.partial;
  k2.red_sites = in.vg.S;
  launch_dslash(c->g, k2, st, in.variant);
}

// y_e = M x_e for one parity block of FP64 even-odd fields (x64, y64: [chunk][cb][rhs] of the
// even parity), computed in storage precision P with the tuned launch variant.
int schur_apply(lqcd_ctx* c, int P, const void* x64, void* y64, int nrhs, int domain, cudaStream_t st) {
  const Geom& g = c->g;
  const VGeom vgH = make_vgeom(g, nrhs, 1);
  const size_t sbP = spinor_bytes(g, P, nrhs);
  const void* xin = x64;
  void* out = y64;
  if (P != P64) {
    void* xp = ws_get(c, "sa_in", sbP);
    out = ws_get(c, "sa_out", sbP);
    if (!xp || !out) return set_error(c, LQCD_ERR_OOM, "schur_apply: out of device memory");
    v_convert(P64, P, x64, xp, vgH, c->d_seg_full, 1, nullptr, st);
    xin = xp;
  }
  void* tmp = ws_get(c, "sa_tmp", sbP);
  if (!tmp) return set_error(c, LQCD_ERR_OOM, "schur_apply: out of device memory");
  const void* U = P == P64 ? c->U64 : (P == P32 ? c->U32 : c->U16);
  const void* Ainv = P == P64 ? c->Ainv64 : (P == P32 ? c->Ainv32 : c->Ainv16);
  const size_t cbP = clover_bytes(g, P);
  const signed char* tc = domain ? c->d_tc_dom : c->d_tc_full;
  const auto tv = c->tuned_variant.find((long)P * 100000 + nrhs);
  const int variant = tv != c->tuned_variant.end() ? tv->second : 0;
  DslashCall k1 = call(c, P, EPI_CH, xin, nullptr, nullptr, tmp, U, off(Ainv, cbP, 1), 1, nrhs, 0.0, 1.0, tc);
  launch_dslash(g, k1, st, variant);
  DslashCall k2 = call(c, P, EPI_Y_CH, tmp, xin, nullptr, out, U, off(Ainv, cbP, 0), 0, nrhs, 1.0,
                       -c->kappa * c->kappa, tc);
  launch_dslash(g, k2, st, variant);
  if (P != P64) v_convert(P, P64, out, y64, vgH, c->d_seg_full, 1, nullptr, st);
  return LQCD_OK;
}

static void bicg_iteration(lqcd_ctx* c, const Inner& in, cudaStream_t st) {
  const int P = in.prec;
  schur(c, in, in.p, in.v, RED_DOT_Z, in.b, st);  // v = M p, partial (r0, v)
  bicg_fin_alpha_only(in.partial, in.partial2, in.nchunk, in.vg, in.si, in.nseg, in.ks, st);
  bicg_s(P, in.r, in.v, in.s, in.vg, in.si, in.nseg, in.ks, st);
  // t = M s, partial (t, s), (t, t), (r0, t), (r0, s), (s, s): the iteration's last reduction
  schur(c, in, in.s, in.t, RED_TS_R0, in.b, st);
  bicg_tail(P, in.x, in.p, in.s, in.t, in.r, in.v, in.partial, in.partial2, in.nchunk, in.vg, in.si, in.nseg,
            in.ks, st);
}

static std::string graph_key(const Inner& in, int chunk) {
  char buf[512];
  snprintf(buf, sizeof buf, "bicg:%d:%d:%d:%d:%d:%d:%p:%p:%p:%p:%p:%p:%p:%p:%p:%p:%p:%p:%p:%p", in.prec, in.nrhs,
           in.nseg, chunk, in.variant, in.nchunk, in.b, in.x, in.r, in.p, in.v, in.s, in.t, in.tmp,
           (void*)in.ks.rho, in.partial, (void*)in.partial2, (const void*)in.tc, (const void*)in.si, in.U);
  return buf;
}

static cudaGraphExec_t capture(lqcd_ctx* c, const std::string& key, int nsys, const KState& ks, int* count_host,
                               const std::function<void(cudaStream_t)>& body) {
  cudaStream_t st = c->work;
  auto f = c->graphs.find(key);
  if (f != c->graphs.end()) return f->second;
  cudaGraph_t graph;
  cudaGraphExec_t exec = nullptr;
  set_capturing(true);
  cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  body(st);
  count_active(ks.active, nsys, ks.count, st);
  cudaMemcpyAsync(count_host, ks.count, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaError_t ce = cudaStreamEndCapture(st, &graph);
  set_capturing(false);
  if (ce == cudaSuccess && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
    c->graphs[key] = exec;
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(graph, nodes.data(), &nn);
    long long nk = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      cudaGraphNodeGetType(nd, &ty);
      nk += ty == cudaGraphNodeTypeKernel;
    }
    c->graph_kernels[exec] = nk;
  } else {
    exec = nullptr;
    cudaGetLastError();
  }
  if (ce == cudaSuccess) cudaGraphDestroy(graph);
  return exec;
}

// Run BiCGStab on the prepared systems until all are inactive or max_iter; returns iterations.
static int run_bicg(lqcd_ctx* c, const Inner& in, int max_iter, int chunk, bool use_graph, int* count_host,
                    long long& dslash_calls) {
  cudaStream_t st = c->work;
  const int nsys = in.nrhs * in.nseg;
  auto body = [&](cudaStream_t s) {
    for (int k = 0; k < chunk; k++) bicg_iteration(c, in, s);
  };
  cudaGraphExec_t exec = use_graph ? capture(c, graph_key(in, chunk), nsys, in.ks, count_host, body) : nullptr;
  int it = 0;
  while (it < max_iter) {
    if (exec) {
      cudaGraphLaunch(exec, st);
      count_launch(c->graph_kernels[exec]);
    } else {
      body(st);
      count_active(in.ks.active, nsys, in.ks.count, st);
      cudaMemcpyAsync(count_host, in.ks.count, sizeof(int), cudaMemcpyDeviceToHost, st);
    }
    it += chunk;
    dslash_calls += 4LL * chunk;
    cudaStreamSynchronize(st);
    if (*count_host == 0) break;
  }
  return it;
}

// ------------------------------------------------------------------ flexible GCR
enum { PREC_NONE = 0, PREC_MR16 = 1, PREC_NN = 2 };

struct Fgcr {
  int m;          // restart length
  VecList Z, W;   // FP32 search directions and their images
  void* x;        // FP32 solution (even half of the correction field)
  void* r;        // FP32 residual
  GState gs;
  int kind;       // PREC_*
  int n_mr;       // MR sweeps of the FP16 preconditioner
  Inner in16;     // FP16 Schur operator (U16, Ainv16) and its work vectors
  void *e16, *r16, *p16;
  double2* omega16;
};

// z = K r
static void precondition(lqcd_ctx* c, const Inner& in, const Fgcr& f, void* z, cudaStream_t st) {
  if (f.kind == PREC_MR16) {
    const Inner& h = f.in16;
    v_convert(P32, P16, f.r, f.r16, in.vg, in.si, in.nseg, f.gs.pscale, st);
    v_zero(P16, f.e16, in.vg, st);
    for (int i = 0; i < f.n_mr; i++) {
      schur(c, h, f.r16, f.p16, RED_DOT_Y_NORM, nullptr, st);  // p = M r, partial (p, r), (p, p)
      mr_finish(h.partial, in.vg, in.si, in.nseg, f.omega16, f.gs.active, st);
      mr_update(P16, f.e16, f.r16, f.p16, in.vg, in.si, in.nseg, f.omega16, f.gs.active, st);
    }
    v_convert(P16, P32, f.e16, z, in.vg, in.si, in.nseg, f.gs.ipscale, st);
  } else if (f.kind == PREC_NN) {
    nn_precondition(c, in, f.r, z, f.gs.pscale, f.gs.ipscale, st);
  } else {
    v_copy(P32, f.r, z, in.vg, st);
  }
}

static void fgcr_cycle(lqcd_ctx* c, const Inner& in, const Fgcr& f, cudaStream_t st) {
  for (int k = 0; k < f.m; k++) {
    precondition(c, in, f, f.Z.v[k], st);
    schur(c, in, f.Z.v[k], f.W.v[k], RED_NONE, nullptr, st);
    gcr_orthogonalise(P32, f.W, f.Z, k, f.r, in.vg, in.si, in.nseg, in.partial, f.gs, st);
    gcr_update(P32, f.x, f.r, f.Z.v[k], f.W.v[k], in.vg, in.si, in.nseg, in.partial, f.gs, st);
  }
}

// Run restarted FGCR(m) until all systems are inactive or max_iter; returns iterations.
static int run_fgcr(lqcd_ctx* c, const Inner& in, const Fgcr& f, int max_iter, bool use_graph, int* count_host,
                    long long& dslash_calls) {
  cudaStream_t st = c->work;
  const int nsys = in.nrhs * in.nseg;
  auto body = [&](cudaStream_t s) { fgcr_cycle(c, in, f, s); };
  char key[256];
  snprintf(key, sizeof key, "fgcr:%d:%d:%d:%d:%d:%p:%p:%p:%p:%p", f.m, f.kind, f.n_mr, in.nrhs, in.nseg, f.x,
           f.Z.v[0], (void*)f.gs.beta, (const void*)in.tc, c->nn_weights);
  GState gs_count = f.gs;
  KState ks_count = in.ks;
  ks_count.active = gs_count.active;
  ks_count.count = gs_count.count;
  cudaGraphExec_t exec = use_graph ? capture(c, key, nsys, ks_count, count_host, body) : nullptr;
  int it = 0;
  const long long per_cycle = (long long)f.m * (2 + (f.kind == PREC_MR16 ? 2 * f.n_mr : 0));
  while (it < max_iter) {
    if (exec) {
      cudaGraphLaunch(exec, st);
      count_launch(c->graph_kernels[exec]);
    } else {
      body(st);
      count_active(gs_count.active, nsys, gs_count.count, st);
      cudaMemcpyAsync(count_host, gs_count.count, sizeof(int), cudaMemcpyDeviceToHost, st);
    }
    it += f.m;
    dslash_calls += per_cycle;
    cudaStreamSynchronize(st);
    if (*count_host == 0) break;
  }
  return it;
}

int solve_batch(lqcd_ctx* c, const double2* b, double2* x, int nrhs, int domain, const lqcd_solve_params& prm,
                BatchStats& bs) {
  cudaStream_t st = c->work;
  const Geom& g = c->g;
  const SegInfo* si = domain ? c->d_seg_dom : c->d_seg_full;
  const int nseg = domain ? c->seg_dom.nseg : 1;
  const int nsys = nrhs * nseg;
  const signed char* tc = domain ? c->d_tc_dom : c->d_tc_full;
  const double tol = prm.tol > 0 ? prm.tol : 1e-10;
  const int max_iter = prm.max_iter > 0 ? prm.max_iter : 20000;
  const int max_outer = prm.max_outer > 0 ? prm.max_outer : 20;
  const int chunk = prm.check_every > 0 ? prm.check_every : 8;

  int P = P64;
  // Residual reduction asked of one inner solve.  FP32 BiCGStab on a unit-norm right-hand side
  // reaches a true residual of a few 1e-7 before rounding stalls it, so asking 2e-6 makes two
  // defect-correction cycles enough for 1e-10 (each FP64 cycle costs two FP64 dslash launches).
  // MIXED with FP16 inner precision and FGCR_NN run FP32 flexible GCR whose preconditioner is
  // FP16-storage MR sweeps or the learned network (MR if no network is loaded).
  double inner_tol = 1e-12;
  bool use_gcr = false;
  int pkind = PREC_NONE;
  if (prm.solver == LQCD_SOLVER_MIXED || prm.solver == LQCD_SOLVER_FGCR_NN) {
    P = P32;
    inner_tol = 2e-6;
    if (prm.solver == LQCD_SOLVER_FGCR_NN) {
      use_gcr = true;
      pkind = c->nn_weights ? PREC_NN : PREC_MR16;
      if (!c->nn_weights) bs.fallback = 1;
    } else if (prm.inner_prec == LQCD_PREC_F16) {
      use_gcr = true;
      pkind = PREC_MR16;
    }
    if (use_gcr && prm.precond_iters < 0) pkind = PREC_NONE;  // unpreconditioned FGCR (reference runs)
  }
  if (prm.inner_tol > 0) inner_tol = prm.inner_tol;

  VGeom vgF = make_vgeom(g, nrhs, 2);  // full lattice
  VGeom vgH = make_vgeom(g, nrhs, 1);  // one parity
  if (vgH.threads() > 128) return set_error(c, LQCD_ERR_INVALID_ARG, "solve: rhs_block > 128");
  const size_t sb64 = spinor_bytes(g, P64, nrhs), sbP = spinor_bytes(g, P, nrhs);
  const size_t cbP = clover_bytes(g, P);

  // FP64 outer fields and per-system bookkeeping
  double2* r64 = (double2*)ws_get(c, "o_r64", 2 * sb64);
  // per-(block, rhs) partial sums: 3 for BiCGStab / norms on the full lattice, up to 2 x 16 for the
  // GCR Gram rows on one parity
  size_t npart = std::max((size_t)vgF.blocks * nrhs * 3, (size_t)vgH.blocks * nrhs * 2 * LQCD_GCR_MAXK);
  double* partial = (double*)ws_get(c, "partial", npart * sizeof(double));
  double* b2 = (double*)ws_get(c, "o_b2", nsys * sizeof(double));
  double* r2 = (double*)ws_get(c, "o_r2", nsys * sizeof(double));
  double* delta = (double*)ws_get(c, "o_delta", nsys * sizeof(double));
  double* scale = (double*)ws_get(c, "o_scale", nsys * sizeof(double));
  double* iscale = (double*)ws_get(c, "o_iscale", nsys * sizeof(double));
  double* rel = (double*)ws_get(c, "o_rel", nsys * sizeof(double));
  int* oact = (int*)ws_get(c, "o_active", nsys * sizeof(int));
  // inner fields (precision P)
  void* rin = ws_get(c, "i_rin", 2 * sbP);  // scaled residual, full lattice
  void* ein = ws_get(c, "i_ein", 2 * sbP);  // correction, full lattice (even part = inner x)
  Inner in;
  in.prec = P;
  in.nrhs = nrhs;
  in.nseg = nseg;
  in.vg = vgH;
  in.si = si;
  in.tc = tc;
  in.U = P == P64 ? c->U64 : (P == P32 ? c->U32 : c->U16);
  const void* Ainv = P == P64 ? c->Ainv64 : (P == P32 ? c->Ainv32 : c->Ainv16);
  in.Ainv_e = off(Ainv, cbP, 0);
  in.Ainv_o = off(Ainv, cbP, 1);
  void* bhat = ws_get(c, "i_bhat", sbP);
  in.b = bhat;
  in.x = ein;  // even half of the full correction field
  in.r = ws_get(c, "i_r", sbP);
  in.p = ws_get(c, "i_p", sbP);
  in.v = ws_get(c, "i_v", sbP);
  in.s = ws_get(c, "i_s", sbP);
  in.t = ws_get(c, "i_t", sbP);
  in.tmp = ws_get(c, "i_tmp", sbP);
  in.kappa = c->kappa;
  in.variant = 0;
  {
    auto it = c->tuned_variant.find((long)P * 100000 + nrhs);
    if (it != c->tuned_variant.end()) in.variant = it->second;
  }
  char* ksb = (char*)ws_get(c, "kstate", (size_t)nsys * (4 * 16 + 3 * 8 + 3 * 4) + 64);
  in.ks.count = (int*)ws_get(c, "kcount", 64);
  if (!r64 || !partial || !b2 || !r2 || !delta || !scale || !iscale || !rel || !oact || !rin || !ein || !bhat ||
      !in.r || !in.p || !in.v || !in.s || !in.t || !in.tmp || !ksb || !in.ks.count)
    return set_error(c, LQCD_ERR_OOM, "solve: out of device memory");
  in.ks.rho = (double2*)ksb;
  in.ks.alpha = in.ks.rho + nsys;
  in.ks.omega = in.ks.alpha + nsys;
  in.ks.beta = in.ks.omega + nsys;
  in.ks.r2 = (double*)(in.ks.beta + nsys);
  in.ks.b2 = in.ks.r2 + nsys;
  in.ks.stop2 = in.ks.b2 + nsys;
  in.ks.active = (int*)(in.ks.stop2 + nsys);
  in.ks.iters = in.ks.active + nsys;
  in.ks.flag = in.ks.iters + nsys;
  in.partial = partial;
  in.nchunk = seg_chunks(vgH, domain ? c->seg_dom : c->seg_full);
  in.partial2 = (double*)ws_get(c, "partial2", (size_t)nseg * in.nchunk * nrhs * 8 * sizeof(double));
  if (!in.partial2) return set_error(c, LQCD_ERR_OOM, "solve: out of device memory");
  int* count_host = (int*)pinned_get(c, 64);
  cudaMemsetAsync(in.ks.iters, 0, nsys * sizeof(int), st);

  Fgcr f;
  if (use_gcr) {
    f.m = prm.gcr_nkrylov > 0 ? std::min(prm.gcr_nkrylov, LQCD_GCR_MAXK) : 8;
    f.kind = pkind;
    f.n_mr = prm.precond_iters > 0 ? prm.precond_iters : 6;
    for (int k = 0; k < f.m; k++) {
      f.Z.v[k] = ws_get(c, "g_z" + std::to_string(k), sbP);
      f.W.v[k] = ws_get(c, "g_w" + std::to_string(k), sbP);
      if (!f.Z.v[k] || !f.W.v[k]) return set_error(c, LQCD_ERR_OOM, "solve: out of device memory (GCR)");
    }
    f.x = in.x;
    f.r = in.r;
    char* gb = (char*)ws_get(c, "gstate", (size_t)nsys * (LQCD_GCR_MAXK * 24 + 16 + 5 * 8) + 64);
    if (!gb) return set_error(c, LQCD_ERR_OOM, "solve: out of device memory (GCR)");
    f.gs.nsys = nsys;
    f.gs.beta = (double2*)gb;
    f.gs.alpha = f.gs.beta + (size_t)LQCD_GCR_MAXK * nsys;
    f.gs.w2 = (double*)(f.gs.alpha + nsys);
    f.gs.r2 = f.gs.w2 + (size_t)LQCD_GCR_MAXK * nsys;
    f.gs.b2 = f.gs.r2 + nsys;
    f.gs.stop2 = f.gs.b2 + nsys;
    f.gs.pscale = f.gs.stop2 + nsys;
    f.gs.ipscale = f.gs.pscale + nsys;
    f.gs.active = in.ks.active;
    f.gs.iters = in.ks.iters;
    f.gs.count = in.ks.count;
    if (pkind == PREC_NN) {
      if (int rc = nn_reserve(c, nrhs)) return rc;
    }
    if (pkind == PREC_MR16) {
      const size_t sb16 = spinor_bytes(g, P16, nrhs);
      f.in16 = in;
      f.in16.prec = P16;
      auto tv = c->tuned_variant.find((long)P16 * 100000 + nrhs);
      f.in16.variant = tv != c->tuned_variant.end() ? tv->second : 0;
      f.in16.U = c->U16;
      f.in16.Ainv_e = off(c->Ainv16, clover_bytes(g, P16), 0);
      f.in16.Ainv_o = off(c->Ainv16, clover_bytes(g, P16), 1);
      f.in16.tmp = ws_get(c, "h_tmp", sb16);
      f.e16 = ws_get(c, "h_e", sb16);
      f.r16 = ws_get(c, "h_r", sb16);
      f.p16 = ws_get(c, "h_p", sb16);
      f.omega16 = (double2*)ws_get(c, "h_omega", nsys * sizeof(double2));
      if (!f.in16.tmp || !f.e16 || !f.r16 || !f.p16 || !f.omega16)
        return set_error(c, LQCD_ERR_OOM, "solve: out of device memory (FP16 preconditioner)");
    }
  }

  // x = 0, r = b, |b|^2
  v_zero(P64, x, vgF, st);
  cudaMemcpyAsync(r64, b, 2 * sb64, cudaMemcpyDeviceToDevice, st);
  v_norm2(P64, b, vgF, si, nseg, partial, b2, st);
  outer_update(b2, b2, nsys, tol, inner_tol, oact, delta, scale, rel, 1, st);

  bs.cycles = 0;
  bs.dslash = 0;
  int total_iters = 0;
  const size_t cb64 = clover_bytes(g, P64);
  const auto tv64 = c->tuned_variant.find((long)P64 * 100000 + nrhs);
  const int v64 = tv64 != c->tuned_variant.end() ? tv64->second : 0;  // FP64 residual launch variant
  for (int cyc = 0; cyc < max_outer; cyc++) {
    count_active(oact, nsys, in.ks.count, st);
    cudaMemcpyAsync(count_host, in.ks.count, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    if (*count_host == 0 || total_iters >= max_iter) break;
    bs.cycles++;
    {  // scaled residual in the inner precision, Schur right-hand side
      PhaseTimer pt(c, "prepare");
      v_convert(P64, P, r64, rin, vgF, si, nseg, scale, st);
      launch_clover_only(g, P, in.Ainv_o, off(rin, sbP, 1), in.tmp, nrhs, st);
      DslashCall kp = call(c, P, EPI_C_YH, in.tmp, off(rin, sbP, 0), nullptr, bhat, in.U, in.Ainv_e, 0, nrhs, 1.0,
                           c->kappa, tc);
      launch_dslash(g, kp, st, in.variant);
      bs.dslash += 1;
    }
    if (use_gcr) {  // inner flexible GCR (FP32) with the FP16 MR or network preconditioner
      PhaseTimer pt(c, pkind == PREC_NN ? "inner_fgcr_nn" : "inner_fgcr_mr16");
      gcr_init(P32, bhat, in.x, in.r, vgH, si, nseg, partial, f.gs, delta, oact, st);
      total_iters += run_fgcr(c, in, f, max_iter - total_iters, prm.use_graph != 0, count_host, bs.dslash);
    } else {  // inner BiCGStab
      PhaseTimer pt(c, P == P64 ? "inner_bicgstab_f64" : "inner_bicgstab_f32");
      bicg_init(P, bhat, in.r, in.p, in.x, vgH, si, nseg, partial, in.ks, delta, oact, st);
      total_iters += run_bicg(c, in, max_iter - total_iters, chunk, prm.use_graph != 0, count_host, bs.dslash);
    }
    {  // odd half of the correction, then x += e / scale
      PhaseTimer pt(c, "reconstruct");
      DslashCall kr = call(c, P, EPI_C_YH, in.x, off(rin, sbP, 1), nullptr, off(ein, sbP, 1), in.U, in.Ainv_o, 1,
                           nrhs, 1.0, c->kappa, tc);
      launch_dslash(g, kr, st, in.variant);
      bs.dslash += 1;
      recip(scale, iscale, nsys, st);
      v_axpy_mixed(P, x, ein, vgF, si, nseg, iscale, oact, st);
    }
    {  // FP64 true residual r = b - D x
      PhaseTimer pt(c, "residual_f64");
      for (int p = 0; p < 2; p++) {
        DslashCall k = call(c, P64, EPI_RES, off(x, sb64, 1 - p), off(x, sb64, p), off(b, sb64, p),
                            off(r64, sb64, p), c->U64, off(c->A64, cb64, p), p, nrhs, 1.0, -c->kappa, tc);
        launch_dslash(g, k, st, v64);
      }
      bs.dslash += 2;
      v_norm2(P64, r64, vgF, si, nseg, partial, r2, st);
      outer_update(r2, b2, nsys, tol, inner_tol, oact, delta, scale, rel, 0, st);
    }
  }
  bs.rel.resize(nsys);
  bs.iters.resize(nsys);
  cudaMemcpyAsync(bs.rel.data(), rel, nsys * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(bs.iters.data(), in.ks.iters, nsys * sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(c, LQCD_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(e));
  if (dslash_pipe_timeouts(true))
    return set_error(c, LQCD_ERR_TIMEOUT, "solve: a staged dslash copy did not complete within its wait limit");
  flush_phase_times(c);
  for (int i = 0; i < nsys; i++) {
    if (!std::isfinite(bs.rel[i])) return set_error(c, LQCD_ERR_NAN, "solve: non-finite residual");
    if (bs.rel[i] > tol) return set_error(c, LQCD_ERR_NOT_CONVERGED, "solve: tolerance not reached");
  }
  return LQCD_OK;
}

}  // namespace lqcd
