// Krylov solver driver for the full operator D and the Dirichlet domain operator D_Lambda
// (Sec. 2.1; the paper's "inversions", Sec. 4).
//
// Every solve is an FP64 defect-correction loop judged by the true residual of the
// unpreconditioned operator, computed from the FP64 fields (in double-float arithmetic, or FP64
// with residual = 1), per system (one right-hand side, or one domain of one right-hand
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
  return (size_t)g.Vh * nrhs * 12 * (prec == P64 || prec == PDF ? 16 : (prec == P32 ? 8 : 4));
}
size_t clover_bytes(const Geom& g, int prec) {
  return (size_t)g.Vh * 2 * (prec == P64 || prec == PDF ? 18 * 16 : (prec == P32 ? 9 * 16 : 9 * 8));
}
size_t link_bytes(const Geom& g, int prec) {
  return (size_t)g.Vh * 8 * (prec == P64 || prec == PDF ? 9 * 16 : (prec == P32 ? 3 * 16 : 3 * 8));
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

static cudaGraphExec_t capture(lqcd_ctx* c, cudaStream_t st, const std::string& key, int nsys, const KState& ks,
                               int* count_host, const std::function<void(cudaStream_t)>& body) {
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
static int run_bicg(lqcd_ctx* c, cudaStream_t st, const Inner& in, int max_iter, int chunk, bool use_graph,
                    int* count_host, long long& dslash_calls) {
  const int nsys = in.nrhs * in.nseg;
  auto body = [&](cudaStream_t s) {
    for (int k = 0; k < chunk; k++) bicg_iteration(c, in, s);
  };
  cudaGraphExec_t exec = use_graph ? capture(c, st, graph_key(in, chunk), nsys, in.ks, count_host, body) : nullptr;
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

static std::string fgcr_key(const Inner& in, const Fgcr& f, const lqcd_ctx* c) {
  char key[256];
  snprintf(key, sizeof key, "fgcr:%d:%d:%d:%d:%d:%p:%p:%p:%p:%p", f.m, f.kind, f.n_mr, in.nrhs, in.nseg, f.x,
           f.Z.v[0], (void*)f.gs.beta, (const void*)in.tc, c->nn_weights);
  return key;
}

// Run restarted FGCR(m) until all systems are inactive or max_iter; returns iterations.
static int run_fgcr(lqcd_ctx* c, cudaStream_t st, const Inner& in, const Fgcr& f, int max_iter, bool use_graph,
                    int* count_host, long long& dslash_calls) {
  const int nsys = in.nrhs * in.nseg;
  auto body = [&](cudaStream_t s) { fgcr_cycle(c, in, f, s); };
  GState gs_count = f.gs;
  KState ks_count = in.ks;
  ks_count.active = gs_count.active;
  ks_count.count = gs_count.count;
  cudaGraphExec_t exec = use_graph ? capture(c, st, fgcr_key(in, f, c), nsys, ks_count, count_host, body) : nullptr;
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

// ------------------------------------------------------------------ one batch of systems
// Workspace, operator data and settings of one batch of right-hand sides.  A context keeps two
// sets of work vectors (slots 0 and 1, on the streams `work` and `slot_stream`) so two batches can
// be in flight at once: one batch's FP64 true residual (FP64-pipe bound) then runs beside the
// other's FP32 iterations (memory and FP32 bound).
struct Batch {
  int slot;
  cudaStream_t st;
  int nrhs, domain, nseg, nsys, P;
  bool use_gcr;
  int pkind;
  double tol, inner_tol;
  int max_iter, max_outer, chunk;
  VGeom vgF, vgH;
  const SegInfo* si;
  const signed char* tc;
  double2* r64;
  double* partial;
  double *b2, *r2, *delta, *scale, *iscale, *rel;
  int* oact;
  void *rin, *ein, *bhat;
  int* ctr;  // device loop counters: inner iterations, cycles, inner chunks
  Inner in;
  Fgcr f;
  int v64;       // launch variant of the true-residual kernel
  int res_prec;  // its arithmetic: PDF (double-float) or P64
  void* xdf;     // PDF: one parity of x split to double-float
  size_t sb64, sbP;
  char* hbuf;  // pinned read-back: rel [nsys] doubles, iters [nsys] ints, counters [4] ints
  long long dslash_host;  // host path: dslash launches counted on the host
  int iters_host;         // host path: inner iterations summed
  bool graph;             // enqueued as one device-loop graph
  int fallback;           // FGCR_NN without a network: MR preconditioner instead
  long long nk_init, nk_cycle, nk_chunk;
};

static std::string wsn(const char* base, int slot) {
  return slot ? std::string(base) + "#" + std::to_string(slot) : std::string(base);
}

cudaStream_t slot_stream(lqcd_ctx* c, int slot) {
  if (slot == 0) return c->work;
  if (!c->slot_stream) {
    cudaStreamCreateWithFlags(&c->slot_stream, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&c->ev_slot, cudaEventDisableTiming);
  }
  return c->slot_stream;
}

static char* slot_pinned(lqcd_ctx* c, int slot, size_t bytes) {
  if (c->slot_pinned_bytes[slot] >= bytes) return (char*)c->slot_pinned[slot];
  if (c->slot_pinned[slot]) {
    cudaStreamSynchronize(slot_stream(c, slot));
    drop_graphs(c);  // captured read-backs target the old buffer
    cudaFreeHost(c->slot_pinned[slot]);
  }
  c->slot_pinned[slot] = nullptr;
  if (cudaMallocHost(&c->slot_pinned[slot], bytes) != cudaSuccess) {
    cudaGetLastError();
    c->slot_pinned_bytes[slot] = 0;
    return nullptr;
  }
  c->slot_pinned_bytes[slot] = bytes;
  return (char*)c->slot_pinned[slot];
}

static int plan_batch(lqcd_ctx* c, int slot, int nrhs, int domain, const lqcd_solve_params& prm, Batch& B) {
  const Geom& g = c->g;
  B.slot = slot;
  B.st = slot_stream(c, slot);
  B.nrhs = nrhs;
  B.domain = domain;
  B.si = domain ? c->d_seg_dom : c->d_seg_full;
  B.nseg = domain ? c->seg_dom.nseg : 1;
  B.nsys = nrhs * B.nseg;
  B.tc = domain ? c->d_tc_dom : c->d_tc_full;
  B.tol = prm.tol > 0 ? prm.tol : 1e-10;
  B.max_iter = prm.max_iter > 0 ? prm.max_iter : 20000;
  B.max_outer = prm.max_outer > 0 ? prm.max_outer : 20;
  // Inner iterations between convergence checks.  A batch runs until its slowest system converges,
  // rounded up to whole chunks, so a large chunk wastes up to chunk - 1 full iterations per cycle;
  // a check costs a few microseconds (a small kernel and a conditional graph node, or a 4-byte
  // read-back).  Default: every iteration once a batch holds >= 2^22 (site, RHS) pairs per parity
  // (an iteration then takes milliseconds), up to every 8th for small batches.
  const long pairs = std::max(1L, g.Vh * (long)nrhs);
  B.chunk = prm.check_every > 0 ? prm.check_every : (int)std::min(8L, std::max(1L, ((1L << 22) + pairs - 1) / pairs));
  B.graph = false;
  B.fallback = 0;
  B.dslash_host = 0;
  B.iters_host = 0;
  const int nsys = B.nsys;

  // Residual reduction asked of one inner solve.  FP32 BiCGStab on a unit-norm right-hand side
  // reaches a true residual of a few 1e-7 before rounding stalls it, so asking 2e-6 makes two
  // defect-correction cycles enough for 1e-10 (each FP64 cycle costs two FP64 dslash launches).
  // MIXED with FP16 inner precision and FGCR_NN run FP32 flexible GCR whose preconditioner is
  // FP16-storage MR sweeps or the learned network (MR if no network is loaded).
  B.P = P64;
  B.inner_tol = 1e-12;
  B.use_gcr = false;
  B.pkind = PREC_NONE;
  if (prm.solver == LQCD_SOLVER_MIXED || prm.solver == LQCD_SOLVER_FGCR_NN) {
    B.P = P32;
    B.inner_tol = 2e-6;
    if (prm.solver == LQCD_SOLVER_FGCR_NN) {
      B.use_gcr = true;
      B.pkind = c->nn_weights ? PREC_NN : PREC_MR16;
      B.fallback = c->nn_weights ? 0 : 1;
    } else if (prm.inner_prec == LQCD_PREC_F16) {
      B.use_gcr = true;
      B.pkind = PREC_MR16;
    }
    if (B.use_gcr && prm.precond_iters < 0) B.pkind = PREC_NONE;  // unpreconditioned FGCR (reference runs)
  }
  if (prm.inner_tol > 0) B.inner_tol = prm.inner_tol;
  const int P = B.P;

  B.vgF = make_vgeom(g, nrhs, 2);  // full lattice
  B.vgH = make_vgeom(g, nrhs, 1);  // one parity
  if (B.vgH.threads() > 128) return set_error(c, LQCD_ERR_INVALID_ARG, "solve: rhs_block > 128");
  B.sb64 = spinor_bytes(g, P64, nrhs);
  B.sbP = spinor_bytes(g, P, nrhs);
  const size_t cbP = clover_bytes(g, P);

  // FP64 outer fields and per-system bookkeeping
  B.r64 = (double2*)ws_get(c, wsn("o_r64", slot), 2 * B.sb64);
  // per-(block, rhs) partial sums: 3 for BiCGStab / norms on the full lattice, up to 2 x 16 for the
  // GCR Gram rows on one parity
  size_t npart = std::max((size_t)B.vgF.blocks * nrhs * 3, (size_t)B.vgH.blocks * nrhs * 2 * LQCD_GCR_MAXK);
  B.partial = (double*)ws_get(c, wsn("partial", slot), npart * sizeof(double));
  double* ob = (double*)ws_get(c, wsn("o_sys", slot), (size_t)nsys * 6 * sizeof(double) + 64);
  B.oact = (int*)ws_get(c, wsn("o_active", slot), nsys * sizeof(int));
  B.ctr = (int*)ws_get(c, wsn("o_ctr", slot), 64);
  // inner fields (precision P)
  B.rin = ws_get(c, wsn("i_rin", slot), 2 * B.sbP);  // scaled residual, full lattice
  B.ein = ws_get(c, wsn("i_ein", slot), 2 * B.sbP);  // correction, full lattice (even part = inner x)
  B.hbuf = slot_pinned(c, slot, (size_t)nsys * 12 + 64);
  if (!B.r64 || !B.partial || !ob || !B.oact || !B.ctr || !B.rin || !B.ein || !B.hbuf)
    return set_error(c, LQCD_ERR_OOM, "solve: out of device memory");
  B.b2 = ob;
  B.r2 = ob + nsys;
  B.delta = ob + 2 * nsys;
  B.scale = ob + 3 * nsys;
  B.iscale = ob + 4 * nsys;
  B.rel = ob + 5 * nsys;
  Inner& in = B.in;
  in.prec = P;
  in.nrhs = nrhs;
  in.nseg = B.nseg;
  in.vg = B.vgH;
  in.si = B.si;
  in.tc = B.tc;
  in.U = P == P64 ? c->U64 : (P == P32 ? c->U32 : c->U16);
  const void* Ainv = P == P64 ? c->Ainv64 : (P == P32 ? c->Ainv32 : c->Ainv16);
  in.Ainv_e = off(Ainv, cbP, 0);
  in.Ainv_o = off(Ainv, cbP, 1);
  B.bhat = ws_get(c, wsn("i_bhat", slot), B.sbP);
  in.b = B.bhat;
  in.x = B.ein;  // even half of the full correction field
  in.r = ws_get(c, wsn("i_r", slot), B.sbP);
  in.p = ws_get(c, wsn("i_p", slot), B.sbP);
  in.v = ws_get(c, wsn("i_v", slot), B.sbP);
  in.s = ws_get(c, wsn("i_s", slot), B.sbP);
  in.t = ws_get(c, wsn("i_t", slot), B.sbP);
  in.tmp = ws_get(c, wsn("i_tmp", slot), B.sbP);
  in.kappa = c->kappa;
  in.variant = 0;
  {
    auto it = c->tuned_variant.find((long)P * 100000 + nrhs);
    if (it != c->tuned_variant.end()) in.variant = it->second;
  }
  char* ksb = (char*)ws_get(c, wsn("kstate", slot), (size_t)nsys * (4 * 16 + 3 * 8 + 3 * 4) + 64);
  in.ks.count = (int*)ws_get(c, wsn("kcount", slot), 64);
  if (!B.bhat || !in.r || !in.p || !in.v || !in.s || !in.t || !in.tmp || !ksb || !in.ks.count)
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
  in.partial = B.partial;
  in.nchunk = seg_chunks(B.vgH, domain ? c->seg_dom : c->seg_full);
  in.partial2 = (double*)ws_get(c, wsn("partial2", slot), (size_t)B.nseg * in.nchunk * nrhs * 8 * sizeof(double));
  if (!in.partial2) return set_error(c, LQCD_ERR_OOM, "solve: out of device memory");

  Fgcr& f = B.f;
  if (B.use_gcr) {
    f.m = prm.gcr_nkrylov > 0 ? std::min(prm.gcr_nkrylov, LQCD_GCR_MAXK) : 8;
    f.kind = B.pkind;
    f.n_mr = prm.precond_iters > 0 ? prm.precond_iters : 6;
    for (int k = 0; k < f.m; k++) {
      f.Z.v[k] = ws_get(c, wsn(("g_z" + std::to_string(k)).c_str(), slot), B.sbP);
      f.W.v[k] = ws_get(c, wsn(("g_w" + std::to_string(k)).c_str(), slot), B.sbP);
      if (!f.Z.v[k] || !f.W.v[k]) return set_error(c, LQCD_ERR_OOM, "solve: out of device memory (GCR)");
    }
    f.x = in.x;
    f.r = in.r;
    char* gb = (char*)ws_get(c, wsn("gstate", slot), (size_t)nsys * (LQCD_GCR_MAXK * 24 + 16 + 5 * 8) + 64);
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
    if (B.pkind == PREC_NN) {
      if (slot != 0) return set_error(c, LQCD_ERR_INVALID_ARG, "solve: the network preconditioner runs in slot 0");
      if (int rc = nn_reserve(c, nrhs)) return rc;
    }
    if (B.pkind == PREC_MR16) {
      const size_t sb16 = spinor_bytes(g, P16, nrhs);
      f.in16 = in;
      f.in16.prec = P16;
      auto tv = c->tuned_variant.find((long)P16 * 100000 + nrhs);
      f.in16.variant = tv != c->tuned_variant.end() ? tv->second : 0;
      f.in16.U = c->U16;
      f.in16.Ainv_e = off(c->Ainv16, clover_bytes(g, P16), 0);
      f.in16.Ainv_o = off(c->Ainv16, clover_bytes(g, P16), 1);
      f.in16.tmp = ws_get(c, wsn("h_tmp", slot), sb16);
      f.e16 = ws_get(c, wsn("h_e", slot), sb16);
      f.r16 = ws_get(c, wsn("h_r", slot), sb16);
      f.p16 = ws_get(c, wsn("h_p", slot), sb16);
      f.omega16 = (double2*)ws_get(c, wsn("h_omega", slot), nsys * sizeof(double2));
      if (!f.in16.tmp || !f.e16 || !f.r16 || !f.p16 || !f.omega16)
        return set_error(c, LQCD_ERR_OOM, "solve: out of device memory (FP16 preconditioner)");
    }
  }
  const auto tv64 = c->tuned_variant.find((long)P64 * 100000 + nrhs);
  B.v64 = tv64 != c->tuned_variant.end() ? tv64->second : 0;  // FP64 residual launch variant
  B.res_prec = prm.residual == 1 ? P64 : PDF;
  B.xdf = nullptr;
  if (B.res_prec == PDF) {
    const auto tvd = c->tuned_variant.find((long)PDF * 100000 + nrhs);
    B.v64 = tvd != c->tuned_variant.end() ? tvd->second : 0;
    B.xdf = ws_get(c, wsn("r_xdf", slot), spinor_bytes(g, P64, nrhs));
    if (!B.xdf) return set_error(c, LQCD_ERR_OOM, "solve: out of device memory (residual)");
  }
  return LQCD_OK;
}

// x = 0, r = b, |b|^2, first bookkeeping
static void batch_start(lqcd_ctx* c, Batch& B, const double2* b, double2* x) {
  cudaStream_t st = B.st;
  cudaMemsetAsync(B.in.ks.iters, 0, B.nsys * sizeof(int), st);
  cudaMemsetAsync(B.ctr, 0, 64, st);
  v_zero(P64, x, B.vgF, st);
  cudaMemcpyAsync(B.r64, b, 2 * B.sb64, cudaMemcpyDeviceToDevice, st);
  v_norm2(P64, b, B.vgF, B.si, B.nseg, B.partial, B.b2, st);
  outer_update(B.b2, B.b2, B.nsys, B.tol, B.inner_tol, B.oact, B.delta, B.scale, B.rel, 1, st);
}

// scaled residual in the inner precision, even-odd Schur right-hand side
static void batch_prepare(lqcd_ctx* c, Batch& B) {
  const Geom& g = c->g;
  const int P = B.P;
  Inner& in = B.in;
  v_convert(P64, P, B.r64, B.rin, B.vgF, B.si, B.nseg, B.scale, B.st);
  launch_clover_only(g, P, in.Ainv_o, off(B.rin, B.sbP, 1), in.tmp, B.nrhs, B.st);
  DslashCall kp = call(c, P, EPI_C_YH, in.tmp, off(B.rin, B.sbP, 0), nullptr, B.bhat, in.U, in.Ainv_e, 0, B.nrhs,
                       1.0, c->kappa, B.tc);
  launch_dslash(g, kp, B.st, in.variant);
}

static void batch_inner_init(Batch& B) {
  Inner& in = B.in;
  if (B.use_gcr)
    gcr_init(P32, B.bhat, in.x, in.r, B.vgH, B.si, B.nseg, B.partial, B.f.gs, B.delta, B.oact, B.st);
  else
    bicg_init(B.P, B.bhat, in.r, in.p, in.x, B.vgH, B.si, B.nseg, B.partial, in.ks, B.delta, B.oact, B.st);
}

// odd half of the correction, x += e / scale, then the FP64 true residual r = b - D x
static void batch_finish_cycle(lqcd_ctx* c, Batch& B, const double2* b, double2* x) {
  const Geom& g = c->g;
  const int P = B.P;
  Inner& in = B.in;
  DslashCall kr = call(c, P, EPI_C_YH, in.x, off(B.rin, B.sbP, 1), nullptr, off(B.ein, B.sbP, 1), in.U, in.Ainv_o, 1,
                       B.nrhs, 1.0, c->kappa, B.tc);
  launch_dslash(g, kr, B.st, in.variant);
  recip(B.scale, B.iscale, B.nsys, B.st);
  v_axpy_mixed(P, x, B.ein, B.vgF, B.si, B.nseg, B.iscale, B.oact, B.st);
  const size_t cb64 = clover_bytes(g, P64);
  for (int p = 0; p < 2; p++) {
    if (B.res_prec == PDF) {
      split_neighbours(off(x, B.sb64, 1 - p), B.xdf, (long)(B.sb64 / 16), B.nrhs, B.st);
      launch_residual_df(g, B.xdf, off(x, B.sb64, p), off(b, B.sb64, p), off(B.r64, B.sb64, p), c->Udf,
                         off(c->Adf, cb64, p), coord_of(c, p), B.tc, p, B.nrhs, c->kappa, B.v64, B.st);
    } else {
      DslashCall k = call(c, P64, EPI_RES, off(x, B.sb64, 1 - p), off(x, B.sb64, p), off(b, B.sb64, p),
                          off(B.r64, B.sb64, p), c->U64, off(c->A64, cb64, p), p, B.nrhs, 1.0, -c->kappa, B.tc);
      launch_dslash(g, k, B.st, B.v64);
    }
  }
  v_norm2(P64, B.r64, B.vgF, B.si, B.nseg, B.partial, B.r2, B.st);
  outer_update(B.r2, B.b2, B.nsys, B.tol, B.inner_tol, B.oact, B.delta, B.scale, B.rel, 0, B.st);
}

static void batch_readback(Batch& B) {
  cudaMemcpyAsync(B.hbuf, B.rel, B.nsys * sizeof(double), cudaMemcpyDeviceToHost, B.st);
  cudaMemcpyAsync(B.hbuf + (size_t)B.nsys * 8, B.in.ks.iters, B.nsys * sizeof(int), cudaMemcpyDeviceToHost, B.st);
  cudaMemcpyAsync(B.hbuf + (size_t)B.nsys * 12, B.ctr, 4 * sizeof(int), cudaMemcpyDeviceToHost, B.st);
}

// Host-driven cycles: a convergence read-back after every chunk of inner iterations (and the
// chunk itself replayed from a CUDA graph when use_graph is set).
static void run_host(lqcd_ctx* c, Batch& B, const double2* b, double2* x, bool use_graph) {
  cudaStream_t st = B.st;
  int* count_host = (int*)pinned_get(c, 64);
  batch_start(c, B, b, x);
  int total_iters = 0, cycles = 0;
  for (int cyc = 0; cyc < B.max_outer; cyc++) {
    count_active(B.oact, B.nsys, B.in.ks.count, st);
    cudaMemcpyAsync(count_host, B.in.ks.count, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    if (*count_host == 0 || total_iters >= B.max_iter) break;
    {
      PhaseTimer pt(c, "prepare");
      batch_prepare(c, B);
      B.dslash_host += 1;
    }
    if (B.use_gcr) {  // inner flexible GCR (FP32) with the FP16 MR or network preconditioner
      PhaseTimer pt(c, B.pkind == PREC_NN ? "inner_fgcr_nn" : "inner_fgcr_mr16");
      batch_inner_init(B);
      total_iters += run_fgcr(c, st, B.in, B.f, B.max_iter - total_iters, use_graph, count_host, B.dslash_host);
    } else {  // inner BiCGStab
      PhaseTimer pt(c, B.P == P64 ? "inner_bicgstab_f64" : "inner_bicgstab_f32");
      batch_inner_init(B);
      total_iters += run_bicg(c, st, B.in, B.max_iter - total_iters, B.chunk, use_graph, count_host, B.dslash_host);
    }
    {
      PhaseTimer pt(c, "reconstruct_residual_f64");
      batch_finish_cycle(c, B, b, x);
      B.dslash_host += 3;
    }
    cycles = cyc + 1;
  }
  cudaMemcpyAsync(B.hbuf, B.rel, B.nsys * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(B.hbuf + (size_t)B.nsys * 8, B.in.ks.iters, B.nsys * sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  int* ctr = (int*)(B.hbuf + (size_t)B.nsys * 12);
  ctr[0] = total_iters;
  ctr[1] = cycles;
  ctr[2] = 0;
  B.iters_host = total_iters;
}

static long long count_kernel_nodes(cudaGraph_t g) {
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  cudaGraphGetNodes(g, nodes.data(), &nn);
  long long nk = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    cudaGraphNodeGetType(nd, &ty);
    nk += ty == cudaGraphNodeTypeKernel;
  }
  return nk;
}

// Append a WHILE node with condition handle h after the current capture position of `st`;
// returns its body graph.
static cudaError_t add_while(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraph_t* body) {
  cudaStreamCaptureStatus stat;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &stat, nullptr, &g, &deps, nullptr, &ndeps);
  if (e != cudaSuccess) return e;
  if (stat != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np);
  if (e != cudaSuccess) return e;
  *body = np.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// The whole solve as one graph with device-side loops (no host round trip until it ends):
//   [x = 0, r = b, |b|^2]  cond(outer)
//   WHILE outer { [prepare, inner init] cond(inner)  WHILE inner { chunk of iterations; cond(inner) }
//                 [reconstruct, x += e, FP64 r = b - D x, |r|^2, bookkeeping]  cond(outer) }
//   [read-back of residuals, iterations, counters to pinned memory]
// The conditions are set by k_loop_cond from the per-system active flags, the iteration and cycle
// counters, max_iter and max_outer: the same decisions the host-driven loop takes.  Returns false
// (nothing recorded) if the driver refuses a step; the caller then runs the host-driven loop.
static bool build_loop_graph(lqcd_ctx* c, const Batch& B0, const double2* b, double2* x, const std::string& key) {
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  Batch B = B0;
  B.st = c->cap_stream;
  cudaStream_t s0 = B.st;
  const int* act_inner = B.use_gcr ? B.f.gs.active : B.in.ks.active;
  const int per_chunk = B.use_gcr ? B.f.m : B.chunk;
  cudaGraph_t G = nullptr, O = nullptr, I = nullptr;
  cudaGraphConditionalHandle ho = 0, hi = 0;
  bool ok = cudaGraphCreate(&G, 0) == cudaSuccess;
  auto end_capture = [&](cudaGraph_t* gr) {
    cudaGraph_t out = nullptr;
    if (cudaStreamEndCapture(s0, &out) != cudaSuccess) ok = false;
    (void)gr;
  };
  set_capturing(true);
  // top level: start, outer condition, outer loop, read-back
  if (ok) ok = cudaStreamBeginCaptureToGraph(s0, G, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) == cudaSuccess;
  if (ok) {
    batch_start(c, B, b, x);
    ok = cudaGraphConditionalHandleCreate(&ho, G, 0, 0) == cudaSuccess;
    if (ok) loop_cond(B.oact, B.nsys, B.ctr, 0, 0, B.max_outer, B.max_iter, ho, s0);
    ok = ok && add_while(s0, ho, &O) == cudaSuccess;
    if (ok) batch_readback(B);
    end_capture(&G);
  }
  // one defect-correction cycle
  if (ok) ok = cudaStreamBeginCaptureToGraph(s0, O, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) == cudaSuccess;
  if (ok) {
    batch_prepare(c, B);
    batch_inner_init(B);
    ok = cudaGraphConditionalHandleCreate(&hi, O, 0, 0) == cudaSuccess;
    if (ok) loop_cond(act_inner, B.nsys, B.ctr, 2, per_chunk, B.max_outer, B.max_iter, hi, s0);
    ok = ok && add_while(s0, hi, &I) == cudaSuccess;
    if (ok) {
      batch_finish_cycle(c, B, b, x);
      loop_cond(B.oact, B.nsys, B.ctr, 1, 0, B.max_outer, B.max_iter, ho, s0);
    }
    end_capture(&O);
  }
  // one chunk of inner iterations
  if (ok) ok = cudaStreamBeginCaptureToGraph(s0, I, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) == cudaSuccess;
  if (ok) {
    if (B.use_gcr)
      fgcr_cycle(c, B.in, B.f, s0);
    else
      for (int k = 0; k < B.chunk; k++) bicg_iteration(c, B.in, s0);
    loop_cond(act_inner, B.nsys, B.ctr, 3, per_chunk, B.max_outer, B.max_iter, hi, s0);
    end_capture(&I);
  }
  set_capturing(false);
  cudaGraphExec_t exec = nullptr;
  if (ok) ok = cudaGraphInstantiate(&exec, G, 0) == cudaSuccess;
  if (ok) {
    lqcd_ctx::LoopGraph lg;
    lg.exec = exec;
    lg.nk_init = count_kernel_nodes(G);
    lg.nk_cycle = count_kernel_nodes(O);
    lg.nk_chunk = count_kernel_nodes(I);
    c->loop_graphs[key] = lg;
  } else {
    cudaStreamCaptureStatus stat;
    if (cudaStreamIsCapturing(s0, &stat) == cudaSuccess && stat != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(s0, &junk);
      if (junk && junk != G) cudaGraphDestroy(junk);
    }
    c->loop_graphs_unavailable = true;  // do not retry on every batch
  }
  if (G) cudaGraphDestroy(G);
  cudaGetLastError();
  return ok;
}

// Decode the read-back of a finished batch.
static int batch_result(lqcd_ctx* c, Batch& B, BatchStats& bs) {
  const int nsys = B.nsys;
  const double* rel = (const double*)B.hbuf;
  const int* its = (const int*)(B.hbuf + (size_t)nsys * 8);
  const int* ctr = (const int*)(B.hbuf + (size_t)nsys * 12);
  bs.rel.assign(rel, rel + nsys);
  bs.iters.assign(its, its + nsys);
  bs.cycles = ctr[1];
  bs.device_loops = B.graph ? 1 : 0;
  bs.fallback = B.fallback;
  if (B.graph) {
    const long long per_chunk_dslash =
        B.use_gcr ? (long long)B.f.m * (2 + (B.f.kind == PREC_MR16 ? 2 * B.f.n_mr : 0)) : 4LL * B.chunk;
    bs.dslash = 4LL * ctr[1] + per_chunk_dslash * ctr[2];
    count_launch(B.nk_init + B.nk_cycle * ctr[1] + B.nk_chunk * ctr[2]);
  } else {
    bs.dslash = B.dslash_host;
  }
  flush_phase_times(c);
  if (dslash_pipe_timeouts(true))
    return set_error(c, LQCD_ERR_TIMEOUT, "solve: a staged dslash copy did not complete within its wait limit");
  for (int i = 0; i < nsys; i++) {
    if (!std::isfinite(bs.rel[i])) return set_error(c, LQCD_ERR_NAN, "solve: non-finite residual");
  }
  for (int i = 0; i < nsys; i++)
    if (bs.rel[i] > B.tol) return set_error(c, LQCD_ERR_NOT_CONVERGED, "solve: tolerance not reached");
  return LQCD_OK;
}

int solve_batch_enqueue(lqcd_ctx* c, int slot, const double2* b, double2* x, int nrhs, int domain,
                        const lqcd_solve_params& prm, BatchHandle& h) {
  h.batch = std::make_shared<Batch>();
  Batch& B = *static_cast<Batch*>(h.batch.get());
  if (int rc = plan_batch(c, slot, nrhs, domain, prm, B)) return rc;
  const bool use_graph = prm.use_graph != 0;
  if (use_graph && !c->loop_graphs_unavailable && !c->timing) {
    char key[512];
    snprintf(key, sizeof key, "loop:%d:%d:%d:%d:%d:%d:%.17g:%.17g:%d:%d:%d:%d:%d:%d:%p:%p:%p:%p:%p:%p:%p:%p", slot, B.P,
             nrhs, domain, B.nseg, B.chunk, B.tol, B.inner_tol, B.max_iter, B.max_outer, B.in.variant, B.v64,
             B.res_prec,
             B.pkind, (const void*)b, (void*)x, (void*)B.r64, B.in.r, (void*)B.hbuf, (const void*)B.tc,
             (const void*)B.si, B.in.U);
    std::string k = key;
    if (B.use_gcr) k += fgcr_key(B.in, B.f, c);
    auto it = c->loop_graphs.find(k);
    if (it == c->loop_graphs.end() && build_loop_graph(c, B, b, x, k)) it = c->loop_graphs.find(k);
    if (it != c->loop_graphs.end()) {
      B.graph = true;
      B.nk_init = it->second.nk_init;
      B.nk_cycle = it->second.nk_cycle;
      B.nk_chunk = it->second.nk_chunk;
      cudaGraphLaunch(it->second.exec, B.st);
      return LQCD_OK;
    }
  }
  run_host(c, B, b, x, use_graph);
  return LQCD_OK;
}

int solve_batch_finish(lqcd_ctx* c, BatchHandle& h, BatchStats& bs) {
  Batch& B = *static_cast<Batch*>(h.batch.get());
  cudaError_t e = cudaStreamSynchronize(B.st);
  if (e != cudaSuccess) return set_error(c, LQCD_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(e));
  int rc = batch_result(c, B, bs);
  h.batch.reset();
  return rc;
}

int solve_batch(lqcd_ctx* c, const double2* b, double2* x, int nrhs, int domain, const lqcd_solve_params& prm,
                BatchStats& bs) {
  BatchHandle h;
  if (int rc = solve_batch_enqueue(c, 0, b, x, nrhs, domain, prm, h)) return rc;
  return solve_batch_finish(c, h, bs);
}

}  // namespace lqcd
