// extern "C" entry points declared in include/lqcd.h: argument checks, host/device staging,
// stream ordering, batching of right-hand sides.  All arithmetic runs in the CUDA kernels of
// this library.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lqcd_blas.h"
#include "lqcd_distill.h"

using namespace lqcd;

static std::string g_create_error;
static std::atomic<long long> g_launches{0};
static thread_local bool g_capturing = false;

namespace lqcd {

void count_launch(long long n) {
  if (!g_capturing) g_launches += n;
}
void set_capturing(bool on) { g_capturing = on; }
bool is_capturing() { return g_capturing; }

void flush_phase_times(lqcd_ctx* c) {
  if (c->pending.empty()) return;
  cudaStreamSynchronize(c->work);
  for (auto& p : c->pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) c->phase_ms[p.first] += ms;
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  cudaGetLastError();
  c->pending.clear();
}

int set_error(lqcd_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

// Message for lqcd_last_error(NULL): failures of calls that take no context.
void set_global_error(const std::string& msg) { g_create_error = msg; }

void* ws_get(lqcd_ctx* c, const std::string& name, size_t bytes) {
  auto it = c->ws.find(name);
  if (it != c->ws.end() && it->second.bytes >= bytes) {
    it->second.gen = c->ws_gen;
    return it->second.p;
  }
  if (it != c->ws.end()) {
    cudaStreamSynchronize(c->work);
    if (c->slot_stream) cudaStreamSynchronize(c->slot_stream);
    cudaFree(it->second.p);
    c->ws.erase(it);
    drop_graphs(c);  // graphs captured on the old buffer are stale
  }
  const size_t sz = bytes < 256 ? 256 : bytes;
  void* p = nullptr;
  if (cudaMalloc(&p, sz) != cudaSuccess) {
    cudaGetLastError();
    // Short of memory: free the buffers that only earlier calls used (another solver's or block
    // size's work vectors), then try once more.
    bool freed = false;
    for (auto& kv : c->ws)
      if (kv.second.gen != c->ws_gen) freed = true;
    if (!freed) return nullptr;
    drop_graphs(c);
    for (auto i = c->ws.begin(); i != c->ws.end();) {
      if (i->second.gen != c->ws_gen) {
        cudaFree(i->second.p);
        i = c->ws.erase(i);
      } else {
        ++i;
      }
    }
    if (cudaMalloc(&p, sz) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
  }
  c->ws[name] = {p, sz, c->ws_gen};
  return p;
}

void drop_graphs(lqcd_ctx* c) {
  if (c->work) cudaStreamSynchronize(c->work);
  if (c->slot_stream) cudaStreamSynchronize(c->slot_stream);
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  c->graph_kernels.clear();
  for (auto& kv : c->loop_graphs) cudaGraphExecDestroy(kv.second.exec);
  c->loop_graphs.clear();
}

void* pinned_get(lqcd_ctx* c, size_t bytes) {
  if (c->pinned_bytes >= bytes) return c->pinned;
  if (c->pinned) {
    cudaStreamSynchronize(c->work);
    cudaFreeHost(c->pinned);
  }
  cudaMallocHost(&c->pinned, bytes);
  c->pinned_bytes = bytes;
  return c->pinned;
}

}  // namespace lqcd

namespace {

// The 16-element Clifford table of the header, built here from the chiral-basis gammas.
struct M4 {
  double re[4][4], im[4][4];
};
M4 m4_zero() {
  M4 m;
  memset(&m, 0, sizeof m);
  return m;
}
M4 m4_mul(const M4& a, const M4& b) {
  M4 c = m4_zero();
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++)
      for (int k = 0; k < 4; k++) {
        c.re[i][j] += a.re[i][k] * b.re[k][j] - a.im[i][k] * b.im[k][j];
        c.im[i][j] += a.re[i][k] * b.im[k][j] + a.im[i][k] * b.re[k][j];
      }
  return c;
}
M4 m4_dag(const M4& a) {
  M4 c;
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) {
      c.re[i][j] = a.re[j][i];
      c.im[i][j] = -a.im[j][i];
    }
  return c;
}
M4 m4_scale_i(const M4& a) {  // i * a
  M4 c;
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) {
      c.re[i][j] = -a.im[i][j];
      c.im[i][j] = a.re[i][j];
    }
  return c;
}
void clifford(M4 out[16], M4 tilde[16]) {
  M4 g[4];
  for (int m = 0; m < 4; m++) g[m] = m4_zero();
  // gamma_x: upper-right block -i sigma_x, lower-left i sigma_x
  g[0].im[0][3] = -1; g[0].im[1][2] = -1; g[0].im[2][1] = 1; g[0].im[3][0] = 1;
  // gamma_y: -i sigma_y = [[0,-1],[1,0]] upper right; i sigma_y = [[0,1],[-1,0]] lower left
  g[1].re[0][3] = -1; g[1].re[1][2] = 1; g[1].re[2][1] = 1; g[1].re[3][0] = -1;
  // gamma_z: -i sigma_z = diag(-i, i) upper right; i sigma_z = diag(i, -i) lower left
  g[2].im[0][2] = -1; g[2].im[1][3] = 1; g[2].im[2][0] = 1; g[2].im[3][1] = -1;
  // gamma_t: identity blocks off the diagonal
  g[3].re[0][2] = 1; g[3].re[1][3] = 1; g[3].re[2][0] = 1; g[3].re[3][1] = 1;
  M4 one = m4_zero();
  for (int i = 0; i < 4; i++) one.re[i][i] = 1;
  M4 g5 = m4_mul(m4_mul(g[0], g[1]), m4_mul(g[2], g[3]));
  out[0] = one;
  for (int m = 0; m < 4; m++) out[1 + m] = g[m];
  out[5] = g5;
  for (int m = 0; m < 4; m++) out[6 + m] = m4_mul(g[m], g5);
  const int pm[6] = {0, 0, 0, 1, 1, 2}, pn[6] = {1, 2, 3, 2, 3, 3};
  for (int k = 0; k < 6; k++) out[10 + k] = m4_scale_i(m4_mul(g[pm[k]], g[pn[k]]));  // sigma = i g g
  for (int k = 0; k < 16; k++) tilde[k] = m4_mul(m4_mul(g[3], m4_dag(out[k])), g[3]);
}

// Order the caller's stream before the library's work stream and back.
struct Scope {
  lqcd_ctx* c;
  explicit Scope(lqcd_ctx* ctx) : c(ctx) {
    c->ws_gen++;
    cudaEventRecord(c->ev_user, c->user_stream);
    cudaStreamWaitEvent(c->work, c->ev_user, 0);
  }
  ~Scope() {
    cudaEventRecord(c->ev_work, c->work);
    cudaStreamWaitEvent(c->user_stream, c->ev_work, 0);
  }
};

// Work-vector slots of a call: slot 1's stream starts after the work stream's queued work, and
// the work stream (hence the caller's stream) waits for slot 1 at the end of the call.
int n_slots(lqcd_ctx* c, const lqcd_solve_params& q, int n_batches) {
  if (q.pipeline < 2 || n_batches < 2 || q.solver == LQCD_SOLVER_FGCR_NN) return 1;
  cudaStream_t s1 = slot_stream(c, 1);
  cudaEventRecord(c->ev_slot, c->work);
  cudaStreamWaitEvent(s1, c->ev_slot, 0);
  return 2;
}
void join_slots(lqcd_ctx* c, int nslots) {
  if (nslots < 2) return;
  cudaEventRecord(c->ev_slot, c->slot_stream);
  cudaStreamWaitEvent(c->work, c->ev_slot, 0);
}

int cuda_check(lqcd_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(c, LQCD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return LQCD_OK;
}

// Stage `bytes` of caller data on the device: returns a device pointer (the caller's when
// where == LQCD_DEVICE).
const void* stage_in(lqcd_ctx* c, const void* p, size_t bytes, int where, const char* name) {
  if (where == LQCD_DEVICE) return p;
  void* d = ws_get(c, name, bytes);
  if (!d) return nullptr;
  cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, c->work);
  return d;
}
void* stage_out(lqcd_ctx* c, void* p, size_t bytes, int where, const char* name) {
  if (where == LQCD_DEVICE) return p;
  return ws_get(c, name, bytes);
}
int finish_out(lqcd_ctx* c, void* host, const void* dev, size_t bytes, int where) {
  if (where == LQCD_HOST) {
    cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, c->work);
    cudaError_t e = cudaStreamSynchronize(c->work);
    if (e != cudaSuccess) return set_error(c, LQCD_ERR_CUDA, cudaGetErrorString(e));
  }
  return LQCD_OK;
}

void fill_tables(lqcd_ctx* c) {
  const int T = c->g.Lt;
  for (int t = 0; t < LQCD_MAXT; t++) c->tc_full[t] = 0;
  for (int t = 0; t < T; t++) c->tc_full[t] = 1;
  c->tc_full[T - 1] = c->bc == LQCD_BC_ANTIPERIODIC ? -1 : (c->bc == LQCD_BC_OPEN ? 0 : 1);
  memset(&c->seg_full, 0, sizeof(SegInfo));
  c->seg_full.nseg = 1;
  c->seg_full.t0[0] = 0;
  c->seg_full.t1[0] = (unsigned short)T;
  // domain tables
  memset(&c->seg_dom, 0, sizeof(SegInfo));
  int n = (int)c->extents.size();
  c->seg_dom.nseg = n;
  int t = c->t_start;  // domain d covers t_start + (e_0 + ... + e_{d-1}) + [0, e_d), mod T
  for (int d = 0; d < n; d++) {
    const int e = c->extents[d];
    for (int k = 0; k < e; k++) c->seg_dom.seg_of_t[(t + k) % T] = (unsigned char)d;
    c->seg_dom.t0[d] = (unsigned short)t;
    if (t + e <= T) {
      c->seg_dom.t1[d] = (unsigned short)(t + e);
    } else {  // wraps: [t, T) and [0, t + e - T)
      c->seg_dom.t1[d] = (unsigned short)T;
      c->seg_dom.t1b[d] = (unsigned short)(t + e - T);
    }
    t = (t + e) % T;
  }
  for (int tt = 0; tt < LQCD_MAXT; tt++) c->tc_dom[tt] = 0;
  for (int tt = 0; tt < T; tt++) {
    int nx = (tt + 1) % T;
    c->tc_dom[tt] = (c->seg_dom.seg_of_t[tt] == c->seg_dom.seg_of_t[nx]) ? c->tc_full[tt] : 0;
  }
  cudaMemcpyAsync(c->d_tc_full, c->tc_full, LQCD_MAXT, cudaMemcpyHostToDevice, c->work);
  cudaMemcpyAsync(c->d_tc_dom, c->tc_dom, LQCD_MAXT, cudaMemcpyHostToDevice, c->work);
  cudaMemcpyAsync(c->d_seg_full, &c->seg_full, sizeof(SegInfo), cudaMemcpyHostToDevice, c->work);
  cudaMemcpyAsync(c->d_seg_dom, &c->seg_dom, sizeof(SegInfo), cudaMemcpyHostToDevice, c->work);
  cudaStreamSynchronize(c->work);
}

lqcd_solve_params resolve(const lqcd_solve_params* p) {
  lqcd_solve_params q;
  lqcd_default_params(&q);
  if (p) q = *p;
  if (q.tol <= 0) q.tol = 1e-10;
  return q;
}

int default_block(int nrhs_total) {
  int b = nrhs_total < 32 ? nrhs_total : 32;
  return b < 1 ? 1 : b;
}

// Accumulate a batch into the caller's stats; per-RHS arrays are written only when
// per_rhs is set (solve calls, whose caller sized them [nrhs] and [nrhs * n_seg]).
void add_stats(lqcd_solve_stats* st, const BatchStats& bs, int rhs0, int nb, int nseg, bool per_rhs = true) {
  if (!st) return;
  st->n_seg = nseg;
  if (bs.cycles > st->outer_cycles) st->outer_cycles = bs.cycles;
  st->dslash_calls += bs.dslash;
  st->fallback |= bs.fallback;
  st->device_loops += bs.device_loops;
  for (int r = 0; r < nb; r++) {
    int it = 0;
    for (int s = 0; s < nseg; s++) {
      double rel = bs.rel[r * nseg + s];
      if (rel > st->max_true_resid) st->max_true_resid = rel;
      if (per_rhs && st->true_resid) st->true_resid[(long)(rhs0 + r) * nseg + s] = rel;
      if (bs.iters[r * nseg + s] > it) it = bs.iters[r * nseg + s];
    }
    if (per_rhs && st->iters) st->iters[rhs0 + r] = it;
    st->total_iters += it;
  }
}

// The more severe of two batch outcomes: a non-finite residual outranks non-convergence.
int worse(int a, int b) {
  if (a == LQCD_ERR_NAN || b == LQCD_ERR_NAN) return LQCD_ERR_NAN;
  return a != LQCD_OK ? a : b;
}

void reset_stats(lqcd_solve_stats* st) {
  if (!st) return;
  st->n_seg = 1;
  st->outer_cycles = 0;
  st->total_iters = 0;
  st->dslash_calls = 0;
  st->max_true_resid = 0;
  st->seconds = 0;
  st->fallback = 0;
  st->device_loops = 0;
}

__global__ void k_scatter_tau(const double2* C, int nsinks, int n_ev, int nrhs, int rhs0, const int* kt_of_z,
                              const int* tp_of_z, int all, int Lt, double2* tau) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long n = (long)nsinks * n_ev * 4 * nrhs;
  if (i >= n) return;
  int r = (int)(i % nrhs);
  long q = i / nrhs;
  int alpha = (int)(q % 4);
  q /= 4;
  int m = (int)(q % n_ev);
  int z = (int)(q / n_ev);
  int jb = rhs0 + r;
  int j = jb / 4, beta = jb % 4;
  long base = all ? ((long)kt_of_z[z] * Lt + tp_of_z[z]) : (long)kt_of_z[z];
  tau[(((base * n_ev + m) * 4 + alpha) * n_ev + j) * 4 + beta] = C[i];
}

}  // namespace

extern "C" {

long long lqcd_kernel_launches(void) { return g_launches.load(); }

void lqcd_default_params(lqcd_solve_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->tol = 1e-10;
  p->max_iter = 20000;
  p->solver = LQCD_SOLVER_BICGSTAB64;
  p->inner_prec = LQCD_PREC_F32;
  p->rhs_block = 0;
  p->use_graph = 1;
  p->inner_tol = 0;
  p->max_outer = 20;
  p->check_every = 0;  // chosen per batch from its size
  p->gcr_nkrylov = 8;
  p->precond_iters = 6;
  p->pipeline = 1;
  p->projection = 0;
  p->residual = 0;
}

int lqcd_create(lqcd_ctx** out, const int L[4], int bc_t, void* stream) {
  if (!out || !L) return LQCD_ERR_INVALID_ARG;
  *out = nullptr;
  for (int m = 0; m < 4; m++)
    if (L[m] < 2 || (L[m] & 1)) {
      g_create_error = "lqcd_create: every extent must be even and >= 2";
      return LQCD_ERR_INVALID_ARG;
    }
  if (L[0] > 256 || L[1] > 256 || L[2] > 256 || L[3] > LQCD_MAXT) {
    g_create_error = "lqcd_create: extents > 256 (Lt > 256)";
    return LQCD_ERR_INVALID_ARG;
  }
  if (bc_t < LQCD_BC_PERIODIC || bc_t > LQCD_BC_OPEN) {
    g_create_error = "lqcd_create: unknown boundary condition";
    return LQCD_ERR_INVALID_ARG;
  }
  lqcd_ctx* c = new lqcd_ctx();
  c->g.Lx = L[0];
  c->g.Ly = L[1];
  c->g.Lz = L[2];
  c->g.Lt = L[3];
  c->g.Lxh = L[0] / 2;
  c->V = (long)L[0] * L[1] * L[2] * L[3];
  c->g.Vh = c->V / 2;
  c->g.Vth = (long)L[0] * L[1] * L[2] / 2;
  c->bc = bc_t;
  c->user_stream = (cudaStream_t)stream;
  cudaGetDevice(&c->device);
  if (cudaStreamCreateWithFlags(&c->work, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_user, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_work, cudaEventDisableTiming) != cudaSuccess ||
      cudaMalloc(&c->d_tc_full, LQCD_MAXT) != cudaSuccess || cudaMalloc(&c->d_tc_dom, LQCD_MAXT) != cudaSuccess ||
      cudaMalloc(&c->d_seg_full, sizeof(SegInfo)) != cudaSuccess ||
      cudaMalloc(&c->d_seg_dom, sizeof(SegInfo)) != cudaSuccess ||
      cudaMalloc(&c->d_gamma, 16 * 2 * 16 * sizeof(double2)) != cudaSuccess) {
    g_create_error = std::string("lqcd_create: ") + cudaGetErrorString(cudaGetLastError());
    lqcd_destroy(c);
    return LQCD_ERR_CUDA;
  }
  {
    // packed coordinates of every checkerboard site of each parity (s = 2 cb + b, b fixing parity)
    std::vector<unsigned> co(2 * c->g.Vh);
    for (int p = 0; p < 2; p++)
      for (long cb = 0; cb < c->g.Vh; cb++) {
        long xh = cb % c->g.Lxh, yzt = cb / c->g.Lxh;
        int y = (int)(yzt % L[1]), z = (int)((yzt / L[1]) % L[2]), t = (int)(yzt / ((long)L[1] * L[2]));
        int x = (int)(2 * xh) + ((p + y + z + t) & 1);
        co[p * c->g.Vh + cb] = (unsigned)x | ((unsigned)y << 8) | ((unsigned)z << 16) | ((unsigned)t << 24);
      }
    if (cudaMalloc(&c->d_coord, co.size() * sizeof(unsigned)) != cudaSuccess ||
        cudaMemcpy(c->d_coord, co.data(), co.size() * sizeof(unsigned), cudaMemcpyHostToDevice) != cudaSuccess) {
      g_create_error = "lqcd_create: cannot allocate the coordinate table";
      cudaGetLastError();
      lqcd_destroy(c);
      return LQCD_ERR_CUDA;
    }
  }
  c->extents.assign(1, L[3]);
  {
    const char* tv = getenv("LQCD_PHASE_TIMING");
    c->timing = tv && tv[0] == '1';
  }
  fill_tables(c);
  M4 G[16], Gt[16];
  clifford(G, Gt);
  std::vector<double2> h(16 * 2 * 16);
  for (int k = 0; k < 16; k++)
    for (int a = 0; a < 4; a++)
      for (int b = 0; b < 4; b++) {
        h[((k * 2 + 0) * 4 + a) * 4 + b] = make_double2(G[k].re[a][b], G[k].im[a][b]);
        h[((k * 2 + 1) * 4 + a) * 4 + b] = make_double2(Gt[k].re[a][b], Gt[k].im[a][b]);
      }
  cudaMemcpy(c->d_gamma, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice);
  if (cuda_check(c, "lqcd_create")) {
    g_create_error = c->err;
    lqcd_destroy(c);
    return LQCD_ERR_CUDA;
  }
  *out = c;
  return LQCD_OK;
}

int lqcd_phase_times(lqcd_ctx* c, char* buf, int len, int reset) {
  if (!c || !buf || len < 3) return set_error(c, LQCD_ERR_INVALID_ARG, "phase_times: bad arguments");
  flush_phase_times(c);
  std::string s = "{";
  for (auto& kv : c->phase_ms) {
    char item[160];
    snprintf(item, sizeof item, "%s\"%s\": %.6f", s.size() > 1 ? ", " : "", kv.first.c_str(), kv.second);
    s += item;
  }
  s += "}";
  if ((int)s.size() >= len) return set_error(c, LQCD_ERR_INVALID_ARG, "phase_times: buffer too small");
  memcpy(buf, s.c_str(), s.size() + 1);
  if (reset) c->phase_ms.clear();
  return LQCD_OK;
}

int lqcd_destroy(lqcd_ctx* c) {
  if (!c) return LQCD_OK;
  if (c->work) cudaStreamSynchronize(c->work);
  flush_phase_times(c);
  drop_graphs(c);
  for (auto& kv : c->ws) cudaFree(kv.second.p);
  for (void* p : c->slot_pinned)
    if (p) cudaFreeHost(p);
  if (c->slot_stream) cudaStreamDestroy(c->slot_stream);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->ev_slot) cudaEventDestroy(c->ev_slot);
  void* bufs[] = {c->U64, c->U32, c->U16, c->Usm, c->A64, c->Ainv64, c->Ainv32, c->Ainv16, c->A32, c->Udf, c->Adf,
                  c->d_tc_full, c->d_tc_dom, c->d_seg_full, c->d_seg_dom, c->d_gamma, c->d_coord,
                  c->nn_weights, c->nn_w16, c->nn_m, c->nn_v};
  for (void* p : bufs)
    if (p) cudaFree(p);
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->ev_user) cudaEventDestroy(c->ev_user);
  if (c->ev_work) cudaEventDestroy(c->ev_work);
  if (c->work) cudaStreamDestroy(c->work);
  delete c;
  return LQCD_OK;
}

int lqcd_release_workspace(lqcd_ctx* c) {
  if (!c) return LQCD_ERR_INVALID_ARG;
  drop_graphs(c);
  for (auto& kv : c->ws) cudaFree(kv.second.p);
  c->ws.clear();
  for (int i = 0; i < 3; i++) c->nn_buf[i] = nullptr;
  return cuda_check(c, "release_workspace");
}

int lqcd_set_stream(lqcd_ctx* c, void* stream) {
  if (!c) return LQCD_ERR_INVALID_ARG;
  c->user_stream = (cudaStream_t)stream;
  return LQCD_OK;
}

const char* lqcd_last_error(const lqcd_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

int lqcd_gauge_upload(lqcd_ctx* c, const double* links, int where, double kappa, double c_sw) {
  if (!c || !links) return set_error(c, LQCD_ERR_INVALID_ARG, "gauge_upload: NULL argument");
  if (!std::isfinite(kappa) || !std::isfinite(c_sw))
    return set_error(c, LQCD_ERR_INVALID_ARG, "gauge_upload: kappa and c_sw must be finite");
  Scope sc(c);
  const Geom& g = c->g;
  auto need = [&](void*& p, size_t b) {
    if (!p && cudaMalloc(&p, b) != cudaSuccess) p = nullptr;
    return p != nullptr;
  };
  bool ok = need(c->U64, link_bytes(g, P64)) && need(c->U32, link_bytes(g, P32)) &&
            need(c->U16, link_bytes(g, P16)) && need(c->A64, 2 * clover_bytes(g, P64)) &&
            need(c->Ainv64, 2 * clover_bytes(g, P64)) && need(c->A32, 2 * clover_bytes(g, P32)) &&
            need(c->Ainv32, 2 * clover_bytes(g, P32)) && need(c->Ainv16, 2 * clover_bytes(g, P16)) &&
            need(c->Udf, link_bytes(g, P64)) && need(c->Adf, 2 * clover_bytes(g, P64));
  if (!ok) {
    cudaGetLastError();
    return set_error(c, LQCD_ERR_OOM, "gauge_upload: out of device memory");
  }
  if (kappa != c->kappa) drop_graphs(c);  // captured Schur launches hold -kappa^2 by value: recapture them
  c->have_gauge = false;
  c->kappa = kappa;
  c->csw = c_sw;
  size_t bytes = (size_t)c->V * 4 * 9 * sizeof(double2);
  const double2* d = (const double2*)stage_in(c, links, bytes, where, "h_links");
  int* bad = (int*)ws_get(c, "bad", 64);
  if (!d || !bad) return set_error(c, LQCD_ERR_OOM, "gauge_upload: out of device memory");
  cudaMemsetAsync(bad, 0, sizeof(int), c->work);
  build_gauge(c, d, bad);
  split_field(c->U64, c->Udf, (long)(link_bytes(g, P64) / 16), c->work);
  split_field(c->A64, c->Adf, (long)(2 * clover_bytes(g, P64) / 16), c->work);
  int hb = 0;
  cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, c->work);
  cudaError_t e = cudaStreamSynchronize(c->work);
  if (e != cudaSuccess) return set_error(c, LQCD_ERR_CUDA, std::string("gauge_upload: ") + cudaGetErrorString(e));
  if (hb) return set_error(c, LQCD_ERR_NAN, "gauge_upload: singular clover block");
  c->have_gauge = true;
  c->have_smeared = false;  // a new field drops the previous smearing
  return LQCD_OK;
}

int lqcd_ape_smear(lqcd_ctx* c, double alpha, int n_iter) {
  if (!c || n_iter < 0 || !(alpha >= 0.0 && alpha <= 1.0))
    return set_error(c, LQCD_ERR_INVALID_ARG, "ape_smear: bad arguments");
  if (!c->have_gauge) return set_error(c, LQCD_ERR_STATE, "ape_smear: no gauge field uploaded");
  Scope sc(c);
  return ape_smear(c, alpha, n_iter);
}

int lqcd_smeared_links(lqcd_ctx* c, double* out, int where) {
  if (!c || !out) return set_error(c, LQCD_ERR_INVALID_ARG, "smeared_links: bad arguments");
  if (!c->have_smeared) return set_error(c, LQCD_ERR_STATE, "smeared_links: no smeared field");
  Scope sc(c);
  const size_t bytes = (size_t)c->V * 27 * sizeof(double2);
  double2* dout = (double2*)stage_out(c, out, bytes, where, "h_sm");
  if (!dout) return set_error(c, LQCD_ERR_OOM, "smeared_links: out of device memory");
  unpack_smeared(c, dout);
  if (int e = cuda_check(c, "smeared_links")) return e;
  return finish_out(c, out, dout, bytes, where);
}

int lqcd_set_domains(lqcd_ctx* c, const int* extents, int n_dom) { return lqcd_set_domains_at(c, 0, extents, n_dom); }

int lqcd_set_domains_at(lqcd_ctx* c, int t_start, const int* extents, int n_dom) {
  if (!c || !extents || n_dom < 1 || n_dom > c->g.Lt || t_start < 0 || t_start >= c->g.Lt)
    return set_error(c, LQCD_ERR_INVALID_ARG, "set_domains: bad arguments");
  int sum = 0;
  for (int d = 0; d < n_dom; d++) {
    if (extents[d] < 1) return set_error(c, LQCD_ERR_INVALID_ARG, "set_domains: extent < 1");
    sum += extents[d];
  }
  if (sum != c->g.Lt) return set_error(c, LQCD_ERR_INVALID_ARG, "set_domains: extents do not tile Lt");
  cudaStreamSynchronize(c->work);
  c->extents.assign(extents, extents + n_dom);
  c->t_start = t_start;
  fill_tables(c);
  return LQCD_OK;
}

int lqcd_dirac_apply(lqcd_ctx* c, const double* in, double* out, int nrhs, int domain, int where) {
  if (!c || !in || !out || nrhs < 1) return set_error(c, LQCD_ERR_INVALID_ARG, "dirac_apply: bad arguments");
  if (!c->have_gauge) return set_error(c, LQCD_ERR_STATE, "dirac_apply: no gauge field uploaded");
  Scope sc(c);
  size_t bytes = (size_t)c->V * 12 * nrhs * sizeof(double2);
  const double2* din = (const double2*)stage_in(c, in, bytes, where, "h_in");
  double2* dout = (double2*)stage_out(c, out, bytes, where, "h_out");
  double2* ein = (double2*)ws_get(c, "eo_in", bytes);
  double2* eout = (double2*)ws_get(c, "eo_out", bytes);
  if (!din || !dout || !ein || !eout) return set_error(c, LQCD_ERR_OOM, "dirac_apply: out of device memory");
  pack_spinor(c->g, din, ein, nrhs, c->work);
  apply_D(c, ein, eout, nrhs, domain, c->work);
  unpack_spinor(c->g, eout, dout, nrhs, c->work);
  if (int e = cuda_check(c, "dirac_apply")) return e;
  return finish_out(c, out, dout, bytes, where);
}

int lqcd_schur_apply(lqcd_ctx* c, int prec, const double* in, double* out, int nrhs, int domain, int where) {
  if (!c || !in || !out || nrhs < 1 ||
      (prec != LQCD_PREC_F64 && prec != LQCD_PREC_F32 && prec != LQCD_PREC_F16))
    return set_error(c, LQCD_ERR_INVALID_ARG, "schur_apply: bad arguments");
  if (!c->have_gauge) return set_error(c, LQCD_ERR_STATE, "schur_apply: no gauge field uploaded");
  const int P = prec == LQCD_PREC_F64 ? P64 : (prec == LQCD_PREC_F32 ? P32 : P16);
  Scope sc(c);
  const size_t bytes = (size_t)c->V * 12 * nrhs * sizeof(double2);
  const double2* din = (const double2*)stage_in(c, in, bytes, where, "h_in");
  double2* dout = (double2*)stage_out(c, out, bytes, where, "h_out");
  double2* ein = (double2*)ws_get(c, "eo_in", bytes);
  double2* eout = (double2*)ws_get(c, "eo_out", bytes);
  if (!din || !dout || !ein || !eout) return set_error(c, LQCD_ERR_OOM, "schur_apply: out of device memory");
  pack_spinor(c->g, din, ein, nrhs, c->work);
  cudaMemsetAsync((char*)eout + bytes / 2, 0, bytes / 2, c->work);  // odd parity block
  if (int e = schur_apply(c, P, ein, eout, nrhs, domain, c->work)) return e;
  unpack_spinor(c->g, eout, dout, nrhs, c->work);
  if (int e = cuda_check(c, "schur_apply")) return e;
  if (dslash_pipe_timeouts(true))
    return set_error(c, LQCD_ERR_TIMEOUT, "schur_apply: a staged dslash copy did not complete within its wait limit");
  return finish_out(c, out, dout, bytes, where);
}

static int solve_common(lqcd_ctx* c, const double* b, double* x, int nrhs, int where, const lqcd_solve_params* p,
                        lqcd_solve_stats* st, int domain) {
  if (!c || !b || !x || nrhs < 1) return set_error(c, LQCD_ERR_INVALID_ARG, "solve: bad arguments");
  if (!c->have_gauge) return set_error(c, LQCD_ERR_STATE, "solve: no gauge field uploaded");
  auto t0 = std::chrono::steady_clock::now();
  lqcd_solve_params q = resolve(p);
  reset_stats(st);
  Scope sc(c);
  const size_t per = (size_t)c->V * 12 * sizeof(double2);
  const double2* db = (const double2*)stage_in(c, b, per * nrhs, where, "h_in");
  double2* dx = (double2*)stage_out(c, x, per * nrhs, where, "h_out");
  if (!db || !dx) return set_error(c, LQCD_ERR_OOM, "solve: out of device memory");
  const int blk = q.rhs_block > 0 ? q.rhs_block : default_block(nrhs);
  int rc = LQCD_OK;
  const int nseg = domain ? c->seg_dom.nseg : 1;
  const int nbatch = (nrhs + blk - 1) / blk;
  const int nsl = n_slots(c, q, nbatch);
  struct Pending {
    BatchHandle h;
    int r0 = -1, nb = 0;
    double2* ex = nullptr;
  } pend[2];
  // finish the batch of a slot: stats, and its solution unpacked on the slot's stream
  auto finish = [&](Pending& pd) -> int {
    if (pd.r0 < 0) return LQCD_OK;
    BatchStats bs;
    int r = solve_batch_finish(c, pd.h, bs);
    if (r != LQCD_OK && r != LQCD_ERR_NOT_CONVERGED && r != LQCD_ERR_NAN) return r;
    rc = worse(rc, r);
    add_stats(st, bs, pd.r0, pd.nb, nseg);
    pd.r0 = -1;
    return LQCD_OK;
  };
  for (int k = 0; k < nbatch; k++) {
    const int s = k % nsl, r0 = k * blk;
    const int nb = nrhs - r0 < blk ? nrhs - r0 : blk;
    if (int e = finish(pend[s])) return e;
    cudaStream_t ss = slot_stream(c, s);
    double2* eb = (double2*)ws_get(c, s ? "eo_b#1" : "eo_b", per * nb);
    double2* ex = (double2*)ws_get(c, s ? "eo_x#1" : "eo_x", per * nb);
    if (!eb || !ex) return set_error(c, LQCD_ERR_OOM, "solve: out of device memory");
    pack_spinor(c->g, db + (size_t)r0 * c->V * 12, eb, nb, ss);
    if (int e = solve_batch_enqueue(c, s, eb, ex, nb, domain, q, pend[s].h)) return e;
    unpack_spinor(c->g, ex, dx + (size_t)r0 * c->V * 12, nb, ss);
    pend[s].r0 = r0;
    pend[s].nb = nb;
    pend[s].ex = ex;
  }
  for (int s = 0; s < nsl; s++)
    if (int e = finish(pend[s])) return e;
  join_slots(c, nsl);
  if (int e = cuda_check(c, "solve")) return e;
  int fo = finish_out(c, x, dx, per * nrhs, where);
  if (fo) return fo;
  if (st) st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (rc == LQCD_ERR_NAN) set_error(c, rc, "solve: non-finite residual (NaN or Inf in a source or iterate)");
  else if (rc != LQCD_OK) set_error(c, rc, "solve: tolerance not reached");
  return rc;
}

int lqcd_solve_full(lqcd_ctx* c, const double* b, double* x, int nrhs, int where, const lqcd_solve_params* p,
                    lqcd_solve_stats* st) {
  return solve_common(c, b, x, nrhs, where, p, st, 0);
}

int lqcd_solve_domain(lqcd_ctx* c, const double* b, double* x, int nrhs, int where, const lqcd_solve_params* p,
                      lqcd_solve_stats* st) {
  return solve_common(c, b, x, nrhs, where, p, st, 1);
}

// Perambulators of the source vectors j in [j0, j0 + nj) (all four spins each).  sinks:
// DIAG / ALL with Vt holding every timeslice, DIAG_SRCV with Vt holding only the source
// timeslices in t_src order.  Columns of tau outside [j0, j0 + nj) are left untouched.
static int perambulator_impl(lqcd_ctx* c, const double* Vt, int n_ev, const int* t_src, int n_tsrc, int mode,
                             int sinks, int j0, int nj, int where, double* tau, const lqcd_solve_params* p,
                             lqcd_solve_stats* st) {
  if (!c || !Vt || !t_src || !tau || n_tsrc < 1) return set_error(c, LQCD_ERR_INVALID_ARG, "perambulator: NULL");
  const Geom& g = c->g;
  const long L3 = (long)g.Lx * g.Ly * g.Lz;
  if (n_ev < 1 || n_ev > 3 * L3) return set_error(c, LQCD_ERR_INVALID_ARG, "perambulator: bad n_ev");
  if (j0 < 0 || nj < 1 || j0 + nj > n_ev)
    return set_error(c, LQCD_ERR_INVALID_ARG, "perambulator: source vector range outside [0, n_ev)");
  if (mode != LQCD_MODE_FULL && mode != LQCD_MODE_DOMAIN)
    return set_error(c, LQCD_ERR_INVALID_ARG, "perambulator: bad mode");
  if (sinks != LQCD_SINKS_DIAG && sinks != LQCD_SINKS_ALL && sinks != LQCD_SINKS_DIAG_SRCV)
    return set_error(c, LQCD_ERR_INVALID_ARG, "perambulator: bad sinks");
  if (sinks == LQCD_SINKS_ALL && mode == LQCD_MODE_DOMAIN)
    return set_error(c, LQCD_ERR_INVALID_ARG, "perambulator: all sinks only in full mode");
  if (n_tsrc > g.Lt) return set_error(c, LQCD_ERR_INVALID_ARG, "perambulator: more source timeslices than Lt");
  for (int k = 0; k < n_tsrc; k++)
    if (t_src[k] < 0 || t_src[k] >= g.Lt) return set_error(c, LQCD_ERR_INVALID_ARG, "perambulator: bad t");
  const bool vsrc = sinks == LQCD_SINKS_DIAG_SRCV;
  std::vector<int> vslot(LQCD_MAXT, -1);  // slot of each timeslice in Vt
  for (int t = 0; t < g.Lt && !vsrc; t++) vslot[t] = t;
  for (int k = 0; k < n_tsrc && vsrc; k++) {
    if (vslot[t_src[k]] >= 0)
      return set_error(c, LQCD_ERR_INVALID_ARG, "perambulator: repeated source timeslice with per-source vectors");
    vslot[t_src[k]] = k;
  }
  if (!c->have_gauge) return set_error(c, LQCD_ERR_STATE, "perambulator: no gauge field uploaded");
  auto t0 = std::chrono::steady_clock::now();
  lqcd_solve_params q = resolve(p);
  reset_stats(st);
  Scope sc(c);
  const int domain = mode == LQCD_MODE_DOMAIN;
  // source groups: full mode one timeslice each; domain mode at most one timeslice per domain
  std::vector<std::vector<int>> groups;  // entries are indices k into t_src
  if (!domain) {
    for (int k = 0; k < n_tsrc; k++) groups.push_back({k});
  } else {
    int nd = c->seg_dom.nseg;
    std::vector<std::vector<int>> q_by_dom(nd);
    for (int k = 0; k < n_tsrc; k++) q_by_dom[c->seg_dom.seg_of_t[t_src[k]]].push_back(k);
    for (size_t level = 0;; level++) {
      std::vector<int> grp;
      for (int d = 0; d < nd; d++)
        if (level < q_by_dom[d].size()) grp.push_back(q_by_dom[d][level]);
      if (grp.empty()) break;
      groups.push_back(grp);
    }
  }
  const size_t vbytes = (size_t)(vsrc ? n_tsrc : g.Lt) * n_ev * L3 * 3 * sizeof(double2);
  const double2* dV = (const double2*)stage_in(c, Vt, vbytes, where, "h_V");
  const long n_tp = sinks == LQCD_SINKS_ALL ? g.Lt : 1;
  const size_t tau_bytes = (size_t)n_tsrc * n_tp * n_ev * 4 * n_ev * 4 * sizeof(double2);
  // host output: untouched columns must survive the round trip through the staging buffer
  double2* dtau = (double2*)(where == LQCD_DEVICE ? (void*)tau
                                                  : (nj < n_ev ? (void*)stage_in(c, tau, tau_bytes, where, "h_tau")
                                                               : stage_out(c, tau, tau_bytes, where, "h_tau")));
  if (!dV || !dtau) return set_error(c, LQCD_ERR_OOM, "perambulator: out of device memory");
  const int rhs_begin = 4 * j0, rhs_end = 4 * (j0 + nj);
  const int nrhs_total = rhs_end - rhs_begin;
  const int blk = q.rhs_block > 0 ? q.rhs_block : default_block(nrhs_total);
  const size_t per = (size_t)c->V * 12 * sizeof(double2);
  const int nseg = domain ? c->seg_dom.nseg : 1;
  const int nbatch = (int)groups.size() * ((nrhs_total + blk - 1) / blk);
  // double-float projection: the colour vectors split once per call, the solution per batch
  float4* Vf = nullptr;
  if (q.projection == 0) {
    const long nv = (long)(vsrc ? n_tsrc : g.Lt) * n_ev * 3 * L3;
    Vf = (float4*)ws_get(c, "p_Vf", (size_t)nv * sizeof(float4));
    if (!Vf) return set_error(c, LQCD_ERR_OOM, "perambulator: OOM");
    split_colour_vectors(dV, Vf, nv, c->work);
  }
  const int nsl = n_slots(c, q, nbatch);
  // per-slot buffers: sources, solutions, tables, projection scratch
  struct Slot {
    int* jb;
    unsigned char* mask;
    int* z;
    double2 *eb, *ex, *C;
    BatchHandle h;
    bool busy = false;
  } sl[2];
  for (int s = 0; s < nsl; s++) {
    const std::string sfx = s ? "#1" : "";
    sl[s].jb = (int*)ws_get(c, "p_jb" + sfx, 2 * blk * sizeof(int));
    sl[s].mask = (unsigned char*)ws_get(c, "p_mask" + sfx, LQCD_MAXT);
    sl[s].z = (int*)ws_get(c, "p_z" + sfx, 3 * LQCD_MAXT * sizeof(int));  // sink t', source slot k, V slot of t
    sl[s].eb = (double2*)ws_get(c, "eo_b" + sfx, per * blk);
    sl[s].ex = (double2*)ws_get(c, "eo_x" + sfx, per * blk);
    sl[s].C = (double2*)ws_get(c, "p_C" + sfx, (size_t)g.Lt * n_ev * 4 * blk * sizeof(double2));
    if (!sl[s].jb || !sl[s].mask || !sl[s].z || !sl[s].eb || !sl[s].ex || !sl[s].C)
      return set_error(c, LQCD_ERR_OOM, "perambulator: OOM");
  }
  int rc = LQCD_OK;
  auto finish = [&](Slot& S) -> int {
    if (!S.busy) return LQCD_OK;
    BatchStats bs;
    int r = solve_batch_finish(c, S.h, bs);
    S.busy = false;
    if (r != LQCD_OK && r != LQCD_ERR_NOT_CONVERGED && r != LQCD_ERR_NAN) return r;
    rc = worse(rc, r);
    add_stats(st, bs, 0, (int)bs.iters.size() / nseg, nseg, false);
    return LQCD_OK;
  };
  int kb = 0;
  for (auto& grp : groups) {
    unsigned char mask[LQCD_MAXT];
    memset(mask, 0, sizeof mask);
    for (int k : grp) mask[t_src[k]] = 1;
    std::vector<int> kz, tz;
    if (sinks != LQCD_SINKS_ALL) {
      for (int k : grp) {
        kz.push_back(k);
        tz.push_back(t_src[k]);
      }
    } else {
      for (int tp = 0; tp < g.Lt; tp++) {
        kz.push_back(grp[0]);
        tz.push_back(tp);
      }
    }
    int nz = (int)kz.size();
    std::vector<int> hz(3 * LQCD_MAXT);
    for (int z = 0; z < nz; z++) {
      hz[z] = tz[z];
      hz[LQCD_MAXT + z] = kz[z];
    }
    for (int t = 0; t < LQCD_MAXT; t++) hz[2 * LQCD_MAXT + t] = vslot[t];
    for (int r0 = rhs_begin; r0 < rhs_end; r0 += blk, kb++) {
      const int s = kb % nsl;
      Slot& S = sl[s];
      if (int e = finish(S)) return e;  // the slot's previous batch (its queued work is ordered anyway)
      cudaStream_t ss = slot_stream(c, s);
      const int nb = rhs_end - r0 < blk ? rhs_end - r0 : blk;
      std::vector<int> hjb(2 * blk);
      for (int r = 0; r < nb; r++) {
        hjb[r] = (r0 + r) / 4;
        hjb[blk + r] = (r0 + r) % 4;
      }
      // pageable sources: the copies complete (staged) before these calls return
      cudaMemcpyAsync(S.mask, mask, LQCD_MAXT, cudaMemcpyHostToDevice, ss);
      cudaMemcpyAsync(S.z, hz.data(), 3 * LQCD_MAXT * sizeof(int), cudaMemcpyHostToDevice, ss);
      cudaMemcpyAsync(S.jb, hjb.data(), 2 * blk * sizeof(int), cudaMemcpyHostToDevice, ss);
      make_sources(g, dV, n_ev, S.jb, S.jb + blk, S.mask, S.z + 2 * LQCD_MAXT, S.eb, nb, ss);
      if (int e = solve_batch_enqueue(c, s, S.eb, S.ex, nb, domain, q, S.h)) return e;
      S.busy = true;
      const int pbs = 4;  // blocks per SM of the projection
      const int ks = project_ksplit(g, n_ev, nb, nz, pbs);
      double2* Cp = (double2*)ws_get(c, s ? "p_Cpart#1" : "p_Cpart", (size_t)ks * nz * n_ev * 4 * nb * sizeof(double2));
      if (!Cp) return set_error(c, LQCD_ERR_OOM, "perambulator: OOM");
      float4* Xf = nullptr;
      if (Vf) {
        Xf = (float4*)ws_get(c, s ? "p_Xf#1" : "p_Xf", (size_t)nz * 4 * nb * 3 * L3 * sizeof(float4));
        if (!Xf) return set_error(c, LQCD_ERR_OOM, "perambulator: OOM");
      }
      project(g, dV, n_ev, S.ex, S.z, S.z + 2 * LQCD_MAXT, nz, S.C, Cp, nb, pbs, nsl > 1, Vf, Xf, ss);
      long n = (long)nz * n_ev * 4 * nb;
      k_scatter_tau<<<(n + 255) / 256, 256, 0, ss>>>(S.C, nz, n_ev, nb, r0, S.z + LQCD_MAXT, S.z,
                                                     sinks == LQCD_SINKS_ALL, g.Lt, dtau); lqcd::count_launch();
      if (int e = cuda_check(c, "perambulator")) return e;
    }
  }
  for (int s = 0; s < nsl; s++)
    if (int e = finish(sl[s])) return e;
  join_slots(c, nsl);
  int fo = finish_out(c, tau, dtau, tau_bytes, where);
  if (fo) return fo;
  cudaStreamSynchronize(c->work);
  if (st) st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (rc == LQCD_ERR_NAN) set_error(c, rc, "perambulator: non-finite residual (NaN or Inf in the colour vectors)");
  else if (rc != LQCD_OK) set_error(c, rc, "perambulator: tolerance not reached");
  return rc;
}

int lqcd_perambulator(lqcd_ctx* c, const double* Vt, int n_ev, const int* t_src, int n_tsrc, int mode, int sinks,
                      int where, double* tau, const lqcd_solve_params* p, lqcd_solve_stats* st) {
  return perambulator_impl(c, Vt, n_ev, t_src, n_tsrc, mode, sinks, 0, n_ev, where, tau, p, st);
}

int lqcd_perambulator_cols(lqcd_ctx* c, const double* Vt, int n_ev, const int* t_src, int n_tsrc, int mode,
                           int sinks, int j0, int nj, int where, double* tau, const lqcd_solve_params* p,
                           lqcd_solve_stats* st) {
  return perambulator_impl(c, Vt, n_ev, t_src, n_tsrc, mode, sinks, j0, nj, where, tau, p, st);
}

int lqcd_loops(lqcd_ctx* c, const double* tau, int n_ev, int n_t, const int* gamma_ids, int n_gamma,
               const double* weights, double* L, double* Lt, int where) {
  if (!c || !tau || !gamma_ids || !L || !Lt || n_ev < 1 || n_t < 1 || n_gamma < 1 || n_gamma > 16)
    return set_error(c, LQCD_ERR_INVALID_ARG, "loops: bad arguments");
  for (int k = 0; k < n_gamma; k++)
    if (gamma_ids[k] < 0 || gamma_ids[k] > 15) return set_error(c, LQCD_ERR_INVALID_ARG, "loops: bad gamma id");
  Scope sc(c);
  size_t tb = (size_t)n_t * n_ev * 4 * n_ev * 4 * sizeof(double2);
  const double2* dt = (const double2*)stage_in(c, tau, tb, where, "l_tau");
  const double* dw = weights ? (const double*)stage_in(c, weights, (size_t)n_t * n_ev * sizeof(double), where,
                                                       "l_w")
                             : nullptr;
  size_t lb = (size_t)n_gamma * n_t * sizeof(double2);
  double2* dL = (double2*)stage_out(c, L, lb, where, "l_L");
  double2* dLt = (double2*)stage_out(c, Lt, lb, where, "l_Lt");
  double2* dG = (double2*)ws_get(c, "l_G", 16 * 2 * 16 * sizeof(double2));
  if (!dt || !dL || !dLt || !dG || (weights && !dw)) return set_error(c, LQCD_ERR_OOM, "loops: OOM");
  for (int k = 0; k < n_gamma; k++)
    cudaMemcpyAsync(dG + (size_t)k * 32, c->d_gamma + (size_t)gamma_ids[k] * 32, 32 * sizeof(double2),
                    cudaMemcpyDeviceToDevice, c->work);
  loops(dt, n_ev, n_t, dG, n_gamma, dw, dL, dLt, c->work);
  if (int e = cuda_check(c, "loops")) return e;
  if (int e = finish_out(c, L, dL, lb, where)) return e;
  return finish_out(c, Lt, dLt, lb, where);
}

int lqcd_conn_correlator(lqcd_ctx* c, const double* tau_all, int n_ev, const int* t_src, int n_t,
                         const int* gamma_ids, int n_gamma, double* C, double* C_avg, int where) {
  if (!c || !tau_all || !t_src || !gamma_ids || !C || n_ev < 1 || n_t < 1 || n_gamma < 1 || n_gamma > 16)
    return set_error(c, LQCD_ERR_INVALID_ARG, "conn_correlator: bad arguments");
  const int T = c->g.Lt;
  for (int k = 0; k < n_t; k++)
    if (t_src[k] < 0 || t_src[k] >= T) return set_error(c, LQCD_ERR_INVALID_ARG, "conn_correlator: bad t");
  for (int k = 0; k < n_gamma; k++)
    if (gamma_ids[k] < 0 || gamma_ids[k] > 15)
      return set_error(c, LQCD_ERR_INVALID_ARG, "conn_correlator: bad gamma id");
  Scope sc(c);
  const size_t tb = (size_t)n_t * T * n_ev * 4 * n_ev * 4 * sizeof(double2);
  const size_t cb = (size_t)n_gamma * T * n_t * sizeof(double2), ab = (size_t)n_gamma * T * sizeof(double2);
  const double2* dtau = (const double2*)stage_in(c, tau_all, tb, where, "cc_tau");
  double2* dC = (double2*)stage_out(c, C, cb, where, "cc_C");
  double2* dA = C_avg ? (double2*)stage_out(c, C_avg, ab, where, "cc_A") : nullptr;
  double2* dG = (double2*)ws_get(c, "cc_G", 16 * 2 * 16 * sizeof(double2));
  int* dts = (int*)ws_get(c, "cc_t", (size_t)n_t * sizeof(int));
  if (!dtau || !dC || (C_avg && !dA) || !dG || !dts) return set_error(c, LQCD_ERR_OOM, "conn_correlator: OOM");
  for (int k = 0; k < n_gamma; k++)
    cudaMemcpyAsync(dG + (size_t)k * 32, c->d_gamma + (size_t)gamma_ids[k] * 32, 32 * sizeof(double2),
                    cudaMemcpyDeviceToDevice, c->work);
  cudaMemcpyAsync(dts, t_src, (size_t)n_t * sizeof(int), cudaMemcpyHostToDevice, c->work);
  conn_correlator(dtau, n_ev, T, dts, n_t, dG, n_gamma, dC, dA, c->work);
  if (int e = cuda_check(c, "conn_correlator")) return e;
  if (int e = finish_out(c, C, dC, cb, where)) return e;
  return C_avg ? finish_out(c, C_avg, dA, ab, where) : LQCD_OK;
}

int lqcd_nr_estimator(lqcd_ctx* c, const double* C_conn_avg, const double* C_disc_avg, const double* dC_avg,
                      int n_delta, int n_gamma, const int* delta_of_dt, double* C_nr, int where) {
  if (!c || !C_conn_avg || !C_disc_avg || !delta_of_dt || !C_nr || n_gamma < 1 || n_delta < 0 ||
      (n_delta > 0 && !dC_avg))
    return set_error(c, LQCD_ERR_INVALID_ARG, "nr_estimator: bad arguments");
  const int T = c->g.Lt;
  for (int t = 0; t < T; t++)
    if (delta_of_dt[t] < -1 || delta_of_dt[t] >= n_delta)
      return set_error(c, LQCD_ERR_INVALID_ARG, "nr_estimator: delta index out of range");
  Scope sc(c);
  const size_t ab = (size_t)n_gamma * T * sizeof(double2);
  const double2* dc = (const double2*)stage_in(c, C_conn_avg, ab, where, "nr_c");
  const double2* dd = (const double2*)stage_in(c, C_disc_avg, ab, where, "nr_d");
  const double2* ddc = n_delta > 0 ? (const double2*)stage_in(c, dC_avg, n_delta * ab, where, "nr_dc") : nullptr;
  double2* dout = (double2*)stage_out(c, C_nr, ab, where, "nr_o");
  int* ddel = (int*)ws_get(c, "nr_del", (size_t)T * sizeof(int));
  if (!dc || !dd || (n_delta > 0 && !ddc) || !dout || !ddel) return set_error(c, LQCD_ERR_OOM, "nr_estimator: OOM");
  cudaMemcpyAsync(ddel, delta_of_dt, (size_t)T * sizeof(int), cudaMemcpyHostToDevice, c->work);
  nr_estimator(dc, dd, ddc, n_gamma, T, ddel, dout, c->work);
  if (int e = cuda_check(c, "nr_estimator")) return e;
  return finish_out(c, C_nr, dout, ab, where);
}

int lqcd_disc_correlator(lqcd_ctx* c, const double* L, const double* Lt, const double* Ld, const double* Ltd,
                         int n_cfg, int n_gamma, int vev, double* C, double* Cdd, double* dC, double* C_avg,
                         double* dC_avg, int* valid, int* n_valid, double* terms, int where) {
  if (!c || !L || !Lt || !Ld || !Ltd || !C || !Cdd || !dC || !C_avg || !dC_avg || !valid || !n_valid ||
      n_cfg < 1 || n_gamma < 1)
    return set_error(c, LQCD_ERR_INVALID_ARG, "disc_correlator: bad arguments");
  if (vev && n_cfg < 2)
    return set_error(c, LQCD_ERR_INVALID_ARG, "disc_correlator: the VEV subtraction needs n_cfg >= 2");
  const int T = c->g.Lt;
  Scope sc(c);
  size_t lb = (size_t)n_cfg * n_gamma * T * sizeof(double2);
  const double2* a = (const double2*)stage_in(c, L, lb, where, "c_L");
  const double2* b = (const double2*)stage_in(c, Lt, lb, where, "c_Lt");
  const double2* ad = (const double2*)stage_in(c, Ld, lb, where, "c_Ld");
  const double2* bd = (const double2*)stage_in(c, Ltd, lb, where, "c_Ltd");
  size_t cb = (size_t)n_gamma * T * T * sizeof(double2), ab = (size_t)n_gamma * T * sizeof(double2);
  double2* dCo = (double2*)stage_out(c, C, cb, where, "c_C");
  double2* dCdd = (double2*)stage_out(c, Cdd, cb, where, "c_Cdd");
  double2* ddC = (double2*)stage_out(c, dC, cb, where, "c_dC");
  double2* dCa = (double2*)stage_out(c, C_avg, ab, where, "c_Ca");
  double2* ddCa = (double2*)stage_out(c, dC_avg, ab, where, "c_dCa");
  int* dvalid = (int*)stage_out(c, valid, (size_t)T * T * sizeof(int), where, "c_valid");
  int* dnv = (int*)stage_out(c, n_valid, (size_t)T * sizeof(int), where, "c_nv");
  double2* dterms = terms ? (double2*)stage_out(c, terms, 4 * cb, where, "c_terms") : nullptr;
  double2* tmp1 = (double2*)ws_get(c, "c_dL", lb);
  double2* tmp2 = (double2*)ws_get(c, "c_dLt", lb);
  int* ddom = (int*)ws_get(c, "c_dom", T * sizeof(int));
  if (!a || !b || !ad || !bd || !dCo || !dCdd || !ddC || !dCa || !ddCa || !dvalid || !dnv || !tmp1 || !tmp2 ||
      !ddom || (terms && !dterms))
    return set_error(c, LQCD_ERR_OOM, "disc_correlator: OOM");
  std::vector<int> dom(T);
  for (int t = 0; t < T; t++) dom[t] = c->seg_dom.seg_of_t[t];
  cudaMemcpyAsync(ddom, dom.data(), T * sizeof(int), cudaMemcpyHostToDevice, c->work);
  correlators(a, b, ad, bd, n_cfg, n_gamma, T, vev, ddom, dCo, dCdd, ddC, dCa, ddCa, dvalid, dnv, dterms, tmp1,
              tmp2, c->work);
  if (int e = cuda_check(c, "disc_correlator")) return e;
  if (where == LQCD_HOST) {
    cudaMemcpyAsync(C, dCo, cb, cudaMemcpyDeviceToHost, c->work);
    cudaMemcpyAsync(Cdd, dCdd, cb, cudaMemcpyDeviceToHost, c->work);
    cudaMemcpyAsync(dC, ddC, cb, cudaMemcpyDeviceToHost, c->work);
    cudaMemcpyAsync(C_avg, dCa, ab, cudaMemcpyDeviceToHost, c->work);
    cudaMemcpyAsync(dC_avg, ddCa, ab, cudaMemcpyDeviceToHost, c->work);
    cudaMemcpyAsync(valid, dvalid, (size_t)T * T * sizeof(int), cudaMemcpyDeviceToHost, c->work);
    cudaMemcpyAsync(n_valid, dnv, (size_t)T * sizeof(int), cudaMemcpyDeviceToHost, c->work);
    if (terms) cudaMemcpyAsync(terms, dterms, 4 * cb, cudaMemcpyDeviceToHost, c->work);
    cudaError_t e = cudaStreamSynchronize(c->work);
    if (e != cudaSuccess) return set_error(c, LQCD_ERR_CUDA, cudaGetErrorString(e));
  }
  return LQCD_OK;
}

int lqcd_window_average(lqcd_ctx* c, const double* C, const double* dC, const int* valid, int n_gamma, int t_lo,
                        int t_hi, double* C_avg, double* dC_avg, int* n_pairs, int* n_valid, int where) {
  if (!c || !C || !dC || !valid || !C_avg || !dC_avg || !n_pairs || !n_valid || n_gamma < 1)
    return set_error(c, LQCD_ERR_INVALID_ARG, "window_average: bad arguments");
  const int T = c->g.Lt;
  if (t_lo < 0 || t_hi < t_lo || t_hi >= T)
    return set_error(c, LQCD_ERR_INVALID_ARG, "window_average: window outside [0, Lt)");
  Scope sc(c);
  const size_t cb = (size_t)n_gamma * T * T * sizeof(double2), ab = (size_t)n_gamma * T * sizeof(double2);
  const double2* dCo = (const double2*)stage_in(c, C, cb, where, "w_C");
  const double2* ddC = (const double2*)stage_in(c, dC, cb, where, "w_dC");
  const int* dv = (const int*)stage_in(c, valid, (size_t)T * T * sizeof(int), where, "w_valid");
  double2* dCa = (double2*)stage_out(c, C_avg, ab, where, "w_Ca");
  double2* ddCa = (double2*)stage_out(c, dC_avg, ab, where, "w_dCa");
  int* dnp = (int*)stage_out(c, n_pairs, (size_t)T * sizeof(int), where, "w_np");
  int* dnv = (int*)stage_out(c, n_valid, (size_t)T * sizeof(int), where, "w_nv");
  if (!dCo || !ddC || !dv || !dCa || !ddCa || !dnp || !dnv) return set_error(c, LQCD_ERR_OOM, "window_average: OOM");
  window_average(dCo, ddC, dv, n_gamma, T, t_lo, t_hi, dCa, ddCa, dnp, dnv, c->work);
  if (int e = cuda_check(c, "window_average")) return e;
  if (int e = finish_out(c, C_avg, dCa, ab, where)) return e;
  if (int e = finish_out(c, dC_avg, ddCa, ab, where)) return e;
  if (int e = finish_out(c, n_pairs, dnp, (size_t)T * sizeof(int), where)) return e;
  return finish_out(c, n_valid, dnv, (size_t)T * sizeof(int), where);
}

}  // extern "C"

static int internal_prec(int prec) {
  return prec == LQCD_PREC_F64 ? P64 : (prec == LQCD_PREC_F32 ? P32 : (prec == LQCD_PREC_F16 ? P16 : PDF));
}

extern "C" int lqcd_tune_dslash(lqcd_ctx* c, int prec, int nrhs, int* best_variant, double* best_ms) {
  if (!c || nrhs < 1 || !best_variant || !best_ms || prec < LQCD_PREC_F64 || prec > LQCD_PREC_DF)
    return set_error(c, LQCD_ERR_INVALID_ARG, "tune_dslash: bad arguments");
  if (!c->have_gauge) return set_error(c, LQCD_ERR_STATE, "tune_dslash: no gauge field uploaded");
  const int P = internal_prec(prec);
  const Geom& g = c->g;
  const size_t sb = spinor_bytes(g, P, nrhs);
  void* in = ws_get(c, "bench_in", sb);
  void* out = ws_get(c, "bench_out", sb);
  if (!in || !out) return set_error(c, LQCD_ERR_OOM, "tune_dslash: OOM");
  Scope sc(c);
  cudaMemsetAsync(in, 0, sb, c->work);
  const void* U = P == P64 || P == PDF ? c->U64 : (P == P32 ? c->U32 : c->U16);
  const void* Ainv = P == P64 ? c->Ainv64 : (P == P32 ? c->Ainv32 : c->Ainv16);
  DslashCall k{P, EPI_CH, 0, in, nullptr, nullptr, out, U, (const char*)Ainv + clover_bytes(g, P), 1, nrhs, 0.0, 1.0,
               c->d_tc_full};
  k.coord = coord_of(c, 1);
  // LQCD_PREC_DF: the true-residual kernel z - (A y - kappa H x) with x = y = z = the input
  auto launch = [&](int var) {
    if (P == PDF)
      launch_residual_df(g, in, in, in, out, c->Udf, (const char*)c->Adf + clover_bytes(g, P64), coord_of(c, 1),
                         c->d_tc_full, 1, nrhs, c->kappa, var, c->work);
    else
      launch_dslash(g, k, c->work, var);
  };
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e30;
  int bt = 0;
  const int nvar = P == P64 || P == PDF ? 3 : 8;  // the staged variants 3-7 are FP32 / FP16 only
  for (int var = 0; var < nvar; var++) {
    launch(var);
    cudaEventRecord(e0, c->work);
    for (int i = 0; i < 5; i++) launch(var);
    cudaEventRecord(e1, c->work);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms / 5 < best) {
      best = ms / 5;
      bt = var;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (int e = cuda_check(c, "tune_dslash")) return e;
  if (dslash_pipe_timeouts(true))
    return set_error(c, LQCD_ERR_TIMEOUT, "tune_dslash: a staged dslash copy did not complete within its wait limit");
  c->tuned_variant[(long)P * 100000 + nrhs] = bt;
  *best_variant = bt;
  *best_ms = best;
  return LQCD_OK;
}

extern "C" int lqcd_set_dslash_variant(lqcd_ctx* c, int prec, int nrhs, int variant) {
  if (!c || nrhs < 1 || variant < 0 || variant > 7 || prec < LQCD_PREC_F64 || prec > LQCD_PREC_DF)
    return set_error(c, LQCD_ERR_INVALID_ARG, "set_dslash_variant: bad arguments");
  const int P = internal_prec(prec);
  c->tuned_variant[(long)P * 100000 + nrhs] = variant;
  return LQCD_OK;
}

extern "C" int lqcd_nn_num_weights(void) { return nn_total_weights(); }

extern "C" int lqcd_nn_set_weights(lqcd_ctx* c, const float* w) {
  if (!c || !w) return set_error(c, LQCD_ERR_INVALID_ARG, "nn_set_weights: NULL");
  Scope sc(c);
  return nn_set_weights(c, w);
}

extern "C" int lqcd_nn_get_weights(lqcd_ctx* c, float* w) {
  if (!c || !w) return set_error(c, LQCD_ERR_INVALID_ARG, "nn_get_weights: NULL");
  Scope sc(c);
  return nn_get_weights(c, w);
}

extern "C" int lqcd_nn_apply(lqcd_ctx* c, const float* in, float* out, int nsamp, int domain, int where) {
  if (!c || !in || !out || nsamp < 1) return set_error(c, LQCD_ERR_INVALID_ARG, "nn_apply: bad arguments");
  if (!c->have_gauge) return set_error(c, LQCD_ERR_STATE, "nn_apply: no gauge field uploaded");
  Scope sc(c);
  const size_t bytes = (size_t)c->V * 12 * nsamp * sizeof(float2);
  const float2* di = (const float2*)stage_in(c, in, bytes, where, "nn_in");
  float2* dout = (float2*)stage_out(c, out, bytes, where, "nn_out");
  if (!di || !dout) return set_error(c, LQCD_ERR_OOM, "nn_apply: OOM");
  if (int rc = nn_apply_lex(c, di, dout, nsamp, domain, false)) return rc;
  if (int e = cuda_check(c, "nn_apply")) return e;
  return finish_out(c, out, dout, bytes, where);
}

extern "C" int lqcd_nn_apply_tc(lqcd_ctx* c, const float* in, float* out, int nsamp, int domain, int where) {
  if (!c || !in || !out || nsamp < 1) return set_error(c, LQCD_ERR_INVALID_ARG, "nn_apply_tc: bad arguments");
  if (!c->have_gauge) return set_error(c, LQCD_ERR_STATE, "nn_apply_tc: no gauge field uploaded");
  Scope sc(c);
  const size_t bytes = (size_t)c->V * 12 * nsamp * sizeof(float2);
  const float2* di = (const float2*)stage_in(c, in, bytes, where, "nn_in");
  float2* dout = (float2*)stage_out(c, out, bytes, where, "nn_out");
  if (!di || !dout) return set_error(c, LQCD_ERR_OOM, "nn_apply_tc: OOM");
  if (int rc = nn_apply_lex(c, di, dout, nsamp, domain, true)) return rc;
  if (int e = cuda_check(c, "nn_apply_tc")) return e;
  if (int e = finish_out(c, out, dout, bytes, where)) return e;
  cudaStreamSynchronize(c->work);
  if (nn_tc_timeouts(true)) return set_error(c, LQCD_ERR_TIMEOUT, "nn_apply_tc: a tensor-core wait ran out");
  return LQCD_OK;
}

extern "C" int lqcd_nn_loss_grad(lqcd_ctx* c, const float* in, const float* target, int nsamp, int domain,
                                 int even_only, int where, double* loss, float* grad) {
  if (!c || !in || !target || !loss || nsamp < 1)
    return set_error(c, LQCD_ERR_INVALID_ARG, "nn_loss_grad: bad arguments");
  if (!c->have_gauge) return set_error(c, LQCD_ERR_STATE, "nn_loss_grad: no gauge field uploaded");
  Scope sc(c);
  const size_t bytes = (size_t)c->V * 12 * nsamp * sizeof(float2);
  const float2* di = (const float2*)stage_in(c, in, bytes, where, "nn_in");
  const float2* dt = (const float2*)stage_in(c, target, bytes, where, "nn_tgt");
  if (!di || !dt) return set_error(c, LQCD_ERR_OOM, "nn_loss_grad: OOM");
  return nn_loss_grad_lex(c, di, dt, nsamp, domain, even_only, loss, grad, false);
}

extern "C" int lqcd_nn_loss_grad_bf16(lqcd_ctx* c, const float* in, const float* target, int nsamp, int domain,
                                      int even_only, int where, double* loss, float* grad) {
  if (!c || !in || !target || !loss || nsamp < 1)
    return set_error(c, LQCD_ERR_INVALID_ARG, "nn_loss_grad_bf16: bad arguments");
  if (!c->have_gauge) return set_error(c, LQCD_ERR_STATE, "nn_loss_grad_bf16: no gauge field uploaded");
  Scope sc(c);
  const size_t bytes = (size_t)c->V * 12 * nsamp * sizeof(float2);
  const float2* di = (const float2*)stage_in(c, in, bytes, where, "nn_in");
  const float2* dt = (const float2*)stage_in(c, target, bytes, where, "nn_tgt");
  if (!di || !dt) return set_error(c, LQCD_ERR_OOM, "nn_loss_grad_bf16: OOM");
  int rc = nn_loss_grad_lex(c, di, dt, nsamp, domain, even_only, loss, grad, true);
  if (rc == LQCD_OK && nn_tc_timeouts(true))
    return set_error(c, LQCD_ERR_TIMEOUT, "nn_loss_grad_bf16: a tensor-core wait ran out");
  return rc;
}

extern "C" int lqcd_nn_train(lqcd_ctx* c, int n_pairs, int epochs, int batch, double lr, int domain, unsigned seed,
                             double* loss_hist) {
  if (!c || n_pairs < 1 || epochs < 1 || batch < 1 || !(lr > 0))
    return set_error(c, LQCD_ERR_INVALID_ARG, "nn_train: bad arguments");
  if (!c->have_gauge) return set_error(c, LQCD_ERR_STATE, "nn_train: no gauge field uploaded");
  if (!c->nn_weights) return set_error(c, LQCD_ERR_STATE, "nn_train: set initial weights first");
  Scope sc(c);
  return nn_train(c, n_pairs, epochs, batch, lr, domain, seed, loss_hist);
}

extern "C" int lqcd_laplace_eigs(lqcd_ctx* c, int n_ev, double* V, double* lambda, int where, double tol,
                                 int* iters) {
  if (!c || !V || !lambda) return set_error(c, LQCD_ERR_INVALID_ARG, "laplace_eigs: NULL argument");
  const Geom& g = c->g;
  const long L3 = (long)g.Lx * g.Ly * g.Lz;
  if (n_ev < 1 || n_ev > 3 * L3) return set_error(c, LQCD_ERR_INVALID_ARG, "laplace_eigs: bad n_ev");
  if (!c->have_gauge) return set_error(c, LQCD_ERR_STATE, "laplace_eigs: no gauge field uploaded");
  Scope sc(c);
  size_t vb = (size_t)g.Lt * n_ev * L3 * 3 * sizeof(double2), lb = (size_t)g.Lt * n_ev * sizeof(double);
  double2* dV = (double2*)stage_out(c, V, vb, where, "e_V");
  double* dl = (double*)stage_out(c, lambda, lb, where, "e_lam");
  if (!dV || !dl) return set_error(c, LQCD_ERR_OOM, "laplace_eigs: OOM");
  int it = 0;
  int rc = laplace_eigs(c, n_ev, dV, dl, tol > 0 ? tol : 1e-10, 500, &it);
  if (iters) *iters = it;
  if (rc != LQCD_OK) return rc;
  if (int e = cuda_check(c, "laplace_eigs")) return e;
  if (int e = finish_out(c, V, dV, vb, where)) return e;
  return finish_out(c, lambda, dl, lb, where);
}

namespace {
__global__ void k_fill_pattern(float* p, long n, unsigned seed) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    unsigned h = (unsigned)i * 2654435761u ^ seed;
    h ^= h >> 13;
    h *= 0x5bd1e995u;
    h ^= h >> 15;
    p[i] = ((h & 0xffff) / 65536.0f - 0.5f) * 0.25f;
  }
}
__global__ void k_flush(float4* p, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = make_float4((float)i, 0.f, 0.f, 1.f);
}
}  // namespace

extern "C" int lqcd_dslash_bench(lqcd_ctx* c, int prec, int nrhs, int n_iter, int flush_l2, double* ms_per_launch,
                                 double* algo_bytes_per_launch) {
  if (!c || nrhs < 1 || n_iter < 1 || !ms_per_launch || !algo_bytes_per_launch || prec < LQCD_PREC_F64 ||
      prec > LQCD_PREC_DF)
    return set_error(c, LQCD_ERR_INVALID_ARG, "dslash_bench: bad arguments");
  if (!c->have_gauge) return set_error(c, LQCD_ERR_STATE, "dslash_bench: no gauge field uploaded");
  const int P = internal_prec(prec);
  const Geom& g = c->g;
  const size_t sb = spinor_bytes(g, P, nrhs);
  void* in = ws_get(c, "bench_in", sb);
  void* out = ws_get(c, "bench_out", sb);
  const size_t flush_n = (256u << 20) / sizeof(float4);
  float4* fl = flush_l2 ? (float4*)ws_get(c, "bench_flush", flush_n * sizeof(float4)) : nullptr;
  if (!in || !out || (flush_l2 && !fl)) return set_error(c, LQCD_ERR_OOM, "dslash_bench: OOM");
  Scope sc(c);
  // P16 fields hold half values; fill through a float view with values that are valid halves too
  if (P == P16) {
    cudaMemsetAsync(in, 0x3c, sb, c->work);  // every half = 1.0 + tiny mantissa pattern
  } else {
    long nf = (long)(sb / sizeof(float));
    k_fill_pattern<<<(nf + 255) / 256, 256, 0, c->work>>>((float*)in, nf, 12345u); lqcd::count_launch();
  }
  if (P == P64 || P == PDF) {
    // reinterpret the float pattern as doubles would give garbage exponents: write doubles instead
    std::vector<double> h(4096);
    for (size_t i = 0; i < h.size(); i++) h[i] = 0.01 * (double)((i * 7919) % 200) - 1.0;
    for (size_t o = 0; o < sb; o += h.size() * sizeof(double)) {
      size_t n = std::min(h.size() * sizeof(double), sb - o);
      cudaMemcpyAsync((char*)in + o, h.data(), n, cudaMemcpyHostToDevice, c->work);
    }
  }
  const void* U = P == P64 || P == PDF ? c->U64 : (P == P32 ? c->U32 : c->U16);
  const void* Ainv = P == P64 ? c->Ainv64 : (P == P32 ? c->Ainv32 : c->Ainv16);
  const void* Ao = (const char*)Ainv + clover_bytes(g, P);
  DslashCall k{P, EPI_CH, 0, in, nullptr, nullptr, out, U, Ao, 1, nrhs, 0.0, 1.0, c->d_tc_full};
  k.coord = coord_of(c, 1);
  // LQCD_PREC_DF: the true-residual kernel z - (A y - kappa H x), reading x (split once, as the
  // solver does), y, z, writing out
  void* xs = P == PDF ? ws_get(c, "bench_split", sb) : nullptr;
  if (P == PDF && !xs) return set_error(c, LQCD_ERR_OOM, "dslash_bench: OOM");
  if (P == PDF) split_neighbours(in, xs, (long)(sb / 16), nrhs, c->work);
  auto launch = [&](int var) {
    if (P == PDF)
      launch_residual_df(g, xs, in, in, out, c->Udf, (const char*)c->Adf + clover_bytes(g, P64), coord_of(c, 1),
                         c->d_tc_full, 1, nrhs, c->kappa, var, c->work);
    else
      launch_dslash(g, k, c->work, var);
  };
  int variant = 0;
  auto it = c->tuned_variant.find((long)P * 100000 + nrhs);
  if (it != c->tuned_variant.end()) variant = it->second;
  // warm-up
  launch(variant);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double total = 0;
  for (int i = 0; i < n_iter; i++) {
    if (fl) {
      k_flush<<<(flush_n + 255) / 256, 256, 0, c->work>>>(fl, (long)flush_n);
      lqcd::count_launch();
    }
    cudaEventRecord(e0, c->work);
    launch(variant);
    cudaEventRecord(e1, c->work);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    total += ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (int e = cuda_check(c, "dslash_bench")) return e;
  *ms_per_launch = total / n_iter;
  const double lb = P == P64 || P == PDF ? 144.0 : (P == P32 ? 48.0 : 24.0);
  const double cb = P == P64 || P == PDF ? 576.0 : (P == P32 ? 288.0 : 144.0);
  const double spb = P == P64 || P == PDF ? 192.0 : (P == P32 ? 96.0 : 48.0);
  *algo_bytes_per_launch = (double)g.Vh * (8 * lb + cb + (P == PDF ? 4.0 : 2.0) * nrhs * spb);
  return LQCD_OK;
}
