// Host-side internals of the lqcd library: the context, workspace, kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <functional>
#include <map>
#include <string>
#include <vector>

#include "lqcd.h"
#include "lqcd_common.cuh"

namespace lqcd {

// ------------------------------------------------------------------ reductions / segments
// Vector kernels run one thread per (site, rhs), rhs fastest, with S sites per block; S is a
// power of two dividing the half-timeslice volume so every block lies inside one timeslice of
// one parity.  Segments are ranges of timeslices (one per domain, or one for the full lattice);
// a Krylov "system" is one (rhs, segment) pair, index sys = rhs * nseg + seg.
// Time segments (domains) of a solve: segment k covers timeslices [t0, t1) and, for a domain
// that wraps around the time boundary (tilings that start at t_start > 0), also [t0b, t1b)
// (empty when t0b == t1b).
struct SegInfo {
  int nseg;
  unsigned char seg_of_t[LQCD_MAXT];
  unsigned short t0[LQCD_MAXT];
  unsigned short t1[LQCD_MAXT];
  unsigned short t0b[LQCD_MAXT];
  unsigned short t1b[LQCD_MAXT];
};

struct VGeom {
  Geom g;
  int nrhs;
  int S;         // sites per block
  int npar;      // 1 (half lattice) or 2 (full lattice, even block then odd block)
  long blocks;   // npar * Vh / S
  long bpt;      // blocks per timeslice per parity = Vth / S
  long bpp;      // blocks per parity = Vh / S
  int threads() const { return S * nrhs; }
};

VGeom make_vgeom(const Geom& g, int nrhs, int npar);

// Per-system Krylov scalars (device arrays of length nsys).
struct KState {
  double2* rho;
  double2* alpha;
  double2* omega;
  double2* beta;
  double* r2;
  double* b2;
  double* stop2;
  int* active;
  int* iters;
  int* flag;    // 1: breakdown
  int* count;   // [1] number of active systems
};

// ------------------------------------------------------------------ dslash
enum Epi {
  EPI_H = 0,     // out = b * H x
  EPI_CH = 1,    // out = b * C (H x)
  EPI_Y_H = 2,   // out = a y + b H x
  EPI_Y_CH = 3,  // out = a y + b C (H x)
  EPI_C_YH = 4,  // out = C (a y + b H x)
  EPI_CY_H = 5,  // out = a C y + b H x
  EPI_RES = 6    // out = z - (C y + b H x)
};

// Dot products fused into the epilogue (second half of the Schur operator, EPI_Y_CH only):
//   RED_DOT_Z:      partial (zred, out)             -> 2 doubles per (block, rhs)
//   RED_DOT_Y_NORM: partial (out, y), (out, out)    -> 3 doubles per (block, rhs)
//   RED_TS_R0:      partial (out, y), (out, out), (zred, out), (zred, y), (y, y)
//                                                   -> 8 doubles per (block, rhs)
// with blocks of red_sites sites x nrhs (the VGeom blocks of the same batch).
enum Red { RED_NONE = 0, RED_DOT_Z = 1, RED_DOT_Y_NORM = 2, RED_TS_R0 = 3 };

struct DslashCall {
  int prec;
  int epi;
  int dagger;
  const void* in;   // parity 1 - out_par
  const void* y;    // parity out_par
  const void* z;    // parity out_par
  void* out;        // parity out_par
  const void* U;
  const void* C;    // packed clover of parity out_par (A or A^-1)
  int out_par;
  int nrhs;
  double a, b;
  const signed char* tc;            // device array [Lt]: forward t-hop coefficient per timeslice
  const unsigned* coord = nullptr;  // packed site coordinates of parity out_par (device)
  double* partial = nullptr;
  const void* zred = nullptr;
  int red = RED_NONE;
  int red_sites = 0;
};

// dslash_df.cu: split an FP64 field of n_complex entries to double-float (float4 per entry), and
// the true residual out = z - (A y - kappa H xn) of parity out_par in double-float arithmetic
// (xn: the neighbour parity, split by split_neighbours; y, z, out: FP64; U_split, A_split: split
// links and the parity's clover; variant 0 / 1 / 2: register caps 255 / 168 / 128).
void split_field(const void* in, void* out, long n_complex, cudaStream_t st);
// the neighbour parity of the residual in the layout launch_residual_df reads for nrhs (pairs of
// right-hand sides interleaved when nrhs is even)
void split_neighbours(const void* in, void* out, long n_complex, int nrhs, cudaStream_t st);
void launch_residual_df(const Geom& g, const void* xn_split, const void* y, const void* z, void* out,
                        const void* U_split, const void* A_split, const unsigned* coord, const signed char* tc,
                        int out_par, int nrhs, double kappa, int variant, cudaStream_t st);

// variant: register cap of the FP32 / FP16 kernels (0: 128, 1: 80, 2: 64 registers per thread)
void launch_dslash(const Geom& g, const DslashCall& c, cudaStream_t st, int variant = 0);
// y_e = M x_e (even-odd Schur operator) on FP64 even-parity blocks, in storage precision P
int schur_apply(lqcd_ctx* c, int P, const void* x64, void* y64, int nrhs, int domain, cudaStream_t st);
// waits of the staged dslash kernel that ran out of their iteration limit since the last reset
unsigned long long dslash_pipe_timeouts(bool reset);
void launch_clover_only(const Geom& g, int prec, const void* C, const void* in, void* out, int nrhs,
                        cudaStream_t st);

}  // namespace lqcd

// ------------------------------------------------------------------ context
struct lqcd_ctx {
  lqcd::Geom g;
  long V;
  int bc;
  double kappa = 0, csw = 0;
  bool have_gauge = false;
  cudaStream_t user_stream = 0;
  cudaStream_t work = 0;
  cudaEvent_t ev_user = 0, ev_work = 0;
  // links: P64 full matrices, P32 / P16 two rows
  void* U64 = nullptr;
  void* U32 = nullptr;
  void* U16 = nullptr;
  // APE-smeared spatial links (FP64, layout of U64 for mu < 3), used by the Laplacian eigensolver
  void* Usm = nullptr;
  bool have_smeared = false;
  // clover A and A^-1 per parity: [par][chir][chunks][Vh]
  void* A64 = nullptr;
  void* Ainv64 = nullptr;
  void* Ainv32 = nullptr;
  void* Ainv16 = nullptr;
  void* A32 = nullptr;
  // U64 and A64 split to double-float (float4 = (re.hi, re.lo, im.hi, im.lo) per complex entry,
  // same indexing), read by the true-residual kernel
  void* Udf = nullptr;
  void* Adf = nullptr;
  // domain tiling of the time axis
  std::vector<int> extents;
  int t_start = 0;  // first timeslice of domain 0 (the tiling wraps around the time boundary)
  signed char tc_full[LQCD_MAXT];
  signed char tc_dom[LQCD_MAXT];
  signed char* d_tc_full = nullptr;  // device copies [Lt]
  signed char* d_tc_dom = nullptr;
  lqcd::SegInfo seg_full, seg_dom;
  lqcd::SegInfo* d_seg_full = nullptr;  // device copies
  lqcd::SegInfo* d_seg_dom = nullptr;
  // workspace: device buffers by name, grown on demand; gen is the API call that last used the
  // buffer (ws_gen counts calls), so that a call short of memory can free buffers only earlier
  // calls used.
  struct WsBuf {
    void* p;
    size_t bytes;
    unsigned long gen;
  };
  std::map<std::string, WsBuf> ws;
  unsigned long ws_gen = 0;
  void* pinned = nullptr;
  size_t pinned_bytes = 0;
  std::string err;
  int device = 0;
  // autotuned threads per block for the dslash, keyed by prec * 100000 + nrhs
  std::map<long, int> tuned_variant;
  // instantiated CUDA graphs of Krylov iteration chunks, keyed by buffers and shape
  std::map<std::string, cudaGraphExec_t> graphs;
  std::map<cudaGraphExec_t, long long> graph_kernels;  // kernel nodes per instantiated graph
  // whole solves captured with device-side loops (conditional WHILE nodes), keyed like `graphs`:
  // the executable and its kernel nodes outside the loops, per cycle and per inner chunk
  struct LoopGraph {
    cudaGraphExec_t exec;
    long long nk_init, nk_cycle, nk_chunk;
  };
  std::map<std::string, LoopGraph> loop_graphs;
  bool loop_graphs_unavailable = false;  // set when the driver refused a conditional graph
  // a second right-hand-side batch in flight (pipelined perambulators): slot 1's stream (slot 0
  // is `work`), an event to order it, and per-slot pinned buffers for the batch read-back
  cudaStream_t slot_stream = 0;
  cudaStream_t cap_stream = 0;  // capture of the loop bodies
  cudaEvent_t ev_slot = 0;
  void* slot_pinned[2] = {nullptr, nullptr};
  size_t slot_pinned_bytes[2] = {0, 0};
  // Clifford table on the device: [16][2][4][4] complex (Gamma, Gamma-tilde)
  double2* d_gamma = nullptr;
  // packed site coordinates x | y << 8 | z << 16 | t << 24 per parity: [2][Vh]
  unsigned* d_coord = nullptr;
  // network preconditioner: FP32 master weights, BF16 inference copy, Adam moments, work fields
  void* nn_weights = nullptr;
  void* nn_w16 = nullptr;
  void* nn_m = nullptr;
  void* nn_v = nullptr;
  int nn_step = 0;
  void* nn_buf[3] = {nullptr, nullptr, nullptr};
  // optional per-phase GPU timing (LQCD_PHASE_TIMING=1): event pairs not yet read, totals in ms
  bool timing = false;
  std::vector<std::pair<std::string, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::map<std::string, double> phase_ms;
};

namespace lqcd {
bool is_capturing();
// Records CUDA events around a phase on the work stream when timing is on (not while capturing).
struct PhaseTimer {
  lqcd_ctx* c;
  const char* name;
  cudaEvent_t e0 = nullptr;
  PhaseTimer(lqcd_ctx* ctx, const char* n) : c(ctx), name(n) {
    if (c->timing && !is_capturing() && cudaEventCreate(&e0) == cudaSuccess) cudaEventRecord(e0, c->work);
  }
  ~PhaseTimer() {
    if (!e0) return;
    cudaEvent_t e1;
    if (cudaEventCreate(&e1) != cudaSuccess) return;
    cudaEventRecord(e1, c->work);
    c->pending.push_back({name, {e0, e1}});
  }
};
// Synchronise the work stream and add the pending phase durations to the totals.
void flush_phase_times(lqcd_ctx* c);
}  // namespace lqcd

inline const unsigned* coord_of(const lqcd_ctx* c, int parity) { return c->d_coord + parity * c->g.Vh; }

namespace lqcd {
// Process-wide count of kernels this library has put on a GPU queue: every launch site calls
// count_launch(); launches recorded while a stream is being captured are not counted, a graph
// replay adds the number of kernel nodes of the graph instead.
void count_launch(long long n = 1);
void set_capturing(bool on);
void* ws_get(lqcd_ctx* c, const std::string& name, size_t bytes);
// Destroy every captured solver graph (buffers or operator scalars they hold changed).
void drop_graphs(lqcd_ctx* c);
void* pinned_get(lqcd_ctx* c, size_t bytes);
int set_error(lqcd_ctx* c, int code, const std::string& msg);
// smear.cu: spatial APE smearing of the uploaded links into c->Usm; unpack to [V][3][3][3]
int ape_smear(lqcd_ctx* c, double alpha, int n_iter);
void unpack_smeared(lqcd_ctx* c, double2* out);
size_t clover_bytes(const Geom& g, int prec);   // one parity
size_t link_bytes(const Geom& g, int prec);     // all mu, both parities
size_t spinor_bytes(const Geom& g, int prec, int nrhs);  // one parity
inline const char* par_ptr(const void* base, size_t bytes_per_par, int p) {
  return reinterpret_cast<const char*>(base) + bytes_per_par * p;
}
}  // namespace lqcd
