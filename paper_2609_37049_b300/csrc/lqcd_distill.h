// Host launchers of the layout and distillation kernels (distill.cu) and the solver driver.
#pragma once
#include <memory>

#include "lqcd_internal.h"

namespace lqcd {
void pack_spinor(const Geom& g, const double2* lex, double2* eo, int nrhs, cudaStream_t st);
void unpack_spinor(const Geom& g, const double2* eo, double2* lex, int nrhs, cudaStream_t st);
// Vt: [slots][n_ev][L3][3], the colour vectors of timeslice t in slot vslot[t] (device [LQCD_MAXT])
void make_sources(const Geom& g, const double2* Vt, int n_ev, const int* jr, const int* br,
                  const unsigned char* srcmask, const int* vslot, double2* b, int nrhs, cudaStream_t st);
// Cpart: scratch of project_ksplit(...) * nsinks * n_ev * 4 * nrhs complex entries.
// blocks_per_sm: about this many 256-thread blocks per SM (split along K to reach it); a batch
// in flight beside the projection wants few (the FP64 pipe needs few warps), a lone one four.
int project_ksplit(const Geom& g, int n_ev, int nrhs, int nsinks, int blocks_per_sm);
// With Vf (the colour vectors split by split_colour_vectors) and Xf (scratch of nsinks * 4 * nrhs
// * 3 L^3 float4) the GEMM runs in double-float arithmetic on the FP32 pipe; with Vf = nullptr in
// FP64.
void project(const Geom& g, const double2* Vt, int n_ev, const double2* X, const int* sinks, const int* vslot,
             int nsinks, double2* C, double2* Cpart, int nrhs, int blocks_per_sm, bool high_priority,
             const float4* Vf, float4* Xf, cudaStream_t st);
// Vf[i] = (re_hi, re_lo, im_hi, im_lo) of V[i], i < n
void split_colour_vectors(const double2* V, float4* Vf, long n, cudaStream_t st);
void loops(const double2* tau, int n_ev, int n_t, const double2* G, int n_gamma, const double* w, double2* L,
           double2* Lt, cudaStream_t st);
// C [n_gamma][T][n_t], C_avg [n_gamma][T] (may be null): connected correlator from all-sink
// perambulators tau [n_t][T][n_ev][4][n_ev][4]; G as for loops.
void conn_correlator(const double2* tau, int n_ev, int T, const int* t_src_dev, int n_t, const double2* G,
                     int n_gamma, double2* C, double2* C_avg, cudaStream_t st);
void nr_estimator(const double2* conn, const double2* disc, const double2* dC, int n_gamma, int T,
                  const int* delta_of_dt_dev, double2* out, cudaStream_t st);
void correlators(const double2* L, const double2* Lt, const double2* Ld, const double2* Ltd, int n_cfg, int n_g,
                 int T, int vev, const int* dom, double2* C, double2* Cdd, double2* dC, double2* C_avg,
                 double2* dC_avg, int* valid, int* n_valid, double2* terms, double2* dL, double2* dLt,
                 cudaStream_t st);
// Bulk-window averages of C, dC [n_g][T][T] (x0, y0) over t_lo <= y0, y0 + dt <= t_hi; outputs
// C_avg, dC_avg [n_g][T], n_pairs, n_valid [T].
void window_average(const double2* C, const double2* dC, const int* valid, int n_g, int T, int t_lo, int t_hi,
                    double2* C_avg, double2* dC_avg, int* n_pairs, int* n_valid, cudaStream_t st);
void build_gauge(lqcd_ctx* c, const double2* links_dev, int* bad_dev);

// Per-batch solver statistics (host side).
struct BatchStats {
  std::vector<double> rel;  // [nsys] final true relative residual
  std::vector<int> iters;   // [nsys] inner iterations summed over cycles
  int cycles = 0;
  long long dslash = 0;
  int fallback = 0;
  int device_loops = 0;  // 1 if the batch ran as one graph with device-side loops
};

// Solve D x = b (domain = 0) or D_Lambda x = b (domain = 1) for nrhs right-hand sides held in
// the full even-odd FP64 layout on the device.  Returns LQCD_OK, LQCD_ERR_NOT_CONVERGED or
// LQCD_ERR_NAN (a non-finite residual), with bs filled in every case.
int solve_batch(lqcd_ctx* c, const double2* b, double2* x, int nrhs, int domain, const lqcd_solve_params& p,
                BatchStats& bs);
// The same in two steps, so two batches can be in flight: enqueue on the stream of work-vector
// slot `slot` (0: the context's work stream, 1: its second stream) -- one graph launch with
// device-side loops where the driver supports it, else the host-driven loop, which returns when
// the batch is done -- and finish (wait for the batch, decode its residuals and iterations).
struct BatchHandle {
  std::shared_ptr<void> batch;
};
int solve_batch_enqueue(lqcd_ctx* c, int slot, const double2* b, double2* x, int nrhs, int domain,
                        const lqcd_solve_params& p, BatchHandle& h);
int solve_batch_finish(lqcd_ctx* c, BatchHandle& h, BatchStats& bs);
// The stream of work-vector slot `slot` (created on first use).
cudaStream_t slot_stream(lqcd_ctx* c, int slot);
// Lowest n_ev eigenpairs of the covariant 3D Laplacian on every timeslice (laplace.cu);
// Vout [Lt][n_ev][L3][3] and lam_out [Lt][n_ev] are device pointers.
int laplace_eigs(lqcd_ctx* c, int n_ev, double2* Vout, double* lam_out_dev, double tol, int max_iter,
                 int* iters_out);
// out = D in (or D_Lambda in), full even-odd FP64 layout.
void apply_D(lqcd_ctx* c, const double2* in, double2* out, int nrhs, int domain, cudaStream_t st);
}  // namespace lqcd
