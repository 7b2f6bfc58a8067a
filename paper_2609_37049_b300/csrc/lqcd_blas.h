// Host launchers of the vector kernels (blas.cu).
#pragma once
#include "lqcd_internal.h"

namespace lqcd {
void v_norm2(int prec, const void* x, const VGeom& vg, const SegInfo* si, int nseg, double* partial, double* out,
             cudaStream_t st);
void v_convert(int pin, int pout, const void* in, void* out, const VGeom& vg, const SegInfo* si, int nseg,
               const double* scale, cudaStream_t st);
void v_axpy_mixed(int pe, void* x, const void* e, const VGeom& vg, const SegInfo* si, int nseg, const double* scale,
                  const int* active, cudaStream_t st);
void v_zero(int prec, void* x, const VGeom& vg, cudaStream_t st);
void v_copy(int prec, const void* a, void* b, const VGeom& vg, cudaStream_t st);
void bicg_init(int prec, const void* b, void* r, void* p, void* x, const VGeom& vg, const SegInfo* si, int nseg,
               double* partial, const KState& ks, const double* delta, const int* outer_active, cudaStream_t st);
void bicg_s(int prec, const void* r, const void* v, void* s, const VGeom& vg, const SegInfo* si, int nseg,
            const KState& ks, cudaStream_t st);
// The BiCGStab finishing steps sum the fused-reduction partials in two levels through p2
// ([nseg][nchunk][nrhs][ND] doubles, nchunk = seg_chunks of the batch, ND <= 8).
int seg_chunks(const VGeom& vg, const SegInfo& si_host);
// after t = M s with the RED_TS_R0 reduction in `partial`: all scalars, then x, r, p in one pass
void bicg_tail(int prec, void* x, void* p, const void* s, const void* t, void* r, const void* v,
               const double* partial, double* p2, int nchunk, const VGeom& vg, const SegInfo* si, int nseg,
               const KState& ks, cudaStream_t st);
// alpha = rho / (r0, v) after v = M p with the RED_DOT_Z reduction in `partial`
void bicg_fin_alpha_only(const double* partial, double* p2, int nchunk, const VGeom& vg, const SegInfo* si,
                         int nseg, const KState& ks, cudaStream_t st);
void count_active(const int* active, int n, int* count, cudaStream_t st);

// ---- flexible GCR and MR preconditioner (gcr.cu)
#define LQCD_GCR_MAXK 16
struct VecList {
  void* v[LQCD_GCR_MAXK];
};
// Per-system GCR scalars (device arrays; beta and w2 have LQCD_GCR_MAXK rows of nsys).
struct GState {
  double2* beta;
  double2* alpha;
  double* w2;
  double* r2;
  double* b2;
  double* stop2;
  double* pscale;   // 1 / |r| (scale of the residual handed to the preconditioner)
  double* ipscale;  // |r|
  int* active;
  int* iters;
  int* count;
  int nsys;
};
void gcr_init(int prec, const void* b, void* x, void* r, const VGeom& vg, const SegInfo* si, int nseg,
              double* partial, const GState& gs, const double* delta, const int* outer_active, cudaStream_t st);
void gcr_orthogonalise(int prec, const VecList& W, const VecList& Z, int k, const void* r, const VGeom& vg,
                       const SegInfo* si, int nseg, double* partial, const GState& gs, cudaStream_t st);
void gcr_update(int prec, void* x, void* r, const void* z, const void* w, const VGeom& vg, const SegInfo* si,
                int nseg, double* partial, const GState& gs, cudaStream_t st);
void mr_finish(const double* partial, const VGeom& vg, const SegInfo* si, int nseg, double2* omega,
               const int* active, cudaStream_t st);
void mr_update(int prec, void* e, void* r, const void* p, const VGeom& vg, const SegInfo* si, int nseg,
               const double2* omega, const int* active, cudaStream_t st);

// One batch's inner (even-odd Schur) Krylov problem: operator data and work vectors.
struct Inner {
  int prec, nrhs, nseg;
  VGeom vg;
  const SegInfo* si;
  const signed char* tc;
  const void* U;
  const void* Ainv_e;
  const void* Ainv_o;
  const void* b;  // prepared right-hand side; also the BiCGStab shadow residual r0
  void *x, *r, *p, *v, *s, *t, *tmp;
  KState ks;
  double* partial;
  double* partial2;  // chunk sums of the two-level reductions
  int nchunk;
  double kappa;
  int variant;  // dslash launch variant (register cap)
};

// ---- gauge-covariant network preconditioner (nn.cu)
int nn_total_weights();
int nn_reserve(lqcd_ctx* c, int nrhs);
void nn_precondition(lqcd_ctx* c, const Inner& in, const void* r, void* z, const double* pscale,
                     const double* ipscale, cudaStream_t st);
int nn_set_weights(lqcd_ctx* c, const float* w_host);
int nn_get_weights(lqcd_ctx* c, float* w_host);
// tc: the inference path (BF16 weights and activations, channel mixing on the tensor cores)
int nn_apply_lex(lqcd_ctx* c, const float2* in_dev, float2* out_dev, int N, int domain, bool tc);
// tensor-core layer waits that ran out of their iteration limit since the last reset
int nn_tc_timeouts(bool reset);
int nn_loss_grad_lex(lqcd_ctx* c, const float2* in_dev, const float2* tgt_dev, int N, int domain, int even_only,
                     double* loss, float* grad_host, bool bf16);
int nn_train(lqcd_ctx* c, int n_pairs, int epochs, int batch, double lr, int domain, unsigned seed,
             double* loss_hist);
void outer_update(const double* r2, const double* b2, int nsys, double tol, double inner_tol, int* active,
                  double* delta, double* scale, double* rel, int first, cudaStream_t st);
void recip(const double* a, double* b, int n, cudaStream_t st);
// Device-side loop condition of a CUDA-graph WHILE node (see k_loop_cond in blas.cu).
void loop_cond(const int* active, int n, int* ctr, int mode, int chunk, int max_outer, int max_iter,
               cudaGraphConditionalHandle h, cudaStream_t st);
}  // namespace lqcd
