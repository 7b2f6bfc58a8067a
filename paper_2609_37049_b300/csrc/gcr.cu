// Vector kernels of the flexible GCR solver and of the minimal-residual (MR) preconditioner.
//
// Flexible GCR(m), right-preconditioned by a variable operator K (Saad, "A flexible inner-outer
// preconditioned GMRES algorithm", SIAM J. Sci. Comput. 14 (1993); GCR form of Eisenstat, Elman
// and Schultz 1983), per system, all systems of a batch in lockstep:
//   z_k = K r;  w_k = M z_k;
//   beta_j = (w_j, w_k) / (w_j, w_j)  (j < k);  w_k -= sum_j beta_j w_j;  z_k -= sum_j beta_j z_j
//   alpha = (w_k, r) / (w_k, w_k);  x += alpha z_k;  r -= alpha w_k
// MR preconditioner sweeps (e = 0, r = input): p = M r; a = (p, r) / (p, p); e += a r; r -= a p.
// Reductions follow the same two-pass per-block / per-segment scheme as blas.cu; scalars stay on
// the device.
#include "lqcd_blas.h"

namespace lqcd {

struct VThreadG {
  int rhs, seg, site_local;
  long idx, stride;
};

LQCD_D VThreadG vthread_g(const VGeom& vg, const SegInfo* si) {
  VThreadG v;
  v.site_local = threadIdx.x / vg.nrhs;
  v.rhs = threadIdx.x - v.site_local * vg.nrhs;
  long cb = (long)blockIdx.x * vg.S + v.site_local;  // one parity (half-lattice fields)
  int t = (int)(cb / vg.g.Vth);
  v.seg = si ? si->seg_of_t[t] : 0;
  v.idx = cb * vg.nrhs + v.rhs;
  v.stride = vg.g.Vh * vg.nrhs;
  return v;
}

// Sum a runtime number of doubles per (block, rhs) one after the other through shared memory.
LQCD_D void block_reduce_many(const double* vals, int nd, double* partial, const VGeom& vg, int site_local,
                              int rhs) {
  extern __shared__ double smg[];
  const int n = blockDim.x;
  for (int k = 0; k < nd; k++) {
    smg[threadIdx.x] = vals[k];
    __syncthreads();
    for (int s = vg.S / 2; s >= 1; s >>= 1) {
      if (site_local < s) smg[threadIdx.x] += smg[threadIdx.x + s * vg.nrhs];
      __syncthreads();
    }
    if (site_local == 0) partial[((long)blockIdx.x * vg.nrhs + rhs) * nd + k] = smg[threadIdx.x];
    __syncthreads();
  }
  (void)n;
}

template <int ND>
LQCD_D void seg_sum_g(const double* partial, const VGeom& vg, const SegInfo* si, int nd_stride, int k0,
                      double (&out)[ND]) {
  __shared__ double sm[ND][128];
  const int rhs = blockIdx.x, seg = blockIdx.y;
  double acc[ND];
#pragma unroll
  for (int k = 0; k < ND; k++) acc[k] = 0.0;
  for (int rg = 0; rg < 2; rg++) {  // the segment's timeslice range(s)
    const long t0 = si ? (rg ? si->t0b[seg] : si->t0[seg]) : 0;
    const long t1 = si ? (rg ? si->t1b[seg] : si->t1[seg]) : (rg ? 0 : vg.g.Lt);
    const long b0 = t0 * vg.bpt, nb = (t1 - t0) * vg.bpt;
    for (long b = threadIdx.x; b < nb; b += blockDim.x) {
#pragma unroll
      for (int k = 0; k < ND; k++) acc[k] += partial[((b0 + b) * vg.nrhs + rhs) * nd_stride + k0 + k];
    }
  }
#pragma unroll
  for (int k = 0; k < ND; k++) sm[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s >= 1; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int k = 0; k < ND; k++) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < ND; k++) out[k] = sm[k][0];
  }
}

LQCD_D double2 cdivd(double2 a, double2 b) {
  double den = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

// ------------------------------------------------------------------ FGCR
// partial (w_j, w_k) for j < k
template <int P>
__global__ void k_gcr_dots(VecList W, int k, VGeom vg, const SegInfo* si, double* partial) {
  using R = typename Traits<P>::real;
  VThreadG v = vthread_g(vg, si);
  cplx<R> wk[12];
  load_spinor<P>(W.v[k], v.stride, v.idx, wk);
  double vals[2 * LQCD_GCR_MAXK];
  for (int j = 0; j < k; j++) {
    cplx<R> wj[12];
    load_spinor<P>(W.v[j], v.stride, v.idx, wj);
    cplx<R> d = {R(0), R(0)};
#pragma unroll
    for (int q = 0; q < 12; q++) d = d + cjmul(wj[q], wk[q]);
    vals[2 * j] = d.re;
    vals[2 * j + 1] = d.im;
  }
  block_reduce_many(vals, 2 * k, partial, vg, v.site_local, v.rhs);
}

// beta_j = (w_j, w_k) / w2_j for the active systems (0 otherwise); beta: [j][nsys]
__global__ void k_gcr_fin_beta(const double* partial, VGeom vg, const SegInfo* si, int nseg, int k, GState gs) {
  const int sys = blockIdx.x * nseg + blockIdx.y;
  for (int j = 0; j < k; j++) {
    double s[2];
    seg_sum_g<2>(partial, vg, si, 2 * k, 2 * j, s);
    if (threadIdx.x == 0) {
      double w2 = gs.w2[j * gs.nsys + sys];
      bool ok = gs.active[sys] && w2 > 0.0;
      gs.beta[j * gs.nsys + sys] = ok ? make_double2(s[0] / w2, s[1] / w2) : make_double2(0.0, 0.0);
    }
    __syncthreads();
  }
}

// w_k -= sum_j beta_j w_j; z_k -= sum_j beta_j z_j; partial |w_k|^2, (w_k, r)
template <int P>
__global__ void k_gcr_orth(VecList W, VecList Z, int k, const void* r, VGeom vg, const SegInfo* si, int nseg,
                           GState gs, double* partial) {
  using R = typename Traits<P>::real;
  VThreadG v = vthread_g(vg, si);
  const int sys = v.rhs * nseg + v.seg;
  cplx<R> wk[12], zk[12];
  load_spinor<P>(W.v[k], v.stride, v.idx, wk);
  load_spinor<P>(Z.v[k], v.stride, v.idx, zk);
  for (int j = 0; j < k; j++) {
    double2 be = gs.beta[j * gs.nsys + sys];
    cplx<R> b = {(R)be.x, (R)be.y};
    cplx<R> a[12];
    load_spinor<P>(W.v[j], v.stride, v.idx, a);
#pragma unroll
    for (int q = 0; q < 12; q++) wk[q] = wk[q] - b * a[q];
    load_spinor<P>(Z.v[j], v.stride, v.idx, a);
#pragma unroll
    for (int q = 0; q < 12; q++) zk[q] = zk[q] - b * a[q];
  }
  if (k > 0) {
    store_spinor<P>(W.v[k], v.stride, v.idx, wk);
    store_spinor<P>(Z.v[k], v.stride, v.idx, zk);
  }
  cplx<R> rv[12];
  load_spinor<P>(r, v.stride, v.idx, rv);
  cplx<R> d = {R(0), R(0)};
  R nn = 0;
#pragma unroll
  for (int q = 0; q < 12; q++) {
    d = d + cjmul(wk[q], rv[q]);
    nn += norm2(wk[q]);
  }
  double vals[3] = {(double)nn, (double)d.re, (double)d.im};
  block_reduce_many(vals, 3, partial, vg, v.site_local, v.rhs);
}

__global__ void k_gcr_fin_alpha(const double* partial, VGeom vg, const SegInfo* si, int nseg, int k, GState gs) {
  double s[3];
  seg_sum_g<3>(partial, vg, si, 3, 0, s);
  if (threadIdx.x) return;
  const int sys = blockIdx.x * nseg + blockIdx.y;
  gs.w2[k * gs.nsys + sys] = s[0];
  bool ok = gs.active[sys] && s[0] > 0.0 && isfinite(s[0]);
  gs.alpha[sys] = ok ? make_double2(s[1] / s[0], s[2] / s[0]) : make_double2(0.0, 0.0);
}

// x += alpha z_k; r -= alpha w_k; partial |r|^2
template <int P>
__global__ void k_gcr_xr(void* x, void* r, const void* z, const void* w, VGeom vg, const SegInfo* si, int nseg,
                         GState gs, double* partial) {
  using R = typename Traits<P>::real;
  VThreadG v = vthread_g(vg, si);
  double2 al = gs.alpha[v.rhs * nseg + v.seg];
  cplx<R> a = {(R)al.x, (R)al.y};
  cplx<R> xv[12], rv[12], zv[12], wv[12];
  load_spinor<P>(x, v.stride, v.idx, xv);
  load_spinor<P>(r, v.stride, v.idx, rv);
  load_spinor<P>(z, v.stride, v.idx, zv);
  load_spinor<P>(w, v.stride, v.idx, wv);
  R nn = 0;
#pragma unroll
  for (int q = 0; q < 12; q++) {
    xv[q] = xv[q] + a * zv[q];
    rv[q] = rv[q] - a * wv[q];
    nn += norm2(rv[q]);
  }
  store_spinor<P>(x, v.stride, v.idx, xv);
  store_spinor<P>(r, v.stride, v.idx, rv);
  double vals[1] = {(double)nn};
  block_reduce_many(vals, 1, partial, vg, v.site_local, v.rhs);
}

__global__ void k_gcr_fin_r2(const double* partial, VGeom vg, const SegInfo* si, int nseg, GState gs) {
  double s[1];
  seg_sum_g<1>(partial, vg, si, 1, 0, s);
  if (threadIdx.x) return;
  const int sys = blockIdx.x * nseg + blockIdx.y;
  if (!gs.active[sys]) return;
  gs.r2[sys] = s[0];
  gs.iters[sys] += 1;
  gs.pscale[sys] = s[0] > 0.0 ? 1.0 / sqrt(s[0]) : 1.0;
  gs.ipscale[sys] = s[0] > 0.0 ? sqrt(s[0]) : 1.0;
  if (!(s[0] > gs.stop2[sys]) || !isfinite(s[0])) gs.active[sys] = 0;
}

// init: x = 0, r = b; partial |b|^2
template <int P>
__global__ void k_gcr_init(const void* b, void* x, void* r, VGeom vg, const SegInfo* si, double* partial) {
  using R = typename Traits<P>::real;
  VThreadG v = vthread_g(vg, si);
  cplx<R> bv[12], z[12];
  load_spinor<P>(b, v.stride, v.idx, bv);
  R nn = 0;
#pragma unroll
  for (int q = 0; q < 12; q++) {
    nn += norm2(bv[q]);
    z[q] = {R(0), R(0)};
  }
  store_spinor<P>(r, v.stride, v.idx, bv);
  store_spinor<P>(x, v.stride, v.idx, z);
  double vals[1] = {(double)nn};
  block_reduce_many(vals, 1, partial, vg, v.site_local, v.rhs);
}

__global__ void k_gcr_fin_init(const double* partial, VGeom vg, const SegInfo* si, int nseg, GState gs,
                               const double* delta, const int* outer_active) {
  double s[1];
  seg_sum_g<1>(partial, vg, si, 1, 0, s);
  if (threadIdx.x) return;
  const int sys = blockIdx.x * nseg + blockIdx.y;
  gs.r2[sys] = s[0];
  gs.b2[sys] = s[0];
  double d = delta ? delta[sys] : 1e-6;
  gs.stop2[sys] = d * d * s[0];
  gs.active[sys] = (s[0] > 0.0) && (!outer_active || outer_active[sys]);
  gs.pscale[sys] = s[0] > 0.0 ? 1.0 / sqrt(s[0]) : 1.0;
  gs.ipscale[sys] = s[0] > 0.0 ? sqrt(s[0]) : 1.0;
  gs.alpha[sys] = make_double2(0.0, 0.0);
}

// ------------------------------------------------------------------ MR sweeps (preconditioner)
// e = 0, r = input (already in place)
template <int P>
__global__ void k_mr_update(void* e, void* r, const void* p, VGeom vg, const SegInfo* si, int nseg,
                            const double2* omega, const int* active) {
  using R = typename Traits<P>::real;
  VThreadG v = vthread_g(vg, si);
  const int sys = v.rhs * nseg + v.seg;
  if (!active[sys]) return;
  double2 om = omega[sys];
  cplx<R> a = {(R)om.x, (R)om.y};
  cplx<R> ev[12], rv[12], pv[12];
  load_spinor<P>(e, v.stride, v.idx, ev);
  load_spinor<P>(r, v.stride, v.idx, rv);
  load_spinor<P>(p, v.stride, v.idx, pv);
#pragma unroll
  for (int q = 0; q < 12; q++) {
    ev[q] = ev[q] + a * rv[q];
    rv[q] = rv[q] - a * pv[q];
  }
  store_spinor<P>(e, v.stride, v.idx, ev);
  store_spinor<P>(r, v.stride, v.idx, rv);
}

// a = (p, r) / (p, p) from the partials of a dslash with RED_DOT_Y_NORM (p = out, r = y)
__global__ void k_mr_fin(const double* partial, VGeom vg, const SegInfo* si, int nseg, double2* omega,
                         const int* active) {
  double s[3];
  seg_sum_g<3>(partial, vg, si, 3, 0, s);
  if (threadIdx.x) return;
  const int sys = blockIdx.x * nseg + blockIdx.y;
  bool ok = active[sys] && s[2] > 0.0 && isfinite(s[2]);
  omega[sys] = ok ? make_double2(s[0] / s[2], s[1] / s[2]) : make_double2(0.0, 0.0);
}

// ------------------------------------------------------------------ host launchers
#define GDISPATCH(prec, KERNEL, ...)                \
  do {                                              \
    if ((prec) == P64) KERNEL<P64> __VA_ARGS__;     \
    else if ((prec) == P32) KERNEL<P32> __VA_ARGS__; \
    else KERNEL<P16> __VA_ARGS__;                   \
    lqcd::count_launch();                           \
  } while (0)

static inline dim3 fgrid(const VGeom& vg, int nseg) { return dim3(vg.nrhs, nseg); }

void gcr_init(int prec, const void* b, void* x, void* r, const VGeom& vg, const SegInfo* si, int nseg,
              double* partial, const GState& gs, const double* delta, const int* outer_active, cudaStream_t st) {
  GDISPATCH(prec, k_gcr_init, <<<vg.blocks, vg.threads(), vg.threads() * sizeof(double), st>>>(b, x, r, vg, si,
                                                                                                 partial));
  k_gcr_fin_init<<<fgrid(vg, nseg), 128, 0, st>>>(partial, vg, si, nseg, gs, delta, outer_active);
  lqcd::count_launch();
}

void gcr_orthogonalise(int prec, const VecList& W, const VecList& Z, int k, const void* r, const VGeom& vg,
                       const SegInfo* si, int nseg, double* partial, const GState& gs, cudaStream_t st) {
  if (k > 0) {
    GDISPATCH(prec, k_gcr_dots,
              <<<vg.blocks, vg.threads(), vg.threads() * sizeof(double), st>>>(W, k, vg, si, partial));
    k_gcr_fin_beta<<<fgrid(vg, nseg), 128, 0, st>>>(partial, vg, si, nseg, k, gs);
    lqcd::count_launch();
  }
  GDISPATCH(prec, k_gcr_orth, <<<vg.blocks, vg.threads(), vg.threads() * sizeof(double), st>>>(
                                  W, Z, k, r, vg, si, nseg, gs, partial));
  k_gcr_fin_alpha<<<fgrid(vg, nseg), 128, 0, st>>>(partial, vg, si, nseg, k, gs);
  lqcd::count_launch();
}

void gcr_update(int prec, void* x, void* r, const void* z, const void* w, const VGeom& vg, const SegInfo* si,
                int nseg, double* partial, const GState& gs, cudaStream_t st) {
  GDISPATCH(prec, k_gcr_xr, <<<vg.blocks, vg.threads(), vg.threads() * sizeof(double), st>>>(
                                x, r, z, w, vg, si, nseg, gs, partial));
  k_gcr_fin_r2<<<fgrid(vg, nseg), 128, 0, st>>>(partial, vg, si, nseg, gs);
  lqcd::count_launch();
}

void mr_finish(const double* partial, const VGeom& vg, const SegInfo* si, int nseg, double2* omega,
               const int* active, cudaStream_t st) {
  k_mr_fin<<<fgrid(vg, nseg), 128, 0, st>>>(partial, vg, si, nseg, omega, active);
  lqcd::count_launch();
}

void mr_update(int prec, void* e, void* r, const void* p, const VGeom& vg, const SegInfo* si, int nseg,
               const double2* omega, const int* active, cudaStream_t st) {
  GDISPATCH(prec, k_mr_update, <<<vg.blocks, vg.threads(), 0, st>>>(e, r, p, vg, si, nseg, omega, active));
}

}  // namespace lqcd
