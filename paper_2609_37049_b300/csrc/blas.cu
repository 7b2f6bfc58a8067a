// Vector kernels of the Krylov solvers: fused BiCGStab updates, segmented (per domain) dot
// products and the finishing kernels that turn per-block partial sums into the per-system
// Krylov scalars on the device, so an iteration needs no host round trip and can be replayed
// from a CUDA graph.
//
// Reductions are two-pass and deterministic: every vector kernel block covers S sites (all in
// one timeslice of one parity) times nrhs right-hand sides and writes one partial sum per
// right-hand side; a finishing kernel with one block per system (rhs, segment) adds the partial
// sums of the blocks that lie in the segment's timeslices.  Per-thread products are formed in
// the storage precision's arithmetic type; block and segment sums are FP64.
#include "lqcd_blas.h"

namespace lqcd {

VGeom make_vgeom(const Geom& g, int nrhs, int npar) {
  VGeom v;
  v.g = g;
  v.nrhs = nrhs;
  v.npar = npar;
  int target = 128 / nrhs;  // blocks of at most 128 threads (the dslash launch bound)
  if (target < 1) target = 1;
  int S = 1;
  while (S * 2 <= target && (g.Vth % (S * 2)) == 0) S *= 2;
  v.S = S;
  v.bpp = g.Vh / S;
  v.bpt = g.Vth / S;
  v.blocks = v.bpp * npar;
  return v;
}

struct VThread {
  int par;
  long cb;
  int rhs;
  int t;
  int seg;
  long idx;     // cb * nrhs + rhs (within a parity block)
  long stride;  // Vh * nrhs (chunk stride)
  int site_local;
};

LQCD_D VThread vthread(const VGeom& vg, const SegInfo* si) {
  VThread v;
  v.site_local = threadIdx.x / vg.nrhs;
  v.rhs = threadIdx.x - v.site_local * vg.nrhs;
  long site = (long)blockIdx.x * vg.S + v.site_local;
  v.par = (int)(site / vg.g.Vh);
  v.cb = site - (long)v.par * vg.g.Vh;
  v.t = (int)(v.cb / vg.g.Vth);
  v.seg = si ? si->seg_of_t[v.t] : 0;
  v.idx = v.cb * vg.nrhs + v.rhs;
  v.stride = vg.g.Vh * vg.nrhs;
  return v;
}

template <int P>
LQCD_D const void* fpar(const void* base, const VGeom& vg, int par) {
  return reinterpret_cast<const char*>(base) + (size_t)par * (size_t)vg.g.Vh * vg.nrhs * 12 *
                                                   (P == P64 ? 16 : (P == P32 ? 8 : 4));
}
template <int P>
LQCD_D void* fpar(void* base, const VGeom& vg, int par) {
  return reinterpret_cast<char*>(base) + (size_t)par * (size_t)vg.g.Vh * vg.nrhs * 12 *
                                             (P == P64 ? 16 : (P == P32 ? 8 : 4));
}

// Reduce ND values over the S sites of the block for each rhs; write partial[block][rhs][ND].
template <int ND>
LQCD_D void block_reduce(double (&v)[ND], double* partial, const VGeom& vg, int site_local, int rhs) {
  extern __shared__ double sm[];
  const int n = blockDim.x;
#pragma unroll
  for (int k = 0; k < ND; k++) sm[k * n + threadIdx.x] = v[k];
  __syncthreads();
  for (int s = vg.S / 2; s >= 1; s >>= 1) {
    if (site_local < s) {
#pragma unroll
      for (int k = 0; k < ND; k++) sm[k * n + threadIdx.x] += sm[k * n + threadIdx.x + s * vg.nrhs];
    }
    __syncthreads();
  }
  if (site_local == 0) {
#pragma unroll
    for (int k = 0; k < ND; k++) partial[((long)blockIdx.x * vg.nrhs + rhs) * ND + k] = sm[k * n + threadIdx.x];
  }
}

// Sum the partials of system (rhs = blockIdx.x, seg = blockIdx.y); result valid in thread 0.
template <int ND>
LQCD_D void seg_sum(const double* partial, const VGeom& vg, const SegInfo* si, double (&out)[ND]) {
  __shared__ double sm[ND][128];
  const int rhs = blockIdx.x, seg = blockIdx.y;
  double acc[ND];
#pragma unroll
  for (int k = 0; k < ND; k++) acc[k] = 0.0;
  for (int rg = 0; rg < 2; rg++) {  // the segment's timeslice range(s)
    const long t0 = si ? (rg ? si->t0b[seg] : si->t0[seg]) : 0;
    const long t1 = si ? (rg ? si->t1b[seg] : si->t1[seg]) : (rg ? 0 : vg.g.Lt);
    const long nb_seg = (t1 - t0) * vg.bpt;
    for (int par = 0; par < vg.npar; par++) {
      const long b0 = par * vg.bpp + t0 * vg.bpt;
      for (long b = threadIdx.x; b < nb_seg; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < ND; k++) acc[k] += partial[((b0 + b) * vg.nrhs + rhs) * ND + k];
      }
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

// Two-level segment sums for the BiCGStab scalars (one parity, vg.npar = 1).  The per-block
// partials of a segment are first summed over chunks of kChunk consecutive blocks, threads over
// the (rhs, k) entries of a block so that every read is coalesced; the finishing kernel of a
// system then adds its segment's chunk sums.  Fixed order: deterministic.
constexpr int kChunk = 64;

template <int ND>
__global__ void k_chunk_sum(const double* partial, VGeom vg, const SegInfo* si, int nchunk, double* p2) {
  const int c = blockIdx.x, seg = blockIdx.y;
  const int e = threadIdx.x;  // rhs * ND + k
  if (e >= vg.nrhs * ND) return;
  const long t0 = si ? si->t0[seg] : 0, t1 = si ? si->t1[seg] : vg.g.Lt;
  const long u0 = si ? si->t0b[seg] : 0, u1 = si ? si->t1b[seg] : 0;
  const long n0 = (t1 - t0) * vg.bpt, n1 = (u1 - u0) * vg.bpt;
  const long f0 = (long)c * kChunk, f1 = min(f0 + kChunk, n0 + n1);
  const long w = (long)vg.nrhs * ND;
  double acc = 0;
#pragma unroll 8
  for (long f = f0; f < f1; f++) {
    const long b = f < n0 ? t0 * vg.bpt + f : u0 * vg.bpt + (f - n0);
    acc += partial[b * w + e];
  }
  p2[((long)seg * nchunk + c) * w + e] = acc;
}

// Sum of the chunk sums of system (rhs = blockIdx.x, seg = blockIdx.y); valid in thread 0.
template <int ND>
LQCD_D void chunk_total(const double* p2, int nchunk, int nrhs, double (&out)[ND]) {
  __shared__ double sm[ND][128];
  const int rhs = blockIdx.x, seg = blockIdx.y;
  double acc[ND];
#pragma unroll
  for (int k = 0; k < ND; k++) acc[k] = 0.0;
  for (int c = threadIdx.x; c < nchunk; c += blockDim.x) {
#pragma unroll
    for (int k = 0; k < ND; k++) acc[k] += p2[(((long)seg * nchunk + c) * nrhs + rhs) * ND + k];
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

// chunks needed by the largest segment of a half-lattice batch
int seg_chunks(const VGeom& vg, const SegInfo& si_host) {
  long most = 0;
  for (int s = 0; s < si_host.nseg; s++) {
    const long n = ((long)(si_host.t1[s] - si_host.t0[s]) + (si_host.t1b[s] - si_host.t0b[s])) * vg.bpt;
    most = n > most ? n : most;
  }
  return (int)((most + kChunk - 1) / kChunk);
}

// ------------------------------------------------------------------ generic kernels
template <int P>
__global__ void k_norm2(const void* x, VGeom vg, const SegInfo* si, double* partial) {
  using R = typename Traits<P>::real;
  VThread v = vthread(vg, si);
  cplx<R> a[12];
  load_spinor<P>(fpar<P>(x, vg, v.par), v.stride, v.idx, a);
  R s = 0;
#pragma unroll
  for (int k = 0; k < 12; k++) s += norm2(a[k]);
  double d[1] = {(double)s};
  block_reduce<1>(d, partial, vg, v.site_local, v.rhs);
}

__global__ void k_fin_sum1(const double* partial, VGeom vg, const SegInfo* si, int nseg, double* out) {
  double s[1];
  seg_sum<1>(partial, vg, si, s);
  if (threadIdx.x == 0) out[blockIdx.x * nseg + blockIdx.y] = s[0];
}

// out = scale[sys] * in  (precision conversion)
template <int PI, int PO>
__global__ void k_convert(const void* in, void* out, VGeom vg, const SegInfo* si, int nseg, const double* scale) {
  using RI = typename Traits<PI>::real;
  using RO = typename Traits<PO>::real;
  VThread v = vthread(vg, si);
  cplx<RI> a[12];
  load_spinor<PI>(fpar<PI>(in, vg, v.par), v.stride, v.idx, a);
  double sc = scale ? scale[v.rhs * nseg + v.seg] : 1.0;
  cplx<RO> b[12];
#pragma unroll
  for (int k = 0; k < 12; k++) b[k] = {(RO)(sc * (double)a[k].re), (RO)(sc * (double)a[k].im)};
  store_spinor<PO>(fpar<PO>(out, vg, v.par), v.stride, v.idx, b);
}

// x (P64) += scale[sys] * e (PE)
template <int PE>
__global__ void k_axpy_mixed(void* x, const void* e, VGeom vg, const SegInfo* si, int nseg, const double* scale,
                             const int* active) {
  using RE = typename Traits<PE>::real;
  VThread v = vthread(vg, si);
  const int sys = v.rhs * nseg + v.seg;
  if (active && !active[sys]) return;
  double sc = scale ? scale[sys] : 1.0;
  cplx<RE> ev[12];
  load_spinor<PE>(fpar<PE>(e, vg, v.par), v.stride, v.idx, ev);
  cplx<double> xv[12];
  void* xp = fpar<P64>(x, vg, v.par);
  load_spinor<P64>(xp, v.stride, v.idx, xv);
#pragma unroll
  for (int k = 0; k < 12; k++) xv[k] = xv[k] + mk(sc * (double)ev[k].re, sc * (double)ev[k].im);
  store_spinor<P64>(xp, v.stride, v.idx, xv);
}

template <int P>
__global__ void k_zero(void* x, VGeom vg) {
  using R = typename Traits<P>::real;
  VThread v = vthread(vg, nullptr);
  cplx<R> z[12];
#pragma unroll
  for (int k = 0; k < 12; k++) z[k] = {R(0), R(0)};
  store_spinor<P>(fpar<P>(x, vg, v.par), v.stride, v.idx, z);
}

template <int P>
__global__ void k_copy(const void* a, void* b, VGeom vg) {
  using R = typename Traits<P>::real;
  VThread v = vthread(vg, nullptr);
  cplx<R> z[12];
  load_spinor<P>(fpar<P>(a, vg, v.par), v.stride, v.idx, z);
  store_spinor<P>(fpar<P>(b, vg, v.par), v.stride, v.idx, z);
}

// ------------------------------------------------------------------ BiCGStab stages
// init: r = b, p = b, x = 0; partial |b|^2
template <int P>
__global__ void k_bicg_init(const void* b, void* r, void* p, void* x, VGeom vg, const SegInfo* si, double* partial) {
  using R = typename Traits<P>::real;
  VThread v = vthread(vg, si);
  cplx<R> a[12], z[12];
  load_spinor<P>(b, v.stride, v.idx, a);
  store_spinor<P>(r, v.stride, v.idx, a);
  store_spinor<P>(p, v.stride, v.idx, a);
  R s = 0;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    s += norm2(a[k]);
    z[k] = {R(0), R(0)};
  }
  store_spinor<P>(x, v.stride, v.idx, z);
  double d[1] = {(double)s};
  block_reduce<1>(d, partial, vg, v.site_local, v.rhs);
}

__global__ void k_bicg_fin_init(const double* partial, VGeom vg, const SegInfo* si, int nseg, KState ks,
                                const double* delta, const int* outer_active) {
  double s[1];
  seg_sum<1>(partial, vg, si, s);
  if (threadIdx.x) return;
  const int sys = blockIdx.x * nseg + blockIdx.y;
  ks.b2[sys] = s[0];
  ks.r2[sys] = s[0];
  ks.rho[sys] = make_double2(s[0], 0.0);
  ks.alpha[sys] = make_double2(0.0, 0.0);
  ks.omega[sys] = make_double2(0.0, 0.0);
  ks.beta[sys] = make_double2(0.0, 0.0);
  double d = delta ? delta[sys] : 1e-6;
  ks.stop2[sys] = d * d * s[0];
  ks.flag[sys] = 0;
  ks.active[sys] = (s[0] > 0.0) && (!outer_active || outer_active[sys]);
}

LQCD_D double2 cdiv(double2 a, double2 b) {
  double den = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
LQCD_D double2 cmul2(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

__global__ void k_bicg_fin_alpha(const double* p2, int nchunk, int nrhs, int nseg, KState ks) {
  double s[2];
  chunk_total<2>(p2, nchunk, nrhs, s);
  if (threadIdx.x) return;
  const int sys = blockIdx.x * nseg + blockIdx.y;
  double2 r0v = make_double2(s[0], s[1]);
  double mag = r0v.x * r0v.x + r0v.y * r0v.y;
  if (!ks.active[sys]) {
    ks.alpha[sys] = make_double2(0.0, 0.0);
    return;
  }
  double2 rho = ks.rho[sys];
  if (!(mag > 0.0) || !isfinite(mag)) {
    ks.alpha[sys] = make_double2(0.0, 0.0);
    ks.active[sys] = 0;
    ks.flag[sys] = 1;
    return;
  }
  ks.alpha[sys] = cdiv(rho, r0v);
}

// s = r - alpha v
template <int P>
__global__ void k_bicg_s(const void* r, const void* vv, void* s, VGeom vg, const SegInfo* si, int nseg, KState ks) {
  using R = typename Traits<P>::real;
  VThread v = vthread(vg, si);
  double2 al = ks.alpha[v.rhs * nseg + v.seg];
  cplx<R> a = {(R)al.x, (R)al.y};
  cplx<R> x[12], y[12];
  load_spinor<P>(r, v.stride, v.idx, x);
  load_spinor<P>(vv, v.stride, v.idx, y);
#pragma unroll
  for (int k = 0; k < 12; k++) x[k] = x[k] - a * y[k];
  store_spinor<P>(s, v.stride, v.idx, x);
}

// One reduction phase per BiCGStab iteration: after t = M s, whose fused reduction gives
// (t,s), (t,t), (r0,t), (r0,s), (s,s), every scalar of the iteration is known:
//   omega = (t,s)/(t,t),  rho' = (r0, s - omega t) = (r0,s) - omega (r0,t),
//   beta = (rho'/rho)(alpha/omega),  |r'|^2 = |s|^2 - |(t,s)|^2/(t,t)  (stopping test),
// so x, r and p are updated in one pass (k_bicg_xrp) instead of two with a reduction between.
__global__ void k_bicg_fin_tail(const double* p2, int nchunk, int nrhs, int nseg, KState ks) {
  double s[8];
  chunk_total<8>(p2, nchunk, nrhs, s);
  if (threadIdx.x) return;
  const int sys = blockIdx.x * nseg + blockIdx.y;
  if (!ks.active[sys]) {
    ks.omega[sys] = make_double2(0.0, 0.0);
    ks.beta[sys] = make_double2(0.0, 0.0);
    return;
  }
  const double tt = s[2];
  if (!(tt > 0.0) || !isfinite(tt)) {  // t = 0 (s = 0) or overflow: stop this system
    ks.omega[sys] = make_double2(0.0, 0.0);
    ks.beta[sys] = make_double2(0.0, 0.0);
    ks.active[sys] = 0;
    ks.flag[sys] = isfinite(tt) ? 1 : 2;
    ks.iters[sys] += 1;
    return;
  }
  const double2 om = make_double2(s[0] / tt, s[1] / tt);
  ks.omega[sys] = om;
  const double2 rho_new = make_double2(s[5] - (om.x * s[3] - om.y * s[4]), s[6] - (om.x * s[4] + om.y * s[3]));
  double r2 = s[7] - (s[0] * s[0] + s[1] * s[1]) / tt;
  r2 = r2 > 0.0 ? r2 : 0.0;
  ks.r2[sys] = r2;
  ks.iters[sys] += 1;
  ks.beta[sys] = make_double2(0.0, 0.0);
  if (!isfinite(r2) || !isfinite(s[7])) {
    ks.active[sys] = 0;
    ks.flag[sys] = 2;
    return;
  }
  if (r2 <= ks.stop2[sys]) {  // converged: this iteration's x and r updates still apply
    ks.active[sys] = 0;
    return;
  }
  const double2 rho = ks.rho[sys];
  const double om2 = om.x * om.x + om.y * om.y, rh2 = rho.x * rho.x + rho.y * rho.y;
  if (!(om2 > 0.0) || !(rh2 > 0.0)) {
    ks.active[sys] = 0;
    ks.flag[sys] = 1;
    return;
  }
  ks.beta[sys] = cmul2(cdiv(rho_new, rho), cdiv(ks.alpha[sys], om));
  ks.rho[sys] = rho_new;
}

// x += alpha p + omega s;  r = s - omega t;  p = r + beta (p - omega v)
template <int P>
__global__ void k_bicg_xrp(void* x, void* p, const void* s, const void* t, void* r, const void* vv, VGeom vg,
                           const SegInfo* si, int nseg, KState ks) {
  using R = typename Traits<P>::real;
  VThread v = vthread(vg, si);
  const int sys = v.rhs * nseg + v.seg;
  const double2 al = ks.alpha[sys], om = ks.omega[sys], be = ks.beta[sys];
  const cplx<R> a = {(R)al.x, (R)al.y}, w = {(R)om.x, (R)om.y}, bt = {(R)be.x, (R)be.y};
  cplx<R> xv[12], pv[12], sv[12], tv[12], vv2[12];
  load_spinor<P>(x, v.stride, v.idx, xv);
  load_spinor<P>(p, v.stride, v.idx, pv);
  load_spinor<P>(s, v.stride, v.idx, sv);
  load_spinor<P>(t, v.stride, v.idx, tv);
  load_spinor<P>(vv, v.stride, v.idx, vv2);
#pragma unroll
  for (int k = 0; k < 12; k++) {
    xv[k] = xv[k] + a * pv[k] + w * sv[k];
    sv[k] = sv[k] - w * tv[k];                     // new r
    pv[k] = sv[k] + bt * (pv[k] - w * vv2[k]);      // new p
  }
  store_spinor<P>(x, v.stride, v.idx, xv);
  store_spinor<P>(r, v.stride, v.idx, sv);
  store_spinor<P>(p, v.stride, v.idx, pv);
}

__global__ void k_count_active(const int* active, int n, int* count) {
  __shared__ int sm[256];
  int s = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += active[i] ? 1 : 0;
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k >= 1; k >>= 1) {
    if (threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) count[0] = sm[0];
}

// Condition of a device-side solver loop (a WHILE node of a CUDA graph): counts the active systems
// and sets the node's condition.  ctr: [0] inner iterations summed over cycles, [1] defect-correction
// cycles, [2] inner chunks run.  mode 0: before the cycles (any active); 1: end of a cycle
// (ctr[1]++; any active and ctr[1] < max_outer and ctr[0] < max_iter); 2: before an inner loop (any
// active and ctr[0] < max_iter); 3: end of an inner chunk (ctr[0] += chunk, ctr[2]++; same test).
__global__ void k_loop_cond(const int* active, int n, int* ctr, int mode, int chunk, int max_outer, int max_iter,
                            cudaGraphConditionalHandle h) {
  __shared__ int sm[256];
  int s = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += active[i] ? 1 : 0;
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k >= 1; k >>= 1) {
    if (threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x) return;
  const int any = sm[0] > 0;
  unsigned go = any;
  if (mode == 1) {
    ctr[1] += 1;
    go = any && ctr[1] < max_outer && ctr[0] < max_iter;
  } else if (mode == 2) {
    go = any && ctr[0] < max_iter;
  } else if (mode == 3) {
    ctr[0] += chunk;
    ctr[2] += 1;
    go = any && ctr[0] < max_iter;
  }
  cudaGraphSetConditional(h, go);
}

// outer-loop bookkeeping: r2 -> active, inner delta and scale per system
__global__ void k_outer_update(const double* r2, const double* b2, int nsys, double tol, double inner_tol,
                               int* active, double* delta, double* scale, double* rel, int first) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsys) return;
  double bn = b2[i], rn = r2[i];
  if (!isfinite(bn) || !isfinite(rn)) {  // a non-finite source or residual: report NaN, stop the system
    rel[i] = __longlong_as_double(0x7ff8000000000000LL);
    active[i] = 0;
    delta[i] = 0.5;
    scale[i] = 1.0;
    return;
  }
  double rr = bn > 0 ? sqrt(rn / bn) : 0.0;
  rel[i] = rr;
  int act = (bn > 0) && (rr > tol);
  if (!first && !active[i]) act = 0;
  active[i] = act;
  // the inner solve must reduce this residual by inner_tol, but no further than needed
  double need = rr > 0 ? 0.5 * tol / rr : 1.0;
  double d = inner_tol > need ? inner_tol : need;
  delta[i] = d < 1.0 ? d : 0.5;
  scale[i] = rn > 0 ? 1.0 / sqrt(rn) : 1.0;
}

__global__ void k_recip(const double* a, double* b, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i] != 0.0 ? 1.0 / a[i] : 0.0;
}

// ------------------------------------------------------------------ host launchers
static inline size_t shm(const VGeom& vg, int nd) { return (size_t)nd * vg.threads() * sizeof(double); }
static inline dim3 fin_grid(const VGeom& vg, int nseg) { return dim3(vg.nrhs, nseg); }

#define DISPATCH_P(prec, KERNEL, ...)            \
  do {                                           \
    if ((prec) == P64) KERNEL<P64> __VA_ARGS__;  \
    else if ((prec) == P32) KERNEL<P32> __VA_ARGS__; \
    else KERNEL<P16> __VA_ARGS__;                \
    lqcd::count_launch();                        \
  } while (0)

void v_norm2(int prec, const void* x, const VGeom& vg, const SegInfo* si, int nseg, double* partial, double* out,
             cudaStream_t st) {
  DISPATCH_P(prec, k_norm2, <<<vg.blocks, vg.threads(), shm(vg, 1), st>>>(x, vg, si, partial));
  k_fin_sum1<<<fin_grid(vg, nseg), 128, 0, st>>>(partial, vg, si, nseg, out); lqcd::count_launch();
}

void v_convert(int pin, int pout, const void* in, void* out, const VGeom& vg, const SegInfo* si, int nseg,
               const double* scale, cudaStream_t st) {
#define CONV(A, B)                                                                    \
  do {                                                                                \
    k_convert<A, B><<<vg.blocks, vg.threads(), 0, st>>>(in, out, vg, si, nseg, scale); \
    lqcd::count_launch();                                                             \
  } while (0)
  if (pin == P64 && pout == P32) CONV(P64, P32);
  else if (pin == P64 && pout == P16) CONV(P64, P16);
  else if (pin == P32 && pout == P64) CONV(P32, P64);
  else if (pin == P16 && pout == P64) CONV(P16, P64);
  else if (pin == P32 && pout == P16) CONV(P32, P16);
  else if (pin == P16 && pout == P32) CONV(P16, P32);
  else if (pin == P64 && pout == P64) CONV(P64, P64);
  else if (pin == P32 && pout == P32) CONV(P32, P32);
  else CONV(P16, P16);
#undef CONV
}

void v_axpy_mixed(int pe, void* x, const void* e, const VGeom& vg, const SegInfo* si, int nseg, const double* scale,
                  const int* active, cudaStream_t st) {
  DISPATCH_P(pe, k_axpy_mixed, <<<vg.blocks, vg.threads(), 0, st>>>(x, e, vg, si, nseg, scale, active));
}

void v_zero(int prec, void* x, const VGeom& vg, cudaStream_t st) {
  DISPATCH_P(prec, k_zero, <<<vg.blocks, vg.threads(), 0, st>>>(x, vg));
}

void v_copy(int prec, const void* a, void* b, const VGeom& vg, cudaStream_t st) {
  DISPATCH_P(prec, k_copy, <<<vg.blocks, vg.threads(), 0, st>>>(a, b, vg));
}

void bicg_init(int prec, const void* b, void* r, void* p, void* x, const VGeom& vg, const SegInfo* si, int nseg,
               double* partial, const KState& ks, const double* delta, const int* outer_active, cudaStream_t st) {
  DISPATCH_P(prec, k_bicg_init, <<<vg.blocks, vg.threads(), shm(vg, 1), st>>>(b, r, p, x, vg, si, partial));
  k_bicg_fin_init<<<fin_grid(vg, nseg), 128, 0, st>>>(partial, vg, si, nseg, ks, delta, outer_active); lqcd::count_launch();
}

void bicg_s(int prec, const void* r, const void* v, void* s, const VGeom& vg, const SegInfo* si, int nseg,
            const KState& ks, cudaStream_t st) {
  DISPATCH_P(prec, k_bicg_s, <<<vg.blocks, vg.threads(), 0, st>>>(r, v, s, vg, si, nseg, ks));
}

// Finishing kernels alone, for partial sums produced by a dslash with fused reductions.
void bicg_fin_alpha_only(const double* partial, double* p2, int nchunk, const VGeom& vg, const SegInfo* si,
                         int nseg, const KState& ks, cudaStream_t st) {
  k_chunk_sum<2><<<dim3(nchunk, nseg), vg.nrhs * 2, 0, st>>>(partial, vg, si, nchunk, p2); lqcd::count_launch();
  k_bicg_fin_alpha<<<fin_grid(vg, nseg), 128, 0, st>>>(p2, nchunk, vg.nrhs, nseg, ks);
  lqcd::count_launch();
}

void bicg_tail(int prec, void* x, void* p, const void* s, const void* t, void* r, const void* v,
               const double* partial, double* p2, int nchunk, const VGeom& vg, const SegInfo* si, int nseg,
               const KState& ks, cudaStream_t st) {
  k_chunk_sum<8><<<dim3(nchunk, nseg), vg.nrhs * 8, 0, st>>>(partial, vg, si, nchunk, p2); lqcd::count_launch();
  k_bicg_fin_tail<<<fin_grid(vg, nseg), 128, 0, st>>>(p2, nchunk, vg.nrhs, nseg, ks); lqcd::count_launch();
  DISPATCH_P(prec, k_bicg_xrp, <<<vg.blocks, vg.threads(), 0, st>>>(x, p, s, t, r, v, vg, si, nseg, ks));
}

void count_active(const int* active, int n, int* count, cudaStream_t st) {
  k_count_active<<<1, 256, 0, st>>>(active, n, count); lqcd::count_launch();
}

void outer_update(const double* r2, const double* b2, int nsys, double tol, double inner_tol, int* active,
                  double* delta, double* scale, double* rel, int first, cudaStream_t st) {
  k_outer_update<<<(nsys + 127) / 128, 128, 0, st>>>(r2, b2, nsys, tol, inner_tol, active, delta, scale, rel,
                                                     first); lqcd::count_launch();
}

void loop_cond(const int* active, int n, int* ctr, int mode, int chunk, int max_outer, int max_iter,
               cudaGraphConditionalHandle h, cudaStream_t st) {
  k_loop_cond<<<1, 256, 0, st>>>(active, n, ctr, mode, chunk, max_outer, max_iter, h);
  lqcd::count_launch();
}

void recip(const double* a, double* b, int n, cudaStream_t st) {
  k_recip<<<(n + 127) / 128, 128, 0, st>>>(a, b, n); lqcd::count_launch();
}

}  // namespace lqcd
