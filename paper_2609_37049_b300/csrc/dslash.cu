// Even-odd hopping term of the clover-Wilson operator (Sec. 2.1 / Sec. 3 of the paper), with
// the clover (or inverse clover) multiplication and the axpy of the Schur complement fused into
// the epilogue, and optionally the Krylov dot products of the output fused into the same pass.
// One thread per (output site, right-hand side), right-hand sides fastest, so the threads of one
// site read its links and clover once per warp (a broadcast) and the spinor loads of a warp are
// contiguous 16-byte chunks.  Site coordinates come from a packed per-site table and the eight
// neighbours from index arithmetic on the lexicographic site (no divisions).
//
//   (H x)(s) = sum_mu (1 + sf gamma_mu) U_mu(s) x(s+mu) + (1 - sf gamma_mu) U_mu(s-mu)^dag x(s-mu)
// with sf = -1 for H and sf = +1 for H^dag.  In the chiral basis gamma_mu = [[0, X],[X^dag, 0]]
// with X_x = -i sigma_x, X_y = -i sigma_y, X_z = -i sigma_z, X_t = 1, so
//   (1 + s gamma_mu) psi = [ h ; s X^dag h ],  h = psi_up + s X psi_down  (two spins x colour):
// only the two-spin half spinor h is multiplied by the link.
#include "lqcd_internal.h"

namespace lqcd {

struct DslashParams {
  Geom g;
  const void* in;
  const void* y;
  const void* z;
  void* out;
  const void* U;
  const void* C;
  const unsigned* coord;  // packed (x, y, z, t) of every site of the output parity
  const signed char* tc;  // device array [Lt]
  double* partial;        // fused reductions: [block][rhs][ND]
  const void* zred;       // vector dotted with the output for RED_DOT_Z
  int out_par;
  int nrhs;
  int S;  // sites per block when reducing
  double a, b;
};

// h = psi_up + s X_mu psi_down
template <int MU, int S, typename R>
LQCD_D void project(const cplx<R> (&p)[12], cplx<R> (&h)[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    cplx<R> p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
    if constexpr (MU == 0) {  // X p_d = (-i p3, -i p2)
      h[0][c] = S > 0 ? p0 + times_mi(p3) : p0 - times_mi(p3);
      h[1][c] = S > 0 ? p1 + times_mi(p2) : p1 - times_mi(p2);
    } else if constexpr (MU == 1) {  // X p_d = (-p3, p2)
      h[0][c] = S > 0 ? p0 - p3 : p0 + p3;
      h[1][c] = S > 0 ? p1 + p2 : p1 - p2;
    } else if constexpr (MU == 2) {  // X p_d = (-i p2, i p3)
      h[0][c] = S > 0 ? p0 + times_mi(p2) : p0 - times_mi(p2);
      h[1][c] = S > 0 ? p1 + times_i(p3) : p1 - times_i(p3);
    } else {  // X p_d = (p2, p3)
      h[0][c] = S > 0 ? p0 + p2 : p0 - p2;
      h[1][c] = S > 0 ? p1 + p3 : p1 - p3;
    }
  }
}

// acc += [ w ; s X^dag w ]
template <int MU, int S, typename R>
LQCD_D void accumulate(cplx<R> (&acc)[12], const cplx<R> (&w)[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    acc[c] = acc[c] + w[0][c];
    acc[3 + c] = acc[3 + c] + w[1][c];
    cplx<R> l2, l3;
    if constexpr (MU == 0) {  // X^dag w = (i w1, i w0)
      l2 = times_i(w[1][c]);
      l3 = times_i(w[0][c]);
    } else if constexpr (MU == 1) {  // X^dag w = (w1, -w0)
      l2 = w[1][c];
      l3 = -w[0][c];
    } else if constexpr (MU == 2) {  // X^dag w = (i w0, -i w1)
      l2 = times_i(w[0][c]);
      l3 = times_mi(w[1][c]);
    } else {
      l2 = w[0][c];
      l3 = w[1][c];
    }
    if constexpr (S > 0) {
      acc[6 + c] = acc[6 + c] + l2;
      acc[9 + c] = acc[9 + c] + l3;
    } else {
      acc[6 + c] = acc[6 + c] - l2;
      acc[9 + c] = acc[9 + c] - l3;
    }
  }
}

template <typename R>
LQCD_D void su3_mul(const cplx<R> (&u)[3][3], const cplx<R> (&h)[2][3], cplx<R> (&w)[2][3]) {
#pragma unroll
  for (int s = 0; s < 2; s++)
#pragma unroll
    for (int a = 0; a < 3; a++) w[s][a] = u[a][0] * h[s][0] + u[a][1] * h[s][1] + u[a][2] * h[s][2];
}

template <typename R>
LQCD_D void su3_dag_mul(const cplx<R> (&u)[3][3], const cplx<R> (&h)[2][3], cplx<R> (&w)[2][3]) {
#pragma unroll
  for (int s = 0; s < 2; s++)
#pragma unroll
    for (int a = 0; a < 3; a++)
      w[s][a] = cjmul(u[0][a], h[s][0]) + cjmul(u[1][a], h[s][1]) + cjmul(u[2][a], h[s][2]);
}

// One direction, forward and backward hop.  cmu / Lmu: coordinate and extent along mu,
// smu: lexicographic stride of mu, coef_f / coef_b: boundary / cut coefficients (+1, -1, 0).
template <int P, int MU, bool DAG>
LQCD_D void hop_dir(const DslashParams& pr, long cb, long s, int cmu, int Lmu, long smu, int coef_f, int coef_b,
                    int rhs, long stride, cplx<typename Traits<P>::real> (&acc)[12]) {
  using R = typename Traits<P>::real;
  constexpr int SF = DAG ? 1 : -1;  // forward projector sign
  constexpr int SB = -SF;
  const int op = pr.out_par, ip = 1 - pr.out_par;
  if (coef_f != 0) {  // U_mu(s) x(s + mu)
    const long sn = s + ((cmu + 1 == Lmu) ? smu * (1 - Lmu) : smu);
    const long nb = sn >> 1;
    cplx<R> p[12];
    load_spinor<P>(pr.in, stride, nb * pr.nrhs + rhs, p);
    cplx<R> h[2][3], w[2][3], u[3][3];
    project<MU, SF>(p, h);
    load_link<P>(pr.U, pr.g.Vh, MU, op, cb, u);
    su3_mul(u, h, w);
    if (coef_f < 0) {
#pragma unroll
      for (int q = 0; q < 2; q++)
#pragma unroll
        for (int a = 0; a < 3; a++) w[q][a] = -w[q][a];
    }
    accumulate<MU, SF>(acc, w);
  }
  if (coef_b != 0) {  // U_mu(s - mu)^dag x(s - mu)
    const long sn = s + ((cmu == 0) ? smu * (Lmu - 1) : -smu);
    const long nb = sn >> 1;
    cplx<R> p[12];
    load_spinor<P>(pr.in, stride, nb * pr.nrhs + rhs, p);
    cplx<R> h[2][3], w[2][3], u[3][3];
    project<MU, SB>(p, h);
    load_link<P>(pr.U, pr.g.Vh, MU, ip, nb, u);
    su3_dag_mul(u, h, w);
    if (coef_b < 0) {
#pragma unroll
      for (int q = 0; q < 2; q++)
#pragma unroll
        for (int a = 0; a < 3; a++) w[q][a] = -w[q][a];
    }
    accumulate<MU, SB>(acc, w);
  }
}

// MINB: minimum resident blocks of 128 threads the compiler must allow (register cap 128 / 80 / 64
// per thread for MINB = 4 / 6 / 8); the autotuner picks the variant per precision and RHS count.
template <int P, int EPI, bool DAG, int RED, int MINB>
__global__ void __launch_bounds__(128, MINB) dslash_kernel(const DslashParams pr) {
  using R = typename Traits<P>::real;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long cb = tid / pr.nrhs;
  const int rhs = (int)(tid - cb * pr.nrhs);
  if (RED == RED_NONE && cb >= pr.g.Vh) return;
  const Geom& g = pr.g;
  const unsigned cw = __ldg(pr.coord + cb);
  const int x = cw & 0xff, y = (cw >> 8) & 0xff, z = (cw >> 16) & 0xff, t = cw >> 24;
  const long sy = g.Lx, sz = (long)g.Lx * g.Ly, st = sz * g.Lz;
  const long s = x + sy * y + sz * z + st * t;
  const long stride = g.Vh * pr.nrhs;
  const long idx = cb * pr.nrhs + rhs;

  cplx<R> acc[12];
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = {R(0), R(0)};
  hop_dir<P, 0, DAG>(pr, cb, s, x, g.Lx, 1, 1, 1, rhs, stride, acc);
  hop_dir<P, 1, DAG>(pr, cb, s, y, g.Ly, sy, 1, 1, rhs, stride, acc);
  hop_dir<P, 2, DAG>(pr, cb, s, z, g.Lz, sz, 1, 1, rhs, stride, acc);
  const int cf = __ldg(pr.tc + t), cbk = __ldg(pr.tc + (t == 0 ? g.Lt - 1 : t - 1));
  hop_dir<P, 3, DAG>(pr, cb, s, t, g.Lt, st, cf, cbk, rhs, stride, acc);

  const R a = (R)pr.a, b = (R)pr.b;
  cplx<R> o[12];
  cplx<R> yv[12];
  if constexpr (EPI == EPI_H) {
#pragma unroll
    for (int k = 0; k < 12; k++) o[k] = b * acc[k];
  } else if constexpr (EPI == EPI_CH) {
    clover_apply<P>(pr.C, g.Vh, cb, acc);
#pragma unroll
    for (int k = 0; k < 12; k++) o[k] = b * acc[k];
  } else if constexpr (EPI == EPI_Y_H || EPI == EPI_Y_CH) {
    if constexpr (EPI == EPI_Y_CH) clover_apply<P>(pr.C, g.Vh, cb, acc);
    load_spinor<P>(pr.y, stride, idx, yv);
#pragma unroll
    for (int k = 0; k < 12; k++) o[k] = a * yv[k] + b * acc[k];
  } else if constexpr (EPI == EPI_C_YH) {
    load_spinor<P>(pr.y, stride, idx, yv);
#pragma unroll
    for (int k = 0; k < 12; k++) o[k] = a * yv[k] + b * acc[k];
    clover_apply<P>(pr.C, g.Vh, cb, o);
  } else if constexpr (EPI == EPI_CY_H) {
    load_spinor<P>(pr.y, stride, idx, yv);
    clover_apply<P>(pr.C, g.Vh, cb, yv);
#pragma unroll
    for (int k = 0; k < 12; k++) o[k] = a * yv[k] + b * acc[k];
  } else {  // EPI_RES: z - (C y + b H x)
    cplx<R> zv[12];
    load_spinor<P>(pr.y, stride, idx, yv);
    clover_apply<P>(pr.C, g.Vh, cb, yv);
    load_spinor<P>(pr.z, stride, idx, zv);
#pragma unroll
    for (int k = 0; k < 12; k++) o[k] = zv[k] - (yv[k] + b * acc[k]);
  }
  store_spinor<P>(pr.out, stride, idx, o);

  if constexpr (RED == RED_DOT_Z) {  // (z, out)
    cplx<R> zv[12];
    load_spinor<P>(pr.zred, stride, idx, zv);
    cplx<R> d = {R(0), R(0)};
#pragma unroll
    for (int k = 0; k < 12; k++) d = d + cjmul(zv[k], o[k]);
    double v[2] = {(double)d.re, (double)d.im};
    block_reduce_rhs<2>(v, pr.partial, pr.S, pr.nrhs, (int)(threadIdx.x / pr.nrhs), rhs);
  } else if constexpr (RED == RED_DOT_Y_NORM) {  // (out, y), (out, out); y is the EPI_Y_* input
    cplx<R> d = {R(0), R(0)};
    R nn = 0;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      d = d + cjmul(o[k], yv[k]);
      nn += norm2(o[k]);
    }
    double v[3] = {(double)d.re, (double)d.im, (double)nn};
    block_reduce_rhs<3>(v, pr.partial, pr.S, pr.nrhs, (int)(threadIdx.x / pr.nrhs), rhs);
  }
}

template <int P>
__global__ void clover_only_kernel(const void* C, const void* in, void* out, long Vh, int nrhs) {
  using R = typename Traits<P>::real;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long cb = tid / nrhs;
  if (cb >= Vh) return;
  const long stride = Vh * nrhs;
  cplx<R> s[12];
  load_spinor<P>(in, stride, tid, s);
  clover_apply<P>(C, Vh, cb, s);
  store_spinor<P>(out, stride, tid, s);
}

template <int P, int EPI, int RED, int MINB>
static void launch_v(const DslashParams& pr, bool dag, long blocks, int tpb, size_t shm, cudaStream_t st) {
  if (dag)
    dslash_kernel<P, EPI, true, RED, MINB><<<blocks, tpb, shm, st>>>(pr);
  else
    dslash_kernel<P, EPI, false, RED, MINB><<<blocks, tpb, shm, st>>>(pr);
  lqcd::count_launch();
}

template <int P, int EPI, int RED>
static void launch_p_e(const DslashParams& pr, bool dag, long blocks, int tpb, size_t shm, int variant,
                       cudaStream_t st) {
  // register-capped variants only where the kernel is not FP64-ALU bound
  if constexpr (P != P64) {
    if (variant == 1) return launch_v<P, EPI, RED, 6>(pr, dag, blocks, tpb, shm, st);
    if (variant == 2) return launch_v<P, EPI, RED, 8>(pr, dag, blocks, tpb, shm, st);
  }
  launch_v<P, EPI, RED, 4>(pr, dag, blocks, tpb, shm, st);
}

template <int P, int RED>
static void launch_p(const DslashParams& pr, int epi, bool dag, long blocks, int tpb, size_t shm, int variant,
                     cudaStream_t st) {
  if constexpr (RED == RED_NONE) {
    switch (epi) {
      case EPI_H: launch_p_e<P, EPI_H, RED>(pr, dag, blocks, tpb, shm, variant, st); break;
      case EPI_CH: launch_p_e<P, EPI_CH, RED>(pr, dag, blocks, tpb, shm, variant, st); break;
      case EPI_Y_H: launch_p_e<P, EPI_Y_H, RED>(pr, dag, blocks, tpb, shm, variant, st); break;
      case EPI_Y_CH: launch_p_e<P, EPI_Y_CH, RED>(pr, dag, blocks, tpb, shm, variant, st); break;
      case EPI_C_YH: launch_p_e<P, EPI_C_YH, RED>(pr, dag, blocks, tpb, shm, variant, st); break;
      case EPI_CY_H: launch_p_e<P, EPI_CY_H, RED>(pr, dag, blocks, tpb, shm, variant, st); break;
      default: launch_p_e<P, EPI_RES, RED>(pr, dag, blocks, tpb, shm, variant, st); break;
    }
  } else {
    // fused reductions are used by the Schur operator's second half only
    launch_p_e<P, EPI_Y_CH, RED>(pr, dag, blocks, tpb, shm, variant, st);
  }
}

template <int RED>
static void launch_prec(int prec, const DslashParams& pr, int epi, bool dag, long blocks, int tpb, size_t shm,
                        int variant, cudaStream_t st) {
  if (prec == P64)
    launch_p<P64, RED>(pr, epi, dag, blocks, tpb, shm, variant, st);
  else if (prec == P32)
    launch_p<P32, RED>(pr, epi, dag, blocks, tpb, shm, variant, st);
  else
    launch_p<P16, RED>(pr, epi, dag, blocks, tpb, shm, variant, st);
}

void launch_dslash(const Geom& g, const DslashCall& c, cudaStream_t st, int variant) {
  DslashParams pr;
  pr.g = g;
  pr.in = c.in;
  pr.y = c.y;
  pr.z = c.z;
  pr.out = c.out;
  pr.U = c.U;
  pr.C = c.C;
  pr.coord = c.coord;
  pr.tc = c.tc;
  pr.partial = c.partial;
  pr.zred = c.zred;
  pr.out_par = c.out_par;
  pr.nrhs = c.nrhs;
  pr.S = c.red_sites;
  pr.a = c.a;
  pr.b = c.b;
  const bool dag = c.dagger != 0;
  if (variant < 0 || variant > 2) variant = 0;
  if (c.red == RED_NONE) {
    long nthreads = g.Vh * (long)c.nrhs;
    const int tpb = 128;
    launch_prec<RED_NONE>(c.prec, pr, c.epi, dag, (nthreads + tpb - 1) / tpb, tpb, 0, variant, st);
  } else {
    // one block = red_sites sites (inside one timeslice) x nrhs right-hand sides (<= 128 threads)
    const int tpb = c.red_sites * c.nrhs;
    const long blocks = g.Vh / c.red_sites;
    const int nd = c.red == RED_DOT_Z ? 2 : 3;
    const size_t shm = (size_t)nd * tpb * sizeof(double);
    if (c.red == RED_DOT_Z)
      launch_prec<RED_DOT_Z>(c.prec, pr, c.epi, dag, blocks, tpb, shm, variant, st);
    else
      launch_prec<RED_DOT_Y_NORM>(c.prec, pr, c.epi, dag, blocks, tpb, shm, variant, st);
  }
}

void launch_clover_only(const Geom& g, int prec, const void* C, const void* in, void* out, int nrhs,
                        cudaStream_t st) {
  long n = g.Vh * (long)nrhs;
  int tpb = 128;
  long blocks = (n + tpb - 1) / tpb;
  if (prec == P64)
    clover_only_kernel<P64><<<blocks, tpb, 0, st>>>(C, in, out, g.Vh, nrhs);
  else if (prec == P32)
    clover_only_kernel<P32><<<blocks, tpb, 0, st>>>(C, in, out, g.Vh, nrhs);
  else
    clover_only_kernel<P16><<<blocks, tpb, 0, st>>>(C, in, out, g.Vh, nrhs);
  lqcd::count_launch();
}

}  // namespace lqcd
