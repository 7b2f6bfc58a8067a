// Building blocks of the even-odd dslash kernels (dslash.cu: direct loads; dslash_staged.cu:
// links, clover or neighbour spinors staged in shared memory): kernel parameters, spin
// projection and reconstruction for the chiral basis, SU(3) products, and the fused epilogue.
#pragma once
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
  int pipe_off;  // staged-spinor kernels: byte offset of the staging buffers in dynamic shared memory
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
    for (int a = 0; a < 3; a++) w[s][a] = cfma(u[a][2], h[s][2], cfma(u[a][1], h[s][1], u[a][0] * h[s][0]));
}

template <typename R>
LQCD_D void su3_dag_mul(const cplx<R> (&u)[3][3], const cplx<R> (&h)[2][3], cplx<R> (&w)[2][3]) {
#pragma unroll
  for (int s = 0; s < 2; s++)
#pragma unroll
    for (int a = 0; a < 3; a++)
      w[s][a] = cjfma(u[2][a], h[s][2], cjfma(u[1][a], h[s][1], cjmul(u[0][a], h[s][0])));
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

// One hop whose neighbour spinor p is already loaded: forward (U_mu(s) p, link of the output site
// cb) or backward (U_mu(s - mu)^dag p, link of the neighbour nb), scaled by the coefficient
// coef (+1 / -1; 0 means the hop is cut and is skipped by the caller).
template <int P, int MU, bool FWD, bool DAG>
LQCD_D void hop_one(const DslashParams& pr, long cb, long nb, int coef, const cplx<typename Traits<P>::real> (&p)[12],
                    cplx<typename Traits<P>::real> (&acc)[12]) {
  using R = typename Traits<P>::real;
  constexpr int SF = DAG ? 1 : -1;
  constexpr int SG = FWD ? SF : -SF;
  cplx<R> h[2][3], w[2][3], u[3][3];
  project<MU, SG>(p, h);
  if constexpr (FWD) {
    load_link<P>(pr.U, pr.g.Vh, MU, pr.out_par, cb, u);
    su3_mul(u, h, w);
  } else {
    load_link<P>(pr.U, pr.g.Vh, MU, 1 - pr.out_par, nb, u);
    su3_dag_mul(u, h, w);
  }
  if (coef < 0) {
#pragma unroll
    for (int q = 0; q < 2; q++)
#pragma unroll
      for (int a = 0; a < 3; a++) w[q][a] = -w[q][a];
  }
  accumulate<MU, SG>(acc, w);
}

// Epilogue shared by the dslash kernels: combine the hopping sum acc of site cb / right-hand side
// rhs with the clover term and the y / z inputs as EPI says, store it, and form the fused partial
// sums.  `idx` = cb * nrhs + rhs, `stride` = Vh * nrhs (the chunk stride of a spinor field).
// The site's clover block (both chiralities) applied to s in place: from global memory, or (SC)
// from the block's shared-memory copy sc = 18 float4 (chirality-major, packed as in global).
template <int P, bool SC>
LQCD_D void clover_site(const DslashParams& pr, long cb, const float4* sc, cplx<typename Traits<P>::real> (&s)[12]) {
  using R = typename Traits<P>::real;
  if constexpr (SC) {
#pragma unroll
    for (int ch = 0; ch < 2; ch++) {
      R r[36];
#pragma unroll
      for (int c = 0; c < 9; c++) {
        const float4 v = sc[ch * 9 + c];
        r[4 * c] = v.x; r[4 * c + 1] = v.y; r[4 * c + 2] = v.z; r[4 * c + 3] = v.w;
      }
      cplx<R> y[6];
      herm6_apply<R>(r, &s[6 * ch], y);
#pragma unroll
      for (int i = 0; i < 6; i++) s[6 * ch + i] = y[i];
    }
  } else {
    clover_apply<P>(pr.C, pr.g.Vh, cb, s);
  }
}

template <int P, int EPI, int RED, bool SC = false>
LQCD_D void dslash_epilogue(const DslashParams& pr, long cb, long idx, long stride, int rhs,
                            cplx<typename Traits<P>::real> (&acc)[12], const float4* sc = nullptr) {
  using R = typename Traits<P>::real;
  const R a = (R)pr.a, b = (R)pr.b;
  cplx<R> o[12];
  cplx<R> yv[12];
  if constexpr (EPI == EPI_H) {
#pragma unroll
    for (int k = 0; k < 12; k++) o[k] = b * acc[k];
  } else if constexpr (EPI == EPI_CH) {
    clover_site<P, SC>(pr, cb, sc, acc);
#pragma unroll
    for (int k = 0; k < 12; k++) o[k] = b * acc[k];
  } else if constexpr (EPI == EPI_Y_H || EPI == EPI_Y_CH) {
    if constexpr (EPI == EPI_Y_CH) clover_site<P, SC>(pr, cb, sc, acc);
    load_spinor<P>(pr.y, stride, idx, yv);
#pragma unroll
    for (int k = 0; k < 12; k++) o[k] = a * yv[k] + b * acc[k];
  } else if constexpr (EPI == EPI_C_YH) {
    load_spinor<P>(pr.y, stride, idx, yv);
#pragma unroll
    for (int k = 0; k < 12; k++) o[k] = a * yv[k] + b * acc[k];
    clover_site<P, SC>(pr, cb, sc, o);
  } else if constexpr (EPI == EPI_CY_H) {
    load_spinor<P>(pr.y, stride, idx, yv);
    clover_site<P, SC>(pr, cb, sc, yv);
#pragma unroll
    for (int k = 0; k < 12; k++) o[k] = a * yv[k] + b * acc[k];
  } else {  // EPI_RES: z - (C y + b H x)
    cplx<R> zv[12];
    load_spinor<P>(pr.y, stride, idx, yv);
    clover_site<P, SC>(pr, cb, sc, yv);
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
  } else if constexpr (RED == RED_TS_R0) {  // (out, y), (out, out), (z, out), (z, y), (y, y)
    cplx<R> zv[12];
    load_spinor<P>(pr.zred, stride, idx, zv);
    cplx<R> ty = {R(0), R(0)}, zo = {R(0), R(0)}, zy = {R(0), R(0)};
    R oo = 0, yy = 0;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      ty = ty + cjmul(o[k], yv[k]);
      zo = zo + cjmul(zv[k], o[k]);
      zy = zy + cjmul(zv[k], yv[k]);
      oo += norm2(o[k]);
      yy += norm2(yv[k]);
    }
    double v[8] = {(double)ty.re, (double)ty.im, (double)oo, (double)zo.re,
                   (double)zo.im, (double)zy.re, (double)zy.im, (double)yy};
    block_reduce_rhs<8>(v, pr.partial, pr.S, pr.nrhs, (int)(threadIdx.x / pr.nrhs), rhs);
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

// dslash_staged.cu: launch the staged kernel of launch variant 3-5; false (nothing launched) where
// it does not apply.  red_shm = dynamic shared memory of the fused reduction.
// dslash_rb2.cu: launch variant 7 (two right-hand sides per thread), FP32 only.
bool launch_dslash_rb2(const DslashParams& pr, int epi, int red, long blocks, int tpb, size_t red_shm,
                       cudaStream_t st);
bool launch_dslash_staged(const DslashParams& pr, int prec, int epi, bool dag, int red, long blocks, int tpb,
                          size_t red_shm, int variant, cudaStream_t st);

}  // namespace lqcd
