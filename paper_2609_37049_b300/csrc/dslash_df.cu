// The defect correction's true residual r_p = b_p - (A_pp x_p - kappa H_p,1-p x_1-p) of one parity
// p, from the FP64 fields, in double-float arithmetic (pairs of floats, lqcd_common.cuh) on the
// FP32 pipe.  On B300 the FP64 pipe issues 1/64 of the FP32 rate, so this FP64-class arithmetic,
// about 20 FP32 operations per FP64 one, runs a few times faster than native FP64.
//
// Data: the neighbour parity x_1-p is split to double-float once per residual (split_field, into
// a scratch field of float4 = (re.hi, re.lo, im.hi, im.lo) per complex), so the eight hops that
// read each neighbour do not split it eight times; the links and the clover are split once per
// gauge field (split_field at upload).  x_p and b_p are split as they are read.
//
// Code size: one generic hop body runs the eight hops in a loop (direction, sign, spin
// projection, link or its adjoint chosen at run time by selects), so the kernel's instructions fit
// the instruction cache; a hop written out per direction, eight times, did not.
//
// Sums are carried unnormalised (hi, lo): each term is added with TwoSum on the high parts and
// its error plus low part folded into lo; products of two double-float numbers use TwoProduct
// (FMA).  The error of every output is a few units of 2^-46 of the sum of its terms' magnitudes.
#include "lqcd_internal.h"

namespace lqcd {
namespace {

struct acc2 {
  float hi, lo;
};

LQCD_D void add_to(acc2& s, dfl x) {
  const float t = s.hi + x.hi;
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (x.hi - bp);
  s.hi = t;
  s.lo += err + x.lo;
}

// s += a b
LQCD_D void mac(acc2& s, dfl a, dfl b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float t = s.hi + p;
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (p - bp);
  s.hi = t;
  s.lo += err + e;
}

LQCD_D dfl norm(acc2 s) { return df_quick(s.hi, s.lo); }

LQCD_D dfl neg_if(dfl a, bool n) { return n ? dfl(-a.hi, -a.lo) : a; }

struct cdf {
  dfl re, im;
};

// a i^k (k = 0..3)
LQCD_D cdf phase(cdf a, int k) {
  const bool sw = k & 1;
  const dfl r = sw ? a.im : a.re, i = sw ? a.re : a.im;
  return {neg_if(r, k == 1 || k == 2), neg_if(i, k >= 2)};
}

LQCD_D cdf ld4(const float4* f, long i) {
  const float4 v = __ldg(f + i);
  return {dfl(v.x, v.y), dfl(v.z, v.w)};
}

LQCD_D cdf ld_split(const double2* f, long i) {
  const double2 v = __ldg(f + i);
  return {split_d(v.x), split_d(v.y)};
}

// The float-to-double conversion by bit manipulation (exact for normal floats and zero; no FP64
// pipe work).
LQCD_D double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;  // zero, subnormal, inf, NaN: the exact conversion
  const unsigned hw = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  return __hiloint2double((int)hw, (int)((b & 0x7u) << 29));
}
// The stored residual: its high part.  The cancellation b - D x is what needs the double-float
// arithmetic; the result, once normalised, is r to 2^-24 of |r| (|lo| <= ulp(hi) / 2), far finer
// than its uses need (its norm against 1e-10 ||b||, and the FP32 right-hand side of the next inner
// solve).
LQCD_D double to_double(dfl a) { return f2d_bits(a.hi); }

struct ResDF {
  Geom g;
  const float4* xn;      // neighbour parity 1 - p, split: [12][Vh * nrhs]
  const double2* y;      // x_p
  const double2* z;      // b_p
  double2* out;          // r_p
  const float4* U;       // split links, layout of the FP64 links: [mu][par][9][Vh]
  const float4* A;       // split clover of parity p: [chir][18][Vh]
  const unsigned* coord;  // packed (x, y, z, t) of the sites of parity p
  const signed char* tc;  // forward t-hop coefficient per timeslice
  int out_par, nrhs;
  double mkappa;  // -kappa
};

// Spin projection (chiral basis) per direction: h_s = p_s + sgn ph_s p_{q_s} (s = 0, 1) and the
// reconstruction of the lower components l_L = sgn ps_L w_{r_L} (L = 2, 3), phases as powers of i.
__constant__ signed char kQ[4][2] = {{3, 2}, {3, 2}, {2, 3}, {2, 3}};
__constant__ signed char kPh[4][2] = {{3, 3}, {2, 0}, {3, 1}, {0, 0}};
__constant__ signed char kR[4][2] = {{1, 0}, {1, 0}, {0, 1}, {0, 1}};
__constant__ signed char kPs[4][2] = {{1, 1}, {0, 2}, {1, 3}, {0, 0}};

template <int MINB>
__global__ void __launch_bounds__(128, MINB) k_res_df(const ResDF pr) {
  const Geom& g = pr.g;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long cb = tid / pr.nrhs;
  const int rhs = (int)(tid - cb * pr.nrhs);
  if (cb >= g.Vh) return;
  const unsigned cw = __ldg(pr.coord + cb);
  const int cx = cw & 0xff, cy = (cw >> 8) & 0xff, cz = (cw >> 16) & 0xff, ct = cw >> 24;
  const long sy = g.Lx, sz = (long)g.Lx * g.Ly, st = sz * g.Lz;
  const long s = cx + sy * cy + sz * cz + st * ct;
  const long stride = g.Vh * pr.nrhs;
  const int op = pr.out_par, ip = 1 - pr.out_par;

  acc2 acc[12][2];
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k][0] = acc[k][1] = {0.f, 0.f};

#pragma unroll 1
  for (int hop = 0; hop < 8; hop++) {
    const int mu = hop >> 1;
    const bool fwd = (hop & 1) == 0;
    const int cm = mu == 0 ? cx : (mu == 1 ? cy : (mu == 2 ? cz : ct));
    const int Lm = mu == 0 ? g.Lx : (mu == 1 ? g.Ly : (mu == 2 ? g.Lz : g.Lt));
    const long sm = mu == 0 ? 1 : (mu == 1 ? sy : (mu == 2 ? sz : st));
    const int coef = mu < 3 ? 1 : (int)__ldg(pr.tc + (fwd ? ct : (ct == 0 ? g.Lt - 1 : ct - 1)));
    if (coef == 0) continue;
    const long sn = fwd ? s + (cm + 1 == Lm ? sm * (1 - Lm) : sm) : s + (cm == 0 ? sm * (Lm - 1) : -sm);
    const long nb = sn >> 1;
    const int sg2 = fwd ? 2 : 0;  // forward projector 1 - gamma_mu: sign -1 = i^2

    // projected half spinor of the neighbour
    cdf h[2][3];
    {
      cdf p[12];
#pragma unroll
      for (int k = 0; k < 12; k++) p[k] = ld4(pr.xn, (long)k * stride + nb * pr.nrhs + rhs);
#pragma unroll
      for (int sp = 0; sp < 2; sp++) {
        const int q = kQ[mu][sp], k = (kPh[mu][sp] + sg2) & 3;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const cdf t = phase(q == 2 ? p[6 + c] : p[9 + c], k);
          acc2 r = {p[3 * sp + c].re.hi, p[3 * sp + c].re.lo}, i = {p[3 * sp + c].im.hi, p[3 * sp + c].im.lo};
          add_to(r, t.re);
          add_to(i, t.im);
          h[sp][c] = {dfl(r.hi, r.lo), dfl(i.hi, i.lo)};
        }
      }
    }
    // M = coef U_mu(s) (forward) or coef U_mu(s - mu)^dag (backward)
    cdf M[3][3];
    {
      const float4* Uf = pr.U + ((long)(mu * 2 + (fwd ? op : ip)) * 9) * g.Vh + (fwd ? cb : nb);
      cdf u[3][3];
#pragma unroll
      for (int e = 0; e < 9; e++) u[e / 3][e % 3] = ld4(Uf, (long)e * g.Vh);
      const bool ng = coef < 0;
#pragma unroll
      for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
          const cdf v = fwd ? u[a][b] : u[b][a];
          M[a][b] = {neg_if(v.re, ng), neg_if(v.im, ng != !fwd)};
        }
    }
    // w = M h, then acc += (w ; sgn X^dag w)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cdf w[2];
#pragma unroll
      for (int sp = 0; sp < 2; sp++) {
        acc2 r = {0.f, 0.f}, i = {0.f, 0.f};
#pragma unroll
        for (int b = 0; b < 3; b++) {
          mac(r, M[a][b].re, h[sp][b].re);
          mac(r, -M[a][b].im, h[sp][b].im);
          mac(i, M[a][b].re, h[sp][b].im);
          mac(i, M[a][b].im, h[sp][b].re);
        }
        w[sp] = {norm(r), norm(i)};
        add_to(acc[3 * sp + a][0], w[sp].re);
        add_to(acc[3 * sp + a][1], w[sp].im);
      }
#pragma unroll
      for (int L = 0; L < 2; L++) {
        const cdf l = phase(kR[mu][L] == 0 ? w[0] : w[1], (kPs[mu][L] + sg2) & 3);
        add_to(acc[3 * (2 + L) + a][0], l.re);
        add_to(acc[3 * (2 + L) + a][1], l.im);
      }
    }
  }

  // epilogue: r = z - (A y - kappa acc), chirality by chirality (A is block diagonal)
  const long idx = cb * pr.nrhs + rhs;
  const dfl mk = dfl(pr.mkappa);
#pragma unroll 1
  for (int ch = 0; ch < 2; ch++) {
    cdf yv[6];
#pragma unroll
    for (int i = 0; i < 6; i++) yv[i] = ld_split(pr.y, (long)(6 * ch + i) * stride + idx);
    const float4* Af = pr.A + (long)ch * 18 * g.Vh + cb;
    acc2 o[6][2];
#pragma unroll
    for (int i = 0; i < 6; i++) {  // o = z - kappa acc
      const cdf zv = ld_split(pr.z, (long)(6 * ch + i) * stride + idx);
      o[i][0] = {zv.re.hi, zv.re.lo};
      o[i][1] = {zv.im.hi, zv.im.lo};
      // (selects, not a run-time index, keep acc in registers)
      const acc2 ar = ch == 0 ? acc[i][0] : acc[6 + i][0], ai = ch == 0 ? acc[i][1] : acc[6 + i][1];
      mac(o[i][0], -mk, norm(ar));
      mac(o[i][1], -mk, norm(ai));
    }
    // o -= A y, A packed Hermitian: diag r[0..5], upper (i < j) row-major at r[6 + 2k], r[7 + 2k]
    dfl r[36];
#pragma unroll
    for (int c = 0; c < 18; c++) {
      const float4 v = __ldg(Af + (long)c * g.Vh);
      r[2 * c] = dfl(v.x, v.y);
      r[2 * c + 1] = dfl(v.z, v.w);
    }
#pragma unroll
    for (int i = 0; i < 6; i++) {
      mac(o[i][0], -r[i], yv[i].re);
      mac(o[i][1], -r[i], yv[i].im);
    }
    int kk = 0;
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
      for (int j = i + 1; j < 6; j++) {
        const dfl cr = r[6 + 2 * kk], ci = r[7 + 2 * kk];
        // o_i -= c y_j ;  o_j -= conj(c) y_i
        mac(o[i][0], -cr, yv[j].re);
        mac(o[i][0], ci, yv[j].im);
        mac(o[i][1], -cr, yv[j].im);
        mac(o[i][1], -ci, yv[j].re);
        mac(o[j][0], -cr, yv[i].re);
        mac(o[j][0], -ci, yv[i].im);
        mac(o[j][1], -cr, yv[i].im);
        mac(o[j][1], ci, yv[i].re);
        kk++;
      }
#pragma unroll
    for (int i = 0; i < 6; i++)
      pr.out[(long)(6 * ch + i) * stride + idx] = make_double2(to_double(norm(o[i][0])), to_double(norm(o[i][1])));
  }
}

// ------------------------------------------------------------------ two right-hand sides per thread
// The same residual for the pair (r, r + 1) of a thread, every float of the double-float
// arithmetic a float2 (value for r, value for r + 1) on paired instructions (add.f32x2,
// mul.f32x2, fma.rn.f32x2): half the arithmetic instructions per right-hand side.  The neighbour
// parity is split into a pair layout: for right-hand sides 2q, 2q + 1 of a spinor entry, float4
// (re.hi_2q, re.hi_2q+1, re.lo_2q, re.lo_2q+1) then float4 (im ...), in the place of the two
// double2 entries.  Even nrhs only.
struct dp {  // double-float pair
  float2 hi, lo;
};
struct cp {
  dp re, im;
};

LQCD_D float2 F2(float a, float b) { return make_float2(a, b); }
LQCD_D float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
LQCD_D float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
LQCD_D float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }

LQCD_D void add_to2(dp& s, dp x) {
  const float2 t = add2(s.hi, x.hi);
  const float2 bp = sub2(t, s.hi);
  const float2 err = add2(sub2(s.hi, sub2(t, bp)), sub2(x.hi, bp));
  s.hi = t;
  s.lo = add2(s.lo, add2(err, x.lo));
}

// s += a b
LQCD_D void mac2(dp& s, dp a, dp b) {
  const float2 p = __fmul2_rn(a.hi, b.hi);
  float2 e = __ffma2_rn(a.hi, b.hi, neg2(p));
  e = __ffma2_rn(a.hi, b.lo, e);
  e = __ffma2_rn(a.lo, b.hi, e);
  const float2 t = add2(s.hi, p);
  const float2 bp = sub2(t, s.hi);
  const float2 err = add2(sub2(s.hi, sub2(t, bp)), sub2(p, bp));
  s.hi = t;
  s.lo = add2(s.lo, add2(err, e));
}

LQCD_D dp norm2p(dp s) {
  const float2 h = add2(s.hi, s.lo);
  return {h, sub2(s.lo, sub2(h, s.hi))};
}
LQCD_D dp neg_if2(dp a, bool n) { return n ? dp{neg2(a.hi), neg2(a.lo)} : a; }
LQCD_D dp bcast(dfl a) { return {F2(a.hi, a.hi), F2(a.lo, a.lo)}; }
LQCD_D dp pair_of(dfl a, dfl b) { return {F2(a.hi, b.hi), F2(a.lo, b.lo)}; }

// a i^k (k = 0..3)
LQCD_D cp phase2(cp a, int k) {
  const bool sw = k & 1;
  const dp r = sw ? a.im : a.re, i = sw ? a.re : a.im;
  return {neg_if2(r, k == 1 || k == 2), neg_if2(i, k >= 2)};
}

LQCD_D cp ld_pair(const float4* f, long i) {
  const float4 a = __ldg(f + i), b = __ldg(f + i + 1);
  return {{F2(a.x, a.y), F2(a.z, a.w)}, {F2(b.x, b.y), F2(b.z, b.w)}};
}

LQCD_D cp ld_split_pair(const double2* f, long i) {
  const double2 a = __ldg(f + i), b = __ldg(f + i + 1);
  return {pair_of(split_d(a.x), split_d(b.x)), pair_of(split_d(a.y), split_d(b.y))};
}

template <int MINB>
__global__ void __launch_bounds__(128, MINB) k_res_df2(const ResDF pr) {
  const Geom& g = pr.g;
  const int half = pr.nrhs >> 1;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long cb = tid / half;
  const int rhs0 = 2 * (int)(tid - cb * half);
  if (cb >= g.Vh) return;
  const unsigned cw = __ldg(pr.coord + cb);
  const int cx = cw & 0xff, cy = (cw >> 8) & 0xff, cz = (cw >> 16) & 0xff, ct = cw >> 24;
  const long sy = g.Lx, sz = (long)g.Lx * g.Ly, st = sz * g.Lz;
  const long s = cx + sy * cy + sz * cz + st * ct;
  const long stride = g.Vh * pr.nrhs;
  const int op = pr.out_par, ip = 1 - pr.out_par;

  dp acc[12][2];
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k][0] = acc[k][1] = {F2(0.f, 0.f), F2(0.f, 0.f)};

#pragma unroll 1
  for (int hop = 0; hop < 8; hop++) {
    const int mu = hop >> 1;
    const bool fwd = (hop & 1) == 0;
    const int cm = mu == 0 ? cx : (mu == 1 ? cy : (mu == 2 ? cz : ct));
    const int Lm = mu == 0 ? g.Lx : (mu == 1 ? g.Ly : (mu == 2 ? g.Lz : g.Lt));
    const long sm = mu == 0 ? 1 : (mu == 1 ? sy : (mu == 2 ? sz : st));
    const int coef = mu < 3 ? 1 : (int)__ldg(pr.tc + (fwd ? ct : (ct == 0 ? g.Lt - 1 : ct - 1)));
    if (coef == 0) continue;
    const long sn = fwd ? s + (cm + 1 == Lm ? sm * (1 - Lm) : sm) : s + (cm == 0 ? sm * (Lm - 1) : -sm);
    const long nb = sn >> 1;
    const int sg2 = fwd ? 2 : 0;  // forward projector 1 - gamma_mu: sign -1 = i^2

    cp h[2][3];
    {
      cp p[12];
#pragma unroll
      for (int k = 0; k < 12; k++) p[k] = ld_pair(pr.xn, (long)k * stride + nb * pr.nrhs + rhs0);
#pragma unroll
      for (int sp = 0; sp < 2; sp++) {
        const int q = kQ[mu][sp], k = (kPh[mu][sp] + sg2) & 3;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const cp t = phase2(q == 2 ? p[6 + c] : p[9 + c], k);
          dp r = p[3 * sp + c].re, i = p[3 * sp + c].im;
          add_to2(r, t.re);
          add_to2(i, t.im);
          h[sp][c] = {r, i};
        }
      }
    }
    cdf M[3][3];
    {
      const float4* Uf = pr.U + ((long)(mu * 2 + (fwd ? op : ip)) * 9) * g.Vh + (fwd ? cb : nb);
      cdf u[3][3];
#pragma unroll
      for (int e = 0; e < 9; e++) u[e / 3][e % 3] = ld4(Uf, (long)e * g.Vh);
      const bool ng = coef < 0;
#pragma unroll
      for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
          const cdf v = fwd ? u[a][b] : u[b][a];
          M[a][b] = {neg_if(v.re, ng), neg_if(v.im, ng != !fwd)};
        }
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cp w[2];
#pragma unroll
      for (int sp = 0; sp < 2; sp++) {
        dp r = {F2(0.f, 0.f), F2(0.f, 0.f)}, i = {F2(0.f, 0.f), F2(0.f, 0.f)};
#pragma unroll
        for (int b = 0; b < 3; b++) {
          const dp mr = bcast(M[a][b].re), mi = bcast(M[a][b].im), mmi = bcast(-M[a][b].im);
          mac2(r, mr, h[sp][b].re);
          mac2(r, mmi, h[sp][b].im);
          mac2(i, mr, h[sp][b].im);
          mac2(i, mi, h[sp][b].re);
        }
        w[sp] = {norm2p(r), norm2p(i)};
        add_to2(acc[3 * sp + a][0], w[sp].re);
        add_to2(acc[3 * sp + a][1], w[sp].im);
      }
#pragma unroll
      for (int L = 0; L < 2; L++) {
        const cp l = phase2(kR[mu][L] == 0 ? w[0] : w[1], (kPs[mu][L] + sg2) & 3);
        add_to2(acc[3 * (2 + L) + a][0], l.re);
        add_to2(acc[3 * (2 + L) + a][1], l.im);
      }
    }
  }

  const long idx = cb * pr.nrhs + rhs0;
  const dp kap = bcast(-dfl(pr.mkappa));  // kappa
#pragma unroll 1
  for (int ch = 0; ch < 2; ch++) {
    cp yv[6];
#pragma unroll
    for (int i = 0; i < 6; i++) yv[i] = ld_split_pair(pr.y, (long)(6 * ch + i) * stride + idx);
    const float4* Af = pr.A + (long)ch * 18 * g.Vh + cb;
    dp o[6][2];
#pragma unroll
    for (int i = 0; i < 6; i++) {  // o = z + kappa acc
      const cp zv = ld_split_pair(pr.z, (long)(6 * ch + i) * stride + idx);
      o[i][0] = zv.re;
      o[i][1] = zv.im;
      const dp ar = ch == 0 ? acc[i][0] : acc[6 + i][0], ai = ch == 0 ? acc[i][1] : acc[6 + i][1];
      mac2(o[i][0], kap, norm2p(ar));
      mac2(o[i][1], kap, norm2p(ai));
    }
    dfl r[36];
#pragma unroll
    for (int c = 0; c < 18; c++) {
      const float4 v = __ldg(Af + (long)c * g.Vh);
      r[2 * c] = dfl(v.x, v.y);
      r[2 * c + 1] = dfl(v.z, v.w);
    }
#pragma unroll
    for (int i = 0; i < 6; i++) {
      const dp mr = bcast(-r[i]);
      mac2(o[i][0], mr, yv[i].re);
      mac2(o[i][1], mr, yv[i].im);
    }
    int kk = 0;
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
      for (int j = i + 1; j < 6; j++) {
        const dp mcr = bcast(-r[6 + 2 * kk]), ci = bcast(r[7 + 2 * kk]), mci = bcast(-r[7 + 2 * kk]);
        // o_i -= c y_j ;  o_j -= conj(c) y_i
        mac2(o[i][0], mcr, yv[j].re);
        mac2(o[i][0], ci, yv[j].im);
        mac2(o[i][1], mcr, yv[j].im);
        mac2(o[i][1], mci, yv[j].re);
        mac2(o[j][0], mcr, yv[i].re);
        mac2(o[j][0], mci, yv[i].im);
        mac2(o[j][1], mcr, yv[i].im);
        mac2(o[j][1], ci, yv[i].re);
        kk++;
      }
#pragma unroll
    for (int i = 0; i < 6; i++) {
      const dp orr = norm2p(o[i][0]), oi = norm2p(o[i][1]);
      double2* dst = pr.out + (long)(6 * ch + i) * stride + idx;
      dst[0] = make_double2(f2d_bits(orr.hi.x), f2d_bits(oi.hi.x));
      dst[1] = make_double2(f2d_bits(orr.hi.y), f2d_bits(oi.hi.y));
    }
  }
}

// pairs of consecutive right-hand sides: n_pairs = (complex entries) / 2
__global__ void k_split_field_pairs(const double2* in, float4* out, long n_pairs) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n_pairs; i += (long)gridDim.x * blockDim.x) {
    const double2 a = in[2 * i], b = in[2 * i + 1];
    const dfl ar = split_d(a.x), ai = split_d(a.y), br = split_d(b.x), bi = split_d(b.y);
    out[2 * i] = make_float4(ar.hi, br.hi, ar.lo, br.lo);
    out[2 * i + 1] = make_float4(ai.hi, bi.hi, ai.lo, bi.lo);
  }
}

__global__ void k_split_field(const double2* in, float4* out, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    const dfl a = split_d(v.x), b = split_d(v.y);
    out[i] = make_float4(a.hi, a.lo, b.hi, b.lo);
  }
}

}  // namespace

void split_field(const void* in, void* out, long n_complex, cudaStream_t st) {
  k_split_field<<<148 * 8, 256, 0, st>>>((const double2*)in, (float4*)out, n_complex);
  count_launch();
}

void split_neighbours(const void* in, void* out, long n_complex, int nrhs, cudaStream_t st) {
  if (nrhs % 2 == 0)
    k_split_field_pairs<<<148 * 8, 256, 0, st>>>((const double2*)in, (float4*)out, n_complex / 2);
  else
    k_split_field<<<148 * 8, 256, 0, st>>>((const double2*)in, (float4*)out, n_complex);
  count_launch();
}

void launch_residual_df(const Geom& g, const void* xn_split, const void* y, const void* z, void* out, const void* U_split,
                        const void* A_split, const unsigned* coord, const signed char* tc, int out_par, int nrhs,
                        double kappa, int variant, cudaStream_t st) {
  ResDF pr;
  pr.g = g;
  pr.xn = (const float4*)xn_split;
  pr.y = (const double2*)y;
  pr.z = (const double2*)z;
  pr.out = (double2*)out;
  pr.U = (const float4*)U_split;
  pr.A = (const float4*)A_split;
  pr.coord = coord;
  pr.tc = tc;
  pr.out_par = out_par;
  pr.nrhs = nrhs;
  pr.mkappa = -kappa;
  if (nrhs % 2 == 0) {  // two right-hand sides per thread (xn_split in the pair layout)
    const long blocks = (g.Vh * (long)(nrhs / 2) + 127) / 128;
    if (variant == 1)  // register caps 168 / 128 / 255
      k_res_df2<3><<<blocks, 128, 0, st>>>(pr);
    else if (variant == 2)
      k_res_df2<4><<<blocks, 128, 0, st>>>(pr);
    else
      k_res_df2<2><<<blocks, 128, 0, st>>>(pr);
  } else {
    const long blocks = (g.Vh * (long)nrhs + 127) / 128;
    if (variant == 1)
      k_res_df<3><<<blocks, 128, 0, st>>>(pr);
    else if (variant == 2)
      k_res_df<4><<<blocks, 128, 0, st>>>(pr);
    else
      k_res_df<2><<<blocks, 128, 0, st>>>(pr);
  }
  count_launch();
}

}  // namespace lqcd
