// Launch variant 7 of the even-odd dslash (FP32 storage): two right-hand sides per thread.
//
// Every arithmetic step of a hop is the same for all right-hand sides of a site (same links, same
// spin projection, same phases), so a thread that holds the pair (r, r + 1) carries each real
// quantity as a float2 (value for r, value for r + 1) and does the SU(3) products, the spin
// reconstruction and the clover block on paired instructions (fma.rn.f32x2 / add.f32x2 /
// mul.f32x2: two lanes per instruction), with every link and clover entry read once from shared
// memory for both.  Links are staged once per site as 9 float4 (re, re, im, im), the clover as 21
// float4 per chirality (diagonal (d, d, 0, 0), upper entries (re, re, im, im)), so an entry read
// is already the broadcast pair.  Only the spin projection (inputs as loaded, per right-hand side)
// and the final stores run per right-hand side.
//
// Blocks: the sites and right-hand sides of the variant-3 launch with half the threads:
// blockDim = S * nrhs / 2 for S sites (128 / nrhs sites, or the fused reductions' red_sites),
// thread = (site_local, pair p), right-hand sides 2p and 2p + 1.  Dynamic shared memory:
// [fused-reduction scratch | links S x 8 x 9 | clover S x 2 x 21] (float4).  The fused reductions
// keep the variant-3 layout of partial sums per (block, right-hand side).
#include "dslash_ops.cuh"

namespace lqcd {
namespace {

struct pcplx {  // a complex number for the two right-hand sides: re = (re_r, re_r+1), im likewise
  float2 re, im;
};

LQCD_D float2 f2(float a, float b) { return make_float2(a, b); }
LQCD_D float2 fneg2(float2 a) { return make_float2(-a.x, -a.y); }
LQCD_D float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
LQCD_D float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
LQCD_D float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// s * a for a power of i: s i^k (k = 0..3), lane-wise
LQCD_D pcplx times_ik(pcplx a, int k) {
  if (k == 0) return a;
  if (k == 1) return {fneg2(a.im), a.re};
  if (k == 2) return {fneg2(a.re), fneg2(a.im)};
  return {a.im, fneg2(a.re)};
}

// Staged link of one hop: 9 float4 (re, re, im, im) row-major.  w = U h (DAG: U^dag h) for the
// two spins s of the projected half spinor h[s][b].
template <bool DAG>
LQCD_D void su3_rb2(const float4* L, const pcplx (&h)[2][3], pcplx (&w)[2][3]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const float4 u = L[DAG ? b * 3 + a : a * 3 + b];
      const float2 ur = f2(u.x, u.y), ui = f2(u.z, u.w), mui = f2(-u.z, -u.w);
#pragma unroll
      for (int s = 0; s < 2; s++) {
        if (b == 0) {
          w[s][a].re = fmul2(ur, h[s][0].re);
          w[s][a].im = fmul2(ur, h[s][0].im);
        } else {
          w[s][a].re = ffma2(ur, h[s][b].re, w[s][a].re);
          w[s][a].im = ffma2(ur, h[s][b].im, w[s][a].im);
        }
        w[s][a].re = ffma2(DAG ? ui : mui, h[s][b].im, w[s][a].re);  // U h: - Im u Im h; U^dag h: + Im u Im h
        w[s][a].im = ffma2(DAG ? mui : ui, h[s][b].re, w[s][a].im);  // U h: + Im u Re h; U^dag h: - Im u Re h
      }
    }
  }
}

// One hop along MU (FWD: U_mu(s) x(s + mu), else U_mu(s - mu)^dag x(s - mu)) for the pair,
// accumulated into acc[12] (spin-colour components).
template <int MU, bool FWD>
LQCD_D void hop_rb2(const DslashParams& pr, int nb_idx, int coef, int stride, const float4* L, pcplx (&acc)[12]) {
  constexpr int S = FWD ? -1 : 1;  // H (not H^dag): forward projector 1 - gamma_mu
  cplx<float> h0[2][3], h1[2][3];
  {
    cplx<float> p[12];
    const float4* f = reinterpret_cast<const float4*>(pr.in) + nb_idx;
#pragma unroll
    for (int c = 0; c < 6; c++) {
      const float4 v = __ldg(f + c * stride);
      p[2 * c] = {v.x, v.y};
      p[2 * c + 1] = {v.z, v.w};
    }
    project<MU, S>(p, h0);
#pragma unroll
    for (int c = 0; c < 6; c++) {
      const float4 v = __ldg(f + c * stride + 1);
      p[2 * c] = {v.x, v.y};
      p[2 * c + 1] = {v.z, v.w};
    }
    project<MU, S>(p, h1);
  }
  pcplx h[2][3], w[2][3];
#pragma unroll
  for (int s = 0; s < 2; s++)
#pragma unroll
    for (int c = 0; c < 3; c++) h[s][c] = {f2(h0[s][c].re, h1[s][c].re), f2(h0[s][c].im, h1[s][c].im)};
  su3_rb2<!FWD>(L, h, w);
  if (coef < 0) {
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
      for (int c = 0; c < 3; c++) w[s][c] = {fneg2(w[s][c].re), fneg2(w[s][c].im)};
  }
  // acc += [ w ; S X^dag w ]: upper spins take w, lower spins a phase times one of its spins
  constexpr int r2 = MU == 0 || MU == 1 ? 1 : 0;              // source spin of lower component 2
  constexpr int k2 = (MU == 0 ? 1 : MU == 1 ? 0 : MU == 2 ? 1 : 0) + (S < 0 ? 2 : 0);
  constexpr int k3 = (MU == 0 ? 1 : MU == 1 ? 2 : MU == 2 ? 3 : 0) + (S < 0 ? 2 : 0);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    acc[c] = {fadd2(acc[c].re, w[0][c].re), fadd2(acc[c].im, w[0][c].im)};
    acc[3 + c] = {fadd2(acc[3 + c].re, w[1][c].re), fadd2(acc[3 + c].im, w[1][c].im)};
    const pcplx l2 = times_ik(w[r2][c], k2 & 3), l3 = times_ik(w[1 - r2][c], k3 & 3);
    acc[6 + c] = {fadd2(acc[6 + c].re, l2.re), fadd2(acc[6 + c].im, l2.im)};
    acc[9 + c] = {fadd2(acc[9 + c].re, l3.re), fadd2(acc[9 + c].im, l3.im)};
  }
}

template <int MU>
LQCD_D void hop_dir_rb2(const DslashParams& pr, int s, int cmu, int Lmu, int smu, int coef_f, int coef_b, int rhs0,
                        int stride, int nrhs, const float4* lf, const float4* lb, pcplx (&acc)[12]) {
  if (coef_f != 0) {
    const int sn = s + ((cmu + 1 == Lmu) ? smu * (1 - Lmu) : smu);
    hop_rb2<MU, true>(pr, (sn >> 1) * nrhs + rhs0, coef_f, stride, lf, acc);
  }
  if (coef_b != 0) {
    const int sn = s + ((cmu == 0) ? smu * (Lmu - 1) : -smu);
    hop_rb2<MU, false>(pr, (sn >> 1) * nrhs + rhs0, coef_b, stride, lb, acc);
  }
}

// y = A x for one chirality's packed Hermitian 6x6 block staged as 21 float4 (6 diagonal
// (d, d, 0, 0), then the upper entries (re, re, im, im) row-major), on the pair.
LQCD_D void clover_rb2(const float4* C, const pcplx* x, pcplx* y) {
#pragma unroll
  for (int i = 0; i < 6; i++) {
    const float4 d = C[i];
    y[i] = {fmul2(f2(d.x, d.y), x[i].re), fmul2(f2(d.x, d.y), x[i].im)};
  }
  int k = 6;
#pragma unroll
  for (int i = 0; i < 6; i++) {
#pragma unroll
    for (int j = i + 1; j < 6; j++) {
      const float4 c = C[k++];
      const float2 cr = f2(c.x, c.y), ci = f2(c.z, c.w), mci = f2(-c.z, -c.w);
      // y_i += c x_j ; y_j += conj(c) x_i
      y[i].re = ffma2(cr, x[j].re, y[i].re);
      y[i].re = ffma2(mci, x[j].im, y[i].re);
      y[i].im = ffma2(cr, x[j].im, y[i].im);
      y[i].im = ffma2(ci, x[j].re, y[i].im);
      y[j].re = ffma2(cr, x[i].re, y[j].re);
      y[j].re = ffma2(ci, x[i].im, y[j].re);
      y[j].im = ffma2(cr, x[i].im, y[j].im);
      y[j].im = ffma2(mci, x[i].re, y[j].im);
    }
  }
}

LQCD_D void clover_both_rb2(const float4* C, pcplx (&s)[12]) {
#pragma unroll
  for (int ch = 0; ch < 2; ch++) {
    pcplx y[6];
    clover_rb2(C + ch * 21, &s[6 * ch], y);
#pragma unroll
    for (int i = 0; i < 6; i++) s[6 * ch + i] = y[i];
  }
}

LQCD_D void load_pair(const void* base, int stride, int idx, pcplx (&s)[12]) {
  const float4* f = reinterpret_cast<const float4*>(base) + idx;
#pragma unroll
  for (int c = 0; c < 6; c++) {
    const float4 a = __ldg(f + c * stride), b = __ldg(f + c * stride + 1);
    s[2 * c] = {f2(a.x, b.x), f2(a.y, b.y)};
    s[2 * c + 1] = {f2(a.z, b.z), f2(a.w, b.w)};
  }
}

LQCD_D void store_pair(void* base, int stride, int idx, const pcplx (&s)[12]) {
  float4* f = reinterpret_cast<float4*>(base) + idx;
#pragma unroll
  for (int c = 0; c < 6; c++) {
    f[c * stride] = make_float4(s[2 * c].re.x, s[2 * c].im.x, s[2 * c + 1].re.x, s[2 * c + 1].im.x);
    f[c * stride + 1] = make_float4(s[2 * c].re.y, s[2 * c].im.y, s[2 * c + 1].re.y, s[2 * c + 1].im.y);
  }
}

// Partial sums of ND values per right-hand side over the block's S sites, written as
// partial[block][rhs][ND] (the variant-3 layout); v[r][k]: value k of right-hand side rhs0 + r.
// Scratch: ND * S * nrhs doubles at the start of dynamic shared memory.
template <int ND>
LQCD_D void block_reduce_rb2(const double (&v)[2][ND], double* partial, int S, int nrhs, int site_local, int rhs0) {
  extern __shared__ double sm_rb2[];
  const int n = S * nrhs;
  const int col = site_local * nrhs + rhs0;
#pragma unroll
  for (int k = 0; k < ND; k++) {
    sm_rb2[k * n + col] = v[0][k];
    sm_rb2[k * n + col + 1] = v[1][k];
  }
  __syncthreads();
  for (int s = S / 2; s >= 1; s >>= 1) {
    if (site_local < s) {
#pragma unroll
      for (int k = 0; k < ND; k++) {
        sm_rb2[k * n + col] += sm_rb2[k * n + col + s * nrhs];
        sm_rb2[k * n + col + 1] += sm_rb2[k * n + col + 1 + s * nrhs];
      }
    }
    __syncthreads();
  }
  if (site_local == 0) {
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
      for (int k = 0; k < ND; k++)
        partial[((long)blockIdx.x * nrhs + rhs0 + r) * ND + k] = sm_rb2[k * n + col + r];
  }
}

template <int EPI, int RED, int MINB>
__global__ void __launch_bounds__(128, MINB) dslash_rb2_kernel(const DslashParams pr) {
  extern __shared__ __align__(16) unsigned char dsm_rb2[];
  const Geom& g = pr.g;
  const int nr = pr.nrhs;
  const int half = nr >> 1;
  const int lgh = __ffs(half) - 1;
  const int S = blockDim.x >> lgh;  // sites of this block
  float4 (*slink)[8][9] = reinterpret_cast<float4 (*)[8][9]>(dsm_rb2 + pr.pipe_off);
  float4 (*sclov)[42] = reinterpret_cast<float4 (*)[42]>(slink + S);
  const int cb0 = blockIdx.x * S;
  const int Vh = (int)g.Vh;
  const int sy = g.Lx, sz = g.Lx * g.Ly, sw = sz * g.Lz;
  for (int j = threadIdx.x; j < 10 * S; j += blockDim.x) {
    if (j < 8 * S) {  // link j & 7 of site j >> 3, third row rebuilt once
      const int site = j >> 3, k = j & 7, c = cb0 + site;
      const int mu = k >> 1;
      int lcb = c, par = pr.out_par;
      if (k & 1) {  // backward hop: the link of the neighbour s - mu
        const int xh = c % g.Lxh, yzt = c / g.Lxh, y = yzt % g.Ly, zt = yzt / g.Ly, z = zt % g.Lz, t = zt / g.Lz;
        const int x = 2 * xh + ((pr.out_par + y + z + t) & 1);
        const int s = x + sy * y + sz * z + sw * t;
        const int cm = mu == 0 ? x : (mu == 1 ? y : (mu == 2 ? z : t));
        const int Lm = mu == 0 ? g.Lx : (mu == 1 ? g.Ly : (mu == 2 ? g.Lz : g.Lt));
        const int sm = mu == 0 ? 1 : (mu == 1 ? sy : (mu == 2 ? sz : sw));
        lcb = (s + (cm == 0 ? sm * (Lm - 1) : -sm)) >> 1;
        par = 1 - pr.out_par;
      }
      cplx<float> u[3][3];
      load_link<P32>(pr.U, g.Vh, mu, par, lcb, u);
      float4* L = slink[site][k];
#pragma unroll
      for (int e = 0; e < 9; e++) {
        const cplx<float> v = u[e / 3][e % 3];
        L[e] = make_float4(v.re, v.re, v.im, v.im);
      }
    } else {  // clover chirality ch of site q >> 1: 36 reals -> 21 broadcast pairs
      const int q = j - 8 * S, site = q >> 1, ch = q & 1, c = cb0 + site;
      float r[36];
#pragma unroll
      for (int e = 0; e < 9; e++) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(pr.C) + (long)(ch * 9 + e) * Vh + c);
        r[4 * e] = v.x;
        r[4 * e + 1] = v.y;
        r[4 * e + 2] = v.z;
        r[4 * e + 3] = v.w;
      }
      float4* C = sclov[site] + ch * 21;
#pragma unroll
      for (int i = 0; i < 6; i++) C[i] = make_float4(r[i], r[i], 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 15; k++) C[6 + k] = make_float4(r[6 + 2 * k], r[6 + 2 * k], r[7 + 2 * k], r[7 + 2 * k]);
    }
  }
  const int sl = threadIdx.x >> lgh;
  const int rhs0 = 2 * (threadIdx.x & (half - 1));
  const int cb = cb0 + sl;
  const unsigned cw = __ldg(pr.coord + cb);  // issued before the barrier
  __syncthreads();

  const int x = cw & 0xff, y = (cw >> 8) & 0xff, z = (cw >> 16) & 0xff, t = cw >> 24;
  const int s = x + sy * y + sz * z + sw * t;
  const int stride = Vh * nr;
  pcplx acc[12];
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = {f2(0.f, 0.f), f2(0.f, 0.f)};
  hop_dir_rb2<0>(pr, s, x, g.Lx, 1, 1, 1, rhs0, stride, nr, slink[sl][0], slink[sl][1], acc);
  hop_dir_rb2<1>(pr, s, y, g.Ly, sy, 1, 1, rhs0, stride, nr, slink[sl][2], slink[sl][3], acc);
  hop_dir_rb2<2>(pr, s, z, g.Lz, sz, 1, 1, rhs0, stride, nr, slink[sl][4], slink[sl][5], acc);
  const int cf = __ldg(pr.tc + t), cbk = __ldg(pr.tc + (t == 0 ? g.Lt - 1 : t - 1));
  hop_dir_rb2<3>(pr, s, t, g.Lt, sw, cf, cbk, rhs0, stride, nr, slink[sl][6], slink[sl][7], acc);

  // epilogue (EPI_CH, EPI_Y_CH, EPI_C_YH), then the fused reductions of the second Schur half
  const int idx = cb * nr + rhs0;
  const float2 a2 = f2((float)pr.a, (float)pr.a), b2 = f2((float)pr.b, (float)pr.b);
  pcplx o[12], yv[12];
  if constexpr (EPI == EPI_CH) {
    clover_both_rb2(sclov[sl], acc);
#pragma unroll
    for (int k = 0; k < 12; k++) o[k] = {fmul2(b2, acc[k].re), fmul2(b2, acc[k].im)};
  } else if constexpr (EPI == EPI_Y_CH) {
    clover_both_rb2(sclov[sl], acc);
    load_pair(pr.y, stride, idx, yv);
#pragma unroll
    for (int k = 0; k < 12; k++)
      o[k] = {ffma2(b2, acc[k].re, fmul2(a2, yv[k].re)), ffma2(b2, acc[k].im, fmul2(a2, yv[k].im))};
  } else {  // EPI_C_YH
    load_pair(pr.y, stride, idx, yv);
#pragma unroll
    for (int k = 0; k < 12; k++)
      o[k] = {ffma2(b2, acc[k].re, fmul2(a2, yv[k].re)), ffma2(b2, acc[k].im, fmul2(a2, yv[k].im))};
    clover_both_rb2(sclov[sl], o);
  }
  store_pair(pr.out, stride, idx, o);

  if constexpr (RED == RED_DOT_Z) {  // (z, out)
    pcplx zv[12];
    load_pair(pr.zred, stride, idx, zv);
    double v[2][2];
#pragma unroll
    for (int r = 0; r < 2; r++) {
      float dr = 0.f, di = 0.f;
#pragma unroll
      for (int k = 0; k < 12; k++) {
        const float zr = r ? zv[k].re.y : zv[k].re.x, zi = r ? zv[k].im.y : zv[k].im.x;
        const float orr = r ? o[k].re.y : o[k].re.x, oi = r ? o[k].im.y : o[k].im.x;
        dr = fmaf(zr, orr, fmaf(zi, oi, dr));  // conj(z) o
        di = fmaf(zr, oi, fmaf(-zi, orr, di));
      }
      v[r][0] = dr;
      v[r][1] = di;
    }
    block_reduce_rb2<2>(v, pr.partial, S, nr, sl, rhs0);
  } else if constexpr (RED == RED_TS_R0) {  // (out, y), (out, out), (z, out), (z, y), (y, y)
    pcplx zv[12];
    load_pair(pr.zred, stride, idx, zv);
    double v[2][8];
#pragma unroll
    for (int r = 0; r < 2; r++) {
      float tyr = 0.f, tyi = 0.f, oo = 0.f, zor = 0.f, zoi = 0.f, zyr = 0.f, zyi = 0.f, yy = 0.f;
#pragma unroll
      for (int k = 0; k < 12; k++) {
        const float orr = r ? o[k].re.y : o[k].re.x, oi = r ? o[k].im.y : o[k].im.x;
        const float yr = r ? yv[k].re.y : yv[k].re.x, yi = r ? yv[k].im.y : yv[k].im.x;
        const float zr = r ? zv[k].re.y : zv[k].re.x, zi = r ? zv[k].im.y : zv[k].im.x;
        tyr = fmaf(orr, yr, fmaf(oi, yi, tyr));  // conj(o) y
        tyi = fmaf(orr, yi, fmaf(-oi, yr, tyi));
        oo = fmaf(orr, orr, fmaf(oi, oi, oo));
        zor = fmaf(zr, orr, fmaf(zi, oi, zor));  // conj(z) o
        zoi = fmaf(zr, oi, fmaf(-zi, orr, zoi));
        zyr = fmaf(zr, yr, fmaf(zi, yi, zyr));  // conj(z) y
        zyi = fmaf(zr, yi, fmaf(-zi, yr, zyi));
        yy = fmaf(yr, yr, fmaf(yi, yi, yy));
      }
      v[r][0] = tyr; v[r][1] = tyi; v[r][2] = oo; v[r][3] = zor;
      v[r][4] = zoi; v[r][5] = zyr; v[r][6] = zyi; v[r][7] = yy;
    }
    block_reduce_rb2<8>(v, pr.partial, S, nr, sl, rhs0);
  } else if constexpr (RED == RED_DOT_Y_NORM) {  // (out, y), (out, out)
    double v[2][3];
#pragma unroll
    for (int r = 0; r < 2; r++) {
      float dr = 0.f, di = 0.f, nn = 0.f;
#pragma unroll
      for (int k = 0; k < 12; k++) {
        const float orr = r ? o[k].re.y : o[k].re.x, oi = r ? o[k].im.y : o[k].im.x;
        const float yr = r ? yv[k].re.y : yv[k].re.x, yi = r ? yv[k].im.y : yv[k].im.x;
        dr = fmaf(orr, yr, fmaf(oi, yi, dr));
        di = fmaf(orr, yi, fmaf(-oi, yr, di));
        nn = fmaf(orr, orr, fmaf(oi, oi, nn));
      }
      v[r][0] = dr; v[r][1] = di; v[r][2] = nn;
    }
    block_reduce_rb2<3>(v, pr.partial, S, nr, sl, rhs0);
  }
}

template <int EPI, int RED>
void launch_rb2_k(const DslashParams& pr, long blocks, int tpb, size_t red_shm, cudaStream_t st) {
  DslashParams q = pr;
  q.pipe_off = (int)((red_shm + 15) / 16 * 16);
  const int S = tpb / pr.nrhs;
  const size_t shm = q.pipe_off + (size_t)S * (72 + 42) * sizeof(float4);
  dslash_rb2_kernel<EPI, RED, 4><<<blocks, tpb / 2, shm, st>>>(q);
  count_launch();
}

}  // namespace

// Variant 7 for the launch (blocks, tpb) of variant 3; false where it does not apply (FP32 only,
// nrhs a power of two in [16, 128], the epilogues of the Schur operator and its reconstruction).
bool launch_dslash_rb2(const DslashParams& pr, int epi, int red, long blocks, int tpb, size_t red_shm,
                       cudaStream_t st) {
  const int nr = pr.nrhs;
  if (nr < 16 || nr > 128 || (nr & (nr - 1)) != 0 || tpb % nr != 0 || tpb > 128) return false;
  if (red_shm > (size_t)8 * 128 * sizeof(double)) return false;
  if (red == RED_TS_R0) {
    if (epi != EPI_Y_CH) return false;
    launch_rb2_k<EPI_Y_CH, RED_TS_R0>(pr, blocks, tpb, red_shm, st);
  } else if (red == RED_DOT_Z) {
    if (epi != EPI_Y_CH) return false;
    launch_rb2_k<EPI_Y_CH, RED_DOT_Z>(pr, blocks, tpb, red_shm, st);
  } else if (red == RED_DOT_Y_NORM) {
    if (epi != EPI_Y_CH) return false;
    launch_rb2_k<EPI_Y_CH, RED_DOT_Y_NORM>(pr, blocks, tpb, red_shm, st);
  } else if (epi == EPI_CH) {
    launch_rb2_k<EPI_CH, RED_NONE>(pr, blocks, tpb, red_shm, st);
  } else if (epi == EPI_Y_CH) {
    launch_rb2_k<EPI_Y_CH, RED_NONE>(pr, blocks, tpb, red_shm, st);
  } else if (epi == EPI_C_YH) {
    launch_rb2_k<EPI_C_YH, RED_NONE>(pr, blocks, tpb, red_shm, st);
  } else {
    return false;
  }
  return true;
}

}  // namespace lqcd
