// Gauge-field preparation on the GPU: clover field strength, the clover term A and its inverse
// (Sec. 3: Wilson-clover action), and the even-odd packed link copies in FP64 / FP32 / FP16.
//
//   Fhat_{mu nu}(x) = (Q_{mu nu} - Q_{mu nu}^dag) / 8,  Q = sum of the four plaquettes in the
//   (mu, nu) plane that start and end at x;   A = 1 + i kappa c_sw sum_{mu<nu} sigma_{mu nu} Fhat.
// In the chiral basis sigma_{mu nu} is block diagonal; with upper (lower) sign for spins 0,1
// (spins 2,3):
//   sigma_{xy} = -s_z, sigma_{xz} = s_y, sigma_{yz} = -s_x, sigma_{kt} = +-s_k   (s = Pauli),
// so each chirality block is the 6x6 Hermitian matrix 1 + i kappa c_sw sum_k s_k (x) G_k with
//   G_x = -F_yz +- F_xt,  G_y = F_xz +- F_yt,  G_z = -F_xy +- F_zt.
// A^{-1} per chirality block by Gauss-Jordan elimination with partial pivoting in FP64.
#include "lqcd_internal.h"

namespace lqcd {

using C64 = cplx<double>;

struct M3 {
  C64 m[3][3];
};

LQCD_D M3 mul(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) c.m[i][j] = a.m[i][0] * b.m[0][j] + a.m[i][1] * b.m[1][j] + a.m[i][2] * b.m[2][j];
  return c;
}
LQCD_D M3 dag(const M3& a) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) c.m[i][j] = cj(a.m[j][i]);
  return c;
}

struct LexLinks {
  const double2* u;  // [V][4][3][3]
  Geom g;
  LQCD_D M3 get(int x, int y, int z, int t, int mu) const {
    x = (x + g.Lx) % g.Lx;
    y = (y + g.Ly) % g.Ly;
    z = (z + g.Lz) % g.Lz;
    t = (t + g.Lt) % g.Lt;
    const double2* p = u + (lex_index(g, x, y, z, t) * 4 + mu) * 9;
    M3 r;
#pragma unroll
    for (int e = 0; e < 9; e++) {
      double2 v = p[e];
      r.m[e / 3][e % 3] = {v.x, v.y};
    }
    return r;
  }
};

// Q_{mu nu}(x): the four leaves, each a closed path from x in the (mu, nu) plane.
LQCD_D M3 leaves(const LexLinks& L, int c[4], int mu, int nu) {
  auto at = [&](int dm, int dn, int dir) {
    int d[4] = {c[0], c[1], c[2], c[3]};
    d[mu] += dm;
    d[nu] += dn;
    return L.get(d[0], d[1], d[2], d[3], dir);
  };
  M3 q;
  // x -> x+mu -> x+mu+nu -> x+nu -> x
  M3 l1 = mul(mul(at(0, 0, mu), at(1, 0, nu)), mul(dag(at(0, 1, mu)), dag(at(0, 0, nu))));
  // x -> x+nu -> x+nu-mu -> x-mu -> x
  M3 l2 = mul(mul(at(0, 0, nu), dag(at(-1, 1, mu))), mul(dag(at(-1, 0, nu)), at(-1, 0, mu)));
  // x -> x-mu -> x-mu-nu -> x-nu -> x
  M3 l3 = mul(mul(dag(at(-1, 0, mu)), dag(at(-1, -1, nu))), mul(at(-1, -1, mu), at(0, -1, nu)));
  // x -> x-nu -> x-nu+mu -> x+mu -> x
  M3 l4 = mul(mul(dag(at(0, -1, nu)), at(0, -1, mu)), mul(at(1, -1, nu), dag(at(0, 0, mu))));
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) q.m[i][j] = l1.m[i][j] + l2.m[i][j] + l3.m[i][j] + l4.m[i][j];
  return q;
}

LQCD_D void pack_herm(const C64 (&a)[6][6], double (&r)[36]) {
  for (int i = 0; i < 6; i++) r[i] = a[i][i].re;
  int k = 0;
  for (int i = 0; i < 6; i++)
    for (int j = i + 1; j < 6; j++) {
      // average with the mirrored element so the packed matrix is exactly Hermitian
      r[6 + 2 * k] = 0.5 * (a[i][j].re + a[j][i].re);
      r[7 + 2 * k] = 0.5 * (a[i][j].im - a[j][i].im);
      k++;
    }
}

// Gauss-Jordan inverse with partial pivoting; returns 0 on a (numerically) singular block.
LQCD_D int invert6(C64 (&a)[6][6], C64 (&inv)[6][6]) {
  for (int i = 0; i < 6; i++)
    for (int j = 0; j < 6; j++) inv[i][j] = {i == j ? 1.0 : 0.0, 0.0};
  for (int col = 0; col < 6; col++) {
    int piv = col;
    double best = norm2(a[col][col]);
    for (int r = col + 1; r < 6; r++) {
      double v = norm2(a[r][col]);
      if (v > best) {
        best = v;
        piv = r;
      }
    }
    if (!(best > 1e-300)) return 0;
    if (piv != col) {
      for (int j = 0; j < 6; j++) {
        C64 t = a[col][j];
        a[col][j] = a[piv][j];
        a[piv][j] = t;
        t = inv[col][j];
        inv[col][j] = inv[piv][j];
        inv[piv][j] = t;
      }
    }
    C64 d = a[col][col];
    double dn = norm2(d);
    C64 di = {d.re / dn, -d.im / dn};
    for (int j = 0; j < 6; j++) {
      a[col][j] = a[col][j] * di;
      inv[col][j] = inv[col][j] * di;
    }
    for (int r = 0; r < 6; r++) {
      if (r == col) continue;
      C64 f = a[r][col];
      for (int j = 0; j < 6; j++) {
        a[r][j] = a[r][j] - f * a[col][j];
        inv[r][j] = inv[r][j] - f * inv[col][j];
      }
    }
  }
  return 1;
}

// P64 layout [p][chir][18 double2][Vh]
LQCD_D void store_c64(double2* base, const Geom& g, int p, int chir, long cb, const double (&r)[36]) {
  double2* f = base + ((long)(p * 2 + chir) * 18) * g.Vh + cb;
  for (int c = 0; c < 18; c++) f[c * g.Vh] = make_double2(r[2 * c], r[2 * c + 1]);
}
LQCD_D void store_c32(float4* base, const Geom& g, int p, int chir, long cb, const double (&r)[36]) {
  float4* f = base + ((long)(p * 2 + chir) * 9) * g.Vh + cb;
  for (int c = 0; c < 9; c++)
    f[c * g.Vh] = make_float4((float)r[4 * c], (float)r[4 * c + 1], (float)r[4 * c + 2], (float)r[4 * c + 3]);
}
LQCD_D void store_c16(uint2* base, const Geom& g, int p, int chir, long cb, const double (&r)[36]) {
  uint2* f = base + ((long)(p * 2 + chir) * 9) * g.Vh + cb;
  for (int c = 0; c < 9; c++) {
    uint2 v;
    v.x = f2h((float)r[4 * c], (float)r[4 * c + 1]);
    v.y = f2h((float)r[4 * c + 2], (float)r[4 * c + 3]);
    f[c * g.Vh] = v;
  }
}

__global__ void k_clover_build(const double2* links, Geom g, double kappa, double csw, double2* A64,
                               double2* Ainv64, float4* A32, float4* Ainv32, uint2* Ainv16, int* bad) {
  long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long V = 2 * g.Vh;
  if (s >= V) return;
  int c[4];
  c[0] = (int)(s % g.Lx);
  c[1] = (int)((s / g.Lx) % g.Ly);
  c[2] = (int)((s / ((long)g.Lx * g.Ly)) % g.Lz);
  c[3] = (int)(s / ((long)g.Lx * g.Ly * g.Lz));
  const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
  const long cb = s >> 1;
  LexLinks L{links, g};
  // F for the planes (x,y),(x,z),(x,t),(y,z),(y,t),(z,t)
  const int pm[6] = {0, 0, 0, 1, 1, 2}, pn[6] = {1, 2, 3, 2, 3, 3};
  M3 F[6];
  for (int k = 0; k < 6; k++) {
    M3 q = leaves(L, c, pm[k], pn[k]);
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) F[k].m[i][j] = 0.125 * (q.m[i][j] - cj(q.m[j][i]));
  }
  const double kc = kappa * csw;
  for (int chir = 0; chir < 2; chir++) {
    const double sg = chir == 0 ? 1.0 : -1.0;
    M3 Gx, Gy, Gz;
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) {
        Gx.m[i][j] = sg * F[2].m[i][j] - F[3].m[i][j];
        Gy.m[i][j] = F[1].m[i][j] + sg * F[4].m[i][j];
        Gz.m[i][j] = sg * F[5].m[i][j] - F[0].m[i][j];
      }
    // block (s, s') of 1 + i kc sum_k sigma_k G_k:
    //  (0,0) = 1 + i kc Gz, (1,1) = 1 - i kc Gz, (0,1) = i kc (Gx - i Gy), (1,0) = i kc (Gx + i Gy)
    C64 a[6][6];
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) {
        C64 gz = Gz.m[i][j], gx = Gx.m[i][j], gy = Gy.m[i][j];
        C64 d = (i == j) ? C64{1.0, 0.0} : C64{0.0, 0.0};
        a[i][j] = d + kc * times_i(gz);
        a[3 + i][3 + j] = d - kc * times_i(gz);
        a[i][3 + j] = kc * times_i(gx - times_i(gy));
        a[3 + i][j] = kc * times_i(gx + times_i(gy));
      }
    double r[36];
    pack_herm(a, r);
    store_c64(A64, g, p, chir, cb, r);
    store_c32(A32, g, p, chir, cb, r);
    C64 inv[6][6];
    if (!invert6(a, inv)) atomicExch(bad, 1);
    pack_herm(inv, r);
    store_c64(Ainv64, g, p, chir, cb, r);
    store_c32(Ainv32, g, p, chir, cb, r);
    store_c16(Ainv16, g, p, chir, cb, r);
  }
}

// Even-odd packed link copies.
__global__ void k_pack_links(const double2* links, Geom g, double2* U64, float4* U32, uint2* U16) {
  long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long V = 2 * g.Vh;
  if (s >= V) return;
  int x = (int)(s % g.Lx), y = (int)((s / g.Lx) % g.Ly), z = (int)((s / ((long)g.Lx * g.Ly)) % g.Lz),
      t = (int)(s / ((long)g.Lx * g.Ly * g.Lz));
  const int p = (x + y + z + t) & 1;
  const long cb = s >> 1;
  for (int mu = 0; mu < 4; mu++) {
    const double2* u = links + (s * 4 + mu) * 9;
    double2* d = U64 + ((long)(mu * 2 + p) * 9) * g.Vh + cb;
    for (int e = 0; e < 9; e++) d[e * g.Vh] = u[e];
    float4* f = U32 + ((long)(mu * 2 + p) * 3) * g.Vh + cb;
    f[0] = make_float4((float)u[0].x, (float)u[0].y, (float)u[1].x, (float)u[1].y);
    f[g.Vh] = make_float4((float)u[2].x, (float)u[2].y, (float)u[3].x, (float)u[3].y);
    f[2 * g.Vh] = make_float4((float)u[4].x, (float)u[4].y, (float)u[5].x, (float)u[5].y);
    uint2* h = U16 + ((long)(mu * 2 + p) * 3) * g.Vh + cb;
    h[0] = make_uint2(f2h((float)u[0].x, (float)u[0].y), f2h((float)u[1].x, (float)u[1].y));
    h[g.Vh] = make_uint2(f2h((float)u[2].x, (float)u[2].y), f2h((float)u[3].x, (float)u[3].y));
    h[2 * g.Vh] = make_uint2(f2h((float)u[4].x, (float)u[4].y), f2h((float)u[5].x, (float)u[5].y));
  }
}

void build_gauge(lqcd_ctx* c, const double2* links_dev, int* bad_dev) {
  const Geom& g = c->g;
  long V = 2 * g.Vh;
  int tpb = 128;
  long blocks = (V + tpb - 1) / tpb;
  k_pack_links<<<blocks, tpb, 0, c->work>>>(links_dev, g, (double2*)c->U64, (float4*)c->U32, (uint2*)c->U16); lqcd::count_launch();
  k_clover_build<<<(V + 63) / 64, 64, 0, c->work>>>(links_dev, g, c->kappa, c->csw, (double2*)c->A64,
                                                    (double2*)c->Ainv64, (float4*)c->A32, (float4*)c->Ainv32,
                                                    (uint2*)c->Ainv16, bad_dev); lqcd::count_launch();
}

}  // namespace lqcd
