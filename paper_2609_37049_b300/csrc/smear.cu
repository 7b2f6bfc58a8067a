// APE smearing of the spatial links, in FP64 (the distillation vectors of Sec. 3.1 are computed on
// APE-smeared links; the paper takes the smearing parameters from elsewhere, so the weight alpha
// and the number of steps are inputs):
//
//   X_k(x)  = (1 - alpha) U_k(x) + (alpha / 4) sum_{j spatial, j != k} [ U_j(x) U_k(x+j) U_j(x+k)^dag
//                                                       + U_j(x-j)^dag U_k(x-j) U_j(x-j+k) ]
//   U'_k(x) = P(X_k(x)),  k = x, y, z,  every link of a step from the previous step's field;
//
// P(X) = W / det(W)^(1/3) with W = X (X^dag X)^(-1/2) the unitary polar factor and the principal
// cube root.  W comes from the scaled Newton iteration W <- (g W + (g W)^-dag) / 2,
// g = (|W^-1|_F / |W|_F)^(1/2) (Higham), which converges quadratically to the polar factor of a
// non-singular matrix; it stops when no entry moves by more than 1e-14 or after 50 steps.
// One thread per (site, spatial direction).  The smeared field lives in the context, in the
// FP64 link layout [mu][parity][9][Vh] for mu < 3, and the Laplacian eigensolver uses it.
#include "lqcd_internal.h"

namespace lqcd {

namespace {

typedef cplx<double> Cd;

struct M3 {
  Cd m[3][3];
};

LQCD_D M3 load_m(const double2* U, const Geom& g, int mu, int x, int y, int z, int t) {
  const long s = lex_index(g, x, y, z, t);
  const int p = (x + y + z + t) & 1;
  const double2* f = U + ((long)(mu * 2 + p) * 9) * g.Vh + (s >> 1);
  M3 r;
#pragma unroll
  for (int e = 0; e < 9; e++) {
    const double2 v = f[(long)e * g.Vh];
    r.m[e / 3][e % 3] = {v.x, v.y};
  }
  return r;
}

LQCD_D M3 mul(const M3& a, const M3& b) {  // a b
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) r.m[i][j] = cfma(a.m[i][2], b.m[2][j], cfma(a.m[i][1], b.m[1][j], a.m[i][0] * b.m[0][j]));
  return r;
}

LQCD_D M3 mul_dag(const M3& a, const M3& b) {  // a b^dag
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      Cd s = {0, 0};
#pragma unroll
      for (int k = 0; k < 3; k++) s = s + a.m[i][k] * cj(b.m[j][k]);
      r.m[i][j] = s;
    }
  return r;
}

LQCD_D M3 dag_mul(const M3& a, const M3& b) {  // a^dag b
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      Cd s = {0, 0};
#pragma unroll
      for (int k = 0; k < 3; k++) s = s + cjmul(a.m[k][i], b.m[k][j]);
      r.m[i][j] = s;
    }
  return r;
}

LQCD_D Cd det3(const M3& a) {
  return a.m[0][0] * (a.m[1][1] * a.m[2][2] - a.m[1][2] * a.m[2][1]) -
         a.m[0][1] * (a.m[1][0] * a.m[2][2] - a.m[1][2] * a.m[2][0]) +
         a.m[0][2] * (a.m[1][0] * a.m[2][1] - a.m[1][1] * a.m[2][0]);
}

LQCD_D Cd cdiv(Cd a, Cd b) {
  const double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// (a^-1)^dag from the cofactors: a^-1 = adj(a) / det(a)
LQCD_D M3 inv_dag(const M3& a, bool& ok) {
  const Cd d = det3(a);
  ok = ok && (d.re * d.re + d.im * d.im) > 1e-200;
  M3 c;  // cofactor matrix: C[i][j] = (-1)^(i+j) minor(i, j); a^-1 = C^T / det
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      c.m[i][j] = a.m[i1][j1] * a.m[i2][j2] - a.m[i1][j2] * a.m[i2][j1];
    }
  M3 r;  // (a^-1)^dag [i][j] = conj(a^-1 [j][i]) = conj(C[i][j] / det)
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) r.m[i][j] = cj(cdiv(c.m[i][j], d));
  return r;
}

LQCD_D double frob2(const M3& a) {
  double s = 0;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) s += norm2(a.m[i][j]);
  return s;
}

// P(X): unitary polar factor by scaled Newton, then the determinant phase removed
LQCD_D M3 project_su3(M3 w, bool& ok) {
  for (int it = 0; it < 50; it++) {
    const M3 wi = inv_dag(w, ok);
    if (!ok) break;
    const double gsc = sqrt(sqrt(frob2(wi) / frob2(w)));
    double moved = 0;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int j = 0; j < 3; j++) {
        const Cd n = {0.5 * (gsc * w.m[i][j].re + wi.m[i][j].re / gsc), 0.5 * (gsc * w.m[i][j].im + wi.m[i][j].im / gsc)};
        moved = fmax(moved, fmax(fabs(n.re - w.m[i][j].re), fabs(n.im - w.m[i][j].im)));
        w.m[i][j] = n;
      }
    if (moved < 1e-14) break;
  }
  const Cd d = det3(w);
  const double ph = atan2(d.im, d.re) / 3.0, mag = cbrt(sqrt(d.re * d.re + d.im * d.im));
  const Cd root = {mag * cos(ph), mag * sin(ph)};
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) w.m[i][j] = cdiv(w.m[i][j], root);
  return w;
}

__global__ void k_ape_step(const double2* in, double2* out, Geom g, double alpha, int* bad) {
  const long V = 2 * g.Vh;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 3 * V) return;
  const int k = (int)(tid / V);
  const long s = tid - (long)k * V;
  const int x = (int)(s % g.Lx), y = (int)((s / g.Lx) % g.Ly), z = (int)((s / ((long)g.Lx * g.Ly)) % g.Lz);
  const int t = (int)(s / ((long)g.Lx * g.Ly * g.Lz));
  const int L[3] = {g.Lx, g.Ly, g.Lz};
  auto shifted = [&](int c0[3], int mu, int n) {
    c0[mu] = (c0[mu] + n + L[mu]) % L[mu];
  };
  M3 X = load_m(in, g, k, x, y, z, t);
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) X.m[i][j] = (1.0 - alpha) * X.m[i][j];
  M3 st;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) st.m[i][j] = {0, 0};
  for (int j = 0; j < 3; j++) {
    if (j == k) continue;
    int pj[3] = {x, y, z}, pk[3] = {x, y, z}, mj[3] = {x, y, z}, mjk[3] = {x, y, z};
    shifted(pj, j, 1);
    shifted(pk, k, 1);
    shifted(mj, j, -1);
    shifted(mjk, j, -1);
    shifted(mjk, k, 1);
    // forward: U_j(x) U_k(x+j) U_j(x+k)^dag
    const M3 f = mul_dag(mul(load_m(in, g, j, x, y, z, t), load_m(in, g, k, pj[0], pj[1], pj[2], t)),
                         load_m(in, g, j, pk[0], pk[1], pk[2], t));
    // backward: U_j(x-j)^dag U_k(x-j) U_j(x-j+k)
    const M3 b = mul(dag_mul(load_m(in, g, j, mj[0], mj[1], mj[2], t), load_m(in, g, k, mj[0], mj[1], mj[2], t)),
                     load_m(in, g, j, mjk[0], mjk[1], mjk[2], t));
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int c = 0; c < 3; c++) st.m[a][c] = st.m[a][c] + f.m[a][c] + b.m[a][c];
  }
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) X.m[i][j] = X.m[i][j] + (0.25 * alpha) * st.m[i][j];
  bool ok = true;
  const M3 W = project_su3(X, ok);
  if (!ok) atomicOr(bad, 1);
  const int p = (x + y + z + t) & 1;
  double2* o = out + ((long)(k * 2 + p) * 9) * g.Vh + (s >> 1);
#pragma unroll
  for (int e = 0; e < 9; e++) o[(long)e * g.Vh] = make_double2(W.m[e / 3][e % 3].re, W.m[e / 3][e % 3].im);
}

// user layout out[t][z][y][x][k][3][3] (k < 3) from the context layout
__global__ void k_unpack_spatial(const double2* U, Geom g, double2* out) {
  const long V = 2 * g.Vh;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= V * 27) return;
  const long s = tid / 27;
  const int r = (int)(tid - s * 27), k = r / 9, e = r % 9;
  const int x = (int)(s % g.Lx), y = (int)((s / g.Lx) % g.Ly), z = (int)((s / ((long)g.Lx * g.Ly)) % g.Lz);
  const int t = (int)(s / ((long)g.Lx * g.Ly * g.Lz));
  const int p = (x + y + z + t) & 1;
  out[tid] = U[((long)(k * 2 + p) * 9 + e) * g.Vh + (s >> 1)];
}

}  // namespace

// Smear n_iter steps from the uploaded links into c->Usm (n_iter = 0 drops the smeared field).
int ape_smear(lqcd_ctx* c, double alpha, int n_iter) {
  const Geom& g = c->g;
  if (n_iter == 0) {
    c->have_smeared = false;
    return LQCD_OK;
  }
  const size_t bytes = (size_t)3 * 2 * 9 * g.Vh * sizeof(double2);
  if (!c->Usm && cudaMalloc(&c->Usm, bytes) != cudaSuccess) {
    c->Usm = nullptr;
    cudaGetLastError();
    return set_error(c, LQCD_ERR_OOM, "ape_smear: out of device memory");
  }
  double2* tmp = (double2*)ws_get(c, "ape_tmp", bytes);
  int* bad = (int*)ws_get(c, "ape_bad", 64);
  if (!tmp || !bad) return set_error(c, LQCD_ERR_OOM, "ape_smear: out of device memory");
  cudaMemsetAsync(bad, 0, sizeof(int), c->work);
  // step i reads the previous field: start so that the last step writes c->Usm
  double2* a = (n_iter % 2) ? tmp : (double2*)c->Usm;
  double2* b = (n_iter % 2) ? (double2*)c->Usm : tmp;
  cudaMemcpyAsync(a, c->U64, bytes, cudaMemcpyDeviceToDevice, c->work);  // spatial blocks mu = 0, 1, 2
  const long n = 3 * 2 * g.Vh;
  for (int it = 0; it < n_iter; it++) {
    k_ape_step<<<(unsigned)((n + 127) / 128), 128, 0, c->work>>>(a, b, g, alpha, bad);
    count_launch();
    double2* sw = a;
    a = b;
    b = sw;
  }
  int hb = 0;
  cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, c->work);
  cudaError_t e = cudaStreamSynchronize(c->work);
  if (e != cudaSuccess) return set_error(c, LQCD_ERR_CUDA, std::string("ape_smear: ") + cudaGetErrorString(e));
  if (hb) {
    c->have_smeared = false;
    return set_error(c, LQCD_ERR_NAN, "ape_smear: singular staple sum (no SU(3) projection)");
  }
  c->have_smeared = true;
  return LQCD_OK;
}

void unpack_smeared(lqcd_ctx* c, double2* out) {
  const long n = 2 * c->g.Vh * 27;
  k_unpack_spatial<<<(unsigned)((n + 255) / 256), 256, 0, c->work>>>((const double2*)c->Usm, c->g, out);
  count_launch();
}

}  // namespace lqcd
