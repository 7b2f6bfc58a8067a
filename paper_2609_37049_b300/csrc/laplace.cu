// Lowest eigenpairs of the gauge-covariant 3D Laplacian on every timeslice (the distillation
// vectors v_i(t) and eigenvalues lambda_i(t) of Sec. 3.1 / 3.2), computed on the GPU.
//
//   (-Lap phi)(x) = sum_{k=x,y,z} [ 2 phi(x) - U_k(x) phi(x+k) - U_k(x-k)^dag phi(x-k) ]
//
// Chebyshev-filtered subspace iteration (Zhou and Saad, "Self-consistent-field calculations
// using Chebyshev-filtered subspace iteration", J. Comput. Phys. 219 (2006)) on all timeslices at
// once (the operator is block diagonal in t): a subspace of m = n_ev + guard vectors per
// timeslice is filtered by a degree-d Chebyshev polynomial that damps [a, b] (b = 12 bounds the
// spectrum of -Lap for unitary links, a = the largest current Ritz value), orthonormalised and
// rotated onto Ritz vectors (Rayleigh-Ritz), until every wanted pair has ||A v - lambda v|| <= tol.
// The large operations (stencil, Gram matrices, rotations, residuals) are CUDA kernels; the m x m
// Hermitian eigenproblems are solved on the host by cyclic Jacobi rotations.
// Vectors are stored per timeslice as N x m row-major matrices (N = 3 L^3, index s3*3 + colour),
// so one thread per (row, column) reads its links once per warp and its neighbours coalesced.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <vector>

#include "lqcd_distill.h"

namespace lqcd {

using cd = std::complex<double>;

// out = a (-Lap) X + b X + c Z  for timeslices [t0, t0 + nt), columns m
__global__ void k_lap(const double2* X, const double2* Z, double2* out, const double2* U64, Geom g, int t0, int nt,
                      int m, double a, double b, double c) {
  const long L3 = (long)g.Lx * g.Ly * g.Lz;
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long total = (long)nt * L3 * m;
  if (tid >= total) return;
  const int k = (int)(tid % m);
  const long row = tid / m;  // (tl, s3)
  const int tl = (int)(row / L3);
  const long s3 = row - (long)tl * L3;
  const int t = t0 + tl;
  const int x = (int)(s3 % g.Lx), y = (int)((s3 / g.Lx) % g.Ly), z = (int)(s3 / ((long)g.Lx * g.Ly));
  const int p = (x + y + z + t) & 1;
  const long cb = lex_index(g, x, y, z, t) >> 1;
  const double2* Xt = X + (long)tl * L3 * 3 * m;
  cplx<double> acc[3];
  for (int q = 0; q < 3; q++) {
    double2 v = Xt[(s3 * 3 + q) * m + k];
    acc[q] = {6.0 * v.x, 6.0 * v.y};
  }
  for (int d = 0; d < 3; d++) {
    int xf = x, yf = y, zf = z, xb = x, yb = y, zb = z;
    if (d == 0) {
      xf = (x + 1) % g.Lx;
      xb = (x + g.Lx - 1) % g.Lx;
    } else if (d == 1) {
      yf = (y + 1) % g.Ly;
      yb = (y + g.Ly - 1) % g.Ly;
    } else {
      zf = (z + 1) % g.Lz;
      zb = (z + g.Lz - 1) % g.Lz;
    }
    const long sf = xf + (long)g.Lx * (yf + (long)g.Ly * zf);
    const long sb = xb + (long)g.Lx * (yb + (long)g.Ly * zb);
    const long cbb = lex_index(g, xb, yb, zb, t) >> 1;
    const double2* uf = U64 + ((long)(d * 2 + p) * 9) * g.Vh + cb;
    const double2* ub = U64 + ((long)(d * 2 + (1 - p)) * 9) * g.Vh + cbb;
    cplx<double> vf[3], vb[3];
    for (int q = 0; q < 3; q++) {
      double2 w = Xt[(sf * 3 + q) * m + k];
      vf[q] = {w.x, w.y};
      w = Xt[(sb * 3 + q) * m + k];
      vb[q] = {w.x, w.y};
    }
    for (int i = 0; i < 3; i++) {
      cplx<double> s = {0, 0};
      for (int j = 0; j < 3; j++) {
        double2 u = __ldg(uf + (i * 3 + j) * g.Vh);
        double2 w = __ldg(ub + (j * 3 + i) * g.Vh);
        s = s + cplx<double>{u.x, u.y} * vf[j] + cjmul(cplx<double>{w.x, w.y}, vb[j]);
      }
      acc[i] = acc[i] - s;
    }
  }
  double2* o = out + (long)tl * L3 * 3 * m;
  const double2* Zt = Z ? Z + (long)tl * L3 * 3 * m : nullptr;
  for (int q = 0; q < 3; q++) {
    long e = (s3 * 3 + q) * m + k;
    double2 xv = Xt[e];
    cplx<double> r = a * acc[q] + b * cplx<double>{xv.x, xv.y};
    if (Zt) r = r + c * cplx<double>{Zt[e].x, Zt[e].y};
    o[e] = make_double2(r.re, r.im);
  }
}

// C_t = A_t^H B_t (m x m) for N x m row-major A_t, B_t
__global__ void k_gram(const double2* A, const double2* B, double2* C, long N, int m) {
  __shared__ double2 As[16][17];
  __shared__ double2 Bs[16][17];
  const int t = blockIdx.z;
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const double2* At = A + (long)t * N * m;
  const double2* Bt = B + (long)t * N * m;
  cplx<double> acc = {0, 0};
  for (long n0 = 0; n0 < N; n0 += 16) {
    long n = n0 + ty;
    As[ty][tx] = (n < N && i0 + tx < m) ? At[n * m + i0 + tx] : make_double2(0, 0);
    Bs[ty][tx] = (n < N && j0 + tx < m) ? Bt[n * m + j0 + tx] : make_double2(0, 0);
    __syncthreads();
    for (int q = 0; q < 16; q++) {
      double2 a = As[q][ty], b = Bs[q][tx];
      acc = acc + cjmul(cplx<double>{a.x, a.y}, cplx<double>{b.x, b.y});
    }
    __syncthreads();
  }
  if (i0 + ty < m && j0 + tx < m) C[((long)t * m + i0 + ty) * m + j0 + tx] = make_double2(acc.re, acc.im);
}

// Out_t = A_t Q_t  (N x m times m x m)
__global__ void k_rotate(const double2* A, const double2* Q, double2* Out, long N, int m, int nt) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long total = (long)nt * N * m;
  if (tid >= total) return;
  const int j = (int)(tid % m);
  const long r = tid / m;
  const int t = (int)(r / N);
  const double2* a = A + r * m;
  const double2* q = Q + (long)t * m * m + j;
  cplx<double> s = {0, 0};
  for (int i = 0; i < m; i++) {
    double2 x = a[i], y = q[(long)i * m];
    s = s + cplx<double>{x.x, x.y} * cplx<double>{y.x, y.y};
  }
  Out[tid] = make_double2(s.re, s.im);
}

// res[t][i] = || W[:, i] - lam[t][i] X[:, i] ||
__global__ void k_colres(const double2* W, const double2* X, const double* lam, double* res, long N, int m) {
  const int t = blockIdx.y, i = blockIdx.x;
  __shared__ double sm[128];
  const double l = lam[(long)t * m + i];
  double s = 0;
  for (long n = threadIdx.x; n < N; n += blockDim.x) {
    long e = ((long)t * N + n) * m + i;
    double2 w = W[e], x = X[e];
    double dr = w.x - l * x.x, di = w.y - l * x.y;
    s += dr * dr + di * di;
  }
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k >= 1; k >>= 1) {
    if (threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) res[(long)t * m + i] = sqrt(sm[0]);
}

// deterministic pseudo-random start vectors
__global__ void k_randfill(double2* X, long n, unsigned seed) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long h = (unsigned long long)i * 0x9E3779B97F4A7C15ull ^ seed;
  h ^= h >> 31;
  h *= 0xBF58476D1CE4E5B9ull;
  h ^= h >> 29;
  double a = (double)(h & 0xFFFFFF) / 16777216.0 - 0.5, b = (double)((h >> 24) & 0xFFFFFF) / 16777216.0 - 0.5;
  X[i] = make_double2(a, b);
}

// Largest-modulus component (first on ties) of each wanted vector made real positive; write
// V[t0 + tl][i][s3][a] (caller layout) from X[tl][s3*3+a][i].
__global__ void k_phase_out(const double2* X, double2* Vout, long N, int m, int n_ev, int t0) {
  const int tl = blockIdx.y, i = blockIdx.x;
  __shared__ double bm[128];
  __shared__ long bi[128];
  double best = -1;
  long arg = 0;
  for (long n = threadIdx.x; n < N; n += blockDim.x) {
    double2 v = X[((long)tl * N + n) * m + i];
    double a = v.x * v.x + v.y * v.y;
    if (a > best) {
      best = a;
      arg = n;
    }
  }
  bm[threadIdx.x] = best;
  bi[threadIdx.x] = arg;
  __syncthreads();
  for (int k = blockDim.x / 2; k >= 1; k >>= 1) {
    if (threadIdx.x < k) {
      double o = bm[threadIdx.x + k];
      long oi = bi[threadIdx.x + k];
      if (o > bm[threadIdx.x] || (o == bm[threadIdx.x] && oi < bi[threadIdx.x])) {
        bm[threadIdx.x] = o;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  double2 pv = X[((long)tl * N + bi[0]) * m + i];
  double mag = sqrt(pv.x * pv.x + pv.y * pv.y);
  cplx<double> ph = {pv.x / mag, -pv.y / mag};  // conj(p) / |p|
  for (long n = threadIdx.x; n < N; n += blockDim.x) {
    double2 v = X[((long)tl * N + n) * m + i];
    cplx<double> r = ph * cplx<double>{v.x, v.y};
    Vout[(((long)(t0 + tl) * n_ev + i) * N) + n] = make_double2(r.re, r.im);
  }
}

// ---------------------------------------------------------------- host dense linear algebra
// Cyclic Jacobi eigendecomposition of a Hermitian m x m matrix (row major): A = V diag(w) V^H,
// eigenvalues ascending.
static void jacobi_eigh(std::vector<cd>& A, int m, std::vector<double>& w, std::vector<cd>& V) {
  V.assign((size_t)m * m, cd(0, 0));
  for (int i = 0; i < m; i++) V[(size_t)i * m + i] = 1.0;
  auto a = [&](int i, int j) -> cd& { return A[(size_t)i * m + j]; };
  for (int sweep = 0; sweep < 100; sweep++) {
    double off = 0, tot = 0;
    for (int i = 0; i < m; i++)
      for (int j = 0; j < m; j++) {
        double v = std::norm(a(i, j));
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < m - 1; p++)
      for (int q = p + 1; q < m; q++) {
        double bq = std::abs(a(p, q));
        if (bq < 1e-300) continue;
        // phase on column/row q so that a(p,q) becomes real positive
        cd ph = a(p, q) / bq;  // e^{i phi}
        cd phc = std::conj(ph);
        for (int k = 0; k < m; k++) {
          a(k, q) *= phc;
          V[(size_t)k * m + q] *= phc;
        }
        for (int k = 0; k < m; k++) a(q, k) *= ph;
        double app = a(p, p).real(), aqq = a(q, q).real();
        double tau = (aqq - app) / (2 * bq);
        double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1 + tau * tau));
        double c = 1 / std::sqrt(1 + t * t), s = t * c;
        // A <- P^T A P with P_pp = P_qq = c, P_pq = s, P_qp = -s
        for (int k = 0; k < m; k++) {
          cd akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < m; k++) {
          cd apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < m; k++) {
          cd vkp = V[(size_t)k * m + p], vkq = V[(size_t)k * m + q];
          V[(size_t)k * m + p] = c * vkp - s * vkq;
          V[(size_t)k * m + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> ord(m);
  for (int i = 0; i < m; i++) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return a(x, x).real() < a(y, y).real(); });
  w.resize(m);
  std::vector<cd> Vs((size_t)m * m);
  for (int j = 0; j < m; j++) {
    w[j] = a(ord[j], ord[j]).real();
    for (int k = 0; k < m; k++) Vs[(size_t)k * m + j] = V[(size_t)k * m + ord[j]];
  }
  V.swap(Vs);
}

struct LapBufs {
  double2 *X, *Y, *Yp, *W, *G, *Q;
  double *lam, *res;
};

static void lap_apply(lqcd_ctx* c, const double2* X, const double2* Z, double2* out, int t0, int nt, int m, double a,
                      double b, double cc) {
  const long L3 = (long)c->g.Lx * c->g.Ly * c->g.Lz;
  long n = (long)nt * L3 * m;
  const double2* U = (const double2*)(c->have_smeared ? c->Usm : c->U64);  // smeared links if present
  k_lap<<<(n + 255) / 256, 256, 0, c->work>>>(X, Z, out, U, c->g, t0, nt, m, a, b, cc);
  count_launch();
}

static void gram(lqcd_ctx* c, const double2* A, const double2* B, double2* C, long N, int m, int nt) {
  dim3 grid((m + 15) / 16, (m + 15) / 16, nt);
  k_gram<<<grid, dim3(16, 16), 0, c->work>>>(A, B, C, N, m);
  count_launch();
}

static void rotate(lqcd_ctx* c, const double2* A, const double2* Q, double2* Out, long N, int m, int nt) {
  long n = (long)nt * N * m;
  k_rotate<<<(n + 255) / 256, 256, 0, c->work>>>(A, Q, Out, N, m, nt);
  count_launch();
}

// Orthonormalise the columns of Y in place (per timeslice) through the eigendecomposition of
// the Gram matrix: Y <- Y W diag(g)^{-1/2}; returns false if a Gram matrix is rank deficient.
static bool orthonormalise(lqcd_ctx* c, LapBufs& B, double2*& Y, double2*& spare, long N, int m, int nt) {
  gram(c, Y, Y, B.G, N, m, nt);
  std::vector<double2> h((size_t)nt * m * m);
  cudaMemcpyAsync(h.data(), B.G, h.size() * sizeof(double2), cudaMemcpyDeviceToHost, c->work);
  cudaStreamSynchronize(c->work);
  std::vector<double2> q((size_t)nt * m * m);
  int ok = 1;
#pragma omp parallel for schedule(dynamic) reduction(min : ok)
  for (int t = 0; t < nt; t++) {
    // unit-diagonal Gram (columns normalised first: the filter scales them very differently)
    std::vector<double> d(m);
    for (int i = 0; i < m; i++) {
      double gii = h[(size_t)t * m * m + (size_t)i * m + i].x;
      d[i] = gii > 0 ? 1.0 / std::sqrt(gii) : 0.0;
      if (!(gii > 0)) ok = 0;
    }
    std::vector<cd> A((size_t)m * m);
    for (int i = 0; i < m; i++)
      for (int j = 0; j < m; j++) {
        double2 x = h[(size_t)t * m * m + (size_t)i * m + j];
        A[(size_t)i * m + j] = d[i] * d[j] * cd(x.x, x.y);
      }
    std::vector<double> w;
    std::vector<cd> V;
    jacobi_eigh(A, m, w, V);
    if (!(w[0] > 1e-14 * w[m - 1])) {
      ok = 0;
      continue;
    }
    for (int i = 0; i < m; i++)
      for (int j = 0; j < m; j++) {
        cd v = d[i] * V[(size_t)i * m + j] / std::sqrt(w[j]);
        q[(size_t)t * m * m + (size_t)i * m + j] = make_double2(v.real(), v.imag());
      }
  }
  if (!ok) return false;
  cudaMemcpyAsync(B.Q, q.data(), q.size() * sizeof(double2), cudaMemcpyHostToDevice, c->work);
  rotate(c, Y, B.Q, spare, N, m, nt);
  std::swap(Y, spare);
  return true;
}

// Rayleigh-Ritz: X <- Y Z with Y^H A Y = Z diag(lam) Z^H; lam to host and device.
static void rayleigh_ritz(lqcd_ctx* c, LapBufs& B, const double2* Y, double2* X, long N, int m, int t0, int nt,
                          std::vector<double>& lam_h) {
  lap_apply(c, Y, nullptr, B.W, t0, nt, m, 1.0, 0.0, 0.0);
  gram(c, Y, B.W, B.G, N, m, nt);
  std::vector<double2> h((size_t)nt * m * m);
  cudaMemcpyAsync(h.data(), B.G, h.size() * sizeof(double2), cudaMemcpyDeviceToHost, c->work);
  cudaStreamSynchronize(c->work);
  std::vector<double2> q((size_t)nt * m * m);
  lam_h.resize((size_t)nt * m);
#pragma omp parallel for schedule(dynamic)
  for (int t = 0; t < nt; t++) {
    std::vector<cd> A((size_t)m * m);
    for (int i = 0; i < m; i++)
      for (int j = 0; j < m; j++) {
        // symmetrise: the Gram of a Hermitian operator is Hermitian up to rounding
        double2 x = h[(size_t)t * m * m + (size_t)i * m + j], y = h[(size_t)t * m * m + (size_t)j * m + i];
        A[(size_t)i * m + j] = 0.5 * (cd(x.x, x.y) + std::conj(cd(y.x, y.y)));
      }
    std::vector<double> w;
    std::vector<cd> V;
    jacobi_eigh(A, m, w, V);
    for (int j = 0; j < m; j++) lam_h[(size_t)t * m + j] = w[j];
    for (size_t e = 0; e < V.size(); e++) q[(size_t)t * m * m + e] = make_double2(V[e].real(), V[e].imag());
  }
  cudaMemcpyAsync(B.Q, q.data(), q.size() * sizeof(double2), cudaMemcpyHostToDevice, c->work);
  cudaMemcpyAsync(B.lam, lam_h.data(), lam_h.size() * sizeof(double), cudaMemcpyHostToDevice, c->work);
  rotate(c, Y, B.Q, X, N, m, nt);
}

int laplace_eigs(lqcd_ctx* c, int n_ev, double2* Vout, double* lam_out_dev, double tol, int max_iter,
                 int* iters_out) {
  const Geom& g = c->g;
  const long L3 = (long)g.Lx * g.Ly * g.Lz;
  const long N = 3 * L3;
  int m = n_ev + std::max(8, n_ev / 2);
  if (m > N) m = (int)N;
  // timeslices per chunk: keep each of the four N x m work buffers under ~2 GB
  long per_t = N * m * (long)sizeof(double2);
  int tchunk = (int)std::max(1L, std::min((long)g.Lt, (2L << 30) / per_t));
  const int max_degree = 16;
  const double bmax = 12.0;
  LapBufs B;
  size_t vb = (size_t)tchunk * N * m * sizeof(double2);
  B.X = (double2*)ws_get(c, "lap_X", vb);
  B.Y = (double2*)ws_get(c, "lap_Y", vb);
  B.Yp = (double2*)ws_get(c, "lap_Yp", vb);
  B.W = (double2*)ws_get(c, "lap_W", vb);
  B.G = (double2*)ws_get(c, "lap_G", (size_t)tchunk * m * m * sizeof(double2));
  B.Q = (double2*)ws_get(c, "lap_Q", (size_t)tchunk * m * m * sizeof(double2));
  B.lam = (double*)ws_get(c, "lap_lam", (size_t)tchunk * m * sizeof(double));
  B.res = (double*)ws_get(c, "lap_res", (size_t)tchunk * m * sizeof(double));
  if (!B.X || !B.Y || !B.Yp || !B.W || !B.G || !B.Q || !B.lam || !B.res)
    return set_error(c, LQCD_ERR_OOM, "laplace_eigs: out of device memory");
  int worst_iters = 0;
  for (int t0 = 0; t0 < g.Lt; t0 += tchunk) {
    const int nt = std::min(tchunk, g.Lt - t0);
    long n = (long)nt * N * m;
    // three N x m buffers rotate between the Ritz block X and the filter recurrence; W holds A Y
    double2* X = B.X;
    double2* Y = B.Y;
    double2* spare = B.Yp;
    k_randfill<<<(n + 255) / 256, 256, 0, c->work>>>(Y, n, 0x1234567u + t0);
    count_launch();
    if (!orthonormalise(c, B, Y, spare, N, m, nt)) return set_error(c, LQCD_ERR_NAN, "laplace_eigs: start");
    std::vector<double> lam;
    rayleigh_ritz(c, B, Y, X, N, m, t0, nt, lam);
    int it = 0;
    bool done = false;
    double worst_res = 0, last_a = 0;
    int last_degree = 0;
    for (; it < max_iter && !done; it++) {
      // filter: damp [a, bmax], a = largest Ritz value of the subspace (minimum over timeslices);
      // y1 = (A - c) X / e,  y_{k+1} = 2 (A - c) y_k / e - y_{k-1}
      double a = bmax, lmin = bmax;
      for (int t = 0; t < nt; t++) {
        a = std::min(a, lam[(size_t)t * m + m - 1]);
        lmin = std::min(lmin, lam[(size_t)t * m]);
      }
      const double e = 0.5 * (bmax - a), cc = 0.5 * (bmax + a);
      // cap the amplification of the lowest mode relative to the cut at 1e4 per iteration
      // (|T_d(x)| = cosh(d acosh|x|)): larger ratios cost the upper wanted vectors precision
      const double xmin = std::fabs((lmin - cc) / e);
      int degree = max_degree;
      if (xmin > 1.0) degree = std::max(2, std::min(max_degree, (int)(std::acosh(1e4) / std::acosh(xmin))));
      double2* free_bufs[2];
      int nf = 0;
      for (double2* q : {B.X, B.Y, B.Yp})
        if (q != X) free_bufs[nf++] = q;
      double2* y0 = X;
      double2* y1 = free_bufs[0];
      double2* y2 = free_bufs[1];
      lap_apply(c, y0, nullptr, y1, t0, nt, m, 1.0 / e, -cc / e, 0.0);
      for (int k = 2; k <= degree; k++) {
        lap_apply(c, y1, y0, y2, t0, nt, m, 2.0 / e, -2.0 * cc / e, -1.0);
        double2* tmp = y0;
        y0 = y1;
        y1 = y2;
        y2 = tmp;
      }
      Y = y1;        // filtered block
      spare = y0;    // free (y2 is free too)
      if (!orthonormalise(c, B, Y, spare, N, m, nt) || !orthonormalise(c, B, Y, spare, N, m, nt))
        return set_error(c, LQCD_ERR_NAN, "laplace_eigs: filtered block lost rank");
      // Ritz vectors into a buffer other than Y
      X = (spare != Y) ? spare : y2;
      rayleigh_ritz(c, B, Y, X, N, m, t0, nt, lam);
      // residuals of the wanted pairs
      lap_apply(c, X, nullptr, B.W, t0, nt, m, 1.0, 0.0, 0.0);
      k_colres<<<dim3(m, nt), 128, 0, c->work>>>(B.W, X, B.lam, B.res, N, m);
      count_launch();
      std::vector<double> res((size_t)nt * m);
      cudaMemcpyAsync(res.data(), B.res, res.size() * sizeof(double), cudaMemcpyDeviceToHost, c->work);
      cudaStreamSynchronize(c->work);
      done = true;
      worst_res = 0;
      for (int t = 0; t < nt; t++)
        for (int i = 0; i < n_ev; i++) {
          double r = res[(size_t)t * m + i];
          if (!(r <= tol)) done = false;
          if (!(r <= worst_res)) worst_res = r;
        }
      last_a = a;
      last_degree = degree;
    }
    worst_iters = std::max(worst_iters, it);
    if (!done) {
      char msg[256];
      snprintf(msg, sizeof msg,
               "laplace_eigs: tolerance not reached (max residual %.3g after %d iterations, filter cut %.6g, "
               "degree %d, subspace %d)", worst_res, it, last_a, last_degree, m);
      return set_error(c, LQCD_ERR_NOT_CONVERGED, msg);
    }
    k_phase_out<<<dim3(n_ev, nt), 128, 0, c->work>>>(X, Vout, N, m, n_ev, t0);
    count_launch();
    std::vector<double> lw((size_t)nt * n_ev);
    for (int t = 0; t < nt; t++)
      for (int i = 0; i < n_ev; i++) lw[(size_t)t * n_ev + i] = lam[(size_t)t * m + i];
    cudaMemcpyAsync(lam_out_dev + (size_t)t0 * n_ev, lw.data(), lw.size() * sizeof(double), cudaMemcpyHostToDevice,
                    c->work);
    cudaStreamSynchronize(c->work);
  }
  if (iters_out) *iters_out = worst_iters;
  return LQCD_OK;
}

}  // namespace lqcd
