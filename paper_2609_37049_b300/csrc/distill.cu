// Layout conversion between the caller's lexicographic spinors and the internal even-odd
// layout, and the distillation kernels: sources (Sec. 3.1), the projection
// tau = V^dagger X on sink timeslices, quark loops (Sec. 2 / Sec. 3.2) and the disconnected
// correlators (Eqs. Cdisc, correlator_factorised, subtracted_correlator, corr1-corr4).
#include "lqcd_distill.h"

namespace lqcd {

// ------------------------------------------------------------------ layouts
// lex [nrhs][V][12] <-> full even-odd FP64 [par][12][Vh][nrhs]
__global__ void k_pack_spinor(const double2* in, double2* out, Geom g, int nrhs, int to_eo) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long n = 2 * g.Vh * (long)nrhs;
  if (tid >= n) return;
  const int rhs = (int)(tid % nrhs);
  const long site = tid / nrhs;
  const int par = (int)(site / g.Vh);
  const long cb = site - par * g.Vh;
  int x, y, z, t;
  cb_coords(g, par, cb, x, y, z, t);
  const long s = lex_index(g, x, y, z, t);
  const long V = 2 * g.Vh;
  double2* eo_base = out;
  const double2* lex = in;
  if (to_eo) {
    for (int k = 0; k < 12; k++)
      eo_base[(long)par * 12 * g.Vh * nrhs + (k * g.Vh + cb) * nrhs + rhs] = lex[((long)rhs * V + s) * 12 + k];
  } else {
    // here `in` is the eo field and `out` the lex field
    for (int k = 0; k < 12; k++)
      out[((long)rhs * V + s) * 12 + k] = in[(long)par * 12 * g.Vh * nrhs + (k * g.Vh + cb) * nrhs + rhs];
  }
}

void pack_spinor(const Geom& g, const double2* lex, double2* eo, int nrhs, cudaStream_t st) {
  long n = 2 * g.Vh * (long)nrhs;
  k_pack_spinor<<<(n + 255) / 256, 256, 0, st>>>(lex, eo, g, nrhs, 1); lqcd::count_launch();
}
void unpack_spinor(const Geom& g, const double2* eo, double2* lex, int nrhs, cudaStream_t st) {
  long n = 2 * g.Vh * (long)nrhs;
  k_pack_spinor<<<(n + 255) / 256, 256, 0, st>>>(eo, lex, g, nrhs, 0); lqcd::count_launch();
}

// ------------------------------------------------------------------ sources
// b_r(x) = [srcmask[t] == 1] e_{beta_r} (x) v_{j_r}(t)(xvec); Vt: [slots][n_ev][L3][3] with the
// vectors of timeslice t in slot vslot[t]
__global__ void k_sources(const double2* Vt, int n_ev, const int* jr, const int* br, const unsigned char* srcmask,
                          const int* vslot, double2* b, Geom g, int nrhs) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long n = 2 * g.Vh * (long)nrhs;
  if (tid >= n) return;
  const int rhs = (int)(tid % nrhs);
  const long site = tid / nrhs;
  const int par = (int)(site / g.Vh);
  const long cb = site - par * g.Vh;
  int x, y, z, t;
  cb_coords(g, par, cb, x, y, z, t);
  const long L3 = (long)g.Lx * g.Ly * g.Lz;
  const long s3 = x + (long)g.Lx * (y + (long)g.Ly * z);
  double2* out = b + (long)par * 12 * g.Vh * nrhs;
  const int on = srcmask[t];
  const int beta = br[rhs], j = jr[rhs];
  for (int spin = 0; spin < 4; spin++)
    for (int a = 0; a < 3; a++) {
      double2 v = make_double2(0.0, 0.0);
      if (on && spin == beta) v = Vt[(((long)vslot[t] * n_ev + j) * L3 + s3) * 3 + a];
      out[((spin * 3 + a) * g.Vh + cb) * nrhs + rhs] = v;
    }
}

void make_sources(const Geom& g, const double2* Vt, int n_ev, const int* jr, const int* br,
                  const unsigned char* srcmask, const int* vslot, double2* b, int nrhs, cudaStream_t st) {
  long n = 2 * g.Vh * (long)nrhs;
  k_sources<<<(n + 255) / 256, 256, 0, st>>>(Vt, n_ev, jr, br, srcmask, vslot, b, g, nrhs); lqcd::count_launch();
}

// ------------------------------------------------------------------ projection
// For every sink timeslice tp = sinks[z]:  C[z][i][alpha][r] = sum_{s3,a} conj(V(tp)[i][s3][a])
//                                                               X_r(tp, s3, alpha, a)
// as a tiled complex GEMM (M = n_ev, N = 4 nrhs with n = alpha * nrhs + r, K = 3 L^3), FP64,
// split along K over blockIdx.z = z * ksplit + kpart so the grid fills the GPU; the ksplit
// partial tiles are then summed in a fixed order (deterministic).
#define PBM 32
#define PBN 32
#define PBK 16
__global__ void __launch_bounds__(256) k_project(const double2* Vt, int n_ev, const double2* X, const int* sinks,
                                                 const int* vslot, double2* Cpart, Geom g, int nrhs, int ksplit) {
  __shared__ double2 As[PBK][PBM + 1];
  __shared__ double2 Bs[PBK][PBN + 1];
  const int z = blockIdx.z / ksplit, kpart = blockIdx.z - z * ksplit;
  const int tp = sinks[z];
  const long L3 = (long)g.Lx * g.Ly * g.Lz;
  const long K = 3 * L3;
  const int N = 4 * nrhs;
  const int m0 = blockIdx.y * PBM, n0 = blockIdx.x * PBN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  cplx<double> acc[2][2];
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) acc[i][j] = {0.0, 0.0};
  const double2* A = Vt + (long)vslot[tp] * n_ev * K;
  const long kchunks = (K + PBK - 1) / PBK;
  const long kc0 = kchunks * kpart / ksplit, kc1 = kchunks * (kpart + 1) / ksplit;
  double2* C = Cpart + (long)blockIdx.z * n_ev * N;
  for (long k0 = kc0 * PBK; k0 < kc1 * PBK; k0 += PBK) {
    // A tile: PBM x PBK; 256 threads load 512 entries (2 each)
    for (int e = threadIdx.x; e < PBM * PBK; e += 256) {
      int mm = e / PBK, kk = e % PBK;
      long k = k0 + kk;
      double2 v = make_double2(0.0, 0.0);
      if (m0 + mm < n_ev && k < K) v = A[(long)(m0 + mm) * K + k];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < PBN * PBK; e += 256) {
      int kk = e / PBN, nn = e % PBN;
      long k = k0 + kk;
      int n = n0 + nn;
      double2 v = make_double2(0.0, 0.0);
      if (n < N && k < K) {
        long s3 = k / 3;
        int a = (int)(k - s3 * 3);
        int alpha = n / nrhs, r = n - alpha * nrhs;
        long s = (long)tp * L3 + s3;
        int x = (int)(s3 % g.Lx), y = (int)((s3 / g.Lx) % g.Ly), zz = (int)(s3 / ((long)g.Lx * g.Ly));
        int par = (x + y + zz + tp) & 1;
        long cb = s >> 1;
        v = X[(long)par * 12 * g.Vh * nrhs + ((long)(alpha * 3 + a) * g.Vh + cb) * nrhs + r];
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < PBK; kk++) {
      cplx<double> a0 = {As[kk][ty].x, As[kk][ty].y}, a1 = {As[kk][ty + 16].x, As[kk][ty + 16].y};
      cplx<double> b0 = {Bs[kk][tx].x, Bs[kk][tx].y}, b1 = {Bs[kk][tx + 16].x, Bs[kk][tx + 16].y};
      acc[0][0] = acc[0][0] + cjmul(a0, b0);
      acc[0][1] = acc[0][1] + cjmul(a0, b1);
      acc[1][0] = acc[1][0] + cjmul(a1, b0);
      acc[1][1] = acc[1][1] + cjmul(a1, b1);
    }
    __syncthreads();
  }
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) {
      int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < n_ev && n < N) {
        int alpha = n / nrhs, r = n - alpha * nrhs;
        C[((long)m * 4 + alpha) * nrhs + r] = make_double2(acc[i][j].re, acc[i][j].im);
      }
    }
}

// ---- the same projection in double-float arithmetic on the FP32 pipe
// B300 issues FP32 at 64 times its FP64 rate, so the FP64 GEMM above is bound by a pipe the
// rest of the solver barely uses.  Here every FP64 input is split once into an unevaluated pair
// hi + lo of floats (hi = fl32(v), lo = fl32(v - hi): 48 significant bits), and the products are
// accumulated with error-free transformations in the "Dot2" manner of Ogita, Rump and Oishi
// (SIAM J. Sci. Comput. 26, 2005): TwoProduct by FMA (Dekker 1971) for the leading product, the
// cross terms hi*lo and lo*hi and all errors into a float correction, TwoSum (Knuth) into the
// leading float.  Every 512 terms the pair is added into an FP64 accumulator, which bounds the
// correction's own rounding; the split-K partials are summed in FP64 as before.

// One complex FP64 number as two float pairs: (re_hi, re_lo, im_hi, im_lo).
LQCD_D float4 split_c(double2 v) {
  const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
  return make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
}

// Vf[slot][i][k] = split(V[slot][i][k]) for the nslots x n_ev x K entries
__global__ void k_split_v(const double2* V, float4* Vf, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    Vf[i] = split_c(V[i]);
}

// Xf[z][n][k] = split(X_r(tp_z, s3, alpha, a)), n = alpha * nrhs + r, k = s3 * 3 + a: the solution on
// the sink timeslices, K contiguous per column
__global__ void k_split_x(const double2* X, const int* sinks, int nsinks, float4* Xf, Geom g, int nrhs) {
  const long L3 = (long)g.Lx * g.Ly * g.Lz, K = 3 * L3;
  const long n_all = (long)nsinks * 4 * nrhs * K;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n_all; i += (long)gridDim.x * blockDim.x) {
    const long k = i % K;
    const long zn = i / K;
    const int n = (int)(zn % (4 * nrhs)), z = (int)(zn / (4 * nrhs));
    const int tp = sinks[z];
    const long s3 = k / 3;
    const int a = (int)(k - s3 * 3);
    const int alpha = n / nrhs, r = n - alpha * nrhs;
    const int x = (int)(s3 % g.Lx), y = (int)((s3 / g.Lx) % g.Ly), zz = (int)(s3 / ((long)g.Lx * g.Ly));
    const int par = (x + y + zz + tp) & 1;
    const long cb = ((long)tp * L3 + s3) >> 1;
    Xf[i] = split_c(X[(long)par * 12 * g.Vh * nrhs + ((long)(alpha * 3 + a) * g.Vh + cb) * nrhs + r]);
  }
}

// hi + lo += a * b for a = ah + al, b = bh + bl (double-float multiply-accumulate)
LQCD_D void df_mac(float& hi, float& lo, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float e = __fmaf_rn(ah, bh, -p);  // TwoProduct: ah bh = p + e exactly
  const float s = __fadd_rn(hi, p);       // TwoSum: hi + p = s + err exactly
  const float bv = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(p, bv));
  hi = s;
  lo = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, __fadd_rn(lo, __fadd_rn(e, err))));
}

#define DFLUSH 32  // k-tiles of PBK between FP64 flushes (512 terms)
__global__ void __launch_bounds__(256) k_project_df(const float4* Vf, int n_ev, const float4* Xf, const int* sinks,
                                                    const int* vslot, double2* Cpart, Geom g, int nrhs, int ksplit) {
  __shared__ float4 As[PBK][PBM + 1];
  __shared__ float4 Bs[PBK][PBN + 1];
  const int z = blockIdx.z / ksplit, kpart = blockIdx.z - z * ksplit;
  const int tp = sinks[z];
  const long K = 3L * g.Lx * g.Ly * g.Lz;
  const int N = 4 * nrhs;
  const int m0 = blockIdx.y * PBM, n0 = blockIdx.x * PBN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float hr[2][2], lr[2][2], hi_[2][2], li[2][2];
  double ar[2][2], ai[2][2];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 2; j++) hr[i][j] = lr[i][j] = hi_[i][j] = li[i][j] = 0.f, ar[i][j] = ai[i][j] = 0.0;
  const float4* A = Vf + (long)vslot[tp] * n_ev * K;
  const float4* B = Xf + (long)z * N * K;
  const long kchunks = (K + PBK - 1) / PBK;
  const long kc0 = kchunks * kpart / ksplit, kc1 = kchunks * (kpart + 1) / ksplit;
  double2* C = Cpart + (long)blockIdx.z * n_ev * N;
  int since = 0;
  for (long k0 = kc0 * PBK; k0 < kc1 * PBK; k0 += PBK) {
    for (int e = threadIdx.x; e < PBM * PBK; e += 256) {
      const int mm = e / PBK, kk = e % PBK;
      const long k = k0 + kk;
      As[kk][mm] = (m0 + mm < n_ev && k < K) ? A[(long)(m0 + mm) * K + k] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int e = threadIdx.x; e < PBN * PBK; e += 256) {
      const int nn = e / PBK, kk = e % PBK;
      const long k = k0 + kk;
      Bs[kk][nn] = (n0 + nn < N && k < K) ? B[(long)(n0 + nn) * K + k] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < PBK; kk++) {
      const float4 a[2] = {As[kk][ty], As[kk][ty + 16]};
      const float4 b[2] = {Bs[kk][tx], Bs[kk][tx + 16]};
#pragma unroll
      for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) {  // conj(a) b: re = ar br + ai bi, im = ar bi - ai br
          df_mac(hr[i][j], lr[i][j], a[i].x, a[i].y, b[j].x, b[j].y);
          df_mac(hr[i][j], lr[i][j], a[i].z, a[i].w, b[j].z, b[j].w);
          df_mac(hi_[i][j], li[i][j], a[i].x, a[i].y, b[j].z, b[j].w);
          df_mac(hi_[i][j], li[i][j], -a[i].z, -a[i].w, b[j].x, b[j].y);
        }
    }
    __syncthreads();
    if (++since == DFLUSH) {
      since = 0;
#pragma unroll
      for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) {
          ar[i][j] += (double)hr[i][j] + (double)lr[i][j];
          ai[i][j] += (double)hi_[i][j] + (double)li[i][j];
          hr[i][j] = lr[i][j] = hi_[i][j] = li[i][j] = 0.f;
        }
    }
  }
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < n_ev && n < N) {
        const int alpha = n / nrhs, r = n - alpha * nrhs;
        C[((long)m * 4 + alpha) * nrhs + r] = make_double2(ar[i][j] + ((double)hr[i][j] + (double)lr[i][j]),
                                                           ai[i][j] + ((double)hi_[i][j] + (double)li[i][j]));
      }
    }
}

void split_colour_vectors(const double2* V, float4* Vf, long n, cudaStream_t st) {
  k_split_v<<<4 * 148, 256, 0, st>>>(V, Vf, n);
  lqcd::count_launch();
}

// C[z] = sum over kpart of Cpart[z * ksplit + kpart]
__global__ void k_project_sum(const double2* Cpart, double2* C, long per_z, int nsinks, int ksplit) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= per_z * nsinks) return;
  const long z = i / per_z, e = i - z * per_z;
  double re = 0, im = 0;
  for (int k = 0; k < ksplit; k++) {
    double2 v = Cpart[(z * ksplit + k) * per_z + e];
    re += v.x;
    im += v.y;
  }
  C[i] = make_double2(re, im);
}

int project_ksplit(const Geom& g, int n_ev, int nrhs, int nsinks, int blocks_per_sm) {
  const long tiles = (long)((4 * nrhs + PBN - 1) / PBN) * ((n_ev + PBM - 1) / PBM) * nsinks;
  const long kchunks = (3L * g.Lx * g.Ly * g.Lz + PBK - 1) / PBK;
  long ks = ((long)blocks_per_sm * 148 + tiles - 1) / tiles;  // about blocks_per_sm blocks per SM
  if (ks > kchunks) ks = kchunks;
  if (ks < 1) ks = 1;
  return (int)ks;
}

void project(const Geom& g, const double2* Vt, int n_ev, const double2* X, const int* sinks, const int* vslot,
             int nsinks, double2* C, double2* Cpart, int nrhs, int blocks_per_sm, bool high_priority,
             const float4* Vf, float4* Xf, cudaStream_t st) {
  const int ksplit = project_ksplit(g, n_ev, nrhs, nsinks, blocks_per_sm);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((4 * nrhs + PBN - 1) / PBN, (n_ev + PBM - 1) / PBM, nsinks * ksplit);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (high_priority) {  // placed before queued blocks of other streams (a batch in flight beside it)
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = hi;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  if (Vf && Xf) {  // double-float on the FP32 pipe: split the solution on the sinks, then the GEMM
    k_split_x<<<4 * 148, 256, 0, st>>>(X, sinks, nsinks, Xf, g, nrhs);
    lqcd::count_launch();
    cudaLaunchKernelEx(&cfg, k_project_df, (const float4*)Vf, n_ev, (const float4*)Xf, sinks, vslot, Cpart, g, nrhs,
                       ksplit);
  } else {
    cudaLaunchKernelEx(&cfg, k_project, Vt, n_ev, X, sinks, vslot, Cpart, g, nrhs, ksplit);
  }
  lqcd::count_launch();
  const long per_z = (long)n_ev * 4 * nrhs;
  k_project_sum<<<(per_z * nsinks + 255) / 256, 256, 0, st>>>(Cpart, C, per_z, nsinks, ksplit);
  lqcd::count_launch();
}

// ------------------------------------------------------------------ loops
// L[g][t] = sum_i w[t][i] sum_{ab} G[a][b] tau[t][i][b][i][a]; Lt with G~; G: [n_gamma][2][4][4]
__global__ void k_loops(const double2* tau, int n_ev, int n_t, const double2* G, int n_gamma, const double* w,
                        double2* L, double2* Lt) {
  const int gi = blockIdx.x, t = blockIdx.y;
  __shared__ double sm[4][128];
  cplx<double> l = {0, 0}, lt = {0, 0};
  for (int i = threadIdx.x; i < n_ev; i += blockDim.x) {
    double wi = w ? w[(long)t * n_ev + i] : 1.0;
    for (int a = 0; a < 4; a++)
      for (int b = 0; b < 4; b++) {
        double2 tv = tau[((((long)t * n_ev + i) * 4 + b) * n_ev + i) * 4 + a];
        double2 g = G[((gi * 2 + 0) * 4 + a) * 4 + b];
        double2 gt = G[((gi * 2 + 1) * 4 + a) * 4 + b];
        cplx<double> T = {tv.x, tv.y};
        l = l + wi * (cplx<double>{g.x, g.y} * T);
        lt = lt + wi * (cplx<double>{gt.x, gt.y} * T);
      }
  }
  sm[0][threadIdx.x] = l.re;
  sm[1][threadIdx.x] = l.im;
  sm[2][threadIdx.x] = lt.re;
  sm[3][threadIdx.x] = lt.im;
  __syncthreads();
  for (int s = blockDim.x / 2; s >= 1; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 4; k++) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    L[(long)gi * n_t + t] = make_double2(sm[0][0], sm[1][0]);
    Lt[(long)gi * n_t + t] = make_double2(sm[2][0], sm[3][0]);
  }
}

void loops(const double2* tau, int n_ev, int n_t, const double2* G, int n_gamma, const double* w, double2* L,
           double2* Lt, cudaStream_t st) {
  k_loops<<<dim3(n_gamma, n_t), 128, 0, st>>>(tau, n_ev, n_t, G, n_gamma, w, L, Lt); lqcd::count_launch();
}

// ------------------------------------------------------------------ connected correlator
// Quark-line connected part of Eq. Cfull with distilled quark lines:
//   C[g][x0][k] = - Tr[G tau(x0,y0) Gt tau(y0,x0)],  y0 = t_src[k],
// with tau(y0,x0)[j c][i d] = eps_c eps_d conj(tau(x0,y0)[i d][j c]) (gamma_5-hermiticity of D,
// eps = diag(gamma_5)), so only the perambulators of the sources y0 are read:
//   C = - sum_ij sum_abcd (eps_d G[d][a]) (Gt[b][c] eps_c) A[a][b] conj(A[d][c]),  A = tau(x0,y0)_ij.
// One block per (gamma, x0, source); threads over the eigenvector pairs (i, j).
__global__ void k_conn(const double2* tau, int n_ev, int T, int n_t, const double2* G, double2* C) {
  const int gi = blockIdx.x, x0 = blockIdx.y, k = blockIdx.z;
  __shared__ cplx<double> ge[4][4], gte[4][4];  // eps_d G[d][a], Gt[b][c] eps_c
  __shared__ double sm[2][128];
  if (threadIdx.x < 32) {
    const int w = threadIdx.x >> 4, r = (threadIdx.x >> 2) & 3, q = threadIdx.x & 3;
    const double2 v = G[((gi * 2 + w) * 4 + r) * 4 + q];
    const double e = w == 0 ? (r < 2 ? 1.0 : -1.0) : (q < 2 ? 1.0 : -1.0);
    if (w == 0)
      ge[r][q] = {e * v.x, e * v.y};
    else
      gte[r][q] = {e * v.x, e * v.y};
  }
  __syncthreads();
  const double2* base = tau + ((long)k * T + x0) * (long)n_ev * 4 * n_ev * 4;
  cplx<double> acc = {0, 0};
  for (int p = threadIdx.x; p < n_ev * n_ev; p += blockDim.x) {
    const int i = p / n_ev, j = p - i * n_ev;
    cplx<double> A[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int b = 0; b < 4; b++) {
        const double2 v = base[(((long)i * 4 + a) * n_ev + j) * 4 + b];
        A[a][b] = {v.x, v.y};
      }
    cplx<double> Q[4][4];  // Q[d][b] = sum_c conj(A[d][c]) gte[b][c]
#pragma unroll
    for (int d = 0; d < 4; d++)
#pragma unroll
      for (int b = 0; b < 4; b++) {
        cplx<double> q = {0, 0};
#pragma unroll
        for (int c = 0; c < 4; c++) q = q + cjmul(A[d][c], gte[b][c]);
        Q[d][b] = q;
      }
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int b = 0; b < 4; b++) {
        cplx<double> m = {0, 0};
#pragma unroll
        for (int d = 0; d < 4; d++) m = m + ge[d][a] * Q[d][b];
        acc = acc + A[a][b] * m;
      }
  }
  sm[0][threadIdx.x] = acc.re;
  sm[1][threadIdx.x] = acc.im;
  __syncthreads();
  for (int s = blockDim.x / 2; s >= 1; s >>= 1) {
    if (threadIdx.x < s) {
      sm[0][threadIdx.x] += sm[0][threadIdx.x + s];
      sm[1][threadIdx.x] += sm[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) C[((long)gi * T + x0) * n_t + k] = make_double2(-sm[0][0], -sm[1][0]);
}

// C_avg[g][dt] = mean over k of C[g][(t_src[k] + dt) mod T][k]
__global__ void k_conn_avg(const double2* C, const int* t_src, int n_t, int T, double2* C_avg) {
  const int gi = blockIdx.x;
  for (int dt = threadIdx.x; dt < T; dt += blockDim.x) {
    double re = 0, im = 0;
    for (int k = 0; k < n_t; k++) {
      const double2 v = C[((long)gi * T + (t_src[k] + dt) % T) * n_t + k];
      re += v.x;
      im += v.y;
    }
    C_avg[(long)gi * T + dt] = make_double2(re / n_t, im / n_t);
  }
}

void conn_correlator(const double2* tau, int n_ev, int T, const int* t_src_dev, int n_t, const double2* G,
                     int n_gamma, double2* C, double2* C_avg, cudaStream_t st) {
  k_conn<<<dim3(n_gamma, T, n_t), 128, 0, st>>>(tau, n_ev, T, n_t, G, C); lqcd::count_launch();
  if (C_avg) {
    k_conn_avg<<<n_gamma, 128, 0, st>>>(C, t_src_dev, n_t, T, C_avg);
    lqcd::count_launch();
  }
}

// Noise-reduced estimator (Sec. 4): C_nr[g][dt] = conn[g][dt] + dC[d][g][dt] for the block size
// d = delta_of_dt[dt] chosen for the separation, or + disc[g][dt] (standard estimator) if d < 0.
__global__ void k_nr(const double2* conn, const double2* disc, const double2* dC, int n_gamma, int T,
                     const int* delta_of_dt, double2* out) {
  const long n = (long)n_gamma * T;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int dt = (int)(e % T);
    const int d = delta_of_dt[dt];
    const double2 a = conn[e], b = d >= 0 ? dC[(long)d * n + e] : disc[e];
    out[e] = make_double2(a.x + b.x, a.y + b.y);
  }
}

void nr_estimator(const double2* conn, const double2* disc, const double2* dC, int n_gamma, int T,
                  const int* delta_of_dt_dev, double2* out, cudaStream_t st) {
  const long n = (long)n_gamma * T;
  k_nr<<<(int)((n + 127) / 128), 128, 0, st>>>(conn, disc, dC, n_gamma, T, delta_of_dt_dev, out);
  lqcd::count_launch();
}

// ------------------------------------------------------------------ correlators
// conn(A, B)[g][x0][y0] = <A(x0) B(y0)> - vev * <A(x0)> <B(y0)>
LQCD_D cplx<double> conn(const double2* A, const double2* B, int n_cfg, int n_g, int T, int g, int x0, int y0,
                         int vev) {
  cplx<double> ab = {0, 0}, ma = {0, 0}, mb = {0, 0};
  for (int c = 0; c < n_cfg; c++) {
    double2 a = A[((long)c * n_g + g) * T + x0], b = B[((long)c * n_g + g) * T + y0];
    cplx<double> ca = {a.x, a.y}, cb = {b.x, b.y};
    ab = ab + ca * cb;
    ma = ma + ca;
    mb = mb + cb;
  }
  double inv = 1.0 / n_cfg;
  cplx<double> r = inv * ab;
  if (vev) r = r - (inv * ma) * (inv * mb);
  return r;
}

__global__ void k_corr(const double2* L, const double2* Lt, const double2* Ld, const double2* Ltd, int n_cfg, int n_g,
                       int T, int vev, const int* dom, double2* C, double2* Cdd, double2* dC, int* valid,
                       double2* terms, double2* dL, double2* dLt) {
  const int g = blockIdx.x;
  const int x0 = blockIdx.y;
  const int y0 = threadIdx.x;
  if (y0 >= T) return;
  cplx<double> c = conn(L, Lt, n_cfg, n_g, T, g, x0, y0, vev);
  cplx<double> cd = conn(Ld, Ltd, n_cfg, n_g, T, g, x0, y0, vev);
  long o = ((long)g * T + x0) * T + y0;
  C[o] = make_double2(c.re, c.im);
  Cdd[o] = make_double2(cd.re, cd.im);
  dC[o] = make_double2(c.re - cd.re, c.im - cd.im);
  if (g == 0) valid[x0 * T + y0] = dom[x0] != dom[y0];
  if (terms) {
    long q = (long)n_g * T * T;
    cplx<double> t1 = conn(Ld, dLt, n_cfg, n_g, T, g, x0, y0, vev);
    cplx<double> t2 = conn(dL, Ltd, n_cfg, n_g, T, g, x0, y0, vev);
    cplx<double> t3 = conn(dL, dLt, n_cfg, n_g, T, g, x0, y0, vev);
    terms[o] = make_double2(cd.re, cd.im);
    terms[q + o] = make_double2(t1.re, t1.im);
    terms[2 * q + o] = make_double2(t2.re, t2.im);
    terms[3 * q + o] = make_double2(t3.re, t3.im);
  }
}

__global__ void k_diff(const double2* a, const double2* b, double2* c, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = make_double2(a[i].x - b[i].x, a[i].y - b[i].y);
}

__global__ void k_corr_avg(const double2* C, const double2* dC, const int* dom, int n_g, int T, double2* C_avg,
                           double2* dC_avg, int* n_valid) {
  const int g = blockIdx.x;
  const int dt = threadIdx.x;
  if (dt >= T) return;
  cplx<double> s = {0, 0}, sd = {0, 0};
  int nv = 0;
  for (int y0 = 0; y0 < T; y0++) {
    int x0 = (y0 + dt) % T;
    long o = ((long)g * T + x0) * T + y0;
    s = s + cplx<double>{C[o].x, C[o].y};
    if (dom[x0] != dom[y0]) {
      sd = sd + cplx<double>{dC[o].x, dC[o].y};
      nv++;
    }
  }
  C_avg[(long)g * T + dt] = make_double2(s.re / T, s.im / T);
  dC_avg[(long)g * T + dt] = nv ? make_double2(sd.re / nv, sd.im / nv) : make_double2(0.0, 0.0);
  if (g == 0) n_valid[dt] = nv;
}

// Bulk-window averages: source and sink both in [t_lo, t_hi], x0 = y0 + dt without wrap-around;
// one thread per (gamma, dt).  n_pairs / n_valid: pairs in the window / of those in distinct domains.
__global__ void k_window_avg(const double2* C, const double2* dC, const int* valid, int n_g, int T, int t_lo,
                             int t_hi, double2* C_avg, double2* dC_avg, int* n_pairs, int* n_valid) {
  const int g = blockIdx.x;
  const int dt = threadIdx.x;
  if (dt >= T) return;
  cplx<double> s = {0, 0}, sd = {0, 0};
  int np = 0, nv = 0;
  for (int y0 = t_lo; y0 + dt <= t_hi; y0++) {
    const int x0 = y0 + dt;
    const long o = ((long)g * T + x0) * T + y0;
    s = s + cplx<double>{C[o].x, C[o].y};
    np++;
    if (valid[(long)x0 * T + y0]) {
      sd = sd + cplx<double>{dC[o].x, dC[o].y};
      nv++;
    }
  }
  C_avg[(long)g * T + dt] = np ? make_double2(s.re / np, s.im / np) : make_double2(0.0, 0.0);
  dC_avg[(long)g * T + dt] = nv ? make_double2(sd.re / nv, sd.im / nv) : make_double2(0.0, 0.0);
  if (g == 0) {
    n_pairs[dt] = np;
    n_valid[dt] = nv;
  }
}

void window_average(const double2* C, const double2* dC, const int* valid, int n_g, int T, int t_lo, int t_hi,
                    double2* C_avg, double2* dC_avg, int* n_pairs, int* n_valid, cudaStream_t st) {
  k_window_avg<<<n_g, ((T + 31) / 32) * 32, 0, st>>>(C, dC, valid, n_g, T, t_lo, t_hi, C_avg, dC_avg, n_pairs,
                                                     n_valid);
  lqcd::count_launch();
}

void correlators(const double2* L, const double2* Lt, const double2* Ld, const double2* Ltd, int n_cfg, int n_g,
                 int T, int vev, const int* dom, double2* C, double2* Cdd, double2* dC, double2* C_avg,
                 double2* dC_avg, int* valid, int* n_valid, double2* terms, double2* dL, double2* dLt,
                 cudaStream_t st) {
  long n = (long)n_cfg * n_g * T;
  if (terms) {
    k_diff<<<(n + 255) / 256, 256, 0, st>>>(L, Ld, dL, n); lqcd::count_launch();
    k_diff<<<(n + 255) / 256, 256, 0, st>>>(Lt, Ltd, dLt, n); lqcd::count_launch();
  }
  k_corr<<<dim3(n_g, T), ((T + 31) / 32) * 32, 0, st>>>(L, Lt, Ld, Ltd, n_cfg, n_g, T, vev, dom, C, Cdd, dC, valid,
                                                        terms, dL, dLt); lqcd::count_launch();
  k_corr_avg<<<n_g, ((T + 31) / 32) * 32, 0, st>>>(C, dC, dom, n_g, T, C_avg, dC_avg, n_valid); lqcd::count_launch();
}

}  // namespace lqcd
