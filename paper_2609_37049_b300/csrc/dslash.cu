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
#include "dslash_ops.cuh"

namespace lqcd {

// MINB: minimum resident blocks of 128 threads the compiler must allow (register cap 255 / 168 /
// 128 / 80 / 64 per thread for MINB = 2 / 3 / 4 / 6 / 8).  Launch variants 0-2 are this kernel
// with MINB 4 / 6 / 8 (FP64: 4 / 2 / 3);
// variants 3-7 are the staged kernels of dslash_staged.cu and dslash_rb2.cu (3: links and clover
// staged once per site in shared memory; 4: neighbour spinors staged by bulk copies; 5: as 3 on
// paired FP32 arithmetic; 6: as 3 with per-thread asynchronous spinor copies; 7: two right-hand
// sides per thread on paired FP32 arithmetic) where they apply (FP32 /
// FP16, the solver's epilogues, RHS counts as stated there), else variant 0.  The autotuner picks
// the variant per precision and RHS count.
template <int P, int EPI, bool DAG, int RED>
LQCD_D void dslash_body(const DslashParams& pr, const long tid) {
  using R = typename Traits<P>::real;
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

  dslash_epilogue<P, EPI, RED>(pr, cb, idx, stride, rhs, acc);
}

template <int P, int EPI, bool DAG, int RED, int MINB>
__global__ void __launch_bounds__(128, MINB) dslash_kernel(const DslashParams pr) {
  dslash_body<P, EPI, DAG, RED>(pr, (long)blockIdx.x * blockDim.x + threadIdx.x);
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
  if constexpr (P != P64) {  // FP32 / FP16: tighter register caps for more resident warps
    if (variant == 1) return launch_v<P, EPI, RED, 6>(pr, dag, blocks, tpb, shm, st);
    if (variant == 2) return launch_v<P, EPI, RED, 8>(pr, dag, blocks, tpb, shm, st);
  } else {  // FP64 (bound by the FP64 pipe, which few warps keep busy): looser caps, no spills
    if (variant == 1) return launch_v<P, EPI, RED, 2>(pr, dag, blocks, tpb, shm, st);
    if (variant == 2) return launch_v<P, EPI, RED, 3>(pr, dag, blocks, tpb, shm, st);
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
  pr.pipe_off = 0;
  const bool dag = c.dagger != 0;
  if (variant < 0 || variant > 7) variant = 0;
  if (c.red == RED_NONE) {
    long nthreads = g.Vh * (long)c.nrhs;
    const int tpb = 128;
    const long blocks = (nthreads + tpb - 1) / tpb;
    if (variant >= 3) {  // staged kernels (dslash_staged.cu), where they apply
      if (launch_dslash_staged(pr, c.prec, c.epi, dag, RED_NONE, blocks, tpb, 0, variant, st)) return;
      variant = 0;
    }
    launch_prec<RED_NONE>(c.prec, pr, c.epi, dag, blocks, tpb, 0, variant, st);
  } else {
    // one block = red_sites sites (inside one timeslice) x nrhs right-hand sides (<= 128 threads)
    const int tpb = c.red_sites * c.nrhs;
    const long blocks = g.Vh / c.red_sites;
    const int nd = c.red == RED_DOT_Z ? 2 : (c.red == RED_TS_R0 ? 8 : 3);
    const size_t shm = (size_t)nd * tpb * sizeof(double);
    if (variant >= 3) {
      if (launch_dslash_staged(pr, c.prec, c.epi, dag, c.red, blocks, tpb, shm, variant, st)) return;
      variant = 0;
    }
    if (c.red == RED_DOT_Z)
      launch_prec<RED_DOT_Z>(c.prec, pr, c.epi, dag, blocks, tpb, shm, variant, st);
    else if (c.red == RED_TS_R0)
      launch_prec<RED_TS_R0>(c.prec, pr, c.epi, dag, blocks, tpb, shm, variant, st);
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
