// Even-odd dslash kernels (same operator and epilogues as dslash.cu) that stage per-site data in
// shared memory, selected by the dslash launch variant:
//
// * variant 3 (dslash_sl_kernel): the eight links of every site of the block are loaded and their
//   third rows rebuilt once per site by a few threads, and the site's clover blocks copied once,
//   into shared memory; the hopping threads then read them as broadcasts instead of each
//   rebuilding the links (the direct kernel repeats the rebuild for every right-hand side).  Site
//   and element indices are 32-bit (the host checks that the fields fit).  Register cap 80.
// * variant 4 (dslash_pipe_kernel): the eight neighbour spinors of every output site staged by
//   bulk asynchronous copies (cp.async.bulk, completion counted on an mbarrier) 3 hops ahead of
//   the arithmetic.  One warp = 32 right-hand sides of one output site (nrhs a multiple of 32),
//   so the warp's share of one 16-byte chunk of a neighbour spinor is one contiguous 512-byte run
//   of the RHS-innermost layout and lane 0 copies all of them for the warp.  Every mbarrier wait
//   has an iteration limit; a wait that runs out is counted in a device counter (read by
//   dslash_pipe_timeouts) and the kernel finishes without waiting further.
#include "dslash_ops.cuh"

namespace lqcd {

__device__ unsigned long long g_pipe_timeouts;

namespace {

constexpr int kWaitLimit = 1 << 22;
constexpr uint32_t kRun = 32 * 16;  // bytes of one chunk for the 32 right-hand sides of a warp

// shared memory of one warp: NS stages of CH chunks, then the NS mbarriers in a 128-byte tail
template <int P, int NS>
constexpr uint32_t warp_bytes() {
  return NS * Traits<P>::SCHUNKS * kRun + 128;
}

LQCD_D uint32_t smem_addr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

LQCD_D void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

LQCD_D void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// orders this warp's earlier generic-proxy reads of a stage before the async-proxy refill
LQCD_D void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

LQCD_D void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
      "r"(bytes)
      : "memory");
}

LQCD_D void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

LQCD_D bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

LQCD_D bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kWaitLimit; i++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// The spinor of this lane from a staged hop (CH chunks, kRun bytes apart).
template <int P>
LQCD_D void load_staged(const unsigned char* base, cplx<typename Traits<P>::real> (&s)[12]) {
  if constexpr (P == P32) {
#pragma unroll
    for (int c = 0; c < 6; c++) {
      const float4 v = *reinterpret_cast<const float4*>(base + c * kRun);
      s[2 * c] = {v.x, v.y};
      s[2 * c + 1] = {v.z, v.w};
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const uint4 v = *reinterpret_cast<const uint4*>(base + c * kRun);
      const float2 a = h2f(v.x), b = h2f(v.y), d = h2f(v.z), e = h2f(v.w);
      s[4 * c] = {a.x, a.y};
      s[4 * c + 1] = {b.x, b.y};
      s[4 * c + 2] = {d.x, d.y};
      s[4 * c + 3] = {e.x, e.y};
    }
  }
}

struct Stage {
  unsigned char* wb;  // this warp's staging buffers (generic address)
  uint32_t buf;       // same, shared-window address
  uint32_t bar;       // NS mbarriers after the buffers
  const char* in;     // input spinor field
  long first;         // nrhs-index of the warp's first right-hand side
  long stride;        // chunk stride of the field, in 16-byte units
  int nrhs;
};

// lane 0: copy hop k's neighbour spinor (neighbour cb index nbk) into stage k % NS
template <int P, int NS>
LQCD_D void issue(const Stage& sg, int k, long nbk) {
  constexpr int CH = Traits<P>::SCHUNKS;
  const int st = k % NS;
  const uint32_t bar = sg.bar + 8u * st;
  mbar_expect_tx(bar, CH * kRun);
  const char* src = sg.in + (nbk * sg.nrhs + sg.first) * 16;
#pragma unroll
  for (int c = 0; c < CH; c++) bulk_g2s(sg.buf + (st * CH + c) * kRun, src + c * sg.stride * 16, kRun, bar);
}

template <int P, bool DAG, int NS, int K>
LQCD_D void pipe_hop(const DslashParams& pr, const Stage& sg, long cb, const long (&nb)[8], int coef, int lane,
                     bool& ok, cplx<typename Traits<P>::real> (&acc)[12]) {
  using R = typename Traits<P>::real;
  constexpr int CH = Traits<P>::SCHUNKS;
  constexpr int ST = K % NS;
  if (ok) ok = mbar_wait(sg.bar + 8u * ST, (K / NS) & 1);
  cplx<R> p[12];
  load_staged<P>(sg.wb + ST * CH * kRun + lane * 16, p);
  __syncwarp();
  if constexpr (K + NS < 8) {
    if (lane == 0 && ok) {
      fence_proxy_async();
      issue<P, NS>(sg, K + NS, nb[K + NS]);
    }
  }
  if (coef != 0) hop_one<P, K / 2, (K % 2) == 0, DAG>(pr, cb, nb[K], coef, p, acc);
}

template <int P, int EPI, bool DAG, int RED, int NS>
__global__ void __launch_bounds__(128, 4) dslash_pipe_kernel(const DslashParams pr) {
  using R = typename Traits<P>::real;
  constexpr int CH = Traits<P>::SCHUNKS;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long cb = tid / pr.nrhs;
  const int rhs = (int)(tid - cb * pr.nrhs);
  if (RED == RED_NONE && cb >= pr.g.Vh) return;  // whole warps: nrhs is a multiple of 32
  const Geom& g = pr.g;
  const unsigned cw = __ldg(pr.coord + cb);
  const int x = cw & 0xff, y = (cw >> 8) & 0xff, z = (cw >> 16) & 0xff, t = cw >> 24;
  const long sy = g.Lx, sz = (long)g.Lx * g.Ly, sw = sz * g.Lz;
  const long s = x + sy * y + sz * z + sw * t;
  const long stride = g.Vh * pr.nrhs;
  const long idx = cb * pr.nrhs + rhs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // neighbour checkerboard indices: hop 2 mu = s + mu, hop 2 mu + 1 = s - mu (periodic wrap)
  long nb[8];
  nb[0] = (s + (x + 1 == g.Lx ? 1 - g.Lx : 1)) >> 1;
  nb[1] = (s + (x == 0 ? g.Lx - 1 : -1)) >> 1;
  nb[2] = (s + (y + 1 == g.Ly ? sy * (1 - g.Ly) : sy)) >> 1;
  nb[3] = (s + (y == 0 ? sy * (g.Ly - 1) : -sy)) >> 1;
  nb[4] = (s + (z + 1 == g.Lz ? sz * (1 - g.Lz) : sz)) >> 1;
  nb[5] = (s + (z == 0 ? sz * (g.Lz - 1) : -sz)) >> 1;
  nb[6] = (s + (t + 1 == g.Lt ? sw * (1 - g.Lt) : sw)) >> 1;
  nb[7] = (s + (t == 0 ? sw * (g.Lt - 1) : -sw)) >> 1;
  const int cf = __ldg(pr.tc + t), cbk = __ldg(pr.tc + (t == 0 ? g.Lt - 1 : t - 1));

  extern __shared__ __align__(128) unsigned char dsm[];
  Stage sg;
  sg.wb = dsm + pr.pipe_off + warp * warp_bytes<P, NS>();
  sg.buf = smem_addr(sg.wb);
  sg.bar = sg.buf + NS * CH * kRun;
  sg.in = reinterpret_cast<const char*>(pr.in);
  sg.first = rhs - lane;
  sg.stride = stride;
  sg.nrhs = pr.nrhs;
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NS; j++) mbar_init(sg.bar + 8u * j, 1);
    mbar_fence_init();
#pragma unroll
    for (int k = 0; k < NS; k++) issue<P, NS>(sg, k, nb[k]);
  }
  __syncwarp();

  cplx<R> acc[12];
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = {R(0), R(0)};
  bool ok = true;
  pipe_hop<P, DAG, NS, 0>(pr, sg, cb, nb, 1, lane, ok, acc);
  pipe_hop<P, DAG, NS, 1>(pr, sg, cb, nb, 1, lane, ok, acc);
  pipe_hop<P, DAG, NS, 2>(pr, sg, cb, nb, 1, lane, ok, acc);
  pipe_hop<P, DAG, NS, 3>(pr, sg, cb, nb, 1, lane, ok, acc);
  pipe_hop<P, DAG, NS, 4>(pr, sg, cb, nb, 1, lane, ok, acc);
  pipe_hop<P, DAG, NS, 5>(pr, sg, cb, nb, 1, lane, ok, acc);
  pipe_hop<P, DAG, NS, 6>(pr, sg, cb, nb, cf, lane, ok, acc);
  pipe_hop<P, DAG, NS, 7>(pr, sg, cb, nb, cbk, lane, ok, acc);
  if (!ok) atomicAdd(&g_pipe_timeouts, 1ull);

  dslash_epilogue<P, EPI, RED>(pr, cb, idx, stride, rhs, acc);
}

// ------------------------------------------------------------------ staged links and clover

// 32-bit addressing of a spinor chunk field: chunk c of element idx at base + c * stride + idx.
template <int P>
LQCD_D void load_spinor32(const void* base, int stride, int idx, cplx<float> (&s)[12]) {
  if constexpr (P == P32) {
    const float4* f = reinterpret_cast<const float4*>(base) + idx;
#pragma unroll
    for (int c = 0; c < 6; c++) {
      const float4 v = __ldg(f + c * stride);
      s[2 * c] = {v.x, v.y};
      s[2 * c + 1] = {v.z, v.w};
    }
  } else {
    const uint4* f = reinterpret_cast<const uint4*>(base) + idx;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const uint4 v = __ldg(f + c * stride);
      const float2 a = h2f(v.x), b = h2f(v.y), d = h2f(v.z), e = h2f(v.w);
      s[4 * c] = {a.x, a.y};
      s[4 * c + 1] = {b.x, b.y};
      s[4 * c + 2] = {d.x, d.y};
      s[4 * c + 3] = {e.x, e.y};
    }
  }
}

// a full 3x3 link stored as 5 float4 (18 floats row-major + 2 pad)
LQCD_D void link_from_shared(const float4* L, cplx<float> (&u)[3][3]) {
  const float4 a = L[0], b = L[1], c = L[2], d = L[3], e = L[4];
  u[0][0] = {a.x, a.y}; u[0][1] = {a.z, a.w}; u[0][2] = {b.x, b.y};
  u[1][0] = {b.z, b.w}; u[1][1] = {c.x, c.y}; u[1][2] = {c.z, c.w};
  u[2][0] = {d.x, d.y}; u[2][1] = {d.z, d.w}; u[2][2] = {e.x, e.y};
}

// forward and backward hop along MU with the links from shared memory (lf: U_mu(s), lb: U_mu(s-mu))
template <int P, int MU>
LQCD_D void hop_dir_sl(const DslashParams& pr, int s, int cmu, int Lmu, int smu, int coef_f, int coef_b, int rhs,
                       int stride, int nrhs, const float4* lf, const float4* lb, cplx<float> (&acc)[12]) {
  constexpr int SF = -1;  // H (not H^dag): forward projector 1 - gamma_mu
  constexpr int SB = 1;
  if (coef_f != 0) {
    const int sn = s + ((cmu + 1 == Lmu) ? smu * (1 - Lmu) : smu);
    cplx<float> p[12], h[2][3], w[2][3], u[3][3];
    load_spinor32<P>(pr.in, stride, (sn >> 1) * nrhs + rhs, p);
    project<MU, SF>(p, h);
    link_from_shared(lf, u);
    su3_mul(u, h, w);
    if (coef_f < 0) {
#pragma unroll
      for (int q = 0; q < 2; q++)
#pragma unroll
        for (int a = 0; a < 3; a++) w[q][a] = -w[q][a];
    }
    accumulate<MU, SF>(acc, w);
  }
  if (coef_b != 0) {
    const int sn = s + ((cmu == 0) ? smu * (Lmu - 1) : -smu);
    cplx<float> p[12], h[2][3], w[2][3], u[3][3];
    load_spinor32<P>(pr.in, stride, (sn >> 1) * nrhs + rhs, p);
    project<MU, SB>(p, h);
    link_from_shared(lb, u);
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

constexpr int kMaxSites = 16;  // sites per 128-thread block: nrhs >= 8

// Blocks of 128 threads = S = 128 / nrhs sites x nrhs right-hand sides (nrhs a power of two in
// [8, 128]); block b holds sites b S .. b S + S - 1.
template <int P, int EPI, int RED, int MINB>
__global__ void __launch_bounds__(128, MINB) dslash_sl_kernel(const DslashParams pr) {
  __shared__ float4 slink[kMaxSites][8][5];  // [site][hop: 2 mu (fwd), 2 mu + 1 (bwd)][link]
  __shared__ float4 sclov[kMaxSites][18];    // [site][chirality x 9 packed chunks]
  const Geom& g = pr.g;
  const int nr = pr.nrhs;
  const int lg = __ffs(nr) - 1;
  const int S = 128 >> lg;
  const int cb0 = blockIdx.x * S;
  const int Vh = (int)g.Vh;
  const int sy = g.Lx, sz = g.Lx * g.Ly, sw = sz * g.Lz;
  for (int j = threadIdx.x; j < 26 * S; j += 128) {
    if (j < 8 * S) {  // link j & 7 of site j >> 3, third row rebuilt once
      const int site = j >> 3, k = j & 7, c = cb0 + site;
      if (c < Vh) {
        const int mu = k >> 1;
        int lcb = c, par = pr.out_par;
        if (k & 1) {  // backward hop: the link of the neighbour s - mu (coordinates by
                      // arithmetic, not the table, so the link load is the only global latency)
          const int xh = c % g.Lxh, yzt = c / g.Lxh, y = yzt % g.Ly, zt = yzt / g.Ly, z = zt % g.Lz,
                    t = zt / g.Lz;
          const int x = 2 * xh + ((pr.out_par + y + z + t) & 1);
          const int s = x + sy * y + sz * z + sw * t;
          const int cm = mu == 0 ? x : (mu == 1 ? y : (mu == 2 ? z : t));
          const int Lm = mu == 0 ? g.Lx : (mu == 1 ? g.Ly : (mu == 2 ? g.Lz : g.Lt));
          const int sm = mu == 0 ? 1 : (mu == 1 ? sy : (mu == 2 ? sz : sw));
          lcb = (s + (cm == 0 ? sm * (Lm - 1) : -sm)) >> 1;
          par = 1 - pr.out_par;
        }
        cplx<float> u[3][3];
        load_link<P>(pr.U, g.Vh, mu, par, lcb, u);
        float4* L = slink[site][k];
        L[0] = make_float4(u[0][0].re, u[0][0].im, u[0][1].re, u[0][1].im);
        L[1] = make_float4(u[0][2].re, u[0][2].im, u[1][0].re, u[1][0].im);
        L[2] = make_float4(u[1][1].re, u[1][1].im, u[1][2].re, u[1][2].im);
        L[3] = make_float4(u[2][0].re, u[2][0].im, u[2][1].re, u[2][1].im);
        L[4] = make_float4(u[2][2].re, u[2][2].im, 0.f, 0.f);
      }
    } else {  // clover chunk e of site q / 18
      const int q = j - 8 * S, site = q / 18, e = q - site * 18, c = cb0 + site;
      if (c < Vh) {
        if constexpr (P == P32) {
          sclov[site][e] = __ldg(reinterpret_cast<const float4*>(pr.C) + (long)e * Vh + c);
        } else {
          const uint2 v = __ldg(reinterpret_cast<const uint2*>(pr.C) + (long)e * Vh + c);
          const float2 a = h2f(v.x), b = h2f(v.y);
          sclov[site][e] = make_float4(a.x, a.y, b.x, b.y);
        }
      }
    }
  }
  const int tid = blockIdx.x * 128 + threadIdx.x;
  const int cb = tid >> lg;
  const int rhs = tid & (nr - 1);
  const unsigned cw = cb < Vh ? __ldg(pr.coord + cb) : 0u;  // issued before the barrier
  __syncthreads();

  if (RED == RED_NONE && cb >= Vh) return;
  const int sl = threadIdx.x >> lg;
  const int x = cw & 0xff, y = (cw >> 8) & 0xff, z = (cw >> 16) & 0xff, t = cw >> 24;
  const int s = x + sy * y + sz * z + sw * t;
  const int stride = Vh * nr;

  cplx<float> acc[12];
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = {0.f, 0.f};
  hop_dir_sl<P, 0>(pr, s, x, g.Lx, 1, 1, 1, rhs, stride, nr, slink[sl][0], slink[sl][1], acc);
  hop_dir_sl<P, 1>(pr, s, y, g.Ly, sy, 1, 1, rhs, stride, nr, slink[sl][2], slink[sl][3], acc);
  hop_dir_sl<P, 2>(pr, s, z, g.Lz, sz, 1, 1, rhs, stride, nr, slink[sl][4], slink[sl][5], acc);
  const int cf = __ldg(pr.tc + t), cbk = __ldg(pr.tc + (t == 0 ? g.Lt - 1 : t - 1));
  hop_dir_sl<P, 3>(pr, s, t, g.Lt, sw, cf, cbk, rhs, stride, nr, slink[sl][6], slink[sl][7], acc);
  dslash_epilogue<P, EPI, RED, true>(pr, cb, (long)cb * nr + rhs, (long)stride, rhs, acc, sclov[sl]);
}

template <int P, int EPI, int RED, int MINB>
void launch_sl(const DslashParams& pr, long blocks, size_t shm, cudaStream_t st) {
  dslash_sl_kernel<P, EPI, RED, MINB><<<blocks, 128, shm, st>>>(pr);
  lqcd::count_launch();
}

template <int P, int MINB>
bool launch_sl_e(const DslashParams& pr, int epi, int red, long blocks, size_t shm, cudaStream_t st) {
  if (red == RED_TS_R0) {
    if (epi != EPI_Y_CH) return false;
    launch_sl<P, EPI_Y_CH, RED_TS_R0, MINB>(pr, blocks, shm, st);
  } else if (red == RED_DOT_Z) {
    if (epi != EPI_Y_CH) return false;
    launch_sl<P, EPI_Y_CH, RED_DOT_Z, MINB>(pr, blocks, shm, st);
  } else if (red == RED_DOT_Y_NORM) {
    if (epi != EPI_Y_CH) return false;
    launch_sl<P, EPI_Y_CH, RED_DOT_Y_NORM, MINB>(pr, blocks, shm, st);
  } else if (epi == EPI_CH) {
    launch_sl<P, EPI_CH, RED_NONE, MINB>(pr, blocks, shm, st);
  } else if (epi == EPI_Y_CH) {
    launch_sl<P, EPI_Y_CH, RED_NONE, MINB>(pr, blocks, shm, st);
  } else if (epi == EPI_C_YH) {
    launch_sl<P, EPI_C_YH, RED_NONE, MINB>(pr, blocks, shm, st);
  } else {
    return false;
  }
  return true;
}

// ------------------------------------------------------------------ bulk-copy staged spinors

// largest dynamic shared memory of a launch: 128 threads, 3-double reduction scratch per thread
template <int P, int NS>
constexpr size_t max_shm() {
  return 3 * 128 * sizeof(double) + 4 * warp_bytes<P, NS>();
}

template <int P, int EPI, int RED, int NS>
void open_k() {
  cudaFuncSetAttribute(dslash_pipe_kernel<P, EPI, false, RED, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)max_shm<P, NS>());
}

template <int P, int NS>
void open_ns() {
  open_k<P, EPI_Y_CH, RED_DOT_Z, NS>();
  open_k<P, EPI_Y_CH, RED_DOT_Y_NORM, NS>();
  open_k<P, EPI_CH, RED_NONE, NS>();
  open_k<P, EPI_Y_CH, RED_NONE, NS>();
  open_k<P, EPI_C_YH, RED_NONE, NS>();
}

// Raise the dynamic shared-memory limit of every instantiation once, before any launch (and so
// before any stream capture).
void open_all() {
  static bool done = false;
  if (done) return;
  done = true;
  open_ns<P32, 3>();
  open_ns<P16, 3>();
}

template <int P, int EPI, int RED, int NS>
void launch_k(const DslashParams& pr, long blocks, int tpb, size_t shm, cudaStream_t st) {
  dslash_pipe_kernel<P, EPI, false, RED, NS><<<blocks, tpb, shm, st>>>(pr);
  lqcd::count_launch();
}

template <int P, int NS>
bool launch_ns(const DslashParams& pr, int epi, int red, long blocks, int tpb, size_t shm, cudaStream_t st) {
  if (red != RED_NONE && red != RED_DOT_Z && red != RED_DOT_Y_NORM) return false;  // direct kernel instead
  if (red == RED_DOT_Z) {
    if (epi != EPI_Y_CH) return false;
    launch_k<P, EPI_Y_CH, RED_DOT_Z, NS>(pr, blocks, tpb, shm, st);
  } else if (red == RED_DOT_Y_NORM) {
    if (epi != EPI_Y_CH) return false;
    launch_k<P, EPI_Y_CH, RED_DOT_Y_NORM, NS>(pr, blocks, tpb, shm, st);
  } else if (epi == EPI_CH) {
    launch_k<P, EPI_CH, RED_NONE, NS>(pr, blocks, tpb, shm, st);
  } else if (epi == EPI_Y_CH) {
    launch_k<P, EPI_Y_CH, RED_NONE, NS>(pr, blocks, tpb, shm, st);
  } else if (epi == EPI_C_YH) {
    launch_k<P, EPI_C_YH, RED_NONE, NS>(pr, blocks, tpb, shm, st);
  } else {
    return false;
  }
  return true;
}

template <int P>
bool launch_p(const DslashParams& pr, int epi, int red, long blocks, int tpb, size_t red_shm, int ns,
              cudaStream_t st) {
  DslashParams q = pr;
  q.pipe_off = (int)((red_shm + 127) / 128 * 128);
  if (tpb > 128 || red_shm > 3 * 128 * sizeof(double)) return false;
  (void)ns;
  return launch_ns<P, 3>(q, epi, red, blocks, tpb, q.pipe_off + (tpb / 32) * warp_bytes<P, 3>(), st);
}

}  // namespace

bool launch_dslash_staged(const DslashParams& pr, int prec, int epi, bool dag, int red, long blocks, int tpb,
                          size_t red_shm, int variant, cudaStream_t st) {
  if (prec == P64 || dag || variant < 3 || variant > 4) return false;
  const long nr = pr.nrhs;
  if (variant == 4) {  // bulk-copy staged spinors, staging depth 3
    if (nr % 32 != 0 || tpb % 32 != 0) return false;
    open_all();
    if (prec == P32) return launch_p<P32>(pr, epi, red, blocks, tpb, red_shm, 3, st);
    return launch_p<P16>(pr, epi, red, blocks, tpb, red_shm, 3, st);
  }
  // staged links and clover: 128-thread blocks of 128 / nrhs whole sites, 32-bit indices
  if (nr < 8 || nr > 128 || (nr & (nr - 1)) != 0 || tpb != 128) return false;
  if (pr.g.Vh % (128 / nr) != 0 || blocks * (128 / nr) != pr.g.Vh) return false;
  if (12 * pr.g.Vh * nr >= (1L << 31)) return false;
  if (prec == P32) return launch_sl_e<P32, 6>(pr, epi, red, blocks, red_shm, st);
  return launch_sl_e<P16, 6>(pr, epi, red, blocks, red_shm, st);
}

unsigned long long dslash_pipe_timeouts(bool reset) {
  unsigned long long n = 0;
  cudaMemcpyFromSymbol(&n, g_pipe_timeouts, sizeof(n));
  if (reset && n) {
    const unsigned long long z = 0;
    cudaMemcpyToSymbol(g_pipe_timeouts, &z, sizeof(z));
  }
  return n;
}

}  // namespace lqcd
