// Even-odd dslash kernels (same operator and epilogues as dslash.cu) that stage per-site data in
// shared memory, selected by the dslash launch variant:
//
// * variant 3 (dslash_sl_kernel): the eight links of every site of the block are loaded and their
//   third rows rebuilt once per site by a few threads, and the site's clover blocks copied once,
//   into shared memory; the hopping threads then read them as broadcasts instead of each
//   rebuilding the links (the direct kernel repeats the rebuild for every right-hand side).  Site
//   and element indices are 32-bit (the host checks that the fields fit).  Register cap 80.
// * variant 5 (dslash_sl2_kernel): variant 3 with the hopping arithmetic on paired FP32 operations
//   (fma.rn.f32x2 / add.f32x2: two lanes per instruction).  The two spin components of a projected
//   half spinor form the pairs, (h_0[c], h_1[c]), so the SU(3) product is 36 paired FMAs per hop
//   instead of 72, with the links staged as (re, re, im, im) per entry; the upper accumulators pair
//   the same way, and the lower ones wherever the direction's spin reconstruction keeps the pair
//   order (mu = z, t).  Same arithmetic as variant 3 (each output lane rounds like the scalar
//   code), other than the order of the two products in an imaginary part.
// * variant 6 (dslash_sl3_kernel): variant 3 with each thread's neighbour spinors copied one hop
//   ahead into its own slots of a shared-memory ring by asynchronous copies (FP32 storage).
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

// ------------------------------------------------------------------ variant 5: paired FP32
// w = U h (DAG: U^dag h) for the spin pair: hr[b] = (Re h_0[b], Re h_1[b]), hi[b] likewise; L holds
// the link as 9 float4 (re, re, im, im), row-major.
template <bool DAG>
LQCD_D void su3_pair(const float4* L, const float2 (&hr)[3], const float2 (&hi)[3], float2 (&wr)[3],
                     float2 (&wi)[3]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const float4 u = L[DAG ? b * 3 + a : a * 3 + b];
      const float2 ur = make_float2(u.x, u.y), ui = make_float2(u.z, u.w), mui = make_float2(-u.z, -u.w);
      if (b == 0) {
        wr[a] = __fmul2_rn(ur, hr[0]);
        wi[a] = __fmul2_rn(ur, hi[0]);
      } else {
        wr[a] = __ffma2_rn(ur, hr[b], wr[a]);
        wi[a] = __ffma2_rn(ur, hi[b], wi[a]);
      }
      wr[a] = __ffma2_rn(DAG ? ui : mui, hi[b], wr[a]);  // U h: - Im u Im h;  U^dag h: + Im u Im h
      wi[a] = __ffma2_rn(DAG ? mui : ui, hr[b], wi[a]);  // U h: + Im u Re h;  U^dag h: - Im u Re h
    }
  }
}

// acc += [ w ; S X_MU^dag w ] on the paired accumulators: ur / ui = (spin 0, spin 1) real / imaginary
// parts per colour, lr / li = (spin 2, spin 3).
template <int MU, int S>
LQCD_D void accumulate_pair(const float2 (&wr)[3], const float2 (&wi)[3], float2 (&ur)[3], float2 (&ui)[3],
                            float2 (&lr)[3], float2 (&li)[3]) {
  constexpr float s = (float)S;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    ur[c] = __fadd2_rn(ur[c], wr[c]);
    ui[c] = __fadd2_rn(ui[c], wi[c]);
    if constexpr (MU == 0) {  // X^dag w = (i w1, i w0)
      lr[c].x -= s * wi[c].y;
      lr[c].y -= s * wi[c].x;
      li[c].x += s * wr[c].y;
      li[c].y += s * wr[c].x;
    } else if constexpr (MU == 1) {  // X^dag w = (w1, -w0)
      lr[c].x += s * wr[c].y;
      lr[c].y -= s * wr[c].x;
      li[c].x += s * wi[c].y;
      li[c].y -= s * wi[c].x;
    } else if constexpr (MU == 2) {  // X^dag w = (i w0, -i w1)
      lr[c] = __ffma2_rn(make_float2(-s, s), wi[c], lr[c]);
      li[c] = __ffma2_rn(make_float2(s, -s), wr[c], li[c]);
    } else {  // X^dag w = (w0, w1)
      lr[c] = __ffma2_rn(make_float2(s, s), wr[c], lr[c]);
      li[c] = __ffma2_rn(make_float2(s, s), wi[c], li[c]);
    }
  }
}

template <int MU, bool FWD>
LQCD_D void hop_pair_p(const cplx<float> (&p)[12], int coef, const float4* L, float2 (&ur)[3], float2 (&ui)[3],
                       float2 (&lr)[3], float2 (&li)[3]) {
  constexpr int S = FWD ? -1 : 1;  // H (not H^dag): forward projector 1 - gamma_mu
  cplx<float> h[2][3];
  project<MU, S>(p, h);
  float2 hr[3], hi[3], wr[3], wi[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    hr[c] = make_float2(h[0][c].re, h[1][c].re);
    hi[c] = make_float2(h[0][c].im, h[1][c].im);
  }
  su3_pair<!FWD>(L, hr, hi, wr, wi);
  if (coef < 0) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      wr[c] = make_float2(-wr[c].x, -wr[c].y);
      wi[c] = make_float2(-wi[c].x, -wi[c].y);
    }
  }
  accumulate_pair<MU, S>(wr, wi, ur, ui, lr, li);
}

template <int P, int MU, bool FWD>
LQCD_D void hop_pair(const DslashParams& pr, int nb_idx, int coef, int stride, const float4* L, float2 (&ur)[3],
                     float2 (&ui)[3], float2 (&lr)[3], float2 (&li)[3]) {
  cplx<float> p[12];
  load_spinor32<P>(pr.in, stride, nb_idx, p);
  hop_pair_p<MU, FWD>(p, coef, L, ur, ui, lr, li);
}

template <int P, int MU>
LQCD_D void hop_dir_pair(const DslashParams& pr, int s, int cmu, int Lmu, int smu, int coef_f, int coef_b, int rhs,
                         int stride, int nrhs, const float4* lf, const float4* lb, float2 (&ur)[3], float2 (&ui)[3],
                         float2 (&lr)[3], float2 (&li)[3]) {
  if (coef_f != 0) {
    const int sn = s + ((cmu + 1 == Lmu) ? smu * (1 - Lmu) : smu);
    hop_pair<P, MU, true>(pr, (sn >> 1) * nrhs + rhs, coef_f, stride, lf, ur, ui, lr, li);
  }
  if (coef_b != 0) {
    const int sn = s + ((cmu == 0) ? smu * (Lmu - 1) : -smu);
    hop_pair<P, MU, false>(pr, (sn >> 1) * nrhs + rhs, coef_b, stride, lb, ur, ui, lr, li);
  }
}

// Blocks as variant 3 (128 threads = 128 / nrhs sites x nrhs right-hand sides).
template <int P, int EPI, int RED, int MINB>
__global__ void __launch_bounds__(128, MINB) dslash_sl2_kernel(const DslashParams pr) {
  __shared__ float4 slink[kMaxSites][8][9];  // [site][hop: 2 mu (fwd), 2 mu + 1 (bwd)][entry]: (re, re, im, im)
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
        if (k & 1) {  // backward hop: the link of the neighbour s - mu
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
#pragma unroll
        for (int e = 0; e < 9; e++) {
          const cplx<float> v = u[e / 3][e % 3];
          L[e] = make_float4(v.re, v.re, v.im, v.im);
        }
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

  float2 ur[3], ui[3], lr[3], li[3];
#pragma unroll
  for (int c = 0; c < 3; c++) ur[c] = ui[c] = lr[c] = li[c] = make_float2(0.f, 0.f);
  hop_dir_pair<P, 0>(pr, s, x, g.Lx, 1, 1, 1, rhs, stride, nr, slink[sl][0], slink[sl][1], ur, ui, lr, li);
  hop_dir_pair<P, 1>(pr, s, y, g.Ly, sy, 1, 1, rhs, stride, nr, slink[sl][2], slink[sl][3], ur, ui, lr, li);
  hop_dir_pair<P, 2>(pr, s, z, g.Lz, sz, 1, 1, rhs, stride, nr, slink[sl][4], slink[sl][5], ur, ui, lr, li);
  const int cf = __ldg(pr.tc + t), cbk = __ldg(pr.tc + (t == 0 ? g.Lt - 1 : t - 1));
  hop_dir_pair<P, 3>(pr, s, t, g.Lt, sw, cf, cbk, rhs, stride, nr, slink[sl][6], slink[sl][7], ur, ui, lr, li);
  cplx<float> acc[12];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    acc[c] = {ur[c].x, ui[c].x};
    acc[3 + c] = {ur[c].y, ui[c].y};
    acc[6 + c] = {lr[c].x, li[c].x};
    acc[9 + c] = {lr[c].y, li[c].y};
  }
  dslash_epilogue<P, EPI, RED, true>(pr, cb, (long)cb * nr + rhs, (long)stride, rhs, acc, sclov[sl]);
}

// ------------------------------------------------------------------ variant 6: pipelined neighbour spinors
// Variant 3 whose eight neighbour spinors are fetched by each thread into its own slots of a
// kPipe-deep ring in shared memory with asynchronous copies (cp.async, 16 bytes each, L2 only),
// kPipe - 1 hops ahead of the arithmetic, so a thread has the next hop's loads in flight while it
// computes without holding them in registers.  Ring layout [stage][chunk][thread] (float4): each
// thread reads back only what it copied (a wait on its own copy groups, no barrier), and a warp's
// accesses are contiguous.  FP32 storage only.
constexpr int kPipe = 2;
constexpr size_t kPipeBytes = (size_t)kPipe * 6 * 128 * sizeof(float4);

LQCD_D void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
LQCD_D void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
LQCD_D void cp_async_wait_pipe() { asm volatile("cp.async.wait_group %0;" ::"n"(kPipe - 1) : "memory"); }

template <int K>
LQCD_D void pipe_issue(const DslashParams& pr, float4* ring, const int (&nb)[8], int stride, bool valid) {
  if constexpr (K < 8) {
    if (valid) {
      float4* dst = ring + (K % kPipe) * 6 * 128 + threadIdx.x;
      const float4* src = reinterpret_cast<const float4*>(pr.in) + nb[K];
#pragma unroll
      for (int c = 0; c < 6; c++) cp_async16(dst + c * 128, src + (long)c * stride);
    }
  }
  cp_async_commit();  // one group per hop (empty past the last), so the wait count stays uniform
}

// hop K = 2 mu (+1 for the backward hop) with its neighbour from the ring and its link from the
// per-site staging (variant-3 format)
template <int K>
LQCD_D void pipe_hop(const DslashParams& pr, float4* ring, const int (&nb)[8], int stride, int coef, bool valid,
                     const float4* L, cplx<float> (&acc)[12]) {
  constexpr int MU = K / 2;
  constexpr bool FWD = (K % 2) == 0;
  constexpr int S = FWD ? -1 : 1;  // H (not H^dag): forward projector 1 - gamma_mu
  pipe_issue<K + kPipe - 1>(pr, ring, nb, stride, valid);
  cp_async_wait_pipe();  // this thread's copies of hop K have landed
  const float4* src = ring + (K % kPipe) * 6 * 128 + threadIdx.x;
  cplx<float> p[12];
#pragma unroll
  for (int c = 0; c < 6; c++) {
    const float4 v = src[c * 128];
    p[2 * c] = {v.x, v.y};
    p[2 * c + 1] = {v.z, v.w};
  }
  if (coef == 0) return;
  cplx<float> h[2][3], w[2][3], u[3][3];
  project<MU, S>(p, h);
  link_from_shared(L, u);
  if constexpr (FWD)
    su3_mul(u, h, w);
  else
    su3_dag_mul(u, h, w);
  if (coef < 0) {
#pragma unroll
    for (int q = 0; q < 2; q++)
#pragma unroll
      for (int a = 0; a < 3; a++) w[q][a] = -w[q][a];
  }
  accumulate<MU, S>(acc, w);
}

// Dynamic shared memory: [ring | links S x 8 x 5 | clover S x 18] (float4); the fused reductions
// scratch (at most 8 doubles per thread, smaller than the ring) overlays the ring once the hops are
// done.
template <int EPI, int RED, int MINB>
__global__ void __launch_bounds__(128, MINB) dslash_sl3_kernel(const DslashParams pr) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int nr = pr.nrhs;
  const int lg = __ffs(nr) - 1;
  const int S = 128 >> lg;
  float4* ring = reinterpret_cast<float4*>(dsm + pr.pipe_off);
  float4 (*slink)[8][5] = reinterpret_cast<float4 (*)[8][5]>(ring + kPipe * 6 * 128);
  float4 (*sclov)[18] = reinterpret_cast<float4 (*)[18]>(slink + S);
  const Geom& g = pr.g;
  const int cb0 = blockIdx.x * S;
  const int Vh = (int)g.Vh;
  const int sy = g.Lx, sz = g.Lx * g.Ly, sw = sz * g.Lz;
  const int tid = blockIdx.x * 128 + threadIdx.x;
  const int cb = tid >> lg;
  const int rhs = tid & (nr - 1);
  const bool valid = cb < Vh;
  const unsigned cw = valid ? __ldg(pr.coord + cb) : 0u;
  const int x = cw & 0xff, y = (cw >> 8) & 0xff, z = (cw >> 16) & 0xff, t = cw >> 24;
  const int s = x + sy * y + sz * z + sw * t;
  const int stride = Vh * nr;
  int nb[8];  // spinor index of the neighbour of each hop (2 mu: s + mu, 2 mu + 1: s - mu)
  {
    const int cm[4] = {x, y, z, t}, Lm[4] = {g.Lx, g.Ly, g.Lz, g.Lt}, sm[4] = {1, sy, sz, sw};
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      nb[2 * mu] = ((s + ((cm[mu] + 1 == Lm[mu]) ? sm[mu] * (1 - Lm[mu]) : sm[mu])) >> 1) * nr + rhs;
      nb[2 * mu + 1] = ((s + ((cm[mu] == 0) ? sm[mu] * (Lm[mu] - 1) : -sm[mu])) >> 1) * nr + rhs;
    }
  }
  static_assert(kPipe == 2, "one hop is issued ahead");
  pipe_issue<0>(pr, ring, nb, stride, valid);  // the first hop's copies run under the link staging
  for (int j = threadIdx.x; j < 26 * S; j += 128) {
    if (j < 8 * S) {  // link j & 7 of site j >> 3, third row rebuilt once
      const int site = j >> 3, k = j & 7, c = cb0 + site;
      if (c < Vh) {
        const int mu = k >> 1;
        int lcb = c, par = pr.out_par;
        if (k & 1) {  // backward hop: the link of the neighbour s - mu
          const int xh = c % g.Lxh, yzt = c / g.Lxh, yy = yzt % g.Ly, zt = yzt / g.Ly, zz = zt % g.Lz,
                    tt = zt / g.Lz;
          const int xx = 2 * xh + ((pr.out_par + yy + zz + tt) & 1);
          const int ss = xx + sy * yy + sz * zz + sw * tt;
          const int cmu = mu == 0 ? xx : (mu == 1 ? yy : (mu == 2 ? zz : tt));
          const int Lmu = mu == 0 ? g.Lx : (mu == 1 ? g.Ly : (mu == 2 ? g.Lz : g.Lt));
          const int smu = mu == 0 ? 1 : (mu == 1 ? sy : (mu == 2 ? sz : sw));
          lcb = (ss + (cmu == 0 ? smu * (Lmu - 1) : -smu)) >> 1;
          par = 1 - pr.out_par;
        }
        cplx<float> u[3][3];
        load_link<P32>(pr.U, g.Vh, mu, par, lcb, u);
        float4* L = slink[site][k];
        L[0] = make_float4(u[0][0].re, u[0][0].im, u[0][1].re, u[0][1].im);
        L[1] = make_float4(u[0][2].re, u[0][2].im, u[1][0].re, u[1][0].im);
        L[2] = make_float4(u[1][1].re, u[1][1].im, u[1][2].re, u[1][2].im);
        L[3] = make_float4(u[2][0].re, u[2][0].im, u[2][1].re, u[2][1].im);
        L[4] = make_float4(u[2][2].re, u[2][2].im, 0.f, 0.f);
      }
    } else {  // clover chunk e of site q / 18
      const int q = j - 8 * S, site = q / 18, e = q - site * 18, c = cb0 + site;
      if (c < Vh) sclov[site][e] = __ldg(reinterpret_cast<const float4*>(pr.C) + (long)e * Vh + c);
    }
  }
  __syncthreads();
  if (RED == RED_NONE && !valid) {
    asm volatile("cp.async.wait_all;" ::: "memory");
    return;
  }
  const int sl = threadIdx.x >> lg;
  const int cf = __ldg(pr.tc + t), cbk = __ldg(pr.tc + (t == 0 ? g.Lt - 1 : t - 1));
  cplx<float> acc[12];
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = {0.f, 0.f};
  pipe_hop<0>(pr, ring, nb, stride, 1, valid, slink[sl][0], acc);
  pipe_hop<1>(pr, ring, nb, stride, 1, valid, slink[sl][1], acc);
  pipe_hop<2>(pr, ring, nb, stride, 1, valid, slink[sl][2], acc);
  pipe_hop<3>(pr, ring, nb, stride, 1, valid, slink[sl][3], acc);
  pipe_hop<4>(pr, ring, nb, stride, 1, valid, slink[sl][4], acc);
  pipe_hop<5>(pr, ring, nb, stride, 1, valid, slink[sl][5], acc);
  pipe_hop<6>(pr, ring, nb, stride, cf, valid, slink[sl][6], acc);
  pipe_hop<7>(pr, ring, nb, stride, cbk, valid, slink[sl][7], acc);
  asm volatile("cp.async.wait_all;" ::: "memory");
  // the fused reductions' scratch overlays the ring (dynamic offset 0): every thread must be done
  // with its ring slots first
  if constexpr (RED != RED_NONE) __syncthreads();
  dslash_epilogue<P32, EPI, RED, true>(pr, cb, (long)cb * nr + rhs, (long)stride, rhs, acc, sclov[sl]);
}

// largest dynamic shared memory of a variant-6 launch: the ring, and the links and clover of 16
// sites
constexpr size_t kSl3MaxShm = kPipeBytes + (size_t)kMaxSites * (40 + 18) * sizeof(float4);

template <int EPI, int RED>
void open_sl3() {
  cudaFuncSetAttribute(dslash_sl3_kernel<EPI, RED, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSl3MaxShm);
}

// Raise the dynamic shared-memory limit of every variant-6 instantiation once, before its first
// launch.
void open_sl3_all() {
  static bool done = false;
  if (done) return;
  done = true;
  open_sl3<EPI_Y_CH, RED_TS_R0>();
  open_sl3<EPI_Y_CH, RED_DOT_Z>();
  open_sl3<EPI_Y_CH, RED_DOT_Y_NORM>();
  open_sl3<EPI_CH, RED_NONE>();
  open_sl3<EPI_Y_CH, RED_NONE>();
  open_sl3<EPI_C_YH, RED_NONE>();
}

template <int EPI, int RED>
void launch_sl3(const DslashParams& pr, long blocks, size_t red_shm, cudaStream_t st) {
  DslashParams q = pr;
  q.pipe_off = 0;
  (void)red_shm;  // fits in the ring (checked by the caller)
  const int S = 128 / pr.nrhs;
  const size_t shm = kPipeBytes + (size_t)S * (40 + 18) * sizeof(float4);
  dslash_sl3_kernel<EPI, RED, 6><<<blocks, 128, shm, st>>>(q);
  lqcd::count_launch();
}

bool launch_sl3_e(const DslashParams& pr, int epi, int red, long blocks, size_t red_shm, cudaStream_t st) {
  if (red_shm > kPipeBytes) return false;
  if (red == RED_TS_R0) {
    if (epi != EPI_Y_CH) return false;
    launch_sl3<EPI_Y_CH, RED_TS_R0>(pr, blocks, red_shm, st);
  } else if (red == RED_DOT_Z) {
    if (epi != EPI_Y_CH) return false;
    launch_sl3<EPI_Y_CH, RED_DOT_Z>(pr, blocks, red_shm, st);
  } else if (red == RED_DOT_Y_NORM) {
    if (epi != EPI_Y_CH) return false;
    launch_sl3<EPI_Y_CH, RED_DOT_Y_NORM>(pr, blocks, red_shm, st);
  } else if (epi == EPI_CH) {
    launch_sl3<EPI_CH, RED_NONE>(pr, blocks, red_shm, st);
  } else if (epi == EPI_Y_CH) {
    launch_sl3<EPI_Y_CH, RED_NONE>(pr, blocks, red_shm, st);
  } else if (epi == EPI_C_YH) {
    launch_sl3<EPI_C_YH, RED_NONE>(pr, blocks, red_shm, st);
  } else {
    return false;
  }
  return true;
}

template <int P, int EPI, int RED, int MINB>
void launch_sl(const DslashParams& pr, long blocks, size_t shm, cudaStream_t st, bool paired) {
  if (paired)
    dslash_sl2_kernel<P, EPI, RED, MINB><<<blocks, 128, shm, st>>>(pr);
  else
    dslash_sl_kernel<P, EPI, RED, MINB><<<blocks, 128, shm, st>>>(pr);
  lqcd::count_launch();
}

template <int P, int MINB>
bool launch_sl_e(const DslashParams& pr, int epi, int red, long blocks, size_t shm, cudaStream_t st,
                 bool paired) {
  if (red == RED_TS_R0) {
    if (epi != EPI_Y_CH) return false;
    launch_sl<P, EPI_Y_CH, RED_TS_R0, MINB>(pr, blocks, shm, st, paired);
  } else if (red == RED_DOT_Z) {
    if (epi != EPI_Y_CH) return false;
    launch_sl<P, EPI_Y_CH, RED_DOT_Z, MINB>(pr, blocks, shm, st, paired);
  } else if (red == RED_DOT_Y_NORM) {
    if (epi != EPI_Y_CH) return false;
    launch_sl<P, EPI_Y_CH, RED_DOT_Y_NORM, MINB>(pr, blocks, shm, st, paired);
  } else if (epi == EPI_CH) {
    launch_sl<P, EPI_CH, RED_NONE, MINB>(pr, blocks, shm, st, paired);
  } else if (epi == EPI_Y_CH) {
    launch_sl<P, EPI_Y_CH, RED_NONE, MINB>(pr, blocks, shm, st, paired);
  } else if (epi == EPI_C_YH) {
    launch_sl<P, EPI_C_YH, RED_NONE, MINB>(pr, blocks, shm, st, paired);
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
  if (prec == P64 || dag || variant < 3 || variant > 7) return false;
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
  if (variant == 7) {  // two right-hand sides per thread on paired arithmetic (dslash_rb2.cu)
    if (prec != P32) return false;
    return launch_dslash_rb2(pr, epi, red, blocks, tpb, red_shm, st);
  }
  if (variant == 6 && prec == P32) {  // pipelined neighbour copies
    open_sl3_all();
    if (launch_sl3_e(pr, epi, red, blocks, red_shm, st)) return true;
  }
  if (variant == 5) {  // paired operands take aligned register pairs: cap 96 instead of 80
    if (prec == P32) return launch_sl_e<P32, 5>(pr, epi, red, blocks, red_shm, st, true);
    return launch_sl_e<P16, 5>(pr, epi, red, blocks, red_shm, st, true);
  }
  if (prec == P32) return launch_sl_e<P32, 6>(pr, epi, red, blocks, red_shm, st, false);
  return launch_sl_e<P16, 6>(pr, epi, red, blocks, red_shm, st, false);
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
