// Even-odd dslash (same operator and epilogues as dslash.cu) with the eight neighbour spinors of
// every output site staged in shared memory by bulk asynchronous copies (cp.async.bulk, completion
// counted on an mbarrier), NS hops ahead of the arithmetic.
//
// One warp = 32 right-hand sides of one output site (nrhs a multiple of 32), so the warp's share of
// one 16-byte chunk of a neighbour spinor is a single contiguous 512-byte run of the RHS-innermost
// layout, and lane 0 copies all of them for the warp.  The neighbour data is in flight without
// per-thread load instructions or registers, which is what limits the direct-load kernel (a serial
// chain of eight dependent neighbour loads per thread at low occupancy).  Links and the clover
// term stay direct loads: every lane of the warp reads the same address (a broadcast).
//
// Every mbarrier wait has an iteration limit; a wait that runs out is counted in a device counter
// (read by dslash_pipe_timeouts) and the kernel finishes without waiting further.
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
  open_ns<P32, 2>();
  open_ns<P32, 3>();
  open_ns<P32, 4>();
  open_ns<P16, 2>();
  open_ns<P16, 3>();
  open_ns<P16, 4>();
}

template <int P, int EPI, int RED, int NS>
void launch_k(const DslashParams& pr, long blocks, int tpb, size_t shm, cudaStream_t st) {
  dslash_pipe_kernel<P, EPI, false, RED, NS><<<blocks, tpb, shm, st>>>(pr);
  lqcd::count_launch();
}

template <int P, int NS>
bool launch_ns(const DslashParams& pr, int epi, int red, long blocks, int tpb, size_t shm, cudaStream_t st) {
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
  if (ns == 2) return launch_ns<P, 2>(q, epi, red, blocks, tpb, q.pipe_off + (tpb / 32) * warp_bytes<P, 2>(), st);
  if (ns == 3) return launch_ns<P, 3>(q, epi, red, blocks, tpb, q.pipe_off + (tpb / 32) * warp_bytes<P, 3>(), st);
  return launch_ns<P, 4>(q, epi, red, blocks, tpb, q.pipe_off + (tpb / 32) * warp_bytes<P, 4>(), st);
}

}  // namespace

bool launch_dslash_pipe(const DslashParams& pr, int prec, int epi, bool dag, int red, long blocks, int tpb,
                        size_t red_shm, int variant, cudaStream_t st) {
  if (prec == P64 || dag || pr.nrhs % 32 != 0 || tpb % 32 != 0 || variant < 3 || variant > 5) return false;
  const int ns = variant - 1;  // variants 3, 4, 5: staging depth 2, 3, 4 hops
  open_all();
  if (prec == P32) return launch_p<P32>(pr, epi, red, blocks, tpb, red_shm, ns, st);
  return launch_p<P16>(pr, epi, red, blocks, tpb, red_shm, ns, st);
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
