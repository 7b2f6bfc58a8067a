// Gauge-covariant parallel-transport network used as the preconditioner of flexible GCR, with
// its training on the GPU (forward, backward and Adam kernels of this file).
//
// A layer maps C_in channels of colour vectors h_c(x) to C_out channels,
//     out_o(x) = sum_{p=0..8} sum_c W[p][o][c] (T_p h_c)(x),
//     T_0 h = h,  T_{1+mu} h(x) = U_mu(x) h(x+mu),  T_{5+mu} h(x) = U_mu(x-mu)^dag h(x-mu),
// on the fermion links (time boundary phase, and Dirichlet cuts for the domain operator, from
// the same per-timeslice coefficients as the dslash).  Each path commutes with gauge
// transformations, so the network is gauge covariant.  Four linear layers, channel widths
// 4 -> 8 -> 8 -> 8 -> 4: a spinor (four spin channels) in, a spinor out.  Inference reads BF16
// weights and accumulates in FP32; training keeps FP32 master weights.
//
// Field layout (FP32 complex): [k = channel * 3 + colour][se][n], se = parity * Vh + cb (even-odd
// full lattice), n = sample; one thread per (site, sample), samples fastest so the links of a
// site are a warp broadcast.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "lqcd_blas.h"
#include "lqcd_distill.h"
#include "tc_bf16.cuh"

namespace lqcd {

constexpr int NN_LAYERS = 4;
constexpr int NN_W[NN_LAYERS + 1] = {4, 8, 8, 8, 4};
constexpr int NN_PATHS = 9;

static int nn_layer_offset(int l) {  // complex entries before layer l
  int o = 0;
  for (int i = 0; i < l; i++) o += NN_PATHS * NN_W[i] * NN_W[i + 1];
  return o;
}
int nn_total_weights() { return nn_layer_offset(NN_LAYERS); }

struct NNGeo {
  Geom g;
  const unsigned* coord;  // [2][Vh]
  const float4* U;        // FP32 links (rows 0, 1)
  const signed char* tc;
  int N;  // samples
};

template <typename WT>
LQCD_D cplx<float> wload(const WT* w, int i);
template <>
LQCD_D cplx<float> wload<float2>(const float2* w, int i) {
  float2 v = w[i];
  return {v.x, v.y};
}
template <>
LQCD_D cplx<float> wload<__nv_bfloat162>(const __nv_bfloat162* w, int i) {
  float2 v = __bfloat1622float2(w[i]);
  return {v.x, v.y};
}

// Transported channels of one path at one (site, sample): th[c][a] = (T_p h_c)(x)[a].
// Returns false if the path is cut (coefficient 0).
template <int C>
LQCD_D bool path_vectors(const NNGeo& G, const float2* h, int p, int par, long cb, int x, int y, int z, int t,
                         int n, cplx<float> (&th)[C][3]) {
  const Geom& g = G.g;
  const long V = 2 * g.Vh;
  const long s = x + (long)g.Lx * (y + (long)g.Ly * (z + (long)g.Lz * t));
  long sn = s;
  int coef = 1;
  int mu = (p - 1) & 3;
  bool fwd = p >= 1 && p <= 4;
  if (p != 0) {
    int cm = mu == 0 ? x : (mu == 1 ? y : (mu == 2 ? z : t));
    int Lm = mu == 0 ? g.Lx : (mu == 1 ? g.Ly : (mu == 2 ? g.Lz : g.Lt));
    long sm = mu == 0 ? 1 : (mu == 1 ? g.Lx : (mu == 2 ? (long)g.Lx * g.Ly : (long)g.Lx * g.Ly * g.Lz));
    if (fwd) {
      sn = s + ((cm + 1 == Lm) ? sm * (1 - Lm) : sm);
      if (mu == 3) coef = __ldg(G.tc + t);
    } else {
      sn = s + ((cm == 0) ? sm * (Lm - 1) : -sm);
      if (mu == 3) coef = __ldg(G.tc + (t == 0 ? g.Lt - 1 : t - 1));
    }
    if (coef == 0) return false;
  }
  const int npar = p == 0 ? par : 1 - par;
  const long nse = (long)npar * g.Vh + (sn >> 1);
  const long VN = V * G.N;  // stride between the channel-colour planes
  const float2* hp = h + nse * G.N + n;
  cplx<float> hv[C][3];
#pragma unroll
  for (int c = 0; c < C; c++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const float2 v = __ldg(hp);
      hp += VN;
      hv[c][a] = {v.x, v.y};
    }
  if (p == 0) {
#pragma unroll
    for (int c = 0; c < C; c++)
#pragma unroll
      for (int a = 0; a < 3; a++) th[c][a] = hv[c][a];
    return true;
  }
  cplx<float> u[3][3];
  if (fwd)
    load_link<P32>(G.U, g.Vh, mu, par, cb, u);
  else
    load_link<P32>(G.U, g.Vh, mu, 1 - par, sn >> 1, u);
  // the backward hop's U^dag and the time-boundary sign, once on the link, so that every path
  // runs the same product below
  cplx<float> w[3][3];
  const float sg = coef < 0 ? -1.f : 1.f;
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++)
      w[a][b] = fwd ? cplx<float>{sg * u[a][b].re, sg * u[a][b].im} : cplx<float>{sg * u[b][a].re, -sg * u[b][a].im};
#pragma unroll
  for (int c = 0; c < C; c++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cplx<float> acc = w[a][0] * hv[c][0];
      acc = cfma(w[a][1], hv[c][1], acc);
      th[c][a] = cfma(w[a][2], hv[c][2], acc);
    }
  return true;
}

LQCD_D void nn_site(const NNGeo& G, long se, int& par, long& cb, int& x, int& y, int& z, int& t) {
  par = se >= G.g.Vh ? 1 : 0;
  cb = se - (long)par * G.g.Vh;
  const unsigned cw = __ldg(G.coord + (long)par * G.g.Vh + cb);
  x = cw & 0xff;
  y = (cw >> 8) & 0xff;
  z = (cw >> 16) & 0xff;
  t = cw >> 24;
}

// out = layer(W, in)  (transport and channel mixing fused; weights staged in shared memory)
template <int CIN, int COUT, typename WT>
__global__ void k_nn_layer(const float2* in, float2* out, const WT* W, NNGeo G) {
  __shared__ cplx<float> Ws[NN_PATHS * COUT * CIN];
  for (int i = threadIdx.x; i < NN_PATHS * COUT * CIN; i += blockDim.x) Ws[i] = wload<WT>(W, i);
  __syncthreads();
  const long V = 2 * G.g.Vh;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long se = tid / G.N;
  const int n = (int)(tid - se * G.N);
  if (se >= V) return;
  int par, x, y, z, t;
  long cb;
  nn_site(G, se, par, cb, x, y, z, t);
  cplx<float> acc[COUT][3];
#pragma unroll
  for (int o = 0; o < COUT; o++)
#pragma unroll
    for (int a = 0; a < 3; a++) acc[o][a] = {0.f, 0.f};
  for (int p = 0; p < NN_PATHS; p++) {
    cplx<float> th[CIN][3];
    if (!path_vectors<CIN>(G, in, p, par, cb, x, y, z, t, n, th)) continue;
#pragma unroll
    for (int o = 0; o < COUT; o++)
#pragma unroll
      for (int c = 0; c < CIN; c++) {
        cplx<float> w = Ws[(p * COUT + o) * CIN + c];
#pragma unroll
        for (int a = 0; a < 3; a++) acc[o][a] = acc[o][a] + w * th[c][a];
      }
  }
#pragma unroll
  for (int o = 0; o < COUT; o++)
#pragma unroll
    for (int a = 0; a < 3; a++) out[((long)(o * 3 + a) * V + se) * G.N + n] = make_float2(acc[o][a].re, acc[o][a].im);
}

// ------------------------------------------------------------------ tensor-core layer (inference)
// The same layer with the channel mixing on the tensor cores (tcgen05, BF16 operands, FP32
// accumulation in tensor memory).  The mixing is a GEMM per colour a whose rows are the
// (site, sample) pairs -- the weights do not mix colours -- with K = (path, re / im part, input
// channel) and N = (re / im part, output channel):
//   A_a[q][(p, 0, c)] = Re (T_p h_c)(q)[a],  A_a[q][(p, 1, c)] = Im (T_p h_c)(q)[a],
//   B[o][(p, 0, c)] = Re W[p][o][c],  B[o][(p, 1, c)] = -Im W,  B[C_out + o][(p, 0, c)] = Im W,
//   B[C_out + o][(p, 1, c)] = Re W,   D_a[q][o] = Re out_o(q)[a],  D_a[q][C_out + o] = Im out_o(q)[a].
//
// Persistent CTA of 128 threads (one thread per pair, row = thread) over tiles of 128 pairs.  Each
// thread transports every input channel along one path chunk (one path for C_in = 8, two for
// C_in = 4: 16 K columns per colour) and writes the three colours' rows into a ring of kRing chunk
// buffers; one lane of warp 0, once the whole chunk is staged, issues its three MMAs (M = 128,
// N = 16, K = 16), accumulating into one of two tensor-memory result buffers (so a tile's MMAs
// overlap the previous tile's read-out); after a tile's last chunk every thread reads its FP32
// result row out of tensor memory and stores it.  No warp is set aside for the MMAs, so four CTAs
// (16 warps of transports) fit an SM.
// Hand-offs are mbarriers: full[s] (128 arrivals) / empty[s] (MMA completion) per ring slot and
// dfull[d] (MMA completion) per result buffer.  A result buffer is reused two tiles later, after
// every thread has read it out and then staged its part of the next tile (so the full barrier of
// that tile's first chunk orders the read-out before the new MMAs).  Every wait has an iteration
// and a time limit; a wait that runs out raises a CTA flag that stops every loop, the kernel
// counts it in g_nn_tc_timeouts, waits (bounded) for its MMAs in flight and frees its tensor
// memory before returning.
constexpr int kNNTile = 128;                      // pairs per tile (MMA M)
constexpr int kRing = 4;                          // staged chunks in flight
constexpr int kChunkColour = kNNTile * 16 * 2;    // bytes of one colour's 128 x 16 BF16 chunk
constexpr int kChunkBytes = 3 * kChunkColour;     // one ring slot
constexpr int kNNWaitLimit = 1 << 22;
constexpr int kNNThreads = 128;
__device__ int g_nn_tc_timeouts;

template <int CIN>
constexpr int nn_tc_chunks() {
  return CIN == 8 ? NN_PATHS : (NN_PATHS + 1) / 2;
}
template <int CIN>
constexpr int nn_tc_k() {
  return 16 * nn_tc_chunks<CIN>();
}

LQCD_D uint32_t bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

LQCD_D bool wait_or_flag(uint64_t* mbar, uint32_t parity, volatile int* fail) {
  if (*fail) return false;
  if (tc::mbar_wait(mbar, parity, kNNWaitLimit)) return true;
  *fail = 1;
  return false;
}

// Tile order.  Sites are visited slab by slab, a slab being Bz consecutive z-planes of one
// timeslice (slabs ordered by z-block, then t), each slab as alternating even / odd tiles of 128
// (site, sample) pairs.  Bz is chosen so that three slabs' input channels fit in L2, so a site's
// channels, read as the centre and as a neighbour in every direction (the z-hops across a block
// edge excepted), come from DRAM about once per layer.
struct NNTiles {
  int Bz;      // z-planes per slab
  long tps;    // tiles per parity per slab
  long ntiles; // all tiles
  int npar;    // 2: even and odd output sites; 1: even output sites only (the odd ones are not needed)
  int in_even; // 1: the input is zero on odd sites, so even outputs take the identity path only and
               // odd outputs the eight hops only
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kNNThreads, 4) k_nn_layer_tc(const float2* in, float2* out,
                                                               const __nv_bfloat162* W, NNGeo G, NNTiles TL) {
  constexpr int NCH = nn_tc_chunks<CIN>();
  constexpr int K = nn_tc_k<CIN>();
  extern __shared__ __align__(128) unsigned char nn_sm[];
  unsigned char* ring = nn_sm;                         // [kRing][3 colours][128 x 16] BF16
  unsigned char* sB = ring + kRing * kChunkBytes;      // 16 x K BF16
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + 16 * K * 2);
  uint64_t* full = bars;                               // [kRing]
  uint64_t* empty = bars + kRing;                      // [kRing]
  uint64_t* dfull = bars + 2 * kRing;                  // [2]
  uint64_t* drain = bars + 2 * kRing + 2;              // [1] (failure path)
  uint32_t* tbase = reinterpret_cast<uint32_t*>(bars + 2 * kRing + 3);
  volatile int* fail = reinterpret_cast<volatile int*>(tbase + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long V = 2 * G.g.Vh;
  const long slab_cb = (long)G.g.Lxh * G.g.Ly * TL.Bz;  // sites of one parity in a slab
  const long slab_pairs = slab_cb * G.N;
  const long ntiles = TL.ntiles;

  // weights -> B in the K-major canonical layout (zero where N is padding)
  for (int e = tid; e < 16 * K; e += kNNThreads) {
    const int j = e / K, k = e - j * K;
    float v = 0.f;
    const int pth = k / (2 * CIN), r = k - pth * 2 * CIN, part = r / CIN, c = r - part * CIN;
    if (j < 2 * COUT && pth < NN_PATHS) {
      const int o = j % COUT, im_out = j / COUT;
      const float2 w = __bfloat1622float2(W[(pth * COUT + o) * CIN + c]);
      v = im_out == 0 ? (part == 0 ? w.x : -w.y) : (part == 0 ? w.y : w.x);
    }
    *reinterpret_cast<__nv_bfloat16*>(sB + tc::kmajor_offset(j, k, K)) = __float2bfloat16(v);
  }
  if (tid == 0) {
    for (int i = 0; i < kRing; i++) {
      tc::mbar_init(full + i, kNNThreads);
      tc::mbar_init(empty + i, 1);
    }
    tc::mbar_init(dfull, 1);
    tc::mbar_init(dfull + 1, 1);
    tc::mbar_init(drain, 1);
    *fail = 0;
  }
  if (warp == 0) tc::tmem_alloc(tbase, 128);
  tc::fence_proxy_async();
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tbase;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 16);
  const uint32_t r0 = tc::smem_u32(ring), b0 = tc::smem_u32(sB);

  long it = 0;     // tiles done by this CTA
  long chunk = 0;  // chunks staged by this CTA
  for (long tile = blockIdx.x; tile < ntiles && !*fail; tile += gridDim.x, it++) {
    const long sl = tile / (TL.npar * TL.tps), r = tile - sl * TL.npar * TL.tps;
    const int tpar = TL.npar == 2 ? (int)(r & 1) : 0;
    const long q = (TL.npar == 2 ? r >> 1 : r) * kNNTile + tid;  // pair within the slab's sites of parity tpar
    const bool valid = q < slab_pairs;
    long se = 0, cb = 0;
    int n = 0, par = 0, x = 0, y = 0, z = 0, t = 0;
    if (valid) {
      const long zb = sl / G.g.Lt, ts = sl - zb * G.g.Lt;
      const long cb0 = (long)G.g.Lxh * G.g.Ly * (zb * TL.Bz + (long)G.g.Lz * ts);
      const long i = q / G.N;
      n = (int)(q - i * G.N);
      se = tpar * G.g.Vh + cb0 + i;
      nn_site(G, se, par, cb, x, y, z, t);
    }
    const int d = (int)(it & 1);
    const uint32_t roff = (uint32_t)((tid >> 3) * 256 + (tid & 7) * 16);  // row offset in a chunk
    for (int ch = 0; ch < NCH; ch++, chunk++) {
      const int slot = (int)(chunk % kRing);
      const long use = chunk / kRing;
      if (use > 0 && !wait_or_flag(empty + slot, (uint32_t)((use - 1) & 1), fail)) break;
      unsigned char* buf = ring + slot * kChunkBytes + roff;
#pragma unroll
      for (int h = 0; h < 16 / (2 * CIN); h++) {  // paths of this chunk
        const int p = ch * (16 / (2 * CIN)) + h;
        cplx<float> th[CIN][3];
        bool on = false;
        const bool live = !TL.in_even || ((tpar == 0) == (p == 0));  // else the input there is zero
        if (valid && p < NN_PATHS && live) on = path_vectors<CIN>(G, in, p, par, cb, x, y, z, t, n, th);
        if (!on) {
#pragma unroll
          for (int c = 0; c < CIN; c++)
#pragma unroll
            for (int a = 0; a < 3; a++) th[c][a] = {0.f, 0.f};
        }
#pragma unroll
        for (int a = 0; a < 3; a++) {
          if (CIN == 8) {  // re of the 8 channels in core column 0, im in core column 1
            uint4 vr, vi;
            vr.x = bf16x2(th[0][a].re, th[1 % CIN][a].re);
            vr.y = bf16x2(th[2 % CIN][a].re, th[3 % CIN][a].re);
            vr.z = bf16x2(th[4 % CIN][a].re, th[5 % CIN][a].re);
            vr.w = bf16x2(th[6 % CIN][a].re, th[7 % CIN][a].re);
            vi.x = bf16x2(th[0][a].im, th[1 % CIN][a].im);
            vi.y = bf16x2(th[2 % CIN][a].im, th[3 % CIN][a].im);
            vi.z = bf16x2(th[4 % CIN][a].im, th[5 % CIN][a].im);
            vi.w = bf16x2(th[6 % CIN][a].im, th[7 % CIN][a].im);
            *reinterpret_cast<uint4*>(buf + a * kChunkColour) = vr;
            *reinterpret_cast<uint4*>(buf + a * kChunkColour + 128) = vi;
          } else {  // 4 channels: re 0..3 then im 0..3 in core column h
            uint4 v;
            v.x = bf16x2(th[0][a].re, th[1 % CIN][a].re);
            v.y = bf16x2(th[2 % CIN][a].re, th[3 % CIN][a].re);
            v.z = bf16x2(th[0][a].im, th[1 % CIN][a].im);
            v.w = bf16x2(th[2 % CIN][a].im, th[3 % CIN][a].im);
            *reinterpret_cast<uint4*>(buf + a * kChunkColour + h * 128) = v;
          }
        }
      }
      tc::fence_proxy_async();  // these generic-proxy writes, before the MMA reads them
      tc::fence_before_sync();  // and this thread's earlier read-out, before the MMAs that follow
      tc::mbar_arrive(full + slot);
      if (warp == 0) {  // the chunk's MMAs, once every thread has staged its row
        if (!wait_or_flag(full + slot, (uint32_t)(use & 1), fail)) break;
        tc::fence_after_sync();
        if (lane == 0) {
#pragma unroll
          for (int a = 0; a < 3; a++)
            tc::mma_bf16(tmem + (uint32_t)(d * 64 + a * 16),
                         tc::smem_desc(r0 + slot * kChunkBytes + a * kChunkColour, 128, 256),
                         tc::smem_desc(b0 + ch * 256, 128, (K / 8) * 128), idesc, ch > 0);
          tc::mma_commit(empty + slot);
          if (ch == NCH - 1) tc::mma_commit(dfull + d);
        }
        __syncwarp();
      }
    }
    if (*fail) break;
    // read-out of this tile's result buffer
    if (!wait_or_flag(dfull + d, (uint32_t)((it >> 1) & 1), fail)) break;
    tc::fence_after_sync();
#pragma unroll
    for (int a = 0; a < 3; a++) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(d * 64 + a * 16), v);
      if (valid) {
#pragma unroll
        for (int o = 0; o < COUT; o++) out[((long)(o * 3 + a) * V + se) * G.N + n] = make_float2(v[o], v[COUT + o]);
      }
    }
  }
  __syncthreads();
  if (*fail) {
    if (tid == 0) atomicAdd(&g_nn_tc_timeouts, 1);
    // let MMAs already issued finish before the tensor memory is freed: one more commit, waited
    // on with a limit
    if (warp == 0) {
      if (lane == 0) tc::mma_commit(drain);
      __syncwarp();
      tc::mbar_wait(drain, 0, kNNWaitLimit);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

template <int CIN, int COUT>
static size_t nn_tc_smem() {
  return (size_t)kRing * kChunkBytes + (size_t)16 * nn_tc_k<CIN>() * 2 + (2 * kRing + 3) * 8 + 16;
}

// Four CTAs per SM: 128 registers x 128 threads each, 52-54 KB of shared memory each, and
// 4 x 128 of the SM's 512 tensor-memory columns.
constexpr int kNNCtasPerSM = 4;

template <int CIN, int COUT>
static void tc_open() {
  const int shm = (int)nn_tc_smem<CIN, COUT>();
  cudaFuncSetAttribute(k_nn_layer_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
  cudaFuncSetAttribute(k_nn_layer_tc<CIN, COUT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
}

// Raise the shared-memory limit of every tensor-core layer instantiation and size its
// persistent grid once, before any launch (and so before any stream capture).
static int g_tc_ctas = 148 * kNNCtasPerSM;
static void tc_open_all() {
  static bool done = false;
  if (done) return;
  done = true;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  g_tc_ctas = sms * kNNCtasPerSM;
  tc_open<4, 8>();
  tc_open<8, 8>();
  tc_open<8, 4>();
  tc_open<4, 4>();
}

template <int CIN, int COUT>
static void tc_launch(const float2* in, float2* out, const __nv_bfloat162* W, const NNGeo& G, cudaStream_t st,
                      bool in_even, bool out_even) {
  tc_open_all();
  // largest Bz dividing Lz whose slab (both parities) holds at most 28 MB of input channels
  const double site_bytes = (double)CIN * 3 * G.N * sizeof(float2);
  NNTiles TL;
  TL.Bz = 1;
  for (int b = 1; b <= G.g.Lz; b++)
    if (G.g.Lz % b == 0 && (double)G.g.Lx * G.g.Ly * b * site_bytes <= 28e6) TL.Bz = b;
  TL.tps = ((long)G.g.Lxh * G.g.Ly * TL.Bz * G.N + kNNTile - 1) / kNNTile;
  TL.npar = out_even ? 1 : 2;
  TL.in_even = in_even ? 1 : 0;
  TL.ntiles = (long)(G.g.Lz / TL.Bz) * G.g.Lt * TL.npar * TL.tps;
  const long blocks = TL.ntiles < g_tc_ctas ? TL.ntiles : g_tc_ctas;
  k_nn_layer_tc<CIN, COUT><<<(unsigned)blocks, kNNThreads, nn_tc_smem<CIN, COUT>(), st>>>(in, out, W, G, TL);
  count_launch();
}

// in_even: the input vanishes on odd sites; out_even: only the even output sites are wanted.
static void layer_launch_tc(int l_in, int l_out, const float2* in, float2* out, const __nv_bfloat162* W,
                            const NNGeo& G, cudaStream_t st, bool in_even = false, bool out_even = false) {
  if (l_in == 4 && l_out == 8)
    tc_launch<4, 8>(in, out, W, G, st, in_even, out_even);
  else if (l_in == 8 && l_out == 8)
    tc_launch<8, 8>(in, out, W, G, st, in_even, out_even);
  else if (l_in == 8 && l_out == 4)
    tc_launch<8, 4>(in, out, W, G, st, in_even, out_even);
  else
    tc_launch<4, 4>(in, out, W, G, st, in_even, out_even);
}

int nn_tc_timeouts(bool reset) {
  int n = 0;
  cudaMemcpyFromSymbol(&n, g_nn_tc_timeouts, sizeof(n));
  if (reset && n) {
    const int z = 0;
    cudaMemcpyToSymbol(g_nn_tc_timeouts, &z, sizeof(z));
  }
  return n;
}

// T[p][k][se][n] = (T_p in)[k] for every path (training: the weight gradient needs them)
LQCD_D void store_t(float2* T, long i, cplx<float> v) { T[i] = make_float2(v.re, v.im); }
LQCD_D void store_t(__nv_bfloat162* T, long i, cplx<float> v) { T[i] = __floats2bfloat162_rn(v.re, v.im); }
LQCD_D float2 load_t(const float2* T, long i) { return T[i]; }
LQCD_D float2 load_t(const __nv_bfloat162* T, long i) { return __bfloat1622float2(T[i]); }

template <int C, typename TT>
__global__ void k_nn_transport(const float2* in, TT* T, NNGeo G) {
  const long V = 2 * G.g.Vh;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long se = tid / G.N;
  const int n = (int)(tid - se * G.N);
  if (se >= V) return;
  int par, x, y, z, t;
  long cb;
  nn_site(G, se, par, cb, x, y, z, t);
  const long VN = V * G.N;
  for (int p = 0; p < NN_PATHS; p++) {
    cplx<float> th[C][3];
    bool on = path_vectors<C>(G, in, p, par, cb, x, y, z, t, n, th);
#pragma unroll
    for (int c = 0; c < C; c++)
#pragma unroll
      for (int a = 0; a < 3; a++)
        store_t(T, ((long)p * C * 3 + c * 3 + a) * VN + se * G.N + n, on ? th[c][a] : cplx<float>{0.f, 0.f});
  }
}

// partial[block][p][o][c] = sum over the block's site-samples of sum_a d_o[a] conj(T_p h_c[a])
template <int CIN, int COUT, typename TT>
__global__ void k_nn_wgrad(const TT* T, const float2* d, float* partial, long VN, long per_block) {
  constexpr int TS = 16;
  extern __shared__ float2 smw[];
  float2* Ds = smw;                       // [TS][COUT*3]
  float2* Ts = smw + TS * COUT * 3;       // [TS][9][CIN*3]
  const int nthr = NN_PATHS * COUT * CIN;
  const int me = threadIdx.x;
  const int p = me / (COUT * CIN), o = (me / CIN) % COUT, c = me % CIN;
  double accr = 0, acci = 0;
  const long q0 = (long)blockIdx.x * per_block;
  const long q1 = q0 + per_block < VN ? q0 + per_block : VN;
  for (long qb = q0; qb < q1; qb += TS) {
    for (int e = threadIdx.x; e < TS * COUT * 3; e += blockDim.x) {
      int i = e / (COUT * 3), k = e % (COUT * 3);
      long q = qb + i;
      Ds[e] = q < q1 ? d[(long)k * VN + q] : make_float2(0.f, 0.f);
    }
    for (int e = threadIdx.x; e < TS * NN_PATHS * CIN * 3; e += blockDim.x) {
      int i = e / (NN_PATHS * CIN * 3), k = e % (NN_PATHS * CIN * 3);
      long q = qb + i;
      Ts[e] = q < q1 ? load_t(T, (long)k * VN + q) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (me < nthr) {
      float sr = 0, si = 0;
      for (int i = 0; i < TS; i++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
          float2 dv = Ds[i * COUT * 3 + o * 3 + a];
          float2 tv = Ts[(i * NN_PATHS + p) * CIN * 3 + c * 3 + a];
          sr += dv.x * tv.x + dv.y * tv.y;  // d * conj(t)
          si += dv.y * tv.x - dv.x * tv.y;
        }
      accr += sr;
      acci += si;
    }
    __syncthreads();
  }
  if (me < nthr) {
    partial[((long)blockIdx.x * nthr + me) * 2] = (float)accr;
    partial[((long)blockIdx.x * nthr + me) * 2 + 1] = (float)acci;
  }
}

__global__ void k_nn_sum_blocks(const float* partial, int nblocks, int nvals, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvals) return;
  double s = 0;
  for (int b = 0; b < nblocks; b++) s += partial[(long)b * nvals + i];
  out[i] = s;
}

// sums[0] += sum mask |tgt|^2, sums[1] += sum mask |out - tgt|^2 (per block partials)
__global__ void k_nn_loss_partial(const float2* out, const float2* tgt, long VN, long Vh, int N, int even_only,
                                  double* partial) {
  __shared__ double sa[256], sb[256];
  double a = 0, b = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < 12 * VN; i += (long)gridDim.x * blockDim.x) {
    long q = i % VN;
    long se = q / N;
    if (even_only && se >= Vh) continue;
    float2 o = out[i], t = tgt[i];
    a += (double)t.x * t.x + (double)t.y * t.y;
    double dx = o.x - t.x, dy = o.y - t.y;
    b += dx * dx + dy * dy;
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int s = blockDim.x / 2; s >= 1; s >>= 1) {
    if (threadIdx.x < s) {
      sa[threadIdx.x] += sa[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = sa[0];
    partial[2 * blockIdx.x + 1] = sb[0];
  }
}

__global__ void k_nn_loss_final(const double* partial, int nb, double* sums) {
  if (threadIdx.x || blockIdx.x) return;
  double a = 0, b = 0;
  for (int i = 0; i < nb; i++) {
    a += partial[2 * i];
    b += partial[2 * i + 1];
  }
  sums[0] = a;
  sums[1] = b;
  sums[2] = a > 0 ? b / a : 0.0;
}

// delta = mask (out - tgt) / sum mask |tgt|^2
__global__ void k_nn_delta(const float2* out, const float2* tgt, float2* delta, long VN, long Vh, int N,
                           int even_only, const double* sums) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 12 * VN) return;
  long se = (i % VN) / N;
  float inv = sums[0] > 0 ? (float)(1.0 / sums[0]) : 0.f;
  float2 o = out[i], t = tgt[i];
  bool on = !(even_only && se >= Vh);
  delta[i] = on ? make_float2((o.x - t.x) * inv, (o.y - t.y) * inv) : make_float2(0.f, 0.f);
}

// Adam on the real and imaginary parts: the real gradient is 2 Re / 2 Im of dL/dconj(W).
__global__ void k_nn_adam(float2* W, __nv_bfloat162* W16, const double* grad, float2* m, float2* v, int n,
                          float lr, float b1, float b2, float eps, int step) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gr = (float)(2.0 * grad[2 * i]), gi = (float)(2.0 * grad[2 * i + 1]);
  float2 mm = m[i], vv = v[i];
  mm.x = b1 * mm.x + (1 - b1) * gr;
  mm.y = b1 * mm.y + (1 - b1) * gi;
  vv.x = b2 * vv.x + (1 - b2) * gr * gr;
  vv.y = b2 * vv.y + (1 - b2) * gi * gi;
  m[i] = mm;
  v[i] = vv;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  float2 w = W[i];
  w.x -= lr * (mm.x / c1) / (sqrtf(vv.x / c2) + eps);
  w.y -= lr * (mm.y / c1) / (sqrtf(vv.y / c2) + eps);
  W[i] = w;
  W16[i] = __floats2bfloat162_rn(w.x, w.y);
}

__global__ void k_nn_to_bf16(const float2* W, __nv_bfloat162* W16, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) W16[i] = __floats2bfloat162_rn(W[i].x, W[i].y);
}

// Adjoint weights: Wa[p][c][o] = conj(W[pbar][o][c]) with pbar the reverse path (FP32 and, for the
// tensor-core backward pass, a BF16 copy).
__global__ void k_nn_adjoint_weights(const float2* W, float2* Wa, __nv_bfloat162* Wa16, int cin, int cout) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NN_PATHS * cin * cout) return;
  int p = i / (cin * cout), c = (i / cout) % cin, o = i % cout;
  int pb = p == 0 ? 0 : (p <= 4 ? p + 4 : p - 4);
  float2 w = W[(pb * cout + o) * cin + c];
  Wa[i] = make_float2(w.x, -w.y);
  if (Wa16) Wa16[i] = __floats2bfloat162_rn(w.x, -w.y);
}

// even-half FP32 spinor [6 float4][cb][nrhs] <-> NN field (4 spin channels, full lattice)
__global__ void k_nn_from_spinor(const void* r, float2* h, Geom g, int nrhs, const SegInfo* si, int nseg,
                                 const double* scale) {
  const long V = 2 * g.Vh;
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= V * nrhs) return;
  const long se = tid / nrhs;
  const int n = (int)(tid - se * nrhs);
  if (se >= g.Vh) {  // odd sites: zero
    for (int k = 0; k < 12; k++) h[((long)k * V + se) * nrhs + n] = make_float2(0.f, 0.f);
    return;
  }
  cplx<float> s[12];
  load_spinor<P32>(r, g.Vh * nrhs, se * nrhs + n, s);
  const int t = (int)(se / g.Vth);
  const float sc = scale ? (float)scale[n * nseg + (si ? si->seg_of_t[t] : 0)] : 1.f;
  for (int k = 0; k < 12; k++) h[((long)k * V + se) * nrhs + n] = make_float2(sc * s[k].re, sc * s[k].im);
}

__global__ void k_nn_to_spinor(const float2* h, void* z, Geom g, int nrhs, const SegInfo* si, int nseg,
                               const double* scale) {
  const long V = 2 * g.Vh;
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.Vh * nrhs) return;
  const long se = tid / nrhs;
  const int n = (int)(tid - se * nrhs);
  const int t = (int)(se / g.Vth);
  const float sc = scale ? (float)scale[n * nseg + (si ? si->seg_of_t[t] : 0)] : 1.f;
  cplx<float> s[12];
  for (int k = 0; k < 12; k++) {
    float2 v = h[((long)k * V + se) * nrhs + n];
    s[k] = {sc * v.x, sc * v.y};
  }
  store_spinor<P32>(z, g.Vh * nrhs, se * nrhs + n, s);
}

// lexicographic FP32 complex [n][V][4][3] <-> NN field
__global__ void k_nn_lex(const float2* a, float2* b, Geom g, int N, int to_nn, const unsigned* coord) {
  const long V = 2 * g.Vh;
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= V * N) return;
  const long se = tid / N;
  const int n = (int)(tid - se * N);
  const int par = se >= g.Vh ? 1 : 0;
  const long cb = se - (long)par * g.Vh;
  const unsigned cw = coord[(long)par * g.Vh + cb];
  const long s = (cw & 0xff) + (long)g.Lx * (((cw >> 8) & 0xff) + (long)g.Ly * (((cw >> 16) & 0xff) + (long)g.Lz * (cw >> 24)));
  for (int k = 0; k < 12; k++) {
    if (to_nn)
      b[((long)k * V + se) * N + n] = a[((long)n * V + s) * 12 + k];
    else
      b[((long)n * V + s) * 12 + k] = a[((long)k * V + se) * N + n];
  }
}

// deterministic Gaussian-like random even-site FP64 spinors (training inputs)
__global__ void k_nn_random_even(double2* b, Geom g, int nrhs, unsigned seed) {
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 2 * g.Vh * nrhs) return;
  const int n = (int)(tid % nrhs);
  const long site = tid / nrhs;
  const int par = (int)(site / g.Vh);
  const long cb = site - (long)par * g.Vh;
  for (int k = 0; k < 12; k++) {
    double2 v = make_double2(0.0, 0.0);
    if (par == 0) {
      unsigned long long h = ((unsigned long long)(cb * nrhs + n) * 12 + k) * 0x9E3779B97F4A7C15ull ^
                             ((unsigned long long)seed << 32);
      h ^= h >> 33;
      h *= 0xff51afd7ed558ccdull;
      h ^= h >> 33;
      h *= 0xc4ceb9fe1a85ec53ull;
      h ^= h >> 33;
      double u1 = ((h & 0xFFFFFFFF) + 0.5) / 4294967296.0, u2 = ((h >> 32) + 0.5) / 4294967296.0;
      double rr = sqrt(-2.0 * log(u1));
      v = make_double2(rr * cos(6.283185307179586 * u2), rr * sin(6.283185307179586 * u2));
    }
    b[((long)par * 12 * g.Vh + (k * g.Vh + cb)) * nrhs + n] = v;
  }
}

// ------------------------------------------------------------------ host side
static NNGeo nn_geo(lqcd_ctx* c, int N, int domain) {
  NNGeo G;
  G.g = c->g;
  G.coord = c->d_coord;
  G.U = (const float4*)c->U32;
  G.tc = domain ? c->d_tc_dom : c->d_tc_full;
  G.N = N;
  return G;
}

template <typename WT>
static void layer_launch(int l_in, int l_out, const float2* in, float2* out, const WT* W, const NNGeo& G,
                         cudaStream_t st) {
  const long n = 2 * G.g.Vh * (long)G.N;
  const int tpb = 128;
  const long blocks = (n + tpb - 1) / tpb;
  if (l_in == 4 && l_out == 8)
    k_nn_layer<4, 8, WT><<<blocks, tpb, 0, st>>>(in, out, W, G);
  else if (l_in == 8 && l_out == 8)
    k_nn_layer<8, 8, WT><<<blocks, tpb, 0, st>>>(in, out, W, G);
  else if (l_in == 8 && l_out == 4)
    k_nn_layer<8, 4, WT><<<blocks, tpb, 0, st>>>(in, out, W, G);
  else
    k_nn_layer<4, 4, WT><<<blocks, tpb, 0, st>>>(in, out, W, G);
  count_launch();
}

static bool nn_ensure(lqcd_ctx* c) {
  if (c->nn_weights) return true;
  const int n = nn_total_weights();
  if (cudaMalloc(&c->nn_weights, n * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&c->nn_w16, n * sizeof(__nv_bfloat162)) != cudaSuccess ||
      cudaMalloc(&c->nn_m, n * sizeof(float2)) != cudaSuccess || cudaMalloc(&c->nn_v, n * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaMemsetAsync(c->nn_m, 0, n * sizeof(float2), c->work);
  cudaMemsetAsync(c->nn_v, 0, n * sizeof(float2), c->work);
  c->nn_step = 0;
  return true;
}

int nn_set_weights(lqcd_ctx* c, const float* w_host) {
  const int n = nn_total_weights();
  if (!nn_ensure(c)) return set_error(c, LQCD_ERR_OOM, "nn: out of device memory");
  cudaMemcpyAsync(c->nn_weights, w_host, n * sizeof(float2), cudaMemcpyHostToDevice, c->work);
  k_nn_to_bf16<<<(n + 255) / 256, 256, 0, c->work>>>((const float2*)c->nn_weights, (__nv_bfloat162*)c->nn_w16, n);
  count_launch();
  cudaMemsetAsync(c->nn_m, 0, n * sizeof(float2), c->work);
  cudaMemsetAsync(c->nn_v, 0, n * sizeof(float2), c->work);
  c->nn_step = 0;
  cudaStreamSynchronize(c->work);
  return LQCD_OK;
}

int nn_get_weights(lqcd_ctx* c, float* w_host) {
  if (!c->nn_weights) return set_error(c, LQCD_ERR_STATE, "nn: no weights");
  cudaMemcpyAsync(w_host, c->nn_weights, nn_total_weights() * sizeof(float2), cudaMemcpyDeviceToHost, c->work);
  cudaStreamSynchronize(c->work);
  return LQCD_OK;
}

// Network on NN-layout fields (N samples); bf16 = 1 uses the inference weights.  a, b: ping-pong
// buffers of 8 channels; the result is in the returned pointer (4 channels).
// eo (tensor-core path): h0 vanishes on odd sites and only the even sites of the result are used
// (the even-odd preconditioned system's residual and correction), so the first layer skips the
// zero paths and the last layer the odd sites.
static float2* nn_forward(lqcd_ctx* c, const float2* h0, float2* a, float2* b, int N, int domain, bool bf16,
                          cudaStream_t st, bool tc = false, bool eo = false) {
  NNGeo G = nn_geo(c, N, domain);
  const float2* cur = h0;
  float2* bufs[2] = {a, b};
  for (int l = 0; l < NN_LAYERS; l++) {
    float2* out = bufs[l & 1];
    const int off = nn_layer_offset(l);
    if (tc)
      layer_launch_tc(NN_W[l], NN_W[l + 1], cur, out, (const __nv_bfloat162*)c->nn_w16 + off, G, st,
                      eo && l == 0, eo && l == NN_LAYERS - 1);
    else if (bf16)
      layer_launch<__nv_bfloat162>(NN_W[l], NN_W[l + 1], cur, out, (const __nv_bfloat162*)c->nn_w16 + off, G, st);
    else
      layer_launch<float2>(NN_W[l], NN_W[l + 1], cur, out, (const float2*)c->nn_weights + off, G, st);
    cur = out;
  }
  return (float2*)cur;
}

void nn_precondition(lqcd_ctx* c, const Inner& in, const void* r, void* z, const double* pscale,
                     const double* ipscale, cudaStream_t st) {
  const Geom& g = c->g;
  const int N = in.nrhs;
  const long V = 2 * g.Vh;
  const size_t fb = (size_t)24 * V * N * sizeof(float2);
  float2* h0 = (float2*)c->nn_buf[0];
  float2* a = (float2*)c->nn_buf[1];
  float2* b = (float2*)c->nn_buf[2];
  (void)fb;
  const long n = V * N;
  k_nn_from_spinor<<<(n + 255) / 256, 256, 0, st>>>(r, h0, g, N, in.si, in.nseg, pscale);
  count_launch();
  const int domain = in.tc == c->d_tc_dom && c->d_tc_dom != c->d_tc_full;
  float2* out = nn_forward(c, h0, a, b, N, domain, true, st, true, true);
  k_nn_to_spinor<<<(g.Vh * N + 255) / 256, 256, 0, st>>>(out, z, g, N, in.si, in.nseg, ipscale);
  count_launch();
}

// Reserve the three NN-layout work fields used by nn_precondition for a batch of nrhs (outside
// graph capture).
int nn_reserve(lqcd_ctx* c, int nrhs) {
  tc_open_all();
  const size_t fb = (size_t)24 * 2 * c->g.Vh * nrhs * sizeof(float2);
  for (int i = 0; i < 3; i++) {
    c->nn_buf[i] = ws_get(c, "nn_buf" + std::to_string(i), fb);
    if (!c->nn_buf[i]) return set_error(c, LQCD_ERR_OOM, "nn: out of device memory");
  }
  return LQCD_OK;
}

// Forward + loss + backward (and optionally Adam) on NN-layout input/target of N samples.
// Returns the loss through *loss; grad_host (may be NULL) receives dL/dconj(W) as float pairs.
// bf16: the training kernels of the BF16 path -- forward and backward-data layers on the tensor
// cores with BF16 weights and activations (FP32 accumulation), the transported activations kept
// in BF16 for the weight gradient (accumulated in FP32), FP32 master weights and Adam.  Otherwise
// everything in FP32 (the reference gradients of lqcd_nn_loss_grad).
static int nn_step(lqcd_ctx* c, const float2* h0, const float2* tgt, int N, int domain, int even_only,
                   double* loss, float* grad_host, bool adam, float lr, bool bf16) {
  cudaStream_t st = c->work;
  const Geom& g = c->g;
  const long V = 2 * g.Vh, VN = V * N;
  NNGeo G = nn_geo(c, N, domain);
  // activations h1..h4 (up to 8 channels) and transported copies of h0..h3
  float2* act[NN_LAYERS + 1];
  act[0] = (float2*)h0;
  void* T[NN_LAYERS];
  const size_t tsz = bf16 ? sizeof(__nv_bfloat162) : sizeof(float2);
  for (int l = 0; l < NN_LAYERS; l++) {
    act[l + 1] = (float2*)ws_get(c, "nn_act" + std::to_string(l), (size_t)NN_W[l + 1] * 3 * VN * sizeof(float2));
    T[l] = ws_get(c, "nn_T" + std::to_string(l), (size_t)NN_PATHS * NN_W[l] * 3 * VN * tsz);
    if (!act[l + 1] || !T[l]) return set_error(c, LQCD_ERR_OOM, "nn: out of device memory (training)");
  }
  __nv_bfloat162* Wa16 = (__nv_bfloat162*)ws_get(c, "nn_Wadj16", (size_t)NN_PATHS * 64 * sizeof(__nv_bfloat162));
  if (!Wa16) return set_error(c, LQCD_ERR_OOM, "nn: out of device memory");
  float2* d0 = (float2*)ws_get(c, "nn_d0", (size_t)24 * VN * sizeof(float2));
  float2* d1 = (float2*)ws_get(c, "nn_d1", (size_t)24 * VN * sizeof(float2));
  float2* Wa = (float2*)ws_get(c, "nn_Wadj", (size_t)NN_PATHS * 64 * sizeof(float2));
  double* grad = (double*)ws_get(c, "nn_grad", (size_t)2 * nn_total_weights() * sizeof(double));
  const int lblocks = 296;
  double* lpart = (double*)ws_get(c, "nn_lpart", (size_t)2 * lblocks * sizeof(double));
  double* sums = (double*)ws_get(c, "nn_sums", 4 * sizeof(double));
  if (!d0 || !d1 || !Wa || !grad || !lpart || !sums) return set_error(c, LQCD_ERR_OOM, "nn: out of device memory");
  const int tpb = 128;
  const long nb = (VN + tpb - 1) / tpb;
  for (int l = 0; l < NN_LAYERS; l++) {
    if (bf16) {
      if (NN_W[l] == 4)
        k_nn_transport<4><<<nb, tpb, 0, st>>>(act[l], (__nv_bfloat162*)T[l], G);
      else
        k_nn_transport<8><<<nb, tpb, 0, st>>>(act[l], (__nv_bfloat162*)T[l], G);
      layer_launch_tc(NN_W[l], NN_W[l + 1], act[l], act[l + 1],
                      (const __nv_bfloat162*)c->nn_w16 + nn_layer_offset(l), G, st);
    } else {
      if (NN_W[l] == 4)
        k_nn_transport<4><<<nb, tpb, 0, st>>>(act[l], (float2*)T[l], G);
      else
        k_nn_transport<8><<<nb, tpb, 0, st>>>(act[l], (float2*)T[l], G);
      layer_launch<float2>(NN_W[l], NN_W[l + 1], act[l], act[l + 1],
                           (const float2*)c->nn_weights + nn_layer_offset(l), G, st);
    }
    count_launch();
  }
  k_nn_loss_partial<<<lblocks, 256, 0, st>>>(act[NN_LAYERS], tgt, VN, g.Vh, N, even_only, lpart);
  k_nn_loss_final<<<1, 1, 0, st>>>(lpart, lblocks, sums);
  k_nn_delta<<<(12 * VN + 255) / 256, 256, 0, st>>>(act[NN_LAYERS], tgt, d0, VN, g.Vh, N, even_only, sums);
  count_launch(3);
  float2* dcur = d0;
  float2* dnext = d1;
  for (int l = NN_LAYERS - 1; l >= 0; l--) {
    const int cin = NN_W[l], cout = NN_W[l + 1], nval = NN_PATHS * cin * cout;
    const long per_block = 4096;
    const int nblk = (int)((VN + per_block - 1) / per_block);
    float* wpart = (float*)ws_get(c, "nn_wpart", (size_t)nblk * 2 * NN_PATHS * 64 * sizeof(float));
    if (!wpart) return set_error(c, LQCD_ERR_OOM, "nn: out of device memory");
    const size_t shm = (size_t)16 * (cout * 3 + NN_PATHS * cin * 3) * sizeof(float2);
    if (bf16) {
      const __nv_bfloat162* Tl = (const __nv_bfloat162*)T[l];
      if (cin == 4)
        k_nn_wgrad<4, 8><<<nblk, nval, shm, st>>>(Tl, dcur, wpart, VN, per_block);
      else if (cout == 8)
        k_nn_wgrad<8, 8><<<nblk, nval, shm, st>>>(Tl, dcur, wpart, VN, per_block);
      else
        k_nn_wgrad<8, 4><<<nblk, nval, shm, st>>>(Tl, dcur, wpart, VN, per_block);
    } else {
      const float2* Tl = (const float2*)T[l];
      if (cin == 4)
        k_nn_wgrad<4, 8><<<nblk, nval, shm, st>>>(Tl, dcur, wpart, VN, per_block);
      else if (cout == 8)
        k_nn_wgrad<8, 8><<<nblk, nval, shm, st>>>(Tl, dcur, wpart, VN, per_block);
      else
        k_nn_wgrad<8, 4><<<nblk, nval, shm, st>>>(Tl, dcur, wpart, VN, per_block);
    }
    k_nn_sum_blocks<<<(2 * nval + 255) / 256, 256, 0, st>>>(wpart, nblk, 2 * nval, grad + 2 * nn_layer_offset(l));
    count_launch(2);
    if (l > 0) {  // delta of the layer input: adjoint layer
      k_nn_adjoint_weights<<<(nval + 127) / 128, 128, 0, st>>>((const float2*)c->nn_weights + nn_layer_offset(l), Wa,
                                                               Wa16, cin, cout);
      count_launch();
      if (bf16)
        layer_launch_tc(cout, cin, dcur, dnext, Wa16, G, st);
      else
        layer_launch<float2>(cout, cin, dcur, dnext, Wa, G, st);
      std::swap(dcur, dnext);
    }
  }
  double hs[4];
  cudaMemcpyAsync(hs, sums, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (grad_host) {
    std::vector<double> gd(2 * nn_total_weights());
    cudaMemcpyAsync(gd.data(), grad, gd.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    for (size_t i = 0; i < gd.size(); i++) grad_host[i] = (float)gd[i];
  }
  if (adam) {
    c->nn_step++;
    const int n = nn_total_weights();
    k_nn_adam<<<(n + 255) / 256, 256, 0, st>>>((float2*)c->nn_weights, (__nv_bfloat162*)c->nn_w16, grad,
                                               (float2*)c->nn_m, (float2*)c->nn_v, n, lr, 0.9f, 0.999f, 1e-8f,
                                               c->nn_step);
    count_launch();
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(c, LQCD_ERR_CUDA, std::string("nn: ") + cudaGetErrorString(e));
  *loss = hs[2];
  return LQCD_OK;
}

int nn_apply_lex(lqcd_ctx* c, const float2* in_dev, float2* out_dev, int N, int domain, bool tc) {
  if (!c->nn_weights) return set_error(c, LQCD_ERR_STATE, "nn: no weights");
  const long VN = 2 * c->g.Vh * (long)N;
  float2* h0 = (float2*)ws_get(c, "nn_h0", (size_t)12 * VN * sizeof(float2));
  float2* a = (float2*)ws_get(c, "nn_pa", (size_t)24 * VN * sizeof(float2));
  float2* b = (float2*)ws_get(c, "nn_pb", (size_t)24 * VN * sizeof(float2));
  if (!h0 || !a || !b) return set_error(c, LQCD_ERR_OOM, "nn: out of device memory");
  k_nn_lex<<<(VN + 255) / 256, 256, 0, c->work>>>(in_dev, h0, c->g, N, 1, c->d_coord);
  count_launch();
  float2* out = nn_forward(c, h0, a, b, N, domain, tc, c->work, tc);
  k_nn_lex<<<(VN + 255) / 256, 256, 0, c->work>>>(out, out_dev, c->g, N, 0, c->d_coord);
  count_launch();
  return LQCD_OK;
}

int nn_loss_grad_lex(lqcd_ctx* c, const float2* in_dev, const float2* tgt_dev, int N, int domain, int even_only,
                     double* loss, float* grad_host, bool bf16) {
  if (!c->nn_weights) return set_error(c, LQCD_ERR_STATE, "nn: no weights");
  const long VN = 2 * c->g.Vh * (long)N;
  float2* h0 = (float2*)ws_get(c, "nn_h0", (size_t)12 * VN * sizeof(float2));
  float2* tg = (float2*)ws_get(c, "nn_tg", (size_t)12 * VN * sizeof(float2));
  if (!h0 || !tg) return set_error(c, LQCD_ERR_OOM, "nn: out of device memory");
  k_nn_lex<<<(VN + 255) / 256, 256, 0, c->work>>>(in_dev, h0, c->g, N, 1, c->d_coord);
  k_nn_lex<<<(VN + 255) / 256, 256, 0, c->work>>>(tgt_dev, tg, c->g, N, 1, c->d_coord);
  count_launch(2);
  return nn_step(c, h0, tg, N, domain, even_only, loss, grad_host, false, 0.f, bf16);
}

// Training pairs (r, e) with M e = r for the even-odd Schur operator M, from the plain FP64
// solver: b = (A_ee r, 0) solved with D gives x_e = M^-1 A_ee^-1 b_e = M^-1 r.  Then Adam on
// the loss |N(r) - e|^2 / |e|^2 over even sites.  loss_hist[epochs] receives the mean loss.
int nn_train(lqcd_ctx* c, int n_pairs, int epochs, int batch, double lr, int domain, unsigned seed,
             double* loss_hist) {
  cudaStream_t st = c->work;
  const Geom& g = c->g;
  if (!nn_ensure(c)) return set_error(c, LQCD_ERR_OOM, "nn: out of device memory");
  const long V = 2 * g.Vh;
  const int nb_pairs = (n_pairs + batch - 1) / batch;
  // Pairs are generated in pools that fit a quarter of the free device memory (a 32^3 x 64 pair
  // in the network layout is 400 MB, so 2000 of them cannot be resident at once): each pool is
  // generated by the solver, trained on for `epochs` passes, and replaced by the next.
  const size_t per_batch = (size_t)12 * V * batch * sizeof(float2);
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const int pool = std::max(1, std::min(nb_pairs, (int)(free_b / 4 / (2 * per_batch))));
  float2* R = (float2*)ws_get(c, "nn_pairs_r", per_batch * pool);
  float2* E = (float2*)ws_get(c, "nn_pairs_e", per_batch * pool);
  double2* b64 = (double2*)ws_get(c, "nn_b64", (size_t)2 * spinor_bytes(g, P64, batch));
  double2* x64 = (double2*)ws_get(c, "nn_x64", (size_t)2 * spinor_bytes(g, P64, batch));
  double2* r64 = (double2*)ws_get(c, "nn_r64", (size_t)2 * spinor_bytes(g, P64, batch));
  void* f32 = ws_get(c, "nn_f32", spinor_bytes(g, P32, batch));
  if (!R || !E || !b64 || !x64 || !r64 || !f32) return set_error(c, LQCD_ERR_OOM, "nn: out of device memory (pairs)");
  // the solver without the network: FP64 defect correction around FP32 BiCGStab, true residual 1e-8
  lqcd_solve_params p;
  lqcd_default_params(&p);
  p.solver = LQCD_SOLVER_MIXED;
  p.inner_prec = LQCD_PREC_F32;
  p.tol = 1e-8;
  const size_t sb64 = spinor_bytes(g, P64, batch);
  VGeom vgH = make_vgeom(g, batch, 1);
  std::vector<double> ep_sum(epochs, 0.0);
  int rounds = 0;
  for (int k0 = 0; k0 < nb_pairs; k0 += pool, rounds++) {
    const int nk = std::min(pool, nb_pairs - k0);
    for (int kk = 0; kk < nk; kk++) {
      const int k = k0 + kk;
      k_nn_random_even<<<(2 * g.Vh * batch + 255) / 256, 256, 0, st>>>(r64, g, batch, seed + 7919u * k);
      count_launch();
      cudaMemsetAsync(b64, 0, 2 * sb64, st);
      launch_clover_only(g, P64, c->A64, r64, b64, batch, st);  // b_e = A_ee r_e
      BatchStats bs;
      int rc = solve_batch(c, b64, x64, batch, domain, p, bs);
      if (rc != LQCD_OK) return rc;
      // even halves to NN layout (odd zero)
      v_convert(P64, P32, r64, f32, vgH, nullptr, 1, nullptr, st);
      k_nn_from_spinor<<<(V * batch + 255) / 256, 256, 0, st>>>(f32, R + (size_t)kk * 12 * V * batch, g, batch,
                                                               nullptr, 1, nullptr);
      v_convert(P64, P32, x64, f32, vgH, nullptr, 1, nullptr, st);
      k_nn_from_spinor<<<(V * batch + 255) / 256, 256, 0, st>>>(f32, E + (size_t)kk * 12 * V * batch, g, batch,
                                                               nullptr, 1, nullptr);
      count_launch(2);
    }
    for (int ep = 0; ep < epochs; ep++) {
      double acc = 0;
      for (int kk = 0; kk < nk; kk++) {
        double L = 0;
        int rc = nn_step(c, R + (size_t)kk * 12 * V * batch, E + (size_t)kk * 12 * V * batch, batch, domain, 1, &L,
                         nullptr, true, (float)lr, true);
        if (rc != LQCD_OK) return rc;
        acc += L;
      }
      ep_sum[ep] += acc / nk;
    }
  }
  if (loss_hist)
    for (int ep = 0; ep < epochs; ep++) loss_hist[ep] = ep_sum[ep] / rounds;
  return LQCD_OK;
}

}  // namespace lqcd
