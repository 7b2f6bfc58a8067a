// Device-side building blocks shared by the lqcd kernels: complex arithmetic, precision
// traits, field accessors for the even-odd RHS-innermost layouts, lattice geometry.
//
// Internal layouts (all half-lattice fields are indexed by parity p and checkerboard index
// cb = s >> 1 of the lexicographic site s = x + Lx (y + Ly (z + Lz t)); Lx even):
//   spinor  [chunk][cb][rhs]      chunk = 12 x double2 (P64) | 6 x float4 (P32) | 3 x uint4 (P16)
//                                 spinor component k = spin*3 + colour
//   links   [mu][p][chunk][cb]    P64: 9 x double2 (full 3x3, row major)
//                                 P32: 3 x float4, P16: 3 x uint2 (rows 0 and 1; row 2 rebuilt)
//   clover  [p][chir][chunk][cb]  packed Hermitian 6x6 per chirality (36 reals: 6 diagonal,
//                                 15 complex upper entries row-major): 18 x double2 | 9 x float4 |
//                                 9 x uint2
// The time-direction boundary phase and Dirichlet domain cuts are not stored in the links: the
// kernels read a per-timeslice coefficient (+1, -1, 0) for the forward t-hop.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define LQCD_MAXT 256
#define LQCD_HD __host__ __device__ __forceinline__
#define LQCD_D __device__ __forceinline__

namespace lqcd {

template <typename R>
struct cplx {
  R re, im;
};

template <typename R> LQCD_HD cplx<R> mk(R a, R b) { return cplx<R>{a, b}; }
template <typename R> LQCD_HD cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> LQCD_HD cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> LQCD_HD cplx<R> operator-(cplx<R> a) { return {-a.re, -a.im}; }
template <typename R> LQCD_HD cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> LQCD_HD cplx<R> operator*(R s, cplx<R> a) { return {s * a.re, s * a.im}; }
template <typename R> LQCD_HD cplx<R> cj(cplx<R> a) { return {a.re, -a.im}; }
// conj(a) * b
template <typename R> LQCD_HD cplx<R> cjmul(cplx<R> a, cplx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename R> LQCD_HD cplx<R> times_i(cplx<R> a) { return {-a.im, a.re}; }
template <typename R> LQCD_HD cplx<R> times_mi(cplx<R> a) { return {a.im, -a.re}; }
template <typename R> LQCD_HD R norm2(cplx<R> a) { return a.re * a.re + a.im * a.im; }

// Fused multiply-adds written out (each real part a chain of two FMAs), so that sums of complex
// products cost 4 FMA per term instead of products followed by separate additions.
LQCD_HD float fmx(float a, float b, float c) { return fmaf(a, b, c); }
LQCD_HD double fmx(double a, double b, double c) { return fma(a, b, c); }
// c + a b
template <typename R> LQCD_HD cplx<R> cfma(cplx<R> a, cplx<R> b, cplx<R> c) {
  return {fmx(-a.im, b.im, fmx(a.re, b.re, c.re)), fmx(a.im, b.re, fmx(a.re, b.im, c.im))};
}
// c + conj(a) b
template <typename R> LQCD_HD cplx<R> cjfma(cplx<R> a, cplx<R> b, cplx<R> c) {
  return {fmx(a.im, b.im, fmx(a.re, b.re, c.re)), fmx(-a.im, b.re, fmx(a.re, b.im, c.im))};
}
// c - a b
template <typename R> LQCD_HD cplx<R> cfms(cplx<R> a, cplx<R> b, cplx<R> c) {
  return {fmx(a.im, b.im, fmx(-a.re, b.re, c.re)), fmx(-a.im, b.re, fmx(-a.re, b.im, c.im))};
}

// ------------------------------------------------------------------ double-float arithmetic
// A value held as an unevaluated sum hi + lo of two floats (|lo| below an ulp of hi): about 48
// significant bits, computed on the FP32 pipe, which on B300 issues 64 times the FP64 pipe's
// operations.  Products use the FMA error-free product (TwoProduct: p = a b, e = fma(a, b, -p)
// exactly); sums add the high parts with Knuth's TwoSum and fold in the low parts, then
// renormalise with Quick-Two-Sum (Dekker 1971; Hida, Li & Bailey 2001).  Each operation errs by
// a few units of 2^-47 of its operands' magnitude.  The compiler must not reassociate these
// expressions, which holds without fast-math flags.
struct dfl {
  float hi, lo;
  dfl() = default;
  LQCD_HD dfl(float h, float l) : hi(h), lo(l) {}
  // conversion of a scalar parameter (a few per thread: FP64 arithmetic is fine here)
  LQCD_HD explicit dfl(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  LQCD_HD explicit dfl(int i) : hi((float)i), lo(0.f) {}
  LQCD_HD explicit operator double() const { return (double)hi + (double)lo; }
};
LQCD_HD dfl df_quick(float s, float e) {
  const float h = s + e;
  return dfl(h, e - (h - s));
}
LQCD_HD dfl operator+(dfl a, dfl b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  return df_quick(s, e);
}
LQCD_HD dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
LQCD_HD dfl operator-(dfl a, dfl b) { return a + (-b); }
LQCD_HD dfl operator*(dfl a, dfl b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return df_quick(p, e);
}
LQCD_HD dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
LQCD_HD dfl fmx(dfl a, dfl b, dfl c) { return a * b + c; }

// hi + lo = d from the bits of d, with integer operations and one int-to-float conversion (no
// FP64 arithmetic): hi = d truncated to 24 significant bits, lo = the remaining 29 bits rounded
// to 24, so |hi + lo - d| <= 2^-47 |d| for |d| >= 2^-74; below that lo loses bits gradually
// (absolute error under 2^-126 while hi is normal; |d| < 2^-126 gives zero).  |d| >= 2^128,
// infinities and NaN go to hi (lo = 0).
LQCD_D dfl split_d(double d) {
  const unsigned hw = (unsigned)__double2hiint(d), lw = (unsigned)__double2loint(d);
  const unsigned sgn = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu) - 1023;  // unbiased exponent
  if (e > 127) return dfl(__double2float_rn(d), 0.f);
  if (e < -126) return dfl(__uint_as_float(sgn), 0.f);
  const float hi = __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  // the low 29 bits are worth m 2^(e - 52): scaled in two steps, a normal power of two first, so
  // that only the last product may underflow
  const float m = __uint2float_rn(lw & 0x1fffffffu);
  const int e1 = e >= -100 ? e - 26 : e;
  const float lo = m * __uint_as_float((unsigned)(e1 + 127) << 23) * (e >= -100 ? 0x1p-26f : 0x1p-52f);
  return dfl(hi, sgn ? -lo : lo);
}

// PDF: FP64 fields, double-float arithmetic (the true-residual kernel of dslash_df.cu)
enum Prec { P64 = 0, P32 = 1, P16 = 2, PDF = 3 };

template <int P> struct Traits;
template <> struct Traits<P64> {
  using real = double;
  using schunk = double2;
  static constexpr int SCHUNKS = 12;  // complex per chunk: 1
  using lchunk = double2;
  static constexpr int LCHUNKS = 9;
  using cchunk = double2;
  static constexpr int CCHUNKS = 18;
};
template <> struct Traits<P32> {
  using real = float;
  using schunk = float4;
  static constexpr int SCHUNKS = 6;  // complex per chunk: 2
  using lchunk = float4;
  static constexpr int LCHUNKS = 3;
  using cchunk = float4;
  static constexpr int CCHUNKS = 9;
};
template <> struct Traits<P16> {
  using real = float;  // arithmetic in FP32, storage in FP16
  using schunk = uint4;
  static constexpr int SCHUNKS = 3;  // complex per chunk: 4
  using lchunk = uint2;
  static constexpr int LCHUNKS = 3;
  using cchunk = uint2;
  static constexpr int CCHUNKS = 9;
};

// ------------------------------------------------------------------ half <-> float helpers
LQCD_D float2 h2f(uint32_t w) {
  __half2 h = *reinterpret_cast<__half2*>(&w);
  return __half22float2(h);
}
LQCD_D uint32_t f2h(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// ------------------------------------------------------------------ spinor accessors
// Load the 12 components of spinor (site cb, rhs) from a half-lattice field.
template <int P>
LQCD_D void load_spinor(const void* base, long stride, long idx, cplx<typename Traits<P>::real> (&s)[12]) {
  if constexpr (P == P64) {
    const double2* f = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int c = 0; c < 12; c++) {
      double2 v = __ldg(f + c * stride + idx);
      s[c] = {v.x, v.y};
    }
  } else if constexpr (P == P32) {
    const float4* f = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int c = 0; c < 6; c++) {
      float4 v = __ldg(f + c * stride + idx);
      s[2 * c] = {v.x, v.y};
      s[2 * c + 1] = {v.z, v.w};
    }
  } else {
    const uint4* f = reinterpret_cast<const uint4*>(base);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      uint4 v = __ldg(f + c * stride + idx);
      float2 a = h2f(v.x), b = h2f(v.y), d = h2f(v.z), e = h2f(v.w);
      s[4 * c] = {a.x, a.y};
      s[4 * c + 1] = {b.x, b.y};
      s[4 * c + 2] = {d.x, d.y};
      s[4 * c + 3] = {e.x, e.y};
    }
  }
}

template <int P, typename R>
LQCD_D void store_spinor(void* base, long stride, long idx, const cplx<R> (&s)[12]) {
  if constexpr (P == P64) {
    double2* f = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int c = 0; c < 12; c++) f[c * stride + idx] = make_double2((double)s[c].re, (double)s[c].im);
  } else if constexpr (P == P32) {
    float4* f = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int c = 0; c < 6; c++)
      f[c * stride + idx] = make_float4((float)s[2 * c].re, (float)s[2 * c].im, (float)s[2 * c + 1].re,
                                        (float)s[2 * c + 1].im);
  } else {
    uint4* f = reinterpret_cast<uint4*>(base);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      uint4 v;
      v.x = f2h((float)s[4 * c].re, (float)s[4 * c].im);
      v.y = f2h((float)s[4 * c + 1].re, (float)s[4 * c + 1].im);
      v.z = f2h((float)s[4 * c + 2].re, (float)s[4 * c + 2].im);
      v.w = f2h((float)s[4 * c + 3].re, (float)s[4 * c + 3].im);
      f[c * stride + idx] = v;
    }
  }
}

// ------------------------------------------------------------------ links
// U[a][b] of link (mu, parity p, cb).  P64 stores all nine entries; P32 / P16 store rows 0 and 1
// (three 16-byte / 8-byte loads) and rebuild row 2 = conj(row0 x row1) (SU(3)): measured on
// B300, the three wide loads plus the rebuild flops beat nine narrow loads.
template <int P>
LQCD_D void load_link(const void* base, long Vh, int mu, int p, long cb, cplx<typename Traits<P>::real> (&u)[3][3]) {
  if constexpr (P == P64) {
    const double2* f = reinterpret_cast<const double2*>(base) + ((long)(mu * 2 + p) * 9) * Vh + cb;
#pragma unroll
    for (int e = 0; e < 9; e++) {
      double2 v = __ldg(f + e * Vh);
      u[e / 3][e % 3] = {v.x, v.y};
    }
  } else {
    if constexpr (P == P32) {
      const float4* f = reinterpret_cast<const float4*>(base) + ((long)(mu * 2 + p) * 3) * Vh + cb;
      float4 a = __ldg(f), b = __ldg(f + Vh), c = __ldg(f + 2 * Vh);
      u[0][0] = {a.x, a.y}; u[0][1] = {a.z, a.w}; u[0][2] = {b.x, b.y};
      u[1][0] = {b.z, b.w}; u[1][1] = {c.x, c.y}; u[1][2] = {c.z, c.w};
    } else {
      const uint2* f = reinterpret_cast<const uint2*>(base) + ((long)(mu * 2 + p) * 3) * Vh + cb;
      uint2 a = __ldg(f), b = __ldg(f + Vh), c = __ldg(f + 2 * Vh);
      float2 t;
      t = h2f(a.x); u[0][0] = {t.x, t.y};
      t = h2f(a.y); u[0][1] = {t.x, t.y};
      t = h2f(b.x); u[0][2] = {t.x, t.y};
      t = h2f(b.y); u[1][0] = {t.x, t.y};
      t = h2f(c.x); u[1][1] = {t.x, t.y};
      t = h2f(c.y); u[1][2] = {t.x, t.y};
    }
    u[2][0] = cj(cfms(u[0][2], u[1][1], u[0][1] * u[1][2]));
    u[2][1] = cj(cfms(u[0][0], u[1][2], u[0][2] * u[1][0]));
    u[2][2] = cj(cfms(u[0][1], u[1][0], u[0][0] * u[1][1]));
  }
}

// ------------------------------------------------------------------ clover (packed Hermitian 6x6)
template <int P>
LQCD_D void load_clover(const void* base, long Vh, int chir, long cb, typename Traits<P>::real (&r)[36]) {
  // base already points at the parity's block: [chir][chunk][cb]
  if constexpr (P == P64) {
    const double2* f = reinterpret_cast<const double2*>(base) + (long)chir * 18 * Vh + cb;
#pragma unroll
    for (int c = 0; c < 18; c++) {
      double2 v = __ldg(f + c * Vh);
      r[2 * c] = v.x;
      r[2 * c + 1] = v.y;
    }

  } else if constexpr (P == P32) {
    const float4* f = reinterpret_cast<const float4*>(base) + (long)chir * 9 * Vh + cb;
#pragma unroll
    for (int c = 0; c < 9; c++) {
      float4 v = __ldg(f + c * Vh);
      r[4 * c] = v.x; r[4 * c + 1] = v.y; r[4 * c + 2] = v.z; r[4 * c + 3] = v.w;
    }
  } else {
    const uint2* f = reinterpret_cast<const uint2*>(base) + (long)chir * 9 * Vh + cb;
#pragma unroll
    for (int c = 0; c < 9; c++) {
      uint2 v = __ldg(f + c * Vh);
      float2 a = h2f(v.x), b = h2f(v.y);
      r[4 * c] = a.x; r[4 * c + 1] = a.y; r[4 * c + 2] = b.x; r[4 * c + 3] = b.y;
    }
  }
}

// y = H x for a packed Hermitian 6x6 H (diag r[0..5], upper (i<j) row-major at r[6+2k], r[7+2k]).
template <typename R>
LQCD_D void herm6_apply(const R (&r)[36], const cplx<R>* x, cplx<R>* y) {
#pragma unroll
  for (int i = 0; i < 6; i++) y[i] = r[i] * x[i];
  int k = 0;
#pragma unroll
  for (int i = 0; i < 6; i++) {
#pragma unroll
    for (int j = i + 1; j < 6; j++) {
      cplx<R> c = {r[6 + 2 * k], r[7 + 2 * k]};
      y[i] = cfma(c, x[j], y[i]);
      y[j] = cjfma(c, x[i], y[j]);
      k++;
    }
  }
}

// Apply the site clover (both chiralities) of parity-block `base` to spinor s in place.
template <int P>
LQCD_D void clover_apply(const void* base, long Vh, long cb, cplx<typename Traits<P>::real> (&s)[12]) {
  using R = typename Traits<P>::real;
#pragma unroll
  for (int ch = 0; ch < 2; ch++) {
    R r[36];
    load_clover<P>(base, Vh, ch, cb, r);
    cplx<R> y[6];
    herm6_apply<R>(r, &s[6 * ch], y);
#pragma unroll
    for (int i = 0; i < 6; i++) s[6 * ch + i] = y[i];
  }
}

// ------------------------------------------------------------------ block reduction
// Sum ND values over the S sites of a block for each of its nrhs right-hand sides (threads are
// (site_local, rhs) with rhs fastest) and write partial[block][rhs][ND].  Needs ND * blockDim
// doubles of dynamic shared memory; S must be a power of two.
template <int ND>
LQCD_D void block_reduce_rhs(double (&v)[ND], double* partial, int S, int nrhs, int site_local, int rhs) {
  extern __shared__ double sm_red[];
  const int n = blockDim.x;
#pragma unroll
  for (int k = 0; k < ND; k++) sm_red[k * n + threadIdx.x] = v[k];
  __syncthreads();
  for (int s = S / 2; s >= 1; s >>= 1) {
    if (site_local < s) {
#pragma unroll
      for (int k = 0; k < ND; k++) sm_red[k * n + threadIdx.x] += sm_red[k * n + threadIdx.x + s * nrhs];
    }
    __syncthreads();
  }
  if (site_local == 0) {
#pragma unroll
    for (int k = 0; k < ND; k++)
      partial[((long)blockIdx.x * nrhs + rhs) * ND + k] = sm_red[k * n + threadIdx.x];
  }
}

// ------------------------------------------------------------------ geometry
struct Geom {
  int Lx, Ly, Lz, Lt;
  int Lxh;     // Lx / 2
  long Vh;     // V / 2
  long Vth;    // Lx Ly Lz / 2: half-lattice sites per timeslice
};

// Coordinates of checkerboard site cb of parity p.
LQCD_D void cb_coords(const Geom& g, int p, long cb, int& x, int& y, int& z, int& t) {
  long xh = cb % g.Lxh;
  long yzt = cb / g.Lxh;
  y = (int)(yzt % g.Ly);
  long zt = yzt / g.Ly;
  z = (int)(zt % g.Lz);
  t = (int)(zt / g.Lz);
  x = (int)(2 * xh) + ((p + y + z + t) & 1);
}

LQCD_HD long lex_index(const Geom& g, int x, int y, int z, int t) {
  return x + (long)g.Lx * (y + (long)g.Ly * (z + (long)g.Lz * t));
}

}  // namespace lqcd
