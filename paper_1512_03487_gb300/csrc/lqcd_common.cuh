// Shared device/host internals of the lqcd library: geometry, field formats,
// complex arithmetic, spinor / link loads and stores, the deterministic
// last-block reduction and the conjugate-gradient control block.
//
// Layout transformation (Grid paper Sec. 2.4): the paper interleaves virtual
// nodes across SIMD lanes so that one instruction serves many sites; here a
// warp's 32 threads are the lanes and the field is stored structure-of-arrays
// with the site index fastest, so every chunk load of a warp is one coalesced
// 256/512-byte transaction.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "df.cuh"
#include "lqcd.h"

namespace lqcd {

// ------------------------------------------------------------------ host utils
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
void count_launches(uint64_t n);
// Checks cudaGetLastError after a launch and counts it.
int after_launch(const char* what);

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// ------------------------------------------------------------------ geometry
// Division of n < 2^31 by a runtime constant d >= 1 with one multiply-high,
// an add and a shift (Granlund and Montgomery, "Division by invariant
// integers using multiplication", PLDI 1994, the round-up multiplier for
// unsigned N-bit operands): s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1,
// q = (mulhi(n, m) + n) >> s. n < 2^31 keeps the sum within 32 bits.
struct FastDiv {
  uint32_t d, m, s;
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.s = 0;
  while ((1ull << f.s) < d) f.s++;
  f.m = (uint32_t)(((1ull << 32) * ((1ull << f.s) - d)) / d + 1);
  return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) { return (__umulhi(n, f.m) + n) >> f.s; }

struct Geom {
  int X, Y, Z, T;
  int Xh;           // X / 2
  int Vh;           // half 4D volume
  int n5;           // inner extent (L_s or number of RHS)
  int64_t nsites;   // Vh * n5: sites of one checkerboard field (< 2^31)
  int64_t sstride;  // chunk stride of a spinor checkerboard field (sites)
  int64_t gstride;  // chunk stride of a gauge (parity, mu) block (cb sites)
  FastDiv fXh, fY, fZ, fn5;
  int st[4];        // lexicographic strides 1, X, X Y, X Y Z (4D volume < 2^31)
  float bcf[4];
  double bcd[4];
  int gp;           // G-parity direction mask of the operator (0: none); n5 = 2 flavours then
};

int make_geom(const lqcd_lattice* lat, Geom* g);  // validates, LQCD_OK or LQCD_ERR_ARG

template <int P> struct PrecTraits;
template <> struct PrecTraits<LQCD_F64> { using real = double; static constexpr int site_bytes = 192; };
template <> struct PrecTraits<LQCD_F32> { using real = float; static constexpr int site_bytes = 96; };
template <> struct PrecTraits<LQCD_F16> { using real = float; static constexpr int site_bytes = 52; };
// FP64 fields, double-float arithmetic
template <> struct PrecTraits<LQCD_F64_DF> { using real = dfl; static constexpr int site_bytes = 192; };

// Format of the iterated CG vectors x_s, r_s for a given sloppy storage format:
// FP64 stays FP64, FP32 and FP16 storage iterate in FP32.
__host__ __device__ constexpr int vec_prec(int sloppy) { return sloppy == LQCD_F64 ? LQCD_F64 : LQCD_F32; }
// Storage of the iterated residual r_s: FP16 with FP16 storage (its rounding is
// relative to the current residual, and the FP32 replacements bound its drift),
// else the vector precision.
__host__ __device__ constexpr int rs_prec(int sloppy) { return sloppy == LQCD_F16 ? LQCD_F16 : vec_prec(sloppy); }

__host__ __device__ inline int spinor_site_bytes(int prec) {
  return prec == LQCD_F64 || prec == LQCD_F64_DF ? 192 : prec == LQCD_F32 ? 96 : prec == LQCD_F16 ? 52 : 0;
}
inline int link_bytes(int prec, int recon) {
  int reals = recon == 12 ? 12 : 18;
  return reals * (prec == LQCD_F64 || prec == LQCD_F64_DF ? 8 : prec == LQCD_F32 ? 4 : 2);
}
// bytes of one checkerboard of a spinor field
__host__ __device__ inline size_t cb_spinor_bytes(const Geom& g, int prec) {
  return (size_t)g.sstride * spinor_site_bytes(prec);
}

// ------------------------------------------------------------------ complex
template <typename T> struct cpx { T r, i; };

template <typename T> __device__ __forceinline__ cpx<T> mk(T r, T i) { cpx<T> c; c.r = r; c.i = i; return c; }
template <typename T> __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.r + b.r, a.i + b.i); }
template <typename T> __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.r - b.r, a.i - b.i); }
template <typename T> __device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return mk(s * a.r, s * a.i); }
// i * a and -i * a
template <typename T> __device__ __forceinline__ cpx<T> times_i(cpx<T> a) { return mk(-a.i, a.r); }
template <typename T> __device__ __forceinline__ cpx<T> times_mi(cpx<T> a) { return mk(a.i, -a.r); }
// acc + a * b
template <typename T> __device__ __forceinline__ cpx<T> cmadd(cpx<T> acc, cpx<T> a, cpx<T> b) {
  acc.r = fma(a.r, b.r, acc.r); acc.r = fma(-a.i, b.i, acc.r);
  acc.i = fma(a.r, b.i, acc.i); acc.i = fma(a.i, b.r, acc.i);
  return acc;
}
// acc + conj(a) * b
template <typename T> __device__ __forceinline__ cpx<T> cmadd_conj(cpx<T> acc, cpx<T> a, cpx<T> b) {
  acc.r = fma(a.r, b.r, acc.r); acc.r = fma(a.i, b.i, acc.r);
  acc.i = fma(a.r, b.i, acc.i); acc.i = fma(-a.i, b.r, acc.i);
  return acc;
}
template <typename T> __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) { return cmadd(mk(T(0), T(0)), a, b); }
template <typename T> __device__ __forceinline__ cpx<T> conj(cpx<T> a) { return mk(a.r, -a.i); }

// Spinor: 12 complexes, index k = spin * 3 + colour.
template <typename T> struct Spinor { cpx<T> v[12]; };
// Half spinor: 2 spin components x 3 colours, index a * 3 + colour.
template <typename T> struct Half { cpx<T> v[6]; };
// SU(3) link, index row * 3 + col.
template <typename T> struct Link { cpx<T> v[9]; };

template <typename T> __device__ __forceinline__ void zero(Spinor<T>& s) {
#pragma unroll
  for (int k = 0; k < 12; k++) s.v[k] = mk(T(0), T(0));
}

// ------------------------------------------------------------------ spinor I/O
// A checkerboard field: base pointer and chunk stride (sites).
struct FieldPtr {
  void* p;
  int64_t stride;
};
struct CFieldPtr {
  const void* p;
  int64_t stride;
};

template <int P> struct SpinorIO;

template <> struct SpinorIO<LQCD_F64> {
  using T = double;
  static __device__ __forceinline__ void load(const void* base, int64_t stride, int64_t j, Spinor<T>& s) {
    const double2* b = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int c = 0; c < 12; c++) {
      double2 w = __ldg(b + c * stride + j);
      s.v[c] = mk(w.x, w.y);
    }
  }
  static __device__ __forceinline__ void store(void* base, int64_t stride, int64_t j, const Spinor<T>& s) {
    double2* b = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int c = 0; c < 12; c++) __stcs(b + c * stride + j, make_double2(s.v[c].r, s.v[c].i));
  }
};

template <> struct SpinorIO<LQCD_F32> {
  using T = float;
  static __device__ __forceinline__ void load(const void* base, int64_t stride, int64_t j, Spinor<T>& s) {
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int c = 0; c < 6; c++) {
      float4 w = __ldg(b + c * stride + j);
      s.v[2 * c] = mk(w.x, w.y);
      s.v[2 * c + 1] = mk(w.z, w.w);
    }
  }
  static __device__ __forceinline__ void store(void* base, int64_t stride, int64_t j, const Spinor<T>& s) {
    float4* b = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int c = 0; c < 6; c++)
      __stcs(b + c * stride + j, make_float4(s.v[2 * c].r, s.v[2 * c].i, s.v[2 * c + 1].r, s.v[2 * c + 1].i));
  }
};

// FP64 fields read into / written from double-float arithmetic (the split and
// the recombination of df.cuh; the layout is the FP64 one).
template <> struct SpinorIO<LQCD_F64_DF> {
  using T = dfl;
  static __device__ __forceinline__ void load(const void* base, int64_t stride, int64_t j, Spinor<T>& s) {
    const double2* b = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int c = 0; c < 12; c++) {
      const double2 w = __ldg(b + c * stride + j);
      s.v[c] = mk(df_split(w.x), df_split(w.y));
    }
  }
  static __device__ __forceinline__ void store(void* base, int64_t stride, int64_t j, const Spinor<T>& s) {
    double2* b = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int c = 0; c < 12; c++) __stcs(b + c * stride + j, make_double2(df_to_double(s.v[c].r), df_to_double(s.v[c].i)));
  }
};

// FP16: 3 chunks of 8 halves (4 complexes), then a float norm per site.
template <> struct SpinorIO<LQCD_F16> {
  using T = float;
  static __device__ __forceinline__ const float* norm_ptr(const void* base, int64_t stride) {
    return reinterpret_cast<const float*>(reinterpret_cast<const char*>(base) + 48 * stride);
  }
  static __device__ __forceinline__ void load(const void* base, int64_t stride, int64_t j, Spinor<T>& s) {
    const uint4* b = reinterpret_cast<const uint4*>(base);
    float nrm = __ldg(norm_ptr(base, stride) + j);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      uint4 w = __ldg(b + c * stride + j);
      unsigned int words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int q = 0; q < 4; q++) {
        __half2 h = *reinterpret_cast<__half2*>(&words[q]);
        float2 f = __half22float2(h);
        s.v[4 * c + q] = mk(f.x * nrm, f.y * nrm);
      }
    }
  }
  // Components without the site norm (returned separately), so that a caller
  // can apply the norm after a linear map that shrinks the data (spin projection).
  static __device__ __forceinline__ void load_unscaled(const void* base, int64_t stride, int64_t j, Spinor<T>& s,
                                                       float& nrm) {
    const uint4* b = reinterpret_cast<const uint4*>(base);
    nrm = __ldg(norm_ptr(base, stride) + j);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      uint4 w = __ldg(b + c * stride + j);
      unsigned int words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int q = 0; q < 4; q++) {
        float2 f = __half22float2(*reinterpret_cast<__half2*>(&words[q]));
        s.v[4 * c + q] = mk(f.x, f.y);
      }
    }
  }
  static __device__ __forceinline__ void store(void* base, int64_t stride, int64_t j, const Spinor<T>& s) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; k++) m = fmaxf(m, fmaxf(fabsf(s.v[k].r), fabsf(s.v[k].i)));
    float inv = m > 0.f ? 1.0f / m : 0.f;
    uint4* b = reinterpret_cast<uint4*>(base);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      unsigned int words[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        __half2 h = __floats2half2_rn(s.v[4 * c + q].r * inv, s.v[4 * c + q].i * inv);
        words[q] = *reinterpret_cast<unsigned int*>(&h);
      }
      __stcs(b + c * stride + j, make_uint4(words[0], words[1], words[2], words[3]));
    }
    float* nb = const_cast<float*>(norm_ptr(base, stride));
    __stcs(nb + j, m);
  }
};

// ------------------------------------------------------------------ link I/O
// Gauge block (parity, mu) starts at chunk (parity * 4 + mu) * NCHUNK.
template <int P, int R> struct LinkIO;

// conj(a b - c d) as two chains of a multiply and three fused multiply-adds
template <typename T> __device__ __forceinline__ cpx<T> conj_cross(cpx<T> a, cpx<T> b, cpx<T> c, cpx<T> d) {
  T re = a.r * b.r;
  re = fma(-a.i, b.i, re);
  re = fma(-c.r, d.r, re);
  re = fma(c.i, d.i, re);
  T im = -(a.r * b.i);
  im = fma(-a.i, b.r, im);
  im = fma(c.r, d.i, im);
  im = fma(c.i, d.r, im);
  return mk(re, im);
}

template <typename T> __device__ __forceinline__ void rebuild_row2(Link<T>& u) {
  // row2 = conj(row0 x row1) (SU(3): the rows are orthonormal and det = 1)
  u.v[6] = conj_cross(u.v[1], u.v[5], u.v[2], u.v[4]);
  u.v[7] = conj_cross(u.v[2], u.v[3], u.v[0], u.v[5]);
  u.v[8] = conj_cross(u.v[0], u.v[4], u.v[1], u.v[3]);
}

template <> struct LinkIO<LQCD_F64, 18> {
  using T = double;
  static constexpr int NCHUNK = 9;
  static __device__ __forceinline__ void load(const void* g, int64_t gs, int blk, int64_t cb, Link<T>& u) {
    const double2* b = reinterpret_cast<const double2*>(g) + (int64_t)blk * NCHUNK * gs + cb;
#pragma unroll
    for (int c = 0; c < 9; c++) { double2 w = __ldg(b + c * gs); u.v[c] = mk(w.x, w.y); }
  }
};
template <> struct LinkIO<LQCD_F64, 12> {
  using T = double;
  static constexpr int NCHUNK = 6;
  static __device__ __forceinline__ void load(const void* g, int64_t gs, int blk, int64_t cb, Link<T>& u) {
    const double2* b = reinterpret_cast<const double2*>(g) + (int64_t)blk * NCHUNK * gs + cb;
#pragma unroll
    for (int c = 0; c < 6; c++) { double2 w = __ldg(b + c * gs); u.v[c] = mk(w.x, w.y); }
    rebuild_row2(u);
  }
};
template <> struct LinkIO<LQCD_F64_DF, 18> {
  using T = dfl;
  static constexpr int NCHUNK = 9;
  static __device__ __forceinline__ void load(const void* g, int64_t gs, int blk, int64_t cb, Link<T>& u) {
    const double2* b = reinterpret_cast<const double2*>(g) + (int64_t)blk * NCHUNK * gs + cb;
#pragma unroll
    for (int c = 0; c < 9; c++) { double2 w = __ldg(b + c * gs); u.v[c] = mk(df_split(w.x), df_split(w.y)); }
  }
};
template <> struct LinkIO<LQCD_F64_DF, 12> {
  using T = dfl;
  static constexpr int NCHUNK = 6;
  static __device__ __forceinline__ void load(const void* g, int64_t gs, int blk, int64_t cb, Link<T>& u) {
    const double2* b = reinterpret_cast<const double2*>(g) + (int64_t)blk * NCHUNK * gs + cb;
#pragma unroll
    for (int c = 0; c < 6; c++) { double2 w = __ldg(b + c * gs); u.v[c] = mk(df_split(w.x), df_split(w.y)); }
    rebuild_row2(u);
  }
};
template <> struct LinkIO<LQCD_F32, 18> {
  using T = float;
  static constexpr int NCHUNK = 9;
  static __device__ __forceinline__ void load(const void* g, int64_t gs, int blk, int64_t cb, Link<T>& u) {
    const float2* b = reinterpret_cast<const float2*>(g) + (int64_t)blk * NCHUNK * gs + cb;
#pragma unroll
    for (int c = 0; c < 9; c++) { float2 w = __ldg(b + c * gs); u.v[c] = mk(w.x, w.y); }
  }
};
template <> struct LinkIO<LQCD_F32, 12> {
  using T = float;
  static constexpr int NCHUNK = 3;
  static __device__ __forceinline__ void load(const void* g, int64_t gs, int blk, int64_t cb, Link<T>& u) {
    const float4* b = reinterpret_cast<const float4*>(g) + (int64_t)blk * NCHUNK * gs + cb;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      float4 w = __ldg(b + c * gs);
      u.v[2 * c] = mk(w.x, w.y);
      u.v[2 * c + 1] = mk(w.z, w.w);
    }
    rebuild_row2(u);
  }
};
template <> struct LinkIO<LQCD_F16, 18> {
  using T = float;
  static constexpr int NCHUNK = 9;
  static __device__ __forceinline__ void load(const void* g, int64_t gs, int blk, int64_t cb, Link<T>& u) {
    const unsigned int* b = reinterpret_cast<const unsigned int*>(g) + (int64_t)blk * NCHUNK * gs + cb;
#pragma unroll
    for (int c = 0; c < 9; c++) {
      unsigned int w = __ldg(b + c * gs);
      float2 f = __half22float2(*reinterpret_cast<__half2*>(&w));
      u.v[c] = mk(f.x, f.y);
    }
  }
};
template <> struct LinkIO<LQCD_F16, 12> {
  using T = float;
  static constexpr int NCHUNK = 3;
  static __device__ __forceinline__ void load(const void* g, int64_t gs, int blk, int64_t cb, Link<T>& u) {
    const uint2* b = reinterpret_cast<const uint2*>(g) + (int64_t)blk * NCHUNK * gs + cb;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      uint2 w = __ldg(b + c * gs);
      float2 f0 = __half22float2(*reinterpret_cast<__half2*>(&w.x));
      float2 f1 = __half22float2(*reinterpret_cast<__half2*>(&w.y));
      u.v[2 * c] = mk(f0.x, f0.y);
      u.v[2 * c + 1] = mk(f1.x, f1.y);
    }
    rebuild_row2(u);
  }
};

// ------------------------------------------------------------------ site coordinates
// 32-bit index arithmetic throughout: the 4D volume is below 2^31 (checked
// when the geometry is made), so lexicographic and checkerboard indices fit.
struct Coord {
  int c[4];      // x, y, z, t
  uint32_t lex;  // x + X (y + Y (z + Z t))
};

__device__ __forceinline__ Coord cb_to_coord(const Geom& g, int64_t cb64, int parity) {
  Coord r;
  const uint32_t cb = (uint32_t)cb64;
  const uint32_t q = fdiv(cb, g.fXh);
  const uint32_t xh = cb - q * (uint32_t)g.Xh;
  const uint32_t q2 = fdiv(q, g.fY);
  r.c[1] = (int)(q - q2 * (uint32_t)g.Y);
  const uint32_t q3 = fdiv(q2, g.fZ);
  r.c[2] = (int)(q2 - q3 * (uint32_t)g.Z);
  r.c[3] = (int)q3;
  r.c[0] = (int)(2 * xh) + ((parity + r.c[1] + r.c[2] + r.c[3]) & 1);
  r.lex = (uint32_t)r.c[0] + 2 * q * (uint32_t)g.Xh;  // x + X (y + Y (z + Z t))
  return r;
}

// Checkerboard index of the neighbour one hop along +-mu, and whether the hop wraps.
template <int MU>
__device__ __forceinline__ int64_t neighbour_cb(const Geom& g, const Coord& x, int sign, bool& wrap) {
  const int L = MU == 0 ? g.X : MU == 1 ? g.Y : MU == 2 ? g.Z : g.T;
  const uint32_t st = (uint32_t)g.st[MU];
  uint32_t lex;
  if (sign > 0) {
    wrap = x.c[MU] == L - 1;
    lex = wrap ? x.lex - (uint32_t)(L - 1) * st : x.lex + st;
  } else {
    wrap = x.c[MU] == 0;
    lex = wrap ? x.lex + (uint32_t)(L - 1) * st : x.lex - st;
  }
  return (int64_t)(lex >> 1);
}

// ------------------------------------------------------------------ CG control
// One independent linear system (one RHS) of a solve.
struct SysState {
  double rr;      // iterated |r|^2 entering the current iteration
  double rr0;     // |b|^2
  double maxrr;   // max iterated |r|^2 since the last reliable update
  double alpha, beta;
  double pAp;
  double rr_new;
  double tol2;    // tol^2 * rr0
  double delta2;  // delta^2 (0 disables reliable updates)
  double rr_true; // last FP64 true |r|^2
  double maxrr_mid;   // max iterated |r|^2 since the last residual replacement of either level
  double delta2_mid;  // delta_mid^2 (0 disables the FP32-arithmetic replacements)
  double ss0;         // CGNR: |b|^2 of the system M x = b
  double tol2_sys;    // CGNR: tol^2 ssx, the exit test on the FP64 |b - M x|^2
  double ssx;         // CGNR: the exit test's scale |b'|^2: ss0, or the full system's |b|^2 of an even-odd solve
  int done;
  int pad;
};

// REASON_MID: an FP32-arithmetic residual replacement is due (three-level scheme).
enum { REASON_CONVERGED = 1, REASON_RELIABLE = 2, REASON_NAN = 4, REASON_MID = 8 };

struct Control {
  int active;      // 1 while inner iterations run; gated kernels return at once when 0
  int reason;      // REASON_* bits explaining a pause / a pending reliable update
  int iter;        // inner iterations completed
  int nsys;
  int n_done;
  int n_reliable;  // FP64 residual recomputations done
  int chunk_left;  // device-driven loop: iterations left in the current graph launch
  int n_mid;       // FP32-arithmetic residual replacements done
};

// What the last block of a reducing kernel does with the per-system totals.
enum Finalize {
  FIN_STORE = 0,     // result[sys] = total
  FIN_ALPHA = 1,     // total = p^dag A p -> alpha
  FIN_UPDATE = 2,    // total = |r_new|^2 -> beta or pause
  FIN_INIT = 3,      // total = |b|^2 -> initial state
  FIN_RELIABLE = 4,  // total = FP64 true |r|^2 -> done flags, beta, resume
  FIN_MID = 5,       // total = |r_ref - A x_s|^2 with FP32 arithmetic -> beta, resume
};

struct ReduceCtx {
  double* partials;       // [nsys][gridDim.x]
  unsigned int* counter;  // zero between uses
  double* result;         // FIN_STORE target [nsys]
  SysState* sys;
  Control* ctrl;
  int nsys;
  int fin;
  double tol2_rel;        // FIN_INIT: tol^2
  double delta2;          // FIN_INIT: delta^2
  double delta2_mid;      // FIN_INIT: delta_mid^2 (0 = no intermediate replacements)
  int sysres;             // FIN_INIT / FIN_RELIABLE of CGNR: result[s] holds |b|^2 / the FP64 |b - M x|^2,
                          // which sets and decides the exit test (tol applies to M x = b)
  const double* scale2;   // FIN_INIT of CGNR, or null: per-system |b|^2 that the exit test scales tol by instead
                          // of result[s] (an even-odd solve: the full system's source, so that tol applies to
                          // ||b - D x|| / ||b||, whose even rows are b_hat - M_hat x_e and odd rows vanish)
  int maxiter;            // FIN_UPDATE: request a final FP64 residual once this many iterations ran
  int cond;               // FIN_UPDATE: 1 = set h_rel / h_mid (device-driven graph), 0 = pause for the host
  cudaGraphConditionalHandle h_rel;  // IF node running the reliable update (when cond)
  cudaGraphConditionalHandle h_mid;  // IF node running the FP32-arithmetic replacement (when cond)
};

__device__ __forceinline__ bool gate_closed(const Control* ctrl) {
  return ctrl != nullptr && *((volatile const int*)&ctrl->active) == 0;
}

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

// Runs on one thread of the last block with the per-system totals.
__device__ inline void finalize_totals(const ReduceCtx& rc, const double* totals) {
  const int nsys = rc.nsys;
  switch (rc.fin) {
    case FIN_STORE:
      for (int s = 0; s < nsys; s++) rc.result[s] = totals[s];
      break;
    case FIN_ALPHA: {
      bool bad = false;
      for (int s = 0; s < nsys; s++) {
        SysState& st = rc.sys[s];
        st.pAp = totals[s];
        if (st.done) { st.alpha = 0.0; continue; }
        if (!(totals[s] > 0.0) || !finite(totals[s])) { bad = true; st.alpha = 0.0; }
        else st.alpha = st.rr / totals[s];
      }
      if (bad) { rc.ctrl->reason |= REASON_NAN; rc.ctrl->active = 0; }
    } break;
    case FIN_UPDATE: {
      int reason = 0;
      for (int s = 0; s < nsys; s++) {
        SysState& st = rc.sys[s];
        st.rr_new = totals[s];
        if (st.done) continue;
        if (!finite(totals[s])) reason |= REASON_NAN;
        else if (totals[s] <= st.tol2) reason |= REASON_CONVERGED;
        else if (totals[s] <= st.delta2 * st.maxrr) reason |= REASON_RELIABLE;
        else if (st.delta2_mid > 0.0 && totals[s] <= st.delta2_mid * st.maxrr_mid) reason |= REASON_MID;
      }
      rc.ctrl->iter += 1;
      const bool at_cap = rc.maxiter > 0 && rc.ctrl->iter >= rc.maxiter;
      const bool rel_due = (reason & (REASON_CONVERGED | REASON_RELIABLE)) || at_cap;
      if (reason & REASON_NAN) {
        rc.ctrl->reason |= REASON_NAN;
        rc.ctrl->active = 0;
      } else if (rel_due || (reason & REASON_MID)) {
        // A residual recomputation is due -- FP64 (convergence, delta, or the
        // iteration cap, where the true residual must be known) or, failing
        // those, the FP32-arithmetic replacement: beta waits for it.
        rc.ctrl->reason |= rel_due ? (reason & ~REASON_MID) : REASON_MID;
        if (rc.cond) cudaGraphSetConditional(rel_due ? rc.h_rel : rc.h_mid, 1);  // run that branch now
        else rc.ctrl->active = 0;                                                  // pause for the host
      } else {
        for (int s = 0; s < nsys; s++) {
          SysState& st = rc.sys[s];
          if (st.done) { st.beta = 0.0; continue; }
          st.beta = totals[s] / st.rr;
          st.rr = totals[s];
          st.maxrr = fmax(st.maxrr, totals[s]);
          st.maxrr_mid = fmax(st.maxrr_mid, totals[s]);
        }
      }
    } break;
    case FIN_INIT: {
      int n_done = 0;
      bool bad = false;
      for (int s = 0; s < nsys; s++) {
        SysState& st = rc.sys[s];
        const double t = totals[s];
        st.rr = st.rr0 = st.maxrr = st.maxrr_mid = st.rr_true = st.rr_new = t;
        st.alpha = st.beta = st.pAp = 0.0;
        st.tol2 = rc.tol2_rel * t;
        st.delta2 = rc.delta2;
        st.delta2_mid = rc.delta2_mid;
        st.ss0 = rc.sysres ? rc.result[s] : t;
        st.ssx = rc.scale2 ? rc.scale2[s] : st.ss0;
        st.tol2_sys = rc.tol2_rel * st.ssx;
        if (!finite(t) || !finite(st.ss0) || !finite(st.ssx)) bad = true;
        st.done = (t == 0.0 || st.ss0 == 0.0) ? 1 : 0;
        n_done += st.done;
      }
      rc.ctrl->nsys = nsys;
      rc.ctrl->n_done = n_done;
      rc.ctrl->iter = 0;
      rc.ctrl->n_reliable = 0;
      rc.ctrl->n_mid = 0;
      rc.ctrl->chunk_left = 0;
      rc.ctrl->reason = bad ? REASON_NAN : 0;
      rc.ctrl->active = (!bad && n_done < nsys) ? 1 : 0;
    } break;
    case FIN_RELIABLE: {
      int n_done = 0;
      bool bad = false;
      for (int s = 0; s < nsys; s++) {
        SysState& st = rc.sys[s];
        const double t = totals[s];
        // CGNR: the exit test is on the FP64 |b - M x|^2; t = |M^dag (b - M x)|^2 restarts the recurrence
        const double ss = rc.sysres ? rc.result[s] : t;
        st.rr_true = ss;
        if (!st.done) {
          if (!finite(t) || !finite(ss)) bad = true;
          else if (ss <= (rc.sysres ? st.tol2_sys : st.tol2)) { st.done = 1; st.beta = 0.0; }
          else {
            st.beta = t / st.rr;
            st.rr = t;
            st.maxrr = t;
            st.maxrr_mid = t;
            // the iterated |r|^2 at which |b - M x|^2 should meet the tolerance, if the two stay
            // proportional (with a factor 2 of margin), requests the next FP64 check
            if (rc.sysres) st.tol2 = fmin(st.tol2, 0.5 * t * st.tol2_sys / ss);
          }
        }
        n_done += st.done;
      }
      rc.ctrl->n_done = n_done;
      rc.ctrl->n_reliable += 1;
      rc.ctrl->reason = bad ? REASON_NAN : 0;
      rc.ctrl->active = (!bad && n_done < nsys) ? 1 : 0;
    } break;
    case FIN_MID: {
      // The replaced residual is only FP32-accurate: it restarts the
      // recurrence (beta, the replacement maximum) but never decides
      // convergence; that stays with the FP64 reliable update.
      bool bad = false;
      for (int s = 0; s < nsys; s++) {
        SysState& st = rc.sys[s];
        if (st.done) continue;
        const double t = totals[s];
        if (!finite(t)) { bad = true; continue; }
        st.beta = t / st.rr;
        st.rr = t;
        st.maxrr = fmax(st.maxrr, t);
        st.maxrr_mid = t;
      }
      rc.ctrl->n_mid += 1;
      rc.ctrl->reason = bad ? REASON_NAN : 0;
      rc.ctrl->active = (!bad && rc.ctrl->n_done < nsys) ? 1 : 0;
    } break;
  }
}

// After every block has written its partials rc.partials[s * gridDim.x +
// blockIdx.x] (s < nsys, written by thread s of the block), the block that
// finishes last (atomic ticket; no block ever waits for another) sums them per
// system in a fixed order and runs the finaliser. `sh` is BLOCK doubles of
// shared scratch. Every thread of the block must call it. Only the writers of
// partials fence: a fence in every thread would also wait for the thread's
// streaming stores of the kernel's output, holding the block's warps
// resident after their work is done.
template <int BLOCK>
__device__ __forceinline__ void last_block_finalize(const ReduceCtx& rc, double* sh) {
  __shared__ double totals[64];
  __shared__ int is_last;
  const int tid = threadIdx.x;
  if (tid < rc.nsys) __threadfence();
  __syncthreads();
  if (tid == 0) {
    unsigned int ticket = atomicAdd(rc.counter, 1u);
    is_last = ticket == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int s = 0; s < rc.nsys; s++) {
    double acc = 0.0;
    const double* part = rc.partials + (int64_t)s * gridDim.x;
    for (int b = tid; b < (int)gridDim.x; b += BLOCK) acc += __ldcg(part + b);
    sh[tid] = acc;
    __syncthreads();
    for (int w = BLOCK / 2; w > 0; w >>= 1) {
      if (tid < w) sh[tid] += sh[tid + w];
      __syncthreads();
    }
    if (tid == 0) totals[s] = sh[0];
    __syncthreads();
  }
  if (tid == 0) {
    finalize_totals(rc, totals);
    *rc.counter = 0u;
  }
}

// Deterministic two-level reduction of one value per thread, grouped by
// system (thread's system = global index mod nsys when nsys > 1). V is the
// field's arithmetic type: a warp sums its 32 values in V (FP32 for FP32 and
// FP16 fields: on GB300 FP64 instructions are scarce, and 32 site norms summed
// in FP32 keep a relative error near 1e-6), everything above the warp is FP64.
// Per-block partials go to rc.partials; the last block to finish (atomic
// ticket, no waiting) sums them in a fixed order and runs the finaliser. Every
// thread of the block must call it.
template <int BLOCK, typename V>
__device__ __forceinline__ void block_reduce_finalize(V v, int64_t block_first_gid, const ReduceCtx& rc) {
  __shared__ double sh[BLOCK];
  const int tid = threadIdx.x;
  const int nsys = rc.nsys;
  if (nsys == 1) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) sh[tid >> 5] = (double)v;
    __syncthreads();
    if (tid == 0) {
      double w = 0.0;
#pragma unroll
      for (int k = 0; k < BLOCK / 32; k++) w += sh[k];
      rc.partials[blockIdx.x] = w;
    }
  } else {
    __shared__ V shv[BLOCK];
    shv[tid] = v;
    __syncthreads();
    if (tid < nsys) {
      int first = (int)((tid - block_first_gid % nsys + nsys) % nsys);
      double s = 0.0;
      for (int k = first; k < BLOCK; k += nsys) s += (double)shv[k];
      rc.partials[(int64_t)tid * gridDim.x + blockIdx.x] = s;
    }
  }
  last_block_finalize<BLOCK>(rc, sh);
}

// block_reduce_finalize for SPT values per thread: value s of thread t belongs to
// global index block_first_gid + s BLOCK + t (the layout of the two-site hop).
template <int BLOCK, int SPT, typename V>
__device__ __forceinline__ void block_reduce_finalize_n(const V (&v)[SPT], int64_t block_first_gid,
                                                        const ReduceCtx& rc) {
  if constexpr (SPT == 1) {
    block_reduce_finalize<BLOCK>(v[0], block_first_gid, rc);
  } else {
    const int nsys = rc.nsys;
    if (nsys == 1) {
      V sum = v[0];
#pragma unroll
      for (int s = 1; s < SPT; s++) sum += v[s];
      block_reduce_finalize<BLOCK>(sum, block_first_gid, rc);
      return;
    }
    __shared__ double sh[BLOCK];
    __shared__ V shv[BLOCK * SPT];
    const int tid = threadIdx.x;
#pragma unroll
    for (int s = 0; s < SPT; s++) shv[s * BLOCK + tid] = v[s];
    __syncthreads();
    if (tid < nsys) {
      const int first = (int)((tid - block_first_gid % nsys + nsys) % nsys);
      double acc = 0.0;
      for (int k = first; k < BLOCK * SPT; k += nsys) acc += (double)shv[k];
      rc.partials[(int64_t)tid * gridDim.x + blockIdx.x] = acc;
    }
    last_block_finalize<BLOCK>(rc, sh);
  }
}

// System index of a site index j = cb * n5 + i5.
__device__ __forceinline__ int sys_of(int64_t j, int nsys) { return nsys == 1 ? 0 : (int)(j % nsys); }

constexpr int MAX_SYS = 64;

}  // namespace lqcd
