// Per-site bodies of the conjugate-gradient vector kernels, shared by the
// single-lattice solver (cg.cu) and the batched solver (batch.cu). VF is the
// format of the iterated solution x_s (FP64 or FP32) and the arithmetic of the
// iterated vectors, RF the storage of the iterated residual r_s (VF, or FP16
// with FP16 storage); SF the format of the vectors the Dslash reads and writes,
// p and Ap (FP64, FP32 or FP16). Each returning function gives the site's
// contribution to the next reduction.
#pragma once

#include "lqcd_common.cuh"

namespace lqcd {

// |s|^2 in the spinor's own arithmetic type (the reductions above the warp are FP64)
template <typename T> __device__ __forceinline__ T site_norm2(const Spinor<T>& s) {
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < 12; k++) acc = fma(s.v[k].r, s.v[k].r, fma(s.v[k].i, s.v[k].i, acc));
  return acc;
}

template <typename TD, typename TS> __device__ __forceinline__ void convert(const Spinor<TS>& a, Spinor<TD>& b) {
#pragma unroll
  for (int k = 0; k < 12; k++) b.v[k] = mk((TD)a.v[k].r, (TD)a.v[k].i);
}

// r = b, r_s = b, p = b, x_s = 0, x = 0; returns |b|^2
template <int VF, int SF, int RF = VF>
__device__ __forceinline__ double init_site(const Geom& g, int64_t j, const double* b64, double* r64, double* x64,
                                            void* rs, void* xs, void* p) {
  using TV = typename PrecTraits<VF>::real;
  using TS = typename PrecTraits<SF>::real;
  Spinor<double> b, z;
  SpinorIO<LQCD_F64>::load(b64, g.sstride, j, b);
  SpinorIO<LQCD_F64>::store(r64, g.sstride, j, b);
  zero(z);
  SpinorIO<LQCD_F64>::store(x64, g.sstride, j, z);
  Spinor<TV> bv, zv;
  convert(b, bv);
  zero(zv);
  SpinorIO<RF>::store(rs, g.sstride, j, bv);
  SpinorIO<VF>::store(xs, g.sstride, j, zv);
  Spinor<TS> bs;
  convert(b, bs);
  SpinorIO<SF>::store(p, g.sstride, j, bs);
  return site_norm2(b);
}

// x_s += alpha p; r_s -= alpha Ap with Ap given in registers; returns |r_s|^2 (in VF's type)
template <int VF, int SF, int RF = VF, typename TA>
__device__ __forceinline__ typename PrecTraits<VF>::real update_site_ap(const Geom& g, int64_t j, double alpha_d, const void* p_,
                                                 const Spinor<TA>& ap, void* xs, void* rs) {
  using TV = typename PrecTraits<VF>::real;
  using TS = typename PrecTraits<SF>::real;
  const TV alpha = (TV)alpha_d;
  Spinor<TS> p;
  SpinorIO<SF>::load(p_, g.sstride, j, p);
  Spinor<TV> x, r;
  SpinorIO<VF>::load(xs, g.sstride, j, x);
  SpinorIO<RF>::load(rs, g.sstride, j, r);
#pragma unroll
  for (int k = 0; k < 12; k++) {
    x.v[k] = mk(fma(alpha, (TV)p.v[k].r, x.v[k].r), fma(alpha, (TV)p.v[k].i, x.v[k].i));
    r.v[k] = mk(fma(-alpha, (TV)ap.v[k].r, r.v[k].r), fma(-alpha, (TV)ap.v[k].i, r.v[k].i));
  }
  SpinorIO<VF>::store(xs, g.sstride, j, x);
  SpinorIO<RF>::store(rs, g.sstride, j, r);
  return site_norm2(r);
}

// x_s += alpha p; r_s -= alpha Ap; returns |r_s|^2 (in VF's type)
template <int VF, int SF, int RF = VF>
__device__ __forceinline__ typename PrecTraits<VF>::real update_site(const Geom& g, int64_t j, double alpha_d, const void* p_,
                                              const void* ap_, void* xs, void* rs) {
  Spinor<typename PrecTraits<SF>::real> ap;
  SpinorIO<SF>::load(ap_, g.sstride, j, ap);
  return update_site_ap<VF, SF, RF>(g, j, alpha_d, p_, ap, xs, rs);
}

// p = r_s + beta p
template <int VF, int SF, int RF = VF>
__device__ __forceinline__ void pupdate_site(const Geom& g, int64_t j, double beta_d, const void* rs, void* pp) {
  using TV = typename PrecTraits<VF>::real;
  using TS = typename PrecTraits<SF>::real;
  const TS beta = (TS)beta_d;
  Spinor<TV> r;
  SpinorIO<RF>::load(rs, g.sstride, j, r);
  Spinor<TS> p;
  SpinorIO<SF>::load(pp, g.sstride, j, p);
#pragma unroll
  for (int k = 0; k < 12; k++) p.v[k] = mk(fma(beta, p.v[k].r, (TS)r.v[k].r), fma(beta, p.v[k].i, (TS)r.v[k].i));
  SpinorIO<SF>::store(pp, g.sstride, j, p);
}

// x += x_s (FP64); x_s = 0
template <int VF>
__device__ __forceinline__ void accumulate_site(const Geom& g, int64_t j, double* x64, void* xs) {
  using TV = typename PrecTraits<VF>::real;
  Spinor<double> x;
  SpinorIO<LQCD_F64>::load(x64, g.sstride, j, x);
  Spinor<TV> d, z;
  SpinorIO<VF>::load(xs, g.sstride, j, d);
#pragma unroll
  for (int k = 0; k < 12; k++) x.v[k] = mk(x.v[k].r + (double)d.v[k].r, x.v[k].i + (double)d.v[k].i);
  zero(z);
  SpinorIO<LQCD_F64>::store(x64, g.sstride, j, x);
  SpinorIO<VF>::store(xs, g.sstride, j, z);
}

// r = b - A x (FP64), r_s = r; returns |r|^2 in FP64. With b64 null, ax64
// already holds the residual (CGNR: M^dag (b - M x)) and r = ax.
template <int VF, int RF = VF>
__device__ __forceinline__ double residual_site(const Geom& g, int64_t j, const double* b64, const double* ax64,
                                                double* r64, void* rs) {
  using TV = typename PrecTraits<VF>::real;
  Spinor<double> b, ax;
  SpinorIO<LQCD_F64>::load(ax64, g.sstride, j, ax);
  if (b64) {
    SpinorIO<LQCD_F64>::load(b64, g.sstride, j, b);
#pragma unroll
    for (int k = 0; k < 12; k++) b.v[k] = b.v[k] - ax.v[k];
  } else {
    b = ax;
  }
  SpinorIO<LQCD_F64>::store(r64, g.sstride, j, b);
  Spinor<TV> rv;
  convert(b, rv);
  SpinorIO<RF>::store(rs, g.sstride, j, rv);
  return site_norm2(b);
}

// CGNR reliable update: r = M^dag (b - M x) applied with FP32 arithmetic (ax32),
// stored as the FP64 r (the replacements' reference) and as r_s; returns |r|^2
template <int VF, int RF = VF>
__device__ __forceinline__ typename PrecTraits<VF>::real residual32_site(const Geom& g, int64_t j, const void* ax32,
                                                                         double* r64, void* rs) {
  using TV = typename PrecTraits<VF>::real;
  Spinor<float> r;
  SpinorIO<LQCD_F32>::load(ax32, g.sstride, j, r);
  Spinor<double> rd;
  convert(r, rd);
  SpinorIO<LQCD_F64>::store(r64, g.sstride, j, rd);
  Spinor<TV> rv;
  convert(r, rv);
  SpinorIO<RF>::store(rs, g.sstride, j, rv);
  return site_norm2(rv);
}

// Intermediate replacement: r_s = r - A x_s, r the FP64 residual of the last
// reliable update and A x_s an FP32 field computed with FP32 arithmetic;
// returns |r_s|^2. The difference is taken in FP32: A x_s carries FP32 error
// already, and the subtraction adds at most one rounding of r_s itself.
template <int VF, int RF = VF>
__device__ __forceinline__ typename PrecTraits<VF>::real mid_residual_site(const Geom& g, int64_t j, const double* r64, const void* ax32,
                                                    void* rs) {
  using TV = typename PrecTraits<VF>::real;
  Spinor<double> r;
  SpinorIO<LQCD_F64>::load(r64, g.sstride, j, r);
  Spinor<float> ax;
  SpinorIO<LQCD_F32>::load(ax32, g.sstride, j, ax);
  Spinor<TV> rv;
#pragma unroll
  for (int k = 0; k < 12; k++)
    rv.v[k] = mk((TV)((float)r.v[k].r - ax.v[k].r), (TV)((float)r.v[k].i - ax.v[k].i));
  SpinorIO<RF>::store(rs, g.sstride, j, rv);
  return site_norm2(rv);
}

}  // namespace lqcd
