// Inverse of the site-local fifth-dimension operator of the Shamir domain-wall
// fermion (the block the L_s-replicated hop of the Grid paper, Sec. 3, is
// preconditioned with):
//
//   M5op = d - P_- S_up - P_+ S_down,   d = 5 - M5,
//   (S_up psi)(s) = psi(s+1), (S_up psi)(L_s-1) = -mf psi(0);  S_down = S_up^T.
//
// On chirality + the matrix is d - L with L the twisted cyclic shift s-1 -> s
// (twist -mf), and L^Ls = -mf, so the Neumann series closes:
//   (d - L)^-1 = sum_{k=0}^{L_s-1} L^k / d^(k+1) / (1 + mf / d^Ls),
// i.e. x(s) = sum_k c_k w_k b(s - k mod L_s), c_k = d^-(k+1) / (1 + mf d^-Ls),
// w_k = -mf if s - k wrapped below 0, else 1. Chirality - uses b(s + k).
// The adjoint swaps the two.
//
// Two kernels. When L_s divides 32 the L_s threads of a 4D site sit in one warp
// (site index j = cb L_s + s) and solve the recurrence itself with shuffles:
// on chirality +, with a = 1/d,
//   y(s) = a (b(s) + y(s-1)), y(-1) = 0      (a Kogge-Stone scan: log2 L_s steps)
//   x(s) = y(s) - mf a^(s+1) y(L_s-1) / (1 + mf a^L_s)
// (the twisted wrap enters once, through y(L_s-1)); chirality - runs the same
// scan from the top. Each thread reads and writes its own spinor once. Other
// L_s use the closed-form sum above, one thread per output site reading the
// L_s source spinors of its 4D site (through L1).
#include <cmath>

#include "lqcd_internal.h"

namespace lqcd {

// Shuffle of one spinor half (6 complex values) within segments of `width` lanes.
template <typename T>
__device__ __forceinline__ cpx<T> shfl_up_c(cpx<T> v, int o, int width) {
  return mk(__shfl_up_sync(0xffffffffu, v.r, o, width), __shfl_up_sync(0xffffffffu, v.i, o, width));
}
template <typename T>
__device__ __forceinline__ cpx<T> shfl_down_c(cpx<T> v, int o, int width) {
  return mk(__shfl_down_sync(0xffffffffu, v.r, o, width), __shfl_down_sync(0xffffffffu, v.i, o, width));
}
template <typename T>
__device__ __forceinline__ cpx<T> shfl_idx_c(cpx<T> v, int lane, int width) {
  return mk(__shfl_sync(0xffffffffu, v.r, lane, width), __shfl_sync(0xffffffffu, v.i, lane, width));
}

// v[q0..q0+5] <- (d - L)^-1 of one chirality, in place. up: L shifts s-1 -> s
// (the recurrence runs upward in s), else s+1 -> s. t = distance of this lane
// from the recurrence's start (s or L_s-1-s).
template <typename T>
__device__ __forceinline__ void m5_scan(Spinor<T>& v, int q0, bool up, int t, int Ls, T a, T corr_t) {
#pragma unroll
  for (int q = 0; q < 6; q++) v.v[q0 + q] = a * v.v[q0 + q];
  T ao = a;  // a^o
  for (int o = 1; o < Ls; o <<= 1) {
#pragma unroll
    for (int q = 0; q < 6; q++) {
      const cpx<T> w = up ? shfl_up_c(v.v[q0 + q], o, Ls) : shfl_down_c(v.v[q0 + q], o, Ls);
      if (t >= o) v.v[q0 + q] = mk(fma(ao, w.r, v.v[q0 + q].r), fma(ao, w.i, v.v[q0 + q].i));
    }
    ao *= ao;
  }
  // wrap: x = y - corr_t y_end, corr_t = mf a^(t+1) / (1 + mf a^Ls)
  const int end = up ? Ls - 1 : 0;
#pragma unroll
  for (int q = 0; q < 6; q++) {
    const cpx<T> ye = shfl_idx_c(v.v[q0 + q], end, Ls);
    v.v[q0 + q] = mk(fma(-corr_t, ye.r, v.v[q0 + q].r), fma(-corr_t, ye.i, v.v[q0 + q].i));
  }
}

// corr[t] = mf a^(t+1) / (1 + mf a^L_s), t < L_s, computed on the host
struct M5Corr {
  double c[32];
};

template <int P>
__global__ void __launch_bounds__(M5_BLOCK) m5inv_scan_kernel(const M5Args a, const M5Corr corr) {
  using T = typename PrecTraits<P>::real;
  using IO = SpinorIO<P>;
  if (gate_closed(a.gate)) return;
  const int64_t j = (int64_t)blockIdx.x * M5_BLOCK + threadIdx.x;
  const bool live = j < a.g.nsites;  // dead lanes still shuffle (whole segments, never stored)
  const int Ls = a.g.n5;
  const int s = (int)(threadIdx.x & (unsigned)(Ls - 1));  // L_s divides 32 and the block size
  Spinor<T> v;
  if (live) IO::load(a.in, a.g.sstride, j, v);
  else zero(v);
  const T ainv = (T)(1.0 / a.d);
  // chirality + recurs upward without dagger, downward with it; chirality - the other way
  const bool plus_up = !a.dagger;
  const int t_up = s, t_down = Ls - 1 - s;
  const T corr_up = (T)corr.c[t_up], corr_down = (T)corr.c[t_down];
  m5_scan(v, 0, plus_up, plus_up ? t_up : t_down, Ls, ainv, plus_up ? corr_up : corr_down);
  m5_scan(v, 6, !plus_up, plus_up ? t_down : t_up, Ls, ainv, plus_up ? corr_down : corr_up);
  if (live) IO::store(a.out, a.g.sstride, j, v);
}

template <int P>
__global__ void __launch_bounds__(M5_BLOCK) m5inv_kernel(const M5Args a, double scale) {
  using T = typename PrecTraits<P>::real;
  using IO = SpinorIO<P>;
  if (gate_closed(a.gate)) return;
  const int64_t j = (int64_t)blockIdx.x * M5_BLOCK + threadIdx.x;
  if (j >= a.g.nsites) return;
  const int Ls = a.g.n5;
  const int64_t base = j / Ls * Ls;
  const int s = (int)(j - base);
  const T dinv = (T)(1.0 / a.d);
  const T mf = (T)a.mf;
  T coef = (T)(scale / a.d);
  Spinor<T> out;
  zero(out);
  for (int k = 0; k < Ls; k++) {
    int sd = s - k;
    T wd = T(1);
    if (sd < 0) { sd += Ls; wd = -mf; }
    int su = s + k;
    T wu = T(1);
    if (su >= Ls) { su -= Ls; wu = -mf; }
    Spinor<T> bd, bu;
    IO::load(a.in, a.g.sstride, base + sd, bd);
    IO::load(a.in, a.g.sstride, base + su, bu);
    const T cd = coef * wd, cu = coef * wu;
    // non-dagger: chirality + (k < 6) takes b(s - k), chirality - takes b(s + k)
#pragma unroll
    for (int q = 0; q < 6; q++) {
      if (!a.dagger) {
        out.v[q] = out.v[q] + cd * bd.v[q];
        out.v[6 + q] = out.v[6 + q] + cu * bu.v[6 + q];
      } else {
        out.v[q] = out.v[q] + cu * bu.v[q];
        out.v[6 + q] = out.v[6 + q] + cd * bd.v[6 + q];
      }
    }
    coef *= dinv;
  }
  IO::store(a.out, a.g.sstride, j, out);
}

int launch_m5inv(int prec, const M5Args& a, cudaStream_t s) {
  const int64_t nb = (a.g.nsites + M5_BLOCK - 1) / M5_BLOCK;
  if (nb == 0) return LQCD_OK;
  const int Ls = a.g.n5;
  if (Ls >= 2 && Ls <= 32 && (Ls & (Ls - 1)) == 0) {  // L_s divides the warp: the shuffle scan
    M5Corr corr;
    const double ainv = 1.0 / a.d, den = 1.0 + a.mf * std::pow(ainv, (double)Ls);
    double at = ainv;  // a^(t+1)
    for (int t = 0; t < 32; t++) {
      corr.c[t] = t < Ls ? a.mf * at / den : 0.0;
      at *= ainv;
    }
    switch (prec) {
      case LQCD_F64: m5inv_scan_kernel<LQCD_F64><<<(unsigned)nb, M5_BLOCK, 0, s>>>(a, corr); break;
      case LQCD_F32: m5inv_scan_kernel<LQCD_F32><<<(unsigned)nb, M5_BLOCK, 0, s>>>(a, corr); break;
      case LQCD_F16: m5inv_scan_kernel<LQCD_F16><<<(unsigned)nb, M5_BLOCK, 0, s>>>(a, corr); break;
      default: return fail(LQCD_ERR_ARG, "bad precision %d", prec);
    }
    return after_launch("m5inv_scan_kernel");
  }
  const double scale = 1.0 / (1.0 + a.mf * std::pow(a.d, -(double)a.g.n5));
  switch (prec) {
    case LQCD_F64: m5inv_kernel<LQCD_F64><<<(unsigned)nb, M5_BLOCK, 0, s>>>(a, scale); break;
    case LQCD_F32: m5inv_kernel<LQCD_F32><<<(unsigned)nb, M5_BLOCK, 0, s>>>(a, scale); break;
    case LQCD_F16: m5inv_kernel<LQCD_F16><<<(unsigned)nb, M5_BLOCK, 0, s>>>(a, scale); break;
    default: return fail(LQCD_ERR_ARG, "bad precision %d", prec);
  }
  return after_launch("m5inv_kernel");
}

}  // namespace lqcd
