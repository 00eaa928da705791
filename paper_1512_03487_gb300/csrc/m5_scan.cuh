// Warp-shuffle scan for the inverse of the domain-wall fifth-dimension
// operator M5op = d - P_- S_up - P_+ S_down (d = 5 - M5, mf-twisted wrap), used
// by the M5op^-1 kernel and fused into the epilogue of the L_s-replicated hop.
// The L_s threads of a 4D site (site index j = cb L_s + s, L_s dividing 32) sit
// in one warp. On chirality +, with a = 1/d, the lower-triangular part is the
// recurrence y(s) = a (b(s) + y(s-1)), solved by a Kogge-Stone scan in
// log2 L_s shuffle steps; the twisted wrap then enters once:
//   x(s) = y(s) - corr(s) y(L_s-1),  corr(t) = mf a^(t+1) / (1 + mf a^L_s).
// Chirality - runs the same scan from the top; the adjoint swaps the two.
#pragma once

#include "lqcd_common.cuh"

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
// double-float values: both halves of each part
__device__ __forceinline__ dfl shfl_up_df(dfl v, int o, int width) {
  return dfl(__shfl_up_sync(0xffffffffu, v.hi, o, width), __shfl_up_sync(0xffffffffu, v.lo, o, width));
}
__device__ __forceinline__ dfl shfl_down_df(dfl v, int o, int width) {
  return dfl(__shfl_down_sync(0xffffffffu, v.hi, o, width), __shfl_down_sync(0xffffffffu, v.lo, o, width));
}
__device__ __forceinline__ dfl shfl_idx_df(dfl v, int lane, int width) {
  return dfl(__shfl_sync(0xffffffffu, v.hi, lane, width), __shfl_sync(0xffffffffu, v.lo, lane, width));
}
template <>
__device__ __forceinline__ cpx<dfl> shfl_up_c<dfl>(cpx<dfl> v, int o, int width) {
  return mk(shfl_up_df(v.r, o, width), shfl_up_df(v.i, o, width));
}
template <>
__device__ __forceinline__ cpx<dfl> shfl_down_c<dfl>(cpx<dfl> v, int o, int width) {
  return mk(shfl_down_df(v.r, o, width), shfl_down_df(v.i, o, width));
}
template <>
__device__ __forceinline__ cpx<dfl> shfl_idx_c<dfl>(cpx<dfl> v, int lane, int width) {
  return mk(shfl_idx_df(v.r, lane, width), shfl_idx_df(v.i, lane, width));
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
    ao = ao * ao;
  }
  // wrap: x = y - corr_t y_end, corr_t = mf a^(t+1) / (1 + mf a^Ls)
  const int end = up ? Ls - 1 : 0;
#pragma unroll
  for (int q = 0; q < 6; q++) {
    const cpx<T> ye = shfl_idx_c(v.v[q0 + q], end, Ls);
    v.v[q0 + q] = mk(fma(-corr_t, ye.r, v.v[q0 + q].r), fma(-corr_t, ye.i, v.v[q0 + q].i));
  }
}

// corr(t) = mf a^(t+1) den_inv, a^(t+1) by binary powering (at most six products)
template <typename T>
__device__ __forceinline__ T m5_corr(int t, T a, T mf, T den_inv) {
  T p = T(1), base = a;
  for (int e = t + 1; e; e >>= 1) {
    if (e & 1) p = p * base;
    base = base * base;
  }
  return mf * p * den_inv;
}

// v <- M5op^-1 v (or its adjoint) across the L_s lanes of each 4D site; s = lane's
// fifth coordinate; every lane of the warp must call it.
template <typename T>
__device__ __forceinline__ void m5inv_lanes(Spinor<T>& v, int s, int Ls, bool dagger, T a, T mf, T den_inv) {
  const bool plus_up = !dagger;  // chirality + recurs upward without dagger, downward with it
  const int t_up = s, t_down = Ls - 1 - s;
  const T corr_up = m5_corr(t_up, a, mf, den_inv), corr_down = m5_corr(t_down, a, mf, den_inv);
  m5_scan(v, 0, plus_up, plus_up ? t_up : t_down, Ls, a, plus_up ? corr_up : corr_down);
  m5_scan(v, 6, !plus_up, plus_up ? t_down : t_up, Ls, a, plus_up ? corr_down : corr_up);
}

// L_s values the shuffle scan serves (the lanes of a 4D site within one warp)
__host__ __device__ inline bool m5_scan_ok(int Ls) { return Ls >= 2 && Ls <= 32 && (Ls & (Ls - 1)) == 0; }

}  // namespace lqcd
