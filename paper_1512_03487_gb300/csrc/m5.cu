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
// Two kernels. When L_s divides 32, the warp-shuffle scan of the recurrence
// (m5_scan.cuh): each thread reads and writes its own spinor once. The
// L_s-replicated hop runs the same scan in its epilogue (EPI_M5INV), so inside
// the Schur operator this kernel is only needed for other L_s, where the
// closed-form sum above runs, one thread per output site reading the L_s
// source spinors of its 4D site (through L1).
#include <cmath>

#include "lqcd_internal.h"
#include "m5_scan.cuh"

namespace lqcd {

template <int P>
__global__ void __launch_bounds__(M5_BLOCK) m5inv_scan_kernel(const M5Args a, double ainv, double den_inv) {
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
  m5inv_lanes(v, s, Ls, a.dagger != 0, (T)ainv, (T)a.mf, (T)den_inv);
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
  if (m5_scan_ok(Ls)) {  // L_s divides the warp: the shuffle scan
    const double ainv = 1.0 / a.d, den_inv = 1.0 / (1.0 + a.mf * std::pow(ainv, (double)Ls));
    switch (prec) {
      case LQCD_F64: m5inv_scan_kernel<LQCD_F64><<<(unsigned)nb, M5_BLOCK, 0, s>>>(a, ainv, den_inv); break;
      case LQCD_F32: m5inv_scan_kernel<LQCD_F32><<<(unsigned)nb, M5_BLOCK, 0, s>>>(a, ainv, den_inv); break;
      case LQCD_F16: m5inv_scan_kernel<LQCD_F16><<<(unsigned)nb, M5_BLOCK, 0, s>>>(a, ainv, den_inv); break;
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
