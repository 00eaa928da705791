// Pseudofermion force for S = phi^dag (M^dag M)^-1 phi, M = D_W.
//
// The Grid paper lists HMC among its algorithms (Sec. 4); the force formula
// is the textbook derivative. With X = (M^dag M)^-1 phi and Y = M X, the only
// terms of dS that involve the link U_mu(x) are the two hops through it:
//   dS = ph Re[ tr(dU A) + tr(dU^dag B) ],
//   A = sum_spin X(x+mu) ((1 - gamma_mu) Y(x))^dag,
//   B = sum_spin ((1 + gamma_mu) X(x)) Y(x+mu)^dag,
// ph = the link's boundary phase. Because (1 -+ gamma) has rank two, each sum
// is two colour outer products of half spinors: A = sum_a g_a h_a^dag with g,
// h the (1 - gamma_mu) projections of X(x+mu) and Y(x) (and likewise B with
// 1 + gamma_mu), which the kernel forms with the same projection code as the
// hop. Outputs per link: the conjugate-Wirtinger gradient A^dag + B, or the
// traceless Hermitian force TA[i (G - G^dag) / 2] with G = U A - B U^dag.
#include "lqcd_internal.h"

namespace lqcd {

constexpr int FORCE_BLOCK = 128;

struct ForceArgs {
  double2* out;
  const void* gauge;
  const void* X;
  const void* Y;
  Geom g;
  int64_t half_bytes;
  int kind;
  int accumulate;  // 1: out -= coef * force (molecular-dynamics momentum update)
  double coef;
};

// M = sum_a g_a h_a^dag (colour outer products of two half spinors)
__device__ __forceinline__ void outer(const Half<double>& g, const Half<double>& h, cpx<double> m[9]) {
#pragma unroll
  for (int r = 0; r < 3; r++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      cpx<double> s = cmadd_conj(mk(0.0, 0.0), h.v[c], g.v[r]);
      m[3 * r + c] = cmadd_conj(s, h.v[3 + c], g.v[3 + r]);
    }
}

template <int MU, int R>
__device__ __forceinline__ void force_dir(const ForceArgs& a, const Coord& x, int64_t cb, int parity,
                                          const Spinor<double>& xs, const Spinor<double>& ys) {
  bool wrap;
  const int64_t nb = neighbour_cb<MU>(a.g, x, +1, wrap);
  const char* Xn = static_cast<const char*>(a.X) + (1 - parity) * a.half_bytes;
  const char* Yn = static_cast<const char*>(a.Y) + (1 - parity) * a.half_bytes;
  Spinor<double> xn, yn;
  SpinorIO<LQCD_F64>::load(Xn, a.g.sstride, nb, xn);
  SpinorIO<LQCD_F64>::load(Yn, a.g.sstride, nb, yn);
  Half<double> ga, ha, gb, hb;
  project<MU, -1>(xn, ga);
  project<MU, -1>(ys, ha);
  project<MU, +1>(xs, gb);
  project<MU, +1>(yn, hb);
  cpx<double> A[9], B[9];
  outer(ga, ha, A);
  outer(gb, hb, B);
  const double ph = wrap ? a.g.bcd[MU] : 1.0;
  cpx<double> out[9];
  if (a.kind == LQCD_FORCE_GRAD) {
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
      for (int c = 0; c < 3; c++) out[3 * r + c] = ph * (conj(A[3 * c + r]) + B[3 * r + c]);
  } else {
    Link<double> u;
    LinkIO<LQCD_F64, R>::load(a.gauge, a.g.gstride, parity * 4 + MU, cb, u);
    cpx<double> G[9];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        cpx<double> s = mk(0.0, 0.0);
#pragma unroll
        for (int k = 0; k < 3; k++) {
          s = cmadd(s, u.v[3 * r + k], A[3 * k + c]);      // (U A)_rc
          s = s - cmul(B[3 * r + k], conj(u.v[3 * c + k]));  // (B U^dag)_rc
        }
        G[3 * r + c] = ph * s;
      }
    // F = i (G - G^dag) / 2, then remove the trace
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        cpx<double> d = G[3 * r + c] - conj(G[3 * c + r]);
        out[3 * r + c] = times_i(0.5 * d);
      }
    const double tr = (out[0].r + out[4].r + out[8].r) / 3.0;
    out[0].r -= tr;
    out[4].r -= tr;
    out[8].r -= tr;
  }
  double2* o = a.out + (int64_t)(parity * 4 + MU) * 9 * a.g.gstride + cb;
  if (a.accumulate) {
#pragma unroll
    for (int k = 0; k < 9; k++) {
      const double2 w = o[k * a.g.gstride];
      o[k * a.g.gstride] = make_double2(w.x - a.coef * out[k].r, w.y - a.coef * out[k].i);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 9; k++) o[k * a.g.gstride] = make_double2(out[k].r, out[k].i);
  }
}

template <int R>
__global__ void __launch_bounds__(FORCE_BLOCK) force_kernel(const ForceArgs a) {
  const int64_t t = (int64_t)blockIdx.x * FORCE_BLOCK + threadIdx.x;
  if (t >= 2 * (int64_t)a.g.Vh) return;
  const int parity = t >= a.g.Vh ? 1 : 0;
  const int64_t cb = t - parity * (int64_t)a.g.Vh;
  const Coord x = cb_to_coord(a.g, cb, parity);
  Spinor<double> xs, ys;
  SpinorIO<LQCD_F64>::load(static_cast<const char*>(a.X) + parity * a.half_bytes, a.g.sstride, cb, xs);
  SpinorIO<LQCD_F64>::load(static_cast<const char*>(a.Y) + parity * a.half_bytes, a.g.sstride, cb, ys);
  force_dir<0, R>(a, x, cb, parity, xs, ys);
  force_dir<1, R>(a, x, cb, parity, xs, ys);
  force_dir<2, R>(a, x, cb, parity, xs, ys);
  force_dir<3, R>(a, x, cb, parity, xs, ys);
}

static int launch_force(const ForceArgs& a, int recon, cudaStream_t s) {
  const unsigned grid = (unsigned)((2 * (int64_t)a.g.Vh + FORCE_BLOCK - 1) / FORCE_BLOCK);
  if (recon == 18) force_kernel<18><<<grid, FORCE_BLOCK, 0, s>>>(a);
  else force_kernel<12><<<grid, FORCE_BLOCK, 0, s>>>(a);
  return after_launch("force_kernel");
}

int force_accumulate(double2* mom, const void* gauge, const void* X, const void* Y, const Geom& g, int recon,
                     double coef, cudaStream_t s) {
  ForceArgs a{mom, gauge, X, Y, g, (int64_t)cb_spinor_bytes(g, LQCD_F64), LQCD_FORCE_TA, 1, coef};
  return launch_force(a, recon, s);
}

}  // namespace lqcd

using namespace lqcd;

extern "C" int lqcd_force(void* out, const void* gauge, const void* X, const void* Y, const lqcd_lattice* lat,
                          const lqcd_operator* op, int kind, void* stream) {
  Geom g;
  int st = make_geom(lat, &g);
  if (st) return st;
  if ((st = check_operator(op, g))) return st;
  if (op->kind != LQCD_WILSON || op->prec != LQCD_F64 || g.n5 != 1)
    return fail(LQCD_ERR_UNSUPPORTED, "lqcd_force: Wilson operator, LQCD_F64 and n5 == 1 only");
  if (kind != LQCD_FORCE_TA && kind != LQCD_FORCE_GRAD) return fail(LQCD_ERR_ARG, "lqcd_force: bad kind %d", kind);
  if (!out || !gauge || !X || !Y || (((uintptr_t)out | (uintptr_t)gauge | (uintptr_t)X | (uintptr_t)Y) & 15))
    return fail(LQCD_ERR_ARG, "lqcd_force: null or misaligned pointer");
  ForceArgs a{static_cast<double2*>(out), gauge, X, Y, g, (int64_t)cb_spinor_bytes(g, LQCD_F64), kind, 0, 0.0};
  return launch_force(a, op->recon, (cudaStream_t)stream);
}
