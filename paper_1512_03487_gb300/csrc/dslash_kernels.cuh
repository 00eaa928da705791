// Fused Wilson hopping kernel (and its L_s-replicated / multi-RHS form).
//
//   out(x) = sum_mu (1 - gamma_mu) U_mu(x) in(x + mu) + (1 + gamma_mu) U_mu(x - mu)^dag in(x - mu)
//
// One thread per output site j = cb * n5 + i5 of one checkerboard. For each
// of the 8 directions the neighbour spinor is loaded (coalesced SoA chunks),
// spin-projected to a half spinor (the paper's Compressor, Sec. 2.6, applied
// in registers instead of to a halo), multiplied by the SU(3) link (2 colour
// vectors), reconstructed to 4 spins and accumulated; the result is written
// once with streaming stores (Sec. 2.6 "streaming stores are used in the
// final write"). With n5 > 1 the n5 threads of a 4D site read the same link
// address, so the link bytes are fetched once per site for all i5 (the
// paper's L_s-fold gauge reuse, Sec. 3 Fig. xc30 caption).
//
// Gamma basis (chiral): gamma_mu = [[0, B_mu], [B_mu^dag, 0]] with
// B_x = -i sigma_1, B_y = -i sigma_2, B_z = -i sigma_3, B_t = 1. For
// (1 + S gamma_mu) psi (S = +-1) the upper half is h = psi_u + S B psi_l and
// the lower half is S B^dag h, so only h is multiplied by the link.
#pragma once

#include "cg_site.cuh"
#include "hop_pair.cuh"
#include "lqcd_common.cuh"
#include "m5_scan.cuh"

namespace lqcd {

// EPI_M5INV: out = M5op^-1 (b H in), the inverse applied across the L_s lanes of
// each 4D site by the warp-shuffle scan (domain wall, L_s dividing 32).
enum Epilogue { EPI_PLAIN = 0, EPI_XPAY = 1, EPI_M5 = 2, EPI_M5INV = 3 };

struct HopArgs {
  void* out;
  const void* in;
  const void* gauge;
  const void* x;          // epilogue operand, same format and subset as out
  Geom g;
  int out_parity;         // single-checkerboard launch: parity of out
  int full;               // 1: out / in / x are full fields, grid covers both parities
  int blocks_per_parity;
  int64_t half_bytes;     // bytes of one checkerboard of a full field
  double a, b;            // EPI_PLAIN: out = b H in; EPI_XPAY: out = a x + b H in
  double m5d, mf;         // EPI_M5: out = M5op(x) + b H in, M5op diagonal m5d = 5 - M5
  int m5_dagger;          // EPI_M5INV: apply the adjoint of M5op^-1
  double m5_a;            // EPI_M5INV: 1 / (5 - M5)
  double m5_den_inv;      // EPI_M5INV: 1 / (1 + mf (5 - M5)^-L_s)
  ReduceCtx red;          // |out|^2 per system (RED_NORM) or |r_s|^2 (RED_CG_UPDATE)
  const Control* gate;    // kernel returns at once when gate->active == 0
  // RED_CG_UPDATE: out = A p is not stored; instead x_s += alpha p and
  // r_s -= alpha A p, alpha = red.sys[system].alpha. p is in the format of
  // out; x_s and r_s in vec_prec of it (upd_half_bytes: one checkerboard).
  const void* upd_p;
  void* upd_xs;
  void* upd_rs;             // in rs_prec of out's format
  int64_t upd_half_bytes;
  int64_t upd_rs_half_bytes;
};

// Reduction / epilogue modes of the hop kernel.
enum HopReduce { RED_NONE = 0, RED_NORM = 1, RED_CG_UPDATE = 2 };

template <int MU, int S, typename T>
__device__ __forceinline__ void project(const Spinor<T>& s, Half<T>& h) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const cpx<T> p0 = s.v[c], p1 = s.v[3 + c], p2 = s.v[6 + c], p3 = s.v[9 + c];
    cpx<T> h0, h1;
    if (MU == 0) {         // h0 = p0 - S i p3, h1 = p1 - S i p2
      h0 = S > 0 ? p0 + times_mi(p3) : p0 + times_i(p3);
      h1 = S > 0 ? p1 + times_mi(p2) : p1 + times_i(p2);
    } else if (MU == 1) {  // h0 = p0 - S p3, h1 = p1 + S p2
      h0 = S > 0 ? p0 - p3 : p0 + p3;
      h1 = S > 0 ? p1 + p2 : p1 - p2;
    } else if (MU == 2) {  // h0 = p0 - S i p2, h1 = p1 + S i p3
      h0 = S > 0 ? p0 + times_mi(p2) : p0 + times_i(p2);
      h1 = S > 0 ? p1 + times_i(p3) : p1 + times_mi(p3);
    } else {               // h0 = p0 + S p2, h1 = p1 + S p3
      h0 = S > 0 ? p0 + p2 : p0 - p2;
      h1 = S > 0 ? p1 + p3 : p1 - p3;
    }
    h.v[c] = h0;
    h.v[3 + c] = h1;
  }
}

// acc += (upper = w, lower = S B_mu^dag w)
template <int MU, int S, typename T>
__device__ __forceinline__ void accumulate(Spinor<T>& acc, const Half<T>& w) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const cpx<T> w0 = w.v[c], w1 = w.v[3 + c];
    acc.v[c] = acc.v[c] + w0;
    acc.v[3 + c] = acc.v[3 + c] + w1;
    if (MU == 0) {         // lower2 = S i w1, lower3 = S i w0
      acc.v[6 + c] = acc.v[6 + c] + (S > 0 ? times_i(w1) : times_mi(w1));
      acc.v[9 + c] = acc.v[9 + c] + (S > 0 ? times_i(w0) : times_mi(w0));
    } else if (MU == 1) {  // lower2 = S w1, lower3 = -S w0
      acc.v[6 + c] = S > 0 ? acc.v[6 + c] + w1 : acc.v[6 + c] - w1;
      acc.v[9 + c] = S > 0 ? acc.v[9 + c] - w0 : acc.v[9 + c] + w0;
    } else if (MU == 2) {  // lower2 = S i w0, lower3 = -S i w1
      acc.v[6 + c] = acc.v[6 + c] + (S > 0 ? times_i(w0) : times_mi(w0));
      acc.v[9 + c] = acc.v[9 + c] + (S > 0 ? times_mi(w1) : times_i(w1));
    } else {               // lower2 = S w0, lower3 = S w1
      acc.v[6 + c] = S > 0 ? acc.v[6 + c] + w0 : acc.v[6 + c] - w0;
      acc.v[9 + c] = S > 0 ? acc.v[9 + c] + w1 : acc.v[9 + c] - w1;
    }
  }
}

// acc + f a and acc + f (i a), one fused multiply-add per real component
template <typename T> __device__ __forceinline__ cpx<T> fmacc(cpx<T> acc, T f, cpx<T> a) {
  return mk(fma(f, a.r, acc.r), fma(f, a.i, acc.i));
}
template <typename T> __device__ __forceinline__ cpx<T> fmacc_i(cpx<T> acc, T f, cpx<T> a) {
  return mk(fma(-f, a.i, acc.r), fma(f, a.r, acc.i));
}

// acc += f (upper = w, lower = S B_mu^dag w): the factor f (boundary phase and,
// for FP16 storage, the neighbour's site norm) rides on the accumulation FMAs.
template <int MU, int S, typename T>
__device__ __forceinline__ void accumulate_scaled(Spinor<T>& acc, const Half<T>& w, T f) {
  const T fs = S > 0 ? f : -f;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const cpx<T> w0 = w.v[c], w1 = w.v[3 + c];
    acc.v[c] = fmacc(acc.v[c], f, w0);
    acc.v[3 + c] = fmacc(acc.v[3 + c], f, w1);
    if (MU == 0) {         // lower2 = S i w1, lower3 = S i w0
      acc.v[6 + c] = fmacc_i(acc.v[6 + c], fs, w1);
      acc.v[9 + c] = fmacc_i(acc.v[9 + c], fs, w0);
    } else if (MU == 1) {  // lower2 = S w1, lower3 = -S w0
      acc.v[6 + c] = fmacc(acc.v[6 + c], fs, w1);
      acc.v[9 + c] = fmacc(acc.v[9 + c], -fs, w0);
    } else if (MU == 2) {  // lower2 = S i w0, lower3 = -S i w1
      acc.v[6 + c] = fmacc_i(acc.v[6 + c], fs, w0);
      acc.v[9 + c] = fmacc_i(acc.v[9 + c], -fs, w1);
    } else {               // lower2 = S w0, lower3 = S w1
      acc.v[6 + c] = fmacc(acc.v[6 + c], fs, w0);
      acc.v[9 + c] = fmacc(acc.v[9 + c], fs, w1);
    }
  }
}

// w_a = U h_a
template <typename T>
__device__ __forceinline__ void link_mul(const Link<T>& u, const Half<T>& h, Half<T>& w) {
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int r = 0; r < 3; r++) {
      cpx<T> s = cmul(u.v[3 * r], h.v[3 * a]);
      s = cmadd(s, u.v[3 * r + 1], h.v[3 * a + 1]);
      s = cmadd(s, u.v[3 * r + 2], h.v[3 * a + 2]);
      w.v[3 * a + r] = s;
    }
}

// w_a = U^dag h_a
template <typename T>
__device__ __forceinline__ void link_mul_dag(const Link<T>& u, const Half<T>& h, Half<T>& w) {
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int r = 0; r < 3; r++) {
      cpx<T> s = cmadd_conj(mk(T(0), T(0)), u.v[r], h.v[3 * a]);
      s = cmadd_conj(s, u.v[3 + r], h.v[3 * a + 1]);
      s = cmadd_conj(s, u.v[6 + r], h.v[3 * a + 2]);
      w.v[3 * a + r] = s;
    }
}

template <typename T> __device__ __forceinline__ T bc_phase(const Geom& g, int mu);
template <> __device__ __forceinline__ double bc_phase<double>(const Geom& g, int mu) { return g.bcd[mu]; }
template <> __device__ __forceinline__ float bc_phase<float>(const Geom& g, int mu) { return g.bcf[mu]; }
template <> __device__ __forceinline__ dfl bc_phase<dfl>(const Geom& g, int mu) { return dfl(g.bcf[mu], 0.f); }

// FP32 a + c and a - c for a the low (H = 0) or high (H = 1) FP16 half of the
// word w (add / sub with an f16 and an f32 operand, sm_100 and later): the
// conversion of a is exact, so each equals the FP32 operation on the converted
// value, rounded once.
template <int H> __device__ __forceinline__ float add_h(unsigned int w, float c) {
  float d;
  if (H == 0) asm("{.reg .b16 l, u; mov.b32 {l, u}, %1; add.rn.f32.f16 %0, l, %2;}" : "=f"(d) : "r"(w), "f"(c));
  else asm("{.reg .b16 l, u; mov.b32 {l, u}, %1; add.rn.f32.f16 %0, u, %2;}" : "=f"(d) : "r"(w), "f"(c));
  return d;
}
template <int H> __device__ __forceinline__ float sub_h(unsigned int w, float c) {
  float d;
  if (H == 0) asm("{.reg .b16 l, u; mov.b32 {l, u}, %1; sub.rn.f32.f16 %0, l, %2;}" : "=f"(d) : "r"(w), "f"(c));
  else asm("{.reg .b16 l, u; mov.b32 {l, u}, %1; sub.rn.f32.f16 %0, u, %2;}" : "=f"(d) : "r"(w), "f"(c));
  return d;
}
// the real (H = 0) or imaginary (H = 1) part of the complex FP16 pair in w
template <int H> __device__ __forceinline__ float part_h(unsigned int w) {
  const __half2 v = *reinterpret_cast<const __half2*>(&w);
  return H == 0 ? __low2float(v) : __high2float(v);
}

// One projected complex component from FP16 data: a + C q with C = +1 (0),
// -1 (1), +i (2), -i (3); a and q are complex FP16 pairs (re low, im high).
template <int C>
__device__ __forceinline__ cpx<float> proj_h(unsigned int a, unsigned int q) {
  if (C == 0) return mk(add_h<0>(a, part_h<0>(q)), add_h<1>(a, part_h<1>(q)));
  if (C == 1) return mk(sub_h<0>(a, part_h<0>(q)), sub_h<1>(a, part_h<1>(q)));
  if (C == 2) return mk(sub_h<0>(a, part_h<1>(q)), add_h<1>(a, part_h<0>(q)));  // a + i q
  return mk(add_h<0>(a, part_h<1>(q)), sub_h<1>(a, part_h<0>(q)));               // a - i q
}

// FP16 storage: (1 + S gamma_mu) applied to the stored halves (each projected
// component one conversion and one mixed-precision add), the same values as
// converting all 24 components and projecting in FP32. w: the 12 complex FP16
// pairs, complex k = spin * 3 + colour in word k.
template <int MU, int S>
__device__ __forceinline__ void project_f16_words(const unsigned int (&w)[12], Half<float>& h) {
  // h0 = p0 + c0 p_k0, h1 = p1 + c1 p_k1 (the chiral-basis projection of project<MU, S>)
  constexpr int K0 = MU < 2 ? 3 : 2, K1 = MU < 2 ? 2 : 3;
  constexpr int C0 = MU == 0 ? (S > 0 ? 3 : 2) : MU == 1 ? (S > 0 ? 1 : 0) : MU == 2 ? (S > 0 ? 3 : 2) : (S > 0 ? 0 : 1);
  constexpr int C1 = MU == 0 ? (S > 0 ? 3 : 2) : MU == 1 ? (S > 0 ? 0 : 1) : MU == 2 ? (S > 0 ? 2 : 3) : (S > 0 ? 0 : 1);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    h.v[c] = proj_h<C0>(w[c], w[3 * K0 + c]);
    h.v[3 + c] = proj_h<C1>(w[3 + c], w[3 * K1 + c]);
  }
}

// The FP16 neighbour at idx loaded and projected; returns its site norm.
template <int MU, int S>
__device__ __forceinline__ float load_project_f16(const void* in, int64_t stride, int64_t idx, Half<float>& h) {
  const uint4* b = reinterpret_cast<const uint4*>(in);
  const float nrm = __ldg(SpinorIO<LQCD_F16>::norm_ptr(in, stride) + idx);
  unsigned int w[12];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const uint4 v = __ldg(b + c * stride + idx);
    w[4 * c] = v.x;
    w[4 * c + 1] = v.y;
    w[4 * c + 2] = v.z;
    w[4 * c + 3] = v.w;
  }
  project_f16_words<MU, S>(w, h);
  return nrm;
}

// Load the neighbour spinor and spin-project it with (1 + S gamma_mu). The
// linear factor the half spinor still needs -- the boundary phase of a
// wrapping hop and, for FP16 storage, the neighbour's site norm -- is returned
// instead of applied; accumulate_scaled folds it into its FMAs.
template <int P, int MU, int S>
__device__ __forceinline__ typename PrecTraits<P>::real load_project(const void* in, const Geom& g, int64_t idx,
                                                                     bool wrap, Half<typename PrecTraits<P>::real>& h) {
  using T = typename PrecTraits<P>::real;
  Spinor<T> s;
  T f;
  if constexpr (P == LQCD_F16) {
    f = load_project_f16<MU, S>(in, g.sstride, idx, h);
    return wrap ? bc_phase<T>(g, MU) * f : f;
  } else {
    SpinorIO<P>::load(in, g.sstride, idx, s);
    f = T(1);
  }
  project<MU, S>(s, h);
  return wrap ? bc_phase<T>(g, MU) * f : f;
}

template <typename T> __device__ __forceinline__ void conj_link(Link<T>& u) {
#pragma unroll
  for (int k = 0; k < 9; k++) u.v[k].i = -u.v[k].i;
}

// Both hops along mu. With GP (G-parity, n5 = 2 flavours i5 = f): a hop that
// wraps in a direction of g.gp reads the other flavour with sign +1 / -1
// (forward, f = 0 / 1) or -1 / +1 (backward) instead of the boundary phase,
// and the link is conjugated when its owner -- the site for the forward hop,
// the neighbour (flavour f') for the backward hop -- is flavour 1.
// sl: this 4D site's eight links staged in shared memory (forward link of mu
// at 2 mu, the backward hop's link at 2 mu + 1), or null to load them here.
template <int MU, int P, int R, bool DAG, bool GP = false>
__device__ __forceinline__ void hop_dir(Spinor<typename PrecTraits<P>::real>& acc, const Geom& g,
                                        const void* gauge, const Coord& x, int64_t cb, int64_t i5,
                                        int parity, const void* in,
                                        const Link<typename PrecTraits<P>::real>* sl = nullptr) {
  using T = typename PrecTraits<P>::real;
  constexpr int SF = DAG ? +1 : -1;  // forward hop carries (1 + SF gamma_mu)
  const int64_t n5 = g.n5;
  {
    bool wrap;
    const int64_t nb = neighbour_cb<MU>(g, x, +1, wrap);
    int64_t f_nb = i5;
    T sgn = T(1);
    if (GP && wrap && ((g.gp >> MU) & 1)) {
      f_nb = 1 - i5;
      sgn = i5 == 0 ? T(1) : T(-1);
      wrap = false;  // the twist replaces the boundary phase
    }
    Half<T> h;
    const T f = sgn * load_project<P, MU, SF>(in, g, nb * n5 + f_nb, wrap, h);
    Link<T> u;
    if (sl) u = sl[2 * MU];
    else LinkIO<P, R>::load(gauge, g.gstride, parity * 4 + MU, cb, u);
    if (GP && i5 == 1) conj_link(u);
    Half<T> w;
    link_mul(u, h, w);
    accumulate_scaled<MU, SF>(acc, w, f);
  }
  {
    bool wrap;
    const int64_t nb = neighbour_cb<MU>(g, x, -1, wrap);
    int64_t f_nb = i5;
    T sgn = T(1);
    if (GP && wrap && ((g.gp >> MU) & 1)) {
      f_nb = 1 - i5;
      sgn = i5 == 0 ? T(-1) : T(1);
      wrap = false;
    }
    Half<T> h;
    const T f = sgn * load_project<P, MU, -SF>(in, g, nb * n5 + f_nb, wrap, h);
    Link<T> u;
    if (sl) u = sl[2 * MU + 1];
    else LinkIO<P, R>::load(gauge, g.gstride, (1 - parity) * 4 + MU, nb, u);
    if (GP && f_nb == 1) conj_link(u);
    Half<T> w;
    link_mul_dag(u, h, w);
    accumulate_scaled<MU, -SF>(acc, w, f);
  }
}

// out_chi(s) += coefficient * x_chi(s'), chirality + = spins 0,1 (k < 6), - = spins 2,3.
template <typename T>
__device__ __forceinline__ void add_chiral(Spinor<T>& out, const Spinor<T>& xs, T coef, bool plus) {
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const int kk = plus ? k : 6 + k;
    out.v[kk] = out.v[kk] + coef * xs.v[kk];
  }
}

// Epilogue coefficients: PLAIN out = b H in; XPAY out = a x + b H in;
// M5 out = M5op(x) + b H in with M5op diagonal m5d and corner mf. (Loading the
// xpay operand before the hop, as the accumulator's start, made the bench step
// 1.8 % slower with FP16 storage: the operand is read at the end.)
struct EpiCoef {
  double a, b, m5d, mf;
};

// ---- the hop with its eight directions in a rolled loop (runtime mu): one copy
// of the per-direction code instead of eight. For the double-float arithmetic a
// fully unrolled hop is about 19,000 instructions long and stalls on
// instruction fetch; this form keeps the loop body in the instruction cache.

// z times c, c = +-1 or +-i: imag selects i, neg the sign
template <typename T> __device__ __forceinline__ cpx<T> times_unit(cpx<T> z, bool imag, bool neg) {
  const cpx<T> r = imag ? mk(-z.i, z.r) : z;
  return neg ? mk(-r.r, -r.i) : r;
}

// The link of direction mu into w: U (forward hop, block blk at checkerboard site
// cb) or U^dag (backward), as the matrix U' with w = U' h. 18-real links are read
// in the transposed order for U^dag; 12-real ones are rebuilt, then transposed.
template <int P, int R>
__device__ __forceinline__ void load_link_rolled(const void* gauge, int64_t gs, int blk, int64_t cb, bool fwd,
                                                 Link<typename PrecTraits<P>::real>& u) {
  using T = typename PrecTraits<P>::real;
  if constexpr (R == 18) {
    const double2* b = reinterpret_cast<const double2*>(gauge) + (int64_t)blk * 9 * gs + cb;
    static_assert(P == LQCD_F64 || P == LQCD_F64_DF, "rolled hop: FP64 fields");
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const double2 w = __ldg(b + (fwd ? 3 * r + c : 3 * c + r) * gs);
        const double im = fwd ? w.y : -w.y;
        if constexpr (P == LQCD_F64_DF) u.v[3 * r + c] = mk(df_split(w.x), df_split(im));
        else u.v[3 * r + c] = mk(w.x, im);
      }
  } else {
    Link<T> v;
    LinkIO<P, 12>::load(gauge, gs, blk, cb, v);
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const cpx<T> a = v.v[3 * r + c], t = conj(v.v[3 * c + r]);
        u.v[3 * r + c] = fwd ? a : t;
      }
  }
}

template <int P, int R, bool DAG>
__device__ __forceinline__ void hop_acc_rolled(const Geom& g, const void* gauge, const void* in, int parity,
                                               int64_t j, Spinor<typename PrecTraits<P>::real>& acc) {
  using T = typename PrecTraits<P>::real;
  const int64_t n5 = g.n5;
  int64_t cb, i5;
  if (n5 == 1) {
    cb = j;
    i5 = 0;
  } else {
    cb = fdiv((uint32_t)j, g.fn5);
    i5 = j - cb * n5;
  }
  const Coord x = cb_to_coord(g, cb, parity);
  zero(acc);
  constexpr int SF = DAG ? +1 : -1;  // forward hop carries (1 + SF gamma_mu)
#pragma unroll 1
  for (int dir = 0; dir < 8; dir++) {
    const int mu = dir >> 1;
    const bool fwd = (dir & 1) == 0;
    const bool sneg = (fwd ? SF : -SF) < 0;  // the projector's sign S is -1
    // neighbour along +-mu
    const int L = mu == 0 ? g.X : mu == 1 ? g.Y : mu == 2 ? g.Z : g.T;
    const int xm = mu == 0 ? x.c[0] : mu == 1 ? x.c[1] : mu == 2 ? x.c[2] : x.c[3];
    const uint32_t st = mu == 0 ? 1u : mu == 1 ? (uint32_t)g.st[1] : mu == 2 ? (uint32_t)g.st[2] : (uint32_t)g.st[3];
    const bool wrap = fwd ? xm == L - 1 : xm == 0;
    const uint32_t lex = fwd ? (wrap ? x.lex - (uint32_t)(L - 1) * st : x.lex + st)
                             : (wrap ? x.lex + (uint32_t)(L - 1) * st : x.lex - st);
    const int64_t nb = (int64_t)(lex >> 1);
    Spinor<T> p;
    SpinorIO<P>::load(in, g.sstride, nb * n5 + i5, p);
    // (1 + S gamma_mu) in the chiral basis: h0 = p0 + c0 p_k0, h1 = p1 + c1 p_k1 with
    // c = sc S (i if mu is even), and the lower spins S B^dag w: spin 2 += d2 w_m2,
    // spin 3 += d3 w_m3 with d = sd S (i if mu is even)
    const bool imag = (mu & 1) == 0;
    const bool k0_is3 = mu < 2;
    const bool c0neg = (mu != 3) != sneg, c1neg = (mu == 0) != sneg;
    const bool d2neg = sneg, d3neg = (mu == 1 || mu == 2) != sneg;
    Half<T> h;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const cpx<T> a0 = k0_is3 ? p.v[9 + c] : p.v[6 + c];
      const cpx<T> a1 = k0_is3 ? p.v[6 + c] : p.v[9 + c];
      h.v[c] = p.v[c] + times_unit(a0, imag, c0neg);
      h.v[3 + c] = p.v[3 + c] + times_unit(a1, imag, c1neg);
    }
    Link<T> u;
    load_link_rolled<P, R>(gauge, g.gstride, fwd ? parity * 4 + mu : (1 - parity) * 4 + mu, fwd ? cb : nb, fwd, u);
    Half<T> w;
    link_mul(u, h, w);
    // a wrapping hop's boundary phase (+-1) flips the signs of its whole contribution
    const float bcm = mu == 0 ? g.bcf[0] : mu == 1 ? g.bcf[1] : mu == 2 ? g.bcf[2] : g.bcf[3];
    const bool pneg = wrap && bcm < 0.f;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const cpx<T> w0 = w.v[c], w1 = w.v[3 + c];
      acc.v[c] = acc.v[c] + times_unit(w0, false, pneg);
      acc.v[3 + c] = acc.v[3 + c] + times_unit(w1, false, pneg);
      acc.v[6 + c] = acc.v[6 + c] + times_unit(k0_is3 ? w1 : w0, imag, d2neg != pneg);
      acc.v[9 + c] = acc.v[9 + c] + times_unit(k0_is3 ? w0 : w1, imag, d3neg != pneg);
    }
  }
}

// Both hops along mu with spin-paired packed arithmetic (hop_pair.cuh): the
// projection and the link as in hop_dir, the products and the accumulation on
// (spin 0, spin 1) pairs. FP32 / FP16 storage, no G-parity.
template <int MU, int P, int R, bool DAG>
__device__ __forceinline__ void hop_dir_sp(SPAcc& acc, const Geom& g, const void* gauge, const Coord& x, int64_t cb,
                                           int64_t i5, int parity, const void* in, const Link<float>* sl) {
  constexpr int SF = DAG ? +1 : -1;
  const int64_t n5 = g.n5;
#pragma unroll
  for (int dir = 0; dir < 2; dir++) {
    bool wrap;
    const int64_t nb = neighbour_cb<MU>(g, x, dir == 0 ? +1 : -1, wrap);
    Half<float> hh;
    const float f = dir == 0 ? load_project<P, MU, SF>(in, g, nb * n5 + i5, wrap, hh)
                             : load_project<P, MU, -SF>(in, g, nb * n5 + i5, wrap, hh);
    SPHalf h, w;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      h.r[c] = make_float2(hh.v[c].r, hh.v[3 + c].r);
      h.i[c] = make_float2(hh.v[c].i, hh.v[3 + c].i);
    }
    Link<float> u;
    if (dir == 0) {
      if (sl) u = sl[2 * MU];
      else LinkIO<P, R>::load(gauge, g.gstride, parity * 4 + MU, cb, u);
      link_mul_sp<false>(u, h, w);
      accumulate_sp<MU, SF>(acc, w, f);
    } else {
      if (sl) u = sl[2 * MU + 1];
      else LinkIO<P, R>::load(gauge, g.gstride, (1 - parity) * 4 + MU, nb, u);
      link_mul_sp<true>(u, h, w);
      accumulate_sp<MU, -SF>(acc, w, f);
    }
  }
}

}  // namespace lqcd

#include "hop_async.cuh"  // the staged hop uses the projections and products above

namespace lqcd {

// H in at output site j (= cb * n5 + i5) of checkerboard `parity`. AS: neighbour
// data streamed through the shared-memory ring `ring` (hop_async.cuh).
template <int P, int R, bool DAG, bool GP = false, bool SP = false, bool AS = false, int BLOCK = 128>
__device__ __forceinline__ void hop_acc(const Geom& g, const void* gauge, const void* in, int parity, int64_t j,
                                        Spinor<typename PrecTraits<P>::real>& acc,
                                        const Link<typename PrecTraits<P>::real>* sl = nullptr,
                                        unsigned char* ring = nullptr) {
  if constexpr (AS) {
    hop_acc_async<P, R, DAG, SP, BLOCK>(g, gauge, in, parity, j, acc, ring);
    return;
  }
  const int64_t n5 = g.n5;
  int64_t cb, i5;
  if (n5 == 1) {
    cb = j;
    i5 = 0;
  } else {
    cb = fdiv((uint32_t)j, g.fn5);
    i5 = j - cb * n5;
  }
  if constexpr (P == LQCD_F64_DF) {
    hop_acc_rolled<P, R, DAG>(g, gauge, in, parity, j, acc);
    return;
  }
  const Coord x = cb_to_coord(g, cb, parity);
  if constexpr (SP) {
    static_assert(P == LQCD_F32 || P == LQCD_F16, "spin-paired hop: FP32 / FP16 storage");
    SPAcc a;
#pragma unroll
    for (int c = 0; c < 3; c++) a.ur[c] = a.ui[c] = a.lr[c] = a.li[c] = make_float2(0.f, 0.f);
    hop_dir_sp<0, P, R, DAG>(a, g, gauge, x, cb, i5, parity, in, sl);
    hop_dir_sp<1, P, R, DAG>(a, g, gauge, x, cb, i5, parity, in, sl);
    hop_dir_sp<2, P, R, DAG>(a, g, gauge, x, cb, i5, parity, in, sl);
    hop_dir_sp<3, P, R, DAG>(a, g, gauge, x, cb, i5, parity, in, sl);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      acc.v[c] = mk(a.ur[c].x, a.ui[c].x);
      acc.v[3 + c] = mk(a.ur[c].y, a.ui[c].y);
      acc.v[6 + c] = mk(a.lr[c].x, a.li[c].x);
      acc.v[9 + c] = mk(a.lr[c].y, a.li[c].y);
    }
    return;
  }
  zero(acc);
  hop_dir<0, P, R, DAG, GP>(acc, g, gauge, x, cb, i5, parity, in, sl);
  hop_dir<1, P, R, DAG, GP>(acc, g, gauge, x, cb, i5, parity, in, sl);
  hop_dir<2, P, R, DAG, GP>(acc, g, gauge, x, cb, i5, parity, in, sl);
  hop_dir<3, P, R, DAG, GP>(acc, g, gauge, x, cb, i5, parity, in, sl);
}

// The epilogue at output site j of the hop result acc = H in (see EpiCoef).
template <int P, bool DAG, int EPI>
__device__ __forceinline__ void hop_epilogue(const Geom& g, const void* xb, int64_t j, const EpiCoef& c,
                                             const Spinor<typename PrecTraits<P>::real>& acc,
                                             Spinor<typename PrecTraits<P>::real>& res) {
  using T = typename PrecTraits<P>::real;
  using IO = SpinorIO<P>;
  const int64_t n5 = g.n5;
  const T b = (T)c.b;
  if (EPI == EPI_PLAIN || EPI == EPI_M5INV) {
#pragma unroll
    for (int k = 0; k < 12; k++) res.v[k] = b * acc.v[k];
  } else if (EPI == EPI_XPAY) {
    Spinor<T> xv;
    IO::load(xb, g.sstride, j, xv);
    const T a = (T)c.a;
#pragma unroll
    for (int k = 0; k < 12; k++) res.v[k] = mk(fma(a, xv.v[k].r, b * acc.v[k].r), fma(a, xv.v[k].i, b * acc.v[k].i));
  } else {
    // M5op(x)(s) = d x(s) - P_- x(s+1) - P_+ x(s-1), mf corners (dagger swaps directions)
    const int64_t i5 = n5 == 1 ? 0 : j - (int64_t)fdiv((uint32_t)j, g.fn5) * n5;
    Spinor<T> xv;
    IO::load(xb, g.sstride, j, xv);
    const T d = (T)c.m5d;
#pragma unroll
    for (int k = 0; k < 12; k++) res.v[k] = mk(fma(d, xv.v[k].r, b * acc.v[k].r), fma(d, xv.v[k].i, b * acc.v[k].i));
    const bool top = i5 + 1 == n5, bottom = i5 == 0;
    const int64_t jp = top ? j - (n5 - 1) : j + 1;
    const int64_t jm = bottom ? j + (n5 - 1) : j - 1;
    const T cp = top ? (T)c.mf : T(-1);
    const T cm = bottom ? (T)c.mf : T(-1);
    Spinor<T> xp, xm;
    IO::load(xb, g.sstride, jp, xp);
    IO::load(xb, g.sstride, jm, xm);
    if (!DAG) {
      add_chiral(res, xp, cp, false);
      add_chiral(res, xm, cm, true);
    } else {
      add_chiral(res, xm, cm, false);
      add_chiral(res, xp, cp, true);
    }
  }
}

// The result at output site j (= cb * n5 + i5) of checkerboard `parity`.
template <int P, int R, bool DAG, int EPI, bool GP = false, bool SP = false, bool AS = false, int BLOCK = 128>
__device__ __forceinline__ void hop_site(const Geom& g, const void* gauge, const void* in, const void* xb,
                                         int parity, int64_t j, const EpiCoef& c,
                                         Spinor<typename PrecTraits<P>::real>& res,
                                         const Link<typename PrecTraits<P>::real>* sl = nullptr,
                                         unsigned char* ring = nullptr) {
  Spinor<typename PrecTraits<P>::real> acc;
  hop_acc<P, R, DAG, GP, SP, AS, BLOCK>(g, gauge, in, parity, j, acc, sl, ring);
  hop_epilogue<P, DAG, EPI>(g, xb, j, c, acc, res);
}

template <typename T> __device__ __forceinline__ T norm2_site(const Spinor<T>& res) {
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 12; k++) s = fma(res.v[k].r, res.v[k].r, fma(res.v[k].i, res.v[k].i, s));
  return s;
}

// ---- link staging for the L_s-replicated / multi-RHS hop (n5 >= 4): the n5
// threads of a 4D site share its eight links (the paper's gauge field reused
// L_s times, Sec. 3), so a block loads (and for 12-real links rebuilds and, for
// FP16, converts) each link of its 4D sites once into shared memory and every
// thread reads them from there instead of repeating that work n5 times.
constexpr int STAGE_MIN_N5 = 4;
template <int BLOCK> constexpr int stage_sites() { return BLOCK / STAGE_MIN_N5 + 2; }

// Checkerboard index of the neighbour of x one hop back along a runtime mu.
__device__ __forceinline__ int64_t back_neighbour_cb(const Geom& g, const Coord& x, int mu) {
  const int L = mu == 0 ? g.X : mu == 1 ? g.Y : mu == 2 ? g.Z : g.T;
  const int xm = mu == 0 ? x.c[0] : mu == 1 ? x.c[1] : mu == 2 ? x.c[2] : x.c[3];
  const uint32_t st = mu == 0 ? 1u : mu == 1 ? (uint32_t)g.st[1] : mu == 2 ? (uint32_t)g.st[2] : (uint32_t)g.st[3];
  const uint32_t lex = xm == 0 ? x.lex + (uint32_t)(L - 1) * st : x.lex - st;
  return (int64_t)(lex >> 1);
}

// Stages the links of the block's 4D sites cb0 .. cb0 + nls - 1 (checkerboard
// `parity`) into sl[ls * 8 + d]; every thread of the block must call it.
template <int P, int R, int BLOCK>
__device__ __forceinline__ void stage_links(const Geom& g, const void* gauge, int parity, int64_t cb0, int nls,
                                            Link<typename PrecTraits<P>::real>* sl) {
  for (int t = threadIdx.x; t < nls * 8; t += BLOCK) {
    const int ls = t >> 3, d = t & 7, mu = d >> 1;
    const int64_t cb = cb0 + ls;
    if (cb >= g.Vh) continue;
    Link<typename PrecTraits<P>::real> u;
    if ((d & 1) == 0) {
      LinkIO<P, R>::load(gauge, g.gstride, parity * 4 + mu, cb, u);
    } else {
      const Coord x = cb_to_coord(g, cb, parity);
      LinkIO<P, R>::load(gauge, g.gstride, (1 - parity) * 4 + mu, back_neighbour_cb(g, x, mu), u);
    }
    sl[t] = u;
  }
  __syncthreads();
}

// One launch computes BLOCK * SPT output sites per block. SPT = 1: one site
// per thread, any precision. SPT = 2 (FP32 and FP16 storage, not G-parity):
// thread t of block blk computes sites j0 = blk BLOCK 2 + t and j1 = j0 +
// BLOCK together in packed FP32x2 arithmetic (hop_pair.cuh), so that every
// load instruction of a warp stays one coalesced access and the two sites
// share each FP32 instruction of the hop.
template <int P, int R, bool DAG, int EPI, int RED, int BLOCK, bool GP, int SPT, bool LS = false, bool SP = false,
          bool AS = false>
__device__ __forceinline__ void hop_body(const HopArgs& A) {
  using T = typename PrecTraits<P>::real;
  static_assert(SPT == 1 || (SPT == 2 && P != LQCD_F64 && !GP), "two sites per thread: FP32 / FP16, no G-parity");
  if (gate_closed(A.gate)) return;
  int parity = A.out_parity;
  int blk = blockIdx.x;
  if (A.full) {
    parity = blk >= A.blocks_per_parity ? 1 : 0;
    blk -= parity * A.blocks_per_parity;
  }
  const char* in = static_cast<const char*>(A.in) + (A.full ? (1 - parity) * A.half_bytes : 0);
  char* out = static_cast<char*>(A.out) + (A.full ? parity * A.half_bytes : 0);
  const char* xb = A.x ? static_cast<const char*>(A.x) + (A.full ? parity * A.half_bytes : 0) : nullptr;
  const EpiCoef c{A.a, A.b, A.m5d, A.mf};
  const int64_t first = (int64_t)blk * (BLOCK * SPT);
  if constexpr (SPT == 1) {
    const int64_t j = first + threadIdx.x;
    // LS: links staged in shared memory once per 4D site when n5 >= STAGE_MIN_N5
    const Link<T>* sl = nullptr;
    if constexpr (LS) {
      __shared__ Link<T> staged[stage_sites<BLOCK>() * 8];
      const int64_t n5 = A.g.n5;
      if (n5 >= STAGE_MIN_N5) {
        const int64_t cb0 = first / n5;
        const int64_t last = (first + BLOCK - 1 < A.g.nsites ? first + BLOCK - 1 : A.g.nsites - 1) / n5;
        stage_links<P, R, BLOCK>(A.g, A.gauge, parity, cb0, (int)(last - cb0 + 1), staged);
        if (j < A.g.nsites) sl = staged + (j / n5 - cb0) * 8;
      }
    }
    // AS: the ring of asynchronously copied neighbour data
    unsigned char* ring = nullptr;
    if constexpr (AS) {
      __shared__ __align__(16) unsigned char stage_ring[stage_nslot<P>() * stage_slot_bytes<P, R>() * BLOCK];
      ring = stage_ring;
    }
    if constexpr (EPI == EPI_M5INV) {
      // every lane takes part in the fifth-dimension scan; lanes past the end
      // (whole 4D sites, since L_s divides the block) carry zeros and store nothing
      static_assert(RED == RED_NONE, "M5op^-1 epilogue without reduction");
      const bool live = j < A.g.nsites;
      Spinor<T> res;
      if (live) hop_site<P, R, DAG, EPI, GP, SP, AS, BLOCK>(A.g, A.gauge, in, xb, parity, j, c, res, sl, ring);
      else zero(res);
      const int Ls = A.g.n5;
      m5inv_lanes(res, (int)(threadIdx.x & (unsigned)(Ls - 1)), Ls, A.m5_dagger != 0, (T)A.m5_a, (T)A.mf,
                  (T)A.m5_den_inv);
      if (live) SpinorIO<P>::store(out, A.g.sstride, j, res);
      return;
    }
    T red = T(0);
    if (j < A.g.nsites) {
      Spinor<T> res;
      hop_site<P, R, DAG, EPI, GP, SP, AS, BLOCK>(A.g, A.gauge, in, xb, parity, j, c, res, sl, ring);
      if constexpr (RED == RED_CG_UPDATE) {
        const int64_t ps = A.full ? parity * A.half_bytes : 0, vs = A.full ? parity * A.upd_half_bytes : 0;
        const int64_t rs = A.full ? parity * A.upd_rs_half_bytes : 0;
        red = update_site_ap<vec_prec(P), P, rs_prec(P)>(A.g, j, A.red.sys[sys_of(j, A.red.nsys)].alpha,
                                                         static_cast<const char*>(A.upd_p) + ps, res,
                                                         static_cast<char*>(A.upd_xs) + vs,
                                                         static_cast<char*>(A.upd_rs) + rs);
      } else {
        SpinorIO<P>::store(out, A.g.sstride, j, res);
        if constexpr (RED == RED_NORM) red = norm2_site(res);
      }
    }
    if constexpr (RED != RED_NONE) block_reduce_finalize<BLOCK>(red, first, A.red);
  } else {
    int64_t j[SPT];
    bool live[SPT];
#pragma unroll
    for (int s = 0; s < SPT; s++) {
      j[s] = first + s * BLOCK + threadIdx.x;
      live[s] = j[s] < A.g.nsites;
    }
    Spinor<T> acc[SPT];
    if (live[0]) {
      // a second site past the end repeats the first one's loads and is not stored
      PSpinor pa;
      hop_acc_pair<P, R, DAG>(A.g, A.gauge, in, parity, j[0], live[1] ? j[1] : j[0], pa);
#pragma unroll
      for (int k = 0; k < 12; k++) {
        acc[0].v[k] = pick(pa.v[k], 0);
        acc[1].v[k] = pick(pa.v[k], 1);
      }
    }
    if constexpr (EPI == EPI_M5INV) {
      static_assert(RED == RED_NONE, "M5op^-1 epilogue without reduction");
      const int Ls = A.g.n5;
#pragma unroll
      for (int s = 0; s < SPT; s++) {
        Spinor<T> res;
        if (live[s]) hop_epilogue<P, DAG, EPI>(A.g, xb, j[s], c, acc[s], res);
        else zero(res);
        m5inv_lanes(res, (int)(threadIdx.x & (unsigned)(Ls - 1)), Ls, A.m5_dagger != 0, (T)A.m5_a, (T)A.mf,
                    (T)A.m5_den_inv);
        if (live[s]) SpinorIO<P>::store(out, A.g.sstride, j[s], res);
      }
    } else {
      T red[SPT];
#pragma unroll
      for (int s = 0; s < SPT; s++) {
        red[s] = T(0);
        if (!live[s]) continue;
        Spinor<T> res;
        hop_epilogue<P, DAG, EPI>(A.g, xb, j[s], c, acc[s], res);
        if constexpr (RED == RED_CG_UPDATE) {
          const int64_t ps = A.full ? parity * A.half_bytes : 0, vs = A.full ? parity * A.upd_half_bytes : 0;
          const int64_t rs = A.full ? parity * A.upd_rs_half_bytes : 0;
          red[s] = update_site_ap<vec_prec(P), P, rs_prec(P)>(A.g, j[s], A.red.sys[sys_of(j[s], A.red.nsys)].alpha,
                                                              static_cast<const char*>(A.upd_p) + ps, res,
                                                              static_cast<char*>(A.upd_xs) + vs,
                                                              static_cast<char*>(A.upd_rs) + rs);
        } else {
          SpinorIO<P>::store(out, A.g.sstride, j[s], res);
          if constexpr (RED == RED_NORM) red[s] = norm2_site(res);
        }
      }
      if constexpr (RED != RED_NONE) block_reduce_finalize_n<BLOCK, SPT>(red, first, A.red);
    }
  }
}

// MINB: minimum resident blocks per SM the register allocation must allow
// (__launch_bounds__; 0 leaves the choice to the compiler), one of the knobs
// of the launch shapes the tuner times.
//
// SPT = -1: one site per thread with the links staged in shared memory (LS);
// SPT = -2: one site per thread in spin-paired packed arithmetic (SP);
// SPT = -3 / -4: as 1 / -2 with the neighbour data copied asynchronously
// through a shared-memory ring (AS, hop_async.cuh).
template <int P, int R, bool DAG, int EPI, int RED, int BLOCK, bool GP = false, int SPT = 1, int MINB = 0>
__global__ void __launch_bounds__(BLOCK, MINB) hop_kernel(const HopArgs A) {
  if constexpr (SPT == -1) hop_body<P, R, DAG, EPI, RED, BLOCK, GP, 1, true>(A);
  else if constexpr (SPT == -2) hop_body<P, R, DAG, EPI, RED, BLOCK, GP, 1, false, true>(A);
  else if constexpr (SPT == -3) hop_body<P, R, DAG, EPI, RED, BLOCK, GP, 1, false, false, true>(A);
  else if constexpr (SPT == -4) hop_body<P, R, DAG, EPI, RED, BLOCK, GP, 1, false, true, true>(A);
  else hop_body<P, R, DAG, EPI, RED, BLOCK, GP, SPT>(A);
}

}  // namespace lqcd
