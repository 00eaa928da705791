// Two output sites per thread in packed FP32x2 arithmetic (the Wilson hop's
// inner loop for FP32 and FP16 storage).
//
// Every real number of the hop is held for two different output sites A and B
// of the same checkerboard as one float2 (A in .x, B in .y), so each FP32 add,
// multiply or fused multiply-add of the one-site hop becomes one packed
// instruction for both sites (add.rn.f32x2 / mul.rn.f32x2 / fma.rn.f32x2,
// sm_100 and later). The two sites use different links and neighbours, so no
// operand is ever broadcast: the pairs are formed for free where the FP16 data
// are converted to FP32 (each conversion writes one half of a pair), and by one
// move per component for FP32 storage. Every packed operation is the one-site
// hop's scalar operation in the same order, so both give bit-identical
// results. This is the paper's "many independent
// small matrix-vector products in lockstep" (Sec. 2.3) applied inside one
// thread, on top of the site-per-lane layout across the warp.
#pragma once

#include "lqcd_common.cuh"

namespace lqcd {

// A complex number at the two sites: r = (Re at A, Re at B), i likewise.
struct pc {
  float2 r, i;
};
struct PSpinor { pc v[12]; };  // index spin * 3 + colour
struct PHalf { pc v[6]; };     // index a * 3 + colour
struct PLink { pc v[9]; };     // index row * 3 + column

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ pc pmk(float2 r, float2 i) {
  pc c;
  c.r = r;
  c.i = i;
  return c;
}
__device__ __forceinline__ pc padd(pc a, pc b) { return pmk(add2(a.r, b.r), add2(a.i, b.i)); }
__device__ __forceinline__ pc psub(pc a, pc b) { return pmk(sub2(a.r, b.r), sub2(a.i, b.i)); }
// a + i b and a - i b
__device__ __forceinline__ pc padd_i(pc a, pc b) { return pmk(sub2(a.r, b.i), add2(a.i, b.r)); }
__device__ __forceinline__ pc psub_i(pc a, pc b) { return pmk(add2(a.r, b.i), sub2(a.i, b.r)); }

// The pair's values at site A (k = 0) or B (k = 1).
__device__ __forceinline__ cpx<float> pick(const pc& c, int k) {
  return k == 0 ? mk(c.r.x, c.i.x) : mk(c.r.y, c.i.y);
}

__device__ __forceinline__ float2 h2lo_hi(unsigned int wa, unsigned int wb, bool hi) {
  const __half2 a = *reinterpret_cast<const __half2*>(&wa);
  const __half2 b = *reinterpret_cast<const __half2*>(&wb);
  return hi ? make_float2(__high2float(a), __high2float(b)) : make_float2(__low2float(a), __low2float(b));
}

// ---- spinor loads of the two sites, as pairs; FP16 leaves the site norms out
template <int P> struct PairSpinorIO;

template <> struct PairSpinorIO<LQCD_F32> {
  static __device__ __forceinline__ void load(const void* base, int64_t stride, int64_t ja, int64_t jb, PSpinor& s,
                                              float2& nrm) {
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int c = 0; c < 6; c++) {
      const float4 wa = __ldg(b + c * stride + ja);
      const float4 wb = __ldg(b + c * stride + jb);
      s.v[2 * c] = pmk(make_float2(wa.x, wb.x), make_float2(wa.y, wb.y));
      s.v[2 * c + 1] = pmk(make_float2(wa.z, wb.z), make_float2(wa.w, wb.w));
    }
    nrm = make_float2(1.f, 1.f);
  }
};

template <> struct PairSpinorIO<LQCD_F16> {
  static __device__ __forceinline__ void load(const void* base, int64_t stride, int64_t ja, int64_t jb, PSpinor& s,
                                              float2& nrm) {
    const uint4* b = reinterpret_cast<const uint4*>(base);
    const float* np = reinterpret_cast<const float*>(reinterpret_cast<const char*>(base) + 48 * stride);
    nrm = make_float2(__ldg(np + ja), __ldg(np + jb));
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const uint4 wa = __ldg(b + c * stride + ja);
      const uint4 wb = __ldg(b + c * stride + jb);
      const unsigned int a4[4] = {wa.x, wa.y, wa.z, wa.w};
      const unsigned int b4[4] = {wb.x, wb.y, wb.z, wb.w};
#pragma unroll
      for (int q = 0; q < 4; q++) s.v[4 * c + q] = pmk(h2lo_hi(a4[q], b4[q], false), h2lo_hi(a4[q], b4[q], true));
    }
  }
};

// ---- links of the two sites (blocks blk_a / blk_b at checkerboard sites cb_a / cb_b)
// conj(a b - c d) with the one-site hop's rounding (conj_cross)
__device__ __forceinline__ pc conj_cross_pair(pc a, pc b, pc c, pc d) {
  float2 re = mul2(a.r, b.r);
  re = fma2(neg2(a.i), b.i, re);
  re = fma2(neg2(c.r), d.r, re);
  re = fma2(c.i, d.i, re);
  float2 im = neg2(mul2(a.r, b.i));
  im = fma2(neg2(a.i), b.r, im);
  im = fma2(c.r, d.i, im);
  im = fma2(c.i, d.r, im);
  return pmk(re, im);
}

// row 2 = conj(row 0 x row 1), with the one-site hop's rounding (rebuild_row2),
// so that both launch shapes give bit-identical results
__device__ __forceinline__ void rebuild_row2_pair(PLink& u) {
  u.v[6] = conj_cross_pair(u.v[1], u.v[5], u.v[2], u.v[4]);
  u.v[7] = conj_cross_pair(u.v[2], u.v[3], u.v[0], u.v[5]);
  u.v[8] = conj_cross_pair(u.v[0], u.v[4], u.v[1], u.v[3]);
}

template <int P, int R> struct PairLinkIO;

template <> struct PairLinkIO<LQCD_F32, 12> {
  static __device__ __forceinline__ void load(const void* g, int64_t gs, int blk_a, int64_t cb_a, int blk_b,
                                              int64_t cb_b, PLink& u) {
    const float4* ba = reinterpret_cast<const float4*>(g) + (int64_t)blk_a * 3 * gs + cb_a;
    const float4* bb = reinterpret_cast<const float4*>(g) + (int64_t)blk_b * 3 * gs + cb_b;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const float4 wa = __ldg(ba + c * gs), wb = __ldg(bb + c * gs);
      u.v[2 * c] = pmk(make_float2(wa.x, wb.x), make_float2(wa.y, wb.y));
      u.v[2 * c + 1] = pmk(make_float2(wa.z, wb.z), make_float2(wa.w, wb.w));
    }
    rebuild_row2_pair(u);
  }
};
template <> struct PairLinkIO<LQCD_F32, 18> {
  static __device__ __forceinline__ void load(const void* g, int64_t gs, int blk_a, int64_t cb_a, int blk_b,
                                              int64_t cb_b, PLink& u) {
    const float2* ba = reinterpret_cast<const float2*>(g) + (int64_t)blk_a * 9 * gs + cb_a;
    const float2* bb = reinterpret_cast<const float2*>(g) + (int64_t)blk_b * 9 * gs + cb_b;
#pragma unroll
    for (int c = 0; c < 9; c++) {
      const float2 wa = __ldg(ba + c * gs), wb = __ldg(bb + c * gs);
      u.v[c] = pmk(make_float2(wa.x, wb.x), make_float2(wa.y, wb.y));
    }
  }
};
template <> struct PairLinkIO<LQCD_F16, 12> {
  static __device__ __forceinline__ void load(const void* g, int64_t gs, int blk_a, int64_t cb_a, int blk_b,
                                              int64_t cb_b, PLink& u) {
    const uint2* ba = reinterpret_cast<const uint2*>(g) + (int64_t)blk_a * 3 * gs + cb_a;
    const uint2* bb = reinterpret_cast<const uint2*>(g) + (int64_t)blk_b * 3 * gs + cb_b;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const uint2 wa = __ldg(ba + c * gs), wb = __ldg(bb + c * gs);
      u.v[2 * c] = pmk(h2lo_hi(wa.x, wb.x, false), h2lo_hi(wa.x, wb.x, true));
      u.v[2 * c + 1] = pmk(h2lo_hi(wa.y, wb.y, false), h2lo_hi(wa.y, wb.y, true));
    }
    rebuild_row2_pair(u);
  }
};
template <> struct PairLinkIO<LQCD_F16, 18> {
  static __device__ __forceinline__ void load(const void* g, int64_t gs, int blk_a, int64_t cb_a, int blk_b,
                                              int64_t cb_b, PLink& u) {
    const unsigned int* ba = reinterpret_cast<const unsigned int*>(g) + (int64_t)blk_a * 9 * gs + cb_a;
    const unsigned int* bb = reinterpret_cast<const unsigned int*>(g) + (int64_t)blk_b * 9 * gs + cb_b;
#pragma unroll
    for (int c = 0; c < 9; c++) {
      const unsigned int wa = __ldg(ba + c * gs), wb = __ldg(bb + c * gs);
      u.v[c] = pmk(h2lo_hi(wa, wb, false), h2lo_hi(wa, wb, true));
    }
  }
};

// ---- spin projection (1 + S gamma_mu) to the upper half h, in the chiral basis
// of the one-site hop: h0 = p0 + S B p_lower(0), h1 = p1 + S B p_lower(1).
template <int MU, int S>
__device__ __forceinline__ void project_pair(const PSpinor& s, PHalf& h) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const pc p0 = s.v[c], p1 = s.v[3 + c], p2 = s.v[6 + c], p3 = s.v[9 + c];
    pc h0, h1;
    if (MU == 0) {         // h0 = p0 - S i p3, h1 = p1 - S i p2
      h0 = S > 0 ? psub_i(p0, p3) : padd_i(p0, p3);
      h1 = S > 0 ? psub_i(p1, p2) : padd_i(p1, p2);
    } else if (MU == 1) {  // h0 = p0 - S p3, h1 = p1 + S p2
      h0 = S > 0 ? psub(p0, p3) : padd(p0, p3);
      h1 = S > 0 ? padd(p1, p2) : psub(p1, p2);
    } else if (MU == 2) {  // h0 = p0 - S i p2, h1 = p1 + S i p3
      h0 = S > 0 ? psub_i(p0, p2) : padd_i(p0, p2);
      h1 = S > 0 ? padd_i(p1, p3) : psub_i(p1, p3);
    } else {               // h0 = p0 + S p2, h1 = p1 + S p3
      h0 = S > 0 ? padd(p0, p2) : psub(p0, p2);
      h1 = S > 0 ? padd(p1, p3) : psub(p1, p3);
    }
    h.v[c] = h0;
    h.v[3 + c] = h1;
  }
}

// w_a = U h_a (DAG false) or U^dag h_a (DAG true)
template <bool DAG>
__device__ __forceinline__ void link_mul_pair(const PLink& u, const PHalf& h, PHalf& w) {
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int r = 0; r < 3; r++) {
      float2 re, im;
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const pc m = DAG ? u.v[3 * c + r] : u.v[3 * r + c];
        const pc x = h.v[3 * a + c];
        if (c == 0) {
          re = mul2(m.r, x.r);
          im = mul2(m.r, x.i);
        } else {
          re = fma2(m.r, x.r, re);
          im = fma2(m.r, x.i, im);
        }
        if (DAG) {  // conj(m) x
          re = fma2(m.i, x.i, re);
          im = fma2(neg2(m.i), x.r, im);
        } else {    // m x
          re = fma2(neg2(m.i), x.i, re);
          im = fma2(m.i, x.r, im);
        }
      }
      w.v[3 * a + r] = pmk(re, im);
    }
}

// acc + f a and acc + f (i a)
__device__ __forceinline__ pc pfma(pc acc, float2 f, pc a) { return pmk(fma2(f, a.r, acc.r), fma2(f, a.i, acc.i)); }
__device__ __forceinline__ pc pfma_i(pc acc, float2 f, pc a) {
  return pmk(fma2(neg2(f), a.i, acc.r), fma2(f, a.r, acc.i));
}

// acc += f (upper = w, lower = S B_mu^dag w), f = boundary phase x site norm of each site
template <int MU, int S>
__device__ __forceinline__ void accumulate_pair(PSpinor& acc, const PHalf& w, float2 f) {
  const float2 fs = S > 0 ? f : neg2(f);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const pc w0 = w.v[c], w1 = w.v[3 + c];
    acc.v[c] = pfma(acc.v[c], f, w0);
    acc.v[3 + c] = pfma(acc.v[3 + c], f, w1);
    if (MU == 0) {         // lower2 = S i w1, lower3 = S i w0
      acc.v[6 + c] = pfma_i(acc.v[6 + c], fs, w1);
      acc.v[9 + c] = pfma_i(acc.v[9 + c], fs, w0);
    } else if (MU == 1) {  // lower2 = S w1, lower3 = -S w0
      acc.v[6 + c] = pfma(acc.v[6 + c], fs, w1);
      acc.v[9 + c] = pfma(acc.v[9 + c], neg2(fs), w0);
    } else if (MU == 2) {  // lower2 = S i w0, lower3 = -S i w1
      acc.v[6 + c] = pfma_i(acc.v[6 + c], fs, w0);
      acc.v[9 + c] = pfma_i(acc.v[9 + c], neg2(fs), w1);
    } else {               // lower2 = S w0, lower3 = S w1
      acc.v[6 + c] = pfma(acc.v[6 + c], fs, w0);
      acc.v[9 + c] = pfma(acc.v[9 + c], fs, w1);
    }
  }
}

// Both hops along mu for the two sites (checkerboard sites cb_a / cb_b, fifth
// coordinates i5_a / i5_b, coordinates xa / xb).
template <int MU, int P, int R, bool DAG>
__device__ __forceinline__ void hop_dir_pair(PSpinor& acc, const Geom& g, const void* gauge, const Coord& xa,
                                             const Coord& xb, int64_t cb_a, int64_t cb_b, int64_t i5_a,
                                             int64_t i5_b, int parity, const void* in) {
  constexpr int SF = DAG ? +1 : -1;  // forward hop carries (1 + SF gamma_mu)
  const int64_t n5 = g.n5;
  const float phase = g.bcf[MU];
#pragma unroll
  for (int dir = 0; dir < 2; dir++) {
    const int sign = dir == 0 ? +1 : -1;
    bool wa, wb;
    const int64_t na = neighbour_cb<MU>(g, xa, sign, wa);
    const int64_t nb = neighbour_cb<MU>(g, xb, sign, wb);
    PSpinor s;
    float2 f;
    PairSpinorIO<P>::load(in, g.sstride, na * n5 + i5_a, nb * n5 + i5_b, s, f);
    f = make_float2(wa ? phase * f.x : f.x, wb ? phase * f.y : f.y);
    PHalf h, w;
    PLink u;
    if (dir == 0) {
      project_pair<MU, SF>(s, h);
      PairLinkIO<P, R>::load(gauge, g.gstride, parity * 4 + MU, cb_a, parity * 4 + MU, cb_b, u);
      link_mul_pair<false>(u, h, w);
      accumulate_pair<MU, SF>(acc, w, f);
    } else {
      project_pair<MU, -SF>(s, h);
      PairLinkIO<P, R>::load(gauge, g.gstride, (1 - parity) * 4 + MU, na, (1 - parity) * 4 + MU, nb, u);
      link_mul_pair<true>(u, h, w);
      accumulate_pair<MU, -SF>(acc, w, f);
    }
  }
}

// H in at the two output sites ja, jb (= cb * n5 + i5) of checkerboard `parity`.
template <int P, int R, bool DAG>
__device__ __forceinline__ void hop_acc_pair(const Geom& g, const void* gauge, const void* in, int parity,
                                             int64_t ja, int64_t jb, PSpinor& acc) {
  const int64_t n5 = g.n5;
  int64_t cb_a, cb_b, i5_a, i5_b;
  if (n5 == 1) {
    cb_a = ja;
    cb_b = jb;
    i5_a = i5_b = 0;
  } else {
    cb_a = fdiv((uint32_t)ja, g.fn5);
    cb_b = fdiv((uint32_t)jb, g.fn5);
    i5_a = ja - cb_a * n5;
    i5_b = jb - cb_b * n5;
  }
  const Coord xa = cb_to_coord(g, cb_a, parity), xb = cb_to_coord(g, cb_b, parity);
#pragma unroll
  for (int k = 0; k < 12; k++) acc.v[k] = pmk(make_float2(0.f, 0.f), make_float2(0.f, 0.f));
  hop_dir_pair<0, P, R, DAG>(acc, g, gauge, xa, xb, cb_a, cb_b, i5_a, i5_b, parity, in);
  hop_dir_pair<1, P, R, DAG>(acc, g, gauge, xa, xb, cb_a, cb_b, i5_a, i5_b, parity, in);
  hop_dir_pair<2, P, R, DAG>(acc, g, gauge, xa, xb, cb_a, cb_b, i5_a, i5_b, parity, in);
  hop_dir_pair<3, P, R, DAG>(acc, g, gauge, xa, xb, cb_a, cb_b, i5_a, i5_b, parity, in);
}

// ---------------------------------------------------------------------------
// One site per thread with the two spin components of each half spinor paired:
// H[c] = (h_0c, h_1c) as float2 of real parts and of imaginary parts, so
// w_a = U h_a for a = 0, 1 is one packed product per term (the link element
// broadcast to both lanes), and the accumulator holds spins (0, 1) and (2, 3)
// as pairs. Same operations in the same order per lane as the one-site hop.
struct SPHalf { float2 r[3], i[3]; };   // (h_0c, h_1c), c = 0..2
struct SPAcc { float2 ur[3], ui[3], lr[3], li[3]; };  // spins (0,1) and (2,3), colour c

__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 swp(float2 a) { return make_float2(a.y, a.x); }

// w = U h (DAG: U^dag h) on spin pairs
template <bool DAG>
__device__ __forceinline__ void link_mul_sp(const Link<float>& u, const SPHalf& h, SPHalf& w) {
#pragma unroll
  for (int r = 0; r < 3; r++) {
    float2 re, im;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const cpx<float> m = DAG ? u.v[3 * c + r] : u.v[3 * r + c];
      const float2 mr = bc2(m.r), mi = bc2(m.i);
      if (c == 0) {
        re = mul2(mr, h.r[c]);
        im = mul2(mr, h.i[c]);
      } else {
        re = fma2(mr, h.r[c], re);
        im = fma2(mr, h.i[c], im);
      }
      if (DAG) {
        re = fma2(mi, h.i[c], re);
        im = fma2(neg2(mi), h.r[c], im);
      } else {
        re = fma2(neg2(mi), h.i[c], re);
        im = fma2(mi, h.r[c], im);
      }
    }
    w.r[r] = re;
    w.i[r] = im;
  }
}

// acc += f (upper = w, lower = S B_mu^dag w) on spin pairs (see accumulate_scaled)
template <int MU, int S>
__device__ __forceinline__ void accumulate_sp(SPAcc& acc, const SPHalf& w, float f) {
  const float fs = S > 0 ? f : -f;
  const float2 F = bc2(f);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    acc.ur[c] = fma2(F, w.r[c], acc.ur[c]);
    acc.ui[c] = fma2(F, w.i[c], acc.ui[c]);
    if (MU == 0) {         // spin 2 += fs i w1, spin 3 += fs i w0
      acc.lr[c] = fma2(bc2(-fs), swp(w.i[c]), acc.lr[c]);
      acc.li[c] = fma2(bc2(fs), swp(w.r[c]), acc.li[c]);
    } else if (MU == 1) {  // spin 2 += fs w1, spin 3 += -fs w0
      acc.lr[c] = fma2(make_float2(fs, -fs), swp(w.r[c]), acc.lr[c]);
      acc.li[c] = fma2(make_float2(fs, -fs), swp(w.i[c]), acc.li[c]);
    } else if (MU == 2) {  // spin 2 += fs i w0, spin 3 += -fs i w1
      acc.lr[c] = fma2(make_float2(-fs, fs), w.i[c], acc.lr[c]);
      acc.li[c] = fma2(make_float2(fs, -fs), w.r[c], acc.li[c]);
    } else {               // spin 2 += fs w0, spin 3 += fs w1
      acc.lr[c] = fma2(bc2(fs), w.r[c], acc.lr[c]);
      acc.li[c] = fma2(bc2(fs), w.i[c], acc.li[c]);
    }
  }
}

}  // namespace lqcd
