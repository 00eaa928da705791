// Hop with asynchronously staged neighbour loads (launch shapes with sites per
// thread -3 / -4; FP32 and FP16 storage, no G-parity).
//
// The plain hop loads each direction's neighbour spinor and link into
// registers; with the register budget of 7 resident blocks per SM the compiler
// keeps about one direction's loads in flight per thread, so the warps spend
// most stall cycles waiting on the L2 / DRAM (one 16-byte load per thread in
// flight on average at 24^3 x 48). Here every thread copies the raw words of
// direction d + NSLOT - 1 into its own slot of a shared-memory ring with
// cp.async (Ampere-style asynchronous copies: no register holds the data in
// flight) while it computes direction d from the slot that has landed, so
// NSLOT - 1 directions' bytes stay in flight per thread at no register cost.
// Each thread reads back only what it copied itself, so the ring needs no
// block barrier: cp.async.wait_group makes a thread's own copies visible to it.
//
// Slot layout (per block, structure of arrays so that a warp's shared-memory
// accesses are conflict-free): the 16-byte spinor chunks [S16][BLOCK], the link
// chunks [LN][BLOCK] of LE bytes, then, for FP16, the site norms [BLOCK].
#pragma once

#include "lqcd_common.cuh"

namespace lqcd {

template <int P, int R> struct StageFmt;
template <> struct StageFmt<LQCD_F16, 12> { static constexpr int S16 = 3, LN = 3, LE = 8, NORM = 1; };
template <> struct StageFmt<LQCD_F16, 18> { static constexpr int S16 = 3, LN = 9, LE = 4, NORM = 1; };
template <> struct StageFmt<LQCD_F32, 12> { static constexpr int S16 = 6, LN = 3, LE = 16, NORM = 0; };
template <> struct StageFmt<LQCD_F32, 18> { static constexpr int S16 = 6, LN = 9, LE = 8, NORM = 0; };

// bytes of one direction's slot per thread
template <int P, int R> constexpr int stage_slot_bytes() {
  return 16 * StageFmt<P, R>::S16 + StageFmt<P, R>::LN * StageFmt<P, R>::LE + 4 * StageFmt<P, R>::NORM;
}
// ring depth: FP16 keeps two directions in flight (3 slots, 228 B per thread),
// FP32 one (2 slots, 288 B per thread), so that 7 / 5 blocks of 128 fit an SM
template <int P> constexpr int stage_nslot() { return P == LQCD_F16 ? 3 : 2; }

template <int BYTES> __device__ __forceinline__ void cp_async(uint32_t dst, const void* src) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copies direction D's neighbour spinor (index nb n5 + i5 of the other
// checkerboard) and link (forward: the site's own, block parity * 4 + mu;
// backward: the neighbour's, block (1 - parity) * 4 + mu) into `slot`.
template <int P, int R, int BLOCK, int D>
__device__ __forceinline__ void stage_issue(unsigned char* slot, const Geom& g, const void* gauge, const void* in,
                                            const Coord& x, int64_t cb, int64_t i5, int parity) {
  using F = StageFmt<P, R>;
  constexpr int MU = D >> 1;
  constexpr bool FWD = (D & 1) == 0;
  bool wrap;
  const int64_t nb = neighbour_cb<MU>(g, x, FWD ? +1 : -1, wrap);
  const int64_t idx = nb * g.n5 + i5;
  const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(slot);
  const char* sp = static_cast<const char*>(in);
#pragma unroll
  for (int c = 0; c < F::S16; c++)
    cp_async<16>(s0 + (c * BLOCK + threadIdx.x) * 16, sp + (c * g.sstride + idx) * 16);
  const int lblk = FWD ? parity * 4 + MU : (1 - parity) * 4 + MU;
  const int64_t lcb = FWD ? cb : nb;
  const char* gp = static_cast<const char*>(gauge);
  const uint32_t l0 = s0 + 16 * F::S16 * BLOCK;
#pragma unroll
  for (int c = 0; c < F::LN; c++)
    cp_async<F::LE>(l0 + (c * BLOCK + threadIdx.x) * F::LE, gp + (((int64_t)lblk * F::LN + c) * g.gstride + lcb) * F::LE);
  if constexpr (F::NORM) {
    const uint32_t n0 = l0 + F::LN * F::LE * BLOCK;
    cp_async<4>(n0 + threadIdx.x * 4, sp + 48 * g.sstride + idx * 4);
  }
}

// The link of a slot, converted to FP32 (12-real links: row 2 rebuilt).
template <int P, int R, int BLOCK>
__device__ __forceinline__ void stage_link(const unsigned char* slot, Link<float>& u) {
  using F = StageFmt<P, R>;
  const unsigned char* l0 = slot + 16 * F::S16 * BLOCK;
  if constexpr (P == LQCD_F16 && R == 12) {
    const uint2* b = reinterpret_cast<const uint2*>(l0) + threadIdx.x;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      uint2 w = b[c * BLOCK];
      const float2 f0 = __half22float2(*reinterpret_cast<__half2*>(&w.x));
      const float2 f1 = __half22float2(*reinterpret_cast<__half2*>(&w.y));
      u.v[2 * c] = mk(f0.x, f0.y);
      u.v[2 * c + 1] = mk(f1.x, f1.y);
    }
    rebuild_row2(u);
  } else if constexpr (P == LQCD_F16) {
    const unsigned int* b = reinterpret_cast<const unsigned int*>(l0) + threadIdx.x;
#pragma unroll
    for (int c = 0; c < 9; c++) {
      unsigned int w = b[c * BLOCK];
      const float2 f = __half22float2(*reinterpret_cast<__half2*>(&w));
      u.v[c] = mk(f.x, f.y);
    }
  } else if constexpr (R == 12) {
    const float4* b = reinterpret_cast<const float4*>(l0) + threadIdx.x;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const float4 w = b[c * BLOCK];
      u.v[2 * c] = mk(w.x, w.y);
      u.v[2 * c + 1] = mk(w.z, w.w);
    }
    rebuild_row2(u);
  } else {
    const float2* b = reinterpret_cast<const float2*>(l0) + threadIdx.x;
#pragma unroll
    for (int c = 0; c < 9; c++) {
      const float2 w = b[c * BLOCK];
      u.v[c] = mk(w.x, w.y);
    }
  }
}

// The spin projection (1 + S gamma_mu) of a slot's spinor; returns the factor
// the half spinor still needs (the FP16 site norm, else 1).
template <int P, int R, int BLOCK, int MU, int S>
__device__ __forceinline__ float stage_project(const unsigned char* slot, Half<float>& h) {
  using F = StageFmt<P, R>;
  const uint4* b = reinterpret_cast<const uint4*>(slot) + threadIdx.x;
  if constexpr (P == LQCD_F16) {
    unsigned int w[12];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const uint4 v = b[c * BLOCK];
      w[4 * c] = v.x;
      w[4 * c + 1] = v.y;
      w[4 * c + 2] = v.z;
      w[4 * c + 3] = v.w;
    }
    project_f16_words<MU, S>(w, h);
    return reinterpret_cast<const float*>(slot + (16 * F::S16 + F::LN * F::LE) * BLOCK)[threadIdx.x];
  } else {
    Spinor<float> s;
#pragma unroll
    for (int c = 0; c < 6; c++) {
      const float4 w = reinterpret_cast<const float4*>(b)[c * BLOCK];
      s.v[2 * c] = mk(w.x, w.y);
      s.v[2 * c + 1] = mk(w.z, w.w);
    }
    project<MU, S>(s, h);
    return 1.f;
  }
}

// Direction D's contribution from its slot: acc (SP = false: Spinor<float>;
// SP = true: the spin-paired SPAcc of hop_pair.cuh).
template <int P, int R, int BLOCK, int D, bool DAG, bool SP, typename Acc>
__device__ __forceinline__ void stage_compute(const unsigned char* slot, Acc& acc, const Geom& g, const Coord& x) {
  constexpr int MU = D >> 1;
  constexpr bool FWD = (D & 1) == 0;
  constexpr int SF = DAG ? +1 : -1;  // forward hop carries (1 + SF gamma_mu)
  constexpr int S = FWD ? SF : -SF;
  bool wrap;
  neighbour_cb<MU>(g, x, FWD ? +1 : -1, wrap);
  Half<float> h;
  float f = stage_project<P, R, BLOCK, MU, S>(slot, h);
  if (wrap) f *= g.bcf[MU];
  Link<float> u;
  stage_link<P, R, BLOCK>(slot, u);
  if constexpr (SP) {
    SPHalf hp, w;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      hp.r[c] = make_float2(h.v[c].r, h.v[3 + c].r);
      hp.i[c] = make_float2(h.v[c].i, h.v[3 + c].i);
    }
    link_mul_sp<!FWD>(u, hp, w);
    accumulate_sp<MU, S>(acc, w, f);
  } else {
    Half<float> w;
    if constexpr (FWD) link_mul(u, h, w);
    else link_mul_dag(u, h, w);
    accumulate_scaled<MU, S>(acc, w, f);
  }
}

// Step D of the ring: issue direction D + NSLOT - 1, wait for direction D, compute it.
template <int P, int R, int BLOCK, int NSLOT, bool DAG, bool SP, int D, typename Acc>
__device__ __forceinline__ void stage_step(unsigned char* ring, Acc& acc, const Geom& g, const void* gauge,
                                           const void* in, const Coord& x, int64_t cb, int64_t i5, int parity) {
  constexpr int SLOT = stage_slot_bytes<P, R>() * BLOCK;
  if constexpr (D + NSLOT - 1 < 8)
    stage_issue<P, R, BLOCK, D + NSLOT - 1>(ring + ((D + NSLOT - 1) % NSLOT) * SLOT, g, gauge, in, x, cb, i5, parity);
  cp_async_commit();  // an empty group past the last direction keeps the count uniform
  cp_async_wait<NSLOT - 1>();
  stage_compute<P, R, BLOCK, D, DAG, SP>(ring + (D % NSLOT) * SLOT, acc, g, x);
  if constexpr (D + 1 < 8) stage_step<P, R, BLOCK, NSLOT, DAG, SP, D + 1>(ring, acc, g, gauge, in, x, cb, i5, parity);
}

// H in at output site j (= cb n5 + i5) of checkerboard `parity`, the neighbour
// data streamed through `ring` (NSLOT slots of stage_slot_bytes * BLOCK bytes).
template <int P, int R, bool DAG, bool SP, int BLOCK>
__device__ __forceinline__ void hop_acc_async(const Geom& g, const void* gauge, const void* in, int parity, int64_t j,
                                              Spinor<float>& out, unsigned char* ring) {
  static_assert(P == LQCD_F32 || P == LQCD_F16, "staged hop: FP32 / FP16 storage");
  constexpr int NSLOT = stage_nslot<P>();
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
  constexpr int SLOT = stage_slot_bytes<P, R>() * BLOCK;
#pragma unroll
  for (int d = 0; d < NSLOT - 1; d++) {
    if (d == 0) stage_issue<P, R, BLOCK, 0>(ring, g, gauge, in, x, cb, i5, parity);
    if (d == 1) stage_issue<P, R, BLOCK, 1>(ring + SLOT, g, gauge, in, x, cb, i5, parity);
    cp_async_commit();
  }
  if constexpr (SP) {
    SPAcc a;
#pragma unroll
    for (int c = 0; c < 3; c++) a.ur[c] = a.ui[c] = a.lr[c] = a.li[c] = make_float2(0.f, 0.f);
    stage_step<P, R, BLOCK, NSLOT, DAG, true, 0>(ring, a, g, gauge, in, x, cb, i5, parity);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      out.v[c] = mk(a.ur[c].x, a.ui[c].x);
      out.v[3 + c] = mk(a.ur[c].y, a.ui[c].y);
      out.v[6 + c] = mk(a.lr[c].x, a.li[c].x);
      out.v[9 + c] = mk(a.lr[c].y, a.li[c].y);
    }
  } else {
    zero(out);
    stage_step<P, R, BLOCK, NSLOT, DAG, false, 0>(ring, out, g, gauge, in, x, cb, i5, parity);
  }
}

}  // namespace lqcd
