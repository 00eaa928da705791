// Conjugate gradient on M^dag M (or M_hat^dag M_hat), plain FP64 or mixed
// precision with FP64 reliable updates.
//
// The Grid paper lists CG among its algorithms (Sec. 4) and relies on global
// reductions for it (Sec. 1); the iteration is the textbook Hestenes-Stiefel
// form. Mixed precision follows the reliable-update scheme of Sleijpen and
// van der Vorst (1996) as used for lattice QCD by Clark et al. (2010): the
// inner iteration runs with a sloppy (FP32 or FP16-storage) operator, x is
// accumulated in FP64, and whenever the iterated |r| falls below delta times
// its maximum since the last update (or below the tolerance) the residual
// r = b - A x is recomputed with the FP64 operator.
//
// With FP16 storage the iterated residual r_s is stored in FP16 as well (its
// rounding is relative to the current residual; x_s stays FP32), and a third
// level sits between the two (delta_mid > 0): FP16
// needs a fresh residual every two to three decades, and on GB300 an FP64
// recomputation costs as much as ten FP32 iterations. So whenever |r_s| falls
// below delta_mid times its maximum since the last replacement, the iterated
// residual is replaced by r - A x_s, with r the residual of the last FP64
// update and A x_s applied in FP32 to an FP32 / 12-real copy of the FP64 links
// made once per solve in the workspace (accurate to about 1e-7 of |r|); the
// FP64 updates then only follow delta, which FP32 accuracy allows down to a
// few times 1e-6.
//
// Every scalar (alpha, beta, the convergence and update decisions) lives on
// the device and is produced by the last block of the reducing kernel, so an
// iteration is a fixed sequence of launches with no host round trip:
//   Mp = M p        (|Mp|^2 = p^dag A p reduced in the epilogue -> alpha)
//   Ap = M^dag Mp
//   x_s += alpha p, r_s -= alpha Ap   (|r_s|^2 -> beta, or pause)
//   p = r_s + beta p
// CGNR (lqcd_cgnr_solve) runs the same iteration for M x = b: each reliable
// update recomputes the system's residual s = b - M x and |s|^2 in FP64, which
// decides the exit (tol applies to |b - M x| / |b|), while r_0 = M^dag b and
// r = M^dag s, which only seed the iterated recurrence, are applied in the inner
// arithmetic. The FP64 work of an update halves and M^dag b is never formed in
// FP64. lqcd_eo_solve wraps it for the full system D x = b: preparation, CGNR
// on the even checkerboard, and (Wilson) the odd half from the H_oe x_e that
// the last update's M x left in the workspace.
//
// A chunk of such iterations is captured once as a CUDA graph and replayed;
// kernels return immediately once the control block is paused, so the host
// only looks at the control block between chunks.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "cg_engine.h"
#include "m5_scan.cuh"
#include "cg_site.cuh"

namespace lqcd {

struct VecArgs {
  Geom g;
  int full;
  int bpp;            // blocks per parity
  double* x64;        // FP64 solution
  const double* b64;  // FP64 source
  double* r64;        // FP64 residual
  const double* ax64; // FP64 A x
  const void* ax32;   // FP32 A x_s of the intermediate replacement (FP32 field)
  void* xs;           // sloppy-vector solution increment (VF)
  void* rs;           // sloppy-vector residual (rs_prec)
  void* p;            // search direction (SF)
  int64_t hb64, hbv, hbs, hbr;  // bytes of one checkerboard per format (FP64, VF, SF, r_s)
  SysState* sys;
  ReduceCtx red;
  const Control* gate;
};

__device__ __forceinline__ bool vec_site(const VecArgs& a, int& parity, int64_t& j, int64_t& first) {
  int blk = blockIdx.x;
  parity = 0;
  if (a.full) {
    parity = blk >= a.bpp ? 1 : 0;
    blk -= parity * a.bpp;
  }
  first = (int64_t)blk * BLAS_BLOCK;
  j = first + threadIdx.x;
  return j < a.g.nsites;
}

#define PAR_PTR(ptr, hb) ((ptr) ? (decltype(ptr))((char*)(ptr) + parity * (hb)) : (ptr))

// r = b, r_s = b, p = b, x_s = 0, x = 0; |b|^2 -> initial state
template <int VF, int SF>
__global__ void __launch_bounds__(BLAS_BLOCK) k_init(VecArgs a) {
  int parity;
  int64_t j, first;
  double red = 0.0;
  if (vec_site(a, parity, j, first))
    red = init_site<VF, SF, rs_prec(SF)>(a.g, j, PAR_PTR(a.b64, a.hb64), PAR_PTR(a.r64, a.hb64),
                                         PAR_PTR(a.x64, a.hb64), PAR_PTR(a.rs, a.hbr), PAR_PTR(a.xs, a.hbv),
                                         PAR_PTR(a.p, a.hbs));
  block_reduce_finalize<BLAS_BLOCK>(red, first, a.red);
}

// p = r_s + beta p
template <int VF, int SF>
__global__ void __launch_bounds__(BLAS_BLOCK) k_pupdate(VecArgs a) {
  if (gate_closed(a.gate)) return;
  int parity;
  int64_t j, first;
  if (!vec_site(a, parity, j, first)) return;
  pupdate_site<VF, SF, rs_prec(SF)>(a.g, j, a.sys[sys_of(j, a.red.nsys)].beta, PAR_PTR(a.rs, a.hbr),
                                    PAR_PTR(a.p, a.hbs));
}

// x += x_s (FP64); x_s = 0
template <int VF>
__global__ void __launch_bounds__(BLAS_BLOCK) k_accumulate(VecArgs a) {
  int parity;
  int64_t j, first;
  if (!vec_site(a, parity, j, first)) return;
  accumulate_site<VF>(a.g, j, PAR_PTR(a.x64, a.hb64), PAR_PTR(a.xs, a.hbv));
}

// r = b - A x (FP64), r_s = r; |r|^2 -> done flags, beta, resume
template <int VF, int RF>
__global__ void __launch_bounds__(BLAS_BLOCK) k_residual(VecArgs a) {
  int parity;
  int64_t j, first;
  double red = 0.0;
  if (vec_site(a, parity, j, first))
    red = residual_site<VF, RF>(a.g, j, PAR_PTR(a.b64, a.hb64), PAR_PTR(a.ax64, a.hb64), PAR_PTR(a.r64, a.hb64),
                                PAR_PTR(a.rs, a.hbr));
  block_reduce_finalize<BLAS_BLOCK>(red, first, a.red);
}
// dst = src between formats (the CGNR start: M^dag b in FP32 arithmetic)
template <int DP, int SP>
__global__ void __launch_bounds__(BLAS_BLOCK) k_copy_field(VecArgs a, void* dst, const void* src) {
  int parity;
  int64_t j, first;
  if (!vec_site(a, parity, j, first)) return;
  const int64_t hd = parity * (int64_t)cb_spinor_bytes(a.g, DP), hs = parity * (int64_t)cb_spinor_bytes(a.g, SP);
  Spinor<typename PrecTraits<SP>::real> v;
  SpinorIO<SP>::load(static_cast<const char*>(src) + hs, a.g.sstride, j, v);
  Spinor<typename PrecTraits<DP>::real> w;
  convert(v, w);
  SpinorIO<DP>::store(static_cast<char*>(dst) + hd, a.g.sstride, j, w);
}

// CGNR: out = b - mx in FP64 and |b - mx|^2 per system (a.red, FIN_STORE);
// with mx null only |b|^2 (out may alias mx)
__global__ void __launch_bounds__(BLAS_BLOCK) k_b_minus(VecArgs a, double* out, const double* mx) {
  int parity;
  int64_t j, first;
  double red = 0.0;
  if (vec_site(a, parity, j, first)) {
    const int64_t h = parity * a.hb64;
    Spinor<double> b, m;
    SpinorIO<LQCD_F64>::load(reinterpret_cast<const char*>(a.b64) + h, a.g.sstride, j, b);
    if (mx) {
      SpinorIO<LQCD_F64>::load(reinterpret_cast<const char*>(mx) + h, a.g.sstride, j, m);
#pragma unroll
      for (int k = 0; k < 12; k++) b.v[k] = b.v[k] - m.v[k];
      SpinorIO<LQCD_F64>::store(reinterpret_cast<char*>(out) + h, a.g.sstride, j, b);
    }
    red = site_norm2(b);
  }
  block_reduce_finalize<BLAS_BLOCK>(red, first, a.red);
}

// CGNR: r = M^dag (b - M x) from its FP32-arithmetic value (a.ax32) -> FP64 r,
// r_s; |r|^2 -> FIN_RELIABLE (exit decided by the FP64 |b - M x|^2)
template <int VF, int RF>
__global__ void __launch_bounds__(BLAS_BLOCK) k_residual32(VecArgs a) {
  int parity;
  int64_t j, first;
  typename PrecTraits<VF>::real red = 0;
  if (vec_site(a, parity, j, first))
    red = residual32_site<VF, RF>(a.g, j, PAR_PTR(a.ax32, a.hbv), PAR_PTR(a.r64, a.hb64), PAR_PTR(a.rs, a.hbr));
  block_reduce_finalize<BLAS_BLOCK>(red, first, a.red);
}

// FP32 / 12-real copy of the FP64 links (rows 0 and 1, rounded once): the operator
// of the CGNR start, of the updates' M^dag and of the intermediate replacements,
// whose FP32 arithmetic needs no more than FP32 links. One thread per (parity, mu, cb).
__global__ void __launch_bounds__(BLAS_BLOCK) k_links_to_f32r12(float4* dst, const double2* src, Geom g, int nchunk64) {
  const int64_t t = (int64_t)blockIdx.x * BLAS_BLOCK + threadIdx.x;
  if (t >= 8 * (int64_t)g.Vh) return;
  const int blk = (int)(t / g.Vh);
  const int64_t cb = t - (int64_t)blk * g.Vh;
  const double2* s = src + (int64_t)blk * nchunk64 * g.gstride + cb;
  float4* d = dst + (int64_t)blk * 3 * g.gstride + cb;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const double2 a = __ldg(s + (2 * c) * g.gstride), b = __ldg(s + (2 * c + 1) * g.gstride);
    d[c * g.gstride] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
  }
}

// Odd half of an even-odd Wilson solve from the last reliable update's hop:
// x_o = (b_o + hx / 2) / c with hx = H_oe x_e (FP64, one checkerboard)
__global__ void __launch_bounds__(BLAS_BLOCK) k_reconstruct_odd(Geom g, double* xo, const double* bo, const double* hx,
                                                                double c) {
  const int64_t j = (int64_t)blockIdx.x * BLAS_BLOCK + threadIdx.x;
  if (j >= g.nsites) return;
  Spinor<double> b, h;
  SpinorIO<LQCD_F64>::load(bo, g.sstride, j, b);
  SpinorIO<LQCD_F64>::load(hx, g.sstride, j, h);
  const double ic = 1.0 / c, ih = 0.5 / c;
#pragma unroll
  for (int k = 0; k < 12; k++) b.v[k] = mk(fma(ih, h.v[k].r, ic * b.v[k].r), fma(ih, h.v[k].i, ic * b.v[k].i));
  SpinorIO<LQCD_F64>::store(xo, g.sstride, j, b);
}

// r_s = r - A x_s (FP32 arithmetic); |r_s|^2 -> beta, resume (FIN_MID)
template <int VF, int RF>
__global__ void __launch_bounds__(BLAS_BLOCK) k_mid_residual(VecArgs a) {
  int parity;
  int64_t j, first;
  double red = 0.0;
  if (vec_site(a, parity, j, first))
    red = mid_residual_site<VF, RF>(a.g, j, PAR_PTR(a.r64, a.hb64), PAR_PTR(a.ax32, a.hbv), PAR_PTR(a.rs, a.hbr));
  block_reduce_finalize<BLAS_BLOCK>(red, first, a.red);
}
#undef PAR_PTR

// ------------------------------------------------------------------ host side

struct Workspace {
  Control* ctrl;
  SysState* sys;
  double* partials;
  unsigned int* counter;
  double* ss;  // CGNR: per-system |b|^2, then |b - M x|^2 of the last reliable update
  double* bb;  // even-odd solve: per-system |b|^2 of the full system's source
  void* g32;   // mixed solves: FP32 / 12-real copy of the FP64 links
  double* r64;
  double* ax64;
  double* mid64;
  void* t1_64;
  void* t2_64;
  void* rs;
  void* xs;
  void* p;
  void* mp;
  void* t1_s;
  void* t2_s;
  size_t total;
};


static int64_t max_blocks(const Geom& g, int subset) {
  const int64_t per = (g.nsites + 63) / 64;  // smallest block size used by reducing kernels is >= 64
  // an even-odd solve also reduces over both checkerboards of its full source (2 x ceil(nsites / 128) blocks)
  return subset == LQCD_FULL ? 2 * per : per + 2;
}

static Workspace carve(void* base, const Geom& g, const lqcd_operator& op, const lqcd_solver_params& p, int subset,
                       int nsys) {
  Workspace w;
  memset(&w, 0, sizeof(w));
  size_t o = 0;
  char* b = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> void* {
    void* r = b ? b + o : nullptr;
    o += round_up((int64_t)bytes, 256);
    return r;
  };
  const int VF = vec_prec(p.sloppy_prec), SF = p.sloppy_prec;
  w.ctrl = (Control*)take(sizeof(Control));
  w.sys = (SysState*)take(sizeof(SysState) * MAX_SYS);
  w.partials = (double*)take(sizeof(double) * nsys * max_blocks(g, subset));
  w.counter = (unsigned int*)take(64);
  w.ss = (double*)take(sizeof(double) * MAX_SYS);
  w.bb = (double*)take(sizeof(double) * MAX_SYS);
  w.r64 = (double*)take(field_bytes(g, LQCD_F64, subset));
  w.ax64 = (double*)take(field_bytes(g, LQCD_F64, subset));
  w.mid64 = (double*)take(field_bytes(g, LQCD_F64, subset));
  if (subset == LQCD_EVEN) {
    w.t1_64 = take(cb_spinor_bytes(g, LQCD_F64));
    if (op.kind == LQCD_DWF) w.t2_64 = take(cb_spinor_bytes(g, LQCD_F64));
  }
  if (p.sloppy_prec != LQCD_F64) w.g32 = take((size_t)8 * g.gstride * link_bytes(LQCD_F32, 12));
  w.rs = take(field_bytes(g, rs_prec(SF), subset));
  w.xs = take(field_bytes(g, VF, subset));
  w.p = take(field_bytes(g, SF, subset));
  w.mp = take(field_bytes(g, SF, subset));
  if (subset == LQCD_EVEN) {
    w.t1_s = take(cb_spinor_bytes(g, SF));
    if (op.kind == LQCD_DWF) w.t2_s = take(cb_spinor_bytes(g, SF));
  }
  w.total = o;
  return w;
}

// Whether a solve runs its FP64-field operator (reliable updates, even-odd source) in double-float
// arithmetic: Wilson without G-parity, or domain wall on 18-real links with L_s dividing 32 (the
// double-float hop fuses M5op^-1 into its epilogue; check_operator states the same rule).
static bool update_df(const lqcd_operator& op, const lqcd_solver_params& p, int n5) {
  if (p.sloppy_prec == LQCD_F64 || p.update_prec != LQCD_F64_DF || op.gparity) return false;
  return op.kind == LQCD_WILSON || (op.kind == LQCD_DWF && op.recon == 18 && m5_scan_ok(n5));
}

static int validate(const lqcd_lattice* lat, const lqcd_operator* op, const lqcd_solver_params* p, int subset,
                    Geom* g) {
  int st = make_geom(lat, g);
  if (st) return st;
  if ((st = check_operator(op, *g))) return st;
  if (!p) return fail(LQCD_ERR_ARG, "null solver params");
  if (op->prec != LQCD_F64) return fail(LQCD_ERR_ARG, "cg: x, b and gauge must be LQCD_F64 (op->prec)");
  if (p->sloppy_prec != LQCD_F64 && p->sloppy_prec != LQCD_F32 && p->sloppy_prec != LQCD_F16)
    return fail(LQCD_ERR_ARG, "cg: bad sloppy precision %d", p->sloppy_prec);
  if (p->sloppy_recon != 18 && p->sloppy_recon != 12) return fail(LQCD_ERR_ARG, "cg: bad sloppy recon");
  if (op->gparity && p->sloppy_prec == LQCD_F16) return fail(LQCD_ERR_UNSUPPORTED, "cg: G-parity with FP16 inner");
  if (!(p->tol > 0.0) || p->maxiter < 1) return fail(LQCD_ERR_ARG, "cg: tol must be > 0 and maxiter >= 1");
  if (p->delta < 0.0 || p->delta >= 1.0) return fail(LQCD_ERR_ARG, "cg: delta must be in [0, 1)");
  if (!(p->delta_mid >= 0.0 && p->delta_mid < 1.0)) return fail(LQCD_ERR_ARG, "cg: delta_mid must be in [0, 1)");
  if (p->update_prec != LQCD_F64 && p->update_prec != LQCD_F64_DF)
    return fail(LQCD_ERR_ARG, "cg: update_prec must be LQCD_F64 or LQCD_F64_DF");
  if (subset != LQCD_EVEN && subset != LQCD_FULL) return fail(LQCD_ERR_ARG, "cg: subset must be EVEN or FULL");
  return LQCD_OK;
}

// Launch helpers for the (VF, SF) instantiations.
enum VecKernel { VK_INIT, VK_PUPDATE, VK_ACCUM, VK_RESIDUAL, VK_MID_RESIDUAL, VK_RESIDUAL32 };

template <int VF, int SF>
static void launch_vec_t(VecKernel k, unsigned grid, const VecArgs& a, cudaStream_t s) {
  switch (k) {
    case VK_INIT: k_init<VF, SF><<<grid, BLAS_BLOCK, 0, s>>>(a); break;
    case VK_PUPDATE: k_pupdate<VF, SF><<<grid, BLAS_BLOCK, 0, s>>>(a); break;
    case VK_ACCUM: k_accumulate<VF><<<grid, BLAS_BLOCK, 0, s>>>(a); break;
    case VK_RESIDUAL: k_residual<VF, rs_prec(SF)><<<grid, BLAS_BLOCK, 0, s>>>(a); break;
    case VK_MID_RESIDUAL: k_mid_residual<VF, rs_prec(SF)><<<grid, BLAS_BLOCK, 0, s>>>(a); break;
    case VK_RESIDUAL32: k_residual32<VF, rs_prec(SF)><<<grid, BLAS_BLOCK, 0, s>>>(a); break;
  }
}

static int launch_vec(VecKernel k, int sloppy, const VecArgs& a, cudaStream_t s) {
  const unsigned grid = (unsigned)(a.full ? 2 * a.bpp : a.bpp);
  if (grid == 0) return LQCD_OK;
  if (sloppy == LQCD_F64) launch_vec_t<LQCD_F64, LQCD_F64>(k, grid, a, s);
  else if (sloppy == LQCD_F32) launch_vec_t<LQCD_F32, LQCD_F32>(k, grid, a, s);
  else launch_vec_t<LQCD_F32, LQCD_F16>(k, grid, a, s);
  return after_launch("cg vector kernel");
}

struct Solver : CgEngine {
  Geom g;
  lqcd_operator op64, ops, opm;  // FP64, sloppy, and FP32 on FP32 / 12-real links from the FP64 field
  lqcd_solver_params prm;
  int subset;
  bool mid_on = false;
  bool normal = false;  // CGNR: b is the right-hand side of M x = b, not of M^dag M x = b
  const double* b_full = nullptr;  // even-odd solve: the full system's FP64 source (scales the exit test)
  Workspace w;
  const void* gauge64;
  const void* gauge_s;
  VecArgs va;
  ReduceCtx rc_init, rc_alpha, rc_update, rc_reliable, rc_mid, rc_ss;

  int init(cudaStream_t s) override {
    cudaError_t e = cudaMemsetAsync(w.counter, 0, 64, s);
    if (e != cudaSuccess) return cuda_fail(e, "cg: memset");
    if (w.g32 && (normal || mid_on)) {  // FP32 links for the FP32-arithmetic operator, from this call's FP64 field
      const unsigned grid = (unsigned)((8 * (int64_t)g.Vh + BLAS_BLOCK - 1) / BLAS_BLOCK);
      k_links_to_f32r12<<<grid, BLAS_BLOCK, 0, s>>>((float4*)w.g32, (const double2*)gauge64, g, op64.recon == 18 ? 9 : 6);
      int st = after_launch("cg: FP32 links");
      if (st) return st;
    }
    VecArgs a = va;
    a.red = rc_init;
    if (b_full) {  // |b|^2 of the full system's source, over both checkerboards
      VecArgs af = va;
      af.full = 1;
      af.b64 = b_full;
      af.red = rc_ss;
      af.red.result = w.bb;
      k_b_minus<<<(unsigned)(2 * af.bpp), BLAS_BLOCK, 0, s>>>(af, nullptr, nullptr);
      int st = after_launch("eo_solve: |b|^2");
      if (st) return st;
    }
    if (normal) {
      // |b|^2 in FP64 (the exit test's scale); r_0 = M^dag b in the inner iteration's
      // arithmetic: the FP64 operator for a plain solve, else the FP32 operator on the
      // FP32 link copy (r only seeds the recurrence; the exit test is on b - M x)
      int st;
      const unsigned grid0 = (unsigned)(a.full ? 2 * a.bpp : a.bpp);
      VecArgs an = a;
      an.red = rc_ss;
      k_b_minus<<<grid0, BLAS_BLOCK, 0, s>>>(an, nullptr, nullptr);
      if ((st = after_launch("cgnr: |b|^2"))) return st;
      if (prm.sloppy_prec == LQCD_F64) {
        OpCtx c64{g, op64, gauge64};
        if ((st = op_apply(c64, w.ax64, a.b64, subset, 1, w.t1_64, w.t2_64, nullptr, nullptr, s))) return st;
        a.b64 = w.ax64;
      } else {
        const unsigned grid = (unsigned)(a.full ? 2 * a.bpp : a.bpp);
        k_copy_field<LQCD_F32, LQCD_F64><<<grid, BLAS_BLOCK, 0, s>>>(a, w.xs, a.b64);
        if ((st = after_launch("cgnr: b to FP32"))) return st;
        OpCtx cm{g, opm, w.g32};
        if ((st = op_apply(cm, w.ax64, w.xs, subset, 1, w.t1_64, w.t2_64, nullptr, nullptr, s))) return st;
        k_copy_field<LQCD_F64, LQCD_F32><<<grid, BLAS_BLOCK, 0, s>>>(a, w.mid64, w.ax64);
        if ((st = after_launch("cgnr: M^dag b to FP64"))) return st;
        a.b64 = w.mid64;
      }
    }
    return launch_vec(VK_INIT, prm.sloppy_prec, a, s);
  }

  // M_hat p with |M_hat p|^2 = p^dag A p -> alpha; then M_hat^dag (M_hat p) = A p,
  // whose last hop applies x_s += alpha p, r_s -= alpha A p and reduces |r_s|^2
  // (beta, or a reliable-update request) instead of storing A p.
  int head(cudaStream_t s, int cond, cudaGraphConditionalHandle h_rel, cudaGraphConditionalHandle h_mid) override {
    OpCtx cs{g, ops, gauge_s};
    int st = op_apply(cs, w.mp, w.p, subset, 0, w.t1_s, w.t2_s, &rc_alpha, w.ctrl, s);
    if (st) return st;
    ReduceCtx ru = rc_update;
    ru.cond = cond;
    ru.h_rel = h_rel;
    ru.h_mid = h_mid;
    const HopUpdate upd{w.p, w.xs, w.rs, va.hbv, va.hbr};
    return op_apply(cs, nullptr, w.mp, subset, 1, w.t1_s, w.t2_s, &ru, w.ctrl, s, &upd);
  }

  int tail(cudaStream_t s) override {
    VecArgs a = va;
    a.gate = w.ctrl;
    return launch_vec(VK_PUPDATE, prm.sloppy_prec, a, s);
  }

  int reliable(cudaStream_t s) override {
    VecArgs a = va;
    int st = launch_vec(VK_ACCUM, prm.sloppy_prec, a, s);
    if (st) return st;
    OpCtx c64{g, op64, gauge64};
    if ((st = op_apply(c64, w.mid64, a.x64, subset, 0, w.t1_64, w.t2_64, nullptr, nullptr, s))) return st;
    if (!normal) {  // r = b - M^dag M x in FP64
      if ((st = op_apply(c64, w.ax64, w.mid64, subset, 1, w.t1_64, w.t2_64, nullptr, nullptr, s))) return st;
      a.red = rc_reliable;
      return launch_vec(VK_RESIDUAL, prm.sloppy_prec, a, s);
    }
    // CGNR: the FP64 residual of the system, s = b - M x and |s|^2, decides the exit;
    // r = M^dag s then only restarts the recurrence, in the inner arithmetic. The first
    // hop's H x stays in t1_64 (the odd half of an even-odd solve reuses it): the
    // adjoint's temporaries are r64 (rewritten last) and t2_64.
    const unsigned grid = (unsigned)(a.full ? 2 * a.bpp : a.bpp);
    VecArgs an = a;
    an.red = rc_ss;
    k_b_minus<<<grid, BLAS_BLOCK, 0, s>>>(an, w.mid64, w.mid64);
    if ((st = after_launch("cgnr: b - M x"))) return st;
    a.red = rc_reliable;
    if (prm.sloppy_prec == LQCD_F64) {
      if ((st = op_apply(c64, w.ax64, w.mid64, subset, 1, w.r64, w.t2_64, nullptr, nullptr, s))) return st;
      a.b64 = nullptr;  // ax64 already holds the residual
      return launch_vec(VK_RESIDUAL, prm.sloppy_prec, a, s);
    }
    k_copy_field<LQCD_F32, LQCD_F64><<<grid, BLAS_BLOCK, 0, s>>>(a, w.ax64, w.mid64);
    if ((st = after_launch("cgnr: b - M x to FP32"))) return st;
    OpCtx cm{g, opm, w.g32};
    if ((st = op_apply(cm, w.mid64, w.ax64, subset, 1, w.r64, w.t2_64, nullptr, nullptr, s))) return st;
    a.ax32 = w.mid64;
    return launch_vec(VK_RESIDUAL32, prm.sloppy_prec, a, s);
  }

  bool has_mid() const override { return mid_on; }

  // Tuning pass, before init: the operator applications of an iteration (M_hat p with
  // its norm, M_hat^dag with the fused update) and of the FP32 level, run once with
  // every reduction sent to scratch (FIN_STORE into ss) and alpha = 0, so that each
  // hop instantiation the captured graph will replay gets its launch shape timed
  // (inside a capture nothing can be timed). The fields it touches are rewritten by
  // init afterwards.
  int tune(cudaStream_t s) {
    TuningPass pass;
    cudaError_t e = cudaMemsetAsync(w.counter, 0, 64, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.sys, 0, sizeof(SysState) * MAX_SYS, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.p, 0, field_bytes(g, prm.sloppy_prec, subset), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.xs, 0, field_bytes(g, vec_prec(prm.sloppy_prec), subset), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.rs, 0, field_bytes(g, rs_prec(prm.sloppy_prec), subset), s);
    if (e != cudaSuccess) return cuda_fail(e, "cg: tuning pass memset");
    ReduceCtx r = rc_ss;  // FIN_STORE into ss
    OpCtx cs{g, ops, gauge_s};
    int st = op_apply(cs, w.mp, w.p, subset, 0, w.t1_s, w.t2_s, &r, nullptr, s);
    const HopUpdate upd{w.p, w.xs, w.rs, va.hbv, va.hbr};
    if (!st) st = op_apply(cs, nullptr, w.mp, subset, 1, w.t1_s, w.t2_s, &r, nullptr, s, &upd);
    if (!st && w.g32 && (normal || mid_on)) {
      e = cudaMemsetAsync(w.g32, 0, (size_t)8 * g.gstride * link_bytes(LQCD_F32, 12), s);
      if (e != cudaSuccess) return cuda_fail(e, "cg: tuning pass memset");
      OpCtx cm{g, opm, w.g32};
      st = op_apply(cm, w.mid64, w.xs, subset, 0, w.t1_64, w.t2_64, nullptr, nullptr, s);
      if (!st) st = op_apply(cm, w.ax64, w.mid64, subset, 1, w.t1_64, w.t2_64, nullptr, nullptr, s);
    }
    return st;
  }

  // r_s = r - M^dag M x_s with the FP32 operator on the FP32 link copy. The
  // FP64 update's buffers (mid64, ax64, t1_64, t2_64) are idle here and hold
  // the FP32 intermediates.
  int mid(cudaStream_t s) override {
    OpCtx cm{g, opm, w.g32};
    int st = op_apply(cm, w.mid64, w.xs, subset, 0, w.t1_64, w.t2_64, nullptr, nullptr, s);
    if (st) return st;
    if ((st = op_apply(cm, w.ax64, w.mid64, subset, 1, w.t1_64, w.t2_64, nullptr, nullptr, s))) return st;
    VecArgs a = va;
    a.ax32 = w.ax64;
    a.red = rc_mid;
    return launch_vec(VK_MID_RESIDUAL, prm.sloppy_prec, a, s);
  }
};

}  // namespace lqcd

using namespace lqcd;

extern "C" {

void lqcd_release_caches(void) {
  release_graph_cache();
  release_noalloc_addresses();
}

size_t lqcd_cg_workspace_bytes(const lqcd_lattice* lat, const lqcd_operator* op, const lqcd_solver_params* p,
                               int subset) {
  Geom g;
  if (validate(lat, op, p, subset, &g)) return 0;
  const int nsys = op->kind == LQCD_WILSON && !op->gparity ? g.n5 : 1;  // G-parity flavours form one system
  return carve(nullptr, g, *op, *p, subset, nsys).total;
}

}  // extern "C"

namespace lqcd {

static int cg_solve_impl(void* x, const void* b, const void* gauge, const void* gauge_sloppy, const lqcd_lattice* lat,
                         const lqcd_operator* op, const lqcd_solver_params* prm, int subset, lqcd_solve_info* info,
                         void* workspace, size_t workspace_bytes, void* stream, bool normal,
                         const void* b_full = nullptr) {
  const auto t0 = std::chrono::steady_clock::now();
  lqcd_solve_info local;
  lqcd_solve_info* inf = info ? info : &local;
  memset(inf, 0, sizeof(*inf));
  auto finish = [&](int status) {
    inf->status = status;
    inf->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return status;
  };
  Solver S;
  int st = validate(lat, op, prm, subset, &S.g);
  if (st) return finish(st);
  if (!x || !b || !gauge || !workspace || ((uintptr_t)workspace & 255) || ((uintptr_t)x & 15) ||
      ((uintptr_t)b & 15))
    return finish(fail(LQCD_ERR_ARG, "cg: null or misaligned pointer (workspace needs 256-byte alignment)"));
  if (prm->sloppy_prec == LQCD_F64) gauge_sloppy = gauge;  // the FP64 field serves both
  if (!gauge_sloppy) return finish(fail(LQCD_ERR_ARG, "cg: gauge_sloppy required"));
  S.prm = *prm;
  if (S.prm.check_interval <= 0) S.prm.check_interval = 16;
  S.subset = subset;
  S.normal = normal;
  S.b_full = static_cast<const double*>(b_full);
  S.nsys = op->kind == LQCD_WILSON && !op->gparity ? S.g.n5 : 1;  // G-parity flavours form one system
  S.w = carve(workspace, S.g, *op, *prm, subset, S.nsys);
  if (workspace_bytes < S.w.total)
    return finish(fail(LQCD_ERR_WORKSPACE, "cg: workspace %zu < %zu bytes", workspace_bytes, S.w.total));
  S.ctrl = S.w.ctrl;
  S.sys = S.w.sys;
  S.op64 = *op;
  // mixed Wilson solves may run the reliable updates' FP64-field operator in double-float arithmetic
  if (update_df(*op, *prm, lat->n5)) S.op64.prec = LQCD_F64_DF;
  S.ops = *op;
  S.ops.prec = prm->sloppy_prec;
  // the FP64 inner operator runs on the FP64 field itself, in that field's format
  S.ops.recon = prm->sloppy_prec == LQCD_F64 ? op->recon : prm->sloppy_recon;
  S.opm = *op;
  S.opm.prec = LQCD_F32;
  S.opm.recon = 12;  // on the workspace's FP32 / 12-real copy of the FP64 links
  S.mid_on = prm->sloppy_prec == LQCD_F16 && prm->delta_mid > 0.0;
  S.gauge64 = gauge;
  S.gauge_s = gauge_sloppy;
  cudaStream_t s = (cudaStream_t)stream;

  const int VF = vec_prec(prm->sloppy_prec), SF = prm->sloppy_prec;
  VecArgs& a = S.va;
  memset(&a, 0, sizeof(a));
  a.g = S.g;
  a.full = subset == LQCD_FULL;
  a.bpp = (int)((S.g.nsites + BLAS_BLOCK - 1) / BLAS_BLOCK);
  a.x64 = (double*)x;
  a.b64 = (const double*)b;
  a.r64 = S.w.r64;
  a.ax64 = S.w.ax64;
  a.xs = S.w.xs;
  a.rs = S.w.rs;
  a.p = S.w.p;
  a.hb64 = (int64_t)cb_spinor_bytes(S.g, LQCD_F64);
  a.hbv = (int64_t)cb_spinor_bytes(S.g, VF);
  a.hbs = (int64_t)cb_spinor_bytes(S.g, SF);
  a.hbr = (int64_t)cb_spinor_bytes(S.g, rs_prec(SF));
  a.sys = S.w.sys;
  ReduceCtx base;
  memset(&base, 0, sizeof(base));
  base.partials = S.w.partials;
  base.counter = S.w.counter;
  base.sys = S.w.sys;
  base.ctrl = S.w.ctrl;
  base.nsys = S.nsys;
  a.red = base;
  S.rc_init = base;
  S.rc_init.fin = FIN_INIT;
  S.rc_init.tol2_rel = prm->tol * prm->tol;
  S.rc_init.delta2 = prm->sloppy_prec == LQCD_F64 ? 0.0 : prm->delta * prm->delta;
  S.rc_alpha = base;
  S.rc_alpha.fin = FIN_ALPHA;
  S.rc_update = base;
  S.rc_update.fin = FIN_UPDATE;
  S.rc_update.maxiter = prm->maxiter;
  S.rc_reliable = base;
  S.rc_reliable.fin = FIN_RELIABLE;
  S.rc_mid = base;
  S.rc_mid.fin = FIN_MID;
  S.rc_ss = base;
  S.rc_ss.fin = FIN_STORE;
  S.rc_ss.result = S.w.ss;
  if (normal) {
    S.rc_init.sysres = S.rc_reliable.sysres = 1;
    S.rc_init.result = S.rc_reliable.result = S.w.ss;
    if (b_full) S.rc_init.scale2 = S.w.bb;
  }
  S.rc_init.delta2_mid = S.mid_on ? prm->delta_mid * prm->delta_mid : 0.0;

  // what the captured graph bakes in (tol and delta live in device state, not in the graph)
  std::vector<unsigned char> key;
  int dev = 0;
  cudaGetDevice(&dev);
  key_append(key, 1);  // single-lattice solver
  key_append(key, dev);
  key_append(key, x);
  key_append(key, b);
  key_append(key, gauge);
  key_append(key, gauge_sloppy);
  key_append(key, workspace);
  for (int mu = 0; mu < 4; mu++) {
    key_append(key, lat->dims[mu]);
    key_append(key, lat->bc[mu]);
  }
  key_append(key, lat->n5);
  key_append(key, op->kind);
  key_append(key, op->mass);
  key_append(key, op->M5);
  key_append(key, op->mf);
  key_append(key, op->recon);
  key_append(key, op->gparity);
  key_append(key, prm->sloppy_prec);
  key_append(key, prm->sloppy_recon);
  key_append(key, S.prm.check_interval);
  key_append(key, prm->maxiter);
  key_append(key, subset);
  key_append(key, S.mid_on);
  key_append(key, S.normal);
  key_append(key, S.op64.prec);
  key_append(key, b_full);

  // one tuning pass per solver configuration (lattice, operator, inner formats), outside any capture
  if (S.ops.prec != LQCD_F64 && !op->gparity && hop_autotune_ready(s)) {
    char tk[200];
    snprintf(tk, sizeof(tk), "%dx%dx%dx%d n5=%d kind=%d prec=%d recon=%d subset=%d mid=%d normal=%d",
             lat->dims[0], lat->dims[1], lat->dims[2], lat->dims[3], lat->n5, op->kind, S.ops.prec, S.ops.recon,
             subset, (int)S.mid_on, (int)normal);
    if (solver_tuning_due(tk)) {
      if ((st = S.tune(s))) return finish(st);
    }
  }

  Control ctrl;
  memset(&ctrl, 0, sizeof(ctrl));
  const int status = run_cg(S, S.prm, key, s, t0, &ctrl);
  // report
  std::vector<SysState> sys(S.nsys);
  cudaError_t e = cudaMemcpyAsync(sys.data(), S.w.sys, sizeof(SysState) * S.nsys, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int out_status = status;
  if (e != cudaSuccess && out_status == LQCD_OK) out_status = cuda_fail(e, "cg: state readback");
  double worst = 0.0;
  for (int i = 0; i < S.nsys; i++) {
    const double den = normal ? sys[i].ssx : sys[i].rr0;  // CGNR: |b - M x| / |b| (full system's |b|: even-odd solve)
    double rel = den > 0 ? std::sqrt(sys[i].rr_true / den) : 0.0;
    if (rel > worst || std::isnan(rel)) worst = rel;
  }
  inf->iterations = ctrl.iter;
  inf->reliable_updates = ctrl.n_reliable;
  inf->residual_replacements = ctrl.n_mid;
  inf->true_rel_residual = worst;
  return finish(out_status);
}

}  // namespace lqcd

extern "C" {

int lqcd_cg_solve(void* x, const void* b, const void* gauge, const void* gauge_sloppy, const lqcd_lattice* lat,
                  const lqcd_operator* op, const lqcd_solver_params* prm, int subset, lqcd_solve_info* info,
                  void* workspace, size_t workspace_bytes, void* stream) {
  return cg_solve_impl(x, b, gauge, gauge_sloppy, lat, op, prm, subset, info, workspace, workspace_bytes, stream,
                       false);
}

int lqcd_cgnr_solve(void* x, const void* b, const void* gauge, const void* gauge_sloppy, const lqcd_lattice* lat,
                    const lqcd_operator* op, const lqcd_solver_params* prm, int subset, lqcd_solve_info* info,
                    void* workspace, size_t workspace_bytes, void* stream) {
  return cg_solve_impl(x, b, gauge, gauge_sloppy, lat, op, prm, subset, info, workspace, workspace_bytes, stream,
                       true);
}

// even-odd solve: [CG workspace (EVEN)][b_hat: one FP64 checkerboard][operator temporary]
size_t lqcd_eo_solve_workspace_bytes(const lqcd_lattice* lat, const lqcd_operator* op,
                                     const lqcd_solver_params* prm) {
  const size_t cgb = lqcd_cg_workspace_bytes(lat, op, prm, LQCD_EVEN);
  if (!cgb) return 0;
  Geom g;
  if (make_geom(lat, &g)) return 0;
  const size_t cb = cb_spinor_bytes(g, LQCD_F64);
  return round_up((int64_t)cgb, 256) + round_up((int64_t)cb, 256) + cb;
}

int lqcd_eo_solve(void* x, const void* b, const void* gauge, const void* gauge_sloppy, const lqcd_lattice* lat,
                  const lqcd_operator* op, const lqcd_solver_params* prm, lqcd_solve_info* info, void* workspace,
                  size_t workspace_bytes, void* stream) {
  lqcd_solve_info local;
  lqcd_solve_info* inf = info ? info : &local;
  const size_t need = lqcd_eo_solve_workspace_bytes(lat, op, prm);
  if (!need) {
    memset(inf, 0, sizeof(*inf));
    inf->status = LQCD_ERR_ARG;
    Geom g;
    int st = validate(lat, op, prm, LQCD_EVEN, &g);
    return st ? st : fail(LQCD_ERR_ARG, "eo_solve: invalid arguments");
  }
  if (!x || !b || !workspace || ((uintptr_t)workspace & 255) || workspace_bytes < need) {
    memset(inf, 0, sizeof(*inf));
    inf->status = LQCD_ERR_WORKSPACE;
    return fail(LQCD_ERR_WORKSPACE, "eo_solve: null pointer or workspace below %zu bytes (256-byte aligned)", need);
  }
  Geom g;
  make_geom(lat, &g);
  const size_t cgb = round_up((int64_t)lqcd_cg_workspace_bytes(lat, op, prm, LQCD_EVEN), 256);
  const size_t cb = cb_spinor_bytes(g, LQCD_F64);
  void* bhat = off(workspace, cgb);
  void* tmp = off(bhat, round_up((int64_t)cb, 256));
  cudaStream_t s = (cudaStream_t)stream;
  lqcd_operator opp = *op;
  // same FP64 fields, double-float arithmetic (Wilson: the domain-wall preparation's separate
  // M5op^-1 kernel has no double-float form)
  if (update_df(*op, *prm, lat->n5) && op->kind == LQCD_WILSON) opp.prec = LQCD_F64_DF;
  int st = lqcd_eo_prepare(bhat, b, gauge, lat, &opp, tmp, stream);
  if (st) {
    memset(inf, 0, sizeof(*inf));
    inf->status = st;
    return st;
  }
  // the even half of x is the first checkerboard of the full field
  // tol applies to the full system: the exit test scales by |b|^2 of the full source
  st = cg_solve_impl(x, bhat, gauge, gauge_sloppy, lat, op, prm, LQCD_EVEN, inf, workspace, cgb, stream, true, b);
  if (st != LQCD_OK && st != LQCD_ERR_NOT_CONVERGED && st != LQCD_ERR_TIMEOUT) return st;
  int rst;
  if (op->kind == LQCD_WILSON && inf->reliable_updates > 0) {
    // the last reliable update computed M_hat x_e for the x_e returned: its first hop, H_oe x_e,
    // is still in the workspace's odd temporary (t1_64)
    Geom gs = g;
    check_operator(op, gs);
    const int nsys = !op->gparity ? gs.n5 : 1;
    const Workspace w = carve(workspace, gs, *op, *prm, LQCD_EVEN, nsys);
    const unsigned grid = (unsigned)((gs.nsites + BLAS_BLOCK - 1) / BLAS_BLOCK);
    k_reconstruct_odd<<<grid, BLAS_BLOCK, 0, s>>>(gs, (double*)off(x, cb), (const double*)off(b, cb),
                                                  (const double*)w.t1_64, 4.0 + op->mass);
    rst = after_launch("eo_solve: odd half");
  } else {
    rst = lqcd_eo_reconstruct(x, b, gauge, lat, op, tmp, stream);
  }
  if (rst) return rst;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "eo_solve: synchronize");
  return st;
}

}  // extern "C"
