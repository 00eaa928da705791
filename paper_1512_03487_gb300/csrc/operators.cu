// Dirac operators built from the fused hop kernel:
//   Wilson   D_W = (4 + m) - H / 2,      M_hat = (4 + m) - H_eo H_oe / (4 (4 + m))
//   DWF      D_DW = M5op - H / 2,        M_hat = M5op - H_eo M5op^-1 H_oe / 4
// and the even-odd source preparation / solution reconstruction.
#include <cmath>
#include <cstring>

#include "lqcd_internal.h"
#include "m5_scan.cuh"

namespace lqcd {

int launch_hop(int prec, int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s) {
  if (a.g.gp) return launch_hop_gparity(prec, recon, dagger, epi, reduce, a, s);
  switch (prec) {
    case LQCD_F64: return launch_hop_f64(recon, dagger, epi, reduce, a, s);
    case LQCD_F32: return launch_hop_f32(recon, dagger, epi, reduce, a, s);
    case LQCD_F16: return launch_hop_f16(recon, dagger, epi, reduce, a, s);
    case LQCD_F64_DF: return launch_hop_df(recon, dagger, epi, reduce, a, s);
  }
  return fail(LQCD_ERR_ARG, "bad precision %d", prec);
}

size_t op_tmp_bytes(const Geom& g, int kind, int prec, int subset) {
  if (subset == LQCD_FULL) return 0;
  const size_t cb = cb_spinor_bytes(g, prec);
  return kind == LQCD_DWF ? 2 * cb : cb;
}

static HopArgs base_args(const OpCtx& c, const ReduceCtx* red, const Control* gate) {
  HopArgs a;
  memset(&a, 0, sizeof(a));
  a.g = c.g;
  a.gauge = c.gauge;
  a.gate = gate;
  if (red) a.red = *red;
  a.m5d = 5.0 - c.op.M5;
  a.mf = c.op.mf;
  a.m5_a = 1.0 / a.m5d;
  a.m5_den_inv = 1.0 / (1.0 + a.mf * std::pow(a.m5_a, (double)c.g.n5));
  return a;
}

int op_apply(const OpCtx& c, void* out, const void* in, int subset, int dagger, void* t1, void* t2,
             const ReduceCtx* red, const Control* gate, cudaStream_t s, const HopUpdate* upd) {
  const int P = c.op.prec, R = c.op.recon;
  if (upd && (!red || !dagger)) return fail(LQCD_ERR_ARG, "fused CG update needs a reduction and dagger");
  const int mode = upd ? RED_CG_UPDATE : red ? RED_NORM : RED_NONE;
  auto set_upd = [&](HopArgs& a) {
    if (!upd) return;
    a.upd_p = upd->p;
    a.upd_xs = upd->xs;
    a.upd_rs = upd->rs;
    a.upd_half_bytes = upd->half_bytes;
    a.upd_rs_half_bytes = upd->rs_half_bytes;
  };
  const bool wilson = c.op.kind == LQCD_WILSON;
  const double cw = 4.0 + c.op.mass;
  if (subset == LQCD_FULL) {
    HopArgs a = base_args(c, red, gate);
    a.full = 1;
    a.half_bytes = (int64_t)cb_spinor_bytes(c.g, P);
    a.out = out;
    a.in = in;
    a.x = in;
    a.a = cw;
    a.b = -0.5;
    set_upd(a);
    return launch_hop(P, R, dagger, wilson ? EPI_XPAY : EPI_M5, mode, a, s);
  }
  if (subset != LQCD_EVEN) return fail(LQCD_ERR_ARG, "operator subset must be LQCD_EVEN or LQCD_FULL");
  HopArgs h1 = base_args(c, nullptr, gate);
  h1.out_parity = LQCD_ODD;
  h1.out = t1;
  h1.in = in;
  h1.b = 1.0;
  // domain wall with L_s dividing 32: M5op^-1 runs in the first hop's epilogue
  const bool fuse_m5 = !wilson && m5_scan_ok(c.g.n5);
  if (fuse_m5) {
    h1.out = t2;
    h1.m5_dagger = dagger;
  }
  int st = launch_hop(P, R, dagger, fuse_m5 ? EPI_M5INV : EPI_PLAIN, RED_NONE, h1, s);
  if (st) return st;
  const void* src = fuse_m5 ? t2 : t1;
  if (!wilson && !fuse_m5) {
    M5Args m;
    m.out = t2;
    m.in = t1;
    m.g = c.g;
    m.d = 5.0 - c.op.M5;
    m.mf = c.op.mf;
    m.dagger = dagger;
    m.gate = gate;
    if ((st = launch_m5inv(P, m, s))) return st;
    src = t2;
  }
  HopArgs h2 = base_args(c, red, gate);
  h2.out_parity = LQCD_EVEN;
  h2.out = out;
  h2.in = src;
  h2.x = in;
  if (wilson) {
    h2.a = cw;
    h2.b = -1.0 / (4.0 * cw);
  } else {
    h2.b = -0.25;
  }
  set_upd(h2);
  return launch_hop(P, R, dagger, wilson ? EPI_XPAY : EPI_M5, mode, h2, s);
}

static bool misaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) != 0; }

static int common_checks(const lqcd_lattice* lat, const lqcd_operator* op, Geom* g) {
  int st = make_geom(lat, g);
  if (st) return st;
  return check_operator(op, *g);
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

int lqcd_dslash(void* out, const void* in, const void* gauge, const lqcd_lattice* lat,
                const lqcd_operator* op, int out_subset, int dagger, void* stream) {
  Geom g;
  int st = common_checks(lat, op, &g);
  if (st) return st;
  if (!out || !in || !gauge || misaligned(out) || misaligned(in) || misaligned(gauge))
    return fail(LQCD_ERR_ARG, "lqcd_dslash: null or misaligned pointer");
  if (out == in) return fail(LQCD_ERR_ARG, "lqcd_dslash: out aliases in");
  if (out_subset != LQCD_EVEN && out_subset != LQCD_ODD && out_subset != LQCD_FULL)
    return fail(LQCD_ERR_ARG, "lqcd_dslash: bad subset %d", out_subset);
  OpCtx c{g, *op, gauge};
  HopArgs a = base_args(c, nullptr, nullptr);
  a.out = out;
  a.in = in;
  a.b = 1.0;
  a.full = out_subset == LQCD_FULL;
  a.out_parity = a.full ? 0 : out_subset;
  a.half_bytes = (int64_t)cb_spinor_bytes(g, op->prec);
  return launch_hop(op->prec, op->recon, dagger != 0, EPI_PLAIN, RED_NONE, a, (cudaStream_t)stream);
}

size_t lqcd_operator_workspace_bytes(const lqcd_lattice* lat, const lqcd_operator* op, int subset) {
  Geom g;
  if (common_checks(lat, op, &g)) return 0;
  if (subset != LQCD_EVEN && subset != LQCD_FULL) return 0;
  return field_bytes(g, op->prec, subset) + op_tmp_bytes(g, op->kind, op->prec, subset);
}

int lqcd_M(void* out, const void* in, const void* gauge, const lqcd_lattice* lat, const lqcd_operator* op,
           int subset, int dagger, void* tmp, void* stream) {
  Geom g;
  int st = common_checks(lat, op, &g);
  if (st) return st;
  if (!out || !in || !gauge || misaligned(out) || misaligned(in) || misaligned(gauge) || misaligned(tmp))
    return fail(LQCD_ERR_ARG, "lqcd_M: null or misaligned pointer");
  if (out == in) return fail(LQCD_ERR_ARG, "lqcd_M: out aliases in");
  if (subset == LQCD_EVEN && !tmp) return fail(LQCD_ERR_ARG, "lqcd_M: workspace required");
  OpCtx c{g, *op, gauge};
  void* t1 = tmp;
  void* t2 = tmp ? off(tmp, cb_spinor_bytes(g, op->prec)) : nullptr;
  return op_apply(c, out, in, subset, dagger != 0, t1, t2, nullptr, nullptr, (cudaStream_t)stream);
}

int lqcd_MdagM(void* out, const void* in, const void* gauge, const lqcd_lattice* lat, const lqcd_operator* op,
               int subset, void* tmp, void* stream) {
  Geom g;
  int st = common_checks(lat, op, &g);
  if (st) return st;
  if (!out || !in || !gauge || !tmp || misaligned(out) || misaligned(in) || misaligned(gauge) || misaligned(tmp))
    return fail(LQCD_ERR_ARG, "lqcd_MdagM: null or misaligned pointer");
  if (subset != LQCD_EVEN && subset != LQCD_FULL) return fail(LQCD_ERR_ARG, "lqcd_MdagM: bad subset");
  OpCtx c{g, *op, gauge};
  void* mid = tmp;
  void* t1 = off(tmp, field_bytes(g, op->prec, subset));
  void* t2 = off(t1, cb_spinor_bytes(g, op->prec));
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = op_apply(c, mid, in, subset, 0, t1, t2, nullptr, nullptr, s))) return st;
  return op_apply(c, out, mid, subset, 1, t1, t2, nullptr, nullptr, s);
}

int lqcd_eo_prepare(void* bhat, const void* b_full, const void* gauge, const lqcd_lattice* lat,
                    const lqcd_operator* op, void* tmp, void* stream) {
  Geom g;
  int st = common_checks(lat, op, &g);
  if (st) return st;
  if (!bhat || !b_full || !gauge || misaligned(bhat) || misaligned(b_full) || misaligned(tmp))
    return fail(LQCD_ERR_ARG, "lqcd_eo_prepare: null or misaligned pointer");
  if (op->kind == LQCD_DWF && !tmp) return fail(LQCD_ERR_ARG, "lqcd_eo_prepare: workspace required");
  const size_t cb = cb_spinor_bytes(g, op->prec);
  const void* b_even = b_full;
  const void* b_odd = off(b_full, cb);
  cudaStream_t s = (cudaStream_t)stream;
  OpCtx c{g, *op, gauge};
  HopArgs a = base_args(c, nullptr, nullptr);
  a.out_parity = LQCD_EVEN;
  a.out = bhat;
  a.x = b_even;
  a.a = 1.0;
  if (op->kind == LQCD_WILSON) {
    a.in = b_odd;
    a.b = 1.0 / (2.0 * (4.0 + op->mass));
  } else {
    M5Args m{tmp, b_odd, g, 5.0 - op->M5, op->mf, 0, nullptr};
    if ((st = launch_m5inv(op->prec, m, s))) return st;
    a.in = tmp;
    a.b = 0.5;
  }
  return launch_hop(op->prec, op->recon, false, EPI_XPAY, RED_NONE, a, s);
}

int lqcd_eo_reconstruct(void* x_full, const void* b_full, const void* gauge, const lqcd_lattice* lat,
                        const lqcd_operator* op, void* tmp, void* stream) {
  Geom g;
  int st = common_checks(lat, op, &g);
  if (st) return st;
  if (!x_full || !b_full || !gauge || misaligned(x_full) || misaligned(b_full) || misaligned(tmp))
    return fail(LQCD_ERR_ARG, "lqcd_eo_reconstruct: null or misaligned pointer");
  if (op->kind == LQCD_DWF && !tmp) return fail(LQCD_ERR_ARG, "lqcd_eo_reconstruct: workspace required");
  const size_t cb = cb_spinor_bytes(g, op->prec);
  cudaStream_t s = (cudaStream_t)stream;
  OpCtx c{g, *op, gauge};
  HopArgs a = base_args(c, nullptr, nullptr);
  a.out_parity = LQCD_ODD;
  a.in = x_full;
  a.x = off(b_full, cb);
  if (op->kind == LQCD_WILSON) {
    const double cw = 4.0 + op->mass;
    a.out = off(x_full, cb);
    a.a = 1.0 / cw;
    a.b = 1.0 / (2.0 * cw);
    return launch_hop(op->prec, op->recon, false, EPI_XPAY, RED_NONE, a, s);
  }
  a.out = tmp;
  a.a = 1.0;
  a.b = 0.5;
  if ((st = launch_hop(op->prec, op->recon, false, EPI_XPAY, RED_NONE, a, s))) return st;
  M5Args m{off(x_full, cb), tmp, g, 5.0 - op->M5, op->mf, 0, nullptr};
  return launch_m5inv(op->prec, m, s);
}

}  // extern "C"
