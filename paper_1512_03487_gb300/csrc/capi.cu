// Library-wide host state: error messages, launch counting, geometry checks.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "lqcd_internal.h"
#include "m5_scan.cuh"

namespace lqcd {

static thread_local char g_last_error[512] = "";
static std::atomic<uint64_t> g_launches{0};
// Set while a thread captures a CUDA graph: captured launches are counted when
// the graph is replayed, not when they are recorded.
thread_local bool g_count_suspended = false;
thread_local uint64_t g_captured_launches = 0;

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(LQCD_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

void count_launches(uint64_t n) {
  if (g_count_suspended) g_captured_launches += n;
  else g_launches.fetch_add(n, std::memory_order_relaxed);
}

int after_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  count_launches(1);
  return LQCD_OK;
}

int make_geom(const lqcd_lattice* lat, Geom* g) {
  if (!lat || !g) return fail(LQCD_ERR_ARG, "null lattice");
  for (int mu = 0; mu < 4; mu++) {
    if (lat->dims[mu] < 2) return fail(LQCD_ERR_ARG, "lattice extent %d in direction %d < 2", lat->dims[mu], mu);
    if (lat->bc[mu] != 1.0 && lat->bc[mu] != -1.0)
      return fail(LQCD_ERR_ARG, "boundary phase %g in direction %d is not +-1", lat->bc[mu], mu);
  }
  // A hop that wraps around an odd extent lands on a site of the same parity,
  // so even-odd checkerboarding needs every extent even.
  for (int mu = 0; mu < 4; mu++)
    if (lat->dims[mu] % 2)
      return fail(LQCD_ERR_ARG, "extent %d in direction %d must be even for checkerboarding", lat->dims[mu], mu);
  if (lat->n5 < 1) return fail(LQCD_ERR_ARG, "n5 = %d < 1", lat->n5);
  const int64_t V = (int64_t)lat->dims[0] * lat->dims[1] * lat->dims[2] * lat->dims[3];
  if (V >= ((int64_t)1 << 31) || V / 2 * lat->n5 >= ((int64_t)1 << 31))
    return fail(LQCD_ERR_ARG, "lattice too large: the 4D volume and V/2 * n5 must stay below 2^31");
  g->X = lat->dims[0];
  g->Y = lat->dims[1];
  g->Z = lat->dims[2];
  g->T = lat->dims[3];
  g->Xh = g->X / 2;
  g->Vh = (int)(V / 2);
  g->n5 = lat->n5;
  g->nsites = (int64_t)g->Vh * g->n5;
  g->sstride = round_up(g->nsites, 32);
  g->gstride = round_up(g->Vh, 32);
  for (int mu = 0; mu < 4; mu++) {
    g->bcd[mu] = lat->bc[mu];
    g->bcf[mu] = (float)lat->bc[mu];
  }
  g->fXh = make_fastdiv((uint32_t)g->Xh);
  g->fY = make_fastdiv((uint32_t)g->Y);
  g->fZ = make_fastdiv((uint32_t)g->Z);
  g->fn5 = make_fastdiv((uint32_t)g->n5);
  g->st[0] = 1;
  g->st[1] = g->X;
  g->st[2] = g->X * g->Y;
  g->st[3] = g->X * g->Y * g->Z;
  g->gp = 0;
  return LQCD_OK;
}

size_t field_bytes(const Geom& g, int prec, int subset) {
  size_t cb = cb_spinor_bytes(g, prec);
  return subset == LQCD_FULL ? 2 * cb : cb;
}

int check_operator(const lqcd_operator* op, Geom& g) {
  if (!op) return fail(LQCD_ERR_ARG, "null operator");
  if (op->kind != LQCD_WILSON && op->kind != LQCD_DWF) return fail(LQCD_ERR_ARG, "bad operator kind %d", op->kind);
  if (op->prec != LQCD_F64 && op->prec != LQCD_F32 && op->prec != LQCD_F16 && op->prec != LQCD_F64_DF)
    return fail(LQCD_ERR_ARG, "bad precision %d", op->prec);
  // double-float arithmetic: Wilson without G-parity, or domain wall on 18-real links whose L_s
  // divides 32 (M5op^-1 fused into the hop's epilogue; the separate M5op^-1 kernels have no
  // double-float form)
  if (op->prec == LQCD_F64_DF &&
      (op->gparity || (op->kind == LQCD_DWF && (op->recon != 18 || !m5_scan_ok(g.n5)))))
    return fail(LQCD_ERR_UNSUPPORTED,
                "double-float arithmetic: Wilson without G-parity, or domain wall with 18-real links and L_s "
                "dividing 32");
  if (op->recon != 18 && op->recon != 12) return fail(LQCD_ERR_ARG, "bad recon %d", op->recon);
  if (op->kind == LQCD_DWF) {
    if (g.n5 > MAX_SYS * 4) return fail(LQCD_ERR_ARG, "L_s = %d too large", g.n5);
    double d = 5.0 - op->M5;
    if (d == 0.0) return fail(LQCD_ERR_ARG, "M5 = 5 makes M5op singular");
  } else if (g.n5 > MAX_SYS) {
    return fail(LQCD_ERR_ARG, "n5 = %d right-hand sides exceed %d", g.n5, MAX_SYS);
  }
  if (op->gparity < 0 || op->gparity > 15) return fail(LQCD_ERR_ARG, "bad G-parity mask %d", op->gparity);
  if (op->gparity) {
    if (op->kind != LQCD_WILSON || g.n5 != 2)
      return fail(LQCD_ERR_ARG, "G-parity needs the Wilson operator and n5 = 2 flavours");
    if (op->prec == LQCD_F16) return fail(LQCD_ERR_UNSUPPORTED, "G-parity with LQCD_F16 storage");
  }
  g.gp = op->gparity;
  return LQCD_OK;
}

}  // namespace lqcd

extern "C" {

const char* lqcd_version(void) { return "lqcd-gb300 0.1 (sm_103a)"; }

const char* lqcd_last_error(void) { return lqcd::g_last_error; }

uint64_t lqcd_launch_count(void) { return lqcd::g_launches.load(); }

size_t lqcd_spinor_bytes(const lqcd_lattice* lat, int prec, int subset) {
  lqcd::Geom g;
  if (lqcd::make_geom(lat, &g) != LQCD_OK) return 0;
  if (lqcd::spinor_site_bytes(prec) == 0) return 0;
  if (subset != LQCD_EVEN && subset != LQCD_ODD && subset != LQCD_FULL) return 0;
  return lqcd::field_bytes(g, prec, subset);
}

size_t lqcd_gauge_bytes(const lqcd_lattice* lat, int prec, int recon) {
  lqcd::Geom g;
  if (lqcd::make_geom(lat, &g) != LQCD_OK) return 0;
  if (lqcd::spinor_site_bytes(prec) == 0 || (recon != 18 && recon != 12)) return 0;
  return (size_t)8 * g.gstride * lqcd::link_bytes(prec, recon);
}

}  // extern "C"
