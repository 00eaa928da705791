// Batched even-odd Wilson CG over independent lattices of different sizes.
//
// All instances advance in lockstep, each with its own alpha, beta,
// reliable-update and convergence state (one SysState per instance). Every
// phase of an iteration is ONE persistent launch over a work list of tiles
// (instance, TILE consecutive sites): a fixed grid of resident blocks strides
// through the list, finds each tile's instance from a prefix table held in
// shared memory, and runs the same per-site code as the single-lattice
// kernels (hop_site, cg_site.cuh). Reductions accumulate per instance in
// shared memory, write one partial per (instance, block), and the last block
// to finish sums them per instance in a fixed order. The tile (64, 128 or 256
// sites, one thread per site) and the grid size (resident blocks per SM) are
// chosen together by timing candidates on the first solve of a given batch
// shape (the autotuner); the choice is cached per shape and can be saved and
// loaded. The iteration loop is the shared conditional-graph driver. With
// update_prec = LQCD_F64_DF the reliable updates' M_hat x runs in double-float
// arithmetic on the FP64 fields (on GB300 about twice as fast as the FP64 pipe).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "cg_engine.h"
#include "cg_site.cuh"
#include "tune.h"

namespace lqcd {

// Tile sizes the tuner chooses among (sites per tile == threads per block).
constexpr int NTILES = 3;
constexpr int TILES[NTILES] = {64, 128, 256};
template <int TILE> constexpr int tile_slot() { return TILE == 64 ? 0 : TILE == 128 ? 1 : 2; }
constexpr int MAX_BATCH = MAX_SYS;

// field selectors of a batch instance
enum BField { BF_X64, BF_B64, BF_R64, BF_AX64, BF_MID64, BF_T1_64, BF_XS, BF_RS, BF_P, BF_AP, BF_MP, BF_T1S, BF_NONE };

struct BInst {
  Geom g;
  const void* gauge64;
  const void* gauge_s;
  double c;  // 4 + m
  double b;  // -1 / (4 c), the Schur hop's coefficient
  void* f[12];
  int64_t tile0[NTILES];  // first tile of this instance in the work list, per tile size
};

struct BatchArgs {
  const BInst* inst;
  int ninst;
  int64_t total_tiles;
  ReduceCtx red;
  const Control* gate;
  int f_out, f_in, f_x;
  int use64;
  int out_parity;
};

__device__ __forceinline__ int find_inst(const int64_t* t0, int n, int64_t t) {
  int lo = 0, hi = n - 1;  // largest i with t0[i] <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t0[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Sum of v over the block, added by thread 0 to acc (all threads call it).
template <int TILE>
__device__ __forceinline__ void block_add(double v, double* sh, double* acc) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < TILE / 32; w++) s += sh[w];
    *acc += s;
  }
  __syncthreads();
}

// RED: RED_NONE, RED_NORM (|out|^2 per instance) or RED_CG_UPDATE (out = A p is
// not stored; x_s += alpha p, r_s -= alpha A p and |r_s|^2 per instance instead).
template <int P, int R, bool DAG, int EPI, int RED, int TILE>
__global__ void __launch_bounds__(TILE) batch_hop_kernel(const BatchArgs A) {
  using T = typename PrecTraits<P>::real;
  if (gate_closed(A.gate)) return;
  __shared__ int64_t s_t0[MAX_BATCH];
  __shared__ double s_acc[MAX_BATCH];
  __shared__ double sh[TILE];
  for (int i = threadIdx.x; i < A.ninst; i += TILE) {
    s_t0[i] = A.inst[i].tile0[tile_slot<TILE>()];
    s_acc[i] = 0.0;
  }
  __syncthreads();
  for (int64_t t = blockIdx.x; t < A.total_tiles; t += gridDim.x) {
    const int k = find_inst(s_t0, A.ninst, t);
    const BInst& I = A.inst[k];
    const int64_t j = (t - s_t0[k]) * TILE + threadIdx.x;
    double v = 0.0;
    if (j < I.g.nsites) {
      EpiCoef c;
      c.a = I.c;
      c.b = EPI == EPI_XPAY ? I.b : 1.0;
      c.m5d = 0.0;
      c.mf = 0.0;
      Spinor<T> res;
      hop_site<P, R, DAG, EPI>(I.g, A.use64 ? I.gauge64 : I.gauge_s, I.f[A.f_in],
                               A.f_x == BF_NONE ? nullptr : I.f[A.f_x], A.out_parity, j, c, res);
      if constexpr (RED == RED_CG_UPDATE) {
        v = update_site_ap<vec_prec(P), P>(I.g, j, A.red.sys[k].alpha, I.f[BF_P], res, I.f[BF_XS], I.f[BF_RS]);
      } else {
        SpinorIO<P>::store(I.f[A.f_out], I.g.sstride, j, res);
        if constexpr (RED == RED_NORM) v = norm2_site(res);
      }
    }
    if constexpr (RED != RED_NONE) block_add<TILE>(v, sh, &s_acc[k]);
  }
  if constexpr (RED != RED_NONE) {
    for (int i = threadIdx.x; i < A.ninst; i += TILE) A.red.partials[(int64_t)i * gridDim.x + blockIdx.x] = s_acc[i];
    last_block_finalize<TILE>(A.red, sh);
  }
}

enum BatchVec { BV_INIT, BV_UPDATE, BV_PUPDATE, BV_ACCUM, BV_RESIDUAL };

template <int VF, int SF, int KIND, int TILE>
__global__ void __launch_bounds__(TILE) batch_vec_kernel(const BatchArgs A) {
  constexpr bool RED = KIND == BV_INIT || KIND == BV_UPDATE || KIND == BV_RESIDUAL;
  constexpr bool GATED = KIND == BV_UPDATE || KIND == BV_PUPDATE;
  if (GATED && gate_closed(A.gate)) return;
  __shared__ int64_t s_t0[MAX_BATCH];
  __shared__ double s_acc[MAX_BATCH];
  __shared__ double sh[TILE];
  for (int i = threadIdx.x; i < A.ninst; i += TILE) {
    s_t0[i] = A.inst[i].tile0[tile_slot<TILE>()];
    s_acc[i] = 0.0;
  }
  __syncthreads();
  for (int64_t t = blockIdx.x; t < A.total_tiles; t += gridDim.x) {
    const int k = find_inst(s_t0, A.ninst, t);
    const BInst& I = A.inst[k];
    const int64_t j = (t - s_t0[k]) * TILE + threadIdx.x;
    double v = 0.0;
    if (j < I.g.nsites) {
      void* const* f = I.f;
      if (KIND == BV_INIT)
        v = init_site<VF, SF>(I.g, j, (const double*)f[BF_B64], (double*)f[BF_R64], (double*)f[BF_X64], f[BF_RS],
                              f[BF_XS], f[BF_P]);
      else if (KIND == BV_UPDATE)
        v = update_site<VF, SF>(I.g, j, A.red.sys[k].alpha, f[BF_P], f[BF_AP], f[BF_XS], f[BF_RS]);
      else if (KIND == BV_PUPDATE)
        pupdate_site<VF, SF>(I.g, j, A.red.sys[k].beta, f[BF_RS], f[BF_P]);
      else if (KIND == BV_ACCUM)
        accumulate_site<VF>(I.g, j, (double*)f[BF_X64], f[BF_XS]);
      else
        v = residual_site<VF>(I.g, j, (const double*)f[BF_B64], (const double*)f[BF_AX64], (double*)f[BF_R64],
                              f[BF_RS]);
    }
    if (RED) block_add<TILE>(v, sh, &s_acc[k]);
  }
  if (RED) {
    for (int i = threadIdx.x; i < A.ninst; i += TILE) A.red.partials[(int64_t)i * gridDim.x + blockIdx.x] = s_acc[i];
    last_block_finalize<TILE>(A.red, sh);
  }
}

// ------------------------------------------------------------------ launchers

template <int P, int R, int TILE>
static void launch_bhop_pr(bool dag, int epi, int red, unsigned grid, const BatchArgs& a, cudaStream_t s) {
#define LQCD_BHOP(DG, EP, RD) batch_hop_kernel<P, R, DG, EP, RD, TILE><<<grid, TILE, 0, s>>>(a)
  if (epi == EPI_PLAIN) {
    if (dag) LQCD_BHOP(true, EPI_PLAIN, RED_NONE);
    else LQCD_BHOP(false, EPI_PLAIN, RED_NONE);
  } else if (red == RED_CG_UPDATE) {  // the last hop of M_hat^dag M_hat
    LQCD_BHOP(true, EPI_XPAY, RED_CG_UPDATE);
  } else if (red == RED_NORM) {
    if (dag) LQCD_BHOP(true, EPI_XPAY, RED_NORM);
    else LQCD_BHOP(false, EPI_XPAY, RED_NORM);
  } else {
    if (dag) LQCD_BHOP(true, EPI_XPAY, RED_NONE);
    else LQCD_BHOP(false, EPI_XPAY, RED_NONE);
  }
#undef LQCD_BHOP
}

// double-float hops on the FP64 fields (the reliable updates' M_hat x): no reduction
template <int R, int TILE>
static void launch_bhop_df(bool dag, int epi, unsigned grid, const BatchArgs& a, cudaStream_t s) {
#define LQCD_BHOP(DG, EP) batch_hop_kernel<LQCD_F64_DF, R, DG, EP, RED_NONE, TILE><<<grid, TILE, 0, s>>>(a)
  if (epi == EPI_PLAIN) {
    if (dag) LQCD_BHOP(true, EPI_PLAIN);
    else LQCD_BHOP(false, EPI_PLAIN);
  } else {
    if (dag) LQCD_BHOP(true, EPI_XPAY);
    else LQCD_BHOP(false, EPI_XPAY);
  }
#undef LQCD_BHOP
}

template <int TILE>
static void launch_bhop_t(int prec, int recon, bool dag, int epi, int red, unsigned grid, const BatchArgs& a,
                          cudaStream_t s) {
  if (prec == LQCD_F64_DF) {  // the caller passes no reduction for it
    if (recon == 18) launch_bhop_df<18, TILE>(dag, epi, grid, a, s);
    else launch_bhop_df<12, TILE>(dag, epi, grid, a, s);
  } else if (prec == LQCD_F64) {
    if (recon == 18) launch_bhop_pr<LQCD_F64, 18, TILE>(dag, epi, red, grid, a, s);
    else launch_bhop_pr<LQCD_F64, 12, TILE>(dag, epi, red, grid, a, s);
  } else if (prec == LQCD_F32) {
    if (recon == 18) launch_bhop_pr<LQCD_F32, 18, TILE>(dag, epi, red, grid, a, s);
    else launch_bhop_pr<LQCD_F32, 12, TILE>(dag, epi, red, grid, a, s);
  } else {
    if (recon == 18) launch_bhop_pr<LQCD_F16, 18, TILE>(dag, epi, red, grid, a, s);
    else launch_bhop_pr<LQCD_F16, 12, TILE>(dag, epi, red, grid, a, s);
  }
}

// tile: index into TILES; a.total_tiles is that tile size's count
static int launch_bhop(int tile, int prec, int recon, bool dag, int epi, int red, unsigned grid, const BatchArgs& a,
                       cudaStream_t s) {
  if (tile == 0) launch_bhop_t<64>(prec, recon, dag, epi, red, grid, a, s);
  else if (tile == 1) launch_bhop_t<128>(prec, recon, dag, epi, red, grid, a, s);
  else launch_bhop_t<256>(prec, recon, dag, epi, red, grid, a, s);
  return after_launch("batch_hop_kernel");
}

template <int VF, int SF, int TILE>
static void launch_bvec_tt(int kind, unsigned grid, const BatchArgs& a, cudaStream_t s) {
  switch (kind) {
    case BV_INIT: batch_vec_kernel<VF, SF, BV_INIT, TILE><<<grid, TILE, 0, s>>>(a); break;
    case BV_UPDATE: batch_vec_kernel<VF, SF, BV_UPDATE, TILE><<<grid, TILE, 0, s>>>(a); break;
    case BV_PUPDATE: batch_vec_kernel<VF, SF, BV_PUPDATE, TILE><<<grid, TILE, 0, s>>>(a); break;
    case BV_ACCUM: batch_vec_kernel<VF, SF, BV_ACCUM, TILE><<<grid, TILE, 0, s>>>(a); break;
    case BV_RESIDUAL: batch_vec_kernel<VF, SF, BV_RESIDUAL, TILE><<<grid, TILE, 0, s>>>(a); break;
  }
}

template <int VF, int SF>
static void launch_bvec_t(int tile, int kind, unsigned grid, const BatchArgs& a, cudaStream_t s) {
  if (tile == 0) launch_bvec_tt<VF, SF, 64>(kind, grid, a, s);
  else if (tile == 1) launch_bvec_tt<VF, SF, 128>(kind, grid, a, s);
  else launch_bvec_tt<VF, SF, 256>(kind, grid, a, s);
}

static int launch_bvec(int tile, int kind, int sloppy, unsigned grid, const BatchArgs& a, cudaStream_t s) {
  if (sloppy == LQCD_F64) launch_bvec_t<LQCD_F64, LQCD_F64>(tile, kind, grid, a, s);
  else if (sloppy == LQCD_F32) launch_bvec_t<LQCD_F32, LQCD_F32>(tile, kind, grid, a, s);
  else launch_bvec_t<LQCD_F32, LQCD_F16>(tile, kind, grid, a, s);
  return after_launch("batch_vec_kernel");
}

// ------------------------------------------------------------------ autotuned grid size

static std::string shape_key(int n, const Geom* geoms, int sloppy, int recon, int sms) {
  std::string k = "batch_hop sms=" + std::to_string(sms) + " prec=" + std::to_string(sloppy) +
                  " recon=" + std::to_string(recon) + " :";
  for (int i = 0; i < n; i++)
    k += " " + std::to_string(geoms[i].X) + "x" + std::to_string(geoms[i].Y) + "x" + std::to_string(geoms[i].Z) +
         "x" + std::to_string(geoms[i].T);
  return k;
}

// ------------------------------------------------------------------ workspace

struct BatchLayout {
  Control* ctrl;
  SysState* sys;
  double* partials;
  unsigned int* counter;
  BInst* inst;  // device copy of the descriptors
  size_t fields_offset[MAX_BATCH];
  size_t total;
};

constexpr int MAX_GRID = 8192;

static size_t inst_field_bytes(const Geom& g, int sloppy) {
  const int VF = sloppy == LQCD_F64 ? LQCD_F64 : LQCD_F32;
  const size_t cb64 = cb_spinor_bytes(g, LQCD_F64);
  return 4 * cb64 + 2 * cb_spinor_bytes(g, VF) + 4 * cb_spinor_bytes(g, sloppy) + 16 * 256;
}

static BatchLayout batch_layout(char* base, int n, const Geom* geoms, int sloppy) {
  BatchLayout L;
  memset(&L, 0, sizeof(L));
  size_t o = 0;
  auto take = [&](size_t bytes) -> char* {
    char* r = base ? base + o : nullptr;
    o += round_up((int64_t)bytes, 256);
    return r;
  };
  L.ctrl = (Control*)take(sizeof(Control));
  L.sys = (SysState*)take(sizeof(SysState) * MAX_SYS);
  L.partials = (double*)take(sizeof(double) * (size_t)n * MAX_GRID);
  L.counter = (unsigned int*)take(64);
  L.inst = (BInst*)take(sizeof(BInst) * n);
  for (int i = 0; i < n; i++) {
    L.fields_offset[i] = o;
    o += round_up((int64_t)inst_field_bytes(geoms[i], sloppy), 256);
  }
  L.total = o;
  return L;
}

static int validate_batch(int n, const lqcd_batch_item* items, int recon, const lqcd_solver_params* p, Geom* geoms) {
  if (n < 1 || n > MAX_BATCH) return fail(LQCD_ERR_ARG, "batch: n = %d outside [1, %d]", n, MAX_BATCH);
  if (!items || !p) return fail(LQCD_ERR_ARG, "batch: null items or params");
  if (recon != 18 && recon != 12) return fail(LQCD_ERR_ARG, "batch: bad recon %d", recon);
  if (p->sloppy_prec != LQCD_F64 && p->sloppy_prec != LQCD_F32 && p->sloppy_prec != LQCD_F16)
    return fail(LQCD_ERR_ARG, "batch: bad sloppy precision %d", p->sloppy_prec);
  if (p->sloppy_recon != 18 && p->sloppy_recon != 12) return fail(LQCD_ERR_ARG, "batch: bad sloppy recon");
  if (!(p->tol > 0.0) || p->maxiter < 1) return fail(LQCD_ERR_ARG, "batch: tol must be > 0 and maxiter >= 1");
  if (p->delta < 0.0 || p->delta >= 1.0) return fail(LQCD_ERR_ARG, "batch: delta must be in [0, 1)");
  if (p->update_prec != LQCD_F64 && p->update_prec != LQCD_F64_DF)
    return fail(LQCD_ERR_ARG, "batch: update_prec must be LQCD_F64 or LQCD_F64_DF");
  for (int i = 0; i < n; i++) {
    int st = make_geom(&items[i].lat, &geoms[i]);
    if (st) return st;
    if (geoms[i].n5 != 1) return fail(LQCD_ERR_ARG, "batch: item %d has n5 = %d (must be 1)", i, geoms[i].n5);
  }
  return LQCD_OK;
}

// ------------------------------------------------------------------ engine

struct BatchSolver : CgEngine {
  int n;
  int sloppy, sloppy_recon, recon;
  bool df;                          // reliable updates in double-float arithmetic
  unsigned grid;
  int tile;                         // index into TILES
  int64_t total_tiles;              // of the chosen tile size
  int64_t tiles_by_size[NTILES];    // work-list length per tile size
  BatchArgs base;
  ReduceCtx rc_init, rc_alpha, rc_update, rc_reliable;

  void set_tile(int t) {
    tile = t;
    total_tiles = tiles_by_size[t];
    base.total_tiles = total_tiles;
  }
  BatchArgs args(int f_out, int f_in, int f_x, int use64, int parity, const Control* gate) const {
    BatchArgs a = base;
    a.f_out = f_out;
    a.f_in = f_in;
    a.f_x = f_x;
    a.use64 = use64;
    a.out_parity = parity;
    a.gate = gate;
    return a;
  }
  // out = M_hat in (dagger), through the odd temporary; with red, red_mode RED_NORM
  // reduces |out|^2 and RED_CG_UPDATE applies the CG update instead of storing out
  int schur(int f_out, int f_in, int f_tmp, bool dag, bool use64, const ReduceCtx* red, const Control* gate,
            cudaStream_t s, int red_mode = RED_NORM) {
    const int P = use64 ? (df ? LQCD_F64_DF : LQCD_F64) : sloppy;
    const int R = use64 ? recon : sloppy_recon;
    BatchArgs a1 = args(f_tmp, f_in, BF_NONE, use64, LQCD_ODD, gate);
    int st = launch_bhop(tile, P, R, dag, EPI_PLAIN, RED_NONE, grid, a1, s);
    if (st) return st;
    BatchArgs a2 = args(f_out, f_tmp, f_in, use64, LQCD_EVEN, gate);
    if (red) a2.red = *red;
    return launch_bhop(tile, P, R, dag, EPI_XPAY, red ? red_mode : RED_NONE, grid, a2, s);
  }
  int init(cudaStream_t s) override {
    cudaError_t e = cudaMemsetAsync(base.red.counter, 0, 64, s);
    if (e != cudaSuccess) return cuda_fail(e, "batch: memset");
    BatchArgs a = base;
    a.red = rc_init;
    return launch_bvec(tile, BV_INIT, sloppy, grid, a, s);
  }
  // M_hat p with |M_hat p|^2 = p^dag A p -> alpha; M_hat^dag (M_hat p) = A p whose last
  // hop applies x_s += alpha p, r_s -= alpha A p and reduces |r_s|^2 instead of storing A p
  int head(cudaStream_t s, int cond, cudaGraphConditionalHandle h_rel, cudaGraphConditionalHandle) override {
    int st = schur(BF_MP, BF_P, BF_T1S, false, false, &rc_alpha, ctrl, s);
    if (st) return st;
    ReduceCtx ru = rc_update;
    ru.cond = cond;
    ru.h_rel = h_rel;
    return schur(BF_AP, BF_MP, BF_T1S, true, false, &ru, ctrl, s, RED_CG_UPDATE);  // BF_AP is not written
  }
  int tail(cudaStream_t s) override {
    BatchArgs a = base;
    a.gate = ctrl;
    return launch_bvec(tile, BV_PUPDATE, sloppy, grid, a, s);
  }
  int reliable(cudaStream_t s) override {
    BatchArgs a = base;
    int st = launch_bvec(tile, BV_ACCUM, sloppy, grid, a, s);
    if (st) return st;
    if ((st = schur(BF_MID64, BF_X64, BF_T1_64, false, true, nullptr, nullptr, s))) return st;
    if ((st = schur(BF_AX64, BF_MID64, BF_T1_64, true, true, nullptr, nullptr, s))) return st;
    a.red = rc_reliable;
    return launch_bvec(tile, BV_RESIDUAL, sloppy, grid, a, s);
  }
};

static int sm_count(int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "batch: device query");
  return LQCD_OK;
}

// Time the sloppy plain hop phase for every tile size and several resident-block
// counts and keep the fastest pair (tile index into TILES, blocks per SM).
static int autotune_batch(BatchSolver& S, int sms, int* best_tile, int* best_bps, cudaStream_t s) {
  const int candidates[] = {1, 2, 4, 6, 8, 12, 16};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(LQCD_ERR_CUDA, "batch autotune: event create");
  float best = 1e30f;
  *best_tile = 1;
  *best_bps = 4;
  int st = LQCD_OK;
  for (int tile = 0; tile < NTILES && st == LQCD_OK; tile++) {
    S.set_tile(tile);
    for (int bps : candidates) {
      int64_t g = (int64_t)bps * sms;
      if (g > S.total_tiles) g = S.total_tiles;
      if (g > MAX_GRID) g = MAX_GRID;
      const unsigned grid = (unsigned)g;
      BatchArgs a = S.args(BF_T1S, BF_P, BF_NONE, 0, LQCD_ODD, nullptr);
      float ms_total = 0.f;
      for (int rep = 0; rep < 4 && st == LQCD_OK; rep++) {
        cudaEventRecord(e0, s);
        st = launch_bhop(tile, S.sloppy, S.sloppy_recon, false, EPI_PLAIN, RED_NONE, grid, a, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) ms_total += ms;  // first launch warms up
      }
      if (st) break;
      if (ms_total < best) {
        best = ms_total;
        *best_tile = tile;
        *best_bps = bps;
      }
      if (g == S.total_tiles) break;  // larger grids cannot differ
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

size_t lqcd_batch_cg_workspace_bytes(int n, const lqcd_batch_item* items, int recon,
                                     const lqcd_solver_params* params) {
  Geom geoms[MAX_BATCH];
  if (validate_batch(n, items, recon, params, geoms)) return 0;
  return batch_layout(nullptr, n, geoms, params->sloppy_prec).total;
}

int lqcd_batch_cg_solve(int n, const lqcd_batch_item* items, int recon, const lqcd_solver_params* prm,
                        lqcd_solve_info* infos, void* workspace, size_t workspace_bytes, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  Geom geoms[MAX_BATCH];
  int st = validate_batch(n, items, recon, prm, geoms);
  auto finish = [&](int status, const Control* c, const SysState* sys) {
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (infos)
      for (int i = 0; i < (n > 0 && n <= MAX_BATCH ? n : 0); i++) {
        memset(&infos[i], 0, sizeof(infos[i]));
        infos[i].status = status;
        infos[i].time_ms = ms;
        if (c) {
          infos[i].iterations = c->iter;
          infos[i].reliable_updates = c->n_reliable;
        }
        if (sys) infos[i].true_rel_residual = sys[i].rr0 > 0 ? std::sqrt(sys[i].rr_true / sys[i].rr0) : 0.0;
      }
    return status;
  };
  if (st) return finish(st, nullptr, nullptr);
  if (!workspace || ((uintptr_t)workspace & 255)) return finish(fail(LQCD_ERR_ARG, "batch: workspace"), 0, 0);
  for (int i = 0; i < n; i++) {
    const lqcd_batch_item& it = items[i];
    if (!it.x || !it.b || !it.gauge || ((uintptr_t)it.x & 15) || ((uintptr_t)it.b & 15))
      return finish(fail(LQCD_ERR_ARG, "batch: item %d has a null or misaligned field", i), 0, 0);
    if (!it.gauge_sloppy && prm->sloppy_prec != LQCD_F64)
      return finish(fail(LQCD_ERR_ARG, "batch: item %d needs gauge_sloppy", i), 0, 0);
  }
  char* base = static_cast<char*>(workspace);
  BatchLayout lay = batch_layout(base, n, geoms, prm->sloppy_prec);
  if (workspace_bytes < lay.total)
    return finish(fail(LQCD_ERR_WORKSPACE, "batch: workspace %zu < %zu bytes", workspace_bytes, lay.total), 0, 0);
  cudaStream_t s = (cudaStream_t)stream;

  // descriptors
  const int VF = prm->sloppy_prec == LQCD_F64 ? LQCD_F64 : LQCD_F32;
  BInst host[MAX_BATCH];
  int64_t tiles_by[NTILES] = {0, 0, 0};
  for (int i = 0; i < n; i++) {
    const Geom& g = geoms[i];
    BInst& I = host[i];
    memset(&I, 0, sizeof(I));
    I.g = g;
    I.gauge64 = items[i].gauge;
    I.gauge_s = (prm->sloppy_prec == LQCD_F64 || !items[i].gauge_sloppy) ? items[i].gauge : items[i].gauge_sloppy;
    I.c = 4.0 + items[i].mass;
    I.b = -1.0 / (4.0 * I.c);
    for (int t = 0; t < NTILES; t++) {
      I.tile0[t] = tiles_by[t];
      tiles_by[t] += (g.nsites + TILES[t] - 1) / TILES[t];
    }
    char* f = base + lay.fields_offset[i];
    size_t o = 0;
    auto take = [&](size_t bytes) -> void* {
      void* r = f + o;
      o += round_up((int64_t)bytes, 256);
      return r;
    };
    I.f[BF_X64] = items[i].x;
    I.f[BF_B64] = const_cast<void*>(items[i].b);
    I.f[BF_R64] = take(cb_spinor_bytes(g, LQCD_F64));
    I.f[BF_AX64] = take(cb_spinor_bytes(g, LQCD_F64));
    I.f[BF_MID64] = take(cb_spinor_bytes(g, LQCD_F64));
    I.f[BF_T1_64] = take(cb_spinor_bytes(g, LQCD_F64));
    I.f[BF_XS] = take(cb_spinor_bytes(g, VF));
    I.f[BF_RS] = take(cb_spinor_bytes(g, VF));
    I.f[BF_P] = take(cb_spinor_bytes(g, prm->sloppy_prec));
    I.f[BF_AP] = take(cb_spinor_bytes(g, prm->sloppy_prec));
    I.f[BF_MP] = take(cb_spinor_bytes(g, prm->sloppy_prec));
    I.f[BF_T1S] = take(cb_spinor_bytes(g, prm->sloppy_prec));
  }
  cudaError_t e = cudaMemcpyAsync(lay.inst, host, sizeof(BInst) * n, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return finish(cuda_fail(e, "batch: descriptor upload"), 0, 0);

  BatchSolver S;
  S.n = n;
  S.nsys = n;
  S.ctrl = lay.ctrl;
  S.sys = lay.sys;
  S.sloppy = prm->sloppy_prec;
  // the FP64 inner operator runs on the FP64 fields themselves, in their format
  S.sloppy_recon = prm->sloppy_prec == LQCD_F64 ? recon : prm->sloppy_recon;
  S.recon = recon;
  S.df = prm->sloppy_prec != LQCD_F64 && prm->update_prec == LQCD_F64_DF;
  memset(&S.base, 0, sizeof(S.base));
  S.base.inst = lay.inst;
  S.base.ninst = n;
  for (int t = 0; t < NTILES; t++) S.tiles_by_size[t] = tiles_by[t];
  S.set_tile(1);
  ReduceCtx rc;
  memset(&rc, 0, sizeof(rc));
  rc.partials = lay.partials;
  rc.counter = lay.counter;
  rc.sys = lay.sys;
  rc.ctrl = lay.ctrl;
  rc.nsys = n;
  S.base.red = rc;
  S.rc_init = rc;
  S.rc_init.fin = FIN_INIT;
  S.rc_init.tol2_rel = prm->tol * prm->tol;
  S.rc_init.delta2 = prm->sloppy_prec == LQCD_F64 ? 0.0 : prm->delta * prm->delta;
  S.rc_alpha = rc;
  S.rc_alpha.fin = FIN_ALPHA;
  S.rc_update = rc;
  S.rc_update.fin = FIN_UPDATE;
  S.rc_update.maxiter = prm->maxiter;
  S.rc_reliable = rc;
  S.rc_reliable.fin = FIN_RELIABLE;

  // persistent grid: autotuned tile size and resident blocks per SM for this batch shape
  int sms = 0;
  if ((st = sm_count(&sms))) return finish(st, 0, 0);
  const std::string skey = shape_key(n, geoms, S.sloppy, S.sloppy_recon, sms);
  const std::string tkey = "batch_tile " + skey.substr(10);  // "batch_hop " -> "batch_tile "
  int bps = 0, tile = 1;
  if (!tune_lookup(skey, &bps) || bps <= 0 || !tune_lookup(tkey, &tile) || tile < 0 || tile >= NTILES) {
    bps = 0;
    S.grid = (unsigned)std::min<int64_t>(std::min<int64_t>((int64_t)4 * sms, S.total_tiles), MAX_GRID);
    if ((st = S.init(s))) return finish(st, 0, 0);  // gives p a defined value to time the hop on
    if ((st = autotune_batch(S, sms, &tile, &bps, s))) return finish(st, 0, 0);
    tune_store(skey, bps);
    tune_store(tkey, tile);
  }
  S.set_tile(tile);
  S.grid = (unsigned)std::min<int64_t>(std::min<int64_t>((int64_t)bps * sms, S.total_tiles), MAX_GRID);

  std::vector<unsigned char> key;
  int dev = 0;
  cudaGetDevice(&dev);
  key_append(key, 2);  // batched solver
  key_append(key, dev);
  key_append(key, workspace);
  key_append(key, n);
  key_append(key, recon);
  key_append(key, prm->sloppy_prec);
  key_append(key, prm->sloppy_recon);
  key_append(key, prm->check_interval);
  key_append(key, prm->maxiter);
  key_append(key, S.grid);
  key_append(key, S.tile);
  key_append(key, (int)S.df);
  for (int i = 0; i < n; i++) {
    key_append(key, geoms[i].X);
    key_append(key, geoms[i].Y);
    key_append(key, geoms[i].Z);
    key_append(key, geoms[i].T);
  }
  lqcd_solver_params p2 = *prm;
  if (p2.check_interval <= 0) p2.check_interval = 16;
  Control ctrl;
  memset(&ctrl, 0, sizeof(ctrl));
  const int status = run_cg(S, p2, key, s, t0, &ctrl);
  SysState sys[MAX_BATCH];
  e = cudaMemcpyAsync(sys, lay.sys, sizeof(SysState) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return finish(status ? status : cuda_fail(e, "batch: state readback"), &ctrl, nullptr);
  return finish(status, &ctrl, sys);
}

}  // extern "C"
