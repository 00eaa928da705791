// Block conjugate gradient (O'Leary, Linear Algebra Appl. 29 (1980) 293) for
// N = n5 right-hand sides sharing one gauge field. The Grid paper lists CG
// (Sec. 4); block CG is its multi-RHS form: one Krylov space of block
// dimension N is shared by all right-hand sides.
//
//   R = B, P = R, S = R^dag R
//   repeat: Q = A P; G = P^dag Q; alpha = G^-1 S
//           X += P alpha; R -= Q alpha; S' = R^dag R; beta = S^-1 S'; P = R + P beta; S = S'
//
// (N x N complex matrices; ^dag is the block inner product over sites, spin
// and colour.) Precision follows the scalar solver: the operator and P, Q are
// sloppy (FP32 or FP16 storage), X_s and R_s are FP32, the Gram matrices are
// accumulated in FP64, and FP64 reliable updates recompute R = B - A X. A
// column whose FP64 residual meets the tolerance is frozen (its rows and
// columns drop out of alpha and beta and its search direction is zeroed),
// which keeps G and S well conditioned as columns converge. If a Cholesky
// factorisation still breaks down (linearly dependent columns) that step and
// the next beta fall back to per-column (independent CG) coefficients.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "cg_engine.h"
#include "cg_site.cuh"

namespace lqcd {

constexpr int BMAX = 16;          // largest block size N
constexpr int GRAM_BLOCK = 256;   // threads of the Gram kernel
constexpr int GRAM_GRID = 1024;   // persistent blocks of the Gram kernel

struct BlockState {
  cpx<double> S[BMAX * BMAX];   // R^dag R of the current iterate
  cpx<double> Sn[BMAX * BMAX];  // R^dag R after the update
  cpx<double> G[BMAX * BMAX];   // P^dag A P
  cpx<double> alpha[BMAX * BMAX];
  cpx<double> beta[BMAX * BMAX];
  double rr0[BMAX];             // |b_j|^2
  double maxrr[BMAX];           // max iterated |r_j|^2 since the last reliable update
  double tol2, delta2;
  int done[BMAX];
  int restart;                  // 1: the last alpha was per-column, so is the next beta
  int pad;
};

enum BFin { BF_S_INIT = 0, BF_ALPHA = 1, BF_UPDATE = 2, BF_RELIABLE = 3 };

struct BlockArgs {
  Geom g;
  int N;
  const void* u;  // Gram: left operand (format FU), right operand v (format FV)
  const void* v;
  cpx<double>* partials;  // [GRAM_GRID][N*N]
  unsigned int* counter;
  BlockState* st;
  Control* ctrl;
  int fin;
  int maxiter;
  int cond;
  cudaGraphConditionalHandle h_rel;
  double tol2, delta2;  // BF_S_INIT: tol^2 and delta^2
  // block axpy / p update fields
  void* xs;
  void* rs;
  void* p;
  const void* q;
  const Control* gate;
};

// ---------------------------------------------------------------- small dense algebra (one thread)

// Solve M X = Y for X on the active index set (Cholesky of the Hermitian positive
// definite M restricted to it). Entries of inactive rows/columns of X are zero.
// Returns false if a pivot is not positive (breakdown).
__device__ bool chol_solve(int N, const int* active, const cpx<double>* M, const cpx<double>* Y, cpx<double>* X) {
  int idx[BMAX];
  int n = 0;
  for (int i = 0; i < N; i++)
    if (active[i]) idx[n++] = i;
  cpx<double> L[BMAX * BMAX];
  double maxd = 0.0;
  for (int i = 0; i < n; i++) maxd = fmax(maxd, M[idx[i] * N + idx[i]].r);
  for (int j = 0; j < n; j++) {
    double d = M[idx[j] * N + idx[j]].r;
    for (int k = 0; k < j; k++) d -= L[j * BMAX + k].r * L[j * BMAX + k].r + L[j * BMAX + k].i * L[j * BMAX + k].i;
    if (!(d > 1e-14 * maxd) || !isfinite(d)) return false;
    const double ljj = sqrt(d);
    L[j * BMAX + j] = mk(ljj, 0.0);
    for (int i = j + 1; i < n; i++) {
      cpx<double> s = M[idx[i] * N + idx[j]];
      for (int k = 0; k < j; k++) s = s - cmul(L[i * BMAX + k], conj(L[j * BMAX + k]));
      L[i * BMAX + j] = (1.0 / ljj) * s;
    }
  }
  for (int i = 0; i < N * N; i++) X[i] = mk(0.0, 0.0);
  for (int c = 0; c < N; c++) {
    if (!active[c]) continue;
    cpx<double> z[BMAX];
    for (int i = 0; i < n; i++) {  // L z = y
      cpx<double> s = Y[idx[i] * N + c];
      for (int k = 0; k < i; k++) s = s - cmul(L[i * BMAX + k], z[k]);
      z[i] = (1.0 / L[i * BMAX + i].r) * s;
    }
    for (int i = n - 1; i >= 0; i--) {  // L^dag x = z
      cpx<double> s = z[i];
      for (int k = i + 1; k < n; k++) s = s - cmul(conj(L[k * BMAX + i]), X[idx[k] * N + c]);
      X[idx[i] * N + c] = (1.0 / L[i * BMAX + i].r) * s;
    }
  }
  return true;
}

// Per-column fallback X = diag(Y) / diag(M) (independent CG steps), used when
// the block factorisation breaks down (e.g. linearly dependent columns).
__device__ void diag_solve(int N, const int* active, const cpx<double>* M, const cpx<double>* Y, cpx<double>* X) {
  for (int i = 0; i < N * N; i++) X[i] = mk(0.0, 0.0);
  for (int j = 0; j < N; j++) {
    const double m = M[j * N + j].r;
    if (active[j] && m > 0.0 && isfinite(m)) X[j * N + j] = mk(Y[j * N + j].r / m, 0.0);
  }
}

__device__ void block_finalize(const BlockArgs& a, const cpx<double>* M) {
  BlockState& s = *a.st;
  Control& c = *a.ctrl;
  const int N = a.N;
  int active[BMAX];
  for (int j = 0; j < N; j++) active[j] = !s.done[j];
  switch (a.fin) {
    case BF_S_INIT: {
      int n_done = 0;
      bool bad = false;
      for (int i = 0; i < N * N; i++) s.S[i] = M[i];
      for (int j = 0; j < N; j++) {
        const double rr = M[j * N + j].r;
        s.rr0[j] = s.maxrr[j] = rr;
        s.done[j] = rr == 0.0 ? 1 : 0;
        if (!isfinite(rr)) bad = true;
        n_done += s.done[j];
      }
      s.tol2 = a.tol2;
      s.delta2 = a.delta2;
      s.restart = 0;
      c.nsys = N;
      c.n_done = n_done;
      c.iter = 0;
      c.n_reliable = 0;
      c.chunk_left = 0;
      c.reason = bad ? REASON_NAN : 0;
      c.active = (!bad && n_done < N) ? 1 : 0;
    } break;
    case BF_ALPHA:
      for (int i = 0; i < N * N; i++) s.G[i] = M[i];
      if (!chol_solve(N, active, s.G, s.S, s.alpha)) {
        diag_solve(N, active, s.G, s.S, s.alpha);  // independent steps this iteration
        s.restart = 1;                             // and a diagonal beta after it
      }
      break;
    case BF_UPDATE: {
      for (int i = 0; i < N * N; i++) s.Sn[i] = M[i];
      int reason = 0;
      bool conv = true;
      for (int j = 0; j < N; j++) {
        if (s.done[j]) continue;
        const double rr = M[j * N + j].r;
        if (!isfinite(rr)) reason |= REASON_NAN;
        if (rr > s.tol2 * s.rr0[j]) conv = false;
        if (rr <= s.delta2 * s.maxrr[j]) reason |= REASON_RELIABLE;
      }
      if (conv) reason |= REASON_CONVERGED;
      c.iter += 1;
      const bool at_cap = a.maxiter > 0 && c.iter >= a.maxiter;
      if (reason & REASON_NAN) {
        c.reason |= REASON_NAN;
        c.active = 0;
      } else if (reason || at_cap) {
        c.reason |= reason;
        if (a.cond) cudaGraphSetConditional(a.h_rel, 1);
        else c.active = 0;
      } else {
        if (s.restart || !chol_solve(N, active, s.S, s.Sn, s.beta)) diag_solve(N, active, s.S, s.Sn, s.beta);
        s.restart = 0;
        for (int i = 0; i < N * N; i++) s.S[i] = s.Sn[i];
        for (int j = 0; j < N; j++) s.maxrr[j] = fmax(s.maxrr[j], M[j * N + j].r);
      }
    } break;
    case BF_RELIABLE: {
      int n_done = 0;
      bool bad = false;
      for (int j = 0; j < N; j++) {
        const double rr = M[j * N + j].r;
        if (!isfinite(rr)) bad = true;
        if (!s.done[j] && rr <= s.tol2 * s.rr0[j]) s.done[j] = 1;
        n_done += s.done[j];
      }
      for (int j = 0; j < N; j++) active[j] = !s.done[j];
      if (s.restart || !chol_solve(N, active, s.S, M, s.beta)) diag_solve(N, active, s.S, M, s.beta);
      s.restart = 0;
      for (int i = 0; i < N * N; i++) s.S[i] = M[i];
      for (int j = 0; j < N; j++) s.maxrr[j] = M[j * N + j].r;
      c.n_done = n_done;
      c.n_reliable += 1;
      c.reason = bad ? REASON_NAN : 0;
      c.active = (!bad && n_done < N) ? 1 : 0;
    } break;
  }
}

// ---------------------------------------------------------------- Gram matrix U^dag V

// Staging type of the Gram kernel: FP64 operands are staged and multiplied in
// FP64 (the plain FP64 block solve needs FP64-accurate alpha and beta), the
// sloppy ones in FP32 with FP64 accumulation across sites.
template <typename T> struct Stage;
template <> struct Stage<double> {
  using V2 = double2;
  static constexpr int SB = 4;
  static __device__ __forceinline__ V2 mk2(double x, double y) { return make_double2(x, y); }
};
template <> struct Stage<float> {
  using V2 = float2;
  static constexpr int SB = 8;
  static __device__ __forceinline__ V2 mk2(float x, float y) { return make_float2(x, y); }
};

template <int FU, int FV>
__global__ void __launch_bounds__(GRAM_BLOCK) k_gram(const BlockArgs a) {
  using TU = typename PrecTraits<FU>::real;
  using TV = typename PrecTraits<FV>::real;
  using TS = TU;  // FU and FV share a precision class
  using ST = Stage<TS>;
  using V2 = typename ST::V2;
  constexpr int SB = ST::SB;  // sites staged per pass
  if (gate_closed(a.gate)) return;
  __shared__ V2 su[SB][BMAX][12];
  __shared__ V2 sv[SB][BMAX][12];
  __shared__ double red[GRAM_BLOCK];
  __shared__ int is_last;
  const int N = a.N, NN = N * N;
  const int tid = threadIdx.x;
  const int pa = tid / N, pb = tid - (tid / N) * N;  // (row, column) of M handled by this thread
  double accr = 0.0, acci = 0.0;
  const int64_t nsite4 = a.g.Vh;
  for (int64_t s0 = (int64_t)blockIdx.x * SB; s0 < nsite4; s0 += (int64_t)gridDim.x * SB) {
    // stage SB sites x N columns of U and V (one spinor per thread)
    for (int e = tid; e < SB * N; e += GRAM_BLOCK) {
      const int ls = e / N, col = e - (e / N) * N;
      const int64_t site = s0 + ls;
      if (site < nsite4) {
        const int64_t j = site * a.g.n5 + col;
        Spinor<TU> x;
        SpinorIO<FU>::load(a.u, a.g.sstride, j, x);
        Spinor<TV> y;
        SpinorIO<FV>::load(a.v, a.g.sstride, j, y);
#pragma unroll
        for (int k = 0; k < 12; k++) {
          su[ls][col][k] = ST::mk2((TS)x.v[k].r, (TS)x.v[k].i);
          sv[ls][col][k] = ST::mk2((TS)y.v[k].r, (TS)y.v[k].i);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 12; k++) su[ls][col][k] = sv[ls][col][k] = ST::mk2(TS(0), TS(0));
      }
    }
    __syncthreads();
    if (tid < NN) {
      TS r = TS(0), im = TS(0);
      for (int ls = 0; ls < SB; ls++)
#pragma unroll
        for (int k = 0; k < 12; k++) {  // conj(u) v
          const V2 p = su[ls][pa][k], q = sv[ls][pb][k];
          r = fma(p.x, q.x, fma(p.y, q.y, r));
          im = fma(p.x, q.y, fma(-p.y, q.x, im));
        }
      accr += (double)r;
      acci += (double)im;
    }
    __syncthreads();
  }
  if (tid < NN) {
    a.partials[(int64_t)blockIdx.x * NN + tid] = mk(accr, acci);
    __threadfence();  // the writers alone fence, before the ticket below
  }
  __syncthreads();
  if (tid == 0) is_last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  __shared__ cpx<double> M[BMAX * BMAX];
  for (int e = 0; e < NN; e++) {
    double sr = 0.0, si = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += GRAM_BLOCK) {
      const double2 w = __ldcg(reinterpret_cast<const double2*>(a.partials + (int64_t)b * NN + e));
      sr += w.x;
      si += w.y;
    }
    red[tid] = sr;
    __syncthreads();
    for (int w = GRAM_BLOCK / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    if (tid == 0) M[e].r = red[0];
    __syncthreads();
    red[tid] = si;
    __syncthreads();
    for (int w = GRAM_BLOCK / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    if (tid == 0) M[e].i = red[0];
    __syncthreads();
  }
  if (tid == 0) {
    block_finalize(a, M);
    *a.counter = 0u;
  }
}

// ---------------------------------------------------------------- block updates

// x_s += P alpha; r_s -= Q alpha (threads of one site in one block: block = N * (128 / N))
template <int VF, int SF>
__global__ void k_block_update(const BlockArgs a) {
  using TV = typename PrecTraits<VF>::real;
  using TS = typename PrecTraits<SF>::real;
  if (gate_closed(a.gate)) return;
  const int N = a.N;
  __shared__ cpx<TV> al[BMAX * BMAX];  // alpha in the precision of the iterated vectors
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) al[e] = mk((TV)a.st->alpha[e].r, (TV)a.st->alpha[e].i);
  __syncthreads();
  const int spb = blockDim.x / N;
  const int ls = threadIdx.x / N, col = threadIdx.x - ls * N;
  const int64_t site = (int64_t)blockIdx.x * spb + ls;
  if (ls >= spb || site >= a.g.Vh) return;
  const int64_t base = site * a.g.n5;
  Spinor<TV> x, r;
  SpinorIO<VF>::load(a.xs, a.g.sstride, base + col, x);
  SpinorIO<VF>::load(a.rs, a.g.sstride, base + col, r);
  for (int k5 = 0; k5 < N; k5++) {
    const cpx<TV> cc = al[k5 * N + col];  // alpha[k5][col]
    if (cc.r == TV(0) && cc.i == TV(0)) continue;
    Spinor<TS> p, q;
    SpinorIO<SF>::load(a.p, a.g.sstride, base + k5, p);
    SpinorIO<SF>::load(a.q, a.g.sstride, base + k5, q);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      x.v[k] = cmadd(x.v[k], mk((TV)p.v[k].r, (TV)p.v[k].i), cc);
      r.v[k] = cmadd(r.v[k], mk((TV)-q.v[k].r, (TV)-q.v[k].i), cc);
    }
  }
  SpinorIO<VF>::store(a.xs, a.g.sstride, base + col, x);
  SpinorIO<VF>::store(a.rs, a.g.sstride, base + col, r);
}

// P = R_s + P beta (in place: every column of a site is read before any is written); frozen columns get P = 0
template <int VF, int SF>
__global__ void k_block_pupdate(const BlockArgs a) {
  using TV = typename PrecTraits<VF>::real;
  using TS = typename PrecTraits<SF>::real;
  if (gate_closed(a.gate)) return;
  const int N = a.N;
  __shared__ cpx<TS> be[BMAX * BMAX];  // beta in the precision of the search directions
  __shared__ int dn[BMAX];
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) be[e] = mk((TS)a.st->beta[e].r, (TS)a.st->beta[e].i);
  for (int e = threadIdx.x; e < N; e += blockDim.x) dn[e] = a.st->done[e];
  __syncthreads();
  const int spb = blockDim.x / N;
  const int ls = threadIdx.x / N, col = threadIdx.x - ls * N;
  const int64_t site = (int64_t)blockIdx.x * spb + ls;
  const bool valid = ls < spb && site < a.g.Vh;
  const int64_t base = site * a.g.n5;
  Spinor<TS> out;
  if (valid) {
    Spinor<TV> r;
    SpinorIO<VF>::load(a.rs, a.g.sstride, base + col, r);
#pragma unroll
    for (int k = 0; k < 12; k++) out.v[k] = mk((TS)r.v[k].r, (TS)r.v[k].i);
    for (int k5 = 0; k5 < N; k5++) {
      const cpx<TS> cc = be[k5 * N + col];  // beta[k5][col]
      if (cc.r == TS(0) && cc.i == TS(0)) continue;
      Spinor<TS> p;
      SpinorIO<SF>::load(a.p, a.g.sstride, base + k5, p);
#pragma unroll
      for (int k = 0; k < 12; k++) out.v[k] = cmadd(out.v[k], p.v[k], cc);
    }
    if (dn[col]) zero(out);
  }
  __syncthreads();  // all old columns of the block's sites are read
  if (valid) SpinorIO<SF>::store(const_cast<void*>(a.p), a.g.sstride, base + col, out);
}

// r = b - A x (FP64), r_s = r
template <int VF>
__global__ void k_block_residual(const Geom g, const double* b, const double* ax, double* r, void* rs) {
  const int64_t j = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (j >= g.nsites) return;
  residual_site<VF>(g, j, b, ax, r, rs);
}

// ---------------------------------------------------------------- engine

struct BlockWorkspace {
  Control* ctrl;
  SysState* sys;
  double* partials;  // scalar reductions (k_init): [nsys][blocks]
  unsigned int* counter;
  BlockState* st;
  cpx<double>* gpart;  // [GRAM_GRID][N*N]
  unsigned int* gcounter;
  double *r64, *ax64, *mid64;
  void* t1_64;
  void *rs, *xs, *p, *q, *mp, *t1s;
  size_t total;
};

static BlockWorkspace block_carve(void* base, const Geom& g, int sloppy) {
  BlockWorkspace w;
  memset(&w, 0, sizeof(w));
  size_t o = 0;
  char* b = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> void* {
    void* r = b ? b + o : nullptr;
    o += round_up((int64_t)bytes, 256);
    return r;
  };
  const int VF = sloppy == LQCD_F64 ? LQCD_F64 : LQCD_F32;
  w.ctrl = (Control*)take(sizeof(Control));
  w.sys = (SysState*)take(sizeof(SysState) * MAX_SYS);
  w.partials = (double*)take(sizeof(double) * g.n5 * ((g.nsites + 63) / 64));
  w.counter = (unsigned int*)take(64);
  w.st = (BlockState*)take(sizeof(BlockState));
  w.gpart = (cpx<double>*)take(sizeof(cpx<double>) * GRAM_GRID * g.n5 * g.n5);
  w.gcounter = (unsigned int*)take(64);
  w.r64 = (double*)take(cb_spinor_bytes(g, LQCD_F64));
  w.ax64 = (double*)take(cb_spinor_bytes(g, LQCD_F64));
  w.mid64 = (double*)take(cb_spinor_bytes(g, LQCD_F64));
  w.t1_64 = take(cb_spinor_bytes(g, LQCD_F64));
  w.rs = take(cb_spinor_bytes(g, VF));
  w.xs = take(cb_spinor_bytes(g, VF));
  w.p = take(cb_spinor_bytes(g, sloppy));
  w.q = take(cb_spinor_bytes(g, sloppy));
  w.mp = take(cb_spinor_bytes(g, sloppy));
  w.t1s = take(cb_spinor_bytes(g, sloppy));
  w.total = o;
  return w;
}

template <int FU, int FV>
static void launch_gram_t(const BlockArgs& a, cudaStream_t s) {
  const unsigned grid = (unsigned)std::min<int64_t>(GRAM_GRID, (a.g.Vh + 3) / 4);
  k_gram<FU, FV><<<grid, GRAM_BLOCK, 0, s>>>(a);
}

struct BlockSolver : CgEngine {
  Geom g;
  int N, sloppy, VF;
  lqcd_operator op64, ops;
  const void* gauge64;
  const void* gauge_s;
  BlockWorkspace w;
  BlockArgs ba;
  double* x64;
  const double* b64;
  double tol2, delta2;
  int maxiter;

  BlockArgs args(int fin, const void* u, const void* v, const Control* gate) const {
    BlockArgs a = ba;
    a.fin = fin;
    a.u = u;
    a.v = v;
    a.gate = gate;
    return a;
  }
  int gram(int fu, int fv, const BlockArgs& a, cudaStream_t s) {
    // formats: FP64 x FP64, VF x VF, SF x SF
    if (fu == LQCD_F64) launch_gram_t<LQCD_F64, LQCD_F64>(a, s);
    else if (fu == LQCD_F32) launch_gram_t<LQCD_F32, LQCD_F32>(a, s);
    else launch_gram_t<LQCD_F16, LQCD_F16>(a, s);
    (void)fv;
    return after_launch("k_gram");
  }
  unsigned upd_grid(int* threads) const {
    const int spb = std::max(1, 128 / N);
    *threads = spb * N;
    return (unsigned)((g.Vh + spb - 1) / spb);
  }
  int init(cudaStream_t s) override;
  int head(cudaStream_t s, int cond, cudaGraphConditionalHandle h_rel, cudaGraphConditionalHandle) override;
  int tail(cudaStream_t s) override;
  int reliable(cudaStream_t s) override;
};

// r = b, r_s = b, p = b, x_s = 0, x = 0 for every column
template <int VF, int SF>
__global__ void k_block_init(const Geom g, const double* b, double* r, double* x, void* rs, void* xs, void* p) {
  const int64_t j = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (j >= g.nsites) return;
  init_site<VF, SF>(g, j, b, r, x, rs, xs, p);
}

// x += x_s (FP64); x_s = 0
template <int VF>
__global__ void k_block_accumulate(const Geom g, double* x, void* xs) {
  const int64_t j = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (j >= g.nsites) return;
  accumulate_site<VF>(g, j, x, xs);
}

#define LQCD_VS_DISPATCH(VF, SF, CALL)                               \
  do {                                                               \
    if (sloppy == LQCD_F64) { constexpr int VF = LQCD_F64, SF = LQCD_F64; (void)SF; CALL; } \
    else if (sloppy == LQCD_F32) { constexpr int VF = LQCD_F32, SF = LQCD_F32; (void)SF; CALL; } \
    else { constexpr int VF = LQCD_F32, SF = LQCD_F16; (void)SF; CALL; }       \
  } while (0)

int BlockSolver::init(cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(w.gcounter, 0, 64, s);
  if (e != cudaSuccess) return cuda_fail(e, "block cg: memset");
  const unsigned grid = (unsigned)((g.nsites + 127) / 128);
  LQCD_VS_DISPATCH(VF_, SF_, (k_block_init<VF_, SF_><<<grid, 128, 0, s>>>(g, b64, w.r64, x64, w.rs, w.xs, w.p)));
  int st = after_launch("k_block_init");
  if (st) return st;
  return gram(LQCD_F64, LQCD_F64, args(BF_S_INIT, w.r64, w.r64, nullptr), s);
}

int BlockSolver::head(cudaStream_t s, int cond, cudaGraphConditionalHandle h_rel, cudaGraphConditionalHandle) {
  OpCtx cs{g, ops, gauge_s};
  int st = op_apply(cs, w.mp, w.p, LQCD_EVEN, 0, w.t1s, nullptr, nullptr, ctrl, s);
  if (st) return st;
  if ((st = op_apply(cs, w.q, w.mp, LQCD_EVEN, 1, w.t1s, nullptr, nullptr, ctrl, s))) return st;
  if ((st = gram(sloppy, sloppy, args(BF_ALPHA, w.p, w.q, ctrl), s))) return st;
  int threads;
  const unsigned grid = upd_grid(&threads);
  BlockArgs a = args(BF_ALPHA, nullptr, nullptr, ctrl);
  LQCD_VS_DISPATCH(VF_, SF_, (k_block_update<VF_, SF_><<<grid, threads, 0, s>>>(a)));
  if ((st = after_launch("k_block_update"))) return st;
  BlockArgs u = args(BF_UPDATE, w.rs, w.rs, ctrl);
  u.cond = cond;
  u.h_rel = h_rel;
  return gram(VF, VF, u, s);
}

int BlockSolver::tail(cudaStream_t s) {
  int threads;
  const unsigned grid = upd_grid(&threads);
  BlockArgs a = args(BF_ALPHA, nullptr, nullptr, ctrl);
  LQCD_VS_DISPATCH(VF_, SF_, (k_block_pupdate<VF_, SF_><<<grid, threads, 0, s>>>(a)));
  return after_launch("k_block_pupdate");
}

int BlockSolver::reliable(cudaStream_t s) {
  const unsigned grid = (unsigned)((g.nsites + 127) / 128);
  LQCD_VS_DISPATCH(VF_, SF_, (k_block_accumulate<VF_><<<grid, 128, 0, s>>>(g, x64, w.xs)));
  int st = after_launch("k_block_accumulate");
  if (st) return st;
  OpCtx c64{g, op64, gauge64};
  if ((st = op_apply(c64, w.mid64, x64, LQCD_EVEN, 0, w.t1_64, nullptr, nullptr, nullptr, s))) return st;
  if ((st = op_apply(c64, w.ax64, w.mid64, LQCD_EVEN, 1, w.t1_64, nullptr, nullptr, nullptr, s))) return st;
  LQCD_VS_DISPATCH(VF_, SF_, (k_block_residual<VF_><<<grid, 128, 0, s>>>(g, b64, w.ax64, w.r64, w.rs)));
  if ((st = after_launch("k_block_residual"))) return st;
  return gram(LQCD_F64, LQCD_F64, args(BF_RELIABLE, w.r64, w.r64, nullptr), s);
}
#undef LQCD_VS_DISPATCH

static int block_validate(const lqcd_lattice* lat, const lqcd_operator* op, const lqcd_solver_params* p, Geom* g) {
  int st = make_geom(lat, g);
  if (st) return st;
  if ((st = check_operator(op, *g))) return st;
  if (!p) return fail(LQCD_ERR_ARG, "block cg: null params");
  if (op->kind != LQCD_WILSON || op->gparity)
    return fail(LQCD_ERR_UNSUPPORTED, "block cg: Wilson operator without G-parity only");
  if (op->prec != LQCD_F64) return fail(LQCD_ERR_ARG, "block cg: x, b and gauge must be LQCD_F64 (op->prec)");
  if (g->n5 > BMAX) return fail(LQCD_ERR_ARG, "block cg: %d right-hand sides exceed %d", g->n5, BMAX);
  if (p->sloppy_prec != LQCD_F64 && p->sloppy_prec != LQCD_F32 && p->sloppy_prec != LQCD_F16)
    return fail(LQCD_ERR_ARG, "block cg: bad sloppy precision %d", p->sloppy_prec);
  if (p->sloppy_recon != 18 && p->sloppy_recon != 12) return fail(LQCD_ERR_ARG, "block cg: bad sloppy recon");
  if (!(p->tol > 0.0) || p->maxiter < 1) return fail(LQCD_ERR_ARG, "block cg: tol must be > 0 and maxiter >= 1");
  if (p->delta < 0.0 || p->delta >= 1.0) return fail(LQCD_ERR_ARG, "block cg: delta must be in [0, 1)");
  return LQCD_OK;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

size_t lqcd_block_cg_workspace_bytes(const lqcd_lattice* lat, const lqcd_operator* op,
                                     const lqcd_solver_params* params) {
  Geom g;
  if (block_validate(lat, op, params, &g)) return 0;
  return block_carve(nullptr, g, params->sloppy_prec).total;
}

int lqcd_block_cg_solve(void* x, const void* b, const void* gauge, const void* gauge_sloppy, const lqcd_lattice* lat,
                        const lqcd_operator* op, const lqcd_solver_params* prm, lqcd_solve_info* info,
                        void* workspace, size_t workspace_bytes, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  lqcd_solve_info local;
  lqcd_solve_info* inf = info ? info : &local;
  memset(inf, 0, sizeof(*inf));
  auto finish = [&](int status) {
    inf->status = status;
    inf->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return status;
  };
  BlockSolver S;
  int st = block_validate(lat, op, prm, &S.g);
  if (st) return finish(st);
  if (!x || !b || !gauge || !workspace || ((uintptr_t)workspace & 255) || ((uintptr_t)x & 15) ||
      ((uintptr_t)b & 15))
    return finish(fail(LQCD_ERR_ARG, "block cg: null or misaligned pointer (workspace needs 256-byte alignment)"));
  if (prm->sloppy_prec == LQCD_F64) gauge_sloppy = gauge;  // the FP64 field serves both
  if (!gauge_sloppy) return finish(fail(LQCD_ERR_ARG, "block cg: gauge_sloppy required"));
  S.w = block_carve(workspace, S.g, prm->sloppy_prec);
  if (workspace_bytes < S.w.total)
    return finish(fail(LQCD_ERR_WORKSPACE, "block cg: workspace %zu < %zu bytes", workspace_bytes, S.w.total));
  S.N = S.g.n5;
  S.nsys = S.N;
  S.ctrl = S.w.ctrl;
  S.sys = S.w.sys;
  S.sloppy = prm->sloppy_prec;
  S.VF = S.sloppy == LQCD_F64 ? LQCD_F64 : LQCD_F32;
  S.op64 = *op;
  S.ops = *op;
  S.ops.prec = prm->sloppy_prec;
  // the FP64 inner operator runs on the FP64 field itself, in that field's format
  S.ops.recon = prm->sloppy_prec == LQCD_F64 ? op->recon : prm->sloppy_recon;
  S.gauge64 = gauge;
  S.gauge_s = gauge_sloppy;
  S.x64 = (double*)x;
  S.b64 = (const double*)b;
  memset(&S.ba, 0, sizeof(S.ba));
  S.ba.g = S.g;
  S.ba.N = S.N;
  S.ba.partials = S.w.gpart;
  S.ba.counter = S.w.gcounter;
  S.ba.st = S.w.st;
  S.ba.ctrl = S.w.ctrl;
  S.ba.maxiter = prm->maxiter;
  S.ba.tol2 = prm->tol * prm->tol;
  S.ba.delta2 = prm->sloppy_prec == LQCD_F64 ? 0.0 : prm->delta * prm->delta;
  S.ba.xs = S.w.xs;
  S.ba.rs = S.w.rs;
  S.ba.p = S.w.p;
  S.ba.q = S.w.q;
  lqcd_solver_params p2 = *prm;
  if (p2.check_interval <= 0) p2.check_interval = 16;

  std::vector<unsigned char> key;
  int dev = 0;
  cudaGetDevice(&dev);
  key_append(key, 3);  // block solver
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
  key_append(key, op->mass);
  key_append(key, op->recon);
  key_append(key, prm->sloppy_prec);
  key_append(key, prm->sloppy_recon);
  key_append(key, p2.check_interval);
  key_append(key, prm->maxiter);

  Control ctrl;
  memset(&ctrl, 0, sizeof(ctrl));
  int status = run_cg(S, p2, key, (cudaStream_t)stream, t0, &ctrl);
  BlockState bs;
  cudaError_t e = cudaMemcpyAsync(&bs, S.w.st, sizeof(BlockState), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess && status == LQCD_OK) status = cuda_fail(e, "block cg: state readback");
  double worst = 0.0;
  for (int j = 0; j < S.N && e == cudaSuccess; j++) {
    const double rel = bs.rr0[j] > 0 ? std::sqrt(bs.S[j * S.N + j].r / bs.rr0[j]) : 0.0;
    if (rel > worst || std::isnan(rel)) worst = rel;
  }
  inf->iterations = ctrl.iter;
  inf->reliable_updates = ctrl.n_reliable;
  inf->true_rel_residual = worst;
  return finish(status);
}

}  // extern "C"
