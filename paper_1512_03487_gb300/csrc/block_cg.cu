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
// sloppy (FP32 or FP16 storage), X_s and R_s are FP32, the Gram matrices'
// partial sums meet in FP64, and FP64 reliable updates recompute R = B - A X. A
// column whose FP64 residual meets the tolerance is frozen (its rows and
// columns drop out of alpha and beta and its search direction is zeroed),
// which keeps G and S well conditioned as columns converge. If a Cholesky
// factorisation still breaks down (linearly dependent columns) that step and
// the next beta fall back to per-column (independent CG) coefficients.
// With update_prec = LQCD_F64_DF the reliable updates' A X runs in double-float
// arithmetic on the FP64 fields. The Gram matrices of FP64 fields are summed in
// double-float arithmetic in the plain FP64 solve and in FP32 in a mixed one
// (they steer the sloppy recurrence; convergence is a sum of squares).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "cg_engine.h"
#include "cg_site.cuh"

namespace lqcd {

constexpr int BMAX = 16;          // largest block size N
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

// ---------------------------------------------------------------- small dense algebra (one warp)

// Solve M X = Y for X on the active index set (Cholesky of the Hermitian positive
// definite M restricted to it), all 32 lanes of one warp together: the
// factorisation column by column (lane 0 the pivot, the lanes the rows below
// it), then one lane per right-hand-side column for the two triangular solves.
// Entries of inactive rows/columns of X are zero. Returns false (on every lane)
// if a pivot is not positive (breakdown). L: BMAX x BMAX shared scratch.
__device__ bool chol_solve_warp(int N, const int* active, const cpx<double>* M, const cpx<double>* Y, cpx<double>* X,
                                cpx<double>* L) {
  const int lane = threadIdx.x & 31;
  int idx[BMAX];
  int n = 0;
  for (int i = 0; i < N; i++)
    if (active[i]) idx[n++] = i;
  double maxd = 0.0;
  for (int i = 0; i < n; i++) maxd = fmax(maxd, M[idx[i] * N + idx[i]].r);
  for (int j = 0; j < n; j++) {
    int ok = 1;
    if (lane == 0) {
      double d = M[idx[j] * N + idx[j]].r;
      for (int k = 0; k < j; k++) d -= L[j * BMAX + k].r * L[j * BMAX + k].r + L[j * BMAX + k].i * L[j * BMAX + k].i;
      ok = (d > 1e-14 * maxd) && isfinite(d);
      L[j * BMAX + j] = mk(ok ? sqrt(d) : 1.0, 0.0);
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    if (!ok) return false;
    const double ljj = L[j * BMAX + j].r;
    const int i = j + 1 + lane;
    if (i < n) {
      cpx<double> t = M[idx[i] * N + idx[j]];
      for (int k = 0; k < j; k++) t = t - cmul(L[i * BMAX + k], conj(L[j * BMAX + k]));
      L[i * BMAX + j] = (1.0 / ljj) * t;
    }
    __syncwarp();
  }
  for (int e = lane; e < N * N; e += 32) X[e] = mk(0.0, 0.0);
  __syncwarp();
  const int c = lane;
  if (c < N && active[c]) {
    cpx<double> z[BMAX];
    for (int i = 0; i < n; i++) {  // L z = y
      cpx<double> t = Y[idx[i] * N + c];
      for (int k = 0; k < i; k++) t = t - cmul(L[i * BMAX + k], z[k]);
      z[i] = (1.0 / L[i * BMAX + i].r) * t;
    }
    for (int i = n - 1; i >= 0; i--) {  // L^dag x = z
      cpx<double> t = z[i];
      for (int k = i + 1; k < n; k++) t = t - cmul(conj(L[k * BMAX + i]), X[idx[k] * N + c]);
      X[idx[i] * N + c] = (1.0 / L[i * BMAX + i].r) * t;
    }
  }
  __syncwarp();
  return true;
}

// Per-column fallback X = diag(Y) / diag(M) (independent CG steps), used when
// the block factorisation breaks down (e.g. linearly dependent columns). One lane.
__device__ void diag_solve(int N, const int* active, const cpx<double>* M, const cpx<double>* Y, cpx<double>* X) {
  for (int i = 0; i < N * N; i++) X[i] = mk(0.0, 0.0);
  for (int j = 0; j < N; j++) {
    const double m = M[j * N + j].r;
    if (active[j] && m > 0.0 && isfinite(m)) X[j * N + j] = mk(Y[j * N + j].r / m, 0.0);
  }
}

// The Gram kernel's finaliser, run by the 32 lanes of one warp of its last block:
// the bookkeeping on lane 0, the dense solves on the whole warp (chol_solve_warp).
// M: the totals (shared memory); L: shared scratch.
__device__ void block_finalize(const BlockArgs& a, const cpx<double>* M, cpx<double>* L) {
  BlockState& s = *a.st;
  Control& c = *a.ctrl;
  const int N = a.N, NN = N * N;
  const int lane = threadIdx.x & 31;
  int active[BMAX];
  for (int j = 0; j < N; j++) active[j] = !s.done[j];
  switch (a.fin) {
    case BF_S_INIT: {
      if (lane == 0) {
        int n_done = 0;
        bool bad = false;
        for (int i = 0; i < NN; i++) s.S[i] = M[i];
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
      }
    } break;
    case BF_ALPHA: {
      for (int i = lane; i < NN; i += 32) s.G[i] = M[i];
      __syncwarp();
      const bool ok = chol_solve_warp(N, active, s.G, s.S, s.alpha, L);
      if (!ok && lane == 0) {
        diag_solve(N, active, s.G, s.S, s.alpha);  // independent steps this iteration
        s.restart = 1;                             // and a diagonal beta after it
      }
    } break;
    case BF_UPDATE: {
      for (int i = lane; i < NN; i += 32) s.Sn[i] = M[i];
      int go = 0;
      if (lane == 0) {
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
          go = 1;
        }
      }
      go = __shfl_sync(0xffffffffu, go, 0);
      __syncwarp();
      if (go) {
        const bool ok = !s.restart && chol_solve_warp(N, active, s.S, s.Sn, s.beta, L);
        if (lane == 0) {
          if (!ok) diag_solve(N, active, s.S, s.Sn, s.beta);
          s.restart = 0;
          for (int i = 0; i < NN; i++) s.S[i] = s.Sn[i];
          for (int j = 0; j < N; j++) s.maxrr[j] = fmax(s.maxrr[j], M[j * N + j].r);
        }
      }
    } break;
    case BF_RELIABLE: {
      int n_done = 0;
      bool bad = false;
      if (lane == 0) {
        for (int j = 0; j < N; j++) {
          const double rr = M[j * N + j].r;
          if (!isfinite(rr)) bad = true;
          if (!s.done[j] && rr <= s.tol2 * s.rr0[j]) s.done[j] = 1;
          n_done += s.done[j];
        }
      }
      __syncwarp();
      for (int j = 0; j < N; j++) active[j] = !s.done[j];
      const bool ok = !s.restart && chol_solve_warp(N, active, s.S, M, s.beta, L);
      if (lane == 0) {
        if (!ok) diag_solve(N, active, s.S, M, s.beta);
        s.restart = 0;
        for (int i = 0; i < NN; i++) s.S[i] = M[i];
        for (int j = 0; j < N; j++) s.maxrr[j] = M[j * N + j].r;
        c.n_done = n_done;
        c.n_reliable += 1;
        c.reason = bad ? REASON_NAN : 0;
        c.active = (!bad && n_done < N) ? 1 : 0;
      }
    } break;
  }
}

// ---------------------------------------------------------------- Gram matrix U^dag V

// M[a][b] = sum over sites s and spin-colour k of conj(u[s][a][k]) v[s][b][k]
// (a, b < N; column c of site s is field index s N + c). A block stages SB
// sites x N columns of u and v in shared memory per pass, then each thread
// accumulates a TT x TT tile of M (NT x NT tiles, NT = ceil(N / TT) <= 4) for
// one staged site, so every shared-memory load feeds TT complex multiply-adds
// and the block's NT^2 SB threads all compute. Sloppy operands (FP32 / FP16
// storage) are multiplied and summed in FP32 per thread (its sites within the
// block: a few hundred terms, like the scalar solver's warp sums), FP64 ones in
// double-float arithmetic (FP64-accurate products and sums on the FP32 pipe:
// GB300's FP64 rate is a sixty-fourth of it); the threads' sums meet in FP64.
template <typename T> struct GramArith;
template <> struct GramArith<float> {
  using A = float;   // arithmetic
  using S2 = float2; // staged complex
  static __device__ __forceinline__ S2 stage(float r, float i) { return make_float2(r, i); }
  static __device__ __forceinline__ A re(S2 c) { return c.x; }
  static __device__ __forceinline__ A im(S2 c) { return c.y; }
  static __device__ __forceinline__ double to_double(A x) { return (double)x; }
};
template <> struct GramArith<double> {
  using A = dfl;
  using S2 = double2;
  static __device__ __forceinline__ S2 stage(double r, double i) { return make_double2(r, i); }
  static __device__ __forceinline__ A re(S2 c) { return df_split(c.x); }
  static __device__ __forceinline__ A im(S2 c) { return df_split(c.y); }
  static __device__ __forceinline__ double to_double(A x) { return df_to_double(x); }
};

// Geometry of one Gram instantiation: N <= NC = 4 TT columns; a staged site
// holds 12 x NC complex, column fastest (so that the threads staging a site's
// columns write consecutive words), its stride padded by one against bank
// conflicts between the two site lanes of a warp; SB sites per pass fit 40 KB
// of shared memory for u and v together.
template <int FU, int TT, bool LOWP = false> struct GramShape {
  using TU = typename PrecTraits<FU>::real;
  using TA = typename std::conditional<LOWP, float, TU>::type;  // arithmetic / staging type
  using S2 = typename GramArith<TA>::S2;
  static constexpr int NC = 4 * TT;
  static constexpr int SSTR = 12 * NC + 1;
  static constexpr int SB0 = 40960 / (2 * SSTR * (int)sizeof(S2));
  static constexpr int SB = (SB0 > 16 ? 16 : SB0) & ~1;  // even: two site lanes per warp
  static constexpr int NTH = 16 * SB;                    // 16 tile slots x SB site lanes
  static constexpr int STAGE_BYTES = 2 * SB * SSTR * (int)sizeof(S2);
  static constexpr int RED_BYTES = (SB / 2) * (4 * TT) * (4 * TT) * 16;
  static constexpr int SMEM = STAGE_BYTES > RED_BYTES ? STAGE_BYTES : RED_BYTES;
};

// LOWP (FP64 operands of a mixed solve, whose Gram matrices only steer the
// sloppy recurrence and test convergence): FP32 products and sums.
template <int FU, int TT, bool LOWP = false>
__global__ void __launch_bounds__(GramShape<FU, TT, LOWP>::NTH) k_gram(const BlockArgs a) {
  using Sh = GramShape<FU, TT, LOWP>;
  using TU = typename Sh::TU;
  using TA = typename Sh::TA;
  using GA = GramArith<TA>;
  using A = typename GA::A;
  using S2 = typename Sh::S2;
  constexpr int SB = Sh::SB, NTH = Sh::NTH, SSTR = Sh::SSTR;
  if (gate_closed(a.gate)) return;
  __shared__ __align__(16) unsigned char smem[Sh::SMEM];
  __shared__ int is_last;
  S2* su = reinterpret_cast<S2*>(smem);
  S2* sv = su + SB * SSTR;
  const int N = a.N, NN = N * N;
  const int NT = (N + TT - 1) / TT;  // tiles per dimension (<= 4)
  const int tid = threadIdx.x;
  const int tile = tid & 15, ls = tid >> 4;
  const int ta = tile >> 2, tb = tile & 3;
  const bool worker = ta < NT && tb < NT;
  const int a0 = ta * TT, b0 = tb * TT;
  A accr[TT][TT], acci[TT][TT];
#pragma unroll
  for (int i = 0; i < TT; i++)
#pragma unroll
    for (int j = 0; j < TT; j++) accr[i][j] = acci[i][j] = A(0);
  const int64_t nsite4 = a.g.Vh;
  for (int64_t s0 = (int64_t)blockIdx.x * SB; s0 < nsite4; s0 += (int64_t)gridDim.x * SB) {
    // stage SB sites x N columns of u and v (one spinor per thread and pass)
    for (int e = tid; e < SB * N; e += NTH) {
      const int es = e / N, col = e - es * N;
      const int64_t site = s0 + es;
      S2* du = su + es * SSTR + col;
      S2* dv = sv + es * SSTR + col;
      if (site < nsite4) {
        const int64_t j = site * a.g.n5 + col;
        Spinor<TU> x, y;
        SpinorIO<FU>::load(a.u, a.g.sstride, j, x);
        SpinorIO<FU>::load(a.v, a.g.sstride, j, y);
#pragma unroll
        for (int k = 0; k < 12; k++) {
          du[k * Sh::NC] = GA::stage((TA)x.v[k].r, (TA)x.v[k].i);
          dv[k * Sh::NC] = GA::stage((TA)y.v[k].r, (TA)y.v[k].i);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 12; k++) du[k * Sh::NC] = dv[k * Sh::NC] = GA::stage(TA(0), TA(0));
      }
    }
    __syncthreads();
    if (worker) {
      const S2* bu = su + ls * SSTR;
      const S2* bv = sv + ls * SSTR;
#pragma unroll 2
      for (int k = 0; k < 12; k++) {
        A ur[TT], ui[TT], vr[TT], vi[TT];
#pragma unroll
        for (int i = 0; i < TT; i++) {
          // rows past N (a ragged last tile) read row N - 1 and are never stored
          const int ra = a0 + i < N ? a0 + i : N - 1, rb = b0 + i < N ? b0 + i : N - 1;
          const S2 cu = bu[k * Sh::NC + ra], cv = bv[k * Sh::NC + rb];
          ur[i] = GA::re(cu);
          ui[i] = GA::im(cu);
          vr[i] = GA::re(cv);
          vi[i] = GA::im(cv);
        }
#pragma unroll
        for (int i = 0; i < TT; i++)
#pragma unroll
          for (int j = 0; j < TT; j++) {  // conj(u) v
            accr[i][j] = fma(ur[i], vr[j], fma(ui[i], vi[j], accr[i][j]));
            acci[i][j] = fma(ur[i], vi[j], fma(-ui[i], vr[j], acci[i][j]));
          }
      }
    }
    __syncthreads();
  }
  // FP64 from here: the two site lanes of a warp (lanes l and l + 16 hold the
  // same tile) by a shuffle, the warps by a fixed-order sum into this block's partial
  double* wred = reinterpret_cast<double*>(smem);  // [SB / 2][NN][2], the staging buffers reused
  const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int i = 0; i < TT; i++)
#pragma unroll
    for (int j = 0; j < TT; j++) {
      double r = worker ? GA::to_double(accr[i][j]) : 0.0;
      double im = worker ? GA::to_double(acci[i][j]) : 0.0;
      r += __shfl_xor_sync(0xffffffffu, r, 16);
      im += __shfl_xor_sync(0xffffffffu, im, 16);
      if (lane < 16 && worker && a0 + i < N && b0 + j < N) {
        const int e = (a0 + i) * N + b0 + j;
        wred[(warp * NN + e) * 2] = r;
        wred[(warp * NN + e) * 2 + 1] = im;
      }
    }
  __syncthreads();
  for (int e = tid; e < NN; e += NTH) {
    double sr = 0.0, si = 0.0;
    for (int w = 0; w < SB / 2; w++) {
      sr += wred[(w * NN + e) * 2];
      si += wred[(w * NN + e) * 2 + 1];
    }
    a.partials[(int64_t)blockIdx.x * NN + e] = mk(sr, si);
  }
  __threadfence();  // every writer fences before the ticket below
  __syncthreads();
  if (tid == 0) is_last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // the last block: each entry summed over the blocks' partials, a warp per
  // entry (lane l takes blocks l, l + 32, ...; then a fixed shuffle tree)
  __shared__ cpx<double> M[BMAX * BMAX];
  __shared__ cpx<double> Lsh[BMAX * BMAX];
  const int nb = (int)gridDim.x;
  for (int e = warp; e < NN; e += NTH / 32) {
    double sr = 0.0, si = 0.0;
    for (int b = lane; b < nb; b += 32) {
      const double2 w = __ldcg(reinterpret_cast<const double2*>(a.partials + (int64_t)b * NN + e));
      sr += w.x;
      si += w.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) M[e] = mk(sr, si);
  }
  __syncthreads();
  if (warp == 0) {
    block_finalize(a, M, Lsh);
    if (lane == 0) *a.counter = 0u;
  }
}

// ---------------------------------------------------------------- block updates

// Threads of the block update kernels: the N columns of spb = UPD_THREADS / N
// sites, so that each site's columns are read from global memory once (by their
// own threads) into shared memory and mixed from there.
template <int SF> constexpr int upd_threads() { return SF == LQCD_F64 ? 64 : 128; }

// x_s += P alpha; r_s -= Q alpha
template <int VF, int SF>
__global__ void __launch_bounds__(upd_threads<SF>()) k_block_update(const BlockArgs a) {
  using TV = typename PrecTraits<VF>::real;
  using TS = typename PrecTraits<SF>::real;
  constexpr int NTH = upd_threads<SF>();
  if (gate_closed(a.gate)) return;
  const int N = a.N;
  __shared__ cpx<TV> al[BMAX * BMAX];  // alpha in the precision of the iterated vectors
  __shared__ cpx<TS> sp[12][NTH];       // the block's columns of P and Q, thread order fastest
  __shared__ cpx<TS> sq[12][NTH];
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) al[e] = mk((TV)a.st->alpha[e].r, (TV)a.st->alpha[e].i);
  const int spb = blockDim.x / N;
  const int ls = threadIdx.x / N, col = threadIdx.x - ls * N;
  const int64_t site = (int64_t)blockIdx.x * spb + ls;
  const bool valid = ls < spb && site < a.g.Vh;
  const int64_t base = site * a.g.n5;
  if (valid) {
    Spinor<TS> p, q;
    SpinorIO<SF>::load(a.p, a.g.sstride, base + col, p);
    SpinorIO<SF>::load(a.q, a.g.sstride, base + col, q);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      sp[k][threadIdx.x] = p.v[k];
      sq[k][threadIdx.x] = q.v[k];
    }
  }
  __syncthreads();
  if (!valid) return;
  Spinor<TV> x, r;
  SpinorIO<VF>::load(a.xs, a.g.sstride, base + col, x);
  SpinorIO<VF>::load(a.rs, a.g.sstride, base + col, r);
  const int t0 = ls * N;
  for (int k5 = 0; k5 < N; k5++) {
    const cpx<TV> cc = al[k5 * N + col];  // alpha[k5][col]
    if (cc.r == TV(0) && cc.i == TV(0)) continue;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const cpx<TS> pk = sp[k][t0 + k5], qk = sq[k][t0 + k5];
      x.v[k] = cmadd(x.v[k], mk((TV)pk.r, (TV)pk.i), cc);
      r.v[k] = cmadd(r.v[k], mk((TV)-qk.r, (TV)-qk.i), cc);
    }
  }
  SpinorIO<VF>::store(a.xs, a.g.sstride, base + col, x);
  SpinorIO<VF>::store(a.rs, a.g.sstride, base + col, r);
}

// P = R_s + P beta (in place: the block's old columns are in shared memory
// before any is written); frozen columns get P = 0
template <int VF, int SF>
__global__ void __launch_bounds__(upd_threads<SF>()) k_block_pupdate(const BlockArgs a) {
  using TV = typename PrecTraits<VF>::real;
  using TS = typename PrecTraits<SF>::real;
  constexpr int NTH = upd_threads<SF>();
  if (gate_closed(a.gate)) return;
  const int N = a.N;
  __shared__ cpx<TS> be[BMAX * BMAX];  // beta in the precision of the search directions
  __shared__ int dn[BMAX];
  __shared__ cpx<TS> sp[12][NTH];
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) be[e] = mk((TS)a.st->beta[e].r, (TS)a.st->beta[e].i);
  for (int e = threadIdx.x; e < N; e += blockDim.x) dn[e] = a.st->done[e];
  const int spb = blockDim.x / N;
  const int ls = threadIdx.x / N, col = threadIdx.x - ls * N;
  const int64_t site = (int64_t)blockIdx.x * spb + ls;
  const bool valid = ls < spb && site < a.g.Vh;
  const int64_t base = site * a.g.n5;
  if (valid) {
    Spinor<TS> p;
    SpinorIO<SF>::load(a.p, a.g.sstride, base + col, p);
#pragma unroll
    for (int k = 0; k < 12; k++) sp[k][threadIdx.x] = p.v[k];
  }
  __syncthreads();
  if (!valid) return;
  Spinor<TS> out;
  Spinor<TV> r;
  SpinorIO<VF>::load(a.rs, a.g.sstride, base + col, r);
#pragma unroll
  for (int k = 0; k < 12; k++) out.v[k] = mk((TS)r.v[k].r, (TS)r.v[k].i);
  const int t0 = ls * N;
  for (int k5 = 0; k5 < N; k5++) {
    const cpx<TS> cc = be[k5 * N + col];  // beta[k5][col]
    if (cc.r == TS(0) && cc.i == TS(0)) continue;
#pragma unroll
    for (int k = 0; k < 12; k++) out.v[k] = cmadd(out.v[k], sp[k][t0 + k5], cc);
  }
  if (dn[col]) zero(out);
  SpinorIO<SF>::store(const_cast<void*>(a.p), a.g.sstride, base + col, out);
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

// One wave of resident blocks (every block makes the same number of passes, so
// none runs alone at the end), at most GRAM_GRID (the partials' capacity).
template <int FU, int TT, bool LOWP>
static void launch_gram_tt(const BlockArgs& a, cudaStream_t s) {
  using Sh = GramShape<FU, TT, LOWP>;
  static const int resident = [] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gram<FU, TT, LOWP>, Sh::NTH, 0);
    return std::max(1, sms * per_sm);
  }();
  const int64_t want = std::min<int64_t>(std::min<int64_t>(GRAM_GRID, resident), (a.g.Vh + Sh::SB - 1) / Sh::SB);
  k_gram<FU, TT, LOWP><<<(unsigned)std::max<int64_t>(1, want), Sh::NTH, 0, s>>>(a);
}

// tile edge TT = ceil(N / 4): NT = ceil(N / TT) <= 4 tiles per dimension fill the 16 tile slots
template <int FU, bool LOWP = false>
static void launch_gram_t(const BlockArgs& a, cudaStream_t s) {
  const int tt = (a.N + 3) / 4;
  if (tt <= 1) launch_gram_tt<FU, 1, LOWP>(a, s);
  else if (tt == 2) launch_gram_tt<FU, 2, LOWP>(a, s);
  else if (tt == 3) launch_gram_tt<FU, 3, LOWP>(a, s);
  else launch_gram_tt<FU, 4, LOWP>(a, s);
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
    // the FP64 residual's Gram in a mixed solve steers the sloppy recurrence and tests
    // convergence (a sum of squares on the diagonal): FP32 arithmetic serves; the plain
    // FP64 solve keeps double-float
    if (fu == LQCD_F64 && sloppy != LQCD_F64) launch_gram_t<LQCD_F64, true>(a, s);
    else if (fu == LQCD_F64) launch_gram_t<LQCD_F64>(a, s);
    else if (fu == LQCD_F32) launch_gram_t<LQCD_F32>(a, s);
    else launch_gram_t<LQCD_F16>(a, s);
    (void)fv;
    return after_launch("k_gram");
  }
  unsigned upd_grid(int* threads) const {
    const int spb = std::max(1, (sloppy == LQCD_F64 ? upd_threads<LQCD_F64>() : upd_threads<LQCD_F32>()) / N);
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
  if (p->update_prec != LQCD_F64 && p->update_prec != LQCD_F64_DF)
    return fail(LQCD_ERR_ARG, "block cg: update_prec must be LQCD_F64 or LQCD_F64_DF");
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
  // reliable updates in double-float arithmetic on the same FP64 fields when asked (mixed solves)
  if (prm->sloppy_prec != LQCD_F64 && prm->update_prec == LQCD_F64_DF) S.op64.prec = LQCD_F64_DF;
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
  key_append(key, S.op64.prec);

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
