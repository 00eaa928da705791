// Two-level adaptive multigrid for the Wilson operator (the Grid paper shows
// the coarse-grid operator of an adaptive multigrid inverter as its stencil
// example, Sec. 2, and lists multigrid-preconditioned solvers, Sec. 4; the
// construction is the standard aggregation-based one):
//
//  * aggregates: blocks of b^4 fine sites split by chirality (spins 0, 1 and
//    2, 3 of the chiral basis); a coarse site carries Nc = 2 Nv components
//    ordered (chirality, k);
//  * P: Nv near-null vectors orthonormalised per aggregate and chirality by
//    modified Gram-Schmidt (one CTA per aggregate and chirality);
//  * restriction c = P^dag psi (one CTA per aggregate) and prolongation
//    psi = P c (one thread per fine site);
//  * the Galerkin coarse operator D_c = P^dag D P, a 9-point stencil of dense
//    Nc x Nc blocks Y_d (d = 0 self, 1 + 2 mu for +mu, 2 + 2 mu for -mu) built
//    in FP64 from the fine hops that stay inside or leave an aggregate (one CTA
//    per coarse site and coarse basis vector), and its application (one thread
//    per coarse site and row);
//  * the solver: flexible GCR in FP64 on the full-lattice Wilson operator,
//    preconditioned by an FP32 V-cycle: MR smoothing, restriction, a fixed
//    number of CGNR iterations on the coarse operator with all scalars on the
//    device, prolongation, MR smoothing. The V-cycle is one captured CUDA graph;
//    the outer iteration reads its scalars on the host.
//
// Fine vectors are full-lattice spinors in the device layout (n5 = 1); a set
// of Nv of them lies at consecutive field offsets. Coarse vectors are
// [coarse site][Nc] complex, coarse sites lexicographic with x fastest; the
// coarse operator is [9][coarse site][Nc][Nc].
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "lqcd_internal.h"

namespace lqcd {

constexpr int MG_BLOCK = 256;
constexpr int MG_MAX_NV = 32;

struct MGGeom {
  Geom g;     // fine
  int b;      // aggregate extent
  int cX, cY, cZ, cT;
  int64_t Vc;
  int nv, nc;
};

static int make_mg_geom(const lqcd_lattice* lat, int nvec, int block, MGGeom* m) {
  int st = make_geom(lat, &m->g);
  if (st) return st;
  if (m->g.n5 != 1) return fail(LQCD_ERR_ARG, "multigrid: n5 must be 1");
  if (block != 2 && block != 4) return fail(LQCD_ERR_ARG, "multigrid: block must be 2 or 4");
  if (nvec < 1 || nvec > MG_MAX_NV) return fail(LQCD_ERR_ARG, "multigrid: nvec must be 1..%d", MG_MAX_NV);
  const int d[4] = {m->g.X, m->g.Y, m->g.Z, m->g.T};
  for (int mu = 0; mu < 4; mu++)
    if (d[mu] % block) return fail(LQCD_ERR_ARG, "multigrid: block %d does not divide extent %d", block, d[mu]);
  m->b = block;
  m->cX = m->g.X / block;
  m->cY = m->g.Y / block;
  m->cZ = m->g.Z / block;
  m->cT = m->g.T / block;
  m->Vc = (int64_t)m->cX * m->cY * m->cZ * m->cT;
  m->nv = nvec;
  m->nc = 2 * nvec;
  return LQCD_OK;
}

// ------------------------------------------------------------------ small device helpers

// Aggregate kernels run max(32, b^4) threads (whole warps for the shuffles); threads
// beyond b^4 hold no site and add zeros to the reductions.
static int agg_threads(const MGGeom& m) { return std::max(32, m.b * m.b * m.b * m.b); }

// Fine site of thread `tid` inside aggregate `agg`: coordinates, parity and cb index.
__device__ __forceinline__ void agg_site(const MGGeom& m, int64_t agg, int tid, int c[4], int& parity, int64_t& cb) {
  const int b = m.b;
  int64_t a = agg;
  const int ax = (int)(a % m.cX);
  a /= m.cX;
  const int ay = (int)(a % m.cY);
  a /= m.cY;
  const int az = (int)(a % m.cZ);
  const int at = (int)(a / m.cZ);
  c[0] = ax * b + tid % b;
  c[1] = ay * b + (tid / b) % b;
  c[2] = az * b + (tid / (b * b)) % b;
  c[3] = at * b + tid / (b * b * b);
  const int64_t lex = c[0] + (int64_t)m.g.X * (c[1] + (int64_t)m.g.Y * (c[2] + (int64_t)m.g.Z * c[3]));
  parity = (c[0] + c[1] + c[2] + c[3]) & 1;
  cb = lex >> 1;
}

__device__ __forceinline__ int64_t agg_of(const MGGeom& m, const int c[4]) {
  const int b = m.b;
  return c[0] / b + (int64_t)m.cX * (c[1] / b + (int64_t)m.cY * (c[2] / b + (int64_t)m.cZ * (c[3] / b)));
}

template <int P>
__device__ __forceinline__ const void* fine_ptr(const void* base, const MGGeom& m, int k, int parity) {
  const int64_t half = (int64_t)cb_spinor_bytes(m.g, P);
  return static_cast<const char*>(base) + (int64_t)k * 2 * half + parity * half;
}

// Sum of N complex values over the block; the result is valid in thread 0.
template <int N>
__device__ __forceinline__ void block_sum(double2 v[N], double2* sh /* [N][MG_BLOCK/32] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int n = 0; n < N; n++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v[n].x += __shfl_down_sync(0xffffffffu, v[n].x, o);
      v[n].y += __shfl_down_sync(0xffffffffu, v[n].y, o);
    }
    if (lane == 0) sh[n * (MG_BLOCK / 32) + warp] = v[n];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int n = 0; n < N; n++) {
      double2 s = make_double2(0.0, 0.0);
      for (int w = 0; w < nw; w++) {
        s.x += sh[n * (MG_BLOCK / 32) + w].x;
        s.y += sh[n * (MG_BLOCK / 32) + w].y;
      }
      v[n] = s;
    }
  }
  __syncthreads();
}

// Grid-wide sum of N doubles per thread: block partials, then the last block
// (atomic ticket, no waiting) sums them in a fixed order into out[] (valid in
// thread 0 of that block); returns true there. Resets the counter.
template <int N>
__device__ __forceinline__ bool grid_sum(double v[N], double* partials, unsigned int* counter, double out[N]) {
  __shared__ double sh[N][MG_BLOCK / 32];
  __shared__ int is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int n = 0; n < N; n++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[n] += __shfl_down_sync(0xffffffffu, v[n], o);
    if (lane == 0) sh[n][warp] = v[n];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int n = 0; n < N; n++) {
      double s = 0.0;
      for (int w = 0; w < nw; w++) s += sh[n][w];
      partials[(int64_t)n * gridDim.x + blockIdx.x] = s;
    }
    __threadfence();
    is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  // every thread sums a fixed strided subset of the partials, then a fixed-order block sum
#pragma unroll
  for (int n = 0; n < N; n++) {
    double s = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) s += __ldcg(partials + (int64_t)n * gridDim.x + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[n][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int n = 0; n < N; n++) {
      double s = 0.0;
      for (int w = 0; w < nw; w++) s += sh[n][w];
      out[n] = s;
    }
    *counter = 0u;
  }
  return threadIdx.x == 0;
}

// ------------------------------------------------------------------ aggregation kernels

// Modified Gram-Schmidt of the Nv vectors restricted to (aggregate, chirality).
__global__ void __launch_bounds__(MG_BLOCK) k_block_orth(void* vecs, MGGeom m) {
  __shared__ double2 sh[2 * (MG_BLOCK / 32)];
  const int64_t agg = blockIdx.x >> 1;
  const int chir = blockIdx.x & 1;
  const int tid = threadIdx.x;
  const bool act = tid < m.b * m.b * m.b * m.b;
  int c[4], parity;
  int64_t cb;
  agg_site(m, agg, act ? tid : 0, c, parity, cb);
  const int s0 = 2 * chir;  // first spin of the chirality
  for (int k = 0; k < m.nv; k++) {
    Spinor<double> a;
    zero(a);
    if (act) SpinorIO<LQCD_F64>::load(fine_ptr<LQCD_F64>(vecs, m, k, parity), m.g.sstride, cb, a);
    for (int j = 0; j < k; j++) {
      Spinor<double> q;
      zero(q);
      if (act) SpinorIO<LQCD_F64>::load(fine_ptr<LQCD_F64>(vecs, m, j, parity), m.g.sstride, cb, q);
      double2 d[1] = {make_double2(0.0, 0.0)};
#pragma unroll
      for (int e = 0; e < 6; e++) {  // <q, a> over the chirality's 2 spins x 3 colours
        const cpx<double> qa = q.v[3 * s0 + e], aa = a.v[3 * s0 + e];
        d[0].x += qa.r * aa.r + qa.i * aa.i;
        d[0].y += qa.r * aa.i - qa.i * aa.r;
      }
      block_sum<1>(d, sh);
      __shared__ double2 proj;
      if (tid == 0) proj = d[0];
      __syncthreads();
      const double2 p = proj;
#pragma unroll
      for (int e = 0; e < 6; e++) {
        cpx<double>& aa = a.v[3 * s0 + e];
        const cpx<double> qa = q.v[3 * s0 + e];
        aa = mk(aa.r - (p.x * qa.r - p.y * qa.i), aa.i - (p.x * qa.i + p.y * qa.r));
      }
      __syncthreads();
    }
    double2 n2[1] = {make_double2(0.0, 0.0)};
#pragma unroll
    for (int e = 0; e < 6; e++) n2[0].x += a.v[3 * s0 + e].r * a.v[3 * s0 + e].r + a.v[3 * s0 + e].i * a.v[3 * s0 + e].i;
    block_sum<1>(n2, sh);
    __shared__ double inv;
    if (tid == 0) inv = n2[0].x > 0.0 ? 1.0 / sqrt(n2[0].x) : 0.0;
    __syncthreads();
    // write back only this chirality's components (the other chirality's CTA owns the rest)
    if (act) {
      double2* base = static_cast<double2*>(const_cast<void*>(fine_ptr<LQCD_F64>(vecs, m, k, parity)));
#pragma unroll
      for (int e = 0; e < 6; e++) {
        const cpx<double> v = inv * a.v[3 * s0 + e];
        base[(3 * s0 + e) * m.g.sstride + cb] = make_double2(v.r, v.i);
      }
    }
    __syncthreads();
  }
}

// c(X)[(s, k)] = sum_{x in X} P_k(x)|_s^dag psi(x)|_s; one CTA per (aggregate X, vector k)
template <int P>
__global__ void __launch_bounds__(MG_BLOCK) k_restrict(void* coarse, const void* fine, const void* vecs, MGGeom m) {
  using T = typename PrecTraits<P>::real;
  __shared__ double2 sh[2 * (MG_BLOCK / 32)];
  const int64_t agg = blockIdx.x;
  const int k = blockIdx.y;
  const bool act = threadIdx.x < m.b * m.b * m.b * m.b;
  int c[4], parity;
  int64_t cb;
  agg_site(m, agg, act ? threadIdx.x : 0, c, parity, cb);
  Spinor<T> psi;
  zero(psi);
  if (act) SpinorIO<P>::load(fine_ptr<P>(fine, m, 0, parity), m.g.sstride, cb, psi);
  cpx<T>* out = static_cast<cpx<T>*>(coarse) + agg * m.nc;
  Spinor<T> v;
  zero(v);
  if (act) SpinorIO<P>::load(fine_ptr<P>(vecs, m, k, parity), m.g.sstride, cb, v);
  T pr[2] = {T(0), T(0)}, pi[2] = {T(0), T(0)};
#pragma unroll
  for (int e = 0; e < 12; e++) {
    const int s = e / 6;
    pr[s] = fma(v.v[e].r, psi.v[e].r, fma(v.v[e].i, psi.v[e].i, pr[s]));
    pi[s] = fma(v.v[e].r, psi.v[e].i, fma(-v.v[e].i, psi.v[e].r, pi[s]));
  }
  double2 d[2] = {make_double2((double)pr[0], (double)pi[0]), make_double2((double)pr[1], (double)pi[1])};
  block_sum<2>(d, sh);
  if (threadIdx.x == 0) {
    out[k] = mk((T)d[0].x, (T)d[0].y);
    out[m.nv + k] = mk((T)d[1].x, (T)d[1].y);
  }
}

// psi(x) = sum_k P_k(x)|_s c(X(x))[(s, k)]  (accumulate: psi += ...)
template <int P>
__global__ void __launch_bounds__(MG_BLOCK) k_prolong(void* fine, const void* coarse, const void* vecs, MGGeom m,
                                                       int accumulate) {
  using T = typename PrecTraits<P>::real;
  const int64_t t = (int64_t)blockIdx.x * MG_BLOCK + threadIdx.x;
  if (t >= 2 * (int64_t)m.g.Vh) return;
  const int parity = t >= m.g.Vh ? 1 : 0;
  const int64_t cb = t - parity * (int64_t)m.g.Vh;
  const Coord x = cb_to_coord(m.g, cb, parity);
  const int64_t agg = agg_of(m, x.c);
  const cpx<T>* cv = static_cast<const cpx<T>*>(coarse) + agg * m.nc;
  Spinor<T> acc;
  if (accumulate) SpinorIO<P>::load(fine_ptr<P>(fine, m, 0, parity), m.g.sstride, cb, acc);
  else zero(acc);
  for (int k = 0; k < m.nv; k++) {
    Spinor<T> v;
    SpinorIO<P>::load(fine_ptr<P>(vecs, m, k, parity), m.g.sstride, cb, v);
    const cpx<T> cp = cv[k], cm = cv[m.nv + k];
#pragma unroll
    for (int e = 0; e < 12; e++) acc.v[e] = cmadd(acc.v[e], v.v[e], e < 6 ? cp : cm);
  }
  SpinorIO<P>::store(const_cast<void*>(fine_ptr<P>(fine, m, 0, parity)), m.g.sstride, cb, acc);
}

// ------------------------------------------------------------------ coarse operator

__device__ __forceinline__ int64_t coarse_nb(const MGGeom& m, int64_t X, int d) {
  if (d == 0) return X;
  const int mu = (d - 1) >> 1;
  const int sgn = (d & 1) ? +1 : -1;
  int64_t a = X;
  int cc[4];
  cc[0] = (int)(a % m.cX);
  a /= m.cX;
  cc[1] = (int)(a % m.cY);
  a /= m.cY;
  cc[2] = (int)(a % m.cZ);
  cc[3] = (int)(a / m.cZ);
  const int L[4] = {m.cX, m.cY, m.cZ, m.cT};
  cc[mu] = (cc[mu] + sgn + L[mu]) % L[mu];
  return cc[0] + (int64_t)m.cX * (cc[1] + (int64_t)m.cY * (cc[2] + (int64_t)m.cZ * cc[3]));
}

// out(X)_i = sum_d sum_j Y_d(X)_ij in(X + d)_j; dagger: sum_d sum_j conj(Y_{-d}(X + d)_ji) in(X + d)_j.
// One warp per (coarse site, row): the lanes take the 9 Nc products in turn
// (consecutive j for consecutive lanes) and the warp sums them.
template <typename T>
__global__ void __launch_bounds__(MG_BLOCK) k_coarse_apply(cpx<T>* out, const cpx<T>* in, const cpx<T>* Y, MGGeom m,
                                                           int dagger) {
  const int64_t wid = ((int64_t)blockIdx.x * MG_BLOCK + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= m.Vc * m.nc) return;  // whole warps exit together
  const int nc = m.nc;
  const int X = (int)(wid / nc);
  const int i = (int)(wid - (int64_t)X * nc);
  // lanes 0..8 find the nine stencil neighbours once (32-bit index arithmetic)
  int nb_l = X;
  if (lane < 9 && lane > 0) {
    const int mu = (lane - 1) >> 1, sgn = (lane & 1) ? 1 : -1;
    int cc[4];
    int a = X;
    cc[0] = a % m.cX;
    a /= m.cX;
    cc[1] = a % m.cY;
    a /= m.cY;
    cc[2] = a % m.cZ;
    cc[3] = a / m.cZ;
    const int L[4] = {m.cX, m.cY, m.cZ, m.cT};
    cc[mu] = (cc[mu] + sgn + L[mu]) % L[mu];
    nb_l = cc[0] + m.cX * (cc[1] + m.cY * (cc[2] + m.cZ * cc[3]));
  }
  float ar = 0.f, ai = 0.f;
  double dr_ = 0.0, di_ = 0.0;
  const int total = 9 * nc;
  for (int base = 0; base < total; base += 32) {  // warp-uniform trip count: every lane joins the shuffle
    const int q = base + lane;
    const int d = q < total ? q / nc : 0;
    const int Xn = __shfl_sync(0xffffffffu, nb_l, d);
    if (q >= total) continue;
    const int j = q - d * nc;
    const cpx<T> v = in[(int64_t)Xn * nc + j];
    cpx<T> y;
    if (!dagger) {
      y = Y[(((int64_t)d * m.Vc + X) * nc + i) * nc + j];
    } else {
      const int dr = d == 0 ? 0 : (((d - 1) ^ 1) + 1);  // opposite direction
      y = conj(Y[(((int64_t)dr * m.Vc + Xn) * nc + j) * nc + i]);
    }
    const cpx<T> p = cmul(y, v);
    if (sizeof(T) == 8) {
      dr_ += (double)p.r;
      di_ += (double)p.i;
    } else {
      ar += (float)p.r;
      ai += (float)p.i;
    }
  }
  if (sizeof(T) == 8) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dr_ += __shfl_down_sync(0xffffffffu, dr_, o);
      di_ += __shfl_down_sync(0xffffffffu, di_, o);
    }
    if (lane == 0) out[wid] = mk((T)dr_, (T)di_);
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar += __shfl_down_sync(0xffffffffu, ar, o);
      ai += __shfl_down_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) out[wid] = mk((T)ar, (T)ai);
  }
}

// One coarse basis vector j of aggregate X + d seen from site x of aggregate X:
// the terms of -1/2 H (and, for d = 0, the mass term) that map it into x.
template <int MU, int S>
__device__ __forceinline__ void hop_term(Spinor<double>& acc, const MGGeom& m, const void* gauge, const void* vecs,
                                         const Coord& x, int64_t cb, int parity, int k, int chir) {
  bool wrap;
  const int64_t nb = neighbour_cb<MU>(m.g, x, S > 0 ? +1 : -1, wrap);
  Spinor<double> s;
  SpinorIO<LQCD_F64>::load(fine_ptr<LQCD_F64>(vecs, m, k, 1 - parity), m.g.sstride, nb, s);
#pragma unroll
  for (int e = 0; e < 12; e++)
    if (e / 6 != chir) s.v[e] = mk(0.0, 0.0);
  Half<double> h, w;
  const double f = -0.5 * (wrap ? m.g.bcd[MU] : 1.0);
  Link<double> u;
  if (S > 0) {  // forward: (1 - gamma_mu) U_mu(x) B(x + mu)
    project<MU, -1>(s, h);
    LinkIO<LQCD_F64, 18>::load(gauge, m.g.gstride, parity * 4 + MU, cb, u);
    link_mul(u, h, w);
    accumulate_scaled<MU, -1>(acc, w, f);
  } else {  // backward: (1 + gamma_mu) U_mu(x - mu)^dag B(x - mu)
    project<MU, +1>(s, h);
    LinkIO<LQCD_F64, 18>::load(gauge, m.g.gstride, (1 - parity) * 4 + MU, nb, u);
    link_mul_dag(u, h, w);
    accumulate_scaled<MU, +1>(acc, w, f);
  }
}

template <int MU>
__device__ __forceinline__ void hop_pair(Spinor<double>& acc, const MGGeom& m, const void* gauge, const void* vecs,
                                         const Coord& x, int64_t cb, int parity, int k, int chir, int d, int lmu) {
  // forward hop leaves the aggregate when x_mu is the last site of the block, backward when the first
  const bool fwd_out = lmu == m.b - 1, bwd_out = lmu == 0;
  if ((d == 0 && !fwd_out) || d == 1 + 2 * MU) hop_term<MU, +1>(acc, m, gauge, vecs, x, cb, parity, k, chir);
  if ((d == 0 && !bwd_out) || d == 2 + 2 * MU) hop_term<MU, -1>(acc, m, gauge, vecs, x, cb, parity, k, chir);
}

// Y_d(X)[:, j] for one coarse site X (blockIdx.x) and coarse basis vector j (blockIdx.y), all d.
__global__ void __launch_bounds__(MG_BLOCK) k_coarse_build(cpx<double>* Y, const void* gauge, const void* vecs,
                                                           MGGeom m, double mass) {
  __shared__ double2 sh[2 * (MG_BLOCK / 32)];
  const int64_t X = blockIdx.x;
  const int j = blockIdx.y;
  const int chir_j = j / m.nv, k_j = j % m.nv;
  const bool act = threadIdx.x < m.b * m.b * m.b * m.b;
  int c[4], parity;
  int64_t cb;
  agg_site(m, X, act ? threadIdx.x : 0, c, parity, cb);
  const Coord x = cb_to_coord(m.g, cb, parity);
  const int lc[4] = {c[0] % m.b, c[1] % m.b, c[2] % m.b, c[3] % m.b};
  const int nc = m.nc;
  for (int d = 0; d < 9; d++) {
    const int dmu = d == 0 ? -1 : (d - 1) >> 1;
    const bool fwd = d != 0 && (d & 1);
    // a site contributes to Y_{+-mu} only from the aggregate's face in that direction
    const bool active = act && (d == 0 || (fwd ? lc[dmu] == m.b - 1 : lc[dmu] == 0));
    Spinor<double> h;
    zero(h);
    if (active) {
      if (d == 0) {
        Spinor<double> s;
        SpinorIO<LQCD_F64>::load(fine_ptr<LQCD_F64>(vecs, m, k_j, parity), m.g.sstride, cb, s);
#pragma unroll
        for (int e = 0; e < 12; e++) h.v[e] = e / 6 == chir_j ? (4.0 + mass) * s.v[e] : mk(0.0, 0.0);
      }
      hop_pair<0>(h, m, gauge, vecs, x, cb, parity, k_j, chir_j, d, lc[0]);
      hop_pair<1>(h, m, gauge, vecs, x, cb, parity, k_j, chir_j, d, lc[1]);
      hop_pair<2>(h, m, gauge, vecs, x, cb, parity, k_j, chir_j, d, lc[2]);
      hop_pair<3>(h, m, gauge, vecs, x, cb, parity, k_j, chir_j, d, lc[3]);
    }
    for (int k = 0; k < m.nv; k++) {
      Spinor<double> v;
      zero(v);
      if (act) SpinorIO<LQCD_F64>::load(fine_ptr<LQCD_F64>(vecs, m, k, parity), m.g.sstride, cb, v);
      double2 s2[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
#pragma unroll
      for (int e = 0; e < 12; e++) {
        const int s = e / 6;
        s2[s].x += v.v[e].r * h.v[e].r + v.v[e].i * h.v[e].i;
        s2[s].y += v.v[e].r * h.v[e].i - v.v[e].i * h.v[e].r;
      }
      block_sum<2>(s2, sh);
      if (threadIdx.x == 0) {
        cpx<double>* blk = Y + ((int64_t)d * m.Vc + X) * nc * nc;
        blk[(int64_t)k * nc + j] = mk(s2[0].x, s2[0].y);
        blk[(int64_t)(m.nv + k) * nc + j] = mk(s2[1].x, s2[1].y);
      }
    }
  }
}

// ------------------------------------------------------------------ vector kernels

// site-aware loop over a full fine field (n5 = 1)
#define MG_FINE_SITE                                                          \
  const int64_t t = (int64_t)blockIdx.x * MG_BLOCK + threadIdx.x;              \
  const bool valid = t < 2 * (int64_t)g.Vh;                                    \
  const int parity = valid && t >= g.Vh ? 1 : 0;                               \
  const int64_t cb = valid ? t - parity * (int64_t)g.Vh : 0;

template <int PD, int PS>
__global__ void __launch_bounds__(MG_BLOCK) k_convert(void* dst, const void* src, Geom g) {
  using TD = typename PrecTraits<PD>::real;
  using TS = typename PrecTraits<PS>::real;
  MG_FINE_SITE
  if (!valid) return;
  const int64_t hd = (int64_t)cb_spinor_bytes(g, PD), hs = (int64_t)cb_spinor_bytes(g, PS);
  Spinor<TS> a;
  SpinorIO<PS>::load(static_cast<const char*>(src) + parity * hs, g.sstride, cb, a);
  Spinor<TD> b;
#pragma unroll
  for (int e = 0; e < 12; e++) b.v[e] = mk((TD)a.v[e].r, (TD)a.v[e].i);
  SpinorIO<PD>::store(static_cast<char*>(dst) + parity * hd, g.sstride, cb, b);
}

// y = a x + s y (a complex: host value times, when coef is set, the device scalar *coef)
template <int P>
__global__ void __launch_bounds__(MG_BLOCK) k_axpby(void* y, const void* x, Geom g, double ar, double ai,
                                                    const double2* coef, double s) {
  using T = typename PrecTraits<P>::real;
  MG_FINE_SITE
  if (!valid) return;
  double cr = ar, ci = ai;
  if (coef) {
    const double2 k = *coef;
    cr = ar * k.x - ai * k.y;
    ci = ar * k.y + ai * k.x;
  }
  const cpx<T> a = mk((T)cr, (T)ci);
  const int64_t h = (int64_t)cb_spinor_bytes(g, P);
  Spinor<T> xv, yv;
  SpinorIO<P>::load(static_cast<const char*>(x) + parity * h, g.sstride, cb, xv);
  if (s != 0.0) SpinorIO<P>::load(static_cast<const char*>(y) + parity * h, g.sstride, cb, yv);
  if (s == 0.0) zero(yv);  // y is overwritten, not read (it may hold anything)
#pragma unroll
  for (int e = 0; e < 12; e++) yv.v[e] = cmadd((T)s * yv.v[e], a, xv.v[e]);
  SpinorIO<P>::store(static_cast<char*>(y) + parity * h, g.sstride, cb, yv);
}

// <x, y> (complex) and |x|^2 into out[0..2]; with mr_alpha also alpha = <x, y> / |x|^2 into *alpha
template <int P>
__global__ void __launch_bounds__(MG_BLOCK) k_dot(const void* x, const void* y, Geom g, double* partials,
                                                  unsigned int* counter, double* out, double2* mr_alpha) {
  using T = typename PrecTraits<P>::real;
  MG_FINE_SITE
  // per-site sums in the field precision (FP64 arithmetic is scarce on this GPU),
  // the sum over sites in FP64
  double v[3] = {0.0, 0.0, 0.0};
  if (valid) {
    const int64_t h = (int64_t)cb_spinor_bytes(g, P);
    Spinor<T> xv, yv;
    SpinorIO<P>::load(static_cast<const char*>(x) + parity * h, g.sstride, cb, xv);
    SpinorIO<P>::load(static_cast<const char*>(y) + parity * h, g.sstride, cb, yv);
    T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
    for (int e = 0; e < 12; e++) {
      a0 = fma(xv.v[e].r, yv.v[e].r, fma(xv.v[e].i, yv.v[e].i, a0));
      a1 = fma(xv.v[e].r, yv.v[e].i, fma(-xv.v[e].i, yv.v[e].r, a1));
      a2 = fma(xv.v[e].r, xv.v[e].r, fma(xv.v[e].i, xv.v[e].i, a2));
    }
    v[0] = (double)a0;
    v[1] = (double)a1;
    v[2] = (double)a2;
  }
  double tot[3];
  if (grid_sum<3>(v, partials, counter, tot)) {
    if (out) {
      out[0] = tot[0];
      out[1] = tot[1];
      out[2] = tot[2];
    }
    if (mr_alpha) *mr_alpha = tot[2] > 0.0 ? make_double2(tot[0] / tot[2], tot[1] / tot[2]) : make_double2(0.0, 0.0);
  }
}

// y64 += x32 (the FP32 correction of a refinement cycle added to the FP64 solution)
__global__ void __launch_bounds__(MG_BLOCK) k_acc64(void* y, const void* x, Geom g) {
  MG_FINE_SITE
  if (!valid) return;
  const int64_t h64 = (int64_t)cb_spinor_bytes(g, LQCD_F64), h32 = (int64_t)cb_spinor_bytes(g, LQCD_F32);
  Spinor<double> yv;
  Spinor<float> xv;
  SpinorIO<LQCD_F64>::load(static_cast<const char*>(y) + parity * h64, g.sstride, cb, yv);
  SpinorIO<LQCD_F32>::load(static_cast<const char*>(x) + parity * h32, g.sstride, cb, xv);
#pragma unroll
  for (int e = 0; e < 12; e++) yv.v[e] = mk(yv.v[e].r + (double)xv.v[e].r, yv.v[e].i + (double)xv.v[e].i);
  SpinorIO<LQCD_F64>::store(static_cast<char*>(y) + parity * h64, g.sstride, cb, yv);
}

// MR step: e += alpha s, s -= alpha t (alpha from the device)
template <int P>
__global__ void __launch_bounds__(MG_BLOCK) k_mr_update(void* e, void* s, const void* tv_, Geom g, const double2* alpha) {
  using T = typename PrecTraits<P>::real;
  MG_FINE_SITE
  if (!valid) return;
  const double2 al = *alpha;
  const cpx<T> a = mk((T)al.x, (T)al.y), ma = mk((T)-al.x, (T)-al.y);
  const int64_t h = (int64_t)cb_spinor_bytes(g, P);
  Spinor<T> ev, sv, tv;
  SpinorIO<P>::load(static_cast<const char*>(e) + parity * h, g.sstride, cb, ev);
  SpinorIO<P>::load(static_cast<const char*>(s) + parity * h, g.sstride, cb, sv);
  SpinorIO<P>::load(static_cast<const char*>(tv_) + parity * h, g.sstride, cb, tv);
#pragma unroll
  for (int k = 0; k < 12; k++) {
    ev.v[k] = cmadd(ev.v[k], a, sv.v[k]);
    sv.v[k] = cmadd(sv.v[k], ma, tv.v[k]);
  }
  SpinorIO<P>::store(static_cast<char*>(e) + parity * h, g.sstride, cb, ev);
  SpinorIO<P>::store(static_cast<char*>(s) + parity * h, g.sstride, cb, sv);
}

// ---- coarse CGNR with device scalars: sc[0] = gamma, sc[1] = alpha, sc[2] = beta
template <typename T>
__global__ void __launch_bounds__(MG_BLOCK) k_c_norm(const cpx<T>* v, int64_t n, double* partials,
                                                     unsigned int* counter, double* sc, int mode) {
  const int64_t t = (int64_t)blockIdx.x * MG_BLOCK + threadIdx.x;
  double a[1] = {0.0};
  if (t < n) a[0] = (double)v[t].r * v[t].r + (double)v[t].i * v[t].i;
  double tot[1];
  if (grid_sum<1>(a, partials, counter, tot)) {
    if (mode == 0) sc[0] = tot[0];                          // gamma = |s|^2 (initial)
    else if (mode == 1) sc[1] = tot[0] > 0.0 ? sc[0] / tot[0] : 0.0;  // alpha = gamma / |q|^2
    else {                                                  // beta = gamma' / gamma
      sc[2] = sc[0] > 0.0 ? tot[0] / sc[0] : 0.0;
      sc[0] = tot[0];
    }
  }
}

// mode 0: x = 0, r = c, (p set later); 1: x += alpha p, r -= alpha q; 2: p = s + beta p; 3: p = s
template <typename T>
__global__ void __launch_bounds__(MG_BLOCK) k_c_update(cpx<T>* x, cpx<T>* r, cpx<T>* p, const cpx<T>* q,
                                                       const cpx<T>* s, const cpx<T>* c, int64_t n, const double* sc,
                                                       int mode) {
  const int64_t t = (int64_t)blockIdx.x * MG_BLOCK + threadIdx.x;
  if (t >= n) return;
  if (mode == 0) {
    x[t] = mk(T(0), T(0));
    r[t] = c[t];
  } else if (mode == 1) {
    const T a = (T)sc[1];
    x[t] = x[t] + a * p[t];
    r[t] = r[t] - a * q[t];
  } else if (mode == 2) {
    p[t] = s[t] + (T)sc[2] * p[t];
  } else {
    p[t] = s[t];
  }
}

// ------------------------------------------------------------------ host side

static unsigned fine_grid(const Geom& g) { return (unsigned)((2 * (int64_t)g.Vh + MG_BLOCK - 1) / MG_BLOCK); }
static unsigned n_grid(int64_t n) { return (unsigned)((n + MG_BLOCK - 1) / MG_BLOCK); }

template <typename F> static int dispatch_prec(int prec, F&& f) {
  if (prec == LQCD_F64) return f(std::integral_constant<int, LQCD_F64>());
  if (prec == LQCD_F32) return f(std::integral_constant<int, LQCD_F32>());
  return fail(LQCD_ERR_ARG, "multigrid: precision must be LQCD_F64 or LQCD_F32");
}

static int restrict_(const MGGeom& m, int prec, void* coarse, const void* fine, const void* vecs, cudaStream_t s) {
  return dispatch_prec(prec, [&](auto P) {
    k_restrict<decltype(P)::value><<<dim3((unsigned)m.Vc, (unsigned)m.nv), agg_threads(m), 0, s>>>(coarse, fine, vecs,
                                                                                                 m);
    return after_launch("k_restrict");
  });
}
static int prolong_(const MGGeom& m, int prec, void* fine, const void* coarse, const void* vecs, int acc,
                    cudaStream_t s) {
  return dispatch_prec(prec, [&](auto P) {
    k_prolong<decltype(P)::value><<<fine_grid(m.g), MG_BLOCK, 0, s>>>(fine, coarse, vecs, m, acc);
    return after_launch("k_prolong");
  });
}
static int coarse_apply_(const MGGeom& m, int prec, void* out, const void* in, const void* Y, int dagger,
                         cudaStream_t s) {
  const unsigned grid = n_grid(m.Vc * m.nc * 32);
  if (prec == LQCD_F64)
    k_coarse_apply<double><<<grid, MG_BLOCK, 0, s>>>(static_cast<cpx<double>*>(out),
                                                     static_cast<const cpx<double>*>(in),
                                                     static_cast<const cpx<double>*>(Y), m, dagger);
  else if (prec == LQCD_F32)
    k_coarse_apply<float><<<grid, MG_BLOCK, 0, s>>>(static_cast<cpx<float>*>(out), static_cast<const cpx<float>*>(in),
                                                    static_cast<const cpx<float>*>(Y), m, dagger);
  else
    return fail(LQCD_ERR_ARG, "multigrid: precision must be LQCD_F64 or LQCD_F32");
  return after_launch("k_coarse_apply");
}
static int orthonormalize_(const MGGeom& m, void* vecs, cudaStream_t s) {
  k_block_orth<<<(unsigned)(2 * m.Vc), agg_threads(m), 0, s>>>(vecs, m);
  return after_launch("k_block_orth");
}
static int coarse_build_(const MGGeom& m, void* Y, const void* gauge, const void* vecs, double mass, cudaStream_t s) {
  dim3 grid((unsigned)m.Vc, (unsigned)m.nc);
  k_coarse_build<<<grid, agg_threads(m), 0, s>>>(static_cast<cpx<double>*>(Y), gauge, vecs, m, mass);
  return after_launch("k_coarse_build");
}

// float conversion of a coarse operator / vector (element-wise)
__global__ void k_c_to_f32(cpx<float>* dst, const cpx<double>* src, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * MG_BLOCK + threadIdx.x;
  if (t < n) dst[t] = mk((float)src[t].r, (float)src[t].i);
}

// The adjoint stencil in FP32, stored explicitly so that D_c^dag runs with the
// coalesced row access of D_c: Yd_d(X)_ij = conj(Y_{-d}(X + d)_ji).
__global__ void k_c_dagger(cpx<float>* Yd, const cpx<double>* Y, MGGeom m) {
  const int64_t t = (int64_t)blockIdx.x * MG_BLOCK + threadIdx.x;
  const int nc = m.nc;
  if (t >= 9 * m.Vc * nc * nc) return;
  const int64_t ij = t % ((int64_t)nc * nc);
  const int64_t dX = t / ((int64_t)nc * nc);
  const int64_t X = dX % m.Vc;
  const int d = (int)(dX / m.Vc);
  const int i = (int)(ij / nc), j = (int)(ij % nc);
  const int dr = d == 0 ? 0 : (((d - 1) ^ 1) + 1);
  const cpx<double> y = Y[(((int64_t)dr * m.Vc + coarse_nb(m, X, d)) * nc + j) * nc + i];
  Yd[t] = mk((float)y.r, (float)-y.i);
}

// ---- solver workspace
struct MGWs {
  double* partials;       // reduction scratch (3 x max blocks)
  unsigned int* counter;
  double* dots;           // host-read results (3 doubles)
  double2* alpha;         // MR alpha (device)
  double* csc;            // coarse CG scalars (3)
  void* P64;              // Nv FP64 fields
  void* P32;              // Nv FP32 fields
  void* Y64;              // coarse operator FP64
  void* Y32;              // coarse operator FP32
  void* Y32d;             // its adjoint stencil FP32
  void* cvec[6];          // FP32 coarse: c, x, r, p, q, s
  void* f32[5];           // FP32 fine: r, e, s (MR residual), t, tmp
  void* r64;              // FP64 true residual of a refinement cycle
  void* x32;              // FP32 correction accumulated within a cycle
  void* Z;                // restart x FP32 fields z_i = K r
  void* W;                // restart x FP32 fields w_i = D z_i
  void* scratch;          // the region of Z and W, lent to the set-up CG
  size_t scratch_bytes;
  size_t total;
};

static MGWs mg_carve(void* base, const MGGeom& m, int restart, size_t setup_cg_bytes) {
  MGWs w;
  memset(&w, 0, sizeof(w));
  size_t o = 0;
  char* b = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> void* {
    void* r = b ? b + o : nullptr;
    o += round_up((int64_t)bytes, 256);
    return r;
  };
  const size_t f64 = 2 * cb_spinor_bytes(m.g, LQCD_F64), f32 = 2 * cb_spinor_bytes(m.g, LQCD_F32);
  const int64_t maxb = std::max<int64_t>((int64_t)fine_grid(m.g), (int64_t)n_grid(m.Vc * m.nc));
  w.partials = static_cast<double*>(take(sizeof(double) * 3 * maxb));
  w.counter = static_cast<unsigned int*>(take(256));
  w.dots = static_cast<double*>(take(256));
  w.alpha = static_cast<double2*>(take(256));
  w.csc = static_cast<double*>(take(256));
  w.P64 = take(f64 * m.nv);
  w.P32 = take(f32 * m.nv);
  const size_t ybytes = (size_t)9 * m.Vc * m.nc * m.nc;
  w.Y64 = take(ybytes * sizeof(cpx<double>));
  w.Y32 = take(ybytes * sizeof(cpx<float>));
  w.Y32d = take(ybytes * sizeof(cpx<float>));
  for (int k = 0; k < 6; k++) w.cvec[k] = take((size_t)m.Vc * m.nc * sizeof(cpx<float>));
  for (int k = 0; k < 5; k++) w.f32[k] = take(f32);
  w.r64 = take(f64);
  w.x32 = take(f32);
  w.scratch_bytes = std::max(2 * f32 * (size_t)restart, setup_cg_bytes);
  w.scratch = take(w.scratch_bytes);
  w.Z = w.scratch;
  w.W = b ? static_cast<char*>(w.scratch) + f32 * (size_t)restart : nullptr;
  w.total = o;
  return w;
}

static void* field_at(void* base, size_t bytes, int k) { return static_cast<char*>(base) + (size_t)k * bytes; }

struct MGSolver {
  MGGeom m;
  lqcd_mg_params mp;
  lqcd_operator op64, op32;
  const void* gauge64;
  const void* gauge32;
  MGWs w;
  cudaStream_t s;

  size_t f64() const { return 2 * cb_spinor_bytes(m.g, LQCD_F64); }
  size_t f32() const { return 2 * cb_spinor_bytes(m.g, LQCD_F32); }

  int D32(void* out, const void* in) {
    OpCtx c{m.g, op32, gauge32};
    return op_apply(c, out, in, LQCD_FULL, 0, nullptr, nullptr, nullptr, nullptr, s);
  }
  int D64(void* out, const void* in) {
    OpCtx c{m.g, op64, gauge64};
    return op_apply(c, out, in, LQCD_FULL, 0, nullptr, nullptr, nullptr, nullptr, s);
  }
  template <int P> int axpby(void* y, const void* x, double ar, double ai, const double2* coef, double sc) {
    k_axpby<P><<<fine_grid(m.g), MG_BLOCK, 0, s>>>(y, x, m.g, ar, ai, coef, sc);
    return after_launch("k_axpby");
  }
  // <x, y>, |x|^2 on the host
  template <int P> int dot(const void* x, const void* y, double out[3]) {
    k_dot<P><<<fine_grid(m.g), MG_BLOCK, 0, s>>>(x, y, m.g, w.partials, w.counter, w.dots, nullptr);
    int st = after_launch("k_dot");
    if (st) return st;
    cudaError_t e = cudaMemcpyAsync(out, w.dots, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? LQCD_OK : cuda_fail(e, "multigrid: dot readback");
  }

  // MR smoothing of D e = r (FP32): starts from e (zero when fresh), residual s = r - D e
  int smooth(void* e, const void* r, int steps, bool fresh) {
    void* sres = w.f32[2];
    void* t = w.f32[3];
    int st;
    if (fresh) {
      if ((st = axpby<LQCD_F32>(e, r, 0.0, 0.0, nullptr, 0.0))) return st;        // e = 0
      if ((st = axpby<LQCD_F32>(sres, r, 1.0, 0.0, nullptr, 0.0))) return st;     // s = r
    } else {
      if ((st = D32(t, e))) return st;
      if ((st = axpby<LQCD_F32>(sres, r, 1.0, 0.0, nullptr, 0.0))) return st;     // s = r
      if ((st = axpby<LQCD_F32>(sres, t, -1.0, 0.0, nullptr, 1.0))) return st;    // s -= D e
    }
    for (int k = 0; k < steps; k++) {
      if ((st = D32(t, sres))) return st;
      k_dot<LQCD_F32><<<fine_grid(m.g), MG_BLOCK, 0, s>>>(t, sres, m.g, w.partials, w.counter, nullptr, w.alpha);
      if ((st = after_launch("k_dot"))) return st;
      k_mr_update<LQCD_F32><<<fine_grid(m.g), MG_BLOCK, 0, s>>>(e, sres, t, m.g, w.alpha);
      if ((st = after_launch("k_mr_update"))) return st;
    }
    return LQCD_OK;
  }

  // fixed-iteration CGNR on D_c x = c (FP32, device scalars)
  int coarse_solve() {
    cpx<float>* c = static_cast<cpx<float>*>(w.cvec[0]);
    cpx<float>* x = static_cast<cpx<float>*>(w.cvec[1]);
    cpx<float>* r = static_cast<cpx<float>*>(w.cvec[2]);
    cpx<float>* p = static_cast<cpx<float>*>(w.cvec[3]);
    cpx<float>* q = static_cast<cpx<float>*>(w.cvec[4]);
    cpx<float>* sv = static_cast<cpx<float>*>(w.cvec[5]);
    const int64_t n = m.Vc * m.nc;
    const unsigned gr = n_grid(n);
    int st;
    k_c_update<float><<<gr, MG_BLOCK, 0, s>>>(x, r, p, q, sv, c, n, w.csc, 0);
    if ((st = coarse_apply_(m, LQCD_F32, sv, r, w.Y32d, 0, s))) return st;
    k_c_update<float><<<gr, MG_BLOCK, 0, s>>>(x, r, p, q, sv, c, n, w.csc, 3);
    k_c_norm<float><<<gr, MG_BLOCK, 0, s>>>(sv, n, w.partials, w.counter, w.csc, 0);
    for (int it = 0; it < mp.coarse_iters; it++) {
      if ((st = coarse_apply_(m, LQCD_F32, q, p, w.Y32, 0, s))) return st;
      k_c_norm<float><<<gr, MG_BLOCK, 0, s>>>(q, n, w.partials, w.counter, w.csc, 1);
      k_c_update<float><<<gr, MG_BLOCK, 0, s>>>(x, r, p, q, sv, c, n, w.csc, 1);
      if ((st = coarse_apply_(m, LQCD_F32, sv, r, w.Y32d, 0, s))) return st;
      k_c_norm<float><<<gr, MG_BLOCK, 0, s>>>(sv, n, w.partials, w.counter, w.csc, 2);
      k_c_update<float><<<gr, MG_BLOCK, 0, s>>>(x, r, p, q, sv, c, n, w.csc, 2);
    }
    return after_launch("coarse cgnr");
  }

  // e = K r (FP32 fields f32[0] = r, f32[1] = e)
  int vcycle() {
    void* r = w.f32[0];
    void* e = w.f32[1];
    void* t = w.f32[3];
    void* res = w.f32[4];
    int st;
    if ((st = smooth(e, r, mp.pre_smooth, true))) return st;
    // res = r - D e
    if ((st = D32(t, e))) return st;
    if ((st = axpby<LQCD_F32>(res, r, 1.0, 0.0, nullptr, 0.0))) return st;
    if ((st = axpby<LQCD_F32>(res, t, -1.0, 0.0, nullptr, 1.0))) return st;
    if ((st = restrict_(m, LQCD_F32, w.cvec[0], res, w.P32, s))) return st;
    if ((st = coarse_solve())) return st;
    if ((st = prolong_(m, LQCD_F32, e, w.cvec[1], w.P32, 1, s))) return st;
    return smooth(e, r, mp.post_smooth, false);
  }

  // The V-cycle is captured on a private stream (capture is not allowed on the
  // legacy default stream) and replayed on the caller's stream.
  cudaGraphExec_t vgraph = nullptr;
  int capture_vcycle() {
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "multigrid: capture stream");
    const cudaStream_t user = s;
    s = cs;
    cudaGraph_t graph = nullptr;
    int st = LQCD_OK;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) st = cuda_fail(e, "multigrid: begin capture");
    if (!st) {
      st = vcycle();
      e = cudaStreamEndCapture(cs, &graph);
      if (!st && e != cudaSuccess) st = cuda_fail(e, "multigrid: end capture");
    }
    s = user;
    cudaStreamDestroy(cs);
    if (st) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    e = cudaGraphInstantiate(&vgraph, graph, 0);
    cudaGraphDestroy(graph);
    return e == cudaSuccess ? LQCD_OK : cuda_fail(e, "multigrid: instantiate");
  }
};

// near-null vectors: a few CG iterations on M^dag M v = (random start), then orthonormalise
static int mg_setup_impl(const MGGeom& m, const MGWs& w, const void* gauge64, const void* gauge32, const double* rnd,
                         const lqcd_lattice* lat, const lqcd_operator* op, const lqcd_mg_params* mp, cudaStream_t s) {
  const size_t f64 = 2 * cb_spinor_bytes(m.g, LQCD_F64);
  lqcd_solver_params sp;
  memset(&sp, 0, sizeof(sp));
  sp.tol = 1e-14;
  sp.maxiter = mp->setup_iters;
  sp.sloppy_prec = LQCD_F32;
  sp.sloppy_recon = 12;
  sp.delta = 0.0;
  sp.check_interval = mp->setup_iters;
  sp.use_graph = 1;
  const size_t cgb = lqcd_cg_workspace_bytes(lat, op, &sp, LQCD_FULL);
  // the CG workspace borrows the outer-solver region (Z, W), unused during set-up
  if (cgb > w.scratch_bytes) return fail(LQCD_ERR_WORKSPACE, "multigrid: set-up CG workspace");
  for (int k = 0; k < m.nv; k++) {
    lqcd_solve_info info;
    const void* src = static_cast<const char*>(static_cast<const void*>(rnd)) + (size_t)k * f64;
    int st = lqcd_cg_solve(field_at(w.P64, f64, k), src, gauge64, gauge32, lat, op, &sp, LQCD_FULL, &info, w.scratch,
                           cgb, s);
    if (st && st != LQCD_ERR_NOT_CONVERGED) return st;
  }
  int st = orthonormalize_(m, w.P64, s);
  if (st) return st;
  const size_t f32 = 2 * cb_spinor_bytes(m.g, LQCD_F32);
  for (int k = 0; k < m.nv; k++) {
    k_convert<LQCD_F32, LQCD_F64><<<fine_grid(m.g), MG_BLOCK, 0, s>>>(field_at(w.P32, f32, k), field_at(w.P64, f64, k),
                                                                      m.g);
    if ((st = after_launch("k_convert"))) return st;
  }
  if ((st = coarse_build_(m, w.Y64, gauge64, w.P64, op->mass, s))) return st;
  const int64_t ny = (int64_t)9 * m.Vc * m.nc * m.nc;
  k_c_to_f32<<<n_grid(ny), MG_BLOCK, 0, s>>>(static_cast<cpx<float>*>(w.Y32), static_cast<const cpx<double>*>(w.Y64),
                                             ny);
  if ((st = after_launch("k_c_to_f32"))) return st;
  k_c_dagger<<<n_grid(ny), MG_BLOCK, 0, s>>>(static_cast<cpx<float>*>(w.Y32d), static_cast<const cpx<double>*>(w.Y64), m);
  return after_launch("k_c_dagger");
}

static size_t setup_cg_bytes(const lqcd_lattice* lat, const lqcd_operator* op, const lqcd_mg_params* mp) {
  lqcd_solver_params sp;
  memset(&sp, 0, sizeof(sp));
  sp.tol = 1e-14;
  sp.maxiter = mp->setup_iters;
  sp.sloppy_prec = LQCD_F32;
  sp.sloppy_recon = 12;
  sp.check_interval = mp->setup_iters;
  sp.use_graph = 1;
  return lqcd_cg_workspace_bytes(lat, op, &sp, LQCD_FULL);
}

static int mg_check(const lqcd_lattice* lat, const lqcd_operator* op, const lqcd_mg_params* mp, MGGeom* m) {
  if (!mp) return fail(LQCD_ERR_ARG, "multigrid: null parameters");
  int st = make_mg_geom(lat, mp->nvec, mp->block, m);
  if (st) return st;
  if (!op) return fail(LQCD_ERR_ARG, "multigrid: null operator");
  if ((st = check_operator(op, m->g))) return st;
  if (op->kind != LQCD_WILSON || op->gparity || op->prec != LQCD_F64 || op->recon != 18)
    return fail(LQCD_ERR_UNSUPPORTED, "multigrid: Wilson operator, LQCD_F64 with 18-real links");
  if (mp->setup_iters < 1 || mp->pre_smooth < 0 || mp->post_smooth < 0 || mp->coarse_iters < 1 || mp->restart < 4)
    return fail(LQCD_ERR_ARG, "multigrid: bad iteration counts");
  return LQCD_OK;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

size_t lqcd_mg_coarse_bytes(const lqcd_lattice* lat, int nvec, int block, int prec) {
  MGGeom m;
  if (make_mg_geom(lat, nvec, block, &m) != LQCD_OK || (prec != LQCD_F64 && prec != LQCD_F32)) return 0;
  return (size_t)m.Vc * m.nc * (prec == LQCD_F64 ? 16 : 8);
}

size_t lqcd_mg_coarse_op_bytes(const lqcd_lattice* lat, int nvec, int block, int prec) {
  MGGeom m;
  if (make_mg_geom(lat, nvec, block, &m) != LQCD_OK || (prec != LQCD_F64 && prec != LQCD_F32)) return 0;
  return (size_t)9 * m.Vc * m.nc * m.nc * (prec == LQCD_F64 ? 16 : 8);
}

int lqcd_mg_block_orthonormalize(void* vecs, int nvec, int block, const lqcd_lattice* lat, void* stream) {
  MGGeom m;
  int st = make_mg_geom(lat, nvec, block, &m);
  if (st) return st;
  if (!vecs || ((uintptr_t)vecs & 15)) return fail(LQCD_ERR_ARG, "lqcd_mg_block_orthonormalize: pointer");
  return orthonormalize_(m, vecs, (cudaStream_t)stream);
}

int lqcd_mg_restrict(void* coarse, const void* fine, const void* vecs, int nvec, int block, int prec,
                     const lqcd_lattice* lat, void* stream) {
  MGGeom m;
  int st = make_mg_geom(lat, nvec, block, &m);
  if (st) return st;
  if (!coarse || !fine || !vecs || (((uintptr_t)coarse | (uintptr_t)fine | (uintptr_t)vecs) & 15))
    return fail(LQCD_ERR_ARG, "lqcd_mg_restrict: pointer");
  return restrict_(m, prec, coarse, fine, vecs, (cudaStream_t)stream);
}

int lqcd_mg_prolong(void* fine, const void* coarse, const void* vecs, int nvec, int block, int prec,
                    const lqcd_lattice* lat, void* stream) {
  MGGeom m;
  int st = make_mg_geom(lat, nvec, block, &m);
  if (st) return st;
  if (!coarse || !fine || !vecs || (((uintptr_t)coarse | (uintptr_t)fine | (uintptr_t)vecs) & 15))
    return fail(LQCD_ERR_ARG, "lqcd_mg_prolong: pointer");
  return prolong_(m, prec, fine, coarse, vecs, 0, (cudaStream_t)stream);
}

int lqcd_mg_coarse_build(void* Y, const void* gauge, const void* vecs, int nvec, int block, const lqcd_lattice* lat,
                         const lqcd_operator* op, void* stream) {
  lqcd_mg_params mp;
  memset(&mp, 0, sizeof(mp));
  mp.nvec = nvec;
  mp.block = block;
  mp.setup_iters = mp.coarse_iters = 1;
  mp.restart = 4;
  MGGeom m;
  int st = mg_check(lat, op, &mp, &m);
  if (st) return st;
  if (!Y || !gauge || !vecs || (((uintptr_t)Y | (uintptr_t)gauge | (uintptr_t)vecs) & 15))
    return fail(LQCD_ERR_ARG, "lqcd_mg_coarse_build: pointer");
  return coarse_build_(m, Y, gauge, vecs, op->mass, (cudaStream_t)stream);
}

int lqcd_mg_coarse_apply(void* out, const void* in, const void* Y, int nvec, int block, int prec, int dagger,
                         const lqcd_lattice* lat, void* stream) {
  MGGeom m;
  int st = make_mg_geom(lat, nvec, block, &m);
  if (st) return st;
  if (!out || !in || !Y || out == in || (((uintptr_t)out | (uintptr_t)in | (uintptr_t)Y) & 15))
    return fail(LQCD_ERR_ARG, "lqcd_mg_coarse_apply: pointer");
  return coarse_apply_(m, prec, out, in, Y, dagger, (cudaStream_t)stream);
}

size_t lqcd_mg_workspace_bytes(const lqcd_lattice* lat, const lqcd_operator* op, const lqcd_mg_params* mp) {
  MGGeom m;
  if (mg_check(lat, op, mp, &m) != LQCD_OK) return 0;
  return mg_carve(nullptr, m, mp->restart, setup_cg_bytes(lat, op, mp)).total;
}

int lqcd_mg_setup(const void* gauge64, const void* gauge32, const double* random_vectors, const lqcd_lattice* lat,
                  const lqcd_operator* op, const lqcd_mg_params* mp, void* workspace, size_t workspace_bytes,
                  void* stream) {
  MGGeom m;
  int st = mg_check(lat, op, mp, &m);
  if (st) return st;
  if (!gauge64 || !gauge32 || !random_vectors || !workspace || ((uintptr_t)workspace & 255))
    return fail(LQCD_ERR_ARG, "lqcd_mg_setup: null or misaligned pointer");
  const MGWs w = mg_carve(workspace, m, mp->restart, setup_cg_bytes(lat, op, mp));
  if (workspace_bytes < w.total) return fail(LQCD_ERR_WORKSPACE, "lqcd_mg_setup: workspace %zu < %zu", workspace_bytes,
                                             w.total);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(workspace, 0, w.total, s);
  if (e != cudaSuccess) return cuda_fail(e, "lqcd_mg_setup: memset");
  return mg_setup_impl(m, w, gauge64, gauge32, random_vectors, lat, op, mp, s);
}

int lqcd_mg_solve(void* x, const void* b, const void* gauge64, const void* gauge32, const lqcd_lattice* lat,
                  const lqcd_operator* op, const lqcd_mg_params* mp, const lqcd_solver_params* prm,
                  lqcd_solve_info* info, void* workspace, size_t workspace_bytes, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  lqcd_solve_info local;
  lqcd_solve_info* inf = info ? info : &local;
  memset(inf, 0, sizeof(*inf));
  auto finish = [&](int status) {
    inf->status = status;
    inf->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return status;
  };
  MGSolver S;
  int st = mg_check(lat, op, mp, &S.m);
  if (st) return finish(st);
  if (!prm || !(prm->tol > 0.0) || prm->maxiter < 1) return finish(fail(LQCD_ERR_ARG, "multigrid: bad solver params"));
  if (!x || !b || !gauge64 || !gauge32 || !workspace || ((uintptr_t)workspace & 255) || (((uintptr_t)x | (uintptr_t)b) & 15))
    return finish(fail(LQCD_ERR_ARG, "lqcd_mg_solve: null or misaligned pointer"));
  S.w = mg_carve(workspace, S.m, mp->restart, setup_cg_bytes(lat, op, mp));
  if (workspace_bytes < S.w.total)
    return finish(fail(LQCD_ERR_WORKSPACE, "lqcd_mg_solve: workspace %zu < %zu", workspace_bytes, S.w.total));
  S.mp = *mp;
  S.op64 = *op;
  S.op32 = *op;
  S.op32.prec = LQCD_F32;
  S.op32.recon = 12;
  S.gauge64 = gauge64;
  S.gauge32 = gauge32;
  S.s = (cudaStream_t)stream;
  const size_t f32 = S.f32();
  const int mres = mp->restart;
  void* r32 = S.w.f32[0];  // the V-cycle graph reads its right-hand side here
  void* e32 = S.w.f32[1];  // and leaves K r here
  // Refinement cycles: FP64 true residual r = b - D x; FP32 flexible GCR on D c = r
  // (Krylov vectors, dots and updates in FP32) until |r| drops by delta_cycle or
  // below the tolerance; x += c in FP64; repeat until the FP64 residual <= tol.
  const double delta_cycle = 1e-5;
  if ((st = S.axpby<LQCD_F64>(x, b, 0.0, 0.0, nullptr, 0.0))) return finish(st);           // x = 0
  if ((st = S.axpby<LQCD_F64>(S.w.r64, b, 1.0, 0.0, nullptr, 0.0))) return finish(st);     // r = b
  double d3[3];
  if ((st = S.dot<LQCD_F64>(b, b, d3))) return finish(st);
  const double bnorm = std::sqrt(d3[2]);
  if (bnorm == 0.0) return finish(LQCD_OK);
  if ((st = S.capture_vcycle())) return finish(st);
  int iters = 0;
  double rel = 1.0;
  int status = LQCD_ERR_NOT_CONVERGED;
  std::vector<double> wnorm2(mres);
  for (;;) {
    if ((st = S.dot<LQCD_F64>(S.w.r64, S.w.r64, d3))) break;
    rel = std::sqrt(d3[2]) / bnorm;
    if (!std::isfinite(rel)) { st = fail(LQCD_ERR_NAN, "multigrid: NaN residual"); break; }
    if (rel <= prm->tol) { status = LQCD_OK; break; }
    if (iters >= prm->maxiter) break;
    if (prm->timeout_ms > 0 &&
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() > prm->timeout_ms) {
      st = fail(LQCD_ERR_TIMEOUT, "multigrid: wall-clock limit exceeded");
      break;
    }
    const double target = std::max(delta_cycle * rel, 0.5 * prm->tol) * bnorm;
    k_convert<LQCD_F32, LQCD_F64><<<fine_grid(S.m.g), MG_BLOCK, 0, S.s>>>(r32, S.w.r64, S.m.g);
    if ((st = after_launch("k_convert"))) break;
    if ((st = S.axpby<LQCD_F32>(S.w.x32, r32, 0.0, 0.0, nullptr, 0.0))) break;  // c = 0
    for (int i = 0; i < mres && iters < prm->maxiter; i++) {
      void* zi = field_at(S.w.Z, f32, i);
      void* wi = field_at(S.w.W, f32, i);
      cudaError_t e = cudaGraphLaunch(S.vgraph, S.s);  // e32 = K r32
      if (e != cudaSuccess) { st = cuda_fail(e, "multigrid: V-cycle launch"); break; }
      if ((st = S.axpby<LQCD_F32>(zi, e32, 1.0, 0.0, nullptr, 0.0)) || (st = S.D32(wi, zi))) break;
      // w_i -= beta_j w_j, z_i -= beta_j z_j with beta_j = <w_j, w_i> / |w_j|^2 (modified Gram-Schmidt)
      for (int j = 0; j < i && !st; j++) {
        void* wj = field_at(S.w.W, f32, j);
        if ((st = S.dot<LQCD_F32>(wj, wi, d3))) break;
        const double br = d3[0] / wnorm2[j], bi = d3[1] / wnorm2[j];
        if ((st = S.axpby<LQCD_F32>(wi, wj, -br, -bi, nullptr, 1.0))) break;
        st = S.axpby<LQCD_F32>(zi, field_at(S.w.Z, f32, j), -br, -bi, nullptr, 1.0);
      }
      if (st) break;
      // alpha = <w_i, r> / |w_i|^2; c += alpha z_i; r -= alpha w_i
      if ((st = S.dot<LQCD_F32>(wi, r32, d3))) break;
      wnorm2[i] = d3[2];
      if (!(d3[2] > 0.0) || !std::isfinite(d3[2])) { st = fail(LQCD_ERR_NAN, "multigrid: GCR breakdown"); break; }
      const double ar = d3[0] / d3[2], ai = d3[1] / d3[2];
      if ((st = S.axpby<LQCD_F32>(S.w.x32, zi, ar, ai, nullptr, 1.0))) break;
      if ((st = S.axpby<LQCD_F32>(r32, wi, -ar, -ai, nullptr, 1.0))) break;
      iters++;
      if ((st = S.dot<LQCD_F32>(r32, r32, d3))) break;
      if (std::sqrt(d3[2]) <= target) break;
    }
    if (st) break;
    // x += c in FP64, then the FP64 true residual
    k_acc64<<<fine_grid(S.m.g), MG_BLOCK, 0, S.s>>>(x, S.w.x32, S.m.g);
    if ((st = after_launch("k_acc64"))) break;
    if ((st = S.D64(S.w.r64, x))) break;
    if ((st = S.axpby<LQCD_F64>(S.w.r64, b, 1.0, 0.0, nullptr, -1.0))) break;
  }
  if (S.vgraph) cudaGraphExecDestroy(S.vgraph);
  inf->iterations = iters;
  inf->true_rel_residual = rel;
  if (st) return finish(st);
  if (status != LQCD_OK) return finish(fail(LQCD_ERR_NOT_CONVERGED, "multigrid: maxiter %d reached", prm->maxiter));
  return finish(LQCD_OK);
}

}  // extern "C"
