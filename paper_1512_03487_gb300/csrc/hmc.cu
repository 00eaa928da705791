// Wilson gauge action, its force, the SU(3) link update and the hybrid Monte
// Carlo trajectory (the Grid paper lists HMC, the Wilson gauge action and the
// leapfrog and minimum-norm integrators among its algorithms, Sec. 4; the
// formulas are the textbook ones):
//
//   S_g = beta sum_{x, mu<nu} (1 - Re tr U_munu(x) / 3), periodic boundaries,
//   Sigma_mu(x) = sum_{nu != mu} [ U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
//                                + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) ],
//   F_mu(x) = (beta / 3) * traceless part of (W - W^dag) / (2 i), W = U_mu(x) Sigma_mu(x),
//   so that dS_g = eps tr(T F) under U -> exp(i eps T) U (the convention of lqcd_force);
//   molecular dynamics: dU/dt = i P U, dP/dt = -(F_g + F_f).
//
// Gauge and momentum fields are FP64 with all 18 reals stored, in the device
// layout [parity][mu][9 chunks of double2][cb]. Every kernel has one thread
// per site (both parities, parity-major) or per link. Reductions are the
// library's deterministic block partials summed in a fixed order by the last
// block. The trajectory driver runs on the host: each momentum step launches
// the gauge-force kernel and, with fermions, one conjugate-gradient solve
// (lqcd_cg_solve, which synchronises), M X and the fermion-force kernel in
// accumulate mode.
#include <cmath>
#include <cstring>

#include "lqcd_internal.h"

namespace lqcd {

constexpr int HMC_BLOCK = 128;
using M3 = Link<double>;

// ------------------------------------------------------------------ 3x3 algebra

__device__ __forceinline__ void m_mul(const M3& a, const M3& b, M3& c) {  // c = a b
#pragma unroll
  for (int r = 0; r < 3; r++)
#pragma unroll
    for (int k = 0; k < 3; k++) {
      cpx<double> s = cmul(a.v[3 * r], b.v[k]);
      s = cmadd(s, a.v[3 * r + 1], b.v[3 + k]);
      c.v[3 * r + k] = cmadd(s, a.v[3 * r + 2], b.v[6 + k]);
    }
}

__device__ __forceinline__ void m_mul_nd(const M3& a, const M3& b, M3& c) {  // c = a b^dag
#pragma unroll
  for (int r = 0; r < 3; r++)
#pragma unroll
    for (int k = 0; k < 3; k++) {
      cpx<double> s = cmul(a.v[3 * r], conj(b.v[3 * k]));
      s = cmadd(s, a.v[3 * r + 1], conj(b.v[3 * k + 1]));
      c.v[3 * r + k] = cmadd(s, a.v[3 * r + 2], conj(b.v[3 * k + 2]));
    }
}

__device__ __forceinline__ void m_mul_dn(const M3& a, const M3& b, M3& c) {  // c = a^dag b
#pragma unroll
  for (int r = 0; r < 3; r++)
#pragma unroll
    for (int k = 0; k < 3; k++) {
      cpx<double> s = cmul(conj(a.v[r]), b.v[k]);
      s = cmadd(s, conj(a.v[3 + r]), b.v[3 + k]);
      c.v[3 * r + k] = cmadd(s, conj(a.v[6 + r]), b.v[6 + k]);
    }
}

__device__ __forceinline__ void m_add(M3& a, const M3& b) {
#pragma unroll
  for (int k = 0; k < 9; k++) a.v[k] = a.v[k] + b.v[k];
}

__device__ __forceinline__ void m_identity(M3& a) {
#pragma unroll
  for (int k = 0; k < 9; k++) a.v[k] = mk(k % 4 == 0 ? 1.0 : 0.0, 0.0);
}

// ------------------------------------------------------------------ link access by coordinate

__device__ __forceinline__ void link_at(const Geom& g, const void* U, int mu, const int c[4], M3& u) {
  const uint32_t lex = (uint32_t)c[0] + (uint32_t)g.X * ((uint32_t)c[1] + (uint32_t)g.Y *
                                                         ((uint32_t)c[2] + (uint32_t)g.Z * (uint32_t)c[3]));
  const int parity = (c[0] + c[1] + c[2] + c[3]) & 1;
  LinkIO<LQCD_F64, 18>::load(U, g.gstride, parity * 4 + mu, (int64_t)(lex >> 1), u);
}

__device__ __forceinline__ int extent(const Geom& g, int mu) {
  return mu == 0 ? g.X : mu == 1 ? g.Y : mu == 2 ? g.Z : g.T;
}

// c + d * mu_hat with periodic wrap (|d| <= 1)
__device__ __forceinline__ void step(const Geom& g, const int c[4], int mu, int d, int out[4]) {
#pragma unroll
  for (int k = 0; k < 4; k++) out[k] = c[k];
  const int L = extent(g, mu);
  int v = c[mu] + d;
  out[mu] = v < 0 ? v + L : (v >= L ? v - L : v);
}

__device__ __forceinline__ double2* link_ptr(double2* base, const Geom& g, int parity, int mu, int64_t cb) {
  return base + (int64_t)(parity * 4 + mu) * 9 * g.gstride + cb;
}

__device__ __forceinline__ void store_link(double2* base, const Geom& g, int parity, int mu, int64_t cb, const M3& u) {
  double2* p = link_ptr(base, g, parity, mu, cb);
#pragma unroll
  for (int k = 0; k < 9; k++) p[k * g.gstride] = make_double2(u.v[k].r, u.v[k].i);
}

// thread -> (parity, cb, coordinates) over both checkerboards
__device__ __forceinline__ bool site_of_thread(const Geom& g, int64_t t, int& parity, int64_t& cb, int c[4]) {
  if (t >= 2 * (int64_t)g.Vh) return false;
  parity = t >= g.Vh ? 1 : 0;
  cb = t - parity * (int64_t)g.Vh;
  const Coord x = cb_to_coord(g, cb, parity);
#pragma unroll
  for (int k = 0; k < 4; k++) c[k] = x.c[k];
  return true;
}

// ------------------------------------------------------------------ kernels

// sum over the six planes of Re tr U_munu(x) / 3 at each site, reduced
__global__ void __launch_bounds__(HMC_BLOCK) plaquette_kernel(const void* U, Geom g, ReduceCtx rc) {
  const int64_t t = (int64_t)blockIdx.x * HMC_BLOCK + threadIdx.x;
  int parity, c[4];
  int64_t cb;
  double v = 0.0;
  if (site_of_thread(g, t, parity, cb, c)) {
    for (int mu = 0; mu < 4; mu++)
      for (int nu = mu + 1; nu < 4; nu++) {
        int cm[4], cn[4];
        step(g, c, mu, +1, cm);
        step(g, c, nu, +1, cn);
        M3 a, b, p, q;
        link_at(g, U, mu, c, a);
        link_at(g, U, nu, cm, b);
        m_mul(a, b, p);  // U_mu(x) U_nu(x+mu)
        link_at(g, U, nu, c, a);
        link_at(g, U, mu, cn, b);
        m_mul(a, b, q);  // U_nu(x) U_mu(x+nu)
        double tr = 0.0;  // Re tr(p q^dag)
#pragma unroll
        for (int k = 0; k < 9; k++) tr += p.v[k].r * q.v[k].r + p.v[k].i * q.v[k].i;
        v += tr / 3.0;
      }
  }
  block_reduce_finalize<HMC_BLOCK>(v, (int64_t)blockIdx.x * HMC_BLOCK, rc);
}

// F_mu(x) of the Wilson gauge action; out = F, or out -= coef F (accumulate)
__global__ void __launch_bounds__(HMC_BLOCK) gauge_force_kernel(double2* out, const void* U, Geom g, double beta,
                                                                double coef, int accumulate) {
  const int64_t t = (int64_t)blockIdx.x * HMC_BLOCK + threadIdx.x;
  int parity, c[4];
  int64_t cb;
  if (!site_of_thread(g, t, parity, cb, c)) return;
  for (int mu = 0; mu < 4; mu++) {
    M3 S;
#pragma unroll
    for (int k = 0; k < 9; k++) S.v[k] = mk(0.0, 0.0);
    int cm[4];
    step(g, c, mu, +1, cm);
    for (int nu = 0; nu < 4; nu++) {
      if (nu == mu) continue;
      int cn[4], cmn[4], cmm[4];
      step(g, c, nu, +1, cn);
      step(g, c, nu, -1, cmm);   // x - nu
      step(g, cm, nu, -1, cmn);  // x + mu - nu
      M3 a, b, tmp, term;
      // upper staple U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
      link_at(g, U, nu, cm, a);
      link_at(g, U, mu, cn, b);
      m_mul_nd(a, b, tmp);
      link_at(g, U, nu, c, a);
      m_mul_nd(tmp, a, term);
      m_add(S, term);
      // lower staple U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) = (U_mu(x-nu) U_nu(x+mu-nu))^dag U_nu(x-nu)
      link_at(g, U, mu, cmm, a);
      link_at(g, U, nu, cmn, b);
      m_mul(a, b, tmp);
      link_at(g, U, nu, cmm, a);
      m_mul_dn(tmp, a, term);
      m_add(S, term);
    }
    M3 u, W;
    link_at(g, U, mu, c, u);
    m_mul(u, S, W);
    // F = (beta / 3) traceless[(W - W^dag) / (2 i)]
    M3 F;
    const double f = beta / 3.0;
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const cpx<double> d = W.v[3 * r + k] - conj(W.v[3 * k + r]);
        F.v[3 * r + k] = mk(0.5 * f * d.i, -0.5 * f * d.r);  // d / (2 i) times f
      }
    const double tr = (F.v[0].r + F.v[4].r + F.v[8].r) / 3.0;
    F.v[0].r -= tr;
    F.v[4].r -= tr;
    F.v[8].r -= tr;
    double2* p = link_ptr(out, g, parity, mu, cb);
    if (accumulate) {
#pragma unroll
      for (int k = 0; k < 9; k++) {
        const double2 w = p[k * g.gstride];
        p[k * g.gstride] = make_double2(w.x - coef * F.v[k].r, w.y - coef * F.v[k].i);
      }
    } else {
      store_link(out, g, parity, mu, cb, F);
    }
  }
}

// U <- exp(i eps P) U per link. The exponential of A = i eps P is a Taylor
// series (degree 16, Horner form) of A / 2^s with |A / 2^s|_F <= 1/4, squared s
// times (scaling and squaring); the truncation error is below 1e-18 of |E|.
__global__ void __launch_bounds__(HMC_BLOCK) exp_update_kernel(void* U, const void* P, Geom g, double eps) {
  const int64_t t = (int64_t)blockIdx.x * HMC_BLOCK + threadIdx.x;
  if (t >= 8 * (int64_t)g.Vh) return;
  const int blk = (int)(t / g.Vh);  // parity * 4 + mu
  const int64_t cb = t - (int64_t)blk * g.Vh;
  M3 p, u;
  LinkIO<LQCD_F64, 18>::load(P, g.gstride, blk, cb, p);
  LinkIO<LQCD_F64, 18>::load(U, g.gstride, blk, cb, u);
  double nrm2 = 0.0;
#pragma unroll
  for (int k = 0; k < 9; k++) nrm2 += p.v[k].r * p.v[k].r + p.v[k].i * p.v[k].i;
  double nrm = fabs(eps) * sqrt(nrm2);
  int s = 0;
  while (nrm > 0.25 && s < 60) {
    nrm *= 0.5;
    s++;
  }
  const double sc = ldexp(eps, -s);
  M3 A;
#pragma unroll
  for (int k = 0; k < 9; k++) A.v[k] = mk(-sc * p.v[k].i, sc * p.v[k].r);  // i sc P
  M3 E, T;
  m_identity(E);
  for (int k = 16; k >= 1; k--) {
    m_mul(A, E, T);
    const double ik = 1.0 / k;
#pragma unroll
    for (int q = 0; q < 9; q++) E.v[q] = mk((q % 4 == 0 ? 1.0 : 0.0) + ik * T.v[q].r, ik * T.v[q].i);
  }
  for (int q = 0; q < s; q++) {
    m_mul(E, E, T);
    E = T;
  }
  m_mul(E, u, T);
  double2* base = static_cast<double2*>(U) + (int64_t)blk * 9 * g.gstride + cb;
#pragma unroll
  for (int k = 0; k < 9; k++) base[k * g.gstride] = make_double2(T.v[k].r, T.v[k].i);
}

// sum over the 4 links of a site of tr(P^2) / 2 = |P|_F^2 / 2 (P Hermitian), reduced
__global__ void __launch_bounds__(HMC_BLOCK) kinetic_kernel(const void* P, Geom g, ReduceCtx rc) {
  const int64_t t = (int64_t)blockIdx.x * HMC_BLOCK + threadIdx.x;
  double v = 0.0;
  if (t < 2 * (int64_t)g.Vh) {
    const int parity = t >= g.Vh ? 1 : 0;
    const int64_t cb = t - parity * (int64_t)g.Vh;
    for (int mu = 0; mu < 4; mu++) {
      M3 p;
      LinkIO<LQCD_F64, 18>::load(P, g.gstride, parity * 4 + mu, cb, p);
#pragma unroll
      for (int k = 0; k < 9; k++) v += 0.5 * (p.v[k].r * p.v[k].r + p.v[k].i * p.v[k].i);
    }
  }
  block_reduce_finalize<HMC_BLOCK>(v, (int64_t)blockIdx.x * HMC_BLOCK, rc);
}

// Re <a, b> of two FP64 full spinor fields (n5 == 1), reduced
__global__ void __launch_bounds__(HMC_BLOCK) dot_kernel(const void* a, const void* b, Geom g, int64_t half_bytes,
                                                        ReduceCtx rc) {
  const int64_t t = (int64_t)blockIdx.x * HMC_BLOCK + threadIdx.x;
  double v = 0.0;
  if (t < 2 * (int64_t)g.Vh) {
    const int parity = t >= g.Vh ? 1 : 0;
    const int64_t cb = t - parity * (int64_t)g.Vh;
    Spinor<double> x, y;
    SpinorIO<LQCD_F64>::load(static_cast<const char*>(a) + parity * half_bytes, g.sstride, cb, x);
    SpinorIO<LQCD_F64>::load(static_cast<const char*>(b) + parity * half_bytes, g.sstride, cb, y);
#pragma unroll
    for (int k = 0; k < 12; k++) v += x.v[k].r * y.v[k].r + x.v[k].i * y.v[k].i;
  }
  block_reduce_finalize<HMC_BLOCK>(v, (int64_t)blockIdx.x * HMC_BLOCK, rc);
}

// ------------------------------------------------------------------ host helpers

static unsigned site_grid(const Geom& g) { return (unsigned)((2 * (int64_t)g.Vh + HMC_BLOCK - 1) / HMC_BLOCK); }
static unsigned link_grid(const Geom& g) { return (unsigned)((8 * (int64_t)g.Vh + HMC_BLOCK - 1) / HMC_BLOCK); }

// Reduction scratch: result (1 double), counter, partials (one per block).
struct ReduceWs {
  double* result;
  unsigned int* counter;
  double* partials;
};
static size_t reduce_ws_bytes(const Geom& g) { return 256 + 256 + (size_t)round_up(8 * (int64_t)site_grid(g), 256); }
static ReduceWs reduce_ws(void* base) {
  char* b = static_cast<char*>(base);
  return ReduceWs{reinterpret_cast<double*>(b), reinterpret_cast<unsigned int*>(b + 256),
                  reinterpret_cast<double*>(b + 512)};
}
static ReduceCtx reduce_ctx(const ReduceWs& w) {
  ReduceCtx rc;
  memset(&rc, 0, sizeof(rc));
  rc.partials = w.partials;
  rc.counter = w.counter;
  rc.result = w.result;
  rc.nsys = 1;
  rc.fin = FIN_STORE;
  return rc;
}
static int read_result(const ReduceWs& w, double* out, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(out, w.result, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "hmc: reduction readback");
  return LQCD_OK;
}
static int zero_counter(const ReduceWs& w, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(w.counter, 0, sizeof(unsigned int), s);
  return e == cudaSuccess ? LQCD_OK : cuda_fail(e, "hmc: memset");
}

static int plaquette(const Geom& g, const void* U, const ReduceWs& w, double* out, cudaStream_t s) {
  plaquette_kernel<<<site_grid(g), HMC_BLOCK, 0, s>>>(U, g, reduce_ctx(w));
  int st = after_launch("plaquette_kernel");
  if (st || (st = read_result(w, out, s))) return st;
  *out /= 6.0 * 2.0 * (double)g.Vh;
  return LQCD_OK;
}
static int kinetic(const Geom& g, const void* P, const ReduceWs& w, double* out, cudaStream_t s) {
  kinetic_kernel<<<site_grid(g), HMC_BLOCK, 0, s>>>(P, g, reduce_ctx(w));
  int st = after_launch("kinetic_kernel");
  if (st) return st;
  return read_result(w, out, s);
}
static int gauge_force(const Geom& g, double2* out, const void* U, double beta, double coef, int acc,
                       cudaStream_t s) {
  gauge_force_kernel<<<site_grid(g), HMC_BLOCK, 0, s>>>(out, U, g, beta, coef, acc);
  return after_launch("gauge_force_kernel");
}
static int exp_update(const Geom& g, void* U, const void* P, double eps, cudaStream_t s) {
  exp_update_kernel<<<link_grid(g), HMC_BLOCK, 0, s>>>(U, P, g, eps);
  return after_launch("exp_update_kernel");
}

static bool mis16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) != 0; }

// ------------------------------------------------------------------ trajectory

struct HmcWs {
  ReduceWs red;
  void* X;        // FP64 full spinor
  void* Y;        // FP64 full spinor
  double* stage;  // host-layout FP64 gauge field (sloppy link refresh)
  void* gs;       // sloppy gauge field
  void* cg;       // CG workspace
  size_t cg_bytes;
  size_t total;
};

static HmcWs carve(void* base, const Geom& g, const lqcd_lattice* lat, const lqcd_operator* op,
                   const lqcd_solver_params* prm) {
  HmcWs w;
  memset(&w, 0, sizeof(w));
  size_t o = 0;
  char* b = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> void* {
    void* r = b ? b + o : nullptr;
    o += round_up((int64_t)bytes, 256);
    return r;
  };
  w.red = reduce_ws(take(reduce_ws_bytes(g)));
  const size_t sp = 2 * cb_spinor_bytes(g, LQCD_F64);
  w.X = take(sp);
  w.Y = take(sp);
  if (prm->sloppy_prec != LQCD_F64) {
    w.stage = static_cast<double*>(take((size_t)8 * g.Vh * 18 * sizeof(double)));
    w.gs = take(lqcd_gauge_bytes(lat, prm->sloppy_prec, prm->sloppy_recon));
  }
  w.cg_bytes = lqcd_cg_workspace_bytes(lat, op, prm, LQCD_FULL);
  w.cg = take(w.cg_bytes);
  w.total = o;
  return w;
}

struct Trajectory {
  Geom g;
  const lqcd_lattice* lat;
  const lqcd_operator* op;
  const lqcd_hmc_params* hp;
  const lqcd_solver_params* sp;
  void* U;
  void* P;
  const void* phi;
  HmcWs w;
  cudaStream_t s;
  lqcd_hmc_info* info;

  // X = (M^dag M)^-1 phi on the full lattice; S_f = Re <phi, X>
  int solve(double* sf) {
    const void* gsl = U;
    if (sp->sloppy_prec != LQCD_F64) {
      int st = lqcd_gauge_unpack(w.stage, U, LQCD_F64, 18, lat, s);
      if (st || (st = lqcd_gauge_pack(w.gs, sp->sloppy_prec, sp->sloppy_recon, w.stage, lat, s))) return st;
      gsl = w.gs;
    }
    lqcd_solve_info ci;
    int st = lqcd_cg_solve(w.X, phi, U, gsl, lat, op, sp, LQCD_FULL, &ci, w.cg, w.cg_bytes, s);
    info->cg_iterations += ci.iterations;
    if (st) return st;
    if (sf) {
      if ((st = zero_counter(w.red, s))) return st;
      dot_kernel<<<site_grid(g), HMC_BLOCK, 0, s>>>(phi, w.X, g, (int64_t)cb_spinor_bytes(g, LQCD_F64),
                                                    reduce_ctx(w.red));
      if ((st = after_launch("dot_kernel")) || (st = read_result(w.red, sf, s))) return st;
    }
    return LQCD_OK;
  }

  int energy(double* H, double* K, double* Sg, double* Sf) {
    int st = zero_counter(w.red, s);
    if (st || (st = kinetic(g, P, w.red, K, s))) return st;
    double plaq;
    if ((st = zero_counter(w.red, s)) || (st = plaquette(g, U, w.red, &plaq, s))) return st;
    *Sg = hp->beta * 6.0 * 2.0 * (double)g.Vh * (1.0 - plaq);
    *Sf = 0.0;
    if (hp->fermion && (st = solve(Sf))) return st;
    *H = *K + *Sg + *Sf;
    return LQCD_OK;
  }

  // P <- P - h (F_g + F_f)
  int kick(double h) {
    info->force_evaluations += 1;
    int st = gauge_force(g, static_cast<double2*>(P), U, hp->beta, h, 1, s);
    if (st || !hp->fermion) return st;
    if ((st = solve(nullptr))) return st;
    if ((st = lqcd_M(w.Y, w.X, U, lat, op, LQCD_FULL, 0, nullptr, s))) return st;
    return force_accumulate(static_cast<double2*>(P), U, w.X, w.Y, g, op->recon, h, s);
  }

  int drift(double h) { return exp_update(g, U, P, h, s); }

  int run() {
    int st = energy(&info->H0, &info->kinetic0, &info->gauge0, &info->fermion0);
    if (st) return st;
    const int n = hp->nsteps;
    const double eps = hp->tau / n;
    if (hp->integrator == LQCD_LEAPFROG) {
      if ((st = kick(0.5 * eps))) return st;
      for (int k = 0; k < n; k++) {
        if ((st = drift(eps))) return st;
        if ((st = kick(k < n - 1 ? eps : 0.5 * eps))) return st;
      }
    } else {
      const double lam = 0.1931833275037836;  // Omelyan, Mryglod and Folk (2003)
      if ((st = kick(lam * eps))) return st;
      for (int k = 0; k < n; k++) {
        if ((st = drift(0.5 * eps))) return st;
        if ((st = kick((1.0 - 2.0 * lam) * eps))) return st;
        if ((st = drift(0.5 * eps))) return st;
        if ((st = kick(k < n - 1 ? 2.0 * lam * eps : lam * eps))) return st;
      }
    }
    return energy(&info->H1, &info->kinetic1, &info->gauge1, &info->fermion1);
  }
};

static int hmc_validate(const lqcd_lattice* lat, const lqcd_operator* op, const lqcd_solver_params* prm,
                        Geom* g) {
  int st = make_geom(lat, g);
  if (st) return st;
  if (g->n5 != 1) return fail(LQCD_ERR_ARG, "hmc: n5 must be 1");
  if (!op || !prm) return fail(LQCD_ERR_ARG, "hmc: null operator or solver parameters");
  if ((st = check_operator(op, *g))) return st;
  if (op->kind != LQCD_WILSON || op->prec != LQCD_F64 || op->recon != 18)
    return fail(LQCD_ERR_UNSUPPORTED, "hmc: Wilson operator with FP64, 18-real links");
  if (prm->sloppy_prec != LQCD_F64 && prm->sloppy_prec != LQCD_F32)
    return fail(LQCD_ERR_UNSUPPORTED, "hmc: sloppy precision must be LQCD_F64 or LQCD_F32");
  if (lqcd_cg_workspace_bytes(lat, op, prm, LQCD_FULL) == 0) return fail(LQCD_ERR_ARG, "hmc: bad solver parameters");
  return LQCD_OK;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

size_t lqcd_reduce_workspace_bytes(const lqcd_lattice* lat) {
  Geom g;
  if (make_geom(lat, &g) != LQCD_OK) return 0;
  return reduce_ws_bytes(g);
}

int lqcd_plaquette(double* plaq, const void* U, const lqcd_lattice* lat, void* ws, size_t ws_bytes, void* stream) {
  Geom g;
  int st = make_geom(lat, &g);
  if (st) return st;
  if (!plaq || !U || !ws || mis16(U) || ((uintptr_t)ws & 255)) return fail(LQCD_ERR_ARG, "lqcd_plaquette: pointer");
  if (ws_bytes < reduce_ws_bytes(g)) return fail(LQCD_ERR_WORKSPACE, "lqcd_plaquette: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const ReduceWs w = reduce_ws(ws);
  if ((st = zero_counter(w, s))) return st;
  return plaquette(g, U, w, plaq, s);
}

int lqcd_spinor_dot_re(double* result, const void* a, const void* b, const lqcd_lattice* lat, void* ws,
                       size_t ws_bytes, void* stream) {
  Geom g;
  int st = make_geom(lat, &g);
  if (st) return st;
  if (g.n5 != 1) return fail(LQCD_ERR_UNSUPPORTED, "lqcd_spinor_dot_re: n5 must be 1");
  if (!result || !a || !b || !ws || mis16(a) || mis16(b) || ((uintptr_t)ws & 255))
    return fail(LQCD_ERR_ARG, "lqcd_spinor_dot_re: pointer");
  if (ws_bytes < reduce_ws_bytes(g)) return fail(LQCD_ERR_WORKSPACE, "lqcd_spinor_dot_re: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const ReduceWs w = reduce_ws(ws);
  if ((st = zero_counter(w, s))) return st;
  dot_kernel<<<site_grid(g), HMC_BLOCK, 0, s>>>(a, b, g, (int64_t)cb_spinor_bytes(g, LQCD_F64), reduce_ctx(w));
  if ((st = after_launch("dot_kernel"))) return st;
  return read_result(w, result, s);
}

int lqcd_momentum_kinetic(double* kin, const void* P, const lqcd_lattice* lat, void* ws, size_t ws_bytes,
                          void* stream) {
  Geom g;
  int st = make_geom(lat, &g);
  if (st) return st;
  if (!kin || !P || !ws || mis16(P) || ((uintptr_t)ws & 255))
    return fail(LQCD_ERR_ARG, "lqcd_momentum_kinetic: pointer");
  if (ws_bytes < reduce_ws_bytes(g)) return fail(LQCD_ERR_WORKSPACE, "lqcd_momentum_kinetic: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const ReduceWs w = reduce_ws(ws);
  if ((st = zero_counter(w, s))) return st;
  return kinetic(g, P, w, kin, s);
}

int lqcd_gauge_force(void* out, const void* U, const lqcd_lattice* lat, double beta, void* stream) {
  Geom g;
  int st = make_geom(lat, &g);
  if (st) return st;
  if (!out || !U || mis16(out) || mis16(U) || out == U) return fail(LQCD_ERR_ARG, "lqcd_gauge_force: pointer");
  return gauge_force(g, static_cast<double2*>(out), U, beta, 0.0, 0, (cudaStream_t)stream);
}

int lqcd_gauge_exp_update(void* U, const void* P, double eps, const lqcd_lattice* lat, void* stream) {
  Geom g;
  int st = make_geom(lat, &g);
  if (st) return st;
  if (!U || !P || mis16(U) || mis16(P) || U == P) return fail(LQCD_ERR_ARG, "lqcd_gauge_exp_update: pointer");
  return exp_update(g, U, P, eps, (cudaStream_t)stream);
}

size_t lqcd_hmc_workspace_bytes(const lqcd_lattice* lat, const lqcd_operator* op, const lqcd_solver_params* prm) {
  Geom g;
  if (hmc_validate(lat, op, prm, &g) != LQCD_OK) return 0;
  return carve(nullptr, g, lat, op, prm).total;
}

int lqcd_hmc_trajectory(void* U, void* P, const void* phi, const lqcd_lattice* lat, const lqcd_operator* op,
                        const lqcd_hmc_params* hp, const lqcd_solver_params* prm, lqcd_hmc_info* info, void* ws,
                        size_t ws_bytes, void* stream) {
  lqcd_hmc_info local;
  lqcd_hmc_info* inf = info ? info : &local;
  memset(inf, 0, sizeof(*inf));
  Geom g;
  int st = hmc_validate(lat, op, prm, &g);
  if (!st && !hp) st = fail(LQCD_ERR_ARG, "hmc: null parameters");
  if (!st && (hp->nsteps < 1 || !(hp->tau > 0.0) || (hp->integrator != LQCD_LEAPFROG &&
                                                     hp->integrator != LQCD_MINNORM2)))
    st = fail(LQCD_ERR_ARG, "hmc: nsteps >= 1, tau > 0 and a known integrator required");
  if (!st && (!U || !P || mis16(U) || mis16(P) || (hp->fermion && (!phi || mis16(phi)))))
    st = fail(LQCD_ERR_ARG, "hmc: null or misaligned field");
  if (!st && (!ws || ((uintptr_t)ws & 255))) st = fail(LQCD_ERR_ARG, "hmc: workspace must be 256-byte aligned");
  Trajectory T;
  if (!st) {
    T.w = carve(ws, g, lat, op, prm);
    if (ws_bytes < T.w.total) st = fail(LQCD_ERR_WORKSPACE, "hmc: workspace %zu < %zu bytes", ws_bytes, T.w.total);
  }
  if (!st) {
    T.g = g;
    T.lat = lat;
    T.op = op;
    T.hp = hp;
    T.sp = prm;
    T.U = U;
    T.P = P;
    T.phi = phi;
    T.s = (cudaStream_t)stream;
    T.info = inf;
    st = T.run();
  }
  inf->status = st;
  return st;
}

}  // extern "C"
