// Layout transformation between the user's lexicographic AoS FP64 layout and
// the device SoA checkerboard layout (the Grid paper's central idea, Sec. 2.4:
// the layout is hidden behind the container and transformed to suit the
// hardware), with precision conversion and optional 12-real link compression
// (the paper's Compressor changes precision, Sec. 2.6).
#include <cstring>

#include "lqcd_internal.h"

namespace lqcd {

constexpr int PACK_BLOCK = 128;

// Host-layout site index of device site j (cb * n5 + i5) of checkerboard `parity`.
__device__ __forceinline__ int64_t host_site(const Geom& g, int64_t j, int parity, bool full) {
  const int64_t n5 = g.n5;
  const int64_t cb = j / n5, i5 = j - cb * n5;
  if (!full) return i5 * g.Vh + cb;
  const Coord x = cb_to_coord(g, cb, parity);
  return i5 * (2 * (int64_t)g.Vh) + x.lex;
}

template <int P>
__global__ void spinor_pack_kernel(void* dst, const double* src, Geom g, int parity, int full,
                                   int blocks_per_parity, int64_t half_bytes) {
  using T = typename PrecTraits<P>::real;
  int blk = blockIdx.x;
  if (full) {
    parity = blk >= blocks_per_parity ? 1 : 0;
    blk -= parity * blocks_per_parity;
  }
  const int64_t j = (int64_t)blk * PACK_BLOCK + threadIdx.x;
  if (j >= g.nsites) return;
  const double* s = src + host_site(g, j, parity, full) * 24;
  Spinor<T> v;
#pragma unroll
  for (int k = 0; k < 12; k++) v.v[k] = mk((T)s[2 * k], (T)s[2 * k + 1]);
  char* d = static_cast<char*>(dst) + (full ? parity * half_bytes : 0);
  SpinorIO<P>::store(d, g.sstride, j, v);
}

template <int P>
__global__ void spinor_unpack_kernel(double* dst, const void* src, Geom g, int parity, int full,
                                     int blocks_per_parity, int64_t half_bytes) {
  using T = typename PrecTraits<P>::real;
  int blk = blockIdx.x;
  if (full) {
    parity = blk >= blocks_per_parity ? 1 : 0;
    blk -= parity * blocks_per_parity;
  }
  const int64_t j = (int64_t)blk * PACK_BLOCK + threadIdx.x;
  if (j >= g.nsites) return;
  const char* sp = static_cast<const char*>(src) + (full ? parity * half_bytes : 0);
  Spinor<T> v;
  SpinorIO<P>::load(sp, g.sstride, j, v);
  double* d = dst + host_site(g, j, parity, full) * 24;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    d[2 * k] = (double)v.v[k].r;
    d[2 * k + 1] = (double)v.v[k].i;
  }
}

// Gauge element addressing: real r of the stored link lives in chunk r / per
// at lane r % per; chunk c of block (parity, mu) at ((blk * nchunk + c) * gstride + cb).
struct LinkFmt {
  int esize;   // bytes per real
  int per;     // reals per chunk
  int nchunk;  // chunks per link
  int nreal;   // stored reals (18 or 12)
};
static LinkFmt link_fmt(int prec, int recon) {
  LinkFmt f;
  f.nreal = recon == 12 ? 12 : 18;
  f.esize = prec == LQCD_F64 ? 8 : prec == LQCD_F32 ? 4 : 2;
  f.per = (prec == LQCD_F64 || recon == 18) ? 2 : 4;
  f.nchunk = f.nreal / f.per;
  return f;
}

__global__ void gauge_pack_kernel(void* dst, const double* src, Geom g, LinkFmt f, int prec) {
  // one thread per (parity, mu, cb)
  const int64_t t = (int64_t)blockIdx.x * PACK_BLOCK + threadIdx.x;
  const int64_t n = 8 * (int64_t)g.Vh;
  if (t >= n) return;
  const int64_t cb = t % g.Vh;
  const int blk = (int)(t / g.Vh);  // parity * 4 + mu
  const int parity = blk >> 2, mu = blk & 3;
  const Coord x = cb_to_coord(g, cb, parity);
  const double* s = src + (x.lex * 4 + mu) * 18;
  char* base = static_cast<char*>(dst);
  const int chunk_bytes = f.esize * f.per;
  for (int r = 0; r < f.nreal; r++) {
    const int c = r / f.per, lane = r % f.per;
    char* p = base + ((int64_t)(blk * f.nchunk + c) * g.gstride + cb) * chunk_bytes + lane * f.esize;
    const double v = s[r];
    if (prec == LQCD_F64) *reinterpret_cast<double*>(p) = v;
    else if (prec == LQCD_F32) *reinterpret_cast<float*>(p) = (float)v;
    else *reinterpret_cast<__half*>(p) = __double2half(v);
  }
}

template <int P, int R>
__global__ void gauge_unpack_kernel(double* dst, const void* src, Geom g) {
  using T = typename PrecTraits<P>::real;
  const int64_t t = (int64_t)blockIdx.x * PACK_BLOCK + threadIdx.x;
  const int64_t n = 8 * (int64_t)g.Vh;
  if (t >= n) return;
  const int64_t cb = t % g.Vh;
  const int blk = (int)(t / g.Vh);
  const int parity = blk >> 2, mu = blk & 3;
  const Coord x = cb_to_coord(g, cb, parity);
  Link<T> u;
  LinkIO<P, R>::load(src, g.gstride, blk, cb, u);
  double* d = dst + (x.lex * 4 + mu) * 18;
#pragma unroll
  for (int k = 0; k < 9; k++) {
    d[2 * k] = (double)u.v[k].r;
    d[2 * k + 1] = (double)u.v[k].i;
  }
}

static bool misaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) != 0; }

static int spinor_xfer(bool pack, void* dev, double* aos, int prec, int subset, const lqcd_lattice* lat,
                       cudaStream_t s) {
  Geom g;
  int st = make_geom(lat, &g);
  if (st) return st;
  if (spinor_site_bytes(prec) == 0) return fail(LQCD_ERR_ARG, "bad precision %d", prec);
  if (subset != LQCD_EVEN && subset != LQCD_ODD && subset != LQCD_FULL)
    return fail(LQCD_ERR_ARG, "bad subset %d", subset);
  if (!dev || !aos || misaligned(dev) || (reinterpret_cast<uintptr_t>(aos) & 7))
    return fail(LQCD_ERR_ARG, "spinor pack/unpack: null or misaligned pointer");
  const bool full = subset == LQCD_FULL;
  const int bpp = (int)((g.nsites + PACK_BLOCK - 1) / PACK_BLOCK);
  const unsigned grid = (unsigned)(full ? 2 * bpp : bpp);
  const int parity = full ? 0 : subset;
  const int64_t hb = (int64_t)cb_spinor_bytes(g, prec);
  if (grid == 0) return LQCD_OK;
#define LQCD_SPINOR_XFER(PR)                                                                             \
  if (pack) spinor_pack_kernel<PR><<<grid, PACK_BLOCK, 0, s>>>(dev, aos, g, parity, full, bpp, hb);     \
  else spinor_unpack_kernel<PR><<<grid, PACK_BLOCK, 0, s>>>(aos, dev, g, parity, full, bpp, hb);
  switch (prec) {
    case LQCD_F64: LQCD_SPINOR_XFER(LQCD_F64) break;
    case LQCD_F32: LQCD_SPINOR_XFER(LQCD_F32) break;
    case LQCD_F16: LQCD_SPINOR_XFER(LQCD_F16) break;
  }
#undef LQCD_SPINOR_XFER
  return after_launch(pack ? "spinor_pack_kernel" : "spinor_unpack_kernel");
}

static int gauge_xfer(bool pack, void* dev, double* aos, int prec, int recon, const lqcd_lattice* lat,
                      cudaStream_t s) {
  Geom g;
  int st = make_geom(lat, &g);
  if (st) return st;
  if (spinor_site_bytes(prec) == 0 || (recon != 18 && recon != 12))
    return fail(LQCD_ERR_ARG, "bad gauge format prec=%d recon=%d", prec, recon);
  if (!dev || !aos || misaligned(dev) || (reinterpret_cast<uintptr_t>(aos) & 7))
    return fail(LQCD_ERR_ARG, "gauge pack/unpack: null or misaligned pointer");
  const int64_t n = 8 * (int64_t)g.Vh;
  const unsigned grid = (unsigned)((n + PACK_BLOCK - 1) / PACK_BLOCK);
  if (pack) {
    gauge_pack_kernel<<<grid, PACK_BLOCK, 0, s>>>(dev, aos, g, link_fmt(prec, recon), prec);
  } else {
#define LQCD_GAUGE_UNPACK(PR, RC) gauge_unpack_kernel<PR, RC><<<grid, PACK_BLOCK, 0, s>>>(aos, dev, g)
    if (prec == LQCD_F64) { if (recon == 18) LQCD_GAUGE_UNPACK(LQCD_F64, 18); else LQCD_GAUGE_UNPACK(LQCD_F64, 12); }
    if (prec == LQCD_F32) { if (recon == 18) LQCD_GAUGE_UNPACK(LQCD_F32, 18); else LQCD_GAUGE_UNPACK(LQCD_F32, 12); }
    if (prec == LQCD_F16) { if (recon == 18) LQCD_GAUGE_UNPACK(LQCD_F16, 18); else LQCD_GAUGE_UNPACK(LQCD_F16, 12); }
#undef LQCD_GAUGE_UNPACK
  }
  return after_launch(pack ? "gauge_pack_kernel" : "gauge_unpack_kernel");
}

static size_t host_spinor_bytes(const Geom& g, int subset) {
  return (size_t)g.nsites * (subset == LQCD_FULL ? 2 : 1) * 24 * sizeof(double);
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

int lqcd_spinor_pack(void* dst, int prec, int subset, const double* src, const lqcd_lattice* lat, void* stream) {
  return spinor_xfer(true, dst, const_cast<double*>(src), prec, subset, lat, (cudaStream_t)stream);
}

int lqcd_spinor_unpack(double* dst, const void* src, int prec, int subset, const lqcd_lattice* lat, void* stream) {
  return spinor_xfer(false, const_cast<void*>(src), dst, prec, subset, lat, (cudaStream_t)stream);
}

int lqcd_gauge_pack(void* dst, int prec, int recon, const double* src, const lqcd_lattice* lat, void* stream) {
  return gauge_xfer(true, dst, const_cast<double*>(src), prec, recon, lat, (cudaStream_t)stream);
}

int lqcd_gauge_unpack(double* dst, const void* src, int prec, int recon, const lqcd_lattice* lat, void* stream) {
  return gauge_xfer(false, const_cast<void*>(src), dst, prec, recon, lat, (cudaStream_t)stream);
}

int lqcd_spinor_upload(void* dst, int prec, int subset, const double* src_host, double* staging,
                       const lqcd_lattice* lat, void* stream) {
  Geom g;
  int st = make_geom(lat, &g);
  if (st) return st;
  if (!src_host || !staging) return fail(LQCD_ERR_ARG, "lqcd_spinor_upload: null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(staging, src_host, host_spinor_bytes(g, subset), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "lqcd_spinor_upload memcpy");
  return lqcd_spinor_pack(dst, prec, subset, staging, lat, stream);
}

int lqcd_spinor_download(double* dst_host, const void* src, int prec, int subset, double* staging,
                         const lqcd_lattice* lat, void* stream) {
  Geom g;
  int st = make_geom(lat, &g);
  if (st) return st;
  if (!dst_host || !staging) return fail(LQCD_ERR_ARG, "lqcd_spinor_download: null pointer");
  if ((st = lqcd_spinor_unpack(staging, src, prec, subset, lat, stream))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(dst_host, staging, host_spinor_bytes(g, subset), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "lqcd_spinor_download memcpy");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "lqcd_spinor_download sync");
  return LQCD_OK;
}

int lqcd_gauge_upload(void* dst, int prec, int recon, const double* src_host, double* staging,
                      const lqcd_lattice* lat, void* stream) {
  Geom g;
  int st = make_geom(lat, &g);
  if (st) return st;
  if (!src_host || !staging) return fail(LQCD_ERR_ARG, "lqcd_gauge_upload: null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)2 * g.Vh * 4 * 18 * sizeof(double);
  cudaError_t e = cudaMemcpyAsync(staging, src_host, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "lqcd_gauge_upload memcpy");
  return lqcd_gauge_pack(dst, prec, recon, staging, lat, stream);
}

}  // extern "C"
