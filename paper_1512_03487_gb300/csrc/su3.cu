// Fields of 3x3 complex (colour) matrices and their site-by-site product
// z(x) = x(x) y(x): the SU(3) x SU(3) kernel the Grid paper benchmarks first
// (Sec. 5, performance against memory footprint). One thread per site; the
// field is streamed once (two matrices read, one written), so the kernel is
// bound by HBM bandwidth beyond the L2 size and by L2 below it.
//
// Device layout (structure of arrays, site fastest, stride = n rounded up to
// 32 sites): FP64 9 chunks of double2 (entries in row-major order); FP32 4
// chunks of float4 (entries 0-7, two per chunk) then 1 chunk of float2
// (entry 8): 72 bytes per site in 5 coalesced loads.
#include "lqcd_internal.h"

namespace lqcd {

constexpr int SU3_BLOCK = 256;

template <typename T> struct CMat {
  cpx<T> e[9];
};

template <int P> struct CMatIO;

template <> struct CMatIO<LQCD_F64> {
  using T = double;
  static __device__ __forceinline__ void load(const void* base, int64_t stride, int64_t i, CMat<T>& m) {
    const double2* b = static_cast<const double2*>(base);
#pragma unroll
    for (int c = 0; c < 9; c++) {
      const double2 w = __ldg(b + c * stride + i);
      m.e[c] = mk(w.x, w.y);
    }
  }
  static __device__ __forceinline__ void store(void* base, int64_t stride, int64_t i, const CMat<T>& m) {
    double2* b = static_cast<double2*>(base);
#pragma unroll
    for (int c = 0; c < 9; c++) __stcs(b + c * stride + i, make_double2(m.e[c].r, m.e[c].i));
  }
};

template <> struct CMatIO<LQCD_F32> {
  using T = float;
  static __device__ __forceinline__ const float2* tail(const void* base, int64_t stride) {
    return reinterpret_cast<const float2*>(static_cast<const float4*>(base) + 4 * stride);
  }
  static __device__ __forceinline__ void load(const void* base, int64_t stride, int64_t i, CMat<T>& m) {
    const float4* b = static_cast<const float4*>(base);
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const float4 w = __ldg(b + c * stride + i);
      m.e[2 * c] = mk(w.x, w.y);
      m.e[2 * c + 1] = mk(w.z, w.w);
    }
    const float2 w = __ldg(tail(base, stride) + i);
    m.e[8] = mk(w.x, w.y);
  }
  static __device__ __forceinline__ void store(void* base, int64_t stride, int64_t i, const CMat<T>& m) {
    float4* b = static_cast<float4*>(base);
#pragma unroll
    for (int c = 0; c < 4; c++)
      __stcs(b + c * stride + i, make_float4(m.e[2 * c].r, m.e[2 * c].i, m.e[2 * c + 1].r, m.e[2 * c + 1].i));
    __stcs(const_cast<float2*>(tail(base, stride)) + i, make_float2(m.e[8].r, m.e[8].i));
  }
};

// z = x y: z_ik = sum_j x_ij y_jk
template <typename T>
__device__ __forceinline__ void cmat_mul(const CMat<T>& x, const CMat<T>& y, CMat<T>& z) {
#pragma unroll
  for (int i = 0; i < 3; i++) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      cpx<T> acc = cmul(x.e[3 * i], y.e[k]);
      acc = cmadd(acc, x.e[3 * i + 1], y.e[3 + k]);
      acc = cmadd(acc, x.e[3 * i + 2], y.e[6 + k]);
      z.e[3 * i + k] = acc;
    }
  }
}

template <int P>
__global__ void __launch_bounds__(SU3_BLOCK) su3_mul_kernel(void* z, const void* x, const void* y, int64_t n,
                                                            int64_t stride) {
  using T = typename PrecTraits<P>::real;
  const int64_t i = (int64_t)blockIdx.x * SU3_BLOCK + threadIdx.x;
  if (i >= n) return;
  CMat<T> a, b, c;
  CMatIO<P>::load(x, stride, i, a);
  CMatIO<P>::load(y, stride, i, b);
  cmat_mul(a, b, c);
  CMatIO<P>::store(z, stride, i, c);
}

// host layout [site][row][col] complex FP64 <-> device layout
template <int P>
__global__ void __launch_bounds__(SU3_BLOCK) cmat_xfer_kernel(bool pack, void* dev, double* host, int64_t n,
                                                              int64_t stride) {
  using T = typename PrecTraits<P>::real;
  const int64_t i = (int64_t)blockIdx.x * SU3_BLOCK + threadIdx.x;
  if (i >= n) return;
  double2* h = reinterpret_cast<double2*>(host) + i * 9;
  CMat<T> m;
  if (pack) {
#pragma unroll
    for (int c = 0; c < 9; c++) {
      const double2 w = h[c];
      m.e[c] = mk((T)w.x, (T)w.y);
    }
    CMatIO<P>::store(dev, stride, i, m);
  } else {
    CMatIO<P>::load(dev, stride, i, m);
#pragma unroll
    for (int c = 0; c < 9; c++) h[c] = make_double2((double)m.e[c].r, (double)m.e[c].i);
  }
}

static int cmat_sites(const lqcd_lattice* lat, int prec, int64_t* n, int64_t* stride) {
  Geom g;
  int st = make_geom(lat, &g);
  if (st) return st;
  if (prec != LQCD_F64 && prec != LQCD_F32)
    return fail(LQCD_ERR_ARG, "colour-matrix fields are LQCD_F64 or LQCD_F32 (got %d)", prec);
  *n = 2 * g.Vh * (int64_t)g.n5;
  *stride = round_up(*n, 32);
  return LQCD_OK;
}

static bool misaligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) != 0; }

static int cmat_xfer(bool pack, void* dev, double* host, int prec, const lqcd_lattice* lat, cudaStream_t s) {
  int64_t n, stride;
  int st = cmat_sites(lat, prec, &n, &stride);
  if (st) return st;
  if (!dev || !host || misaligned16(dev) || misaligned16(host))
    return fail(LQCD_ERR_ARG, "colour matrix %s: null or misaligned pointer", pack ? "pack" : "unpack");
  const unsigned grid = (unsigned)((n + SU3_BLOCK - 1) / SU3_BLOCK);
  if (prec == LQCD_F64) cmat_xfer_kernel<LQCD_F64><<<grid, SU3_BLOCK, 0, s>>>(pack, dev, host, n, stride);
  else cmat_xfer_kernel<LQCD_F32><<<grid, SU3_BLOCK, 0, s>>>(pack, dev, host, n, stride);
  return after_launch("cmat_xfer_kernel");
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

size_t lqcd_colour_matrix_bytes(const lqcd_lattice* lat, int prec) {
  int64_t n, stride;
  if (cmat_sites(lat, prec, &n, &stride) != LQCD_OK) return 0;
  return (size_t)stride * (prec == LQCD_F64 ? 144 : 72);
}

int lqcd_colour_matrix_pack(void* dst, int prec, const double* src, const lqcd_lattice* lat, void* stream) {
  return cmat_xfer(true, dst, const_cast<double*>(src), prec, lat, (cudaStream_t)stream);
}

int lqcd_colour_matrix_unpack(double* dst, const void* src, int prec, const lqcd_lattice* lat, void* stream) {
  return cmat_xfer(false, const_cast<void*>(src), dst, prec, lat, (cudaStream_t)stream);
}

int lqcd_su3_mul(void* z, const void* x, const void* y, const lqcd_lattice* lat, int prec, void* stream) {
  int64_t n, stride;
  int st = cmat_sites(lat, prec, &n, &stride);
  if (st) return st;
  if (!z || !x || !y || misaligned16(z) || misaligned16(x) || misaligned16(y))
    return fail(LQCD_ERR_ARG, "lqcd_su3_mul: null or misaligned pointer");
  const unsigned grid = (unsigned)((n + SU3_BLOCK - 1) / SU3_BLOCK);
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == LQCD_F64) su3_mul_kernel<LQCD_F64><<<grid, SU3_BLOCK, 0, s>>>(z, x, y, n, stride);
  else su3_mul_kernel<LQCD_F32><<<grid, SU3_BLOCK, 0, s>>>(z, x, y, n, stride);
  return after_launch("su3_mul_kernel");
}

}  // extern "C"
