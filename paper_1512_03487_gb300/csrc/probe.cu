// Register-resident FMA chains: the arithmetic rate, FP64 or FP32, that the
// ALU-bound kernels (the FP64 hop of the reliable updates, the FP64 SU(3)
// product) are quoted against beside the nominal figure. Eight independent
// chains per thread keep the pipe busy at any occupancy; the chains' sums go
// to `sink` so the compiler keeps every FMA.
#include "lqcd_internal.h"

namespace lqcd {

constexpr int PROBE_BLOCK = 256;

template <typename T>
__global__ void __launch_bounds__(PROBE_BLOCK) fma_chain_kernel(T* sink, int64_t iters, T a, T b) {
  const int64_t tid = (int64_t)blockIdx.x * PROBE_BLOCK + threadIdx.x;
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; k++) x[k] = (T)(tid % 97) * (T)1e-3 + (T)k;
  for (int64_t i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) s += x[k];
  sink[tid] = s;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

int lqcd_fma_probe(void* sink, int prec, int64_t iters, int blocks, void* stream) {
  if (!sink || iters < 1 || blocks < 1) return fail(LQCD_ERR_ARG, "lqcd_fma_probe: bad arguments");
  if (((uintptr_t)sink & 7) != 0) return fail(LQCD_ERR_ARG, "lqcd_fma_probe: sink must be 8-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  // a slightly below 1 and b small: every chain converges to b / (1 - a) and stays finite
  if (prec == LQCD_F64)
    fma_chain_kernel<double><<<blocks, PROBE_BLOCK, 0, s>>>((double*)sink, iters, 0.999999, 1e-6);
  else if (prec == LQCD_F32)
    fma_chain_kernel<float><<<blocks, PROBE_BLOCK, 0, s>>>((float*)sink, iters, 0.9999f, 1e-4f);
  else
    return fail(LQCD_ERR_ARG, "lqcd_fma_probe: precision must be LQCD_F64 or LQCD_F32");
  return after_launch("fma_chain_kernel");
}

}  // extern "C"
