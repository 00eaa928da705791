// Measurement only, not part of the method or of liblqcd's ABI: register-
// resident FMA chains that give the arithmetic rate, FP64 or FP32, that the
// bench quotes its ALU-bound kernels against (the FP64 hop of the reliable
// updates, the double-float hop, the FP64 SU(3) product, the force) beside the
// rate derived from unit counts and clock. Eight independent chains per thread
// keep the pipe busy at any occupancy; the chains' sums go to `sink` so the
// compiler keeps every FMA. Built as its own library, libfma_probe.so.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

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

}  // namespace

extern "C" {

// `blocks` blocks of 256 threads each run 8 chains of `iters` fused
// multiply-adds in FP64 (prec 0) or FP32 (prec 1) and store one value per
// thread into sink (blocks * 256 elements of that precision, device memory,
// 8-byte aligned): 16 * iters * blocks * 256 flop, asynchronous on `stream`.
// Returns 0, -1 for a bad argument (nothing launched), or the CUDA error code
// of the launch.
int fma_probe(void* sink, int prec, int64_t iters, int blocks, void* stream) {
  if (!sink || iters < 1 || blocks < 1 || ((uintptr_t)sink & 7) != 0 || (prec != 0 && prec != 1)) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  // a slightly below 1 and b small: every chain converges to b / (1 - a) and stays finite
  if (prec == 0) fma_chain_kernel<double><<<blocks, PROBE_BLOCK, 0, s>>>((double*)sink, iters, 0.999999, 1e-6);
  else fma_chain_kernel<float><<<blocks, PROBE_BLOCK, 0, s>>>((float*)sink, iters, 0.9999f, 1e-4f);
  return (int)cudaGetLastError();
}

}  // extern "C"
