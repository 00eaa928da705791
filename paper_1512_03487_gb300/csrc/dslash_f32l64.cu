// Hop kernel instantiations with FP32 spinors and arithmetic on FP64 links:
// the operator of the intermediate (FP32-accurate) residual replacement of the
// three-level mixed-precision CG and of the CGNR start M^dag b. Plain, xpay,
// M5 and M5op^-1 epilogues (G-parity: plain and xpay), no reduction.
#include "lqcd_internal.h"

namespace lqcd {

template <int R, bool DAG, int EPI, bool GP>
static int launch_f32l64_inst(const HopArgs& a, cudaStream_t s) {
  const int64_t nb = (a.g.nsites + HOP_BLOCK - 1) / HOP_BLOCK;
  const int64_t grid = a.full ? 2 * nb : nb;
  if (grid == 0) return LQCD_OK;
  hop_kernel<LQCD_F32, R, DAG, EPI, RED_NONE, HOP_BLOCK, GP, LQCD_F64><<<(unsigned)grid, HOP_BLOCK, 0, s>>>(a);
  return after_launch("hop_kernel (FP64 links)");
}

template <int R, bool DAG, bool GP>
static int launch_f32l64_epi(int epi, const HopArgs& a, cudaStream_t s) {
  if (epi == EPI_PLAIN) return launch_f32l64_inst<R, DAG, EPI_PLAIN, GP>(a, s);
  if (epi == EPI_XPAY) return launch_f32l64_inst<R, DAG, EPI_XPAY, GP>(a, s);
  if (!GP && epi == EPI_M5) return launch_f32l64_inst<R, DAG, GP ? EPI_XPAY : EPI_M5, GP>(a, s);
  if (!GP && epi == EPI_M5INV) return launch_f32l64_inst<R, DAG, GP ? EPI_PLAIN : EPI_M5INV, GP>(a, s);
  return fail(LQCD_ERR_ARG, "bad epilogue %d", epi);
}

template <int R, bool DAG>
static int launch_f32l64_gp(int epi, const HopArgs& a, cudaStream_t s) {
  return a.g.gp ? launch_f32l64_epi<R, DAG, true>(epi, a, s) : launch_f32l64_epi<R, DAG, false>(epi, a, s);
}

int launch_hop_f32_link64(int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s) {
  if (reduce != RED_NONE) return fail(LQCD_ERR_UNSUPPORTED, "FP64-link hop with a reduction");
  a.blocks_per_parity = (int)((a.g.nsites + HOP_BLOCK - 1) / HOP_BLOCK);
  if (recon == 18)
    return dagger ? launch_f32l64_gp<18, true>(epi, a, s) : launch_f32l64_gp<18, false>(epi, a, s);
  if (recon == 12)
    return dagger ? launch_f32l64_gp<12, true>(epi, a, s) : launch_f32l64_gp<12, false>(epi, a, s);
  return fail(LQCD_ERR_ARG, "bad recon %d", recon);
}

}  // namespace lqcd
