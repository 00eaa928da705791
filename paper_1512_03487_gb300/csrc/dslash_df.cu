// Hop kernel instantiations for FP64 fields with double-float arithmetic
// (LQCD_F64_DF): the Wilson epilogues without reductions, and for 18-real
// links the domain-wall M5op and fused M5op^-1 epilogues: all that the
// reliable updates and the even-odd helpers apply.
#include "dslash_launch.cuh"

namespace lqcd {

template <bool DAG, int R>
static int launch_df_epi(int epi, const HopArgs& a, cudaStream_t s) {
  if (epi == EPI_PLAIN) return launch_hop_inst<LQCD_F64_DF, R, DAG, EPI_PLAIN, RED_NONE, false>(a, s);
  if (epi == EPI_XPAY) return launch_hop_inst<LQCD_F64_DF, R, DAG, EPI_XPAY, RED_NONE, false>(a, s);
  if constexpr (R == 18) {
    if (epi == EPI_M5) return launch_hop_inst<LQCD_F64_DF, R, DAG, EPI_M5, RED_NONE, false>(a, s);
    if (epi == EPI_M5INV) return launch_hop_inst<LQCD_F64_DF, R, DAG, EPI_M5INV, RED_NONE, false>(a, s);
  }
  return fail(LQCD_ERR_UNSUPPORTED, "double-float hop: epilogue %d with %d-real links", epi, R);
}

int launch_hop_df(int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s) {
  if (reduce != RED_NONE) return fail(LQCD_ERR_UNSUPPORTED, "double-float hop with a reduction");
  if (recon == 18) return dagger ? launch_df_epi<true, 18>(epi, a, s) : launch_df_epi<false, 18>(epi, a, s);
  if (recon == 12) return dagger ? launch_df_epi<true, 12>(epi, a, s) : launch_df_epi<false, 12>(epi, a, s);
  return fail(LQCD_ERR_ARG, "bad recon %d", recon);
}

}  // namespace lqcd
