// Hop kernel instantiations with G-parity boundary conditions (FP64 and FP32
// storage, Wilson epilogues), compiled apart from the plain ones.
#include "dslash_launch.cuh"

namespace lqcd {
int launch_hop_gparity(int prec, int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s) {
  if (prec == LQCD_F64) return launch_hop_prec<LQCD_F64, true>(recon, dagger, epi, reduce, a, s);
  if (prec == LQCD_F32) return launch_hop_prec<LQCD_F32, true>(recon, dagger, epi, reduce, a, s);
  return fail(LQCD_ERR_UNSUPPORTED, "G-parity hop with precision %d", prec);
}
}  // namespace lqcd
