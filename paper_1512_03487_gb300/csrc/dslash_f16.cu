// Hop kernel instantiations for LQCD_F16 storage, hops without dagger (the
// dagger ones are in dslash_f16_dag.cu: the two halves compile in parallel).
#include "dslash_launch.cuh"

namespace lqcd {
int launch_hop_f16_dag(int recon, int epi, int reduce, const HopArgs& a, cudaStream_t s);

int launch_hop_f16(int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s) {
  if (dagger) return launch_hop_f16_dag(recon, epi, reduce, a, s);
  return launch_hop_dag<LQCD_F16, false>(recon, epi, reduce, a, s);
}
}  // namespace lqcd
