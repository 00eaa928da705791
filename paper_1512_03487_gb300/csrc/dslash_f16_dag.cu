// Hop kernel instantiations for LQCD_F16 storage, dagger hops.
#include "dslash_launch.cuh"

namespace lqcd {
int launch_hop_f16_dag(int recon, int epi, int reduce, const HopArgs& a, cudaStream_t s) {
  return launch_hop_dag<LQCD_F16, true>(recon, epi, reduce, a, s);
}
}  // namespace lqcd
