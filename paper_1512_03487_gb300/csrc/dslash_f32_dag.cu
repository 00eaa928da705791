// Hop kernel instantiations for LQCD_F32 storage, dagger hops.
#include "dslash_launch.cuh"

namespace lqcd {
int launch_hop_f32_dag(int recon, int epi, int reduce, const HopArgs& a, cudaStream_t s) {
  return launch_hop_dag<LQCD_F32, true>(recon, epi, reduce, a, s);
}
}  // namespace lqcd
