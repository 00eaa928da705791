// Hop kernel instantiations for LQCD_F32 storage, hops without dagger (the
// dagger ones are in dslash_f32_dag.cu: the two halves compile in parallel).
#include "dslash_launch.cuh"

namespace lqcd {
int launch_hop_f32_dag(int recon, int epi, int reduce, const HopArgs& a, cudaStream_t s);

int launch_hop_f32(int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s) {
  if (dagger) return launch_hop_f32_dag(recon, epi, reduce, a, s);
  return launch_hop_dag<LQCD_F32, false>(recon, epi, reduce, a, s);
}
}  // namespace lqcd
