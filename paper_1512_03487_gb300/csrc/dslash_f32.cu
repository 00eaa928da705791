// Hop kernel instantiations for LQCD_F32 storage.
#include "dslash_launch.cuh"

namespace lqcd {
int launch_hop_f32(int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s) {
  return launch_hop_prec<LQCD_F32>(recon, dagger, epi, reduce, a, s);
}
}  // namespace lqcd
