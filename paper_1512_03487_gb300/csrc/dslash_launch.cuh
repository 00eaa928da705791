// Launch dispatch for the hop kernel; included by one translation unit per
// precision so the instantiations compile in parallel.
#pragma once

#include "lqcd_internal.h"

namespace lqcd {

template <int P, int R, bool DAG, int EPI, int RED, bool GP>
static int launch_hop_inst(const HopArgs& a, cudaStream_t s) {
  const int64_t nb = (a.g.nsites + HOP_BLOCK - 1) / HOP_BLOCK;
  const int64_t grid = a.full ? 2 * nb : nb;
  if (grid == 0) return LQCD_OK;
  hop_kernel<P, R, DAG, EPI, RED, HOP_BLOCK, GP><<<(unsigned)grid, HOP_BLOCK, 0, s>>>(a);
  return after_launch("hop_kernel");
}

template <int P, int R, bool DAG, int EPI, bool GP>
static int launch_hop_red(int red, const HopArgs& a, cudaStream_t s) {
  if (red == RED_NONE) return launch_hop_inst<P, R, DAG, EPI, RED_NONE, GP>(a, s);
  if (red == RED_NORM) return launch_hop_inst<P, R, DAG, EPI, RED_NORM, GP>(a, s);
  // the fused CG update follows the last hop of M^dag M, always a dagger hop
  if (DAG && red == RED_CG_UPDATE)
    return launch_hop_inst<P, R, DAG, EPI, DAG ? RED_CG_UPDATE : RED_NONE, GP>(a, s);
  return fail(LQCD_ERR_UNSUPPORTED, "hop reduction mode %d (dagger %d)", red, (int)DAG);
}

// GP: G-parity instantiations (Wilson epilogues only; they live in their own translation unit)
template <int P, int R, bool DAG, bool GP>
static int launch_hop_epi(int epi, int red, const HopArgs& a, cudaStream_t s) {
  if (epi == EPI_PLAIN) return launch_hop_inst<P, R, DAG, EPI_PLAIN, RED_NONE, GP>(a, s);
  if (epi == EPI_XPAY) return launch_hop_red<P, R, DAG, EPI_XPAY, GP>(red, a, s);
  if (!GP && epi == EPI_M5) return launch_hop_red<P, R, DAG, GP ? EPI_XPAY : EPI_M5, GP>(red, a, s);
  if (!GP && epi == EPI_M5INV && red == RED_NONE)
    return launch_hop_inst<P, R, DAG, GP ? EPI_PLAIN : EPI_M5INV, RED_NONE, GP>(a, s);
  return fail(LQCD_ERR_ARG, "bad epilogue %d", epi);
}

template <int P, bool GP = false>
static int launch_hop_prec(int recon, bool dagger, int epi, int red, HopArgs a, cudaStream_t s) {
  a.blocks_per_parity = (int)((a.g.nsites + HOP_BLOCK - 1) / HOP_BLOCK);
  if (epi == EPI_PLAIN && red) return fail(LQCD_ERR_UNSUPPORTED, "plain hop with reduction");
  if (recon == 18)
    return dagger ? launch_hop_epi<P, 18, true, GP>(epi, red, a, s) : launch_hop_epi<P, 18, false, GP>(epi, red, a, s);
  if (recon == 12)
    return dagger ? launch_hop_epi<P, 12, true, GP>(epi, red, a, s) : launch_hop_epi<P, 12, false, GP>(epi, red, a, s);
  return fail(LQCD_ERR_ARG, "bad recon %d", recon);
}

}  // namespace lqcd
