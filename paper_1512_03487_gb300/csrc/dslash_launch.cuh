// Launch dispatch for the hop kernel; included by one translation unit per
// precision so the instantiations compile in parallel.
#pragma once

#include "lqcd_internal.h"

namespace lqcd {

template <int P, int R, bool DAG, int EPI, int RED, bool GP, int BLOCK, int SPT, int MINB>
static int launch_hop_shape(HopArgs a, cudaStream_t s) {
  constexpr int SITES = SPT < 0 ? 1 : SPT;  // SPT -1 .. -4: one site per thread
  const int64_t nb = (a.g.nsites + BLOCK * SITES - 1) / (BLOCK * SITES);
  a.blocks_per_parity = (int)nb;
  const int64_t grid = a.full ? 2 * nb : nb;
  if (grid == 0) return LQCD_OK;
  if constexpr (SPT <= -3) {
    // the staged hop's ring: ask for the largest shared-memory carveout so that
    // MINB blocks of it fit an SM
    static const cudaError_t carve = cudaFuncSetAttribute(hop_kernel<P, R, DAG, EPI, RED, BLOCK, GP, SPT, MINB>,
                                                          cudaFuncAttributePreferredSharedMemoryCarveout,
                                                          (int)cudaSharedmemCarveoutMaxShared);
    if (carve != cudaSuccess) return cuda_fail(carve, "hop_kernel: shared-memory carveout");
  }
  hop_kernel<P, R, DAG, EPI, RED, BLOCK, GP, SPT, MINB><<<(unsigned)grid, BLOCK, 0, s>>>(a);
  return after_launch("hop_kernel");
}

template <int P, int R, bool DAG, int EPI, int RED, bool GP>
static int launch_hop_index(int idx, const HopArgs& a, cudaStream_t s) {
  switch (idx) {
#define LQCD_HOP_CASE(I, B, S, M) \
  case I: return launch_hop_shape<P, R, DAG, EPI, RED, GP, B, S, M>(a, s);
    LQCD_HOP_SHAPES(LQCD_HOP_CASE)
#undef LQCD_HOP_CASE
  }
  return fail(LQCD_ERR_ARG, "hop launch shape %d out of range", idx);
}

// FP64 and G-parity hops have one launch shape; FP32 and FP16 hops take the
// tuner table's shape for their key, timing every shape on the first launch
// that may be timed (see TuningPass), else the default shape.
template <int P, int R, bool DAG, int EPI, int RED, bool GP>
static int launch_hop_inst(const HopArgs& a, cudaStream_t s) {
  if constexpr (P == LQCD_F64 || P == LQCD_F64_DF || GP) {
    return launch_hop_shape<P, R, DAG, EPI, RED, GP, HOP_BLOCK, 1, 0>(a, s);
  } else {
    const HopKey k{P, R, DAG ? 1 : 0, EPI, RED, a.full, a.g.X, a.g.Y, a.g.Z, a.g.T, a.g.n5};
    int idx = HOP_SHAPE_DEFAULT;
    if (!hop_shape_lookup(k, &idx)) {
      idx = HOP_SHAPE_DEFAULT;
      const bool repeatable = RED == RED_NONE ? (a.gate == nullptr && a.out != a.in && a.out != a.x)
                                              : hop_tuning_pass();
      if (repeatable && a.g.nsites > 0 && hop_autotune_ready(s)) {
        const int st = tune_hop_shapes(
            k, [&](int i) { return launch_hop_index<P, R, DAG, EPI, RED, GP>(i, a, s); }, s, &idx);
        if (st) return st;
      }
    }
    return launch_hop_index<P, R, DAG, EPI, RED, GP>(idx, a, s);
  }
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

template <int P, bool DAG, bool GP = false>
static int launch_hop_dag(int recon, int epi, int red, const HopArgs& a, cudaStream_t s) {
  if (epi == EPI_PLAIN && red) return fail(LQCD_ERR_UNSUPPORTED, "plain hop with reduction");
  if (recon == 18) return launch_hop_epi<P, 18, DAG, GP>(epi, red, a, s);
  if (recon == 12) return launch_hop_epi<P, 12, DAG, GP>(epi, red, a, s);
  return fail(LQCD_ERR_ARG, "bad recon %d", recon);
}

template <int P, bool GP = false>
static int launch_hop_prec(int recon, bool dagger, int epi, int red, const HopArgs& a, cudaStream_t s) {
  return dagger ? launch_hop_dag<P, true, GP>(recon, epi, red, a, s) : launch_hop_dag<P, false, GP>(recon, epi, red, a, s);
}

}  // namespace lqcd
