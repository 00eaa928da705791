// The conjugate-gradient driver shared by the single-lattice solver (cg.cu)
// and the batched solver (batch.cu). An engine supplies the kernels of one
// solve; the driver owns the loop, the CUDA graph and the host checks.
#pragma once

#include <chrono>
#include <vector>

#include "lqcd_internal.h"

namespace lqcd {

struct CgEngine {
  Control* ctrl = nullptr;
  SysState* sys = nullptr;
  int nsys = 0;
  virtual ~CgEngine() {}
  // r = b, x = 0, p = b; |b|^2 per system -> initial state (FIN_INIT)
  virtual int init(cudaStream_t s) = 0;
  // Mp = M p (p^dag A p -> alpha), Ap = M^dag Mp, x_s += alpha p, r_s -= alpha Ap
  // (|r_s|^2 -> beta, or a reliable update / replacement is requested: through
  // the IF node handles when cond = 1, by pausing for the host when cond = 0). Gated.
  virtual int head(cudaStream_t s, int cond, cudaGraphConditionalHandle h_rel, cudaGraphConditionalHandle h_mid) = 0;
  // p = r_s + beta p. Gated.
  virtual int tail(cudaStream_t s) = 0;
  // x += x_s; r = b - A x with the FP64 operator; |r|^2 -> done flags, beta (FIN_RELIABLE)
  virtual int reliable(cudaStream_t s) = 0;
  // Three-level scheme: r_s = r - A x_s with FP32 arithmetic on the FP64
  // links, r the residual of the last FP64 update; |r_s|^2 -> beta (FIN_MID).
  // Engines without the intermediate level never request it.
  virtual bool has_mid() const { return false; }
  virtual int mid(cudaStream_t) { return fail(LQCD_ERR_UNSUPPORTED, "cg: no intermediate replacement level"); }
};

// Runs a solve with engine E. `key` identifies everything the captured graph
// bakes in (pointers, shapes, formats, chunk length, iteration cap); graphs
// are cached across calls under it. On return *ctrl holds the final control
// block.
int run_cg(CgEngine& E, const lqcd_solver_params& prm, const std::vector<unsigned char>& key, cudaStream_t s,
           std::chrono::steady_clock::time_point t0, Control* ctrl);

// Kernel launches are counted when they run: a thread capturing a graph
// suspends counting (and tallies the captured launches instead).
extern thread_local bool g_count_suspended;
extern thread_local uint64_t g_captured_launches;

void release_graph_cache();

template <typename T>
inline void key_append(std::vector<unsigned char>& key, const T& v) {
  const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
  key.insert(key.end(), p, p + sizeof(T));
}

}  // namespace lqcd
