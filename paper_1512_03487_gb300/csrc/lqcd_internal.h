// Host-side internal interfaces shared by the library's translation units.
#pragma once

#include <functional>
#include <string>

#include "dslash_kernels.cuh"
#include "lqcd_common.cuh"

namespace lqcd {

// ---- hop launchers (one translation unit per precision)
int launch_hop(int prec, int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s);
int launch_hop_f64(int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s);
int launch_hop_f32(int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s);
int launch_hop_f16(int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s);
int launch_hop_gparity(int prec, int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s);
int launch_hop_df(int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s);

// Threads per block of the one-site hop (FP64, G-parity, the batch solver's tiles).
// Every hop launch shape covers at least 64 sites per block: the solvers size
// their reduction partials for that.
constexpr int HOP_BLOCK = 128;

// Launch shapes of the FP32 / FP16 hop that the autotuner chooses among:
// X(index, threads per block, sites per thread, minimum resident blocks per SM;
// 0 leaves the register count to the compiler). Measured on GB300 at 24^3 x 48
// (warm, back to back): the plain FP16 / 12-real hop takes 26.6-27.1 us with one
// site per thread, 25.2-26.8 us spin-paired (21 % fewer instructions, the FMA
// pipe as busy), 25.7 us with the neighbour data staged asynchronously (long-
// scoreboard stalls 3.6 -> 0.5 per issue, issue slots 69 -> 77 % busy, 9 % more
// instructions), 30 us with two sites per thread (32 % fewer instructions,
// 168-222 registers); the FP32 / 12-real hop is fastest staged (34.8 us cold,
// 0.81 of the copy bandwidth, against 36.9 us). Shape 0 is the default; the
// tuner times all of them per key.
// Sites per thread -1: one site per thread with the links of each 4D site staged
// in shared memory once for its n5 threads (L_s-replicated and multi-RHS hops,
// n5 >= 4; otherwise as shape 0). -2: one site per thread with the two spin
// components of each half spinor paired in packed FP32x2 instructions. -3 / -4:
// as 1 / -2 with each direction's neighbour spinor and link copied with
// cp.async into a per-thread shared-memory ring while an earlier direction is
// computed (hop_async.cuh).
#define LQCD_HOP_SHAPES(X) X(0, 128, 1, 0) X(1, 128, 1, 7) X(2, 128, -2, 7) X(3, 128, 1, 5) X(4, 128, 2, 3) \
  X(5, 128, -1, 6) X(6, 128, -2, 0) X(7, 128, -3, 7) X(8, 128, -4, 7)
constexpr int HOP_SHAPES = 9;
// The shape used when the table holds no choice for a hop.
constexpr int HOP_SHAPE_DEFAULT = 0;

// What identifies one tunable hop launch: the kernel instantiation and the lattice.
struct HopKey {
  int prec, recon, dagger, epi, red, full, X, Y, Z, T, n5;
};
// Text form of k, the autotuner table's key.
std::string hop_key_string(const HopKey& k);
// The table's shape index for k, if it holds one.
bool hop_shape_lookup(const HopKey& k, int* idx);
// Whether an untuned hop launch on stream s may be timed now: autotuning is
// on (lqcd_tune_set_enabled) and s is not capturing a graph.
bool hop_autotune_ready(cudaStream_t s);
// Times launch(i) for every shape i on s (a warm-up each, then three interleaved
// rounds of two back-to-back launches; a shape's time is its fastest round),
// stores the fastest under k -- the default unless another shape is at least
// 3 % faster -- and returns it in *best.
int tune_hop_shapes(const HopKey& k, const std::function<int(int)>& launch, cudaStream_t s, int* best);
// A hop launch is timed in place only if running it again cannot change what
// it leaves behind: no reduction, no gate, out not aliasing in or x. Inside a
// tuning pass (an object of this type alive on the thread) the caller
// guarantees that a reducing hop's partials, counter, result and update
// fields are scratch, so reducing hops are tuned too.
struct TuningPass {
  TuningPass();
  ~TuningPass();
  bool prev;
};
bool hop_tuning_pass();
// While an object of this type is alive on the thread, no hop launch is timed
// (hop_autotune_ready is false): for entry points that must not synchronise.
struct NoTuning {
  NoTuning();
  ~NoTuning();
  bool prev;
};
// True the first time it is called for a solver configuration key (its tuning
// pass is then due), false afterwards.
bool solver_tuning_due(const std::string& key);
// Forgets which configurations had their tuning pass (lqcd_tune_clear).
void solver_tuning_reset();
constexpr int BLAS_BLOCK = 128;
constexpr int M5_BLOCK = 128;

// ---- fifth-dimension inverse M5op^-1 (domain wall), out and in checkerboard fields
struct M5Args {
  void* out;
  const void* in;
  Geom g;
  double d;    // 5 - M5
  double mf;
  int dagger;
  const Control* gate;
};
int launch_m5inv(int prec, const M5Args& a, cudaStream_t s);

// ---- operators
struct OpCtx {
  Geom g;
  lqcd_operator op;   // kind, mass, M5, mf, prec, recon
  const void* gauge;
};
// out = M in (subset LQCD_FULL) or M_hat in (LQCD_EVEN), dagger; optional |out|^2
// reduction and gate. t1, t2: odd checkerboard temporaries (EVEN subset).
// With upd (and red) the last hop does not store out but runs the fused CG
// update of HopArgs::upd_* instead (dagger only).
struct HopUpdate {
  const void* p;
  void* xs;
  void* rs;
  int64_t half_bytes;     // one checkerboard of x_s
  int64_t rs_half_bytes;  // one checkerboard of r_s
};
int op_apply(const OpCtx& c, void* out, const void* in, int subset, int dagger,
             void* t1, void* t2, const ReduceCtx* red, const Control* gate, cudaStream_t s,
             const HopUpdate* upd = nullptr);
// Bytes of the temporaries op_apply needs (t1 + t2) for a subset.
size_t op_tmp_bytes(const Geom& g, int kind, int prec, int subset);
// Bytes of a field of the given subset.
size_t field_bytes(const Geom& g, int prec, int subset);
// Validates op against g and records the operator's G-parity mask in g.gp.
int check_operator(const lqcd_operator* op, Geom& g);

// ---- fermion force accumulated into a momentum field: mom -= coef * F (traceless
// Hermitian force of lqcd_force, kind LQCD_FORCE_TA); FP64 fields, gauge in recon.
int force_accumulate(double2* mom, const void* gauge, const void* X, const void* Y, const Geom& g, int recon,
                     double coef, cudaStream_t s);

// Forgets the cached device addresses of the allocation-free operator's array.
void release_noalloc_addresses();

// Host pointer offset helper.
inline void* off(void* p, size_t bytes) { return static_cast<char*>(p) + bytes; }
inline const void* off(const void* p, size_t bytes) { return static_cast<const char*>(p) + bytes; }

}  // namespace lqcd
