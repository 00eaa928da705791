// Host-side internal interfaces shared by the library's translation units.
#pragma once

#include "dslash_kernels.cuh"
#include "lqcd_common.cuh"

namespace lqcd {

// ---- hop launchers (one translation unit per precision)
int launch_hop(int prec, int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s);
int launch_hop_f64(int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s);
int launch_hop_f32(int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s);
int launch_hop_f16(int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s);
int launch_hop_gparity(int prec, int recon, bool dagger, int epi, int reduce, HopArgs a, cudaStream_t s);

// Blocks of the hop kernel per checkerboard (the reduction buffers are sized from it).
constexpr int HOP_BLOCK = 128;
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

// Host pointer offset helper.
inline void* off(void* p, size_t bytes) { return static_cast<char*>(p) + bytes; }
inline const void* off(const void* p, size_t bytes) { return static_cast<const char*>(p) + bytes; }

}  // namespace lqcd
