// lqcd_M_noalloc: the Dirac operator of lqcd_M with its scratch space in a
// fixed device array inside this library, for callers that cannot allocate
// device memory themselves.
//
// Who cannot allocate: code that runs where a cudaMalloc is forbidden or
// harmful -- inside a host callback enqueued with cudaLaunchHostFunc (which
// must not call CUDA API functions that allocate), on a latency-critical path
// where cudaMalloc's implicit device synchronisation is not acceptable, or in
// a plugin whose host framework owns the whole device memory pool so that a
// private allocation would fail or fragment it. Such callers still pass the
// input and output fields; only the operator's temporaries move here.
//
// The scratch array is a file-scope __device__ array, so every GPU that loads
// the library holds its LQCD_NOALLOC_SCRATCH_BYTES until the process exits.
// In host code the symbol is only a host-side stand-in; the device address is
// obtained once per device with cudaGetSymbolAddress, on the first call made
// with that device current.
#include <mutex>

#include "lqcd_internal.h"

namespace lqcd {

static __device__ __align__(256) unsigned char g_noalloc_scratch[LQCD_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
static void* g_scratch_addr[MAX_DEVICES] = {nullptr};
static std::mutex g_scratch_mutex;

// Device address of the scratch array on the current device (looked up once per device).
static int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "lqcd_M_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) return fail(LQCD_ERR_UNSUPPORTED, "lqcd_M_noalloc: device %d", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "lqcd_M_noalloc: cudaGetSymbolAddress");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return LQCD_OK;
}

// Forgets the looked-up addresses (lqcd_release_caches): after a device reset
// the module is loaded again and the array may move.
void release_noalloc_addresses() {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  for (int d = 0; d < MAX_DEVICES; d++) g_scratch_addr[d] = nullptr;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" int lqcd_M_noalloc(void* out, const void* in, const void* gauge, const lqcd_lattice* lat,
                              const lqcd_operator* op, int subset, int dagger, void* stream) {
  Geom g;
  int st = make_geom(lat, &g);
  if (st) return st;
  if ((st = check_operator(op, g))) return st;
  if (subset != LQCD_EVEN && subset != LQCD_FULL) return fail(LQCD_ERR_ARG, "lqcd_M_noalloc: bad subset %d", subset);
  if (!out || !in || !gauge || (((uintptr_t)out | (uintptr_t)in | (uintptr_t)gauge) & 15))
    return fail(LQCD_ERR_ARG, "lqcd_M_noalloc: null or misaligned pointer");
  if (out == in) return fail(LQCD_ERR_ARG, "lqcd_M_noalloc: out aliases in");
  const size_t need = op_tmp_bytes(g, op->kind, op->prec, subset);
  if (need > LQCD_NOALLOC_SCRATCH_BYTES)
    return fail(LQCD_ERR_ARG,
                "lqcd_M_noalloc: the operator needs %zu bytes of scratch, more than the fixed %zu-byte "
                "array; use lqcd_M with a caller-provided workspace",
                need, (size_t)LQCD_NOALLOC_SCRATCH_BYTES);
  void* t1 = nullptr;
  void* t2 = nullptr;
  if (need > 0) {
    void* base = nullptr;
    if ((st = scratch_address(&base))) return st;
    t1 = base;
    t2 = off(base, cb_spinor_bytes(g, op->prec));
  }
  OpCtx c{g, *op, gauge};
  NoTuning quiet;  // never time launch shapes here: that would synchronise the stream
  return op_apply(c, out, in, subset, dagger != 0, t1, t2, nullptr, nullptr, (cudaStream_t)stream);
}
