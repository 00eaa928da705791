// Process-wide autotuner table (see tune.h) and its C entry points.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <atomic>
#include <functional>
#include <mutex>
#include <set>

#include "lqcd_common.cuh"
#include "lqcd_internal.h"
#include "tune.h"

namespace lqcd {

static std::mutex g_tune_mutex;
static std::map<std::string, int> g_tune;

bool tune_lookup(const std::string& key, int* value) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  *value = it->second;
  return true;
}

void tune_store(const std::string& key, int value) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune[key] = value;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

int lqcd_tune_save(const char* path) {
  if (!path) return fail(LQCD_ERR_ARG, "lqcd_tune_save: null path");
  FILE* f = fopen(path, "w");
  if (!f) return fail(LQCD_ERR_ARG, "lqcd_tune_save: cannot open %s", path);
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  for (auto& kv : g_tune) fprintf(f, "%d\t%s\n", kv.second, kv.first.c_str());
  fclose(f);
  return LQCD_OK;
}

int lqcd_tune_load(const char* path) {
  if (!path) return fail(LQCD_ERR_ARG, "lqcd_tune_load: null path");
  FILE* f = fopen(path, "r");
  if (!f) return fail(LQCD_ERR_ARG, "lqcd_tune_load: cannot open %s", path);
  char line[4096];
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  while (fgets(line, sizeof(line), f)) {
    char* tab = strchr(line, '\t');
    if (!tab) continue;
    *tab = 0;
    char* end = nullptr;
    const long v = strtol(line, &end, 10);
    if (end == line || *end != 0) continue;
    std::string k(tab + 1);
    while (!k.empty() && (k.back() == '\n' || k.back() == '\r')) k.pop_back();
    if (k.empty() || v < 0 || v > 64) continue;
    g_tune[k] = (int)v;
  }
  fclose(f);
  return LQCD_OK;
}

int lqcd_tune_entries(void) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  return (int)g_tune.size();
}

void lqcd_tune_clear(void) {
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune.clear();
  }
  lqcd::solver_tuning_reset();
}

}  // extern "C"

namespace lqcd {

static std::atomic<bool> g_autotune{true};
static thread_local bool g_tuning_pass = false;
static thread_local bool g_no_tuning = false;

std::string hop_key_string(const HopKey& k) {
  char buf[160];
  snprintf(buf, sizeof(buf), "hop prec=%d recon=%d dagger=%d epi=%d red=%d full=%d lat=%dx%dx%dx%d n5=%d", k.prec,
           k.recon, k.dagger, k.epi, k.red, k.full, k.X, k.Y, k.Z, k.T, k.n5);
  return buf;
}

bool hop_shape_lookup(const HopKey& k, int* idx) {
  int v = 0;
  if (tune_lookup(hop_key_string(k), &v) && v >= 0 && v < HOP_SHAPES) {
    *idx = v;
    return true;
  }
  return false;
}

bool hop_tuning_pass() { return g_tuning_pass; }

static std::mutex g_solver_mutex;
static std::set<std::string> g_solver_tuned;

bool solver_tuning_due(const std::string& key) {
  std::lock_guard<std::mutex> lock(g_solver_mutex);
  return g_solver_tuned.insert(key).second;
}

void solver_tuning_reset() {
  std::lock_guard<std::mutex> lock(g_solver_mutex);
  g_solver_tuned.clear();
}

TuningPass::TuningPass() : prev(g_tuning_pass) { g_tuning_pass = true; }
TuningPass::~TuningPass() { g_tuning_pass = prev; }
NoTuning::NoTuning() : prev(g_no_tuning) { g_no_tuning = true; }
NoTuning::~NoTuning() { g_no_tuning = prev; }

bool hop_autotune_ready(cudaStream_t s) {
  if (!g_autotune.load() || g_no_tuning) return false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs == cudaStreamCaptureStatusNone;
}

int tune_hop_shapes(const HopKey& k, const std::function<int(int)>& launch, cudaStream_t s, int* best) {
  // Every shape is launched once to warm up, then timed in ROUNDS interleaved
  // rounds of PAIR back-to-back launches; a shape's time is its fastest round.
  // The default shape is kept unless another one is faster by at least MARGIN:
  // differences of a few per cent between shapes are within the spread of such
  // timings and would make the choice change from run to run.
  constexpr int ROUNDS = 3, PAIR = 2;
  constexpr float MARGIN = 0.97f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "hop autotune: event create");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError(), "hop autotune: event create");
  }
  float t[HOP_SHAPES];
  int st = LQCD_OK;
  for (int i = 0; i < HOP_SHAPES && st == LQCD_OK; i++) {
    t[i] = 3.0e38f;
    st = launch(i);
  }
  for (int r = 0; r < ROUNDS && st == LQCD_OK; r++) {
    for (int i = 0; i < HOP_SHAPES && st == LQCD_OK; i++) {
      cudaEventRecord(e0, s);
      for (int q = 0; q < PAIR && st == LQCD_OK; q++) st = launch(i);
      cudaEventRecord(e1, s);
      if (st) break;
      cudaError_t e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        st = cuda_fail(e, "hop autotune: timing");
        break;
      }
      if (ms < t[i]) t[i] = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  int b = HOP_SHAPE_DEFAULT;
  for (int i = 0; i < HOP_SHAPES; i++)
    if (t[i] < MARGIN * t[HOP_SHAPE_DEFAULT] && t[i] < t[b]) b = i;
  *best = b;
  tune_store(hop_key_string(k), b);
  return LQCD_OK;
}

}  // namespace lqcd

extern "C" {

void lqcd_tune_set_enabled(int on) { lqcd::g_autotune.store(on != 0); }

int lqcd_tune_get(const char* key) {
  int v = 0;
  if (!key || !lqcd::tune_lookup(key, &v)) return -1;
  return v;
}

}  // extern "C"
