// CG driver: the device-driven conditional graph, its cache, and the host loop.
//
// Graph of one launch (one "chunk" of up to check_interval iterations):
//
//   chunk_start --> WHILE (go) {
//                     head: 4 sloppy hops (alpha), x_s / r_s update (beta, or request)
//                     IF (replacement requested) { r_s = r - A x_s, FP32 arithmetic }  [three-level only]
//                     IF (reliable update requested) { x += x_s; r = b - A x in FP64 }
//                     tail: p = r_s + beta p
//                     loop control: go = active && chunks left && iter < maxiter
//                   }
//
// The WHILE and IF conditions are set on the device (cudaGraphSetConditional)
// by a one-thread control kernel and by the finaliser of the update kernel,
// so reliable updates cost no host round trip. Every body execution
// decrements the chunk counter, so one launch runs at most check_interval
// iterations whatever the state says. The host only reads the control block
// between launches (convergence, NaN, iteration cap, wall-clock limit).
//
// With use_graph = 0 the same kernels are launched directly and a requested
// reliable update pauses the chunk for the host instead.
#include <cstring>
#include <mutex>

#include "cg_engine.h"

namespace lqcd {

__global__ void k_chunk_start(Control* c, int chunk, int maxiter, cudaGraphConditionalHandle h_loop) {
  c->chunk_left = chunk;
  const int go = c->active && c->iter < maxiter && c->n_done < c->nsys && !(c->reason & REASON_NAN);
  cudaGraphSetConditional(h_loop, go ? 1u : 0u);
}

__global__ void k_loop_control(Control* c, int maxiter, cudaGraphConditionalHandle h_loop,
                               cudaGraphConditionalHandle h_rel, cudaGraphConditionalHandle h_mid, int has_mid) {
  cudaGraphSetConditional(h_rel, 0u);  // the next iteration's update decides afresh
  if (has_mid) cudaGraphSetConditional(h_mid, 0u);
  c->chunk_left -= 1;
  const int go = c->active && c->chunk_left > 0 && c->iter < maxiter && c->n_done < c->nsys &&
                 !(c->reason & REASON_NAN);
  cudaGraphSetConditional(h_loop, go ? 1u : 0u);
}

struct GraphEntry {
  std::vector<unsigned char> key;
  cudaGraphExec_t exec;
  uint64_t head_kernels, tail_kernels, reliable_kernels, mid_kernels;
  uint64_t last_use;
};

static std::mutex g_graph_mutex;
static std::vector<GraphEntry> g_graphs;
static uint64_t g_graph_clock = 0;
constexpr size_t MAX_GRAPHS = 16;

void release_graph_cache() {
  std::lock_guard<std::mutex> lock(g_graph_mutex);
  for (auto& e : g_graphs) cudaGraphExecDestroy(e.exec);
  g_graphs.clear();
}

namespace {

struct Capture {
  cudaStream_t s = nullptr;
  ~Capture() {
    if (s) {
      cudaStreamCaptureStatus cs;
      if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
      }
      cudaStreamDestroy(s);
    }
    g_count_suspended = false;
  }
};

}  // namespace

#define LQCD_TRY_CUDA(expr, what)                  \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

static int build_graph(CgEngine& E, int chunk, int maxiter, GraphEntry* out) {
  Capture cap;
  LQCD_TRY_CUDA(cudaStreamCreateWithFlags(&cap.s, cudaStreamNonBlocking), "cg graph: stream");
  cudaGraph_t outer = nullptr;
  LQCD_TRY_CUDA(cudaGraphCreate(&outer, 0), "cg graph: create");
  struct GraphGuard {
    cudaGraph_t g;
    ~GraphGuard() { if (g) cudaGraphDestroy(g); }
  } guard{outer};
  cudaGraphConditionalHandle h_loop;
  LQCD_TRY_CUDA(cudaGraphConditionalHandleCreate(&h_loop, outer, 1, cudaGraphCondAssignDefault),
                "cg graph: loop handle");
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  g_count_suspended = true;

  // chunk start
  LQCD_TRY_CUDA(cudaStreamBeginCaptureToGraph(cap.s, outer, nullptr, nullptr, 0, mode), "cg graph: capture");
  k_chunk_start<<<1, 1, 0, cap.s>>>(E.ctrl, chunk, maxiter, h_loop);
  int st = after_launch("k_chunk_start");
  LQCD_TRY_CUDA(cudaStreamEndCapture(cap.s, &outer), "cg graph: end capture");
  if (st) return st;
  cudaGraphNode_t start = nullptr;
  size_t n = 1;
  LQCD_TRY_CUDA(cudaGraphGetNodes(outer, &start, &n), "cg graph: nodes");

  // WHILE node and its body
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = h_loop;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  LQCD_TRY_CUDA(cudaGraphAddNode(&wnode, outer, &start, nullptr, 1, &wp), "cg graph: while node");
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  cudaGraphConditionalHandle h_rel, h_mid = 0;
  LQCD_TRY_CUDA(cudaGraphConditionalHandleCreate(&h_rel, body, 0, cudaGraphCondAssignDefault),
                "cg graph: reliable handle");
  const bool has_mid = E.has_mid();
  if (has_mid)
    LQCD_TRY_CUDA(cudaGraphConditionalHandleCreate(&h_mid, body, 0, cudaGraphCondAssignDefault),
                  "cg graph: replacement handle");

  // body: head
  LQCD_TRY_CUDA(cudaStreamBeginCaptureToGraph(cap.s, body, nullptr, nullptr, 0, mode), "cg graph: capture");
  uint64_t c0 = g_captured_launches;
  st = E.head(cap.s, 1, h_rel, h_mid);
  out->head_kernels = g_captured_launches - c0;
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cap.s, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
  std::vector<cudaGraphNode_t> frontier(deps, deps + (e == cudaSuccess ? ndeps : 0));
  LQCD_TRY_CUDA(cudaStreamEndCapture(cap.s, &body), "cg graph: end capture");
  if (st) return st;
  if (e != cudaSuccess) return cuda_fail(e, "cg graph: capture info");

  // body: IF (FP32-arithmetic replacement requested)
  out->mid_kernels = 0;
  if (has_mid) {
    cudaGraphNodeParams mp = {};
    mp.type = cudaGraphNodeTypeConditional;
    mp.conditional.handle = h_mid;
    mp.conditional.type = cudaGraphCondTypeIf;
    mp.conditional.size = 1;
    cudaGraphNode_t mnode;
    LQCD_TRY_CUDA(cudaGraphAddNode(&mnode, body, frontier.data(), nullptr, frontier.size(), &mp),
                  "cg graph: replacement node");
    cudaGraph_t mg = mp.conditional.phGraph_out[0];
    LQCD_TRY_CUDA(cudaStreamBeginCaptureToGraph(cap.s, mg, nullptr, nullptr, 0, mode), "cg graph: capture");
    c0 = g_captured_launches;
    st = E.mid(cap.s);
    out->mid_kernels = g_captured_launches - c0;
    LQCD_TRY_CUDA(cudaStreamEndCapture(cap.s, &mg), "cg graph: end capture");
    if (st) return st;
    frontier.assign(1, mnode);
  }

  // body: IF (reliable update requested)
  cudaGraphNodeParams ip = {};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = h_rel;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  cudaGraphNode_t inode;
  LQCD_TRY_CUDA(cudaGraphAddNode(&inode, body, frontier.data(), nullptr, frontier.size(), &ip),
                "cg graph: if node");
  cudaGraph_t rel = ip.conditional.phGraph_out[0];
  LQCD_TRY_CUDA(cudaStreamBeginCaptureToGraph(cap.s, rel, nullptr, nullptr, 0, mode), "cg graph: capture");
  c0 = g_captured_launches;
  st = E.reliable(cap.s);
  out->reliable_kernels = g_captured_launches - c0;
  LQCD_TRY_CUDA(cudaStreamEndCapture(cap.s, &rel), "cg graph: end capture");
  if (st) return st;

  // body: tail and loop control, after the IF node
  LQCD_TRY_CUDA(cudaStreamBeginCaptureToGraph(cap.s, body, &inode, nullptr, 1, mode), "cg graph: capture");
  c0 = g_captured_launches;
  st = E.tail(cap.s);
  if (!st) {
    k_loop_control<<<1, 1, 0, cap.s>>>(E.ctrl, maxiter, h_loop, h_rel, h_mid, has_mid ? 1 : 0);
    st = after_launch("k_loop_control");
  }
  out->tail_kernels = g_captured_launches - c0;
  LQCD_TRY_CUDA(cudaStreamEndCapture(cap.s, &body), "cg graph: end capture");
  if (st) return st;

  LQCD_TRY_CUDA(cudaGraphInstantiate(&out->exec, outer, 0), "cg graph: instantiate");
  return LQCD_OK;
}

static int cached_graph(CgEngine& E, const std::vector<unsigned char>& key, int chunk, int maxiter,
                        GraphEntry* out) {
  std::lock_guard<std::mutex> lock(g_graph_mutex);
  for (auto& e : g_graphs) {
    if (e.key == key) {
      e.last_use = ++g_graph_clock;
      *out = e;
      return LQCD_OK;
    }
  }
  GraphEntry ne;
  ne.key = key;
  ne.exec = nullptr;
  int st = build_graph(E, chunk, maxiter, &ne);
  if (st) {
    if (ne.exec) cudaGraphExecDestroy(ne.exec);
    return st;
  }
  if (g_graphs.size() >= MAX_GRAPHS) {
    size_t lru = 0;
    for (size_t i = 1; i < g_graphs.size(); i++)
      if (g_graphs[i].last_use < g_graphs[lru].last_use) lru = i;
    cudaGraphExecDestroy(g_graphs[lru].exec);
    g_graphs.erase(g_graphs.begin() + lru);
  }
  ne.last_use = ++g_graph_clock;
  g_graphs.push_back(ne);
  *out = ne;
  return LQCD_OK;
}

static int read_ctrl(const Control* d, Control* h, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(h, d, sizeof(Control), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cg: control readback");
  return LQCD_OK;
}

int run_cg(CgEngine& E, const lqcd_solver_params& prm, const std::vector<unsigned char>& key, cudaStream_t s,
           std::chrono::steady_clock::time_point t0, Control* ctrl) {
  int st = E.init(s);
  if (st) return st;
  const int chunk = prm.check_interval > 0 ? prm.check_interval : 16;
  GraphEntry ge;
  ge.exec = nullptr;
  if (prm.use_graph && (st = cached_graph(E, key, chunk, prm.maxiter, &ge))) return st;
  auto timed_out = [&]() {
    if (prm.timeout_ms <= 0) return false;
    const double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return el > prm.timeout_ms;
  };
  for (;;) {
    if ((st = read_ctrl(E.ctrl, ctrl, s))) return st;
    if (ctrl->reason & REASON_NAN) return fail(LQCD_ERR_NAN, "cg: NaN/Inf or non-positive p^dag A p");
    if (ctrl->n_done == ctrl->nsys) return LQCD_OK;
    if (ge.exec) {
      // device-driven: the final FP64 check at the iteration cap already ran
      if (ctrl->iter >= prm.maxiter) return fail(LQCD_ERR_NOT_CONVERGED, "cg: maxiter %d reached", prm.maxiter);
      if (timed_out()) return fail(LQCD_ERR_TIMEOUT, "cg: wall-clock limit %.1f ms exceeded", prm.timeout_ms);
      const Control before = *ctrl;
      cudaError_t e = cudaGraphLaunch(ge.exec, s);
      if (e != cudaSuccess) return cuda_fail(e, "cg: graph launch");
      if ((st = read_ctrl(E.ctrl, ctrl, s))) return st;
      const uint64_t iters = (uint64_t)(ctrl->iter - before.iter);
      const uint64_t rels = (uint64_t)(ctrl->n_reliable - before.n_reliable);
      const uint64_t mids = (uint64_t)(ctrl->n_mid - before.n_mid);
      count_launches(1 + iters * (ge.head_kernels + ge.tail_kernels) + rels * ge.reliable_kernels +
                     mids * ge.mid_kernels);
      continue;
    }
    // host-driven
    if (ctrl->iter >= prm.maxiter) {
      if ((st = E.reliable(s)) || (st = E.tail(s))) return st;
      if ((st = read_ctrl(E.ctrl, ctrl, s))) return st;
      if (ctrl->reason & REASON_NAN) return fail(LQCD_ERR_NAN, "cg: NaN/Inf in the true residual");
      if (ctrl->n_done != ctrl->nsys) return fail(LQCD_ERR_NOT_CONVERGED, "cg: maxiter %d reached", prm.maxiter);
      return LQCD_OK;
    }
    if (ctrl->active == 0) {
      // paused by the update's finaliser: the reason bits say which recomputation is due
      const bool mid_only = (ctrl->reason & REASON_MID) && !(ctrl->reason & (REASON_CONVERGED | REASON_RELIABLE));
      if ((st = mid_only ? E.mid(s) : E.reliable(s)) || (st = E.tail(s))) return st;
      continue;
    }
    if (timed_out()) return fail(LQCD_ERR_TIMEOUT, "cg: wall-clock limit %.1f ms exceeded", prm.timeout_ms);
    for (int i = 0; i < chunk; i++)
      if ((st = E.head(s, 0, 0, 0)) || (st = E.tail(s))) return st;
  }
}

}  // namespace lqcd
