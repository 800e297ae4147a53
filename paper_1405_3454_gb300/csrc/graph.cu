// graph.cu -- hull_batch_ranges run as a CUDA graph (include/cudapre.h,
// hull_graph_*).  The paper has no counterpart: this is how a caller that
// repeats a batch call replays all of its kernels with one launch.
//
// A call with the same arguments and options as the previous one on the same
// object replays the instantiated graph.  Any other call captures its work
// anew (the launch sequence of hull_batch_ranges, enqueued on a capturing
// stream) and updates the instantiated graph in place, or instantiates a new
// one when CUDA refuses the update (a different sequence of kernels, e.g.
// other options).  Every size the kernels need is read on the device, so a
// replay may run on new point data, offsets and starts in the same buffers.
#include <cstring>

#include "internal.cuh"

struct hull_graph {
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;
  int64_t kernels = 0;  // kernel nodes of the instantiated graph
  // the arguments of the captured call
  const float* d_xy = nullptr;
  int64_t n_xy = 0;
  const int64_t* d_starts = nullptr;
  const int64_t* d_offsets = nullptr;
  int32_t S = 0;
  int64_t n_total = 0;
  void* d_ws = nullptr;
  size_t ws_bytes = 0;
  int64_t* d_hull_idx = nullptr;
  int64_t* d_hull_offsets = nullptr;
  hull_options opt{};
  // counters: calls, captures, in-place updates, instantiations, replays
  int64_t count[5] = {0, 0, 0, 0, 0};
};

namespace {

int64_t kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
  cudaGraphNode_t* nodes = new cudaGraphNode_t[n];
  int64_t k = 0;
  if (cudaGraphGetNodes(g, nodes, &n) == cudaSuccess) {
    for (size_t i = 0; i < n; ++i) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
  }
  delete[] nodes;
  return k;
}

}  // namespace

extern "C" {

hull_graph* hull_graph_create(void) { return new hull_graph(); }

void hull_graph_destroy(hull_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
}

void hull_graph_counts(const hull_graph* g, int64_t* h_out) {
  if (!g || !h_out) return;
  for (int k = 0; k < 5; ++k) h_out[k] = g->count[k];
  h_out[5] = g->kernels;
}

hull_status hull_graph_batch_ranges(hull_graph* g, const float* d_xy, int64_t n_xy, const int64_t* d_starts,
                                    const int64_t* d_offsets, int32_t S, int64_t n_total, void* d_ws,
                                    size_t ws_bytes, int64_t* d_hull_idx, int64_t* d_hull_offsets,
                                    const hull_options* opt, void* stream) {
  if (!g || !stream) return HULL_ERR_INVALID_ARG;  // the legacy default stream cannot be captured
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  hull_options o;
  hull_default_options(&o);
  if (opt) o = *opt;
  ++g->count[0];
  const bool same = g->exec && g->stream == st && g->d_xy == d_xy && g->n_xy == n_xy && g->d_starts == d_starts &&
                    g->d_offsets == d_offsets && g->S == S && g->n_total == n_total && g->d_ws == d_ws &&
                    g->ws_bytes == ws_bytes && g->d_hull_idx == d_hull_idx && g->d_hull_offsets == d_hull_offsets &&
                    std::memcmp(&g->opt, &o, sizeof(o)) == 0;
  if (same) {
    if (cudaGraphLaunch(g->exec, st) != cudaSuccess) return HULL_ERR_CUDA;
    cudapre::count_launches((int)g->kernels);
    ++g->count[4];
    return HULL_OK;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return HULL_ERR_INVALID_ARG;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HULL_ERR_CUDA;
  const int64_t launched0 = hull_launch_count();
  const hull_status s = hull_batch_ranges(d_xy, n_xy, d_starts, d_offsets, S, n_total, d_ws, ws_bytes, d_hull_idx,
                                          d_hull_offsets, &o, stream);
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(st, &graph);
  // the captured launches did not run: take them off the launch count
  cudapre::count_launches(-(int)(hull_launch_count() - launched0));
  if (s != HULL_OK || ec != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    return s != HULL_OK ? s : HULL_ERR_CUDA;
  }
  ++g->count[1];
  bool ready = false;
  if (g->exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(g->exec, graph, &info) == cudaSuccess) {
      ready = true;
      ++g->count[2];
    } else {
      (void)cudaGetLastError();
      cudaGraphExecDestroy(g->exec);
      g->exec = nullptr;
    }
  }
  if (!ready) {
    if (cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
      g->exec = nullptr;
      cudaGraphDestroy(graph);
      return HULL_ERR_CUDA;
    }
    ++g->count[3];
  }
  g->kernels = kernel_nodes(graph);
  cudaGraphDestroy(graph);
  g->stream = st;
  g->d_xy = d_xy;
  g->n_xy = n_xy;
  g->d_starts = d_starts;
  g->d_offsets = d_offsets;
  g->S = S;
  g->n_total = n_total;
  g->d_ws = d_ws;
  g->ws_bytes = ws_bytes;
  g->d_hull_idx = d_hull_idx;
  g->d_hull_offsets = d_hull_offsets;
  g->opt = o;
  if (cudaGraphLaunch(g->exec, st) != cudaSuccess) return HULL_ERR_CUDA;
  cudapre::count_launches((int)g->kernels);
  return HULL_OK;
}

}  // extern "C"
