// Replay of fixed launch sequences as CUDA graphs.
//
// Several steps of the library issue the same few hundred launches every time for a given size on
// given buffers (the Cholesky recursion, the eigensolver's orthonormalisation and back-
// transformation), most of them small.  On a capturable stream such a sequence is recorded once
// per key as a CUDA graph and replayed afterwards, which takes the host launch cost and most gaps
// off the device timeline.  Graphs are kept per host thread (each handle's work runs on one host
// thread at a time), at most 64, the oldest dropped first.  The legacy default stream cannot be
// captured and a stream that is already capturing is not nested into: both run the sequence
// directly, as does everything while per-launch-site timing is on (so that each kernel stays
// bracketed by its own events).
#include <vector>

#include "common.cuh"
#include "kernels.hpp"

namespace mpsgb {

namespace {
struct Entry {
  GraphKey key;
  cudaGraphExec_t exec;
  unsigned long long kernels;
};
struct Cache {
  std::vector<Entry> v;
  ~Cache() {
    for (auto& e : v) cudaGraphExecDestroy(e.exec);
  }
};
thread_local Cache t_cache;
}  // namespace

int replay_or_issue(cudaStream_t st, const GraphKey& key, const std::function<int()>& issue) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capturable = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread && !g_kt_enabled &&
                          cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
  if (!capturable) {
    if (issue() != 0) return -4;
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
  }
  for (auto& e : t_cache.v)
    if (e.key == key) {
      if (cudaGraphLaunch(e.exec, st) != cudaSuccess) return -4;
      count_launch(e.kernels);
      return 0;
    }
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return -4;
  unsigned long long kernels = 0;  // the captured kernels run (and are counted) at each graph launch
  t_launch_sink = &kernels;
  const int issued = issue();
  t_launch_sink = nullptr;
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(st, &graph);
  if (issued != 0 || ec != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return -4;
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess || !exec) return -4;
  if (t_cache.v.size() >= 64) {
    cudaGraphExecDestroy(t_cache.v.front().exec);
    t_cache.v.erase(t_cache.v.begin());
  }
  t_cache.v.push_back(Entry{key, exec, kernels});
  if (cudaGraphLaunch(exec, st) != cudaSuccess) return -4;
  count_launch(kernels);
  return 0;
}

}  // namespace mpsgb
