// Replay of fixed launch sequences as CUDA graphs.
//
// Several steps of the library issue the same few hundred launches every time for a given size on
// given buffers (the Cholesky recursion, the eigensolver's orthonormalisation and back-
// transformation), most of them small.  On a capturable stream such a sequence is recorded once
// per key as a CUDA graph and replayed afterwards, which takes the host launch cost and most gaps
// off the device timeline.  The recording is made on a stream private to the calling host thread
// (nothing runs during a recording, and no other thread's launches onto the caller's stream can
// enter it, also where several handles share one stream); the graph is then launched on the
// caller's stream, after the work already issued there.  Graphs live in the cache of the handle
// whose work is being issued (selected by GraphScope; a handle's work runs on one host thread at a
// time, so its cache needs no lock; at most 128 graphs, the least recently used dropped first), or,
// outside any handle, in one process-wide cache (a lock, at most 512 graphs).  A key holds the
// stream and every buffer address.  The legacy default stream cannot be captured and a stream
// that is already capturing is not nested into: both run the sequence directly, as does
// everything while per-launch-site timing is on (so that each kernel stays bracketed by its own
// events) or while the calling thread has graphs switched off (set_graphs_enabled).
#include <cstdlib>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.hpp"

namespace mpsgb {

namespace {
struct Entry {
  GraphKey key;
  cudaGraphExec_t exec;
  unsigned long long kernels;
  unsigned long long used;
  cudaEvent_t done;  // recorded after every launch: an evicted graph is destroyed once it is idle
};
}  // namespace

struct GraphCache {
  std::mutex mu;  // taken for the process-wide cache only
  std::vector<Entry> v;
  unsigned long long clock = 0;
  size_t cap = 128;
  void clear() {
    for (auto& e : v) {
      cudaEventSynchronize(e.done);
      cudaGraphExecDestroy(e.exec);
      cudaEventDestroy(e.done);
    }
    v.clear();
  }
};
GraphCache* new_graph_cache() { return new GraphCache(); }
void free_graph_cache(GraphCache* c) {
  if (!c) return;
  c->clear();
  delete c;
}
thread_local GraphCache* t_graph_cache = nullptr;
GraphScope::GraphScope(GraphCache* c) : prev(t_graph_cache) { t_graph_cache = c; }
GraphScope::~GraphScope() { t_graph_cache = prev; }

namespace {
using Cache = GraphCache;
void release_all();
Cache& cache() {
  // never destroyed: the graphs are released by an exit handler registered after the CUDA runtime
  // initialised (so it runs before the runtime's own teardown)
  static Cache* c = [] {
    Cache* p = new Cache();
    p->cap = 512;
    std::atexit(release_all);
    return p;
  }();
  return *c;
}
void release_all() {
  Cache& c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  c.clear();
}
thread_local bool t_graphs = true;

// the calling thread's capture stream, created on first use and destroyed with the thread
struct CaptureStream {
  cudaStream_t s = nullptr;
  ~CaptureStream() {
    if (s) cudaStreamDestroy(s);
  }
  cudaStream_t get() {
    if (!s && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
    return s;
  }
};
thread_local CaptureStream t_capture;
}  // namespace

void set_graphs_enabled(bool on) { t_graphs = on; }
bool graphs_enabled() { return t_graphs; }

int replay_or_issue(cudaStream_t st, const GraphKey& key, const std::function<int(cudaStream_t)>& issue) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capturable = t_graphs && st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread &&
                          !g_kt_enabled && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
  cudaStream_t cap = capturable ? t_capture.get() : nullptr;
  if (!cap) {
    if (issue(st) != 0) return -4;
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
  }
  Cache& c = t_graph_cache ? *t_graph_cache : cache();
  const bool shared = !t_graph_cache;
  {
    // launch under the lock (shared cache), so that no other thread evicts the graph in between
    std::unique_lock<std::mutex> lk(c.mu, std::defer_lock);
    if (shared) lk.lock();
    for (auto& e : c.v)
      if (e.key == key) {
        e.used = ++c.clock;
        if (cudaGraphLaunch(e.exec, st) != cudaSuccess || cudaEventRecord(e.done, st) != cudaSuccess) return -4;
        count_launch(e.kernels);
        return 0;
      }
  }
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return -4;
  unsigned long long kernels = 0;  // the captured kernels run (and are counted) at each graph launch
  t_launch_sink = &kernels;
  const int issued = issue(cap);
  t_launch_sink = nullptr;
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(cap, &graph);
  if (issued != 0 || ec != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return -4;
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess || !exec) return -4;
  cudaEvent_t done = nullptr;
  if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGraphExecDestroy(exec);
    return -4;
  }
  if (cudaGraphLaunch(exec, st) != cudaSuccess || cudaEventRecord(done, st) != cudaSuccess) {
    cudaStreamSynchronize(st);
    cudaGraphExecDestroy(exec);
    cudaEventDestroy(done);
    return -4;
  }
  bool evicted = false;
  Entry drop{};
  {
    std::unique_lock<std::mutex> lk(c.mu, std::defer_lock);
    if (shared) lk.lock();
    if (c.v.size() >= c.cap) {
      size_t old = 0;
      for (size_t i = 1; i < c.v.size(); ++i)
        if (c.v[i].used < c.v[old].used) old = i;
      drop = c.v[old];
      evicted = true;
      c.v.erase(c.v.begin() + old);
    }
    c.v.push_back(Entry{key, exec, kernels, ++c.clock, done});
  }
  // the evicted graph (of another size, or of another handle) is no longer reachable from the
  // cache; its last launch is waited for before its resources are released
  if (evicted) {
    cudaEventSynchronize(drop.done);
    cudaGraphExecDestroy(drop.exec);
    cudaEventDestroy(drop.done);
  }
  count_launch(kernels);
  return 0;
}

}  // namespace mpsgb
