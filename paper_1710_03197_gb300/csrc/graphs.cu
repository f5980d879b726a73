// graphs.cu - CUDA graphs of the entry points' kernel sequences.
//
// A forward or adjoint NUFFT is a fixed sequence of 3 to 10 kernel launches
// (and a solver iteration a dozen more); for small problems the host launch
// cost is comparable to the GPU work.  The plan therefore records each entry
// point's sequence, per set of buffers and stream, into an executable CUDA
// graph on its second use and replays it afterwards with one launch.
#include "internal.cuh"

namespace nufft {

void drop_graphs(nufft_plan_t* p) {
  ++p->generation;   // graphs recorded elsewhere (frame sets) over this plan are stale too
  for (int i = 0; i < kGraphSlots; ++i) {
    if (p->graphs[i].state == 2 && p->graphs[i].exec) cudaGraphExecDestroy(p->graphs[i].exec);
    p->graphs[i] = GraphEntry{};
  }
}

int run_graphed_impl(nufft_plan_t* p, int kind, const void* a, const void* b, int64_t extra, int (*fn)(void*),
                     void* ctx) {
  if (!p->graphs_enabled) return fn(ctx);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(p->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return fn(ctx);   // the caller is capturing: our launches become part of its graph
  }
  GraphEntry* e = nullptr;
  for (int i = 0; i < kGraphSlots; ++i) {
    GraphEntry& g = p->graphs[i];
    if (g.kind == kind && g.a == a && g.b == b && g.extra == extra && g.stream == p->stream) { e = &g; break; }
  }
  if (!e) {   // first use: remember the key and run eagerly (lazy allocations happen here)
    GraphEntry* slot = &p->graphs[0];
    for (int i = 0; i < kGraphSlots; ++i) {
      if (p->graphs[i].kind == 0) { slot = &p->graphs[i]; break; }
      if (p->graphs[i].last_use < slot->last_use) slot = &p->graphs[i];
    }
    if (slot->state == 2 && slot->exec) cudaGraphExecDestroy(slot->exec);
    *slot = GraphEntry{kind, a, b, extra, p->stream, 1, nullptr, ++p->graph_clock};
    const int rc = fn(ctx);
    // a failed first call (e.g. a work-space allocation) does not count: the
    // next call runs eagerly again instead of allocating inside a capture
    if (rc != NUFFT_OK) *slot = GraphEntry{};
    return rc;
  }
  e->last_use = ++p->graph_clock;
  if (e->state == 3) return fn(ctx);
  if (e->state == 1) {   // second use: capture on the plan's own stream, then instantiate
    if (!p->capture_stream) {
      cudaError_t ce = cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking);
      if (ce != cudaSuccess) { p->capture_stream = nullptr; e->state = 3; cudaGetLastError(); return fn(ctx); }
    }
    cudaStream_t user = p->stream;
    p->stream = p->capture_stream;
    cudaGraph_t graph = nullptr;
    int rc = NUFFT_OK;
    cudaError_t be = cudaStreamBeginCapture(p->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (be == cudaSuccess) {
      rc = fn(ctx);
      cudaError_t ee = cudaStreamEndCapture(p->capture_stream, &graph);
      if (ee != cudaSuccess) rc = rc == NUFFT_OK ? NUFFT_ECUDA : rc;
    } else {
      rc = NUFFT_ECUDA;
    }
    p->stream = user;
    cudaGraphExec_t exec = nullptr;
    if (rc == NUFFT_OK && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
      e->exec = exec;
      e->state = 2;
    } else {
      e->state = 3;      // this sequence is not capturable: keep running it eagerly
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    snprintf(p->err, sizeof(p->err), "no error");
    if (e->state != 2) return fn(ctx);
  }
  const cudaError_t le = cudaGraphLaunch(e->exec, p->stream);
  return le == cudaSuccess ? NUFFT_OK : cuda_check(p, le, "graph launch");
}

}  // namespace nufft

using namespace nufft;

extern "C" int nufft_set_graphs(nufft_plan_t* p, int enable) {
  if (!p) return set_error(nullptr, NUFFT_EINVAL, "plan is NULL");
  if (!enable) drop_graphs(p);
  p->graphs_enabled = enable ? 1 : 0;
  return NUFFT_OK;
}
