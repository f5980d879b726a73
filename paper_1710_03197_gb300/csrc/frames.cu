// frames.cu - dynamic series: the multi-coil normal operator of every frame in
// one recorded CUDA graph.
//
// Section 2.2.3 (Eqs. 32-33) per frame f of a dynamic acquisition: the frames
// share the image geometry and the coil maps but each has its own trajectory
// (its own plan, with any number of points), and
//   out_f = sum_i conj(c_i) . A_f^H A_f (c_i . x_f).
// A frame set records the launches of all frames once, each frame on a branch
// of its own (fork from one event, join on the frames' events), and replays
// that graph as one launch into the caller's stream: the frames run
// concurrently and the host issues one launch per call.
#include <vector>

#include "internal.cuh"

namespace nufft {
int selfadjoint_multicoil_impl(nufft_plan_t* p, const float2* coils, int nc, const float2* x, float2* out);
}  // namespace nufft

using namespace nufft;

struct nufft_frames {
  std::vector<nufft_plan_t*> plans;
  cudaStream_t stream = nullptr;        // replays go here
  cudaStream_t cap = nullptr;           // capture origin
  std::vector<cudaStream_t> branch;     // one per frame, used while capturing
  std::vector<cudaEvent_t> done;        // one per frame (join)
  cudaEvent_t fork = nullptr;
  // the one recorded call: key, state (0 none, 1 seen once, 2 recorded, 3 eager only)
  const void* kcoils = nullptr;
  const void* kx = nullptr;
  const void* kout = nullptr;
  int knc = 0;
  std::vector<uint64_t> kgen;           // the plans' generations when the key was taken
  int state = 0;
  cudaGraphExec_t exec = nullptr;
};

namespace {
void release(nufft_frames* fs) {
  if (fs->exec) cudaGraphExecDestroy(fs->exec);
  for (cudaStream_t s : fs->branch)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : fs->done)
    if (e) cudaEventDestroy(e);
  if (fs->fork) cudaEventDestroy(fs->fork);
  if (fs->cap) cudaStreamDestroy(fs->cap);
  delete fs;
}

int run_frames(nufft_frames* fs, const float2* coils, int nc, const float2* x, float2* out, bool branches) {
  const int nf = (int)fs->plans.size();
  const int64_t n = fs->plans[0]->Nprod;
  cudaStream_t origin = branches ? fs->cap : fs->stream;
  if (branches && cudaEventRecord(fs->fork, origin) != cudaSuccess) return NUFFT_ECUDA;
  int rc = NUFFT_OK;
  for (int f = 0; f < nf && rc == NUFFT_OK; ++f) {
    nufft_plan_t* p = fs->plans[f];
    cudaStream_t keep = p->stream;
    p->stream = branches ? fs->branch[f] : fs->stream;
    if (branches && cudaStreamWaitEvent(p->stream, fs->fork, 0) != cudaSuccess) rc = NUFFT_ECUDA;
    if (rc == NUFFT_OK) rc = selfadjoint_multicoil_impl(p, coils, nc, x + f * n, out + f * n);
    if (rc == NUFFT_OK && branches) {
      if (cudaEventRecord(fs->done[f], p->stream) != cudaSuccess ||
          cudaStreamWaitEvent(origin, fs->done[f], 0) != cudaSuccess)
        rc = NUFFT_ECUDA;
    }
    p->stream = keep;
  }
  return rc;
}
}  // namespace

extern "C" int nufft_frames_create(nufft_plan_t* const* plans, int nframes, void* stream, nufft_frames_t** out) {
  if (!out) return set_error(nullptr, NUFFT_EINVAL, "out is NULL");
  *out = nullptr;
  if (!plans || nframes < 1) return set_error(nullptr, NUFFT_EINVAL, "plans is NULL or nframes < 1");
  for (int f = 0; f < nframes; ++f) {
    if (!plans[f]) return set_error(nullptr, NUFFT_EINVAL, "plans[%d] is NULL", f);
    const Geom &a = plans[0]->g, &b = plans[f]->g;
    bool same = a.d == b.d;
    for (int i = 0; same && i < a.d; ++i) same = a.N[i] == b.N[i];
    if (!same) return set_error(nullptr, NUFFT_EINVAL, "plans[%d] has another image geometry than plans[0]", f);
    for (int g = 0; g < f; ++g)
      if (plans[g] == plans[f]) return set_error(nullptr, NUFFT_EINVAL, "plans[%d] repeats plans[%d]", f, g);
  }
  nufft_frames* fs = new (std::nothrow) nufft_frames;
  if (!fs) return set_error(nullptr, NUFFT_ENOMEM, "host allocation of the frame set failed");
  fs->plans.assign(plans, plans + nframes);
  fs->stream = (cudaStream_t)stream;
  fs->branch.assign(nframes, nullptr);
  fs->done.assign(nframes, nullptr);
  cudaError_t e = cudaStreamCreateWithFlags(&fs->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fs->fork, cudaEventDisableTiming);
  for (int f = 0; f < nframes && e == cudaSuccess; ++f) {
    e = cudaStreamCreateWithFlags(&fs->branch[f], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fs->done[f], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    release(fs);
    return cuda_check(nullptr, e, "frame set streams");
  }
  *out = fs;
  return NUFFT_OK;
}

extern "C" int nufft_frames_destroy(nufft_frames_t* fs) {
  if (!fs) return NUFFT_OK;
  cudaStreamSynchronize(fs->stream);
  release(fs);
  return NUFFT_OK;
}

extern "C" int nufft_frames_set_stream(nufft_frames_t* fs, void* stream) {
  if (!fs) return set_error(nullptr, NUFFT_EINVAL, "frame set is NULL");
  fs->stream = (cudaStream_t)stream;
  return NUFFT_OK;
}

extern "C" int nufft_frames_selfadjoint_multicoil(nufft_frames_t* fs, const float* coils_dev, int nc, const float* x_dev,
                                                  float* out_dev) {
  if (!fs) return set_error(nullptr, NUFFT_EINVAL, "frame set is NULL");
  if (!coils_dev || !x_dev || !out_dev || nc < 1)
    return set_error(nullptr, NUFFT_EINVAL, "coils_dev, x_dev or out_dev is NULL, or nc < 1");
  if ((const void*)x_dev == (const void*)out_dev) return set_error(nullptr, NUFFT_EINVAL, "x_dev and out_dev alias");
  const float2* coils = reinterpret_cast<const float2*>(coils_dev);
  const float2* x = reinterpret_cast<const float2*>(x_dev);
  float2* out = reinterpret_cast<float2*>(out_dev);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(fs->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return run_frames(fs, coils, nc, x, out, false);   // inside the caller's capture
  }
  bool same = fs->kcoils == coils_dev && fs->kx == x_dev && fs->kout == out_dev && fs->knc == nc &&
              fs->kgen.size() == fs->plans.size();
  for (size_t f = 0; same && f < fs->plans.size(); ++f) same = fs->kgen[f] == fs->plans[f]->generation;
  if (!same || fs->state == 0) {   // first use of these buffers (or a plan changed): eager
    if (fs->exec) cudaGraphExecDestroy(fs->exec);
    fs->exec = nullptr;
    fs->kcoils = coils_dev;
    fs->kx = x_dev;
    fs->kout = out_dev;
    fs->knc = nc;
    fs->state = 1;
    const int rc = run_frames(fs, coils, nc, x, out, false);   // lazy allocations happen here
    fs->kgen.resize(fs->plans.size());
    for (size_t f = 0; f < fs->plans.size(); ++f) fs->kgen[f] = fs->plans[f]->generation;
    return rc;
  }
  if (fs->state == 3) return run_frames(fs, coils, nc, x, out, false);
  if (fs->state == 1) {   // second use: record the frames as branches of one graph
    cudaGraph_t graph = nullptr;
    int rc = NUFFT_ECUDA;
    if (cudaStreamBeginCapture(fs->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      rc = run_frames(fs, coils, nc, x, out, true);
      if (cudaStreamEndCapture(fs->cap, &graph) != cudaSuccess) rc = NUFFT_ECUDA;
    }
    if (rc == NUFFT_OK && graph && cudaGraphInstantiate(&fs->exec, graph, 0) == cudaSuccess) {
      fs->state = 2;
    } else {
      fs->exec = nullptr;
      fs->state = 3;   // not capturable: keep running eagerly
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (fs->state != 2) return run_frames(fs, coils, nc, x, out, false);
  }
  const cudaError_t le = cudaGraphLaunch(fs->exec, fs->stream);
  return le == cudaSuccess ? NUFFT_OK : cuda_check(nullptr, le, "frame set graph launch");
}
