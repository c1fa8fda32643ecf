// Many independent assimilation problems (instances of uneven grid, ensemble
// size and radius) run as one CUDA graph.  The paper analyses independent
// sub-domains in parallel (Section 3, Algorithm 2); here whole instances are
// independent as well.  Each instance keeps its own handle (tables, workspace,
// status word).  Its estimate -> assemble -> analyze sequence is recorded on
// one of several side streams forked from the batch's stream.  Instances are
// placed longest first on the least loaded stream, by the handle's algorithmic
// work, so small and large instances overlap.  The whole fan-out is captured
// once and replayed with a single graph launch per cycle.
#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "enkfmc_internal.h"

struct enkfmc_batch {
  std::vector<enkfmc_handle*> h;
  struct Bind {
    const void *Xb = nullptr, *y = nullptr, *R = nullptr, *Z = nullptr;
    void *T = nullptr, *D = nullptr, *Xa = nullptr;
    bool set = false;
  };
  std::vector<Bind> bind;
  std::vector<int> stream_of;  // side stream of each instance
  cudaStream_t stream = nullptr;  // the caller's stream: graph launches, status reads
  cudaStream_t origin = nullptr;  // capture origin (the legacy default stream cannot be captured)
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;  // fork, then one join event per side stream
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

enkfmc_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return ENKFMC_OK;
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? ENKFMC_ENOMEM : ENKFMC_ECUDA;
}

void free_batch(enkfmc_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  for (cudaStream_t s : b->side) cudaStreamDestroy(s);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

// One analysis cycle of instance i on stream s (the handle's stream meanwhile).
enkfmc_status run_instance(enkfmc_batch* b, int i, cudaStream_t s) {
  enkfmc_handle* h = b->h[i];
  const enkfmc_batch::Bind& x = b->bind[i];
  enkfmc_status st = enkfmc_set_stream(h, s);
  if (!st) st = enkfmc_estimate(h, x.Xb, x.T, x.D);
  if (!st) st = enkfmc_assemble(h, x.Xb, x.T, x.D, x.R);
  if (!st) st = enkfmc_analyze(h, x.Xb, x.y, x.R, x.Z, x.Xa);
  return st;
}

}  // namespace

extern "C" enkfmc_status enkfmc_batch_create(enkfmc_batch** out, enkfmc_handle* const* handles,
                                  int32_t nprob, int32_t nstreams, void* cuda_stream) {
  if (!out || !handles || nprob < 1 || nstreams < 1 || nstreams > 64) return ENKFMC_EINVAL;
  *out = nullptr;
  enkfmc_batch* b = new (std::nothrow) enkfmc_batch();
  if (!b) return ENKFMC_ENOMEM;
  b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  for (int i = 0; i < nprob; ++i) {
    if (!handles[i]) {
      delete b;
      return ENKFMC_EINVAL;
    }
    b->h.push_back(handles[i]);
  }
  b->bind.resize(nprob);
  const int ns = std::min(nstreams, nprob);
  if (enkfmc_status st = cuda_status(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking))) {
    free_batch(b);
    return st;
  }
  for (int k = 0; k < ns; ++k) {
    cudaStream_t s = nullptr;
    enkfmc_status st = cuda_status(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    if (st) {
      free_batch(b);
      return st;
    }
    b->side.push_back(s);
  }
  for (int k = 0; k <= ns; ++k) {
    cudaEvent_t e = nullptr;
    enkfmc_status st = cuda_status(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (st) {
      free_batch(b);
      return st;
    }
    b->ev.push_back(e);
  }
  // longest processing time first onto the least loaded stream
  std::vector<double> cost(nprob, 0.0);
  for (int i = 0; i < nprob; ++i)
    for (int k = 0; k < ENKFMC_NKERNEL; ++k) cost[i] += b->h[i]->work_flops[k];
  std::vector<int> order(nprob);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  std::vector<double> load(ns, 0.0);
  b->stream_of.assign(nprob, 0);
  for (int i : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->stream_of[i] = k;
    load[k] += cost[i];
  }
  *out = b;
  return ENKFMC_OK;
}

extern "C" enkfmc_status enkfmc_batch_bind(enkfmc_batch* b, int32_t i, const void* Xb, void* Tvals, void* D,
                                const void* y, const void* Rdiag, const void* Z, void* Xa) {
  if (!b || i < 0 || i >= (int)b->h.size() || !Xb || !Tvals || !D || !Xa || Xa == Xb)
    return ENKFMC_EINVAL;
  enkfmc_info info;
  enkfmc_query(b->h[i], &info);
  if (info.m < 0) return ENKFMC_ESTATE;
  if (info.m > 0 && (!y || !Rdiag || !Z)) return ENKFMC_EINVAL;
  b->bind[i] = {Xb, y, Rdiag, Z, Tvals, D, Xa, true};
  if (b->exec) {  // a new binding invalidates the captured graph
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  return ENKFMC_OK;
}

namespace {

// The eager cycle and the capture (see enkfmc_batch_capture); the handles'
// streams are the side streams meanwhile.
enkfmc_status capture_cycle(enkfmc_batch* b) {
  const int n = (int)b->h.size(), ns = (int)b->side.size();
  // the side streams do not order against the caller's stream: let the
  // caller's work on the inputs finish first
  if (enkfmc_status st = cuda_status(cudaStreamSynchronize(b->stream))) return st;
  // one eager cycle per instance: the lazy set-up of every launch happens
  // outside the capture, and numerical failures show before any replay
  for (int i = 0; i < n; ++i) {
    enkfmc_status st = run_instance(b, i, b->side[b->stream_of[i]]);
    if (st) return st;
  }
  for (cudaStream_t s : b->side)
    if (enkfmc_status st = cuda_status(cudaStreamSynchronize(s))) return st;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  // capture: fork the side streams from the origin stream, run every
  // instance on its stream, join them back.  The graph is launched on the
  // caller's stream, which may be the legacy default stream.
  enkfmc_status st =
      cuda_status(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed));
  if (st) return st;
  cudaError_t e = cudaEventRecord(b->ev[0], b->origin);
  for (int k = 0; k < ns && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[k], b->ev[0], 0);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    st = run_instance(b, i, b->side[b->stream_of[i]]);
    if (st) e = cudaErrorUnknown;
  }
  for (int k = 0; k < ns && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b->ev[k + 1], b->side[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->ev[k + 1], 0);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(b->origin, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    (void)cudaGetLastError();
    return st ? st : ENKFMC_ECUDA;
  }
  b->graph = g;
  if ((st = cuda_status(cudaGraphInstantiate(&b->exec, g, 0)))) {
    cudaGraphDestroy(g);
    b->graph = nullptr;
    b->exec = nullptr;
    return st;
  }
  return ENKFMC_OK;
}

}  // namespace

extern "C" enkfmc_status enkfmc_batch_capture(enkfmc_batch* b) {
  if (!b) return ENKFMC_EINVAL;
  const int n = (int)b->h.size();
  for (int i = 0; i < n; ++i)
    if (!b->bind[i].set) return ENKFMC_ESTATE;
  for (enkfmc_handle* h : b->h) enkfmc_profile(h, 0);
  const enkfmc_status st = capture_cycle(b);
  // success or not, every handle is back on the batch's stream: the side
  // streams end with the batch
  for (int i = 0; i < n; ++i) enkfmc_set_stream(b->h[i], b->stream);
  return st;
}

extern "C" {

enkfmc_status enkfmc_batch_run(enkfmc_batch* b) {
  if (!b) return ENKFMC_EINVAL;
  if (!b->exec) return ENKFMC_ESTATE;
  return cuda_status(cudaGraphLaunch(b->exec, b->stream));
}

enkfmc_status enkfmc_batch_get_status(enkfmc_batch* b, int32_t* status, int64_t* info) {
  if (!b || !status) return ENKFMC_EINVAL;
  if (enkfmc_status st = cuda_status(cudaStreamSynchronize(b->stream))) return st;
  enkfmc_status first = ENKFMC_OK;
  for (size_t i = 0; i < b->h.size(); ++i) {
    int64_t inf = 0;
    const enkfmc_status s = enkfmc_get_status(b->h[i], &inf);
    status[i] = (int32_t)s;
    if (info) info[i] = inf;
    if (s && !first) first = s;
  }
  return first;
}

enkfmc_status enkfmc_batch_query(const enkfmc_batch* b, int32_t* nstreams, int32_t* stream_of) {
  if (!b) return ENKFMC_EINVAL;
  if (nstreams) *nstreams = (int32_t)b->side.size();
  if (stream_of)
    for (size_t i = 0; i < b->h.size(); ++i) stream_of[i] = b->stream_of[i];
  return ENKFMC_OK;
}

void enkfmc_batch_destroy(enkfmc_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  for (cudaStream_t s : b->side) cudaStreamSynchronize(s);
  free_batch(b);
}

enkfmc_status enkfmc_set_tuning(enkfmc_handle* h, int32_t knob, int32_t value) {
  if (!h || value < 0) return ENKFMC_EINVAL;
  switch (knob) {
    case ENKFMC_TUNE_REGRESS_CTAS_PER_SM:
      if (value > 1024) return ENKFMC_EINVAL;
      h->g.regress_cap = value;
      return ENKFMC_OK;
    case ENKFMC_TUNE_REGRESS_KERNEL:
      if (value > 3) return ENKFMC_EINVAL;
      h->g.regress_kernel = value;
      return ENKFMC_OK;
  }
  return ENKFMC_EINVAL;
}

}  // extern "C"
