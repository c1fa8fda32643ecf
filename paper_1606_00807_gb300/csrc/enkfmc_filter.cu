// Filter cycling (Algorithm 1) on one handle: M analysis cycles with the
// synthetic forecast operator as the model step between them.  Cycle 0 runs
// eagerly (it also does every lazy set-up of the launches); the later cycles
// replay one CUDA graph of estimate -> assemble -> analyze -> squared error ->
// forecast, captured from a private stream on fixed buffers the handle keeps
// for it.  Before each replay the cycle's observations, perturbations and
// reference state are copied into those buffers on the caller's stream.
#include "enkfmc_internal.h"

namespace {

enkfmc_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return ENKFMC_OK;
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? ENKFMC_ENOMEM : ENKFMC_ECUDA;
}

enkfmc_status alloc_once(void** p, size_t bytes) {
  if (*p) return ENKFMC_OK;
  return cuda_status(cudaMalloc(p, bytes ? bytes : 16));
}

// One cycle on the handle's current stream from the fixed buffers.
enkfmc_status one_cycle(enkfmc_handle* h, void* Xb, const void* R, void* Tv, void* D, void* Xa,
                        int shift, double inflation) {
  enkfmc_status st = enkfmc_estimate(h, Xb, Tv, D);
  if (!st) st = enkfmc_assemble(h, Xb, Tv, D, R);
  if (!st) st = enkfmc_analyze(h, Xb, h->d_fy, R, h->d_fZ, Xa);
  if (!st) st = enkfmc_ensemble_sqerr(h, Xa, h->d_fx, h->d_fsq);
  if (!st) st = enkfmc_forecast_shift(h, Xa, Xb, h->g.N, shift, inflation);
  return st;
}

}  // namespace

extern "C" enkfmc_status enkfmc_filter_run(enkfmc_handle* h, void* Xb, const void* ys,
                                           const void* Zs, const void* Rdiag, const void* xrefs,
                                           void* Tvals, void* D, void* Xa, int32_t M,
                                           int32_t shift, double inflation, double* sqerr) {
  if (!h || !Xb || !xrefs || !Tvals || !D || !Xa || !sqerr || M < 1 || Xa == Xb ||
      !(inflation > 0.0) || inflation > 1e3)
    return ENKFMC_EINVAL;
  enkfmc_info info;
  enkfmc_query(h, &info);
  const int64_t m = info.m;
  if (m < 0) return ENKFMC_ESTATE;
  if (m > 0 && (!ys || !Zs || !Rdiag)) return ENKFMC_EINVAL;
  const size_t es = h->esize;
  const int64_t n = h->g.n, N = h->g.N;
  enkfmc_status st = alloc_once(&h->d_fy, es * m);
  if (!st) st = alloc_once(&h->d_fZ, es * N * m);
  if (!st) st = alloc_once(&h->d_fx, es * n);
  if (!st) st = alloc_once(reinterpret_cast<void**>(&h->d_fsq), sizeof(double));
  if (!st && !h->f_stream)
    st = cuda_status(cudaStreamCreateWithFlags(&h->f_stream, cudaStreamNonBlocking));
  if (st) return st;
  const void* R = m > 0 ? Rdiag : h->d_fy;
  cudaStream_t user = h->stream;
  auto stage = [&](int k) -> enkfmc_status {  // cycle k's inputs into the fixed buffers
    cudaError_t e = cudaSuccess;
    if (m > 0) {
      e = cudaMemcpyAsync(h->d_fy, (const char*)ys + (size_t)k * m * es, m * es,
                          cudaMemcpyDeviceToDevice, user);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_fZ, (const char*)Zs + (size_t)k * N * m * es, N * m * es,
                            cudaMemcpyDeviceToDevice, user);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->d_fx, (const char*)xrefs + (size_t)k * n * es, n * es,
                          cudaMemcpyDeviceToDevice, user);
    return cuda_status(e);
  };
  auto read_sq = [&](int k) {
    return cuda_status(
        cudaMemcpyAsync(sqerr + k, h->d_fsq, sizeof(double), cudaMemcpyDeviceToDevice, user));
  };
  st = stage(0);
  if (!st) st = one_cycle(h, Xb, R, Tvals, D, Xa, shift, inflation);
  if (!st) st = read_sq(0);
  if (st || M == 1) return st;

  // capture one cycle on the private stream (the caller's stream may be the
  // legacy default stream, which cannot be captured), kernel timing off
  if ((st = cuda_status(cudaStreamSynchronize(user)))) return st;
  const bool prof = h->prof;
  h->prof = false;
  h->stream = h->f_stream;
  cudaGraph_t graph = nullptr;
  st = cuda_status(cudaStreamBeginCapture(h->f_stream, cudaStreamCaptureModeRelaxed));
  if (!st) {
    const enkfmc_status sc = one_cycle(h, Xb, R, Tvals, D, Xa, shift, inflation);
    const cudaError_t e = cudaStreamEndCapture(h->f_stream, &graph);
    st = sc ? sc : cuda_status(e);
  }
  h->stream = user;
  h->prof = prof;
  cudaGraphExec_t exec = nullptr;
  if (!st) st = cuda_status(cudaGraphInstantiate(&exec, graph, 0));
  for (int k = 1; k < M && !st; ++k) {
    st = stage(k);
    if (!st) st = cuda_status(cudaGraphLaunch(exec, user));
    if (!st) st = read_sq(k);
  }
  const enkfmc_status ss = cuda_status(cudaStreamSynchronize(user));
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  return st ? st : ss;
}
