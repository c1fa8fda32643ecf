// enkfmc_estimate_noalloc: the estimate step (anomalies and regressions of
// every component) without any device allocation.
//
// Some callers cannot let a library allocate device memory: a service that
// budgets every byte of GPU memory up front and hands out only what it has
// reserved, a host application whose own allocator owns the device, or a
// latency-critical loop that cannot afford cudaMalloc/cudaFree because they
// may synchronise the whole device and stall every other stream.  For them
// this entry point takes no handle and uses, as its only scratch, one
// file-scope device array of fixed size that exists on every GPU that loads
// the library, for as long as the process lives.
//
// Scratch layout (each part starting on a 256-byte boundary): the
// component-major anomalies U[n][ldN], the covariance table C[n][nC] (nC pair
// offsets per component), and for single-precision problems with rows where
// 2p > N their FP64 copies U64[n][ldN], C64[n][nC].  Every byte a call reads
// it has written first in the same call, so nothing needs clearing.
#include <cstring>
#include <mutex>

#include "enkfmc_internal.h"

using namespace enkfmc;

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on `dev` (looked up once per device,
// with that device current).  In host code the symbol itself is only a
// host-side stand-in, never a device address.
enkfmc_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return ENKFMC_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return ENKFMC_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return ENKFMC_OK;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Scratch bytes of a validated geometry (n < 2^31, ldN <= 128, nC < 2^15:
// no product below can wrap in 64 bits).
size_t scratch_need(const Geom& g, bool single, size_t* offC, size_t* offU64, size_t* offC64) {
  const size_t n = (size_t)g.n, nC = (size_t)cov_offset_count(g.r, g.vr);
  const size_t es = single ? sizeof(float) : sizeof(double);
  size_t off = round256(es * n * (size_t)g.ldN);
  *offC = off;
  off += round256(es * n * nC);
  *offU64 = *offC64 = 0;
  if (has_fp64_rows(g, single)) {
    *offU64 = off;
    off += round256(sizeof(double) * n * (size_t)g.ldN);
    *offC64 = off;
    off += round256(sizeof(double) * n * nC);
  }
  return off;
}

template <typename T>
enkfmc_status run(const Geom& g, double ridge_c, const T* Xb, T* Tv, T* D, unsigned char* base,
                  size_t offC, size_t offU64, size_t offC64, cudaStream_t s) {
  EstStats<T> st{reinterpret_cast<T*>(base), reinterpret_cast<T*>(base + offC),
                 offU64 ? reinterpret_cast<double*>(base + offU64) : nullptr,
                 offC64 ? reinterpret_cast<double*>(base + offC64) : nullptr};
  int nk = 0;
  cudaError_t e = launch_stat_anomalies<T>(g, Xb, st, s, &nk);
  if (e == cudaSuccess) e = launch_stat_covtables<T>(g, st, s, &nk);
  // no status word: a failed row shows as D = NaN with a zero T row
  if (e == cudaSuccess)
    e = launch_regressions<T>(g, st, nullptr, g.n, nullptr, Tv, D, ridge_c, nullptr, s, &nk);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return ENKFMC_ECUDA;
  }
  return ENKFMC_OK;
}

}  // namespace

extern "C" enkfmc_status enkfmc_estimate_noalloc(const enkfmc_problem* p, const void* Xb,
                                                 void* Tvals, void* D, void* cuda_stream) {
  if (!p || !Xb || !Tvals || !D) return ENKFMC_EINVAL;
  Geom g;
  enkfmc_status st = problem_geom(*p, g);  // every unsupported geometry: EINVAL here
  if (st) return st;
  const bool single = p->precision != ENKFMC_FP64;
  size_t offC, offU64, offC64;
  if (scratch_need(g, single, &offC, &offU64, &offC64) > kNoallocScratchBytes)
    return ENKFMC_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return ENKFMC_ECUDA;
  }
  if (cudaDeviceGetAttribute(&g.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    g.sm_count = 0;
  }
  void* base = nullptr;
  if ((st = scratch_address(dev, &base))) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  unsigned char* b = static_cast<unsigned char*>(base);
  if (!single)
    return run<double>(g, p->ridge_c, (const double*)Xb, (double*)Tvals, (double*)D, b, offC,
                       offU64, offC64, s);
  return run<float>(g, p->ridge_c, (const float*)Xb, (float*)Tvals, (float*)D, b, offC, offU64,
                    offC64, s);
}
