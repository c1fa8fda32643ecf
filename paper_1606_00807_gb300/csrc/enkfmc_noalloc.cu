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
// Scratch layout: [0, 256) a 16-byte status word (cleared at every call),
// then the component-major anomalies U[n][ldN], then the covariance table
// C[n][nC] (nC pair offsets per component).
#include <cstring>
#include <mutex>

#include "enkfmc_internal.h"

using namespace enkfmc;

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr size_t kStatusBytes = 256;
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

// Geometry of a problem for the global regressions (no sub-domain tables).
enkfmc_status noalloc_geom(const enkfmc_problem& p, Geom& g) {
  const int nvar = p.nvar_3d + p.nvar_2d;
  if (p.nlon < 1 || p.nlat < 1 || p.nlev < 1 || p.nvar_3d < 0 || p.nvar_2d < 0 || nvar < 1 ||
      nvar > kMaxVar || p.r < 0 || p.r > 16 || p.vert_reach < 0 || p.N < 2 || p.N > 128 ||
      !(p.ridge_c >= 0.0))
    return ENKFMC_EINVAL;
  if (p.precision != ENKFMC_FP64 && p.precision != ENKFMC_FP32) return ENKFMC_EINVAL;
  if (p.lon_periodic && p.nlon < 2 * p.r + 1) return ENKFMC_EINVAL;
  std::memset(&g, 0, sizeof(g));
  g.nlon = p.nlon;
  g.nlat = p.nlat;
  g.nlev = p.nlev;
  g.nvar3 = p.nvar_3d;
  g.nvar2 = p.nvar_2d;
  g.nvar = nvar;
  g.r = p.r;
  g.vr = p.nvar_3d > 0 ? (p.vert_reach < p.nlev - 1 ? p.vert_reach : p.nlev - 1) : 0;
  g.periodic = p.lon_periodic ? 1 : 0;
  g.N = p.N;
  g.ldN = (p.N + 3) / 4 * 4;
  g.pmax = slot_count(g.r, g.vr, g.periodic);
  int64_t off = 0;
  for (int v = 0; v < nvar; ++v) {
    g.var_off[v] = off;
    g.var_lev[v] = v < p.nvar_3d ? p.nlev : 1;
    off += (int64_t)g.var_lev[v] * p.nlat * p.nlon;
  }
  g.var_off[nvar] = off;
  g.n = off;
  return ENKFMC_OK;
}

template <typename T>
enkfmc_status run(const Geom& g, double ridge_c, const T* Xb, T* Tv, T* D, unsigned char* base,
                  cudaStream_t s) {
  int32_t* status = reinterpret_cast<int32_t*>(base);
  T* U = reinterpret_cast<T*>(base + kStatusBytes);
  T* Cv = U + (size_t)g.n * g.ldN;
  if (cudaMemsetAsync(status, 0, 16, s) != cudaSuccess) {
    (void)cudaGetLastError();
    return ENKFMC_ECUDA;
  }
  cudaError_t e = launch_anomalies<T>(g, Xb, U, s);
  if (e == cudaSuccess) e = launch_covtable<T>(g, U, Cv, s);
  if (e == cudaSuccess)
    e = launch_regress<T>(g, U, Cv, nullptr, g.n, nullptr, Tv, D, ridge_c, status, s);
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
  enkfmc_status st = noalloc_geom(*p, g);
  if (st) return st;
  const size_t esize = p->precision == ENKFMC_FP64 ? sizeof(double) : sizeof(float);
  const size_t need =
      kStatusBytes + esize * (size_t)g.n * ((size_t)g.ldN + (size_t)cov_offset_count(g.r, g.vr));
  if (need > kNoallocScratchBytes) return ENKFMC_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return ENKFMC_ECUDA;
  }
  void* base = nullptr;
  if ((st = scratch_address(dev, &base))) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  unsigned char* b = static_cast<unsigned char*>(base);
  if (p->precision == ENKFMC_FP64)
    return run<double>(g, p->ridge_c, (const double*)Xb, (double*)Tvals, (double*)D, b, s);
  return run<float>(g, p->ridge_c, (const float*)Xb, (float*)Tvals, (float*)D, b, s);
}
