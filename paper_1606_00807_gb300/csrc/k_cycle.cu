// Filter cycling (Algorithm 1): the model step between analyses and the
// analysis error of Eq. 18.  The paper's model (SPEEDY) is replaced by a
// synthetic forecast operator: advection of every field along its latitude
// circle by a whole number of cells per step (periodic in longitude), which
// carries the seeded random fields without changing their statistics, with
// optional multiplicative covariance inflation about the ensemble mean (a
// permutation has no model error, so without it the spread only shrinks).
#include "enkfmc_internal.h"

namespace enkfmc {

namespace {

// Y[row][(x + shift) mod nlon] = X[row][x] for rows of nlon values (every
// latitude circle of every level, variable and state vector); 0 <= shift < nlon.
template <typename T>
__global__ void __launch_bounds__(256) k_shift(const T* __restrict__ X, T* __restrict__ Y,
                                               int64_t nrows, int nlon, int shift) {
  const int64_t total = nrows * nlon;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / nlon;
    int xs = (int)(e - row * nlon) + shift;
    if (xs >= nlon) xs -= nlon;
    Y[row * nlon + xs] = X[e];
  }
}

// The same advection with multiplicative covariance inflation about the
// ensemble mean: Y[v][l'] = mean + rho (X[v][l] - mean), mean over the nvec
// vectors (member-major, stride n) in double precision; one thread per
// component of a latitude circle, the vectors in a loop.
template <typename T>
__global__ void __launch_bounds__(256) k_shift_inflate(const T* __restrict__ X, T* __restrict__ Y,
                                                       int64_t n, int nvec, int nlon, int shift,
                                                       double rho) {
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = l / nlon;
    int xs = (int)(l - row * nlon) + shift;
    if (xs >= nlon) xs -= nlon;
    const int64_t lo = row * nlon + xs;
    double s = 0.0;
    for (int v = 0; v < nvec; ++v) s += (double)X[(int64_t)v * n + l];
    const double mean = s / nvec;
    for (int v = 0; v < nvec; ++v)
      Y[(int64_t)v * n + lo] = (T)(mean + rho * ((double)X[(int64_t)v * n + l] - mean));
  }
}

// Partial sums of (mean_m Xa[m][l] - xref[l])^2, the ensemble mean and the
// squares in double precision; block b sums the components l = b * 256 + t +
// k * kSqGrid * 256 and reduces them in a fixed tree, so the result does not
// depend on scheduling.
template <typename T>
__global__ void __launch_bounds__(256) k_sqerr_part(const T* __restrict__ Xa,
                                                    const T* __restrict__ xref, int64_t n, int N,
                                                    double* __restrict__ part) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t l = (int64_t)blockIdx.x * 256 + threadIdx.x; l < n; l += (int64_t)kSqGrid * 256) {
    double s = 0.0;
    for (int m = 0; m < N; ++m) s += (double)Xa[(int64_t)m * n + l];
    const double e = s / N - (double)xref[l];
    acc = fma(e, e, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) k_sqerr_final(const double* __restrict__ part,
                                                     double* __restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < kSqGrid; i += 256) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

template <typename T>
cudaError_t launch_shift(const Geom& g, const T* X, T* Y, int nvec, int shift, double rho,
                         cudaStream_t s) {
  if (rho != 1.0) {
    int64_t grid = (g.n + 255) / 256;
    const int64_t cap = (int64_t)(g.sm_count > 0 ? g.sm_count : 152) * 8;
    if (grid > cap) grid = cap;
    k_shift_inflate<T><<<(unsigned)grid, 256, 0, s>>>(X, Y, g.n, nvec, g.nlon, shift, rho);
    return cudaGetLastError();
  }
  const int64_t nrows = (int64_t)nvec * (g.n / g.nlon);
  const int64_t total = nrows * g.nlon;
  if (total <= 0) return cudaSuccess;
  int64_t grid = (total + 255) / 256;
  const int64_t cap = (int64_t)(g.sm_count > 0 ? g.sm_count : 152) * 8;
  if (grid > cap) grid = cap;
  k_shift<T><<<(unsigned)grid, 256, 0, s>>>(X, Y, nrows, g.nlon, shift);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sqerr(const Geom& g, const T* Xa, const T* xref, double* part, double* out,
                         cudaStream_t s) {
  k_sqerr_part<T><<<kSqGrid, 256, 0, s>>>(Xa, xref, g.n, g.N, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sqerr_final<<<1, 256, 0, s>>>(part, out);
  return cudaGetLastError();
}

template cudaError_t launch_shift<float>(const Geom&, const float*, float*, int, int, double,
                                         cudaStream_t);
template cudaError_t launch_shift<double>(const Geom&, const double*, double*, int, int, double,
                                          cudaStream_t);
template cudaError_t launch_sqerr<float>(const Geom&, const float*, const float*, double*,
                                         double*, cudaStream_t);
template cudaError_t launch_sqerr<double>(const Geom&, const double*, const double*, double*,
                                          double*, cudaStream_t);

}  // namespace enkfmc
