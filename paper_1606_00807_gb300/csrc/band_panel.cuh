// Panel steps shared by the band Cholesky kernels (k_band.cu, k_band_tc.cu).
//
// Storage: column-major lower band of one block, AB[c (hb + 1) + d] = A[c + d][c].
// A panel of nbc <= 32 columns starting at c0 and its rows [c0, c0 + rows) is
// staged column-major in shared memory, P[t ldP + i] = A[c0 + i][c0 + t].
#pragma once

#include <math.h>

#include "enkfmc_internal.h"

namespace enkfmc {

__device__ __forceinline__ bool finite_val(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_val(double v) { return isfinite(v); }

// Asynchronous global -> shared copy of one element (completed by
// panel_wait before the barrier that publishes the panel).
__device__ __forceinline__ void cp_elem(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_elem(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void panel_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Stage panel c0 (entries outside the band read as 0): every element is an
// independent asynchronous copy, so one thread's copies are all in flight at
// once; the caller runs panel_wait() and a barrier before reading P.
template <typename T>
__device__ __forceinline__ void load_panel(const T* __restrict__ AB, int ld, int hb, int c0,
                                           int nbc, int rows, T* P, int ldP) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = warp; t < nbc; t += nw) {
    const T* col = AB + (int64_t)(c0 + t) * ld;
    T* dst = P + t * ldP;
    for (int i = lane; i < rows; i += 32) {
      const int d = i - t;
      if (d >= 0 && d <= hb) cp_elem(dst + i, col + d);
      else dst[i] = T(0);
    }
  }
  panel_wait();
}

// Left-looking Cholesky of the staged panel, one thread per row: column t
// takes the products of the finished columns u < t, then its pivot.  Writes
// 1 / L[c0+t][c0+t] to inv_out[t] when inv_out is not null.  Returns false
// (the same value in every thread) at a pivot that is not positive: a finite
// one sets bfail[id] when bfail is given (the block is factored again in
// double precision), else records ENOTSPD; a non-finite one records
// ENONFINITE.
template <typename T>
__device__ bool factor_panel(T* P, int ldP, int nbc, int rows, T* inv_out, int32_t* status,
                             int* bfail, int id) {
  const int tid = threadIdx.x;
  for (int t = 0; t < nbc; ++t) {
    for (int i = t + tid; i < rows; i += blockDim.x) {
      T acc = P[t * ldP + i];
      for (int u = 0; u < t; ++u) acc = fma(-P[u * ldP + i], P[u * ldP + t], acc);
      P[t * ldP + i] = acc;
    }
    __syncthreads();
    T dg = P[t * ldP + t];
    if (!finite_val(dg) || !(dg > T(0))) {
      if (tid == 0) {
        if (bfail && finite_val(dg)) bfail[id] = 1;
        else record_error(status, finite_val(dg) ? ENKFMC_ENOTSPD : ENKFMC_ENONFINITE, (int64_t)id);
      }
      return false;
    }
    dg = sqrt(dg);
    const T inv = T(1) / dg;
    __syncthreads();
    for (int i = t + 1 + tid; i < rows; i += blockDim.x) P[t * ldP + i] *= inv;
    if (tid == 0) {
      P[t * ldP + t] = dg;
      if (inv_out) inv_out[t] = inv;
    }
    __syncthreads();
  }
  return true;
}

// Write the factored panel back to the band.
template <typename T>
__device__ __forceinline__ void write_panel(T* __restrict__ AB, int ld, int hb, int c0, int nbc,
                                            int rows, const T* P, int ldP) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = warp; t < nbc; t += nw) {
    T* col = AB + (int64_t)(c0 + t) * ld;
    for (int i = t + lane; i < rows && i - t <= hb; i += 32) col[i - t] = P[t * ldP + i];
  }
}

}  // namespace enkfmc
