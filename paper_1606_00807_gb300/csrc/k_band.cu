// Batched banded Cholesky A = L L^T and the solves L L^T dX = rhs with N
// right-hand sides (Eq. 11), one thread block per (sub-domain, variable)
// block of A.
//
// Storage: column-major lower band, band[c * (hb + 1) + d] = A[c + d][c];
// the factor overwrites A.  Right-hand sides are column-major per block,
// rhs[m * nb + i].
//
// Factorisation (right-looking, panel width NB): a panel of NB columns and
// its nb_rows = NB + hb rows is staged in shared memory, factored column by
// column, written back, and its rank-NB update is applied to the trailing
// hb x hb window of the band with 4x4 register tiles.  The window of a block
// in flight is a few hundred KB, so the read-modify-write traffic stays in L2.
//
// Forward solve: per panel, the NB x NB triangle is solved for every member
// (one thread per member), then the rows below are updated with a 4x4 tiled
// product.  Back solve: per panel from the last one, the already solved rows
// below the panel are staged in chunks and contracted against the panel, then
// the triangle is solved backwards.
#include <math.h>

#include "enkfmc_internal.h"

namespace enkfmc {

namespace {

constexpr int NB = 32;
constexpr int kThreads = 256;

__device__ __forceinline__ bool finite_val(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_val(double v) { return isfinite(v); }

// Column-major tile index over the lower triangle of an nT x nT tile grid:
// tiles of column C are (C, C), (C+1, C), ..., (nT-1, C).
__device__ __forceinline__ void tri_tile(int idx, int nT, int& I, int& C) {
  // number of tiles before column C: S(C) = C*nT - C*(C-1)/2
  const float fn = (float)nT + 0.5f;
  int c = (int)(fn - sqrtf(fn * fn - 2.f * (float)idx));
  if (c < 0) c = 0;
  if (c > nT - 1) c = nT - 1;
  while (c > 0 && c * nT - c * (c - 1) / 2 > idx) --c;
  while ((c + 1) * nT - (c + 1) * c / 2 <= idx) ++c;
  C = c;
  I = C + (idx - (C * nT - C * (C - 1) / 2));
}

template <typename T>
__device__ __forceinline__ void load_panel(const T* __restrict__ AB, int ld, int hb, int c0,
                                           int nbc, int rows, T* P, int ldP) {
  for (int idx = threadIdx.x; idx < nbc * rows; idx += blockDim.x) {
    const int t = idx / rows, i = idx - t * rows;
    const int d = i - t;
    T v = T(0);
    if (d >= 0 && d <= hb) v = AB[(int64_t)(c0 + t) * ld + d];
    P[t * ldP + i] = v;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_bandchol(const Block* __restrict__ blocks,
                                                       T* __restrict__ band, int32_t* status,
                                                       int ldP) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* P = reinterpret_cast<T*>(smem);  // [NB][ldP]: P[t*ldP + i] = A[c0+i][c0+t]
  const Block b = blocks[blockIdx.x];
  const int nb = b.nb, hb = b.hb, ld = hb + 1;
  T* AB = band + b.band_off;
  const int tid = threadIdx.x;
  for (int c0 = 0; c0 < nb; c0 += NB) {
    const int nbc = min(NB, nb - c0);
    const int rows = min(nbc + hb, nb - c0);
    load_panel(AB, ld, hb, c0, nbc, rows, P, ldP);
    __syncthreads();
    for (int t = 0; t < nbc; ++t) {
      T dg = P[t * ldP + t];
      if (!finite_val(dg) || !(dg > T(0))) {
        if (tid == 0)
          record_error(status, finite_val(dg) ? ENKFMC_ENOTSPD : ENKFMC_ENONFINITE,
                       (int64_t)blockIdx.x);
        return;  // uniform: every thread read the same pivot
      }
      dg = sqrt(dg);
      __syncthreads();
      const T inv = T(1) / dg;
      for (int i = t + 1 + tid; i < rows; i += blockDim.x) P[t * ldP + i] *= inv;
      if (tid == 0) P[t * ldP + t] = dg;
      __syncthreads();
      const int ncol = nbc - t - 1;
      for (int idx = tid; idx < ncol * rows; idx += blockDim.x) {
        const int u = t + 1 + idx / rows;
        const int i = idx - (u - t - 1) * rows;
        if (i >= u) P[u * ldP + i] -= P[t * ldP + i] * P[t * ldP + u];
      }
      __syncthreads();
    }
    // write the factored panel
    for (int idx = tid; idx < nbc * rows; idx += blockDim.x) {
      const int t = idx / rows, i = idx - t * rows;
      const int d = i - t;
      if (d >= 0 && d <= hb) AB[(int64_t)(c0 + t) * ld + d] = P[t * ldP + i];
    }
    // trailing update of the window [c0+nbc, c0+rows)
    const int W = rows - nbc;
    if (W > 0) {
      const int nT = (W + 3) >> 2;
      const int ntiles = nT * (nT + 1) / 2;
      for (int tile = tid; tile < ntiles; tile += blockDim.x) {
        int I, C;
        tri_tile(tile, nT, I, C);
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][c] = T(0);
        const int i0 = nbc + 4 * I, j0 = nbc + 4 * C;
        for (int t = 0; t < nbc; ++t) {
          const T* Pt = P + t * ldP;
          T av[4], bv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) av[a] = (i0 + a < rows) ? Pt[i0 + a] : T(0);
#pragma unroll
          for (int c = 0; c < 4; ++c) bv[c] = (j0 + c < rows) ? Pt[j0 + c] : T(0);
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int jj = 4 * C + c;  // window-relative column
          if (jj >= W) continue;
          T* colp = AB + (int64_t)(c0 + nbc + jj) * ld;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int ii = 4 * I + a;
            if (ii < W && ii >= jj) colp[ii - jj] -= acc[a][c];
          }
        }
      }
    }
    __syncthreads();
  }
}

constexpr int NM = 32;       // members per thread block in the solves
constexpr int NMP = NM + 4;  // padded row of the right-hand-side window

// Solve L L^T X = B for members [m0, m0 + NM) of one block.  The rows of B
// the current panel touches (NB + hb of them) live in a circular window of WR
// rows in shared memory (row i in slot i % WR); finished rows go back to
// global memory and the next ones are read in their place.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bandsolve(const Block* __restrict__ blocks,
                                                        const T* __restrict__ band,
                                                        T* __restrict__ rhs, int N, int ldP,
                                                        int WRmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* P = reinterpret_cast<T*>(smem);   // [NB][ldP]
  T* Wn = P + (size_t)NB * ldP;        // [WRmax][NMP]
  T* Red = Wn + (size_t)WRmax * NMP;   // [4][NB][NM] partial sums
  const Block b = blocks[blockIdx.x];
  const int m0 = blockIdx.y * NM;
  const int nm = min(NM, N - m0);
  const int nb = b.nb, hb = b.hb, ld = hb + 1;
  const int WR = ((NB + hb + NB - 1) / NB) * NB;
  const T* AB = band + b.band_off;
  T* B = rhs + b.row_off * N + (int64_t)m0 * nb;  // B[m * nb + i], m relative to m0
  const int tid = threadIdx.x;

  auto load_rows = [&](int r0, int cnt) {
    for (int idx = tid; idx < cnt * nm; idx += blockDim.x) {
      const int m = idx / cnt, i = idx - m * cnt;
      Wn[((r0 + i) % WR) * NMP + m] = B[(int64_t)m * nb + r0 + i];
    }
  };
  auto store_rows = [&](int r0, int cnt) {
    for (int idx = tid; idx < cnt * nm; idx += blockDim.x) {
      const int m = idx / cnt, i = idx - m * cnt;
      B[(int64_t)m * nb + r0 + i] = Wn[((r0 + i) % WR) * NMP + m];
    }
  };

  // ---- forward: L Y = B ----
  load_rows(0, min(WR, nb));
  for (int c0 = 0; c0 < nb; c0 += NB) {
    const int nbc = min(NB, nb - c0);
    const int rows = min(nbc + hb, nb - c0);
    load_panel(AB, ld, hb, c0, nbc, rows, P, ldP);
    __syncthreads();
    if (tid < nm) {
      for (int t = 0; t < nbc; ++t) {
        T* wt = Wn + ((c0 + t) % WR) * NMP + tid;
        const T yt = *wt / P[t * ldP + t];
        *wt = yt;
        for (int i = t + 1; i < nbc; ++i) Wn[((c0 + i) % WR) * NMP + tid] -= P[t * ldP + i] * yt;
      }
    }
    __syncthreads();
    const int Wr = rows - nbc;
    const int nTi = (Wr + 3) >> 2;
    for (int tile = tid; tile < nTi * (NM / 8); tile += blockDim.x) {
      const int Ti = tile / (NM / 8), Tm = tile - Ti * (NM / 8);
      const int i0 = nbc + 4 * Ti, mm0 = 8 * Tm;
      if (mm0 >= nm) continue;
      T acc[4][8];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[a][c] = T(0);
      for (int t = 0; t < nbc; ++t) {
        T av[4], yv[8];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = (i0 + a < rows) ? P[t * ldP + i0 + a] : T(0);
        const T* yr = Wn + ((c0 + t) % WR) * NMP + mm0;
#pragma unroll
        for (int c = 0; c < 8; ++c) yv[c] = yr[c];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[a][c] = fma(av[a], yv[c], acc[a][c]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        if (i0 + a >= rows) break;
        T* wr = Wn + ((c0 + i0 + a) % WR) * NMP + mm0;
#pragma unroll
        for (int c = 0; c < 8; ++c) wr[c] -= acc[a][c];
      }
    }
    __syncthreads();
    store_rows(c0, nbc);
    __syncthreads();
    if (c0 + WR < nb) load_rows(c0 + WR, min(nbc, nb - (c0 + WR)));
    __syncthreads();
  }

  // ---- backward: L^T X = Y ----
  const int last = ((nb - 1) / NB) * NB;
  for (int c0 = last; c0 >= 0; c0 -= NB) {
    const int nbc = min(NB, nb - c0);
    const int rows = min(nbc + hb, nb - c0);
    load_rows(c0, nbc);  // Y of this panel (its slots held rows >= c0 + hb)
    load_panel(AB, ld, hb, c0, nbc, rows, P, ldP);
    __syncthreads();
    // partial sums of L[c0+i][c0+t] X[c0+i][m] over i in [nbc, rows), 4 groups of i
    {
      const int tile = tid & 63, kg = tid >> 6;
      const int t0 = 4 * (tile >> 3), mm0 = 4 * (tile & 7);
      T acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = T(0);
      for (int i = nbc + kg; i < rows; i += 4) {
        T lv[4], xv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) lv[a] = (t0 + a < nbc) ? P[(t0 + a) * ldP + i] : T(0);
        const T* xr = Wn + ((c0 + i) % WR) * NMP + mm0;
#pragma unroll
        for (int c = 0; c < 4; ++c) xv[c] = xr[c];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][c] = fma(lv[a], xv[c], acc[a][c]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) Red[(kg * NB + t0 + a) * NM + mm0 + c] = acc[a][c];
    }
    __syncthreads();
    for (int idx = tid; idx < nbc * nm; idx += blockDim.x) {
      const int t = idx / nm, m = idx - t * nm;
      const T sum = Red[(0 * NB + t) * NM + m] + Red[(1 * NB + t) * NM + m] +
                    Red[(2 * NB + t) * NM + m] + Red[(3 * NB + t) * NM + m];
      Wn[((c0 + t) % WR) * NMP + m] -= sum;
    }
    __syncthreads();
    if (tid < nm) {
      for (int t = nbc - 1; t >= 0; --t) {
        T* wt = Wn + ((c0 + t) % WR) * NMP + tid;
        const T xt = *wt / P[t * ldP + t];
        *wt = xt;
        for (int i = 0; i < t; ++i) Wn[((c0 + i) % WR) * NMP + tid] -= P[i * ldP + t] * xt;
      }
    }
    __syncthreads();
    store_rows(c0, nbc);
    __syncthreads();
  }
}

}  // namespace

template <typename T>
cudaError_t launch_bandchol(const Block* blocks, int nblock, int hb_max, T* band, int32_t* status,
                            cudaStream_t s) {
  const int ldP = NB + hb_max + 1;
  const size_t smem = sizeof(T) * (size_t)NB * ldP;
  cudaError_t e = cudaFuncSetAttribute(k_bandchol<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_bandchol<T><<<nblock, kThreads, smem, s>>>(blocks, band, status, ldP);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bandsolve(const Block* blocks, int nblock, int hb_max, int N, const T* band,
                             T* rhs, cudaStream_t s) {
  const int ldP = (NB + hb_max + 1 + 3) / 4 * 4;
  const int WRmax = ((NB + hb_max + NB - 1) / NB) * NB;
  const size_t smem =
      sizeof(T) * ((size_t)NB * ldP + (size_t)WRmax * NMP + 4 * (size_t)NB * NM);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_bandsolve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid(nblock, (N + NM - 1) / NM);
  k_bandsolve<T><<<grid, kThreads, smem, s>>>(blocks, band, rhs, N, ldP, WRmax);
  return cudaGetLastError();
}

#define INST(T)                                                                                  \
  template cudaError_t launch_bandchol<T>(const Block*, int, int, T*, int32_t*, cudaStream_t);  \
  template cudaError_t launch_bandsolve<T>(const Block*, int, int, int, const T*, T*,           \
                                           cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace enkfmc
