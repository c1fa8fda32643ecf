// Step (a): ensemble anomalies (Eq. 5) and the modified Cholesky regressions
// (Section 2.1, Eq. 1-3; Section 2.3, Eq. 8 with S = U).
//
// Layout.  The anomaly kernel turns the member-major ensemble X[m][l] into a
// component-major array U[l][ldN] (ldN = N rounded up to 4, zero padded), so
// that the N samples of one component are contiguous and a warp reads them
// with one coalesced request.
//
// Regression.  One warp per row j.  The predecessor list P_j (stencil slots
// that are predecessors, optionally cut to a sub-domain's extended box) is
// compacted with a ballot.  The augmented Gram matrix [U_P; u_j][U_P; u_j]^T
// is accumulated in 4x4 register tiles over chunks of 32 members staged in
// shared memory.  G + lambda I is factored by a warp Cholesky, beta solves
// the normal equations and, in single precision, one step of iterative
// refinement corrects beta with the residual e = u_j - U_P^T beta computed in
// compensated (double-float) arithmetic: beta += (L L^T)^-1 U_P e
// (corrected semi-normal equations, Bjorck 1987).  The final residual gives
// D_j = |e|^2 / (N - 1).
#include <math.h>

#include "enkfmc_internal.h"

namespace enkfmc {

namespace {

constexpr int kChunk = 32;  // members staged per pass
constexpr int kMCP = 33;    // padded chunk stride (odd: conflict-free stores)

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ bool finite_val(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_val(double v) { return isfinite(v); }

// ---------------------------------------------------------------------------
// Anomalies: U[l][m] = X[m][l] - mean_m X[m][l]
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_anomalies(const T* __restrict__ X, T* __restrict__ U,
                                                   int64_t n, int N, int ldN) {
  __shared__ T tile[32][33];
  __shared__ T mean_s[32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t c0 = (int64_t)blockIdx.x * 32;
  const int64_t c = c0 + tx;
  T acc = 0;
  if (c < n)
    for (int m = ty; m < N; m += 8) acc += X[(int64_t)m * n + c];
  tile[ty][tx] = acc;
  __syncthreads();
  if (ty == 0) {
    T s = 0;
    for (int i = 0; i < 8; ++i) s += tile[i][tx];
    mean_s[tx] = s / T(N);
  }
  __syncthreads();
  for (int m0 = 0; m0 < ldN; m0 += 32) {
    for (int i = ty; i < 32; i += 8) {
      const int m = m0 + i;
      T v = 0;
      if (c < n && m < N) v = X[(int64_t)m * n + c] - mean_s[tx];
      tile[i][tx] = v;
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
      const int64_t cc = c0 + i;
      const int m = m0 + tx;
      if (cc < n && m < ldN) U[cc * ldN + m] = tile[tx][i];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Warp-level helpers on a dense lower-triangular matrix in shared memory.
// ---------------------------------------------------------------------------
// In-place Cholesky of G[0:p][0:p] (row stride ld).  Returns 0 on success,
// otherwise ENKFMC_EDNONPOS / ENKFMC_ENONFINITE.  Warp-uniform.
template <typename T>
__device__ int warp_cholesky(T* G, int ld, int p, int lane) {
  for (int k = 0; k < p; ++k) {
    T d = G[k * ld + k];
    if (!finite_val(d)) return ENKFMC_ENONFINITE;
    if (!(d > T(0))) return ENKFMC_EDNONPOS;
    d = sqrt(d);
    __syncwarp();
    if (lane == 0) G[k * ld + k] = d;
    const T inv = T(1) / d;
    for (int i = k + 1 + lane; i < p; i += 32) G[i * ld + k] *= inv;
    __syncwarp();
    for (int i = k + 1 + lane; i < p; i += 32) {
      const T lik = G[i * ld + k];
      T* gi = G + i * ld;
      for (int l = k + 1; l <= i; ++l) gi[l] -= lik * G[l * ld + k];
    }
    __syncwarp();
  }
  return 0;
}

// v <- (L L^T)^-1 v with L the Cholesky factor stored in G.
template <typename T>
__device__ void warp_chol_solve(const T* G, int ld, int p, T* v, int lane) {
  for (int k = 0; k < p; ++k) {
    const T wk = v[k] / G[k * ld + k];
    __syncwarp();
    if (lane == 0) v[k] = wk;
    for (int i = k + 1 + lane; i < p; i += 32) v[i] -= G[i * ld + k] * wk;
    __syncwarp();
  }
  for (int k = p - 1; k >= 0; --k) {
    const T bk = v[k] / G[k * ld + k];
    __syncwarp();
    if (lane == 0) v[k] = bk;
    for (int i = lane; i < k; i += 32) v[i] -= G[k * ld + i] * bk;
    __syncwarp();
  }
}

// Stage members [m0, m0 + 32) of rows qrow[0..nrow) into Us[i][mm].
template <typename T>
__device__ __forceinline__ void stage_chunk(const T* __restrict__ U, const int64_t* qrow, int nrow,
                                            int nrow_pad, int m0, int N, T* Us, int lane) {
  const bool live = (m0 + lane) < N;
  for (int i = 0; i < nrow_pad; ++i) {
    T v = 0;
    if (i < nrow && live) v = U[qrow[i] + m0 + lane];
    Us[i * kMCP + lane] = v;
  }
  __syncwarp();
}

// e = u - sum_i U_i beta_i for the warp's member, compensated for float.
__device__ __forceinline__ float residual_member(const float* Us, int p, const float* beta,
                                                 int lane) {
  float s = Us[p * kMCP + lane], c = 0.f;
  for (int i = 0; i < p; ++i) {
    const float a = Us[i * kMCP + lane];
    const float prod = a * beta[i];
    const float perr = fmaf(a, beta[i], -prod);
    const float t = s - prod;
    const float z = t - s;
    const float e = (s - (t - z)) + (-prod - z);
    s = t;
    c += e - perr;
  }
  return s + c;
}
__device__ __forceinline__ double residual_member(const double* Us, int p, const double* beta,
                                                  int lane) {
  double e = Us[p * kMCP + lane];
  for (int i = 0; i < p; ++i) e -= Us[i * kMCP + lane] * beta[i];
  return e;
}

// ---------------------------------------------------------------------------
// Regression kernel
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_regress(const Geom g, const T* __restrict__ U,
                                                 const int32_t* __restrict__ halo, int64_t nitems,
                                                 const Block* __restrict__ blocks,
                                                 T* __restrict__ Tout, T* __restrict__ Dout,
                                                 double ridge_c, int32_t* status, int ldp,
                                                 int warp_bytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  unsigned char* base = smem + (size_t)warp * warp_bytes;
  int64_t* qrow = reinterpret_cast<int64_t*>(base);  // [ldp]
  int* sidx = reinterpret_cast<int*>(qrow + ldp);      // [ldp]
  T* Us = reinterpret_cast<T*>(sidx + ldp);            // [ldp][kMCP]
  T* G = Us + ldp * kMCP;                              // [ldp][ldp]
  T* va = G + ldp * ldp;                               // [ldp]
  T* vb = va + ldp;                                    // [ldp]
  T* es = vb + ldp;                                    // [kMCP]
  const int N = g.N, pmax = g.pmax;
  const bool refine = sizeof(T) == 4;

  for (int64_t item = (int64_t)blockIdx.x * wpc + warp; item < nitems;
       item += (int64_t)gridDim.x * wpc) {
    int v, k, y, x;
    int64_t orow;
    const Block* b = nullptr;
    if (halo) {
      const int blk = halo[2 * item], loc = halo[2 * item + 1];
      b = blocks + blk;
      const int plane = b->ey * b->ex;
      k = loc / plane;
      const int rem = loc - k * plane;
      const int yy = rem / b->ex, xx = rem - yy * b->ex;
      y = b->lat_lo + yy;
      x = imod(b->lon_lo + xx, g.nlon);
      v = b->var;
      orow = b->row_off + loc;
    } else {
      label_coords(g, item, v, k, y, x);
      orow = item;
    }
    // predecessor list
    int p = 0;
    for (int s0 = 0; s0 < pmax; s0 += 32) {
      const int s = s0 + lane;
      bool pres = false;
      int64_t q = 0;
      if (s < pmax) {
        int kq, yq, xq;
        pres = slot_pred(g, k, y, x, s, kq, yq, xq);
        if (pres && b) {
          int yy, xx;
          pres = in_ext(*b, g.nlon, yq, xq, yy, xx);
        }
        if (pres) q = coords_label(g, v, kq, yq, xq);
      }
      const unsigned mask = __ballot_sync(0xffffffffu, pres);
      const int idx = p + __popc(mask & ((1u << lane) - 1u));
      if (s < pmax) sidx[s] = pres ? idx : -1;
      if (pres) qrow[idx] = q * g.ldN;
      p += __popc(mask);
    }
    if (lane == 0) qrow[p] = coords_label(g, v, k, y, x) * g.ldN;
    __syncwarp();
    const int p1 = p + 1;
    const int P4 = (p1 + 3) >> 2;
    int err = 0;

    if (p > 0) {
      // augmented Gram [U_P; u_j][U_P; u_j]^T, lower 4x4 tiles
      const int ntile = P4 * (P4 + 1) / 2;
      for (int m0 = 0; m0 < N; m0 += kChunk) {
        stage_chunk(U, qrow, p1, P4 * 4, m0, N, Us, lane);
        const int mmax = min(kChunk, N - m0);
        for (int bi = lane; bi < ntile; bi += 32) {
          int I = (int)((sqrtf(8.f * bi + 1.f) - 1.f) * 0.5f);
          while ((I + 1) * (I + 2) / 2 <= bi) ++I;
          while (I * (I + 1) / 2 > bi) --I;
          const int J = bi - I * (I + 1) / 2;
          T acc[4][4];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] = (m0 == 0) ? T(0) : G[(4 * I + a) * ldp + 4 * J + c];
          const T* ra = Us + (4 * I) * kMCP;
          const T* rb = Us + (4 * J) * kMCP;
          for (int mm = 0; mm < mmax; ++mm) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = ra[a * kMCP + mm];
#pragma unroll
            for (int c = 0; c < 4; ++c) bv[c] = rb[c * kMCP + mm];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int c = 0; c < 4; ++c) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) G[(4 * I + a) * ldp + 4 * J + c] = acc[a][c];
        }
        __syncwarp();
      }
      // ridge where p >= N - 1
      if (ridge_c > 0.0 && p >= N - 1) {
        T tr = 0;
        for (int i = lane; i < p; i += 32) tr += G[i * ldp + i];
        tr = warp_sum(tr);
        const T lam = T(ridge_c) * tr / T(p);
        __syncwarp();
        for (int i = lane; i < p; i += 32) G[i * ldp + i] += lam;
        __syncwarp();
      }
      // g = row p of the augmented Gram
      for (int i = lane; i < p; i += 32) va[i] = G[p * ldp + i];
      __syncwarp();
      err = warp_cholesky(G, ldp, p, lane);
      if (!err) {
        warp_chol_solve(G, ldp, p, va, lane);
        if (refine) {
          for (int i = lane; i < p; i += 32) vb[i] = 0;
          __syncwarp();
          for (int m0 = 0; m0 < N; m0 += kChunk) {
            stage_chunk(U, qrow, p1, p1, m0, N, Us, lane);
            es[lane] = (m0 + lane < N) ? residual_member(Us, p, va, lane) : T(0);
            __syncwarp();
            const int mmax = min(kChunk, N - m0);
            for (int i = lane; i < p; i += 32) {
              T a = vb[i];
              for (int mm = 0; mm < mmax; ++mm) a = fma(Us[i * kMCP + mm], es[mm], a);
              vb[i] = a;
            }
            __syncwarp();
          }
          warp_chol_solve(G, ldp, p, vb, lane);
          for (int i = lane; i < p; i += 32) va[i] += vb[i];
          __syncwarp();
        }
      }
    }
    // residual variance
    T ssq = 0;
    if (!err) {
      for (int m0 = 0; m0 < N; m0 += kChunk) {
        stage_chunk(U, qrow, p1, p1, m0, N, Us, lane);
        if (m0 + lane < N) {
          const T e = residual_member(Us, p, va, lane);
          ssq = fma(e, e, ssq);
        }
        __syncwarp();
      }
      ssq = warp_sum(ssq);
    }
    T Dj = ssq / T(N - 1);
    if (!err && !finite_val(Dj)) err = ENKFMC_ENONFINITE;
    if (!err && !(Dj > T(0))) err = ENKFMC_EDNONPOS;
    if (err && lane == 0) record_error(status, err, orow);
    T* trow = Tout + orow * pmax;
    for (int s = lane; s < pmax; s += 32) {
      const int i = sidx[s];
      trow[s] = (i >= 0 && !err) ? -va[i] : T(0);
    }
    if (lane == 0) Dout[orow] = err ? T(NAN) : Dj;
    __syncwarp();
  }
}

}  // namespace

template <typename T>
cudaError_t launch_anomalies(const Geom& g, const T* Xb, T* U, cudaStream_t s) {
  const dim3 blk(32, 8);
  const int64_t grid = (g.n + 31) / 32;
  k_anomalies<T><<<(unsigned)grid, blk, 0, s>>>(Xb, U, g.n, g.N, g.ldN);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_regress(const Geom& g, const T* U, const int32_t* halo, int64_t nitems,
                           const Block* blocks, T* Tout, T* Dout, double ridge_c,
                           int32_t* status, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  const int ldp = ((g.pmax + 1) + 3) / 4 * 4;
  size_t wb = (size_t)ldp * (sizeof(int64_t) + sizeof(int)) +
              sizeof(T) * ((size_t)ldp * kMCP + (size_t)ldp * ldp + 2 * (size_t)ldp + kMCP);
  wb = (wb + 15) / 16 * 16;
  int wpc = (int)(200 * 1024 / wb);
  if (wpc > 8) wpc = 8;
  if (wpc < 1) return cudaErrorInvalidConfiguration;
  const size_t smem = wb * wpc;
  cudaError_t e = cudaFuncSetAttribute(k_regress<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int64_t grid = (nitems + wpc - 1) / wpc;
  if (grid > 152 * 64) grid = 152 * 64;
  k_regress<T><<<(unsigned)grid, 32 * wpc, smem, s>>>(g, U, halo, nitems, blocks, Tout, Dout,
                                                      ridge_c, status, ldp, (int)wb);
  return cudaGetLastError();
}

template cudaError_t launch_anomalies<float>(const Geom&, const float*, float*, cudaStream_t);
template cudaError_t launch_anomalies<double>(const Geom&, const double*, double*, cudaStream_t);
template cudaError_t launch_regress<float>(const Geom&, const float*, const int32_t*, int64_t,
                                           const Block*, float*, float*, double, int32_t*,
                                           cudaStream_t);
template cudaError_t launch_regress<double>(const Geom&, const double*, const int32_t*, int64_t,
                                            const Block*, double*, double*, double, int32_t*,
                                            cudaStream_t);

}  // namespace enkfmc
