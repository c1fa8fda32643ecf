// Step (a): ensemble anomalies (Eq. 5) and the modified Cholesky regressions
// (Section 2.1, Eq. 1-3; Section 2.3, Eq. 8 with S = U).
//
// Layout.  The anomaly kernel turns the member-major ensemble X[m][l] into a
// component-major array U[l][ldN] (ldN = N rounded up to 4, zero padded), so
// that the N samples of one component are contiguous.
//
// Covariance table.  Every Gram entry a regression needs is the dot product
// of two components of the same variable whose offset (dk, dlat, dlon) lies in
// the box |dk| <= vr, |dlat|, |dlon| <= 2r (both lie in one local box).  The
// table C[a][h] holds U_a . U_{a+delta_h} for the half of that box with
// delta >= 0 in (dk, dlat, dlon) lexicographic order, so each pair is
// computed once for the whole grid and shared by the global rows and the
// boundary rows of every sub-domain (about 6x fewer flops than forming each
// row's Gram matrix).  One block computes a line of W components against a
// staged (lat, lon) window with 4x4 register tiles over (component, dlon).
//
// Rows.  One warp per row j: the predecessor list P_j (stencil slots that are
// predecessors, optionally cut to a sub-domain's extended box) is compacted
// with a ballot, the augmented Gram matrix [U_P; u_j][U_P; u_j]^T is gathered
// from the table and factored by a right-looking Cholesky in 4 x 4 tiles
// (tiled_cholesky) whose last row yields w = L^-1 g; then beta = L^-T w.  In
// single precision one step of iterative refinement corrects beta with the
// residual e = u_j - U_P^T beta of the anomalies themselves (FMA, single
// precision): beta += (L L^T)^-1 U_P e (corrected semi-normal equations,
// Bjorck 1987), which removes the error of the single-precision Gram entries;
// D_j = |e'|^2 / (N - 1) for the refined residual.  In double precision (and
// for the rows a single-precision problem regresses in double) D_j is formed
// from the explicit residual e = u_j - U_P^T beta.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "enkfmc_internal.h"

namespace enkfmc {

namespace {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over each group of G consecutive lanes (G = 16: each half of the warp;
// every lane of the warp takes part).
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ bool finite_val(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_val(double v) { return isfinite(v); }

// four consecutive elements from 16-byte aligned shared memory
__device__ __forceinline__ void lds4v(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void lds4v(const double* p, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void sts4v(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void sts4v(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
// four consecutive elements from 16-byte aligned global memory
__device__ __forceinline__ void ldg4v(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ldg4v(const double* p, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
// four consecutive elements to 16-byte aligned global memory
__device__ __forceinline__ void sts4g(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void sts4g(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
// ---------------------------------------------------------------------------
// Anomalies: U[l][m] = X[m][l] - mean_m X[m][l], accumulated and subtracted in
// TU; U32 (optional) receives the same anomalies rounded to single precision
// (the FP32 path with FP64 rows keeps both).
// ---------------------------------------------------------------------------
template <typename TX, typename TU>
__global__ void __launch_bounds__(256) k_anomalies(const TX* __restrict__ X, TU* __restrict__ U,
                                                   float* __restrict__ U32, int64_t n, int N,
                                                   int ldN) {
  __shared__ TU tile[32][33];
  __shared__ TU mean_s[32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t c0 = (int64_t)blockIdx.x * 32;
  const int64_t c = c0 + tx;
  TU acc = 0;
  if (c < n)
    for (int m = ty; m < N; m += 8) acc += (TU)X[(int64_t)m * n + c];
  tile[ty][tx] = acc;
  __syncthreads();
  if (ty == 0) {
    TU s = 0;
    for (int i = 0; i < 8; ++i) s += tile[i][tx];
    mean_s[tx] = s / TU(N);
  }
  __syncthreads();
  for (int m0 = 0; m0 < ldN; m0 += 32) {
    for (int i = ty; i < 32; i += 8) {
      const int m = m0 + i;
      TU v = 0;
      if (c < n && m < N) v = (TU)X[(int64_t)m * n + c] - mean_s[tx];
      tile[i][tx] = v;
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
      const int64_t cc = c0 + i;
      const int m = m0 + tx;
      if (cc < n && m < ldN) {
        U[cc * ldN + m] = tile[tx][i];
        if (U32) U32[cc * ldN + m] = (float)tile[tx][i];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Covariance table
// ---------------------------------------------------------------------------
// Offset rows of the half box: rho -> (dk, dy, first dlon).  rho 0 is
// (0, 0) with dlon in [0, 2r]; rho 1..2r are (0, dy) with dy = 1..2r; then
// vr levels of (dk, dy), dy = -2r..2r, with dlon in [-2r, 2r].
__device__ __forceinline__ void cov_row(int rho, int r, int& dk, int& dy, int& dxlo) {
  if (rho <= 2 * r) {
    dk = 0;
    dy = rho;
    dxlo = rho == 0 ? 0 : -2 * r;
    return;
  }
  const int t = rho - (2 * r + 1);
  const int w4 = 4 * r + 1;
  dk = 1 + t / w4;
  dy = t % w4 - 2 * r;
  dxlo = -2 * r;
}

// Region row (staging) of an offset row: level k rows first (dy = 0..2r), then
// the rows of the levels above (dy = -2r..2r).
template <typename T, int MC>
__global__ void __launch_bounds__(256) k_covtable(const Geom g, const T* __restrict__ U,
                                                  T* __restrict__ C, int W, int nH, int nrho) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int MCP = MC + 1;  // odd stride: cells 4 apart fall in different banks
  const int r = g.r, r2 = 2 * r, w4 = 4 * r + 1;
  const int Wp = W + 4 * r;
  const int R = nrho;  // region rows coincide with offset rows
  T* S = reinterpret_cast<T*>(smem);        // [R][Wp][MCP]
  T* Cs = S + (size_t)R * Wp * MCP;         // [W][nH]
  // plane -> (variable, level)
  int plane = blockIdx.z, v = 0;
  while (plane >= g.var_lev[v]) {
    plane -= g.var_lev[v];
    ++v;
  }
  const int k = plane, y = blockIdx.y, x0 = blockIdx.x * W;
  const int nlev_v = g.var_lev[v];
  const int tid = threadIdx.x;
  // tiles: (rho, dx tile, a tile)
  const int atiles = W / 4;
  const int dxt_full = (w4 + 3) / 4, dxt_half = (r2 + 1 + 3) / 4;
  const int ntiles = (dxt_half + (nrho - 1) * dxt_full) * atiles;
  for (int i = tid; i < W * nH; i += blockDim.x) Cs[i] = T(0);

  for (int m0 = 0; m0 < g.N; m0 += MC) {
    __syncthreads();
    // stage the window for members [m0, m0 + MC): one thread per (row, column)
    // cell, MC contiguous members copied with 16-byte vectors
    constexpr int VEC = 16 / sizeof(T);
    const bool full = m0 + MC <= g.ldN;
    for (int cell = tid; cell < R * Wp; cell += blockDim.x) {
      const int chi = cell % Wp, rho = cell / Wp;
      int dk, dy, dxlo;
      cov_row(rho, r, dk, dy, dxlo);
      const int kk = k + dk, yy = y + dy;
      int xx = x0 - r2 + chi;
      bool ok = kk < nlev_v && yy >= 0 && yy < g.nlat;
      if (ok && (xx < 0 || xx >= g.nlon)) {
        if (g.periodic) xx = imod(xx, g.nlon);
        else ok = false;
      }
      T* dst = S + (size_t)cell * MCP;
      if (ok && full) {
        const T* src = U + coords_label(g, v, kk, yy, xx) * g.ldN + m0;
#pragma unroll
        for (int q = 0; q < MC / VEC; ++q) {
          const float4 f = reinterpret_cast<const float4*>(src)[q];
          const T* e = reinterpret_cast<const T*>(&f);
#pragma unroll
          for (int u = 0; u < VEC; ++u) dst[q * VEC + u] = e[u];
        }
      } else {
        const T* src = ok ? U + coords_label(g, v, kk, yy, xx) * g.ldN : nullptr;
#pragma unroll
        for (int mm = 0; mm < MC; ++mm) dst[mm] = (ok && m0 + mm < g.N) ? src[m0 + mm] : T(0);
      }
    }
    __syncthreads();
    const int mcnt = min(MC, g.N - m0);
    for (int tile = tid; tile < ntiles; tile += blockDim.x) {
      const int at = tile % atiles;
      int rest = tile / atiles;
      int rho, dxt;
      if (rest < dxt_half) {
        rho = 0;
        dxt = rest;
      } else {
        rest -= dxt_half;
        rho = 1 + rest / dxt_full;
        dxt = rest % dxt_full;
      }
      int dk, dy, dxlo;
      cov_row(rho, r, dk, dy, dxlo);
      const int dx0 = dxlo + 4 * dxt;
      T acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
      const T* Sa = S + ((size_t)0 * Wp + (r2 + 4 * at)) * MCP;           // a cells
      const T* Sb = S + ((size_t)rho * Wp + (r2 + 4 * at + dx0)) * MCP;   // b cells
      for (int mm = 0; mm < mcnt; ++mm) {
        T av[4], bv[7];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = Sa[i * MCP + mm];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
          const int chi = r2 + 4 * at + dx0 + q;
          bv[q] = (chi >= 0 && chi < Wp) ? Sb[q * MCP + mm] : T(0);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[i + j], acc[i][j]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int dx = dx0 + j;
        if (dx > r2) continue;
        const int t = ((dk + g.vr) * w4 + (dy + r2)) * w4 + (dx + r2);
        const int h = t - ((2 * g.vr + 1) * w4 * w4 - 1) / 2;
#pragma unroll
        for (int i = 0; i < 4; ++i) Cs[(4 * at + i) * nH + h] += acc[i][j];
      }
    }
  }
  __syncthreads();
  for (int idx = tid; idx < W * nH; idx += blockDim.x) {
    const int a = idx / nH, h = idx - a * nH;
    const int x = x0 + a;
    if (x < g.nlon) C[coords_label(g, v, k, y, x) * nH + h] = Cs[idx];
  }
}

// Covariance table, member-major staging (even r): the window of a member
// chunk is stored as S[m][cell], rows of Wp4 cells padded with zeros, so a
// thread's 4 a-cells are one 16-byte read and its 7 b-cells two aligned 16-byte
// reads (the b window starts at dx = -2r or 0, a multiple of 4 from the a
// cells): 3 shared-memory reads per 16 multiply-adds, no bounds tests.  A
// thread keeps the same TPT tiles for every member chunk, their 4 x 4 sums in
// registers; the [W][nH] output is staged once, at the end, in the space of S.
template <typename T, int MC, int TPT>
__global__ void __launch_bounds__(256) k_covtable4(const Geom g, const T* __restrict__ U,
                                                   T* __restrict__ C, int W, int nH, int nrho,
                                                   int Wp4) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int r = g.r, r2 = 2 * r, w4 = 4 * r + 1;
  const int Wp = W + 4 * r;
  const int SLD = nrho * Wp4;  // cells per member (a multiple of 4)
  T* S = reinterpret_cast<T*>(smem);   // [MC][SLD]; at the end [W][nH]
  int plane = blockIdx.z, v = 0;
  while (plane >= g.var_lev[v]) {
    plane -= g.var_lev[v];
    ++v;
  }
  const int k = plane, y = blockIdx.y, x0 = blockIdx.x * W;
  const int nlev_v = g.var_lev[v];
  const int tid = threadIdx.x;
  const int atiles = W / 4;
  const int dxt_full = (w4 + 3) / 4, dxt_half = (r2 + 1 + 3) / 4;
  const int ntiles = (dxt_half + (nrho - 1) * dxt_full) * atiles;
  // this thread's tiles: a-cell group, b window offset, first output column
  int offa[TPT], offb[TPT], h0[TPT], at4[TPT], dx0s[TPT];
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int tile = min(tid + u * (int)blockDim.x, ntiles - 1);
    const int at = tile % atiles;
    int rest = tile / atiles;
    int rho, dxt;
    if (rest < dxt_half) {
      rho = 0;
      dxt = rest;
    } else {
      rest -= dxt_half;
      rho = 1 + rest / dxt_full;
      dxt = rest % dxt_full;
    }
    int dk, dy, dxlo;
    cov_row(rho, r, dk, dy, dxlo);
    const int dx0 = dxlo + 4 * dxt;
    offa[u] = r2 + 4 * at;
    offb[u] = rho * Wp4 + (r2 + 4 * at + dx0);
    const int t = ((dk + g.vr) * w4 + (dy + r2)) * w4 + (dx0 + r2);
    h0[u] = t - ((2 * g.vr + 1) * w4 * w4 - 1) / 2;  // column of dx0; dx0 + j -> h0 + j
    at4[u] = 4 * at;
    dx0s[u] = dx0;
  }
  T acc[TPT][4][4];
#pragma unroll
  for (int u = 0; u < TPT; ++u)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[u][i][j] = T(0);

  for (int m0 = 0; m0 < g.N; m0 += MC) {
    __syncthreads();
    constexpr int VEC = 16 / sizeof(T);
    const bool full = m0 + MC <= g.ldN;
    for (int cell = tid; cell < SLD; cell += blockDim.x) {
      const int rho = cell / Wp4, chi = cell - rho * Wp4;
      int dk, dy, dxlo;
      cov_row(rho, r, dk, dy, dxlo);
      const int kk = k + dk, yy = y + dy;
      int xx = x0 - r2 + chi;
      bool ok = chi < Wp && kk < nlev_v && yy >= 0 && yy < g.nlat;
      if (ok && (xx < 0 || xx >= g.nlon)) {
        if (g.periodic) xx = imod(xx, g.nlon);
        else ok = false;
      }
      if (ok && full) {
        const T* src = U + coords_label(g, v, kk, yy, xx) * g.ldN + m0;
#pragma unroll
        for (int q = 0; q < MC / VEC; ++q) {
          const float4 f = reinterpret_cast<const float4*>(src)[q];
          const T* e = reinterpret_cast<const T*>(&f);
#pragma unroll
          for (int u = 0; u < VEC; ++u) S[(size_t)(q * VEC + u) * SLD + cell] = e[u];
        }
      } else {
        const T* src = ok ? U + coords_label(g, v, kk, yy, xx) * g.ldN : nullptr;
#pragma unroll
        for (int mm = 0; mm < MC; ++mm)
          S[(size_t)mm * SLD + cell] = (ok && m0 + mm < g.N) ? src[m0 + mm] : T(0);
      }
    }
    __syncthreads();
    const int mcnt = min(MC, g.N - m0);
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      if (tid + u * (int)blockDim.x >= ntiles) break;
      const T* Sa = S + offa[u];  // row 0: the a cells
      const T* Sb = S + offb[u];  // row rho: the b cells
      for (int mm = 0; mm < mcnt; ++mm) {
        T av[4], b0[4], b1[4];
        lds4v(Sa + (size_t)mm * SLD, av);
        lds4v(Sb + (size_t)mm * SLD, b0);
        lds4v(Sb + (size_t)mm * SLD + 4, b1);
        const T bv[7] = {b0[0], b0[1], b0[2], b0[3], b1[0], b1[1], b1[2]};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[u][i][j] = fma(av[i], bv[i + j], acc[u][i][j]);
      }
    }
  }
  __syncthreads();
  T* Cs = S;  // [W][nH]; every entry is written by exactly one tile
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    if (tid + u * (int)blockDim.x >= ntiles) break;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (dx0s[u] + j > r2) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) Cs[(at4[u] + i) * nH + h0[u] + j] = acc[u][i][j];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < W * nH; idx += blockDim.x) {
    const int a = idx / nH, h = idx - a * nH;
    const int x = x0 + a;
    if (x < g.nlon) C[coords_label(g, v, k, y, x) * nH + h] = Cs[idx];
  }
}

// ---------------------------------------------------------------------------
// Row regressions
// ---------------------------------------------------------------------------
// Table entry for the pair (a, b) at geometric offset (dk, dy, dx) = b - a.
template <typename T>
__device__ __forceinline__ T cov_lookup(const T* __restrict__ C, int nH, int r, int vr, int a,
                                        int b, int dk, int dy, int dx) {
  const int w4 = 4 * r + 1;
  const int B = (2 * vr + 1) * w4 * w4;
  const int t0 = (B - 1) / 2;
  const int t = ((dk + vr) * w4 + (dy + 2 * r)) * w4 + (dx + 2 * r);
  if (t >= t0) return C[(int64_t)a * nH + (t - t0)];
  return C[(int64_t)b * nH + (B - 1 - t - t0)];
}

// sqrt(x) and 1 / sqrt(x) for a pivot x > 0.  Single precision: Newton's
// iteration for the reciprocal square root, one step from rsqrtf (a few
// instructions instead of the IEEE square root and division), IEEE below the
// normal range; double precision: IEEE.
__device__ __forceinline__ void sqrt_and_inv(float x, float& s, float& inv) {
  if (x < 1.17549435e-38f) {  // subnormal pivot
    s = sqrtf(x);
    inv = 1.f / s;
    return;
  }
  float r = rsqrtf(x);
  r = r * fmaf(-0.5f * x * r, r, 1.5f);
  inv = r;
  s = x * r;
}
__device__ __forceinline__ void sqrt_and_inv(double x, double& s, double& inv) {
  s = sqrt(x);
  inv = 1.0 / s;
}

// Element (r, c) of a warp's lower-triangular matrix (c <= r, or inside the
// diagonal 4 x 4 tile): packed 4 x 4 tiles, tile (I, J), J <= I, at
// (I (I + 1) / 2 + J) * S with S = 20 floats or 18 doubles (80 or 144 bytes:
// the tiles of 8 consecutive lanes start in distinct 16-byte bank groups, and
// a row of a tile is 16-byte aligned).  About half the shared memory of the
// row-major square: more warps per SM (four CTAs of eight warps in single
// precision at 39 slots; more warps sharing the FP64 pipes in double).
template <typename T>
struct Addr;
template <>
struct Addr<float> {
  int ld;  // unused
  __device__ __forceinline__ int operator()(int r, int c) const {
    const int I = r >> 2;
    return (I * (I + 1) / 2 + (c >> 2)) * 20 + ((r & 3) << 2) + (c & 3);
  }
};
template <>
struct Addr<double> {
  int ld;  // unused
  __device__ __forceinline__ int operator()(int r, int c) const {
    const int I = r >> 2;
    return (I * (I + 1) / 2 + (c >> 2)) * 18 + ((r & 3) << 2) + (c & 3);
  }
};
// Elements of the matrix storage for ldp rows (a multiple of 4) and row stride ldg.
__host__ __device__ inline int64_t addr_elems(size_t esize, int ldp, int ldg) {
  const int nt = ldp / 4;
  return (int64_t)nt * (nt + 1) / 2 * (esize == 4 ? 20 : 18);
}

// Right-looking Cholesky, in 4 x 4 tiles, of the leading nrows x nrows block
// of the warp's lower-triangular matrix L (addressed by at),
// rows padded with identity rows up to a multiple of 4.  Pivots are taken for
// the first npiv columns only (npiv = nrows - 1 leaves the last row as
// L^-1 times itself: the solve of an augmented system).  Step K: lane 0
// factors diagonal tile K, lanes solve the tiles (I, K) below it against it,
// then lanes update the trailing tiles (I, J), K < J <= I, with 4 x 4 register
// tiles (64 multiply-adds per 12 vector loads).  invd[u] = 1 / L[u][u] for
// u < npiv; *code (a slot not among those) carries the error code between
// lanes.  Returns 0 or ENKFMC_EDNONPOS / ENKFMC_ENONFINITE (same in every lane).
template <typename T, int G = 32>
__device__ int tiled_cholesky(T* L, const Addr<T> at, T* invd, T* code, int nrows, int npiv, int lane,
                              const uint16_t* tri = nullptr) {
  const int p1 = nrows, p = npiv;
  const int P4 = (p1 + 3) & ~3;
  for (int i = p1 + lane; i < P4; i += G) {
    for (int l = 0; l < i; ++l) L[at(i, l)] = T(0);
    L[at(i, i)] = T(1);
  }
  __syncwarp();
  const int nt = P4 >> 2;
  int err = 0;
  for (int K = 0; K < nt; ++K) {
    const int k0 = 4 * K;
    if (lane == 0) {
      T a[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r) lds4v(L + at(k0 + r, k0), a[r]);
      int e = 0;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int u = k0 + c;
        T inv = T(1);
        if (u < p) {
          const T piv = a[c][c];
          const bool fin = finite_val(piv);
          if (fin && piv > T(0)) {
            T sd;
            sqrt_and_inv(piv, sd, inv);
            a[c][c] = sd;
          } else if (!e) {
            e = fin ? ENKFMC_EDNONPOS : ENKFMC_ENONFINITE;
          }
          invd[u] = inv;
        }
#pragma unroll
        for (int r = c + 1; r < 4; ++r) a[r][c] *= inv;
#pragma unroll
        for (int r = c + 1; r < 4; ++r)
#pragma unroll
          for (int q2 = c + 1; q2 <= r; ++q2) a[r][q2] = fma(-a[r][c], a[q2][c], a[r][q2]);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) sts4v(L + at(k0 + r, k0), a[r]);
      *code = T(e);  // error code of this step (uniform read below)
    }
    __syncwarp();
    {
      const int e = (int)*code;
      if (G == 32) {  // a warp per matrix: stop at the first failure
        if (e) {
          err = e;
          break;
        }
      } else if (e && !err) {  // groups in step with each other: finish the steps
        err = e;
      }
    }
    // tiles (I, K) below: X L_KK^T = A_IK, rows of X solved left to right
    const int nrem = nt - K - 1;
    for (int tI = lane; tI < nrem; tI += G) {
      T lk[4][4], iv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        lds4v(L + at(k0 + r, k0), lk[r]);
        iv[r] = (k0 + r < p) ? invd[k0 + r] : T(1);
      }
      const int i0 = k0 + 4 * (tI + 1);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        T xr[4];
        lds4v(L + at(i0 + r, k0), xr);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          T acc = xr[c];
#pragma unroll
          for (int t = 0; t < c; ++t) acc = fma(-lk[c][t], xr[t], acc);
          xr[c] = acc * iv[c];
        }
        sts4v(L + at(i0 + r, k0), xr);
      }
    }
    __syncwarp();
    // trailing tiles (I, J), K < J <= I < nt
    const int ntile = nrem * (nrem + 1) / 2;
    for (int tix = lane; tix < ntile; tix += G) {
      int Ip, Jp;
      if (tri) {  // lower-triangle index table: tix -> (Ip, Jp)
        const uint32_t il = tri[tix];
        Ip = il & 0xff;
        Jp = il >> 8;
      } else {
        Ip = (int)((sqrtf(8.f * tix + 1.f) - 1.f) * 0.5f);
        while ((Ip + 1) * (Ip + 2) / 2 <= tix) ++Ip;
        while (Ip * (Ip + 1) / 2 > tix) --Ip;
        Jp = tix - Ip * (Ip + 1) / 2;
      }
      const int i0 = k0 + 4 * (Ip + 1), j0 = k0 + 4 * (Jp + 1);
      T li[4][4], lj[4][4], acc[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        lds4v(L + at(i0 + r, k0), li[r]);
        lds4v(L + at(j0 + r, k0), lj[r]);
        lds4v(L + at(i0 + r, j0), acc[r]);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int t = 0; t < 4; ++t) acc[r][c] = fma(-li[r][t], lj[c][t], acc[r][c]);
#pragma unroll
      for (int r = 0; r < 4; ++r) sts4v(L + at(i0 + r, j0), acc[r]);
    }
    __syncwarp();
  }

  return err;
}

// The pair table of the typical row (pair_table_entry) in shared memory,
// built by the CTA.
__device__ inline void build_pair_table(const Geom& g, int pf, int2* ptab) {
  const int np = (pf + 1) * (pf + 2) / 2;
  for (int pi = threadIdx.x; pi < np; pi += blockDim.x) ptab[pi] = pair_table_entry(g, pf, pi);
}

__host__ __device__ inline int pair_table_bytes(int pmax, int r, int periodic) {
  const int pf = pmax - (periodic ? r : 0);
  return ((pf + 1) * (pf + 2) / 2 * 8 + 15) / 16 * 16;
}

// The regressions' gather tables (gather_table_entry) in shared memory, built
// by the CTA: tri then ftab, (pmax + 1)(pmax + 2) / 2 entries each.
__device__ inline void build_gather_tables(const Geom& g, int pmax, uint16_t* tri,
                                           uint16_t* ftab) {
  const int np = (pmax + 1) * (pmax + 2) / 2;
  for (int pi = threadIdx.x; pi < np; pi += blockDim.x)
    gather_table_entry(g, pmax, pi, tri[pi], ftab[pi]);
}

__host__ __device__ inline int gather_table_bytes(int pmax) {
  return ((pmax + 1) * (pmax + 2) / 2 * 4 + 15) / 16 * 16;
}

// v := L^-1 v for the first n unknowns (L lower, stored in 4 x 4 tiles as
// tiled_cholesky leaves it, invd[u] = 1 / L[u][u]); v is 16-byte aligned with
// room for n rounded up to 4.  Per tile step lane 0 solves the 4 unknowns of
// the diagonal tile, then the lanes update the unknowns below it, one 16-byte
// read of L per row.
template <typename T, int G = 32>
__device__ void tiled_forward(const T* L, const Addr<T> at, const T* invd, T* v, int n, int lane) {
  const int nt = (n + 3) >> 2;
  for (int K = 0; K < nt; ++K) {
    const int k0 = 4 * K;
    if (lane == 0) {
      T x[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        T acc = k0 + c < n ? v[k0 + c] : T(0);
#pragma unroll
        for (int t = 0; t < c; ++t) acc = fma(-L[at(k0 + c, k0 + t)], x[t], acc);
        x[c] = k0 + c < n ? acc * invd[k0 + c] : T(0);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) v[k0 + c] = x[c];
    }
    __syncwarp();
    T x4[4];
    lds4v(v + k0, x4);
    for (int i = k0 + 4 + lane; i < n; i += G) {
      T l4[4];
      lds4v(L + at(i, k0), l4);
      T acc = v[i];
#pragma unroll
      for (int c = 0; c < 4; ++c) acc = fma(-l4[c], x4[c], acc);
      v[i] = acc;
    }
    __syncwarp();
  }
}

// v := L^-T v for the first n unknowns (same storage as tiled_forward).
template <typename T, int G = 32>
__device__ void tiled_backward(const T* L, const Addr<T> at, const T* invd, T* v, int n, int lane) {
  const int nt = (n + 3) >> 2;
  for (int K = nt - 1; K >= 0; --K) {
    const int k0 = 4 * K;
    if (lane == 0) {
      T x[4];
#pragma unroll
      for (int c = 3; c >= 0; --c) {
        T acc = k0 + c < n ? v[k0 + c] : T(0);
#pragma unroll
        for (int t = c + 1; t < 4; ++t) acc = fma(-L[at(k0 + t, k0 + c)], x[t], acc);
        x[c] = k0 + c < n ? acc * invd[k0 + c] : T(0);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) v[k0 + c] = x[c];
    }
    __syncwarp();
    T x4[4];
    lds4v(v + k0, x4);
    for (int j = lane; j < k0; j += G) {
      T acc = v[j];
#pragma unroll
      for (int c = 0; c < 4; ++c) acc = fma(-L[at(k0 + c, j)], x4[c], acc);
      v[j] = acc;
    }
    __syncwarp();
  }
}

constexpr int kMaxRounds = 4;  // N <= 128 members: 4 rounds of 32 lanes

// One warp per row of the item list (every component, or the boundary rows of
// the blocks when `halo` is given).  T: the arithmetic and the element type of
// U and C; TO: the element type of Tout and Dout.  MR: rounds of 32 members
// covering N.  sel selects rows by their predecessor count p: 0 every row,
// 1 the rows with 2p <= N, 2 the rows with 2p > N (p/N > 0.5: the rows a
// single-precision problem regresses in double precision, from FP64 U and C).
// status may be null (errors then show only as D = NaN with a zero T row).
// use_ptab = 0 leaves out the typical row's pair table (large stencils whose
// per-warp workspace would not fit beside it): every row then gathers
// through the slot-pair tables.
template <typename T, typename TO, int MR>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1)
    k_regress(const Geom g, const T* __restrict__ U, const T* __restrict__ C, int nH,
              const int32_t* __restrict__ halo, int64_t nitems, const Block* __restrict__ blocks,
              TO* __restrict__ Tout, TO* __restrict__ Dout, double ridge_c, int32_t* status,
              int ldp, int ldg, int warp_bytes, int sel, int use_ptab) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  // per-block slot offsets
  signed char* off = reinterpret_cast<signed char*>(smem);  // [3][pmax], padded to 16
  const int pmax = g.pmax;
  const int offbytes = (3 * pmax + 15) / 16 * 16;
  for (int s = threadIdx.x; s < pmax; s += blockDim.x) {
    int dk, dy, dx;
    slot_offset(s, g.r, g.vr, dk, dy, dx);
    off[s] = (signed char)dk;
    off[pmax + s] = (signed char)dy;
    off[2 * pmax + s] = (signed char)dx;
  }
  const int pf = pmax - (g.periodic ? g.r : 0);
  int2* ptab = reinterpret_cast<int2*>(smem + offbytes);
  const int ptab_bytes = use_ptab ? pair_table_bytes(pmax, g.r, g.periodic) : 0;
  if (use_ptab) build_pair_table(g, pf, ptab);
  const int nfull = (pmax + 1) * (pmax + 2) / 2;
  uint16_t* tri = reinterpret_cast<uint16_t*>(smem + offbytes + ptab_bytes);
  uint16_t* ftab = tri + nfull;
  build_gather_tables(g, pmax, tri, ftab);
  __syncthreads();
  unsigned char* base = smem + offbytes + ptab_bytes +
                        gather_table_bytes(pmax) + (size_t)warp * warp_bytes;
  int* q = reinterpret_cast<int*>(base);   // [ldp] component labels (q[p] = j)
  int* sl = q + ldp;                        // [ldp] slot of compacted entry (-1 = j)
  int* sidx = sl + ldp;                     // [ldp] compacted index of slot s
  T* L = reinterpret_cast<T*>(sidx + ldp);  // the Gram matrix, then its factor (Addr<T>)
  const Addr<T> at{ldg};
  T* va = L + addr_elems(sizeof(T), ldp, ldg);  // [ldp]
  T* vb = va + ldp;                         // [ldp]
  T* gv = vb + ldp;                         // [ldp]
  T* invd = gv + ldp;                       // [ldp]
  const int N = g.N;

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
      int qq = 0;
      if (s < pmax) {
        int kq, yq, xq;
        pres = slot_pred_off(g, k, y, x, off[s], off[pmax + s], off[2 * pmax + s], kq, yq, xq);
        if (pres && b) {
          int yy, xx;
          pres = in_ext(*b, g.nlon, yq, xq, yy, xx);
        }
        if (pres) qq = (int)coords_label(g, v, kq, yq, xq);
      }
      const unsigned mask = __ballot_sync(0xffffffffu, pres);
      const int idx = p + __popc(mask & ((1u << lane) - 1u));
      if (s < pmax) sidx[s] = pres ? idx : -1;
      if (pres) {
        q[idx] = qq;
        sl[idx] = s;
      }
      p += __popc(mask);
    }
    const int jlab = (int)coords_label(g, v, k, y, x);
    if (lane == 0) {
      q[p] = jlab;
      sl[p] = -1;
    }
    __syncwarp();
    if (sel && ((2 * p > N) != (sel == 2))) continue;  // the other launch's row
    const int p1 = p + 1;

    // gather the augmented Gram matrix, lower triangle, rows 0..p: the typical
    // row through its pair table, any other row through the slots of i and l
    const int npair = p1 * (p1 + 1) / 2;
    const bool typical = use_ptab && p == pf && (p == 0 || sl[p - 1] == pf - 1);
    if (typical) {
#pragma unroll 4
      for (int pi = lane; pi < npair; pi += 32) {
        const int2 e = ptab[pi];
        const int i = e.x & 0xff, l = (e.x >> 8) & 0xff;
        L[at(i, l)] = C[(int64_t)((e.x >> 16) ? q[l] : q[i]) * nH + e.y];
      }
    } else
#pragma unroll 4
    for (int pi = lane; pi < npair; pi += 32) {
      const uint32_t il = tri[pi];
      const int i = il & 0xff, l = il >> 8;
      // the ballot compaction keeps the slots rising with the compact index
      // and the row itself (slot pmax) is last, so sm <= si whenever l <= i:
      // (si, sm) is an entry of the lower-triangle slot-pair table
      int si = sl[i], sm = sl[l];
      si = si < 0 ? pmax : si;  // the row itself
      sm = sm < 0 ? pmax : sm;
#ifdef ENKFMC_CHECK
      if (sm > si && status) record_error(status, ENKFMC_EINVAL, orow);
#endif
      const uint32_t e = ftab[si * (si + 1) / 2 + sm];
      L[at(i, l)] = C[(int64_t)((e & 0x8000u) ? q[l] : q[i]) * nH + (e & 0x7fffu)];
    }
    __syncwarp();
    T lam = T(0);
    if (p > 0 && ridge_c > 0.0 && p >= N - 1) {
      T tr = 0;
      for (int i = lane; i < p; i += 32) tr += L[at(i, i)];
      tr = warp_sum(tr);
      lam = T(ridge_c) * tr / T(p);
    }
    for (int i = lane; i < p; i += 32) {
      gv[i] = L[at(p, i)];
      L[at(i, i)] += lam;
    }
    __syncwarp();

    // right-looking tiled Cholesky; pivots for the first p columns, so row p
    // becomes w = L^-1 g
    // (the trailing tiles of a step number at most nfull, the size of tri)
    const int err0 = tiled_cholesky(L, at, invd, invd + (ldp - 1), p1, p, lane, tri);
    int err = err0;

    T Dj = T(0);
    if (!err) {
      // beta = L^-T w  (w = row p of L), result in vb
      for (int i = lane; i < p; i += 32) va[i] = L[at(p, i)];
      __syncwarp();
      tiled_backward(L, at, invd, va, p, lane);
      for (int i = lane; i < p; i += 32) vb[i] = va[i];
      __syncwarp();
      if constexpr (sizeof(T) == 4) {
        // residual e = u - U_P^T beta, members m0 .. m0 + 3 of this lane
        // (m0 = 4 lane < ldN; U is zero past N)
        // (single precision with FMA: the correction needs the residual of the
        // data, not extra digits of it; measured on the T63 statistics against
        // the FP64 regressions, the refined beta and D match a compensated
        // residual's to within 2e-7)
        const int m0 = 4 * lane;
        const bool mv = m0 < g.ldN;
        float4 e4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (mv) e4 = *reinterpret_cast<const float4*>(U + (int64_t)jlab * g.ldN + m0);
#pragma unroll 4
        for (int i = 0; i < p; ++i) {
          const float bi = vb[i];
          if (mv) {
            const float4 u4 = *reinterpret_cast<const float4*>(U + (int64_t)q[i] * g.ldN + m0);
            e4.x = fmaf(-u4.x, bi, e4.x);
            e4.y = fmaf(-u4.y, bi, e4.y);
            e4.z = fmaf(-u4.z, bi, e4.z);
            e4.w = fmaf(-u4.w, bi, e4.w);
          }
        }
        // c = U_P e - lambda beta, the residual of (G + lambda I) beta = g -> va.
        // Full batches of 32 predecessors: each lane forms its partial dot
        // products, then a reduce-scatter (31 shuffles) leaves predecessor
        // i0 + lane's sum in lane lane; the rest one warp sum each
        auto udot = [&](int i) {
          if (!mv) return 0.f;
          const float4 u4 = *reinterpret_cast<const float4*>(U + (int64_t)q[i] * g.ldN + m0);
          return fmaf(u4.w, e4.w, fmaf(u4.z, e4.z, fmaf(u4.y, e4.y, u4.x * e4.x)));
        };
        const int pfull32 = p & ~31;
        for (int i0 = 0; i0 < pfull32; i0 += 32) {
          float part[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) part[j] = udot(i0 + j);
#pragma unroll
          for (int o = 16; o >= 1; o >>= 1) {
            const bool hi = (lane & o) != 0;
#pragma unroll
            for (int j = 0; j < o; ++j) {
              const float send = hi ? part[j] : part[j + o];
              const float keep = hi ? part[j + o] : part[j];
              part[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
          }
          const int i = i0 + lane;
          va[i] = (T)(part[0] - (float)lam * (float)vb[i]);
        }
        for (int i = pfull32; i < p; ++i) {
          const float part = warp_sum(udot(i));
          if (lane == (i & 31)) va[i] = (T)(part - (float)lam * (float)vb[i]);
        }
        __syncwarp();
        // c (the residual) is kept in gv for D below
        for (int i = lane; i < p; i += 32) gv[i] = va[i];
        // solve L z = c (forward), then L^T delta = z (backward), in va
        tiled_forward(L, at, invd, va, p, lane);
        float zz = 0.f;  // |z|^2 = delta^T (G + lambda I) delta
        for (int i = lane; i < p; i += 32) zz = fmaf((float)va[i], (float)va[i], zz);
        zz = warp_sum(zz);
        tiled_backward(L, at, invd, va, p, lane);
        // D from the refined residual e' = e - U_P^T delta without reading U:
        //   |e'|^2 = |e|^2 - 2 delta.(U_P e) + delta^T G delta,
        //   U_P e = c + lambda beta,  delta^T G delta = |z|^2 - lambda |delta|^2;
        // the corrections are small next to |e|^2
        const float ee = warp_sum(
            fmaf(e4.w, e4.w, fmaf(e4.z, e4.z, fmaf(e4.y, e4.y, e4.x * e4.x))));
        float dc = 0.f, dd = 0.f;
        for (int i = lane; i < p; i += 32) {
          const float di = (float)va[i];
          dc = fmaf(di, (float)gv[i] + (float)lam * (float)vb[i], dc);
          dd = fmaf(di, di, dd);
        }
        dc = warp_sum(dc);
        dd = warp_sum(dd);
        // beta += delta
        for (int i = lane; i < p; i += 32) vb[i] += va[i];
        const float ssq = ee - 2.f * dc + (zz - (float)lam * dd);
        Dj = (T)(ssq / (float)(N - 1));
        __syncwarp();
      } else {
        // D from the explicit residual e = u - U_P^T beta, members m = lane + 32 t
        // (the closed form u.u - beta.g - lambda beta.beta cancels when the
        // residual is small next to u)
        T ee = 0;
#pragma unroll
        for (int t = 0; t < MR; ++t) {
          const int m = lane + 32 * t;
          if (m < N) {
            T e = U[(int64_t)jlab * g.ldN + m];
            for (int i = 0; i < p; ++i) e = fma(-U[(int64_t)q[i] * g.ldN + m], vb[i], e);
            ee = fma(e, e, ee);
          }
        }
        ee = warp_sum(ee);
        Dj = ee / T(N - 1);
      }
      if (!finite_val(Dj)) err = ENKFMC_ENONFINITE;
      else if (!(Dj > T(0))) err = ENKFMC_EDNONPOS;
    }
    if (err && lane == 0 && status) record_error(status, err, orow);
    TO* trow = Tout + orow * pmax;
    for (int s = lane; s < pmax; s += 32) {
      const int i = sidx[s];
      trow[s] = (i >= 0 && !err) ? (TO)(-vb[i]) : TO(0);
    }
    if (lane == 0) Dout[orow] = err ? TO(NAN) : (TO)Dj;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Single-precision regressions, two rows per warp (16 lanes each).  The tiled
// factorisation leaves most lanes idle in its serial steps (lane 0 factors a
// 4 x 4 diagonal tile, the tile solves and the triangular solves use a few
// lanes); with a row per half-warp the same instructions serve two rows.  A
// warp takes the items 2e and 2e + 1 of the list; each half builds its row's
// predecessor list, and when the two rows have the same predecessor count p
// (the usual case: neighbouring components) the halves run in step through
// the same loops and barriers.  Otherwise the warp runs the two rows one after
// the other, both halves on the same row (the same result; the second half's
// writes repeat the first's).  Per half: the workspace of k_regress (Gram
// matrix row-major, vectors); members 4 * (lane + 16 k) .. + 3 of a row.
// Arithmetic as k_regress's single-precision rows (FP32 Cholesky, one
// corrected semi-normal step from the residual of the anomalies).
// ---------------------------------------------------------------------------
template <int MV>
__global__ void __launch_bounds__(192, 3)
    k_regress_pair(const Geom g, const float* __restrict__ U, const float* __restrict__ C, int nH,
                   const int32_t* __restrict__ halo, int64_t nitems,
                   const Block* __restrict__ blocks, float* __restrict__ Tout,
                   float* __restrict__ Dout, double ridge_c, int32_t* status, int ldp, int ldg,
                   int half_bytes, int sel, int use_ptab) {
  constexpr int G = 16;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  const int hw = lane >> 4, gl = lane & 15;
  signed char* off = reinterpret_cast<signed char*>(smem);
  const int pmax = g.pmax;
  const int offbytes = (3 * pmax + 15) / 16 * 16;
  for (int s = threadIdx.x; s < pmax; s += blockDim.x) {
    int dk, dy, dx;
    slot_offset(s, g.r, g.vr, dk, dy, dx);
    off[s] = (signed char)dk;
    off[pmax + s] = (signed char)dy;
    off[2 * pmax + s] = (signed char)dx;
  }
  const int pf = pmax - (g.periodic ? g.r : 0);
  int2* ptab = reinterpret_cast<int2*>(smem + offbytes);
  const int ptab_bytes = use_ptab ? pair_table_bytes(pmax, g.r, g.periodic) : 0;
  if (use_ptab) build_pair_table(g, pf, ptab);
  const int nfull = (pmax + 1) * (pmax + 2) / 2;
  uint16_t* tri = reinterpret_cast<uint16_t*>(smem + offbytes + ptab_bytes);
  uint16_t* ftab = tri + nfull;
  build_gather_tables(g, pmax, tri, ftab);
  __syncthreads();
  unsigned char* base = smem + offbytes + ptab_bytes + gather_table_bytes(pmax) +
                        ((size_t)warp * 2 + hw) * half_bytes;
  int* q = reinterpret_cast<int*>(base);        // [ldp] component labels (q[p] = j)
  int* sl = q + ldp;                             // [ldp] slot of compacted entry (-1 = j)
  int* sidx = sl + ldp;                          // [ldp] compacted index of slot s
  float* L = reinterpret_cast<float*>(sidx + ldp);  // [ldp][ldg]
  const Addr<float> at{ldg};
  float* va = L + addr_elems(sizeof(float), ldp, ldg);  // [ldp]
  float* vb = va + ldp;                          // [ldp]
  float* gv = vb + ldp;                          // [ldp]
  float* invd = gv + ldp;                        // [ldp]
  const int N = g.N;

  // predecessor list of item `it` in this half (sets q, sl, sidx; returns p)
  auto pred_list = [&](int64_t it, int& v, int& k, int& y, int& x, int64_t& orow, int& jlab,
                       const Block*& b) {
    b = nullptr;
    if (halo) {
      const int blk = halo[2 * it], loc = halo[2 * it + 1];
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
      label_coords(g, it, v, k, y, x);
      orow = it;
    }
    int p = 0;
    for (int s0 = 0; s0 < pmax; s0 += G) {
      const int s = s0 + gl;
      bool pres = false;
      int qq = 0;
      if (s < pmax) {
        int kq, yq, xq;
        pres = slot_pred_off(g, k, y, x, off[s], off[pmax + s], off[2 * pmax + s], kq, yq, xq);
        if (pres && b) {
          int yy, xx;
          pres = in_ext(*b, g.nlon, yq, xq, yy, xx);
        }
        if (pres) qq = (int)coords_label(g, v, kq, yq, xq);
      }
      const unsigned mask = (__ballot_sync(FULL, pres) >> (16 * hw)) & 0xffffu;
      const int idx = p + __popc(mask & ((1u << gl) - 1u));
      if (s < pmax) sidx[s] = pres ? idx : -1;
      if (pres) {
        q[idx] = qq;
        sl[idx] = s;
      }
      p += __popc(mask);
    }
    jlab = (int)coords_label(g, v, k, y, x);
    if (gl == 0) {
      q[p] = jlab;
      sl[p] = -1;
    }
    __syncwarp();
    return p;
  };

  // the regression of this half's row, its predecessor list built; p is the
  // same in both halves
  auto regress_row = [&](int p, int64_t orow, int jlab) {
    if (sel && ((2 * p > N) != (sel == 2))) return;  // the other launch's row
    const int p1 = p + 1;
    const int npair = p1 * (p1 + 1) / 2;
    const bool typical = use_ptab && p == pf && (p == 0 || sl[p - 1] == pf - 1);
    if (typical) {
#pragma unroll 4
      for (int pi = gl; pi < npair; pi += G) {
        const int2 e = ptab[pi];
        const int i = e.x & 0xff, l = (e.x >> 8) & 0xff;
        L[at(i, l)] = C[(int64_t)((e.x >> 16) ? q[l] : q[i]) * nH + e.y];
      }
    } else {
#pragma unroll 4
      for (int pi = gl; pi < npair; pi += G) {
        const uint32_t il = tri[pi];
        const int i = il & 0xff, l = il >> 8;
        // slots rise with the compact index and the row itself is last: sm <= si
        int si = sl[i], sm = sl[l];
        si = si < 0 ? pmax : si;
        sm = sm < 0 ? pmax : sm;
        const uint32_t e = ftab[si * (si + 1) / 2 + sm];
        L[at(i, l)] = C[(int64_t)((e & 0x8000u) ? q[l] : q[i]) * nH + (e & 0x7fffu)];
      }
    }
    __syncwarp();
    float lam = 0.f;
    if (p > 0 && ridge_c > 0.0 && p >= N - 1) {
      float tr = 0.f;
      for (int i = gl; i < p; i += G) tr += L[at(i, i)];
      tr = group_sum<G>(tr);
      lam = (float)ridge_c * tr / (float)p;
    }
    for (int i = gl; i < p; i += G) {
      gv[i] = L[at(p, i)];
      L[at(i, i)] += lam;
    }
    __syncwarp();
    int err = tiled_cholesky<float, G>(L, at, invd, invd + (ldp - 1), p1, p, gl, tri);
    // beta = L^-T w (w = row p of L), in vb
    for (int i = gl; i < p; i += G) va[i] = L[at(p, i)];
    __syncwarp();
    tiled_backward<float, G>(L, at, invd, va, p, gl);
    for (int i = gl; i < p; i += G) vb[i] = va[i];
    __syncwarp();
    // residual e = u - U_P^T beta, members 4 (gl + 16 k) .. + 3 of this lane
    float4 e4[MV];
#pragma unroll
    for (int k = 0; k < MV; ++k) {
      const int m0 = 4 * (gl + G * k);
      e4[k] = m0 < g.ldN ? *reinterpret_cast<const float4*>(U + (int64_t)jlab * g.ldN + m0)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll 2
    for (int i = 0; i < p; ++i) {
      const float bi = vb[i];
      const float* Ui = U + (int64_t)q[i] * g.ldN;
#pragma unroll
      for (int k = 0; k < MV; ++k) {
        const int m0 = 4 * (gl + G * k);
        if (m0 < g.ldN) {
          const float4 u4 = *reinterpret_cast<const float4*>(Ui + m0);
          e4[k].x = fmaf(-u4.x, bi, e4[k].x);
          e4[k].y = fmaf(-u4.y, bi, e4[k].y);
          e4[k].z = fmaf(-u4.z, bi, e4[k].z);
          e4[k].w = fmaf(-u4.w, bi, e4[k].w);
        }
      }
    }
    // c = U_P e - lambda beta -> va: 16 predecessors at a time by a
    // reduce-scatter over the half, the rest one group sum each
    auto udot = [&](int i) {
      const float* Ui = U + (int64_t)q[i] * g.ldN;
      float sdot = 0.f;
#pragma unroll
      for (int k = 0; k < MV; ++k) {
        const int m0 = 4 * (gl + G * k);
        if (m0 < g.ldN) {
          const float4 u4 = *reinterpret_cast<const float4*>(Ui + m0);
          sdot = fmaf(u4.w, e4[k].w, fmaf(u4.z, e4[k].z, fmaf(u4.y, e4[k].y,
                      fmaf(u4.x, e4[k].x, sdot))));
        }
      }
      return sdot;
    };
    const int pfull = p & ~(G - 1);
    for (int i0 = 0; i0 < pfull; i0 += G) {
      float part[G];
#pragma unroll
      for (int j = 0; j < G; ++j) part[j] = udot(i0 + j);
#pragma unroll
      for (int o = G / 2; o >= 1; o >>= 1) {
        const bool hi = (gl & o) != 0;
#pragma unroll
        for (int j = 0; j < o; ++j) {
          const float send = hi ? part[j] : part[j + o];
          const float keep = hi ? part[j + o] : part[j];
          part[j] = keep + __shfl_xor_sync(FULL, send, o);
        }
      }
      const int i = i0 + gl;
      va[i] = part[0] - lam * vb[i];
    }
    for (int i = pfull; i < p; ++i) {
      const float part = group_sum<G>(udot(i));
      if (gl == (i & (G - 1))) va[i] = part - lam * vb[i];
    }
    __syncwarp();
    for (int i = gl; i < p; i += G) gv[i] = va[i];
    tiled_forward<float, G>(L, at, invd, va, p, gl);
    float zz = 0.f;
    for (int i = gl; i < p; i += G) zz = fmaf(va[i], va[i], zz);
    zz = group_sum<G>(zz);
    tiled_backward<float, G>(L, at, invd, va, p, gl);
    float ee = 0.f;
#pragma unroll
    for (int k = 0; k < MV; ++k)
      ee = fmaf(e4[k].w, e4[k].w, fmaf(e4[k].z, e4[k].z, fmaf(e4[k].y, e4[k].y,
                fmaf(e4[k].x, e4[k].x, ee))));
    ee = group_sum<G>(ee);
    float dc = 0.f, dd = 0.f;
    for (int i = gl; i < p; i += G) {
      const float di = va[i];
      dc = fmaf(di, gv[i] + lam * vb[i], dc);
      dd = fmaf(di, di, dd);
    }
    dc = group_sum<G>(dc);
    dd = group_sum<G>(dd);
    for (int i = gl; i < p; i += G) vb[i] += va[i];
    const float ssq = ee - 2.f * dc + (zz - lam * dd);
    const float Dj = ssq / (float)(N - 1);
    if (!err) {
      if (!finite_val(Dj)) err = ENKFMC_ENONFINITE;
      else if (!(Dj > 0.f)) err = ENKFMC_EDNONPOS;
    }
    __syncwarp();
    if (err && gl == 0 && status) record_error(status, err, orow);
    float* trow = Tout + orow * pmax;
    for (int s = gl; s < pmax; s += G) {
      const int i = sidx[s];
      trow[s] = (i >= 0 && !err) ? -vb[i] : 0.f;
    }
    if (gl == 0) Dout[orow] = err ? NAN : Dj;
    __syncwarp();
  };

  const int64_t nent = (nitems + 1) / 2;
  for (int64_t e = (int64_t)blockIdx.x * wpc + warp; e < nent; e += (int64_t)gridDim.x * wpc) {
    const int64_t iA = 2 * e, iB = (2 * e + 1 < nitems) ? 2 * e + 1 : 2 * e;
    int v, k, y, x, jlab;
    int64_t orow;
    const Block* b;
    int p = pred_list(hw ? iB : iA, v, k, y, x, orow, jlab, b);
    const int pA = __shfl_sync(FULL, p, 0), pB = __shfl_sync(FULL, p, 16);
    if (pA == pB) {
      regress_row(p, orow, jlab);
    } else {  // one row after the other, both halves on it
      for (int pass = 0; pass < 2; ++pass) {
        p = pred_list(pass ? iB : iA, v, k, y, x, orow, jlab, b);
        regress_row(p, orow, jlab);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Single-precision regressions with the Gram matrix in registers, for stencils
// of 16 to 31 + NX predecessor slots and N <= 128 members (the rows of
// k_regress and k_adj_regress with sel 0 or 1).  One warp per row.  The
// augmented Gram matrix is padded to NP = 32 + NX rows: predecessors at
// 0..p-1, identity rows from p, the row itself last (NA = NP - 1).  Lane i
// holds row i of the leading 32 x 32 block (a[0..31], lower part); lane c
// holds column c of the last NX rows (b[r] = A[32 + r][c]).  Right-looking
// Cholesky over the leading columns: at step k every lane takes lane k's
// diagonal, scales its own entry of column k and publishes it in shared
// memory; every lane then updates its row and its column of the last rows,
// so the whole warp works at every step.  The Schur complement
// A22 - L21 L21^T of the last NX rows is factored in lanes 0..NX-1; the row
// itself ends as w = L^-1 g.  Solves with L11 sweep over its columns (a
// broadcast and one multiply-add per lane and column), from a copy of L11 in
// shared memory; the small solves with L22 run redundantly in every lane.
// The refinement step is that of k_regress (residual of the anomalies,
// corrected semi-normal equations, D from the refined residual), with four
// members per lane.
//
// Per-warp shared memory: G [NP][NP + 1] (the Gram matrix; after the
// factorisation L11 in its leading 32 x 32 block, L21^T in rows 0..31 from
// column 32, L22 in rows 32.. from column 32), and vectors col, bv, cv [NP],
// dv [8] (1 / L22 diagonal).
// ---------------------------------------------------------------------------
template <int NX>
struct Lane {
  static constexpr int NP = 32 + NX, LDG = NP + 1, NA = NP - 1;
  static constexpr int NU = NX ? 32 : 31;  // pivots of the leading block
  static constexpr int ND = NX > 1 ? NX - 1 : 1;
};

__host__ __device__ inline int lane_warp_bytes(int NX, int ints) {
  const int NP = 32 + NX, LDG = NP + 1;
  const int floats = (NP * LDG + 3) / 4 * 4 + 3 * NP + 8;
  return (((ints + 3) / 4 * 4 + floats) * 4 + 15) / 16 * 16;
}

// Column sweep of L11^T x = rhs (lane c holds x_c; L11 row t at G + t * LDG,
// inv = 1 / L_cc in lane c): unknowns 0..NU-1, the rest left as they are.
template <int NU, int LDG>
__device__ __forceinline__ float lane_backward(const float* G, float x, float inv, int lane) {
#pragma unroll
  for (int t = NU - 1; t >= 0; --t) {
    const float xt = __shfl_sync(0xffffffffu, x * inv, t);
    if (lane == t) x = xt;
    else if (lane < t) x = fmaf(-G[t * LDG + lane], xt, x);
  }
  return x;
}

// Column sweep of L11 z = c (lane i holds z_i, L11 row i at G + i * LDG).
template <int NU, int LDG>
__device__ __forceinline__ float lane_forward(const float* G, float z, float inv, int lane) {
#pragma unroll
  for (int t = 0; t < NU; ++t) {
    const float zt = __shfl_sync(0xffffffffu, z * inv, t);
    if (lane == t) z = zt;
    else if (lane > t) z = fmaf(-G[lane * LDG + t], zt, z);
  }
  return z;
}

__device__ __forceinline__ float dot4(const float4 a, const float4 b) {
  return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
}

// Members 4 m0 .. 4 m0 + 3 of a row (stride ldN, zero past N; m0 < ldN).
__device__ __forceinline__ float4 ld_members(const float* row, int m0, int N) {
  float4 u = *reinterpret_cast<const float4*>(row + m0);
  if (m0 + 4 > N) {
    if (m0 + 1 >= N) u.y = 0.f;
    if (m0 + 2 >= N) u.z = 0.f;
    if (m0 + 3 >= N) u.w = 0.f;
    if (m0 >= N) u.x = 0.f;
  }
  return u;
}

// The augmented Gram matrix of a row, lower triangle: identity rows p..NA-1,
// the row itself at NA (compact index p), gathered from the covariance table
// through the typical row's pair table or the slot-pair tables (tri, ftab).
template <int NX>
__device__ __forceinline__ void lane_gather(float* G, const int* q, const int* sl, int p,
                                            int pmax, bool typical, const int2* ptab,
                                            const uint16_t* tri, const uint16_t* ftab,
                                            const float* __restrict__ C, int nH, int lane) {
  constexpr int LDG = Lane<NX>::LDG, NA = Lane<NX>::NA;
  for (int i = p; i < NA; ++i)
    for (int l = lane; l <= i; l += 32) G[i * LDG + l] = (l == i) ? 1.f : 0.f;
  for (int l = p + lane; l < NA; l += 32) G[NA * LDG + l] = 0.f;
  const int p1 = p + 1, npair = p1 * (p1 + 1) / 2;
  if (typical) {
#pragma unroll 4
    for (int pi = lane; pi < npair; pi += 32) {
      const int2 e = ptab[pi];
      const int i = e.x & 0xff, l = (e.x >> 8) & 0xff;
      const int ii = i == p ? NA : i, ll = l == p ? NA : l;
      G[ii * LDG + ll] = C[(int64_t)((e.x >> 16) ? q[ll] : q[ii]) * nH + e.y];
    }
  } else {
#pragma unroll 4
    for (int pi = lane; pi < npair; pi += 32) {
      const uint32_t il = tri[pi];
      const int i = il & 0xff, l = il >> 8;
      const int ii = i == p ? NA : i, ll = l == p ? NA : l;
      // slots rise with the compact index and the row itself (pmax) is last,
      // so sm <= si: the entry of the lower-triangle table exists
      int si = sl[ii], sm = sl[ll];
      si = si < 0 ? pmax : si;
      sm = sm < 0 ? pmax : sm;
      const uint32_t e = ftab[si * (si + 1) / 2 + sm];
      G[ii * LDG + ll] = C[(int64_t)((e & 0x8000u) ? q[ll] : q[ii]) * nH + (e & 0x7fffu)];
    }
  }
  __syncwarp();
}

// lambda = c tr(G) / p added to the predecessors' diagonal where p >= N - 1.
template <int NX>
__device__ __forceinline__ float lane_ridge(float* G, int p, int N, double ridge_c, int lane) {
  constexpr int LDG = Lane<NX>::LDG;
  float lam = 0.f;
  if (p > 0 && ridge_c > 0.0 && p >= N - 1) {
    float tr = 0.f;
    for (int i = lane; i < p; i += 32) tr += G[i * LDG + i];
    tr = warp_sum(tr);
    lam = (float)ridge_c * tr / (float)p;
    for (int i = lane; i < p; i += 32) G[i * LDG + i] += lam;
    __syncwarp();
  }
  return lam;
}

// Cholesky of G (pivots for rows 0..NA-1), leaving the factor in G as
// described above; myinv = 1 / L_ll in lane l < NU, dv[r] = 1 / L22_rr.
// Returns 0 or ENKFMC_EDNONPOS / ENKFMC_ENONFINITE (same in every lane).
template <int NX>
__device__ __forceinline__ int lane_factor(float* G, float* col, float* dv, float& myinv,
                                           int lane) {
  constexpr int LDG = Lane<NX>::LDG, NU = Lane<NX>::NU;
  constexpr unsigned FULL = 0xffffffffu;
  float a[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) a[j] = (j <= lane) ? G[lane * LDG + j] : 0.f;
  float bx[NX > 0 ? NX : 1];
#pragma unroll
  for (int r = 0; r < NX; ++r) bx[r] = G[(32 + r) * LDG + lane];

  int err = 0;
  myinv = 1.f;
#pragma unroll
  for (int kk = 0; kk < NU; ++kk) {
    const float d = __shfl_sync(FULL, a[kk], kk);
    const bool ok = finite_val(d) && d > 0.f;
    if (!ok && !err) err = finite_val(d) ? ENKFMC_EDNONPOS : ENKFMC_ENONFINITE;
    float sd, inv;
    sqrt_and_inv(ok ? d : 1.f, sd, inv);
    const float lk = a[kk] * inv;  // lane kk: sqrt(d); lanes below: L[i][kk]
    a[kk] = lk;
    if (lane == kk) {
      myinv = inv;
#pragma unroll
      for (int r = 0; r < NX; ++r) bx[r] *= inv;
    }
    col[lane] = lk;
    if (NX > 0 && lane == kk) {
#pragma unroll
      for (int r = 0; r < NX; r += 4) {
        const float t4[4] = {bx[r], bx[r + 1], bx[r + 2], bx[r + 3]};
        sts4v(col + 32 + r, t4);
      }
    }
    __syncwarp();
#pragma unroll
    for (int j4 = (kk + 1) / 4 * 4; j4 < 32; j4 += 4) {
      float c4[4];
      lds4v(col + j4, c4);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j4 + u > kk) a[j4 + u] = fmaf(-lk, c4[u], a[j4 + u]);
    }
    if (NX > 0 && lane > kk) {
#pragma unroll
      for (int r = 0; r < NX; r += 4) {
        float c4[4];
        lds4v(col + 32 + r, c4);
#pragma unroll
        for (int u = 0; u < 4; ++u) bx[r + u] = fmaf(-c4[u], lk, bx[r + u]);
      }
    }
    __syncwarp();
  }

  if constexpr (NX > 0) {
    // L21^T beside L11 (rows 0..31, columns 32..), then the Schur complement
    // of the last rows, lower part, one entry per lane
#pragma unroll
    for (int r = 0; r < NX; ++r) G[lane * LDG + 32 + r] = bx[r];
    __syncwarp();
    constexpr int NS = NX * (NX + 1) / 2;
    for (int e = lane; e < NS; e += 32) {
      int r = 0;
      while ((r + 1) * (r + 2) / 2 <= e) ++r;
      const int s = e - r * (r + 1) / 2;
      float acc = G[(32 + r) * LDG + 32 + s];
#pragma unroll 8
      for (int c = 0; c < 32; ++c) acc = fmaf(-G[c * LDG + 32 + r], G[c * LDG + 32 + s], acc);
      G[(32 + r) * LDG + 32 + s] = acc;
    }
    __syncwarp();
    // Cholesky of the Schur complement: lane r holds its row r < NX; the
    // last row (the row itself) takes no pivot
    float sr[NX];
#pragma unroll
    for (int t = 0; t < NX; ++t)
      sr[t] = (lane < NX && t <= lane) ? G[(32 + lane) * LDG + 32 + t] : 0.f;
    float sinv = 1.f;
#pragma unroll
    for (int kk = 0; kk < NX - 1; ++kk) {
      const float d = __shfl_sync(FULL, sr[kk], kk);
      const bool ok = finite_val(d) && d > 0.f;
      if (!ok && !err) err = finite_val(d) ? ENKFMC_EDNONPOS : ENKFMC_ENONFINITE;
      float sd, inv;
      sqrt_and_inv(ok ? d : 1.f, sd, inv);
      const float lk = sr[kk] * inv;
      sr[kk] = lk;
      if (lane == kk) sinv = inv;
#pragma unroll
      for (int j = kk + 1; j < NX; ++j) sr[j] = fmaf(-lk, __shfl_sync(FULL, lk, j), sr[j]);
    }
    if (lane < NX) {
#pragma unroll
      for (int t = 0; t < NX; ++t)
        if (t <= lane) G[(32 + lane) * LDG + 32 + t] = sr[t];
      dv[lane] = sinv;
    }
  }
  // L11 (lower part of the registers) to shared memory for the sweeps
#pragma unroll
  for (int j = 0; j < 32; ++j) G[lane * LDG + j] = a[j];
  __syncwarp();
  return err;
}

// x = (L L^T)^-1 c for the predecessor unknowns (c in cv, zero at padded
// positions): x_l in lane l < NU, the last unknowns in d2 (every lane);
// zz = |L^-1 c|^2.
template <int NX>
__device__ __forceinline__ float lane_solve(const float* G, const float* cv, const float* dv,
                                            float myinv, int lane,
                                            float (&d2)[Lane<NX>::ND], float& zz) {
  constexpr int LDG = Lane<NX>::LDG, NU = Lane<NX>::NU;
  float z = lane < NU ? cv[lane] : 0.f;
  z = lane_forward<NU, LDG>(G, z, myinv, lane);
  zz = lane < NU ? z * z : 0.f;
  if constexpr (NX > 0) {
    // z2 = L22^-1 (c2 - L21 z1), every lane
    float z2[NX - 1];
#pragma unroll
    for (int r = 0; r < NX - 1; ++r) z2[r] = warp_sum(G[lane * LDG + 32 + r] * z);
#pragma unroll
    for (int r = 0; r < NX - 1; ++r) {
      float acc = cv[32 + r] - z2[r];
#pragma unroll
      for (int j = 0; j < r; ++j) acc = fmaf(-G[(32 + r) * LDG + 32 + j], z2[j], acc);
      z2[r] = acc * dv[r];
    }
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < NX - 1; ++r) zz = fmaf(z2[r], z2[r], zz);
    }
    // x2 = L22^-T z2, then z1 - L21^T x2 for the leading sweep
#pragma unroll
    for (int t = NX - 2; t >= 0; --t) {
      float acc = z2[t];
#pragma unroll
      for (int j = t + 1; j < NX - 1; ++j) acc = fmaf(-G[(32 + j) * LDG + 32 + t], d2[j], acc);
      d2[t] = acc * dv[t];
    }
#pragma unroll
    for (int r = 0; r < NX - 1; ++r) z = fmaf(-G[lane * LDG + 32 + r], d2[r], z);
  }
  zz = warp_sum(zz);
  return lane_backward<NU, LDG>(G, z, myinv, lane);
}

// c_i = <U_qi, e> * s - t * w_i for the p predecessors (c into cv, zero at the
// padded positions up to NA): 32 predecessors at a time by a reduce-scatter
// (31 shuffles leave predecessor i0 + lane's sum in lane lane), the rest one
// warp sum each.  dot(i) gives the lane's partial product of predecessor i.
template <int NX, typename Dot>
__device__ __forceinline__ void lane_reduce_to(float* cv, int p, const float* w, float s, float t,
                                               int lane, Dot dot) {
  constexpr unsigned FULL = 0xffffffffu;
  const int pfull32 = p & ~31;
  for (int i0 = 0; i0 < pfull32; i0 += 32) {
    float part[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) part[j] = dot(i0 + j);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      const bool hi = (lane & o) != 0;
#pragma unroll
      for (int j = 0; j < o; ++j) {
        const float send = hi ? part[j] : part[j + o];
        const float keep = hi ? part[j + o] : part[j];
        part[j] = keep + __shfl_xor_sync(FULL, send, o);
      }
    }
    cv[i0 + lane] = part[0] * s - t * w[i0 + lane];
  }
  for (int i = pfull32; i < p; ++i) {
    const float part = warp_sum(dot(i));
    if (lane == (i & 31)) cv[i] = part * s - t * w[i];
  }
  for (int i = p + lane; i < Lane<NX>::NA; i += 32) cv[i] = 0.f;
  __syncwarp();
}

template <int NX>
__global__ void __launch_bounds__(256, 2)
    k_regress_lane(const Geom g, const float* __restrict__ U, const float* __restrict__ C,
                   int nH, const int32_t* __restrict__ halo, int64_t nitems,
                   const Block* __restrict__ blocks, float* __restrict__ Tout,
                   float* __restrict__ Dout, double ridge_c, int32_t* status, int warp_bytes,
                   int sel, int use_ptab) {
  using S = Lane<NX>;
  constexpr int NP = S::NP, LDG = S::LDG, NA = S::NA, NU = S::NU;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  signed char* off = reinterpret_cast<signed char*>(smem);  // [3][pmax], padded to 16
  const int pmax = g.pmax;
  const int offbytes = (3 * pmax + 15) / 16 * 16;
  for (int s = threadIdx.x; s < pmax; s += blockDim.x) {
    int dk, dy, dx;
    slot_offset(s, g.r, g.vr, dk, dy, dx);
    off[s] = (signed char)dk;
    off[pmax + s] = (signed char)dy;
    off[2 * pmax + s] = (signed char)dx;
  }
  const int pf = pmax - (g.periodic ? g.r : 0);
  int2* ptab = reinterpret_cast<int2*>(smem + offbytes);
  const int ptab_bytes = use_ptab ? pair_table_bytes(pmax, g.r, g.periodic) : 0;
  if (use_ptab) build_pair_table(g, pf, ptab);
  const int nfull = (pmax + 1) * (pmax + 2) / 2;
  uint16_t* tri = reinterpret_cast<uint16_t*>(smem + offbytes + ptab_bytes);
  uint16_t* ftab = tri + nfull;
  build_gather_tables(g, pmax, tri, ftab);
  __syncthreads();
  unsigned char* base = smem + offbytes + ptab_bytes + gather_table_bytes(pmax) +
                        (size_t)warp * warp_bytes;
  int* q = reinterpret_cast<int*>(base);   // [NP] component labels (q[NA] = j)
  int* sl = q + NP;                         // [NP] slot of a compacted entry (-1 = j)
  int* sidx = sl + NP;                      // [pmax] compacted index of slot s
  float* G = reinterpret_cast<float*>(sidx + (pmax + 3) / 4 * 4);  // [NP][LDG]
  float* col = G + (NP * LDG + 3) / 4 * 4;  // [NP] the column of a step
  float* bv = col + NP;                     // [NP] beta
  float* cv = bv + NP;                      // [NP] residual of the normal equations
  float* dv = cv + NP;                      // [8] 1 / L22 diagonal
  const int N = g.N;
  const int m0 = 4 * lane;                  // lane's members m0 .. m0 + 3
  const bool mv = m0 < g.ldN;

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
    // predecessor list (as k_regress)
    int p = 0;
    for (int s0 = 0; s0 < pmax; s0 += 32) {
      const int s = s0 + lane;
      bool pres = false;
      int qq = 0;
      if (s < pmax) {
        int kq, yq, xq;
        pres = slot_pred_off(g, k, y, x, off[s], off[pmax + s], off[2 * pmax + s], kq, yq, xq);
        if (pres && b) {
          int yy, xx;
          pres = in_ext(*b, g.nlon, yq, xq, yy, xx);
        }
        if (pres) qq = (int)coords_label(g, v, kq, yq, xq);
      }
      const unsigned mask = __ballot_sync(FULL, pres);
      const int idx = p + __popc(mask & ((1u << lane) - 1u));
      if (s < pmax) sidx[s] = pres ? idx : -1;
      if (pres) {
        q[idx] = qq;
        sl[idx] = s;
      }
      p += __popc(mask);
    }
    const int jlab = (int)coords_label(g, v, k, y, x);
    if (lane == 0) {
      q[NA] = jlab;
      sl[NA] = -1;
    }
    __syncwarp();
    if (sel && ((2 * p > N) != (sel == 2))) continue;  // the other launch's row

    const bool typical = use_ptab && p == pf && (p == 0 || sl[p - 1] == pf - 1);
    lane_gather<NX>(G, q, sl, p, pmax, typical, ptab, tri, ftab, C, nH, lane);
    const float lam = lane_ridge<NX>(G, p, N, ridge_c, lane);
    float myinv;
    int err = lane_factor<NX>(G, col, dv, myinv, lane);

    // beta = L^-T w
    float d2[S::ND];
    float xb;
    if constexpr (NX > 0) {
      // last unknowns: L22^T beta2 = w2 (w2 = row NA of the Schur factor)
#pragma unroll
      for (int t = NX - 2; t >= 0; --t) {
        float acc = G[NA * LDG + 32 + t];
#pragma unroll
        for (int j = t + 1; j < NX - 1; ++j) acc = fmaf(-G[(32 + j) * LDG + 32 + t], d2[j], acc);
        d2[t] = acc * dv[t];
      }
      // leading unknowns: L11^T beta1 = w1 - L21^T beta2 (w1 in L21^T's last column)
      xb = G[lane * LDG + 32 + NX - 1];
#pragma unroll
      for (int r = 0; r < NX - 1; ++r) xb = fmaf(-G[lane * LDG + 32 + r], d2[r], xb);
    } else {
      xb = lane < NU ? G[NA * LDG + lane] : 0.f;  // w = row NA of L11
    }
    xb = lane_backward<NU, LDG>(G, xb, myinv, lane);
    if (lane < NU) bv[lane] = xb;
    if constexpr (NX > 0) {
      if (lane == 0) {
#pragma unroll
        for (int r = 0; r < NX - 1; ++r) bv[32 + r] = d2[r];
      }
    }
    __syncwarp();

    // refinement: residual e = u - U_P^T beta of the anomalies
    float4 e4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (mv) e4 = *reinterpret_cast<const float4*>(U + (int64_t)jlab * g.ldN + m0);
#pragma unroll 4
    for (int i = 0; i < p; ++i) {
      const float bi = bv[i];
      if (mv) {
        const float4 u4 = *reinterpret_cast<const float4*>(U + (int64_t)q[i] * g.ldN + m0);
        e4.x = fmaf(-u4.x, bi, e4.x);
        e4.y = fmaf(-u4.y, bi, e4.y);
        e4.z = fmaf(-u4.z, bi, e4.z);
        e4.w = fmaf(-u4.w, bi, e4.w);
      }
    }
    // c = U_P e - lambda beta, then delta = (L L^T)^-1 c
    lane_reduce_to<NX>(cv, p, bv, 1.f, lam, lane, [&](int i) {
      float4 u4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (mv) u4 = *reinterpret_cast<const float4*>(U + (int64_t)q[i] * g.ldN + m0);
      return dot4(u4, e4);
    });
    float zz;
    const float z = lane_solve<NX>(G, cv, dv, myinv, lane, d2, zz);
    // D from the refined residual e' = e - U_P^T delta without reading U:
    //   |e'|^2 = |e|^2 - 2 delta.(U_P e) + delta^T G delta,
    //   U_P e = c + lambda beta,  delta^T G delta = |z|^2 - lambda |delta|^2
    float dc = 0.f, dd = 0.f;
    if (lane < NU) {
      dc = z * (cv[lane] + lam * bv[lane]);
      dd = z * z;
    }
    if constexpr (NX > 0) {
      if (lane == 0) {
#pragma unroll
        for (int r = 0; r < NX - 1; ++r) {
          dc = fmaf(d2[r], cv[32 + r] + lam * bv[32 + r], dc);
          dd = fmaf(d2[r], d2[r], dd);
        }
      }
    }
    const float ee = warp_sum(dot4(e4, e4));
    dc = warp_sum(dc);
    dd = warp_sum(dd);
    __syncwarp();
    if (lane < NU) bv[lane] += z;
    if constexpr (NX > 0) {
      if (lane == 0) {
#pragma unroll
        for (int r = 0; r < NX - 1; ++r) bv[32 + r] += d2[r];
      }
    }
    const float ssq = ee - 2.f * dc + (zz - lam * dd);
    const float Dj = ssq / (float)(N - 1);
    if (!err) {
      if (!finite_val(Dj)) err = ENKFMC_ENONFINITE;
      else if (!(Dj > 0.f)) err = ENKFMC_EDNONPOS;
    }
    __syncwarp();
    if (err && lane == 0 && status) record_error(status, err, orow);
    float* trow = Tout + orow * pmax;
    for (int s = lane; s < pmax; s += 32) {
      const int i = sidx[s];
      trow[s] = (i >= 0 && !err) ? -bv[i] : 0.f;
    }
    if (lane == 0) Dout[orow] = err ? NAN : Dj;
    __syncwarp();
  }
}

// The adjoint of the regressions (as k_adj_regress, whose comment gives the
// formulas) with the register factorisation of the rows above: one warp per
// extended row of one block; the pair and gather tables from global memory.
template <int NX>
__global__ void __launch_bounds__(256, 2) k_adj_regress_lane(
    const Geom g, const Block* __restrict__ blocks, const float* __restrict__ U,
    const float* __restrict__ C, int nH, const float* __restrict__ Tg,
    const float* __restrict__ Dg, const float* __restrict__ Te, const float* __restrict__ De,
    const float* __restrict__ aT, const float* __restrict__ bT, const float* __restrict__ dxT,
    const float* __restrict__ lamT, const int2* __restrict__ ptab,
    const uint16_t* __restrict__ gtab, float* __restrict__ Eo, float* __restrict__ Fo,
    float* __restrict__ Vo, float* __restrict__ Ko, double ridge_c, int32_t* status,
    int warp_bytes, int sel) {
  using S = Lane<NX>;
  constexpr int NP = S::NP, LDG = S::LDG, NA = S::NA, NU = S::NU;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  signed char* off = reinterpret_cast<signed char*>(smem);
  const int pmax = g.pmax;
  const int offbytes = (3 * pmax + 15) / 16 * 16;
  for (int s = threadIdx.x; s < pmax; s += blockDim.x) {
    int dk, dy, dx;
    slot_offset(s, g.r, g.vr, dk, dy, dx);
    off[s] = (signed char)dk;
    off[pmax + s] = (signed char)dy;
    off[2 * pmax + s] = (signed char)dx;
  }
  __syncthreads();
  unsigned char* base = smem + offbytes + (size_t)warp * warp_bytes;
  int* q = reinterpret_cast<int*>(base);  // [NP] labels (q[NA] = j)
  int* sl = q + NP;                        // [NP] slots
  int* qr = sl + NP;                       // [NP] extended rows (block-relative)
  float* G = reinterpret_cast<float*>(qr + NP);  // [NP][LDG]
  float* col = G + (NP * LDG + 3) / 4 * 4;
  float* bv = col + NP;                    // [NP] beta
  float* cv = bv + NP;                     // [NP] betabar, then v
  float* dv = cv + NP;                     // [8]
  const int N = g.N, ldN = g.ldN;
  const Block b = blocks[blockIdx.y];
  const int loc = blockIdx.x * wpc + warp;
  if (loc >= b.nb) return;
  const int plane = b.ey * b.ex;
  const int k = loc / plane;
  const int yy0 = (loc - k * plane) / b.ex, xx0 = loc - k * plane - yy0 * b.ex;
  const int y = b.lat_lo + yy0, x = imod(b.lon_lo + xx0, g.nlon);
  const int v = b.var;
  const int64_t rowj = b.row_off + loc;
  // predecessors inside the extended box
  int p = 0;
  for (int s0 = 0; s0 < pmax; s0 += 32) {
    const int s = s0 + lane;
    bool pres = false;
    int qq = 0, rr = 0;
    if (s < pmax) {
      int kq, yq, xq, yyq, xxq;
      pres = slot_pred_off(g, k, y, x, off[s], off[pmax + s], off[2 * pmax + s], kq, yq, xq) &&
             in_ext(b, g.nlon, yq, xq, yyq, xxq);
      if (pres) {
        qq = (int)coords_label(g, v, kq, yq, xq);
        rr = (kq * b.ey + yyq) * b.ex + xxq;
      }
    }
    const unsigned mask = __ballot_sync(FULL, pres);
    const int idx = p + __popc(mask & ((1u << lane) - 1u));
    if (pres) {
      q[idx] = qq;
      sl[idx] = s;
      qr[idx] = rr;
    }
    p += __popc(mask);
  }
  const int jlab = (int)coords_label(g, v, k, y, x);
  if (lane == 0) {
    q[NA] = jlab;
    sl[NA] = -1;
  }
  __syncwarp();
  if (sel && ((2 * p > N) != (sel == 2))) return;  // the other launch's row
  // beta and D of this instance
  const bool inner = in_interior(b, y, x);
  const float* trow = inner ? Tg + (int64_t)jlab * pmax : Te + rowj * pmax;
  const float Dj = inner ? Dg[jlab] : De[rowj];
  for (int i = lane; i < p; i += 32) bv[i] = -trow[sl[i]];
  __syncwarp();
  const int m0 = 4 * lane;  // lane's members m0 .. m0 + 3 (zero past N)
  const bool mv = m0 < ldN;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 e4 = z4, aj = z4, bj = z4;
  if (mv) {
    e4 = ld_members(U + (int64_t)jlab * ldN, m0, N);
    aj = ld_members(aT + rowj * ldN, m0, N);
    bj = ld_members(bT + rowj * ldN, m0, N);
  }
  // e = u - U_P^T beta
  for (int i = 0; i < p; ++i) {
    const float bi = bv[i];
    if (mv) {
      const float4 u4 = ld_members(U + (int64_t)q[i] * ldN, m0, N);
      e4.x = fmaf(-u4.x, bi, e4.x);
      e4.y = fmaf(-u4.y, bi, e4.y);
      e4.z = fmaf(-u4.z, bi, e4.z);
      e4.w = fmaf(-u4.w, bi, e4.w);
    }
  }
  const float ab = warp_sum(dot4(aj, bj));
  const float Dbar = ab / (Dj * Dj);
  const float ebs = 2.f * Dbar / (float)(N - 1);
  // Gram matrix and ridge
  const int pf = pmax - (g.periodic ? g.r : 0);
  const bool typical = p == pf && (p == 0 || sl[p - 1] == pf - 1);
  const int nfull = (pmax + 1) * (pmax + 2) / 2;
  lane_gather<NX>(G, q, sl, p, pmax, typical, ptab, gtab, gtab + nfull, C, nH, lane);
  const float lam = lane_ridge<NX>(G, p, N, ridge_c, lane);
  // betabar_i = (<a_j, dX_qi> + <b_j, Lambda_qi>) / D_j - 2 Dbar lambda beta_i / (N - 1)
  // (<U_qi, ebar> by the normal equations U_P e = lambda beta)
  lane_reduce_to<NX>(cv, p, bv, 1.f / Dj, 2.f * Dbar * lam / (float)(N - 1), lane, [&](int i) {
    if (!mv) return 0.f;
    const int64_t r = (b.row_off + qr[i]) * ldN;
    return dot4(aj, ld_members(dxT + r, m0, N)) + dot4(bj, ld_members(lamT + r, m0, N));
  });
  float myinv;
  const int err = lane_factor<NX>(G, col, dv, myinv, lane);
  float4 f4 = make_float4(ebs * e4.x, ebs * e4.y, ebs * e4.z, ebs * e4.w);
  float kappa = 0.f;
  if (err) {
    if (lane == 0) record_error(status, err, rowj);
    e4 = z4;
    f4 = z4;
    p = 0;  // defined (zero) terms for the failed row
  } else {
    // v = (G + lambda I)^-1 betabar into cv
    float d2[S::ND], zz;
    const float vl = lane_solve<NX>(G, cv, dv, myinv, lane, d2, zz);
    if (lane < NU) cv[lane] = vl;
    if constexpr (NX > 0) {
      if (lane == 0) {
#pragma unroll
        for (int r = 0; r < NX - 1; ++r) cv[32 + r] = d2[r];
      }
    }
    __syncwarp();
    float vbeta = 0.f;
    for (int i = lane; i < p; i += 32) vbeta = fmaf(cv[i], bv[i], vbeta);
    vbeta = warp_sum(vbeta);
    if (lam > 0.f) kappa = 2.f * (float)ridge_c / (float)p * vbeta;
    // f = ebar + U_P^T v
    for (int i = 0; i < p; ++i) {
      const float vi = cv[i];
      if (mv) {
        const float4 u4 = ld_members(U + (int64_t)q[i] * ldN, m0, N);
        f4.x = fmaf(u4.x, vi, f4.x);
        f4.y = fmaf(u4.y, vi, f4.y);
        f4.z = fmaf(u4.z, vi, f4.z);
        f4.w = fmaf(u4.w, vi, f4.w);
      }
    }
  }
  // this row's outputs: e, f (members m0 .. m0 + 3), v in its slots, kappa
  if (mv) {
    *reinterpret_cast<float4*>(Eo + rowj * ldN + m0) = e4;
    *reinterpret_cast<float4*>(Fo + rowj * ldN + m0) = f4;
  }
  float* vrow = Vo + rowj * pmax;
  for (int s = lane; s < pmax; s += 32) vrow[s] = 0.f;
  __syncwarp();
  for (int i = lane; i < p; i += 32) vrow[sl[i]] = cv[i];
  if (lane == 0) Ko[rowj] = kappa;
}

// ---------------------------------------------------------------------------
// Adjoint of the regressions of one (sub-domain, variable) block.  One warp
// per extended row j (a regression instance of Algorithm 3): with
// a_j = (T Lambda)_j, b_j = (T dX)_j (row-major, N samples),
//   betabar_i = (<a_j, dX_qi> + <b_j, Lambda_qi>) / D_j - <U_qi, ebar>,
//   Dbar_j = <a_j, b_j> / D_j^2, ebar = 2 Dbar e / (N - 1),
//   v = (G + lambda I)^-1 betabar (factor recomputed from the covariance table),
//   f = ebar + U_P^T v,  Ubar_qi += v_i e - beta_i f - kappa U_qi,  Ubar_j += f,
// kappa = 2 (c / p) v.beta when the ridge is active.  Rows share predecessors,
// so the row does not add into Ubar itself: it stores e and f (Eo, Fo
// [ext row][ldN]), v in its slots (Vo [ext row][pmax]) and kappa (Ko), and
// k_adj_gather sums each component's terms in a fixed order (deterministic).
// ---------------------------------------------------------------------------
// T: the arithmetic and the element type of U and C (FP64 for the rows a
// single-precision problem regressed in double precision); TS: the element
// type of T, D, the adjoint rows and the stored terms.  sel as in k_regress.
template <typename T, typename TS>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1) k_adj_regress(
    const Geom g, const Block* __restrict__ blocks, const T* __restrict__ U,
    const T* __restrict__ C, int nH, const TS* __restrict__ Tg, const TS* __restrict__ Dg,
    const TS* __restrict__ Te, const TS* __restrict__ De, const TS* __restrict__ aT,
    const TS* __restrict__ bT, const TS* __restrict__ dxT, const TS* __restrict__ lamT,
    const int2* __restrict__ ptab, const uint16_t* __restrict__ gtab, TS* __restrict__ Eo,
    TS* __restrict__ Fo, TS* __restrict__ Vo, TS* __restrict__ Ko, double ridge_c,
    int32_t* status, int ldp, int ldg, int warp_bytes, int sel) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  signed char* off = reinterpret_cast<signed char*>(smem);
  const int pmax = g.pmax;
  const int offbytes = (3 * pmax + 15) / 16 * 16;
  for (int s = threadIdx.x; s < pmax; s += blockDim.x) {
    int dk, dy, dx;
    slot_offset(s, g.r, g.vr, dk, dy, dx);
    off[s] = (signed char)dk;
    off[pmax + s] = (signed char)dy;
    off[2 * pmax + s] = (signed char)dx;
  }
  __syncthreads();
  unsigned char* base = smem + offbytes + (size_t)warp * warp_bytes;
  int* q = reinterpret_cast<int*>(base);    // [ldp] labels (q[p] = j)
  int* sl = q + ldp;                         // [ldp] slots
  int* qr = sl + ldp;                        // [ldp] extended rows (block-relative)
  T* L = reinterpret_cast<T*>(qr + ldp);     // the Gram matrix, then its factor (Addr<T>)
  const Addr<T> at{ldg};
  T* va = L + addr_elems(sizeof(T), ldp, ldg);  // [ldp] betabar -> v
  T* vb = va + ldp;                          // [ldp] beta
  T* invd = vb + ldp;                        // [ldp]
  const int N = g.N, ldN = g.ldN;
  const Block b = blocks[blockIdx.y];
  const int loc = blockIdx.x * wpc + warp;
  if (loc >= b.nb) return;
  const int plane = b.ey * b.ex;
  const int k = loc / plane;
  const int yy0 = (loc - k * plane) / b.ex, xx0 = loc - k * plane - yy0 * b.ex;
  const int y = b.lat_lo + yy0, x = imod(b.lon_lo + xx0, g.nlon);
  const int v = b.var;
  const int64_t rowj = b.row_off + loc;
  // predecessors inside the extended box
  int p = 0;
  for (int s0 = 0; s0 < pmax; s0 += 32) {
    const int s = s0 + lane;
    bool pres = false;
    int qq = 0, rr = 0;
    if (s < pmax) {
      int kq, yq, xq, yyq, xxq;
      pres = slot_pred_off(g, k, y, x, off[s], off[pmax + s], off[2 * pmax + s], kq, yq, xq) &&
             in_ext(b, g.nlon, yq, xq, yyq, xxq);
      if (pres) {
        qq = (int)coords_label(g, v, kq, yq, xq);
        rr = (kq * b.ey + yyq) * b.ex + xxq;
      }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, pres);
    const int idx = p + __popc(mask & ((1u << lane) - 1u));
    if (pres) {
      q[idx] = qq;
      sl[idx] = s;
      qr[idx] = rr;
    }
    p += __popc(mask);
  }
  const int jlab = (int)coords_label(g, v, k, y, x);
  if (lane == 0) {
    q[p] = jlab;
    sl[p] = -1;
  }
  __syncwarp();
  if (sel && ((2 * p > N) != (sel == 2))) return;  // the other launch's row
  // beta and D of this instance
  const bool inner = in_interior(b, y, x);
  const TS* trow = inner ? Tg + (int64_t)jlab * pmax : Te + rowj * pmax;
  const T Dj = (T)(inner ? Dg[jlab] : De[rowj]);
  for (int i = lane; i < p; i += 32) vb[i] = -(T)trow[sl[i]];
  __syncwarp();
  // members 4 lane .. 4 lane + 3 of this lane (N <= 128): vector loads, and
  // one vector atomic per predecessor for U-bar
  const int m0 = 4 * lane;
  auto ld4 = [&](const auto* row, T (&o)[4]) {
    if (m0 < ldN) {
      using E = typename std::remove_cv<typename std::remove_pointer<decltype(row)>::type>::type;
      E r4[4];
      ldg4v(row + m0, r4);
#pragma unroll
      for (int a = 0; a < 4; ++a) o[a] = (m0 + a < N) ? (T)r4[a] : T(0);
    } else {
#pragma unroll
      for (int a = 0; a < 4; ++a) o[a] = T(0);
    }
  };
  // this row's outputs: e, f (members 4 lane .. 4 lane + 3), v in its slots, kappa
  auto store = [&](const T (&e4)[4], const T (&f4)[4], int np, T kap) {
    if (m0 < ldN) {
      TS a4[4], c4[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        a4[a] = (TS)e4[a];
        c4[a] = (TS)f4[a];
      }
      sts4g(Eo + rowj * ldN + m0, a4);
      sts4g(Fo + rowj * ldN + m0, c4);
    }
    TS* vrow = Vo + rowj * pmax;
    for (int s = lane; s < pmax; s += 32) vrow[s] = TS(0);
    __syncwarp();
    for (int i = lane; i < np; i += 32) vrow[sl[i]] = (TS)va[i];
    if (lane == 0) Ko[rowj] = (TS)kap;
  };
  // e = u - U_P^T beta; a_j, b_j in registers
  T e[4], aj[4], bj[4];
  ld4(U + (int64_t)jlab * ldN, e);
  ld4(aT + rowj * ldN, aj);
  ld4(bT + rowj * ldN, bj);
  for (int i = 0; i < p; ++i) {
    const T bi = vb[i];
    T u4[4];
    ld4(U + (int64_t)q[i] * ldN, u4);
#pragma unroll
    for (int a = 0; a < 4; ++a) e[a] = fma(-u4[a], bi, e[a]);
  }
  T ab = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a) ab = fma(aj[a], bj[a], ab);
  ab = warp_sum(ab);
  const T Dbar = ab / (Dj * Dj);
  const T ebs = T(2) * Dbar / T(N - 1);
  T eb[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) eb[a] = ebs * e[a];
  // Gram matrix from the covariance table (as in the forward pass) and the ridge
  T lam = 0;
  if (p > 0) {
    const int npair = p * (p + 1) / 2;
    const int pf = pmax - (g.periodic ? g.r : 0);
    if (ptab && p == pf && sl[p - 1] == pf - 1) {
      // typical row: the handle's pair table (global memory, cached)
      for (int pi = lane; pi < npair; pi += 32) {
        const int2 e = ptab[pi];
        const int i = e.x & 0xff, l = (e.x >> 8) & 0xff;
        L[at(i, l)] = C[(int64_t)((e.x >> 16) ? q[l] : q[i]) * nH + e.y];
      }
    } else if (gtab) {  // any other row: the handle's gather tables, through the slots
      // The ballot compaction above keeps the slots in increasing order, so
      // sl[l] <= sl[i] whenever l <= i: (sl[i], sl[l]) is a lower-triangle entry
      // of the slot-pair table, the only half it stores.
      const int nfull = (pmax + 1) * (pmax + 2) / 2;
      for (int pi = lane; pi < npair; pi += 32) {
        const uint32_t il = gtab[pi];
        const int i = il & 0xff, l = il >> 8;
        const int si = sl[i], sm = sl[l];
#ifdef ENKFMC_CHECK
        if (sm > si && status) record_error(status, ENKFMC_EINVAL, rowj);
#endif
        const uint32_t e = gtab[nfull + si * (si + 1) / 2 + sm];
        L[at(i, l)] = C[(int64_t)((e & 0x8000u) ? q[l] : q[i]) * nH + (e & 0x7fffu)];
      }
    } else
    for (int pi = lane; pi < npair; pi += 32) {
      int i = (int)((sqrtf(8.f * pi + 1.f) - 1.f) * 0.5f);
      while ((i + 1) * (i + 2) / 2 <= pi) ++i;
      while (i * (i + 1) / 2 > pi) --i;
      const int l = pi - i * (i + 1) / 2;
      const int si = sl[i], sm = sl[l];
      const int dk = off[sm] - off[si];
      const int dy = off[pmax + sm] - off[pmax + si];
      const int dx = off[2 * pmax + sm] - off[2 * pmax + si];
      L[at(i, l)] = cov_lookup(C, nH, g.r, g.vr, q[i], q[l], dk, dy, dx);
    }
    __syncwarp();
    if (ridge_c > 0.0 && p >= N - 1) {
      T tr = 0;
      for (int i = lane; i < p; i += 32) tr += L[at(i, i)];
      tr = warp_sum(tr);
      lam = T(ridge_c) * tr / T(p);
      __syncwarp();
      for (int i = lane; i < p; i += 32) L[at(i, i)] += lam;
    }
    __syncwarp();
  }
  // betabar_i = (<a_j, dX_qi> + <b_j, Lambda_qi>) / D_j - <U_qi, ebar>.  The
  // regression residual satisfies the normal equations, U_P e = lambda beta
  // (G = U_P U_P^T, (G + lambda I) beta = U_P u), so <U_qi, ebar> =
  // 2 Dbar lambda beta_i / (N - 1): no pass over U_P for it.
  const T invD = T(1) / Dj;
  const T ebu = T(2) * Dbar * lam / T(N - 1);
  for (int i = 0; i < p; ++i) {
    T x4[4], l4[4];
    ld4(dxT + (b.row_off + qr[i]) * ldN, x4);
    ld4(lamT + (b.row_off + qr[i]) * ldN, l4);
    T s1 = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      s1 = fma(aj[a], x4[a], s1);
      s1 = fma(bj[a], l4[a], s1);
    }
    s1 = warp_sum(s1);
    if (lane == (i & 31)) va[i] = s1 * invD - ebu * vb[i];
  }
  __syncwarp();
  T f[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) f[a] = eb[a];
  T kappa = 0;
  if (p > 0) {
    const int err = tiled_cholesky(L, at, invd, invd + (ldp - 1), p, p, lane, gtab);
    if (err) {
      if (lane == 0) record_error(status, err, rowj);
      const T z4[4] = {T(0), T(0), T(0), T(0)};
      store(z4, z4, 0, T(0));  // defined (zero) terms for the failed row
      return;
    }
    // v = (L L^T)^-1 betabar in va
    tiled_forward(L, at, invd, va, p, lane);
    tiled_backward(L, at, invd, va, p, lane);
    // f = ebar + U_P^T v; kappa
    T vbeta = 0;
    for (int i = lane; i < p; i += 32) vbeta = fma(va[i], vb[i], vbeta);
    vbeta = warp_sum(vbeta);
    if (lam > T(0)) kappa = T(2) * T(ridge_c) / T(p) * vbeta;
    for (int i = 0; i < p; ++i) {
      const T vi = va[i];
      T u4[4];
      ld4(U + (int64_t)q[i] * ldN, u4);
#pragma unroll
      for (int a = 0; a < 4; ++a) f[a] = fma(u4[a], vi, f[a]);
    }
  }
  store(e, f, p, kappa);
}

}  // namespace

int cov_offset_count(int r, int vr) {
  const int w4 = 4 * r + 1;
  return ((2 * vr + 1) * w4 * w4 + 1) / 2;
}

namespace {

// Launch shape of the covariance table for elements of `esize` bytes: the
// member-major kernel (k_covtable4, even r) when its window and tiles fit,
// else the general one (k_covtable).  False when neither fits.
struct CovShape {
  bool mm;
  int W, tpt, Wp4, mc;
  size_t smem;
};

bool covtable_shape(const Geom& g, size_t esize, CovShape& cs) {
  const int r = g.r;
  const int MC = esize == 4 ? 16 : 8;
  const int nH = cov_offset_count(r, g.vr);
  const int nrho = 1 + 2 * r + g.vr * (4 * r + 1);
  cs.mc = MC;
  if (r % 2 == 0) {
    int W = r <= 2 ? 64 : 32;
    auto bytes = [&](int w) {
      const int wp4 = (w + 4 * r + 4 + 3) / 4 * 4;
      return esize * std::max((size_t)MC * nrho * wp4, (size_t)w * nH);
    };
    while (bytes(W) > 200 * 1024 && W > 8) W /= 2;
    const int w4 = 4 * r + 1;
    const int ntiles = ((2 * r + 1 + 3) / 4 + (nrho - 1) * ((w4 + 3) / 4)) * (W / 4);
    const int tpt = (ntiles + 255) / 256;
    if (bytes(W) <= 220 * 1024 && tpt <= 4) {
      cs.mm = true;
      cs.W = W;
      cs.tpt = tpt;
      cs.Wp4 = (W + 4 * r + 4 + 3) / 4 * 4;
      cs.smem = bytes(W);
      return true;
    }
  }
  int W = r <= 2 ? 64 : 32;
  auto bytes = [&](int w) {
    return esize * ((size_t)nrho * (w + 4 * r) * (MC + 1) + (size_t)w * nH);
  };
  while (bytes(W) > 200 * 1024 && W > 8) W /= 2;
  cs.mm = false;
  cs.W = W;
  cs.tpt = 0;
  cs.Wp4 = 0;
  cs.smem = bytes(W);
  return cs.smem <= 220 * 1024;
}

// Launch shape of k_regress (reg = true) or k_adj_regress for elements of
// `esize` bytes: per-warp workspace, warps per CTA, shared memory.
struct RegShape {
  int ldp, ldg, wpc, use_ptab;
  size_t wb, smem;
};

bool regress_shape(const Geom& g, size_t esize, bool reg, RegShape& rs) {
  rs.ldp = ((g.pmax + 1) + 3) / 4 * 4;
  // (ldg: unused by the packed tiles of Addr, kept in the launch arguments)
  rs.ldg = ((g.pmax + 1) + 7) / 8 * 8 + 4;
  size_t wb = (size_t)rs.ldp * 3 * sizeof(int) +
              esize * ((size_t)addr_elems(esize, rs.ldp, rs.ldg) + (reg ? 4 : 3) * (size_t)rs.ldp);
  rs.wb = (wb + 15) / 16 * 16;
  // single precision: up to 96 KB per CTA (at 39 slots about 54 KB: four CTAs
  // of eight warps per SM), with the typical row's pair table if it fits;
  // double precision: one CTA of
  // up to eight warps per SM in up to 220 KB, without the pair table (the
  // double-precision pipes, not the gather, bound those rows: more warps share
  // them)
  const bool single = esize == 4;
  for (int ptab = reg && single ? 1 : 0; ptab >= 0; --ptab) {  // without the pair table if need be
    size_t offbytes = (3 * (size_t)g.pmax + 15) / 16 * 16;
    if (reg)
      offbytes += (ptab ? pair_table_bytes(g.pmax, g.r, g.periodic) : 0) +
                  gather_table_bytes(g.pmax);
    const size_t budget = (size_t)(single ? 96 : 220) * 1024;
    int wpc = (int)((budget - std::min<size_t>(offbytes, budget)) / rs.wb);
    if (wpc > 8) wpc = 8;
    if (wpc < 1 && single) {
      wpc = (int)(((size_t)200 * 1024 - std::min<size_t>(offbytes, 200 * 1024)) / rs.wb);
      if (wpc > 8) wpc = 8;
    }
    if (wpc >= 1) {
      rs.wpc = wpc;
      rs.use_ptab = ptab;
      rs.smem = offbytes + rs.wb * wpc;
      return true;
    }
  }
  return false;
}

}  // namespace

bool has_fp64_rows(const Geom& g, bool single) {
  return single && !g.plain_fp32 && 2 * g.pmax > g.N;
}

bool estimate_supported(const Geom& g, bool single) {
  // 8-bit row indices in the gather tables, 15-bit table columns, members in
  // at most four rounds of 32 lanes
  if (g.pmax + 1 > 32 * 8 || g.N > 32 * kMaxRounds || g.N < 2) return false;
  if (cov_offset_count(g.r, g.vr) >= 0x8000) return false;
  CovShape cs;
  RegShape rs;
  const size_t es = single ? 4 : 8;
  if (!covtable_shape(g, es, cs) || !regress_shape(g, es, true, rs) ||
      !regress_shape(g, es, false, rs))
    return false;
  if (has_fp64_rows(g, single) &&
      (!covtable_shape(g, 8, cs) || !regress_shape(g, 8, true, rs) ||
       !regress_shape(g, 8, false, rs)))
    return false;
  return true;
}

template <typename T>
cudaError_t launch_anomalies(const Geom& g, const T* Xb, T* U, cudaStream_t s) {
  const dim3 blk(32, 8);
  const int64_t grid = (g.n + 31) / 32;
  k_anomalies<T, T><<<(unsigned)grid, blk, 0, s>>>(Xb, U, nullptr, g.n, g.N, g.ldN);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_covtable(const Geom& g, const T* U, T* C, cudaStream_t s) {
  constexpr int MC = sizeof(T) == 4 ? 16 : 8;
  CovShape cs;
  if (!covtable_shape(g, sizeof(T), cs)) return cudaErrorInvalidConfiguration;
  const int r = g.r;
  const int nH = cov_offset_count(r, g.vr);
  const int nrho = 1 + 2 * r + g.vr * (4 * r + 1);
  int planes = 0;
  for (int v = 0; v < g.nvar; ++v) planes += g.var_lev[v];
  const dim3 grid((g.nlon + cs.W - 1) / cs.W, g.nlat, planes);
  auto run = [&](auto kern, auto... args) -> cudaError_t {
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs.smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 256, cs.smem, s>>>(g, U, C, cs.W, nH, nrho, args...);
    return cudaGetLastError();
  };
  if (cs.mm) {  // aligned b windows: member-major staging
    if (cs.tpt <= 1) return run(k_covtable4<T, MC, 1>, cs.Wp4);
    if (cs.tpt <= 2) return run(k_covtable4<T, MC, 2>, cs.Wp4);
    if (cs.tpt <= 3) return run(k_covtable4<T, MC, 3>, cs.Wp4);
    return run(k_covtable4<T, MC, 4>, cs.Wp4);
  }
  return run(k_covtable<T, MC>);
}

template <typename T, typename TO, int MR>
cudaError_t launch_regress_rm(const Geom& g, const T* U, const T* C, const int32_t* halo,
                              int64_t nitems, const Block* blocks, TO* Tout, TO* Dout,
                              double ridge_c, int32_t* status, int sel, cudaStream_t s) {
  const int nH = cov_offset_count(g.r, g.vr);
  RegShape rs;
  if (!regress_shape(g, sizeof(T), true, rs)) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_regress<T, TO, MR>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs.smem);
  if (e != cudaSuccess) return e;
  // a grid-stride loop over the rows: enough CTAs for an even tail, few enough
  // that each amortises its shared tables (measured on the T63 rows: 64 CTAs
  // per SM beat 24, 32, 128 and one CTA per 8 rows; a handle's tuning can
  // change the cap)
  int64_t grid = (nitems + rs.wpc - 1) / rs.wpc;
  const int64_t cap = (int64_t)(g.sm_count > 0 ? g.sm_count : 152) *
                      (g.regress_cap > 0 ? g.regress_cap : 64);
  if (grid > cap) grid = cap;
  k_regress<T, TO, MR><<<(unsigned)grid, 32 * rs.wpc, rs.smem, s>>>(
      g, U, C, nH, halo, nitems, blocks, Tout, Dout, ridge_c, status, rs.ldp, rs.ldg,
      (int)rs.wb, sel, rs.use_ptab);
  return cudaGetLastError();
}

// The register kernels (k_regress_lane, k_adj_regress_lane) can serve
// single-precision rows of stencils with 16 to 39 predecessor slots (NX = 8
// when the padded Gram matrix needs rows past the 32 lanes).  Measured on the
// T63 rows (N = 80, 39 slots) the tiled kernels are faster: 5.98 against 7.29
// ms for the global rows, 3.49 against 6.01 ms for the boundary rows (whose
// short predecessor lists the register kernel pads to 39), 12.1 against 15.6
// ms for the adjoint.  Two rows per warp (k_regress_pair, choice 3) executes
// 41% fewer instructions than a row per warp but, with shared memory holding
// the same 24 rows per SM in half as many warps, becomes latency bound: 7.04
// against 5.78 ms for the global rows, 6.67 against 3.47 ms for the boundary
// rows (whose neighbouring items often differ in p and then run one after the
// other).  Kernel choice 0 (default) and 1: tiled, a row per warp; 2: the
// register kernels wherever they apply; 3: two rows per warp.
bool regress_lane_applies(const Geom& g, int sel, bool adjoint) {
  (void)adjoint;
  return g.regress_kernel == 2 && sel != 2 && g.N <= 32 * kMaxRounds && g.pmax + 1 > 16 &&
         g.pmax + 1 <= 40;
}

template <int NX>
cudaError_t launch_regress_lane(const Geom& g, const float* U, const float* C,
                                const int32_t* halo, int64_t nitems, const Block* blocks,
                                float* Tout, float* Dout, double ridge_c, int32_t* status,
                                int sel, cudaStream_t s) {
  const int nH = cov_offset_count(g.r, g.vr);
  const int wpc = 8;
  const int wb = lane_warp_bytes(NX, 2 * (32 + NX) + (g.pmax + 3) / 4 * 4);
  const size_t tables = (3 * (size_t)g.pmax + 15) / 16 * 16 + gather_table_bytes(g.pmax);
  const size_t ptab = pair_table_bytes(g.pmax, g.r, g.periodic);
  int use_ptab = 1;
  size_t smem = tables + ptab + (size_t)wpc * wb;
  if (smem > 110 * 1024) {  // two CTAs per SM before the typical row's pair table
    use_ptab = 0;
    smem -= ptab;
  }
  cudaError_t e = cudaFuncSetAttribute(k_regress_lane<NX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t grid = (nitems + wpc - 1) / wpc;
  const int64_t cap = (int64_t)(g.sm_count > 0 ? g.sm_count : 152) *
                      (g.regress_cap > 0 ? g.regress_cap : 64);
  if (grid > cap) grid = cap;
  k_regress_lane<NX><<<(unsigned)grid, 32 * wpc, smem, s>>>(
      g, U, C, nH, halo, nitems, blocks, Tout, Dout, ridge_c, status, wb, sel, use_ptab);
  return cudaGetLastError();
}

// Launch shape of k_regress_pair: two half-warp workspaces of k_regress per
// warp, up to six warps per CTA in up to 72 KB (three CTAs per SM, 96
// registers), with or without the typical row's pair table, whichever fits
// more warps; larger stencils in up to 220 KB; false when not even one warp
// fits.
bool regress_pair_shape(const Geom& g, RegShape& rs) {
  if (!regress_shape(g, 4, true, rs)) return false;
  for (size_t budget : {(size_t)72 * 1024, (size_t)220 * 1024}) {
    int best = 0, best_ptab = 0;
    size_t best_tables = 0;
    for (int ptab = 1; ptab >= 0; --ptab) {
      const size_t tables = (3 * (size_t)g.pmax + 15) / 16 * 16 +
                            (ptab ? pair_table_bytes(g.pmax, g.r, g.periodic) : 0) +
                            gather_table_bytes(g.pmax);
      int wpc = (int)((budget - std::min(tables, budget)) / (2 * rs.wb));
      if (wpc > 6) wpc = 6;
      if (wpc > best) {
        best = wpc;
        best_ptab = ptab;
        best_tables = tables;
      }
    }
    if (best >= 1) {
      rs.wpc = best;
      rs.use_ptab = best_ptab;
      rs.smem = best_tables + 2 * rs.wb * best;
      return true;
    }
  }
  return false;
}

template <int MV>
cudaError_t launch_regress_pair_mv(const Geom& g, const float* U, const float* C,
                                   const int32_t* halo, int64_t nitems, const Block* blocks,
                                   float* Tout, float* Dout, double ridge_c, int32_t* status,
                                   int sel, const RegShape& rs, cudaStream_t s) {
  const int nH = cov_offset_count(g.r, g.vr);
  cudaError_t e = cudaFuncSetAttribute(k_regress_pair<MV>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs.smem);
  if (e != cudaSuccess) return e;
  const int64_t nent = (nitems + 1) / 2;
  int64_t grid = (nent + rs.wpc - 1) / rs.wpc;
  const int64_t cap = (int64_t)(g.sm_count > 0 ? g.sm_count : 152) *
                      (g.regress_cap > 0 ? g.regress_cap : 64);
  if (grid > cap) grid = cap;
  k_regress_pair<MV><<<(unsigned)grid, 32 * rs.wpc, rs.smem, s>>>(
      g, U, C, nH, halo, nitems, blocks, Tout, Dout, ridge_c, status, rs.ldp, rs.ldg, (int)rs.wb,
      sel, rs.use_ptab);
  return cudaGetLastError();
}

template <typename T, typename TO>
cudaError_t launch_regress(const Geom& g, const T* U, const T* C, const int32_t* halo,
                           int64_t nitems, const Block* blocks, TO* Tout, TO* Dout, double ridge_c,
                           int32_t* status, int sel, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if (g.pmax + 1 > 32 * 8 || g.N > 32 * kMaxRounds) return cudaErrorInvalidConfiguration;
  if constexpr (std::is_same<T, float>::value && std::is_same<TO, float>::value) {
    RegShape ps;
    if (g.regress_kernel == 3 && sel != 2 && regress_pair_shape(g, ps)) {
      if (g.ldN <= 64)
        return launch_regress_pair_mv<1>(g, U, C, halo, nitems, blocks, Tout, Dout, ridge_c,
                                         status, sel, ps, s);
      return launch_regress_pair_mv<2>(g, U, C, halo, nitems, blocks, Tout, Dout, ridge_c, status,
                                       sel, ps, s);
    }
    if (regress_lane_applies(g, sel, false)) {
      if (g.pmax + 1 > 32)
        return launch_regress_lane<8>(g, U, C, halo, nitems, blocks, Tout, Dout, ridge_c, status,
                                      sel, s);
      return launch_regress_lane<0>(g, U, C, halo, nitems, blocks, Tout, Dout, ridge_c, status,
                                    sel, s);
    }
  }
  const int mr = (g.N + 31) / 32;
  if (mr <= 2)
    return launch_regress_rm<T, TO, 2>(g, U, C, halo, nitems, blocks, Tout, Dout, ridge_c,
                                       status, sel, s);
  if (mr == 3)
    return launch_regress_rm<T, TO, 3>(g, U, C, halo, nitems, blocks, Tout, Dout, ridge_c,
                                       status, sel, s);
  return launch_regress_rm<T, TO, 4>(g, U, C, halo, nitems, blocks, Tout, Dout, ridge_c, status,
                                     sel, s);
}

template <int NX>
cudaError_t launch_adj_regress_lane(const Geom& g, const Block* blocks, int nblock, int nb_max,
                                    const float* U, const float* C, const float* Tg,
                                    const float* Dg, const float* Te, const float* De,
                                    const float* aT, const float* bT, const float* dxT,
                                    const float* lamT, const int2* ptab, const uint16_t* gtab,
                                    float* Eo, float* Fo, float* Vo, float* Ko, double ridge_c,
                                    int32_t* status, int sel, cudaStream_t s) {
  const int nH = cov_offset_count(g.r, g.vr);
  const int wpc = 8;
  const int wb = lane_warp_bytes(NX, 3 * (32 + NX));
  const size_t smem = (3 * (size_t)g.pmax + 15) / 16 * 16 + (size_t)wpc * wb;
  cudaError_t e = cudaFuncSetAttribute(k_adj_regress_lane<NX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((nb_max + wpc - 1) / wpc, nblock);
  k_adj_regress_lane<NX><<<grid, 32 * wpc, smem, s>>>(g, blocks, U, C, nH, Tg, Dg, Te, De, aT,
                                                      bT, dxT, lamT, ptab, gtab, Eo, Fo, Vo, Ko,
                                                      ridge_c, status, wb, sel);
  return cudaGetLastError();
}

template <typename T, typename TS>
cudaError_t launch_adj_regress(const Geom& g, const Block* blocks, int nblock, int nb_max,
                               const T* U, const T* C, const TS* Tg, const TS* Dg, const TS* Te,
                               const TS* De, const TS* aT, const TS* bT, const TS* dxT,
                               const TS* lamT, const int2* ptab, const uint16_t* gtab,
                               TS* Eo, TS* Fo, TS* Vo, TS* Ko, double ridge_c, int32_t* status,
                               int sel,
                               cudaStream_t s) {
  if (g.pmax + 1 > 32 * kMaxRounds * 2 || g.N > 32 * kMaxRounds)
    return cudaErrorInvalidConfiguration;
  if constexpr (std::is_same<T, float>::value && std::is_same<TS, float>::value) {
    if (regress_lane_applies(g, sel, true) && ptab && gtab) {
      if (g.pmax + 1 > 32)
        return launch_adj_regress_lane<8>(g, blocks, nblock, nb_max, U, C, Tg, Dg, Te, De, aT,
                                          bT, dxT, lamT, ptab, gtab, Eo, Fo, Vo, Ko, ridge_c,
                                          status, sel, s);
      return launch_adj_regress_lane<0>(g, blocks, nblock, nb_max, U, C, Tg, Dg, Te, De, aT, bT,
                                        dxT, lamT, ptab, gtab, Eo, Fo, Vo, Ko, ridge_c, status,
                                        sel, s);
    }
  }
  const int nH = cov_offset_count(g.r, g.vr);
  RegShape rs;
  if (!regress_shape(g, sizeof(T), false, rs)) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_adj_regress<T, TS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs.smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((nb_max + rs.wpc - 1) / rs.wpc, nblock);
  k_adj_regress<T, TS><<<grid, 32 * rs.wpc, rs.smem, s>>>(
      g, blocks, U, C, nH, Tg, Dg, Te, De, aT, bT, dxT, lamT, ptab, gtab, Eo, Fo, Vo, Ko, ridge_c,
      status,
      rs.ldp, rs.ldg, (int)rs.wb, sel);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The estimate's launch sequence with the precision rule: double-precision
// problems run in double; single-precision problems run in single, except the
// rows with 2p > N (p/N > 0.5), whose nearly singular Gram matrices are formed
// from FP64 anomalies and an FP64 covariance table and factored and solved in
// double precision (st.U64 / st.C64 present exactly when has_fp64_rows).
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_stat_anomalies(const Geom& g, const T* Xb, const EstStats<T>& st,
                                  cudaStream_t s, int* nk) {
  ++*nk;
  if constexpr (std::is_same<T, float>::value) {
    if (st.U64) {
      const dim3 blk(32, 8);
      const int64_t grid = (g.n + 31) / 32;
      k_anomalies<float, double><<<(unsigned)grid, blk, 0, s>>>(Xb, st.U64, st.U, g.n, g.N,
                                                                g.ldN);
      return cudaGetLastError();
    }
  }
  return launch_anomalies<T>(g, Xb, st.U, s);
}

template <typename T>
cudaError_t launch_stat_covtables(const Geom& g, const EstStats<T>& st, cudaStream_t s,
                                  int* nk) {
  ++*nk;
  cudaError_t e = launch_covtable<T>(g, st.U, st.C, s);
  if (e == cudaSuccess && st.C64) {
    ++*nk;
    e = launch_covtable<double>(g, st.U64, st.C64, s);
  }
  return e;
}

template <typename T>
cudaError_t launch_regressions(const Geom& g, const EstStats<T>& st, const int32_t* halo,
                               int64_t nitems, const Block* blocks, T* Tout, T* Dout,
                               double ridge_c, int32_t* status, cudaStream_t s, int* nk) {
  if (nitems <= 0) return cudaSuccess;
  if (!st.C64) {
    ++*nk;
    return launch_regress<T, T>(g, st.U, st.C, halo, nitems, blocks, Tout, Dout, ridge_c, status,
                                0, s);
  }
  *nk += 2;
  cudaError_t e = launch_regress<T, T>(g, st.U, st.C, halo, nitems, blocks, Tout, Dout, ridge_c,
                                       status, 1, s);
  if (e != cudaSuccess) return e;
  return launch_regress<double, T>(g, st.U64, st.C64, halo, nitems, blocks, Tout, Dout, ridge_c,
                                   status, 2, s);
}

template <typename T>
cudaError_t launch_adj_regressions(const Geom& g, const Block* blocks, int nblock, int nb_max,
                                   const EstStats<T>& st, const T* Tg, const T* Dg, const T* Te,
                                   const T* De, const T* aT, const T* bT, const T* dxT,
                                   const T* lamT, const int2* ptab, const uint16_t* gtab, T* Eo,
                                   T* Fo, T* Vo, T* Ko,
                                   double ridge_c, int32_t* status, cudaStream_t s, int* nk) {
  if (!st.C64) {
    ++*nk;
    return launch_adj_regress<T, T>(g, blocks, nblock, nb_max, st.U, st.C, Tg, Dg, Te, De, aT, bT,
                                    dxT, lamT, ptab, gtab, Eo, Fo, Vo, Ko, ridge_c, status, 0,
                                    s);
  }
  *nk += 2;
  cudaError_t e = launch_adj_regress<T, T>(g, blocks, nblock, nb_max, st.U, st.C, Tg, Dg, Te, De,
                                           aT, bT, dxT, lamT, ptab, gtab, Eo, Fo, Vo, Ko, ridge_c,
                                           status, 1, s);
  if (e != cudaSuccess) return e;
  return launch_adj_regress<double, T>(g, blocks, nblock, nb_max, st.U64, st.C64, Tg, Dg, Te, De,
                                       aT, bT, dxT, lamT, ptab, gtab, Eo, Fo, Vo, Ko, ridge_c,
                                       status, 2, s);
}

#define INST(T)                                                                                  \
  template cudaError_t launch_anomalies<T>(const Geom&, const T*, T*, cudaStream_t);            \
  template cudaError_t launch_covtable<T>(const Geom&, const T*, T*, cudaStream_t);             \
  template cudaError_t launch_stat_anomalies<T>(const Geom&, const T*, const EstStats<T>&,      \
                                                cudaStream_t, int*);                             \
  template cudaError_t launch_stat_covtables<T>(const Geom&, const EstStats<T>&, cudaStream_t,  \
                                                int*);                                           \
  template cudaError_t launch_regressions<T>(const Geom&, const EstStats<T>&, const int32_t*,   \
                                             int64_t, const Block*, T*, T*, double, int32_t*,    \
                                             cudaStream_t, int*);                                \
  template cudaError_t launch_adj_regressions<T>(                                               \
      const Geom&, const Block*, int, int, const EstStats<T>&, const T*, const T*, const T*,     \
      const T*, const T*, const T*, const T*, const T*, const int2*, const uint16_t*, T*, T*, T*, \
      T*, double, int32_t*, cudaStream_t, int*);
INST(float)
INST(double)
#undef INST

}  // namespace enkfmc
