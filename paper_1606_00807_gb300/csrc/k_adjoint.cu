// Reverse pass of the analysis (the gradient of a scalar loss of X^a with
// respect to X^b, y and diag(R)), per (sub-domain, variable) block, reusing the
// forward factor of A:
//   seed:   W = dL/dX^a on the interior rows, 0 on the boundary; Lambda = A^-1 W
//   obs:    ybar_o += sum_i Lambda_ci / R_o,
//           Rbar_o += (<Lambda_c, dX_c> - <Lambda_c, Delta_o>) / R_o^2
//                     + <Lambda_c, Z_o> / (2 R_o sqrt(R_o)),
//           Xbbar_c -= Lambda_c / R_o            (Delta = Y^s - H X^b, Eq. 11)
//   ab:     a_j = (T Lambda)_j, b_j = (T dX)_j, and row-major copies of dX, Lambda
//   (regressions: k_adj_regress in k_estimate.cu)
//   finish: Xbbar += dL/dX^a + Ubar - mean_members(Ubar)   (Eq. 10, Eq. 5)
// Contributions of overlapping extended boxes meet in atomic adds.
#include "enkfmc_internal.h"

namespace enkfmc {

namespace {

constexpr int kRows = 32;
constexpr int kWarps = 4;

template <typename T>
__global__ void __launch_bounds__(128) k_adj_seed(const Geom g, const Block* __restrict__ blocks,
                                                  const T* __restrict__ Xa_bar,
                                                  T* __restrict__ W) {
  const Block b = blocks[blockIdx.y];
  const int loc = blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= b.nb) return;
  const int plane = b.ey * b.ex;
  const int k = loc / plane;
  const int yy = (loc - k * plane) / b.ex;
  const int xx = loc - k * plane - yy * b.ex;
  const int y = b.lat_lo + yy, x = imod(b.lon_lo + xx, g.nlon);
  const bool inner = in_interior(b, y, x);
  const int64_t l = coords_label(g, b.var, k, y, x);
  T* out = W + b.row_off * g.N + loc;
  for (int m = 0; m < g.N; ++m)
    out[(int64_t)m * b.nb] = inner ? Xa_bar[(int64_t)m * g.n + l] : T(0);
}

template <typename T>
__global__ void __launch_bounds__(128) k_adj_obs(
    const Geom g, const Block* __restrict__ blocks, const int32_t* __restrict__ obs_of,
    int64_t mobs, const T* __restrict__ Xb, const T* __restrict__ y, const T* __restrict__ R,
    const T* __restrict__ Z, const T* __restrict__ lam, const T* __restrict__ dX,
    const T* __restrict__ dX2, T* __restrict__ Xb_bar, T* __restrict__ y_bar,
    T* __restrict__ R_bar) {
  const Block b = blocks[blockIdx.y];
  const int loc = blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= b.nb) return;
  const int plane = b.ey * b.ex;
  const int k = loc / plane;
  const int yy = (loc - k * plane) / b.ex;
  const int xx = loc - k * plane - yy * b.ex;
  const int64_t l = coords_label(g, b.var, k, b.lat_lo + yy, imod(b.lon_lo + xx, g.nlon));
  const int o = obs_of[l];
  if (o < 0) return;
  const T Ro = R[o], yo = y[o];
  const T sq = sqrt(Ro), rinv = T(1) / Ro;
  T s_l = 0, s_ldx = 0, s_ldel = 0, s_lz = 0;
  for (int m = 0; m < g.N; ++m) {
    const int64_t e = b.row_off * g.N + (int64_t)m * b.nb + loc;
    const T lm = lam[e];
    const T dx = dX2 ? dX[e] + dX2[e] : dX[e];
    const T z = Z[(int64_t)m * mobs + o];
    const T del = fma(sq, z, yo) - Xb[(int64_t)m * g.n + l];
    s_l += lm;
    s_ldx = fma(lm, dx, s_ldx);
    s_ldel = fma(lm, del, s_ldel);
    s_lz = fma(lm, z, s_lz);
    atomicAdd(Xb_bar + (int64_t)m * g.n + l, -lm * rinv);
  }
  atomicAdd(y_bar + o, s_l * rinv);
  atomicAdd(R_bar + o, (s_ldx - s_ldel) * rinv * rinv + s_lz * rinv / (T(2) * sq));
}

// a = T Lambda, b = T dX for 32 extended rows per thread block, written
// row-major ([row][ldN]) together with row-major copies of dX and Lambda.
template <typename T>
__global__ void __launch_bounds__(kRows* kWarps) k_adj_ab(
    const Geom g, const Block* __restrict__ blocks, const T* __restrict__ Tg,
    const T* __restrict__ Te, const T* __restrict__ lam, const T* __restrict__ dX,
    const T* __restrict__ dX2, T* __restrict__ aT, T* __restrict__ bT, T* __restrict__ dxT,
    T* __restrict__ lamT) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int pmax = g.pmax, N = g.N, ldo = N + 1;
  T* tv = reinterpret_cast<T*>(smem);                  // [kRows][pmax]
  T* Oa = tv + kRows * pmax;                           // [kRows][ldo] x 4 outputs
  T* Ob = Oa + kRows * ldo;
  T* Ox = Ob + kRows * ldo;
  T* Ol = Ox + kRows * ldo;
  int* nbr = reinterpret_cast<int*>(Ol + kRows * ldo);  // [kRows][pmax]
  const Block b = blocks[blockIdx.y];
  const int loc0 = blockIdx.x * kRows;
  if (loc0 >= b.nb) return;
  const int nr = min(kRows, b.nb - loc0);
  const int plane = b.ey * b.ex;
  for (int idx = threadIdx.x; idx < nr * pmax; idx += blockDim.x) {
    const int i = idx / pmax, s = idx - i * pmax;
    const int loc = loc0 + i;
    const int k = loc / plane, yy = (loc - k * plane) / b.ex, xx = loc - k * plane - yy * b.ex;
    const int y = b.lat_lo + yy, x = imod(b.lon_lo + xx, g.nlon);
    const T* trow = in_interior(b, y, x) ? Tg + coords_label(g, b.var, k, y, x) * pmax
                                         : Te + (b.row_off + loc) * pmax;
    const T t = trow[s];
    int kq, yq, xq, yyq, xxq, qq = -1;
    if (t != T(0) && slot_pred(g, k, y, x, s, kq, yq, xq) && in_ext(b, g.nlon, yq, xq, yyq, xxq))
      qq = (kq * b.ey + yyq) * b.ex + xxq;
    nbr[i * pmax + s] = qq;
    tv[i * pmax + s] = qq >= 0 ? t : T(0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < nr) {
    const int* nb_i = nbr + lane * pmax;
    const T* t_i = tv + lane * pmax;
    for (int m = warp; m < N; m += kWarps) {
      const int64_t base = b.row_off * N + (int64_t)m * b.nb;
      const T* lm = lam + base;
      const T* d1 = dX + base;
      const T* d2 = dX2 ? dX2 + base : nullptr;
      const int a0 = loc0 + lane;
      T sa = lm[a0];
      T dxa = d2 ? d1[a0] + d2[a0] : d1[a0];
      T sb = dxa;
      for (int sl = 0; sl < pmax; ++sl) {
        const int qq = nb_i[sl];
        if (qq < 0) continue;
        const T t = t_i[sl];
        sa = fma(t, lm[qq], sa);
        sb = fma(t, d2 ? d1[qq] + d2[qq] : d1[qq], sb);
      }
      Oa[lane * ldo + m] = sa;
      Ob[lane * ldo + m] = sb;
      Ox[lane * ldo + m] = dxa;
      Ol[lane * ldo + m] = lm[a0];
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nr * N; idx += blockDim.x) {
    const int i = idx / N, m = idx - i * N;
    const int64_t o = (b.row_off + loc0 + i) * g.ldN + m;
    aT[o] = Oa[i * ldo + m];
    bT[o] = Ob[i * ldo + m];
    dxT[o] = Ox[i * ldo + m];
    lamT[o] = Ol[i * ldo + m];
  }
}

// Xbbar[m][l] += Xabar[m][l] + Ubar[l][m] - mean_m Ubar[l][m]
template <typename T>
__global__ void __launch_bounds__(256) k_adj_finish(const T* __restrict__ Ubar,
                                                    const T* __restrict__ Xa_bar,
                                                    T* __restrict__ Xb_bar, int64_t n, int N,
                                                    int ldN) {
  __shared__ T tile[32][33];
  __shared__ T mean_s[32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t c0 = (int64_t)blockIdx.x * 32;
  // means over members of components c0..c0+31 (rows of Ubar)
  for (int i = ty; i < 32; i += 8) {
    const int64_t c = c0 + i;
    T s = 0;
    if (c < n)
      for (int m = tx; m < N; m += 32) s += Ubar[c * ldN + m];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (tx == 0) mean_s[i] = s / T(N);
  }
  __syncthreads();
  for (int m0 = 0; m0 < N; m0 += 32) {
    for (int i = ty; i < 32; i += 8) {
      const int64_t c = c0 + i;
      const int m = m0 + tx;
      tile[i][tx] = (c < n && m < N) ? Ubar[c * ldN + m] - mean_s[i] : T(0);
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
      const int m = m0 + i;
      const int64_t c = c0 + tx;
      if (m < N && c < n) {
        const int64_t e = (int64_t)m * n + c;
        Xb_bar[e] += Xa_bar[e] + tile[tx][i];
      }
    }
    __syncthreads();
  }
}

}  // namespace

template <typename T>
cudaError_t launch_adj_seed(const Geom& g, const Block* blocks, int nblock, int nb_max,
                            const T* Xa_bar, T* W, cudaStream_t s) {
  const dim3 grid((nb_max + 127) / 128, nblock);
  k_adj_seed<T><<<grid, 128, 0, s>>>(g, blocks, Xa_bar, W);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_obs(const Geom& g, const Block* blocks, int nblock, int nb_max,
                           const int32_t* obs_of, int64_t m, const T* Xb, const T* y, const T* R,
                           const T* Z, const T* lam, const T* dX, const T* dX2, T* Xb_bar,
                           T* y_bar, T* R_bar, cudaStream_t s) {
  const dim3 grid((nb_max + 127) / 128, nblock);
  k_adj_obs<T><<<grid, 128, 0, s>>>(g, blocks, obs_of, m, Xb, y, R, Z, lam, dX, dX2, Xb_bar,
                                    y_bar, R_bar);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_ab(const Geom& g, const Block* blocks, int nblock, int nb_max,
                          const T* Tg, const T* Te, const T* lam, const T* dX, const T* dX2,
                          T* aT, T* bT, T* dxT, T* lamT, cudaStream_t s) {
  const size_t smem = sizeof(T) * ((size_t)kRows * g.pmax + 4 * (size_t)kRows * (g.N + 1)) +
                      sizeof(int) * (size_t)kRows * g.pmax;
  cudaError_t e = cudaFuncSetAttribute(k_adj_ab<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((nb_max + kRows - 1) / kRows, nblock);
  k_adj_ab<T><<<grid, kRows * kWarps, smem, s>>>(g, blocks, Tg, Te, lam, dX, dX2, aT, bT, dxT,
                                                 lamT);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_finish(const Geom& g, const T* Ubar, const T* Xa_bar, T* Xb_bar,
                              cudaStream_t s) {
  const dim3 blk(32, 8);
  k_adj_finish<T><<<(unsigned)((g.n + 31) / 32), blk, 0, s>>>(Ubar, Xa_bar, Xb_bar, g.n, g.N,
                                                               g.ldN);
  return cudaGetLastError();
}

#define INST(T)                                                                                  \
  template cudaError_t launch_adj_seed<T>(const Geom&, const Block*, int, int, const T*, T*,    \
                                          cudaStream_t);                                         \
  template cudaError_t launch_adj_obs<T>(const Geom&, const Block*, int, int, const int32_t*,   \
                                         int64_t, const T*, const T*, const T*, const T*,       \
                                         const T*, const T*, const T*, T*, T*, T*, cudaStream_t); \
  template cudaError_t launch_adj_ab<T>(const Geom&, const Block*, int, int, const T*, const T*,\
                                        const T*, const T*, const T*, T*, T*, T*, T*,           \
                                        cudaStream_t);                                           \
  template cudaError_t launch_adj_finish<T>(const Geom&, const T*, const T*, T*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace enkfmc
