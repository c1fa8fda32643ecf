// Reverse pass of the analysis (the gradient of a scalar loss of X^a with
// respect to X^b, y and diag(R)), per (sub-domain, variable) block, reusing the
// forward factor of A:
//   seed:   W = dL/dX^a on the interior rows, 0 on the boundary; Lambda = A^-1 W
//   ab:     a_j = (T Lambda)_j, b_j = (T dX)_j, and row-major copies of dX, Lambda
//   (regressions: k_adj_regress in k_estimate.cu stores per extended row the
//    terms e, f, v, kappa of its contribution to Ubar)
//   gather: Ubar of every extended row c = f_c + sum over the rows j holding c
//           in slot s of (v_j[s] e_j - beta_j[s] f_j - kappa_j U_c), s in order
//   owner:  every component and observation from the blocks whose extended set
//           holds it, in block order:
//           Xbbar = dL/dX^a + Ubar - mean_members(Ubar) - sum_b Lambda_c / R_o
//           ybar_o = sum_b sum_i Lambda_ci / R_o,
//           Rbar_o = sum_b (<Lambda_c, dX_c> - <Lambda_c, Delta_o>) / R_o^2
//                    + <Lambda_c, Z_o> / (2 R_o sqrt(R_o))   (Delta = Y^s - H X^b)
// Every sum runs in a fixed order (no atomics): the gradient is reproducible
// bit for bit.
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

// a = T Lambda, b = T dX for 32 extended rows per thread block, written
// row-major ([row][ldN]) together with row-major copies of dX and Lambda;
// kAbWarps warps over the members (the shared tile of the outputs, not the
// threads, bounds the CTAs per SM).
constexpr int kAbWarps = 8;
template <typename T>
__global__ void __launch_bounds__(kRows* kAbWarps) k_adj_ab(
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
    for (int m = warp; m < N; m += kAbWarps) {
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

// Four consecutive members (16-byte aligned rows of ldN, a multiple of 4).
template <typename T>
__device__ __forceinline__ void ld4r(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 c = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = c.x; v[3] = c.y;
  }
}
template <typename T>
__device__ __forceinline__ void st4r(T* p, const T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
}

// Ubar of the extended rows of one block, one warp per row c, members 4 lane ..
// 4 lane + 3 (N <= 128).  The rows j that hold c are j = c - offset(s) for the
// slots s whose predecessor, seen from j inside the block, is c; they are
// listed in slot order (ballot compaction) with their scalars (-beta_j[s],
// v_j[s], kappa_j, found by the lane of slot s), then their terms are added in
// that order: Ubar_c = f_c + sum (v_j[s] e_j - beta_j[s] f_j - kappa_j U_c).
template <typename T>
__global__ void __launch_bounds__(256) k_adj_gather(
    const Geom g, const Block* __restrict__ blocks, const T* __restrict__ Tg,
    const T* __restrict__ Te, const T* __restrict__ U, const T* __restrict__ Eo,
    const T* __restrict__ Fo, const T* __restrict__ Vo, const T* __restrict__ Ko,
    T* __restrict__ Ub) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  const int pmax = g.pmax, ldN = g.ldN;
  // per warp: [pmax] block-relative row j, then [pmax] each of -beta_j[s], v_j[s], kappa_j
  int* cj = reinterpret_cast<int*>(smem) + (size_t)warp * 4 * pmax;
  T* ct = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(smem) +
                               (size_t)wpc * 4 * pmax * sizeof(int)) +
          (size_t)warp * 3 * pmax;
  T* cv = ct + pmax;
  T* ck = cv + pmax;
  const Block b = blocks[blockIdx.y];
  const int c = blockIdx.x * wpc + warp;
  if (c >= b.nb) return;
  const int plane = b.ey * b.ex;
  const int kc = c / plane, yyc = (c - kc * plane) / b.ex, xxc = c - kc * plane - yyc * b.ex;
  const int yc = b.lat_lo + yyc, xc = imod(b.lon_lo + xxc, g.nlon);
  const int v = b.var;
  int nc = 0;
  for (int s0 = 0; s0 < pmax; s0 += 32) {
    const int s = s0 + lane;
    int locj = -1;
    if (s < pmax) {
      int dk, dy, dx;
      slot_offset(s, g.r, g.vr, dk, dy, dx);
      const int kj = kc - dk, yj = yc - dy;
      int xj = xc - dx;
      bool ok = kj >= 0 && kj < b.nlev_b && yj >= 0 && yj < g.nlat;
      if (ok && (xj < 0 || xj >= g.nlon)) {
        if (g.periodic) xj = imod(xj, g.nlon);
        else ok = false;
      }
      int yyj, xxj, kq, yq, xq;
      // row j inside the block, and its slot s lands on c
      if (ok && in_ext(b, g.nlon, yj, xj, yyj, xxj) &&
          slot_pred_off(g, kj, yj, xj, dk, dy, dx, kq, yq, xq) && kq == kc && yq == yc && xq == xc)
        locj = (kj * b.ey + yyj) * b.ex + xxj;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, locj >= 0);
    const int idx = nc + __popc(mask & ((1u << lane) - 1u));
    if (locj >= 0) {
      // the row's scalars for this slot, read once by the lane that found it
      const int kj = locj / plane, yyj = (locj - kj * plane) / b.ex;
      const int xxj = locj - kj * plane - yyj * b.ex;
      const int yj = b.lat_lo + yyj, xj = imod(b.lon_lo + xxj, g.nlon);
      const int64_t rowj = b.row_off + locj;
      cj[idx] = locj;
      ct[idx] = in_interior(b, yj, xj) ? Tg[coords_label(g, v, kj, yj, xj) * pmax + s]
                                       : Te[rowj * pmax + s];  // -beta_j[s]
      cv[idx] = Vo[rowj * pmax + s];
      ck[idx] = Ko[rowj];
    }
    nc += __popc(mask);
  }
  __syncwarp();
  const int m0 = 4 * lane;
  if (m0 >= ldN) return;
  T acc[4], u4[4];
  ld4r(Fo + (b.row_off + c) * ldN + m0, acc);
  ld4r(U + coords_label(g, v, kc, yc, xc) * ldN + m0, u4);
  for (int i = 0; i < nc; ++i) {
    const int64_t rowj = b.row_off + cj[i];
    const T t = ct[i], vv = cv[i], kap = ck[i];
    T e4[4], f4[4];
    ld4r(Eo + rowj * ldN + m0, e4);
    ld4r(Fo + rowj * ldN + m0, f4);
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a] = fma(vv, e4[a], fma(t, f4[a], fma(-kap, u4[a], acc[a])));
  }
  st4r(Ub + (b.row_off + c) * ldN + m0, acc);
}

// The gradients of 32 consecutive components per thread block (a warp per
// component, lanes over members), from the blocks whose extended set holds
// the component, in increasing block order; then the member-major write of
// dL/dX^b through a shared tile (coalesced).
template <typename T>
__global__ void __launch_bounds__(256) k_adj_owner(
    const Geom g, const Block* __restrict__ blocks, int nsubx, int nsuby, int sub_lon,
    int sub_lat, const int32_t* __restrict__ obs_of, int64_t mobs, const T* __restrict__ Xb,
    const T* __restrict__ y, const T* __restrict__ R, const T* __restrict__ Z,
    const T* __restrict__ Ub, const T* __restrict__ lamT, const T* __restrict__ dxT,
    const T* __restrict__ Xa_bar, T* __restrict__ Xb_bar, T* __restrict__ y_bar,
    T* __restrict__ R_bar) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = g.N, ldN = g.ldN, ldS = N + 1;
  T* S = reinterpret_cast<T*>(smem);  // [32][N + 1]: dL/dX^b - dL/dX^a of the components
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * 32;
  const int r = g.r;
  for (int i = warp; i < 32; i += nw) {
    const int64_t c = c0 + i;
    if (c >= g.n) break;
    int v, k, yc, xc;
    label_coords(g, c, v, k, yc, xc);
    // tile columns reached by longitudes xc - r .. xc + r, increasing (at most 8);
    // every column when a tile and its boundary can span the whole ring
    int sxs[8], nsx = 0;
    const bool ring = g.periodic && sub_lon + 2 * r >= g.nlon;
    for (int d = ring ? 0 : -r; d <= (ring ? -1 : r); ++d) {
      int x = xc + d;
      if (x < 0 || x >= g.nlon) {
        if (!g.periodic) continue;
        x = imod(x, g.nlon);
      }
      const int t = x / sub_lon;
      bool seen = false;
      for (int q = 0; q < nsx; ++q) seen |= sxs[q] == t;
      if (!seen && nsx < 8) {
        int q = nsx++;
        while (q > 0 && sxs[q - 1] > t) {
          sxs[q] = sxs[q - 1];
          --q;
        }
        sxs[q] = t;
      }
    }
    if (ring)
      for (int t = 0; t < nsubx && t < 8; ++t) sxs[nsx++] = t;
    const int sy0 = max(0, yc - r) / sub_lat, sy1 = min(nsuby - 1, min(g.nlat - 1, yc + r) / sub_lat);
    const int o = obs_of[c];
    T us[4] = {T(0), T(0), T(0), T(0)}, ls[4] = {T(0), T(0), T(0), T(0)};
    T sldx = 0;
    for (int sy = sy0; sy <= sy1; ++sy)
      for (int q = 0; q < nsx; ++q) {
        const Block& b = blocks[(sy * nsubx + sxs[q]) * g.nvar + v];
        int yy, xx;
        if (!in_ext(b, g.nlon, yc, xc, yy, xx)) continue;
        const int64_t row = b.row_off + (k * b.ey + yy) * b.ex + xx;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int m = lane + 32 * t;
          if (m < N) {
            us[t] += Ub[row * ldN + m];
            if (o >= 0) {
              const T lm = lamT[row * ldN + m];
              ls[t] += lm;
              sldx = fma(lm, dxT[row * ldN + m], sldx);
            }
          }
        }
      }
    T su = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) su += us[t];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) su += __shfl_xor_sync(0xffffffffu, su, off);
    const T mean = su / T(N);
    T rinv = 0;
    if (o >= 0) {
      const T Ro = R[o], yo = y[o], sq = sqrt(Ro);
      rinv = T(1) / Ro;
      T s_l = 0, s_ldel = 0, s_lz = 0;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int m = lane + 32 * t;
        if (m < N) {
          const T z = Z[(int64_t)m * mobs + o];
          const T del = fma(sq, z, yo) - Xb[(int64_t)m * g.n + c];
          s_l += ls[t];
          s_ldel = fma(ls[t], del, s_ldel);
          s_lz = fma(ls[t], z, s_lz);
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        s_l += __shfl_xor_sync(0xffffffffu, s_l, off);
        s_ldel += __shfl_xor_sync(0xffffffffu, s_ldel, off);
        s_lz += __shfl_xor_sync(0xffffffffu, s_lz, off);
        sldx += __shfl_xor_sync(0xffffffffu, sldx, off);
      }
      if (lane == 0) {
        y_bar[o] = s_l * rinv;
        R_bar[o] = (sldx - s_ldel) * rinv * rinv + s_lz * rinv / (T(2) * sq);
      }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int m = lane + 32 * t;
      if (m < N) S[i * ldS + m] = us[t] - mean - ls[t] * rinv;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 32 * N; idx += blockDim.x) {
    const int m = idx / 32, i = idx - m * 32;
    const int64_t c = c0 + i;
    if (c < g.n) {
      const int64_t e = (int64_t)m * g.n + c;
      Xb_bar[e] = Xa_bar[e] + S[i * ldS + m];
    }
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
cudaError_t launch_adj_ab(const Geom& g, const Block* blocks, int nblock, int nb_max,
                          const T* Tg, const T* Te, const T* lam, const T* dX, const T* dX2,
                          T* aT, T* bT, T* dxT, T* lamT, cudaStream_t s) {
  const size_t smem = sizeof(T) * ((size_t)kRows * g.pmax + 4 * (size_t)kRows * (g.N + 1)) +
                      sizeof(int) * (size_t)kRows * g.pmax;
  cudaError_t e = cudaFuncSetAttribute(k_adj_ab<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((nb_max + kRows - 1) / kRows, nblock);
  k_adj_ab<T><<<grid, kRows * kAbWarps, smem, s>>>(g, blocks, Tg, Te, lam, dX, dX2, aT, bT,
                                                   dxT, lamT);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_gather(const Geom& g, const Block* blocks, int nblock, int nb_max,
                              const T* Tg, const T* Te, const T* U, const T* Eo, const T* Fo,
                              const T* Vo, const T* Ko, T* Ub, cudaStream_t s) {
  const int wpc = 8;
  const size_t smem = (sizeof(int) * 4 + sizeof(T) * 3) * (size_t)g.pmax * wpc;
  cudaError_t e = cudaFuncSetAttribute(k_adj_gather<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((nb_max + wpc - 1) / wpc, nblock);
  k_adj_gather<T><<<grid, 32 * wpc, smem, s>>>(g, blocks, Tg, Te, U, Eo, Fo, Vo, Ko, Ub);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_owner(const Geom& g, const Block* blocks, int nsubx, int nsuby,
                             int sub_lon, int sub_lat, const int32_t* obs_of, int64_t m,
                             const T* Xb, const T* y, const T* R, const T* Z, const T* Ub,
                             const T* lamT, const T* dxT, const T* Xa_bar, T* Xb_bar, T* y_bar,
                             T* R_bar, cudaStream_t s) {
  const size_t smem = sizeof(T) * 32 * (size_t)(g.N + 1);
  cudaError_t e = cudaFuncSetAttribute(k_adj_owner<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_adj_owner<T><<<(unsigned)((g.n + 31) / 32), 256, smem, s>>>(
      g, blocks, nsubx, nsuby, sub_lon, sub_lat, obs_of, m, Xb, y, R, Z, Ub, lamT, dxT, Xa_bar,
      Xb_bar, y_bar, R_bar);
  return cudaGetLastError();
}

#define INST(T)                                                                                  \
  template cudaError_t launch_adj_seed<T>(const Geom&, const Block*, int, int, const T*, T*,    \
                                          cudaStream_t);                                         \
  template cudaError_t launch_adj_ab<T>(const Geom&, const Block*, int, int, const T*, const T*,\
                                        const T*, const T*, const T*, T*, T*, T*, T*,           \
                                        cudaStream_t);                                           \
  template cudaError_t launch_adj_gather<T>(const Geom&, const Block*, int, int, const T*,      \
                                            const T*, const T*, const T*, const T*, const T*,    \
                                            const T*, T*, cudaStream_t);                         \
  template cudaError_t launch_adj_owner<T>(const Geom&, const Block*, int, int, int, int,        \
                                           const int32_t*, int64_t, const T*, const T*,        \
                                           const T*, const T*, const T*, const T*, const T*,   \
                                           const T*, T*, T*, T*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace enkfmc
