// Iterative refinement of the sub-domain solves (Eq. 11) in the
// single-precision path: r = rhs - A dX with A = T^T D^-1 T + H^T R^-1 H applied
// in its factored form, every product and sum carried as a double-float pair
// (FMA two-product, two-sum), so that the residual is exact to about 2^-44
// relative to the terms; the correction A c = r is then solved with the same
// single-precision factor.  Each step but the last adds c into dX
// (k_accumulate); after the last, Xa = Xb + dX + c.  The right-hand side is
// Eq. 11's H^T R^-1 (Y^s - H X^b), formed here from the observations, or a
// given array (the reverse pass refines Lambda = A^-1 W the same way).
//
// Pass 1 (k_whiten): v_j = (T dX)_j / D_j for every extended row j, member m.
// Pass 2 (k_residual): r_a = rhs_a - dX_a / R_a - sum_{j: a in row j} T[j][a] v_j,
// gathering the rows j = a - offset(s) that hold a in slot s.
//
// A thread block takes 32 consecutive rows of one block; the slot geometry
// (neighbour positions and coefficients) is resolved once into shared memory,
// then each warp sweeps its share of the members with one row per lane, so the
// inner loops read only shared memory and coalesced rows of dX / v.
#include "enkfmc_internal.h"

namespace enkfmc {

namespace {

constexpr int kRows = 32;
constexpr int kWarps = 4;
constexpr int kMB = 5;  // members per pass (they share the slot reads)

__device__ __forceinline__ void ff_add_prod(float& s, float& c, float t, float x) {
  const float prod = t * x;
  const float perr = fmaf(t, x, -prod);
  const float u = s + prod;
  const float z = u - s;
  const float e = (s - (u - z)) + (prod - z);
  s = u;
  c += e + perr;
}

__device__ __forceinline__ void ff_add(float& s, float& c, float x) {
  const float u = s + x;
  const float z = u - s;
  c += (s - (u - z)) + (x - z);
  s = u;
}

__device__ __forceinline__ void row_coords(const Block& b, int nlon, int loc, int& k, int& yy,
                                           int& xx, int& y, int& x) {
  const int plane = b.ey * b.ex;
  k = loc / plane;
  yy = (loc - k * plane) / b.ex;
  xx = loc - k * plane - yy * b.ex;
  y = b.lat_lo + yy;
  x = imod(b.lon_lo + xx, nlon);
}

// Row j of the block's T and its D (global row inside the tile interior,
// re-estimated boundary row otherwise).
__device__ __forceinline__ const float* row_of(const Geom& g, const Block& b, int v, int kj,
                                               int yj, int xj, int locj, const float* Tg,
                                               const float* Dg, const float* Te, const float* De,
                                               float& Dj) {
  if (in_interior(b, yj, xj)) {
    const int64_t lj = coords_label(g, v, kj, yj, xj);
    Dj = Dg[lj];
    return Tg + lj * g.pmax;
  }
  Dj = De[b.row_off + locj];
  return Te + (b.row_off + locj) * g.pmax;
}

__global__ void __launch_bounds__(kRows* kWarps) k_whiten(
    const Geom g, const Block* __restrict__ blocks, const float* __restrict__ Tg,
    const float* __restrict__ Dg, const float* __restrict__ Te, const float* __restrict__ De,
    const float* __restrict__ dX, float* __restrict__ vhi, float* __restrict__ vlo) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int pmax = g.pmax;
  int* nbr = reinterpret_cast<int*>(smem);              // [kRows][pmax] local index or -1
  float* tv = reinterpret_cast<float*>(nbr + kRows * pmax);  // [kRows][pmax]
  float* dj = tv + kRows * pmax;                        // [kRows]
  signed char* so = reinterpret_cast<signed char*>(dj + kRows);  // [3][pmax] slot offsets
  const Block b = blocks[blockIdx.y];
  const int loc0 = blockIdx.x * kRows;
  if (loc0 >= b.nb) return;
  const int nr = min(kRows, b.nb - loc0);
  for (int s = threadIdx.x; s < pmax; s += blockDim.x) {
    int dk, dy, dx;
    slot_offset(s, g.r, g.vr, dk, dy, dx);
    so[s] = (signed char)dk;
    so[pmax + s] = (signed char)dy;
    so[2 * pmax + s] = (signed char)dx;
  }
  __syncthreads();
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < nr; i += kWarps) {  // a row per warp, its slots over the lanes
      int k, yy, xx, y, x;
      row_coords(b, g.nlon, loc0 + i, k, yy, xx, y, x);
      float Dj;
      const float* trow = row_of(g, b, b.var, k, y, x, loc0 + i, Tg, Dg, Te, De, Dj);
      for (int s = lane; s < pmax; s += 32) {
        const float t = trow[s];
        int kq, yq, xq, yyq, xxq, q = -1;
        if (t != 0.f && slot_pred_off(g, k, y, x, so[s], so[pmax + s], so[2 * pmax + s], kq, yq,
                                      xq) &&
            in_ext(b, g.nlon, yq, xq, yyq, xxq))
          q = (kq * b.ey + yyq) * b.ex + xxq;
        nbr[i * pmax + s] = q;
        tv[i * pmax + s] = q >= 0 ? t : 0.f;
      }
      if (lane == 0) dj[i] = Dj;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane >= nr) return;
  const int* nb_i = nbr + lane * pmax;
  const float* t_i = tv + lane * pmax;
  const float Dj = dj[lane];
  const float invDj = 1.f / Dj;
  // kMB members per pass share the slot reads; members past N are skipped
  for (int m0 = kMB * warp; m0 < g.N; m0 += kMB * kWarps) {
    const float* dXm[kMB];
    float s[kMB], c[kMB];
#pragma unroll
    for (int u = 0; u < kMB; ++u) {
      const int m = min(m0 + u, g.N - 1);
      dXm[u] = dX + b.row_off * g.N + (int64_t)m * b.nb;
      s[u] = dXm[u][loc0 + lane];
      c[u] = 0.f;
    }
    for (int sl = 0; sl < pmax; ++sl) {
      const int q = nb_i[sl];
      if (q >= 0) {
        const float t = t_i[sl];
#pragma unroll
        for (int u = 0; u < kMB; ++u) ff_add_prod(s[u], c[u], t, dXm[u][q]);
      }
    }
#pragma unroll
    for (int u = 0; u < kMB; ++u) {
      if (m0 + u >= g.N) break;
      const float hi = s[u] + c[u];
      const float lo = c[u] - (hi - s[u]);
      // qh ~ hi / D_j; the remainder hi + lo - qh D_j is formed exactly by the
      // FMA, so qh + rem / D_j carries the quotient to double-float accuracy
      const float qh = hi * invDj;
      const float rem = fmaf(-qh, Dj, hi) + lo;
      const int64_t o = b.row_off * g.N + (int64_t)(m0 + u) * b.nb + loc0 + lane;
      vhi[o] = qh;
      vlo[o] = rem * invDj;
    }
  }
}

__global__ void __launch_bounds__(kRows* kWarps) k_residual(
    const Geom g, const Block* __restrict__ blocks, const int32_t* __restrict__ obs_of,
    int64_t mobs, const float* __restrict__ Xb, const float* __restrict__ y,
    const float* __restrict__ R, const float* __restrict__ Z, const float* __restrict__ Tg,
    const float* __restrict__ Dg, const float* __restrict__ Te, const float* __restrict__ De,
    const float* __restrict__ dX, const float* __restrict__ vhi, const float* __restrict__ vlo,
    const float* __restrict__ rhs_in, float* __restrict__ res) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int pmax = g.pmax;
  int* cand = reinterpret_cast<int*>(smem);                  // [kRows][pmax] row j or -1
  float* ct = reinterpret_cast<float*>(cand + kRows * pmax);  // [kRows][pmax] T[j][s]
  int* obs = reinterpret_cast<int*>(ct + kRows * pmax);      // [kRows]
  int64_t* lab = reinterpret_cast<int64_t*>(obs + kRows + (kRows & 1));  // [kRows]
  signed char* so = reinterpret_cast<signed char*>(lab + kRows);  // [3][pmax] slot offsets
  const Block b = blocks[blockIdx.y];
  const int loc0 = blockIdx.x * kRows;
  if (loc0 >= b.nb) return;
  const int nr = min(kRows, b.nb - loc0);
  const int v = b.var;
  for (int s = threadIdx.x; s < pmax; s += blockDim.x) {
    int dk, dy, dx;
    slot_offset(s, g.r, g.vr, dk, dy, dx);
    so[s] = (signed char)dk;
    so[pmax + s] = (signed char)dy;
    so[2 * pmax + s] = (signed char)dx;
  }
  __syncthreads();
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < nr; i += kWarps) {  // a row per warp, its slots over the lanes
      int kc, yyc, xxc, yc, xc;
      row_coords(b, g.nlon, loc0 + i, kc, yyc, xxc, yc, xc);
      if (lane == 0) {
        const int64_t l = coords_label(g, v, kc, yc, xc);
        lab[i] = l;
        obs[i] = obs_of[l];
      }
      for (int sj = lane; sj < pmax; sj += 32) {
        // row j = c - offset(sj) holds c in its slot sj
        const int kj = kc - so[sj], yj = yc - so[pmax + sj];
        int xj = xc - so[2 * pmax + sj], jloc = -1;
        float t = 0.f;
        bool ok = kj < b.nlev_b && yj >= 0 && yj < g.nlat;
        if (ok && (xj < 0 || xj >= g.nlon)) {
          if (g.periodic) xj = imod(xj, g.nlon);
          else ok = false;
        }
        int yyj, xxj;
        if (ok && in_ext(b, g.nlon, yj, xj, yyj, xxj)) {
          const int locj = (kj * b.ey + yyj) * b.ex + xxj;
          float Dj;
          t = row_of(g, b, v, kj, yj, xj, locj, Tg, Dg, Te, De, Dj)[sj];
          if (t != 0.f) jloc = locj;
        }
        cand[i * pmax + sj] = jloc;
        ct[i * pmax + sj] = jloc >= 0 ? t : 0.f;
      }
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane >= nr) return;
  const int* cj = cand + lane * pmax;
  const float* tj = ct + lane * pmax;
  const int o = obs[lane];
  const int64_t l = lab[lane];
  float Ro = 1.f, yo = 0.f, sq = 0.f, rinv = 0.f;
  if (o >= 0) {
    Ro = R[o];
    yo = y[o];
    sq = sqrtf(Ro);
    rinv = 1.f / Ro;
  }
  const int a = loc0 + lane;
  // kMB members per pass share the slot reads; members past N are skipped
  for (int m0 = kMB * warp; m0 < g.N; m0 += kMB * kWarps) {
    int64_t base[kMB];
    float s[kMB], c[kMB];
#pragma unroll
    for (int u = 0; u < kMB; ++u) {
      const int m = min(m0 + u, g.N - 1);
      base[u] = b.row_off * g.N + (int64_t)m * b.nb;
      s[u] = rhs_in ? rhs_in[base[u] + a] : 0.f;
      c[u] = 0.f;
      if (o >= 0) {
        if (!rhs_in)
          s[u] = rhs_entry(yo, sq, Z[(int64_t)m * mobs + o], Xb[(int64_t)m * g.n + l], rinv);
        ff_add_prod(s[u], c[u], -dX[base[u] + a], rinv);
      }
      ff_add(s[u], c[u], -vhi[base[u] + a]);
      c[u] -= vlo[base[u] + a];
    }
    for (int sj = 0; sj < pmax; ++sj) {
      const int j = cj[sj];
      if (j < 0) continue;
      const float t = tj[sj];
#pragma unroll
      for (int u = 0; u < kMB; ++u) {
        ff_add_prod(s[u], c[u], -t, vhi[base[u] + j]);
        c[u] -= t * vlo[base[u] + j];
      }
    }
#pragma unroll
    for (int u = 0; u < kMB; ++u)
      if (m0 + u < g.N) res[base[u] + a] = s[u] + c[u];
  }
}

__global__ void __launch_bounds__(256) k_accumulate(float* __restrict__ y,
                                                    const float* __restrict__ x, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}

}  // namespace

cudaError_t launch_accumulate(float* y, const float* x, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  int64_t grid = (count + 255) / 256;
  if (grid > 152 * 16) grid = 152 * 16;
  k_accumulate<<<(unsigned)grid, 256, 0, s>>>(y, x, count);
  return cudaGetLastError();
}

cudaError_t launch_refine_residual(const Geom& g, const Block* blocks, int nblock, int nb_max,
                                   const int32_t* obs_of, int64_t m, const float* Xb,
                                   const float* y, const float* R, const float* Z,
                                   const float* Tg, const float* Dg, const float* Te,
                                   const float* De, const float* dX, float* vhi, float* vlo,
                                   const float* rhs_in, float* res, cudaStream_t s) {
  const dim3 grid((nb_max + kRows - 1) / kRows, nblock);
  const size_t sm1 = (size_t)kRows * g.pmax * 8 + kRows * 4 + 3 * g.pmax;
  const size_t sm2 = (size_t)kRows * g.pmax * 8 + kRows * 4 + 8 + kRows * 8 + 3 * g.pmax;
  k_whiten<<<grid, kRows * kWarps, sm1, s>>>(g, blocks, Tg, Dg, Te, De, dX, vhi, vlo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_residual<<<grid, kRows * kWarps, sm2, s>>>(g, blocks, obs_of, m, Xb, y, R, Z, Tg, Dg, Te, De,
                                               dX, vhi, vlo, rhs_in, res);
  return cudaGetLastError();
}

}  // namespace enkfmc
