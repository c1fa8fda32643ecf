// One step of iterative refinement of the sub-domain solves (Eq. 11) in the
// single-precision path: r = rhs - A dX with A = T^T D^-1 T + H^T R^-1 H applied
// in its factored form, every product and sum carried as a double-float pair
// (FMA two-product, two-sum), so that the residual is exact to about 2^-44
// relative to the terms; the correction A c = r is then solved with the same
// single-precision factor and Xa = Xb + dX + c.
//
// Pass 1 (k_whiten): v_j = (T dX)_j / D_j for every extended row j, member m.
// Pass 2 (k_residual): r_a = rhs_a - dX_a / R_a - sum_{j: a in row j} T[j][a] v_j,
// gathering the rows j = a - offset(s) that hold a in slot s.
#include "enkfmc_internal.h"

namespace enkfmc {

namespace {

struct ff {
  float hi, lo;
};

// s + t*x exactly up to the low-order accumulation: (s, c) += t * x
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

__global__ void __launch_bounds__(128) k_whiten(const Geom g, const Block* __restrict__ blocks,
                                                const float* __restrict__ Tg,
                                                const float* __restrict__ Dg,
                                                const float* __restrict__ Te,
                                                const float* __restrict__ De,
                                                const float* __restrict__ dX,
                                                float* __restrict__ vhi, float* __restrict__ vlo) {
  const Block b = blocks[blockIdx.y];
  const int loc = blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= b.nb) return;
  const int m = blockIdx.z;
  const int plane = b.ey * b.ex;
  const int k = loc / plane;
  const int yy = (loc - k * plane) / b.ex;
  const int xx = loc - k * plane - yy * b.ex;
  const int y = b.lat_lo + yy, x = imod(b.lon_lo + xx, g.nlon);
  float Dj;
  const float* trow = row_of(g, b, b.var, k, y, x, loc, Tg, Dg, Te, De, Dj);
  const float* dXm = dX + b.row_off * g.N + (int64_t)m * b.nb;
  float s = dXm[loc], c = 0.f;
  for (int sl = 0; sl < g.pmax; ++sl) {
    const float t = trow[sl];
    if (t == 0.f) continue;
    int kq, yq, xq, yyq, xxq;
    if (!slot_pred(g, k, y, x, sl, kq, yq, xq) || !in_ext(b, g.nlon, yq, xq, yyq, xxq)) continue;
    ff_add_prod(s, c, t, dXm[(kq * b.ey + yyq) * b.ex + xxq]);
  }
  // (s + c) / Dj as a pair
  const float hi = s + c;
  const float lo = c - (hi - s);
  const float qh = hi / Dj;
  const float rem = fmaf(-qh, Dj, hi) + lo;
  const int64_t o = b.row_off * g.N + (int64_t)m * b.nb + loc;
  vhi[o] = qh;
  vlo[o] = rem / Dj;
}

__global__ void __launch_bounds__(128) k_residual(
    const Geom g, const Block* __restrict__ blocks, const int32_t* __restrict__ obs_of,
    int64_t mobs, const float* __restrict__ Xb, const float* __restrict__ y,
    const float* __restrict__ R, const float* __restrict__ Z, const float* __restrict__ Tg,
    const float* __restrict__ Dg, const float* __restrict__ Te, const float* __restrict__ De,
    const float* __restrict__ dX, const float* __restrict__ vhi, const float* __restrict__ vlo,
    float* __restrict__ res) {
  const Block b = blocks[blockIdx.y];
  const int loc = blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= b.nb) return;
  const int m = blockIdx.z;
  const int plane = b.ey * b.ex;
  const int kc = loc / plane;
  const int yyc = (loc - kc * plane) / b.ex;
  const int xxc = loc - kc * plane - yyc * b.ex;
  const int yc = b.lat_lo + yyc, xc = imod(b.lon_lo + xxc, g.nlon);
  const int v = b.var;
  const int64_t base = b.row_off * g.N + (int64_t)m * b.nb;
  float s = 0.f, c = 0.f;
  const int64_t l = coords_label(g, v, kc, yc, xc);
  const int o = obs_of[l];
  if (o >= 0) {
    const float Ro = R[o];
    const float rinv = 1.f / Ro;
    s = rhs_entry(y[o], sqrtf(Ro), Z[(int64_t)m * mobs + o], Xb[(int64_t)m * g.n + l], rinv);
    ff_add_prod(s, c, -dX[base + loc], rinv);
  }
  // j = a itself (T[a][a] = 1)
  ff_add(s, c, -vhi[base + loc]);
  c -= vlo[base + loc];
  for (int sj = 0; sj < g.pmax; ++sj) {
    int dk, dy, dx;
    slot_offset(sj, g.r, g.vr, dk, dy, dx);
    const int kj = kc - dk, yj = yc - dy;
    int xj = xc - dx;
    if (kj >= b.nlev_b || yj < 0 || yj >= g.nlat) continue;
    if (xj < 0 || xj >= g.nlon) {
      if (!g.periodic) continue;
      xj = imod(xj, g.nlon);
    }
    int yyj, xxj;
    if (!in_ext(b, g.nlon, yj, xj, yyj, xxj)) continue;
    const int locj = (kj * b.ey + yyj) * b.ex + xxj;
    float Dj;
    const float* trow = row_of(g, b, v, kj, yj, xj, locj, Tg, Dg, Te, De, Dj);
    const float t = trow[sj];
    if (t == 0.f) continue;
    ff_add_prod(s, c, -t, vhi[base + locj]);
    c -= t * vlo[base + locj];
  }
  res[base + loc] = s + c;
}

}  // namespace

cudaError_t launch_refine_residual(const Geom& g, const Block* blocks, int nblock, int nb_max,
                                   const int32_t* obs_of, int64_t m, const float* Xb,
                                   const float* y, const float* R, const float* Z,
                                   const float* Tg, const float* Dg, const float* Te,
                                   const float* De, const float* dX, float* vhi, float* vlo,
                                   float* res, cudaStream_t s) {
  const dim3 grid((nb_max + 127) / 128, nblock, g.N);
  k_whiten<<<grid, 128, 0, s>>>(g, blocks, Tg, Dg, Te, De, dX, vhi, vlo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_residual<<<grid, 128, 0, s>>>(g, blocks, obs_of, m, Xb, y, R, Z, Tg, Dg, Te, De, dX, vhi,
                                  vlo, res);
  return cudaGetLastError();
}

}  // namespace enkfmc
