// Step (b) assembly and step (c) right-hand side / write-back.
//
// A_k = T_k^T D_k^-1 T_k + H_k^T R_k^-1 H_k (Eq. 8, Eq. 11) on every
// (sub-domain, variable) block of the extended set.  Neighbours share the
// variable, so A_k is block diagonal over variables.  In local order
// loc = (k * ey + yy) * ex + xx a row of T and its predecessors span at most
// hb positions, so A is banded with half-bandwidth hb and is stored as a
// column-major lower band: band[c * (hb + 1) + d] = A[c + d][c].
//
// A[a][b] = sum_j T[j][a] T[j][b] / D[j]: the rows j that contain component c
// are c itself and c - offset(s) for every stencil slot s.  One warp builds
// column c: for each such row j (in slot order, so the sum order is fixed and
// the result deterministic) its lanes add T[j][c] T[j][b] / D[j] for every
// entry b >= c of the row into a shared column buffer.  Rows of the tile
// interior read the global T; boundary rows read the re-estimated rows.
#include "enkfmc_internal.h"

namespace enkfmc {

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_assemble(const Geom g, const Block* __restrict__ blocks,
                                                  const T* __restrict__ Tg, const T* __restrict__ Dg,
                                                  const T* __restrict__ Te, const T* __restrict__ De,
                                                  const int32_t* __restrict__ obs_of,
                                                  const T* __restrict__ R, T* __restrict__ band,
                                                  int32_t* status, int hbp1_max) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  T* col = reinterpret_cast<T*>(smem) + (size_t)warp * hbp1_max;
  const Block b = blocks[blockIdx.y];
  const int c = blockIdx.x * wpc + warp;
  if (c >= b.nb) return;
  const int hb = b.hb, pmax = g.pmax, nlon = g.nlon;
  for (int d = lane; d <= hb; d += 32) col[d] = T(0);
  __syncwarp();
  const int plane = b.ey * b.ex;
  const int kc = c / plane;
  const int yyc = (c - kc * plane) / b.ex;
  const int xxc = c - kc * plane - yyc * b.ex;
  const int yc = b.lat_lo + yyc;
  const int xc = imod(b.lon_lo + xxc, nlon);
  const int v = b.var;

  for (int sj = -1; sj < pmax; ++sj) {
    int kj = kc, yj = yc, xj = xc, yyj = yyc, xxj = xxc;
    if (sj >= 0) {
      int dk, dy, dx;
      slot_offset(sj, g.r, g.vr, dk, dy, dx);
      kj = kc - dk;
      yj = yc - dy;
      xj = xc - dx;
      if (kj >= b.nlev_b || yj < 0 || yj >= g.nlat) continue;
      if (xj < 0 || xj >= nlon) {
        if (!g.periodic) continue;
        xj = imod(xj, nlon);
      }
      if (!in_ext(b, nlon, yj, xj, yyj, xxj)) continue;
    }
    const int locj = (kj * b.ey + yyj) * b.ex + xxj;
    const T* trow;
    T Dj;
    if (in_interior(b, yj, xj)) {
      const int64_t lj = coords_label(g, v, kj, yj, xj);
      trow = Tg + lj * pmax;
      Dj = Dg[lj];
    } else {
      trow = Te + (b.row_off + locj) * pmax;
      Dj = De[b.row_off + locj];
    }
    const T tjc = (sj < 0) ? T(1) : trow[sj];
    if (tjc == T(0)) continue;
    const T scale = tjc / Dj;
    if (lane == 0) {
      const int d = locj - c;
      if (d >= 0) {
        if (d <= hb) col[d] += scale;
        else record_error(status, ENKFMC_EINVAL, (int64_t)blockIdx.y);
      }
    }
    for (int s2 = lane; s2 < pmax; s2 += 32) {
      const T tjb = trow[s2];
      if (tjb == T(0)) continue;
      int kq, yq, xq, yyq, xxq;
      if (!slot_pred(g, kj, yj, xj, s2, kq, yq, xq) || !in_ext(b, nlon, yq, xq, yyq, xxq)) {
        record_error(status, ENKFMC_EINVAL, (int64_t)blockIdx.y);
        continue;
      }
      const int d = (kq * b.ey + yyq) * b.ex + xxq - c;
      if (d >= 0) {
        if (d <= hb) col[d] += scale * tjb;
        else record_error(status, ENKFMC_EINVAL, (int64_t)blockIdx.y);
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    const int o = obs_of[coords_label(g, v, kc, yc, xc)];
    if (o >= 0) col[0] += T(1) / R[o];
  }
  __syncwarp();
  T* out = band + b.band_off + (int64_t)c * (hb + 1);
  for (int d = lane; d <= hb; d += 32) out[d] = (c + d < b.nb) ? col[d] : T(0);
}

// Band entries A[c + d][c] for a tile of kCols columns from the slot pairs of
// each diagonal d.  The rows j = c - o(s2) that can touch the tile (local
// indices [c0 - r, c0 + kCols + hb]) are staged in shared memory with their D,
// and so is the block shape's pair list; each thread then builds entries with
// d fastest (contiguous stores), summing its pairs in a fixed order
// (deterministic results).
constexpr int kCols = 32;

template <typename T>
__global__ void __launch_bounds__(256) k_assemble_pairs(
    const Geom g, const Block* __restrict__ blocks, const int2* __restrict__ pairs,
    const int32_t* __restrict__ dptr, const T* __restrict__ Tg, const T* __restrict__ Dg,
    const T* __restrict__ Te, const T* __restrict__ De, const int32_t* __restrict__ obs_of,
    const T* __restrict__ R, T* __restrict__ band, int stage_rows, int npair_max) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Block b = blocks[blockIdx.y];
  const int c0 = blockIdx.x * kCols;
  if (c0 >= b.nb) return;
  const int pmax = g.pmax, ldt = pmax + 1;  // staged row: pmax coefficients then 1/D
  const int ns = pmax + 1;                   // slots plus the row itself
  T* Ts = reinterpret_cast<T*>(smem);                         // [stage_rows][ldt]
  const size_t ts_bytes = (sizeof(T) * (size_t)stage_rows * ldt + 15) / 16 * 16;
  int4* Ps = reinterpret_cast<int4*>(smem + ts_bytes);        // [npair_max], 16-byte aligned
  int2* Dl = reinterpret_cast<int2*>(Ps + npair_max);         // non-empty diagonals: [start, end)
  int* Dd = reinterpret_cast<int*>(Dl + (g.pmax + 1) * (g.pmax + 2) / 2 + 1);  // their d
  unsigned char* Vm = reinterpret_cast<unsigned char*>(Dd + (g.pmax + 1) * (g.pmax + 2) / 2 + 1);
  __shared__ int n_nz;
  const int hp1 = b.hb + 1;
  const int jlo = c0 - g.r;
  const int nrow = min(stage_rows, kCols + hp1 + g.r);
  const int plane = b.ey * b.ex;
  const int ncol = min(kCols, b.nb - c0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // zero the tile's band columns (non-empty diagonals are overwritten below)
  for (int e = threadIdx.x; e < ncol * hp1; e += blockDim.x) band[b.band_off + (int64_t)c0 * hp1 + e] = T(0);
  // stage rows j in [jlo, jlo + nrow): one warp per row, lanes over its slots
  for (int jj = warp; jj < nrow; jj += nw) {
    const int j = jlo + jj;
    T* dst = Ts + jj * ldt;
    if (j < 0 || j >= b.nb) {
      for (int s = lane; s < ldt; s += 32) dst[s] = T(0);
      continue;
    }
    const int kj = j / plane, yyj = (j - kj * plane) / b.ex, xxj = j - kj * plane - yyj * b.ex;
    const int yj = b.lat_lo + yyj, xj = imod(b.lon_lo + xxj, g.nlon);
    const bool in = in_interior(b, yj, xj);
    const int64_t rsrc = in ? coords_label(g, b.var, kj, yj, xj) : b.row_off + j;
    const T* src = (in ? Tg : Te) + rsrc * pmax;
    for (int s = lane; s < pmax; s += 32) dst[s] = src[s];
    if (lane == 0) dst[pmax] = T(1) / (in ? Dg[rsrc] : De[rsrc]);
  }
  // pair list with each pair's local row offset; compact list of non-empty diagonals
  const int np = dptr[b.dptr_base + b.hb + 1];
  for (int q = threadIdx.x; q < np; q += blockDim.x) {
    const int2 pr = pairs[b.pair_base + q];
    const int dk = (signed char)(pr.y & 0xff);
    const int dy = (signed char)((pr.y >> 8) & 0xff);
    const int dx = (signed char)((pr.y >> 16) & 0xff);
    Ps[q] = make_int4(pr.x, pr.y, (dk * b.ey + dy) * b.ex + dx, 0);
  }
  if (threadIdx.x == 0) {
    int cnt = 0;
    for (int d = 0; d < hp1; ++d) {
      const int a = dptr[b.dptr_base + d], e = dptr[b.dptr_base + d + 1];
      if (e > a) {
        Dl[cnt] = make_int2(a, e);
        Dd[cnt] = d;
        ++cnt;
      }
    }
    n_nz = cnt;
  }
  // validity of each slot (row j = c - offset(s) inside the box) per column
  for (int idx = threadIdx.x; idx < ncol * ns; idx += blockDim.x) {
    const int cc = idx / ns, s = idx - cc * ns;
    const int c = c0 + cc;
    const int kc = c / plane, yyc = (c - kc * plane) / b.ex, xxc = c - kc * plane - yyc * b.ex;
    int dk = 0, dy = 0, dx = 0;
    if (s < pmax) slot_offset(s, g.r, g.vr, dk, dy, dx);
    const int kj = kc - dk, yyj = yyc - dy, xxj = xxc - dx;
    Vm[cc * ns + s] = (kj >= 0 && kj < b.nlev_b && yyj >= 0 && yyj < b.ey && xxj >= 0 && xxj < b.ex);
  }
  __syncthreads();
  // entries of the non-empty diagonals: threads over (diagonal, column)
  const int nz = n_nz;
  for (int e = threadIdx.x; e < nz * ncol; e += blockDim.x) {
    const int zi = e % nz, cc = e / nz;
    const int d = Dd[zi];
    const int c = c0 + cc;
    if (c + d >= b.nb) continue;
    const unsigned char* vm = Vm + cc * ns;
    T sum = T(0);
    const int2 rg = Dl[zi];
    for (int q = rg.x; q < rg.y; ++q) {
      const int4 pr = Ps[q];
      const int s1 = pr.x & 0xffff, s2 = pr.x >> 16;
      if (!vm[s2]) continue;
      const T* tr = Ts + (c - pr.z - jlo) * ldt;
      const T t1 = s1 == pmax ? T(1) : tr[s1];
      const T t2 = s2 == pmax ? T(1) : tr[s2];
      sum += (t1 * tr[pmax]) * t2;
    }
    if (d == 0) {
      const int kc = c / plane, yyc = (c - kc * plane) / b.ex, xxc = c - kc * plane - yyc * b.ex;
      const int o = obs_of[coords_label(g, b.var, kc, b.lat_lo + yyc, imod(b.lon_lo + xxc, g.nlon))];
      if (o >= 0) sum += T(1) / R[o];
    }
    band[b.band_off + (int64_t)c * hp1 + d] = sum;
  }
}

// rhs[blk][m][loc] = (y_o + sqrt(R_o) Z[m][o] - Xb[m][l]) / R_o when component
// l = label(loc) is observed by o, else 0 (Eq. 11 right-hand side).
template <typename T>
__global__ void __launch_bounds__(128) k_rhs(const Geom g, const Block* __restrict__ blocks,
                                             const int32_t* __restrict__ obs_of, int64_t mobs,
                                             const T* __restrict__ Xb, const T* __restrict__ y,
                                             const T* __restrict__ R, const T* __restrict__ Z,
                                             T* __restrict__ rhs) {
  const Block b = blocks[blockIdx.y];
  const int loc = blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= b.nb) return;
  const int plane = b.ey * b.ex;
  const int k = loc / plane;
  const int yy = (loc - k * plane) / b.ex;
  const int xx = loc - k * plane - yy * b.ex;
  const int64_t l = coords_label(g, b.var, k, b.lat_lo + yy, imod(b.lon_lo + xx, g.nlon));
  const int o = obs_of[l];
  T* out = rhs + b.row_off * g.N + loc;
  if (o < 0) {
    for (int m = 0; m < g.N; ++m) out[(int64_t)m * b.nb] = T(0);
    return;
  }
  const T Ro = R[o], yo = y[o];
  const T sq = sqrt(Ro), rinv = T(1) / Ro;
  for (int m = 0; m < g.N; ++m)
    out[(int64_t)m * b.nb] = rhs_entry(yo, sq, Z[(int64_t)m * mobs + o], Xb[(int64_t)m * g.n + l],
                                       rinv);
}

// Xa[m][l] = Xb[m][l] + dX[blk][m][loc] for the sub-domain whose interior
// holds l (Eq. 10; interiors are disjoint, so plain stores suffice).
template <typename T>
__global__ void __launch_bounds__(256) k_writeback(const Geom g, const Block* __restrict__ blocks,
                                                   int nsubx, int sub_lon, int sub_lat,
                                                   const T* __restrict__ Xb,
                                                   const T* __restrict__ dX,
                                                   const T* __restrict__ dX2, T* __restrict__ Xa) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= g.n) return;
  const int m = blockIdx.y;
  int v, k, y, x;
  label_coords(g, l, v, k, y, x);
  const int sub = (y / sub_lat) * nsubx + x / sub_lon;
  const Block& b = blocks[sub * g.nvar + v];
  const int loc = (k * b.ey + (y - b.lat_lo)) * b.ex + imod(x - b.lon_lo, g.nlon);
  const int64_t i = (int64_t)m * g.n + l;
  const int64_t e = b.row_off * g.N + (int64_t)m * b.nb + loc;
  Xa[i] = dX2 ? Xb[i] + (dX[e] + dX2[e]) : Xb[i] + dX[e];
}

}  // namespace

template <typename T>
cudaError_t launch_assemble(const Geom& g, const Block* blocks, int nblock, int nb_max,
                            const T* Tg, const T* Dg, const T* Te, const T* De,
                            const int32_t* obs_of, const T* R, T* band, int32_t* status,
                            cudaStream_t s, int hb_max) {
  const int wpc = 8;
  const int hbp1 = hb_max + 1;
  const size_t smem = sizeof(T) * (size_t)hbp1 * wpc;
  cudaError_t e = cudaFuncSetAttribute(k_assemble<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((nb_max + wpc - 1) / wpc, nblock);
  k_assemble<T><<<grid, 32 * wpc, smem, s>>>(g, blocks, Tg, Dg, Te, De, obs_of, R, band, status,
                                             hbp1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_assemble_pairs(const Geom& g, const Block* blocks, int nblock, int nb_max,
                                  int hb_max, int npair_max, const int2* pairs,
                                  const int32_t* dptr, const T* Tg, const T* Dg, const T* Te,
                                  const T* De, const int32_t* obs_of, const T* R, T* band,
                                  cudaStream_t s) {
  const int stage_rows = kCols + hb_max + 1 + g.r;
  const size_t nd = (size_t)(g.pmax + 1) * (g.pmax + 2) / 2 + 1;  // bound on non-empty diagonals
  const size_t smem = (sizeof(T) * (size_t)stage_rows * (g.pmax + 1) + 15) / 16 * 16 +
                      sizeof(int4) * (size_t)npair_max + nd * (sizeof(int2) + sizeof(int)) +
                      (size_t)kCols * (g.pmax + 1);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_assemble_pairs<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((nb_max + kCols - 1) / kCols, nblock);
  k_assemble_pairs<T><<<grid, 256, smem, s>>>(g, blocks, pairs, dptr, Tg, Dg, Te, De, obs_of, R,
                                              band, stage_rows, npair_max);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rhs(const Geom& g, const Block* blocks, int nblock, int nb_max,
                       const int32_t* obs_of, int64_t m, const T* Xb, const T* y, const T* R,
                       const T* Z, T* rhs, cudaStream_t s) {
  const dim3 grid((nb_max + 127) / 128, nblock);
  k_rhs<T><<<grid, 128, 0, s>>>(g, blocks, obs_of, m, Xb, y, R, Z, rhs);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_writeback(const Geom& g, const Block* blocks, int nsubx, int sub_lon,
                             int sub_lat, const T* Xb, const T* dX, const T* dX2, T* Xa,
                             cudaStream_t s) {
  const dim3 grid((unsigned)((g.n + 255) / 256), g.N);
  k_writeback<T><<<grid, 256, 0, s>>>(g, blocks, nsubx, sub_lon, sub_lat, Xb, dX, dX2, Xa);
  return cudaGetLastError();
}

#define INST(T)                                                                                  \
  template cudaError_t launch_assemble_pairs<T>(const Geom&, const Block*, int, int, int, int,  \
                                                const int2*, const int32_t*, const T*, const T*,  \
                                                const T*, const T*, const int32_t*, const T*, T*, \
                                                cudaStream_t);                                     \
  template cudaError_t launch_assemble<T>(const Geom&, const Block*, int, int, const T*,        \
                                          const T*, const T*, const T*, const int32_t*,         \
                                          const T*, T*, int32_t*, cudaStream_t, int);           \
  template cudaError_t launch_rhs<T>(const Geom&, const Block*, int, int, const int32_t*,       \
                                     int64_t, const T*, const T*, const T*, const T*, T*,       \
                                     cudaStream_t);                                              \
  template cudaError_t launch_writeback<T>(const Geom&, const Block*, int, int, int, const T*,  \
                                           const T*, const T*, T*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace enkfmc
