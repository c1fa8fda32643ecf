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

// T: the type of T, D and R; TB: the band's type and the arithmetic (double
// for the blocks whose single-precision factorisation failed: their A is
// assembled again from the same single-precision T and D, in double).  rng
// (optional, device {lo, hi}): only the entries [lo, hi) of `blocks`.
template <typename T, typename TB>
__global__ void __launch_bounds__(256) k_assemble(const Geom g, const Block* __restrict__ blocks,
                                                  const T* __restrict__ Tg, const T* __restrict__ Dg,
                                                  const T* __restrict__ Te, const T* __restrict__ De,
                                                  const int32_t* __restrict__ obs_of,
                                                  const T* __restrict__ R, TB* __restrict__ band,
                                                  int32_t* status, int hbp1_max,
                                                  const int* __restrict__ rng) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  TB* col = reinterpret_cast<TB*>(smem) + (size_t)warp * hbp1_max;
  if (rng && ((int)blockIdx.y < rng[0] || (int)blockIdx.y >= rng[1])) return;
  const Block b = blocks[blockIdx.y];
  const int c = blockIdx.x * wpc + warp;
  if (c >= b.nb) return;
  const int hb = b.hb, pmax = g.pmax, nlon = g.nlon;
  for (int d = lane; d <= hb; d += 32) col[d] = TB(0);
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
    const TB tjc = (sj < 0) ? TB(1) : (TB)trow[sj];
    if (tjc == TB(0)) continue;
    const TB scale = tjc / (TB)Dj;
    if (lane == 0) {
      const int d = locj - c;
      if (d >= 0) {
        if (d <= hb) col[d] += scale;
        else record_error(status, ENKFMC_EINVAL, (int64_t)blockIdx.y);
      }
    }
    for (int s2 = lane; s2 < pmax; s2 += 32) {
      const TB tjb = (TB)trow[s2];
      if (tjb == TB(0)) continue;
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
    if (o >= 0) col[0] += TB(1) / (TB)R[o];
  }
  __syncwarp();
  TB* out = band + b.band_off + (int64_t)c * (hb + 1);
  for (int d = lane; d <= hb; d += 32) out[d] = (c + d < b.nb) ? col[d] : TB(0);
}

// Band assembly of tiles of 32 NH columns of one block from the pair list of
// its shape.  Records {s1, s2, o(s2), d} sorted by d: row j = c - o(s2) adds
// T[j][s1] T[j][s2] / D[j] to A[c + d][c] when row j lies in the block.
//  * A CTA walks consecutive tiles of one block; the rows a tile reads sit in
//    a ring in shared memory (source rows from the handle's per-row table):
//    pmax coefficients, 1 (the row's own unit entry, slot pmax), then 1/D[j];
//    odd row stride, so lanes on consecutive columns hit distinct banks.  Each
//    tile after the first stages only the rows it adds.
//  * Warps take about equal chunks of the pair list, each chunk moved to start
//    at a diagonal boundary, so every entry is summed by one warp in list
//    order (deterministic).  Lane l owns columns c0 + l + 32 h (h < NH): every
//    lane runs the same pairs, the pair record is a broadcast read and the slot
//    validity a bit of a per-column mask.  A warp stores its sums into the
//    shared output tile at each change of diagonal.
//  * The tile's band columns are contiguous in the band: one coalesced write,
//    zeros included, with 1/R on the diagonal of observed components.
constexpr int kAsmThreads = 512;

__host__ __device__ inline int asm_ldt(int pmax) { return (pmax + 2) | 1; }
__host__ __device__ inline int asm_ldo(int hb) { return (hb + 1) | 1; }
__host__ __device__ inline int asm_rows(int cols, int hb, int r) { return cols + hb + 1 + r; }

template <typename T, int NH>
__global__ void __launch_bounds__(kAsmThreads) k_assemble_pairs(
    const Geom g, const Block* __restrict__ blocks, const int4* __restrict__ pairs,
    const int32_t* __restrict__ srcrow, const T* __restrict__ Tg, const T* __restrict__ Dg,
    const T* __restrict__ Te, const T* __restrict__ De, const int32_t* __restrict__ obs_of,
    const T* __restrict__ R, T* __restrict__ band, int hb_max, int tiles_per_cta) {
  constexpr int kCols = 32 * NH;
  extern __shared__ __align__(16) unsigned char smem[];
  const Block b = blocks[blockIdx.y];
  const int ntiles = (b.nb + kCols - 1) / kCols;
  const int t0 = blockIdx.x * tiles_per_cta, t1 = min(ntiles, t0 + tiles_per_cta);
  if (t0 >= t1) return;
  const int pmax = g.pmax, ldt = asm_ldt(pmax);
  const int hp1 = b.hb + 1, ldo = asm_ldo(hb_max);
  const int nrow = asm_rows(kCols, b.hb, g.r);  // rows a tile reads: the ring's length
  const int plane = b.ey * b.ex;
  const int npair = b.npair;
  int4* Ps = reinterpret_cast<int4*>(smem);                           // [npair]
  T* Os = reinterpret_cast<T*>(Ps + npair);                           // [kCols][ldo]
  T* Ts = Os + (size_t)kCols * ldo;                                   // [nrow][ldt] ring
  // slot-validity bit masks by level, latitude and longitude position in the box
  uint64_t* Mk = reinterpret_cast<uint64_t*>(Ts + (size_t)nrow * ldt + 1);  // 8-byte aligned below
  Mk = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(Mk) + 7) & ~(uintptr_t)7);
  uint64_t* My = Mk + b.nlev_b;
  uint64_t* Mx = My + b.ey;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kAsmThreads / 32;

  for (int q = threadIdx.x; q < npair; q += kAsmThreads) Ps[q] = pairs[b.pair_base + q];
  for (int e = threadIdx.x; e < kCols * ldo; e += kAsmThreads) Os[e] = T(0);
  // bit s of Mk[k] / My[yy] / Mx[xx]: the row at offset s from that position
  // stays inside the box along that axis (bit pmax: the row itself); a warp per
  // position, lanes over the slots
  for (int e = warp; e < b.nlev_b + b.ey + b.ex; e += nw) {
    const int axis = e < b.nlev_b ? 0 : (e < b.nlev_b + b.ey ? 1 : 2);
    const int pos = e - (axis == 0 ? 0 : (axis == 1 ? b.nlev_b : b.nlev_b + b.ey));
    const int lim = axis == 0 ? b.nlev_b : (axis == 1 ? b.ey : b.ex);
    uint64_t m = (uint64_t)1 << pmax;
    for (int s0 = 0; s0 < pmax; s0 += 32) {
      const int sl = s0 + lane;
      bool in = false;
      if (sl < pmax) {
        int o3[3];
        slot_offset(sl, g.r, g.vr, o3[0], o3[1], o3[2]);
        const int q = pos - o3[axis];
        in = q >= 0 && q < lim;
      }
      m |= (uint64_t)__ballot_sync(0xffffffffu, in) << s0;
    }
    if (lane == 0) (axis == 0 ? Mk : (axis == 1 ? My : Mx))[pos] = m;
  }

  // The CTA walks tiles t0 .. t1 - 1; tile t reads rows [c0 - r, c0 - r + nrow)
  // (c0 = kCols t), kept in a ring: row j in slot (j - jbase) mod nrow.  The
  // first tile stages all its rows, each later one the kCols rows it adds.
  const int jbase = t0 * kCols - g.r;
  // stage rows [jfrom, jto): a warp per row, lanes over the slots (slot pmax
  // = 1, slot pmax + 1 = 1 / D[j]); the loads of kStage rows are issued
  // before any is stored
  auto stage = [&](int jfrom, int jto) {
    constexpr int kStage = 4, kSlotRounds = 3;  // ldt <= 96 (pmax <= 63 here)
    for (int j0 = jfrom + warp * kStage; j0 < jto; j0 += nw * kStage) {
      T v[kStage][kSlotRounds];
#pragma unroll
      for (int u = 0; u < kStage; ++u) {
        const int j = j0 + u;
        const int sr = (j < jto && j >= 0 && j < b.nb) ? srcrow[b.row_off + j] : INT32_MIN;
#pragma unroll
        for (int h = 0; h < kSlotRounds; ++h) {
          const int sl = lane + 32 * h;
          T x = T(0);
          if (sr != INT32_MIN) {
            if (sl < pmax)
              x = sr >= 0 ? Tg[(int64_t)sr * pmax + sl] : Te[(int64_t)(~sr) * pmax + sl];
            else if (sl == pmax) x = T(1);
            else if (sl == pmax + 1) x = T(1) / (sr >= 0 ? Dg[sr] : De[~sr]);
          }
          v[u][h] = x;
        }
      }
#pragma unroll
      for (int u = 0; u < kStage; ++u) {
        const int j = j0 + u;
        if (j >= jto) continue;
        T* dst = Ts + (size_t)((j - jbase) % nrow) * ldt;
#pragma unroll
        for (int h = 0; h < kSlotRounds; ++h) {
          const int sl = lane + 32 * h;
          if (sl < ldt) dst[sl] = v[u][h];
        }
      }
    }
  };
  const int per = (npair + nw - 1) / nw;
  auto at_diag_start = [&](int q) {  // first q' >= q that starts a diagonal
    if (q <= 0) return 0;
    while (q < npair && Ps[q].w == Ps[q - 1].w) ++q;
    return min(q, npair);
  };
  __syncthreads();
  const int q0 = at_diag_start(warp * per), q1 = at_diag_start((warp + 1) * per);

  for (int t = t0; t < t1; ++t) {
    const int c0 = t * kCols;
    const int ncol = min(kCols, b.nb - c0);
    const int jhi = c0 - g.r + nrow;
    stage(t == t0 ? c0 - g.r : jhi - kCols, jhi);
    __syncthreads();

    // this lane's columns and the slots whose row lies in the block (bit s)
    uint64_t vmask[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      const int cc = lane + 32 * h, c = c0 + cc;
      vmask[h] = 0;
      if (cc < ncol) {
        const int kc = c / plane, yyc = (c - kc * plane) / b.ex, xxc = c - kc * plane - yyc * b.ex;
        vmask[h] = Mk[kc] & My[yyc] & Mx[xxc];
      }
    }
    // row c - o(s2) of column c = c0 + lane + 32 h sits in slot rel - o(s2)
    // (mod nrow), rel = the slot of row c; o(s2) lies in (-nrow, r]
    int rel[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) rel[h] = (c0 + lane + 32 * h - jbase) % nrow;
    T sum[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) sum[h] = T(0);
    int dcur = q0 < q1 ? Ps[q0].w : 0;
    for (int q = q0; q < q1; ++q) {
      const int4 pr = Ps[q];
      if (pr.w != dcur) {
#pragma unroll
        for (int h = 0; h < NH; ++h) {
          Os[(lane + 32 * h) * ldo + dcur] = sum[h];
          sum[h] = T(0);
        }
        dcur = pr.w;
      }
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        if ((vmask[h] >> pr.y) & 1) {
          int sl = rel[h] - pr.z;
          sl += sl < 0 ? nrow : 0;
          sl -= sl >= nrow ? nrow : 0;
          const T* tr = Ts + (size_t)sl * ldt;
          sum[h] += (tr[pr.x] * tr[pmax + 1]) * tr[pr.y];
        }
      }
    }
    if (q0 < q1) {
#pragma unroll
      for (int h = 0; h < NH; ++h) Os[(lane + 32 * h) * ldo + dcur] = sum[h];
    }
    __syncthreads();
    if (threadIdx.x < ncol) {  // H^T R^-1 H on the diagonal
      const int cq = c0 + threadIdx.x;
      const int kc = cq / plane, yyc = (cq - kc * plane) / b.ex,
                xxc = cq - kc * plane - yyc * b.ex;
      const int o =
          obs_of[coords_label(g, b.var, kc, b.lat_lo + yyc, imod(b.lon_lo + xxc, g.nlon))];
      if (o >= 0) Os[threadIdx.x * ldo] += T(1) / R[o];
    }
    __syncthreads();
    // write the tile's band columns (zeros past the block) and clear the
    // output tile for the next one
    T* out = band + b.band_off + (int64_t)c0 * hp1;
    for (int col = warp; col < kCols; col += nw)
      for (int d = lane; d < hp1; d += 32) {
        if (col < ncol) out[(int64_t)col * hp1 + d] = (c0 + col + d < b.nb) ? Os[col * ldo + d] : T(0);
        Os[col * ldo + d] = T(0);
      }
    __syncthreads();
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
// holds l (Eq. 10; interiors are disjoint, so plain stores suffice).  TD: the
// increments' type (rounded to T when added).
template <typename T, typename TD>
__global__ void __launch_bounds__(256) k_writeback(const Geom g, const Block* __restrict__ blocks,
                                                   int nsubx, int sub_lon, int sub_lat,
                                                   const T* __restrict__ Xb,
                                                   const TD* __restrict__ dX,
                                                   const TD* __restrict__ dX2, T* __restrict__ Xa) {
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
  Xa[i] = dX2 ? Xb[i] + (T)(dX[e] + dX2[e]) : Xb[i] + (T)dX[e];
}

}  // namespace

template <typename T, typename TB>
cudaError_t launch_assemble(const Geom& g, const Block* blocks, int nblock, int nb_max,
                            const T* Tg, const T* Dg, const T* Te, const T* De,
                            const int32_t* obs_of, const T* R, TB* band, int32_t* status,
                            cudaStream_t s, int hb_max, const int* rng) {
  const int wpc = 8;
  const int hbp1 = hb_max + 1;
  const size_t smem = sizeof(TB) * (size_t)hbp1 * wpc;
  cudaError_t e = cudaFuncSetAttribute(k_assemble<T, TB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((nb_max + wpc - 1) / wpc, nblock);
  k_assemble<T, TB><<<grid, 32 * wpc, smem, s>>>(g, blocks, Tg, Dg, Te, De, obs_of, R, band,
                                                 status, hbp1, rng);
  return cudaGetLastError();
}

// 32 columns per tile in both precisions: at the T63 shape (hb = 290) a tile's
// shared memory (pair list, output tile, staged rows) stays near 104 KB, so two
// CTAs share an SM and one's staging overlaps the other's sums.
template <typename T>
constexpr int asm_halves() { return 1; }

size_t assemble_pairs_smem(size_t esize, int pmax, int hb_max, int r, int npair_max,
                           int box_sum) {
  const int cols = 32 * (esize == sizeof(float) ? asm_halves<float>() : asm_halves<double>());
  const int rows = asm_rows(cols, hb_max, r);
  return 16 * (size_t)npair_max + esize * (size_t)cols * asm_ldo(hb_max) +
         esize * (size_t)rows * asm_ldt(pmax) + 16 + 8 * (size_t)box_sum + 4 * (size_t)rows;
}

template <typename T>
cudaError_t launch_assemble_pairs(const Geom& g, const Block* blocks, int nblock, int nb_max,
                                  int hb_max, int npair_max, const int4* pairs,
                                  const int32_t* srcrow, const T* Tg, const T* Dg, const T* Te,
                                  const T* De, const int32_t* obs_of, const T* R, T* band,
                                  int box_sum, cudaStream_t s) {
  constexpr int NH = asm_halves<T>();
  const size_t smem = assemble_pairs_smem(sizeof(T), g.pmax, hb_max, g.r, npair_max, box_sum);
  cudaError_t e = cudaFuncSetAttribute(k_assemble_pairs<T, NH>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  constexpr int kTilesPerCta = 8;
  const int ntiles = (nb_max + 32 * NH - 1) / (32 * NH);
  const dim3 grid((ntiles + kTilesPerCta - 1) / kTilesPerCta, nblock);
  k_assemble_pairs<T, NH><<<grid, kAsmThreads, smem, s>>>(g, blocks, pairs, srcrow, Tg, Dg, Te,
                                                          De, obs_of, R, band, hb_max,
                                                          kTilesPerCta);
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

template <typename T, typename TD>
cudaError_t launch_writeback(const Geom& g, const Block* blocks, int nsubx, int sub_lon,
                             int sub_lat, const T* Xb, const TD* dX, const TD* dX2, T* Xa,
                             cudaStream_t s) {
  const dim3 grid((unsigned)((g.n + 255) / 256), g.N);
  k_writeback<T, TD><<<grid, 256, 0, s>>>(g, blocks, nsubx, sub_lon, sub_lat, Xb, dX, dX2, Xa);
  return cudaGetLastError();
}

#define INST(T)                                                                                  \
  template cudaError_t launch_assemble_pairs<T>(const Geom&, const Block*, int, int, int, int,  \
                                                const int4*, const int32_t*, const T*, const T*,  \
                                                const T*, const T*, const int32_t*, const T*, T*, \
                                                int, cudaStream_t);                                \
  template cudaError_t launch_assemble<T, T>(const Geom&, const Block*, int, int, const T*,     \
                                             const T*, const T*, const T*, const int32_t*,      \
                                             const T*, T*, int32_t*, cudaStream_t, int,         \
                                             const int*);                                        \
  template cudaError_t launch_rhs<T>(const Geom&, const Block*, int, int, const int32_t*,       \
                                     int64_t, const T*, const T*, const T*, const T*, T*,       \
                                     cudaStream_t);                                              \
  template cudaError_t launch_writeback<T, T>(const Geom&, const Block*, int, int, int,        \
                                              const T*, const T*, const T*, T*, cudaStream_t);
INST(float)
INST(double)
#undef INST
template cudaError_t launch_assemble<float, double>(const Geom&, const Block*, int, int,
                                                    const float*, const float*, const float*,
                                                    const float*, const int32_t*, const float*,
                                                    double*, int32_t*, cudaStream_t, int,
                                                    const int*);

}  // namespace enkfmc
