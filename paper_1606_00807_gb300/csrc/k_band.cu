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

#include "band_panel.cuh"
#include "enkfmc_internal.h"

namespace enkfmc {

namespace {

constexpr int NB = 32;
constexpr int kThreads = 256;
constexpr int kSolveThreads = 320;

// Four consecutive elements from 16-byte aligned shared memory.
template <typename T>
__device__ __forceinline__ void lds4(const T* p, T (&v)[4]) {
  if (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = (T)q.x; v[1] = (T)q.y; v[2] = (T)q.z; v[3] = (T)q.w;
  } else {
    const double2 q0 = reinterpret_cast<const double2*>(p)[0];
    const double2 q1 = reinterpret_cast<const double2*>(p)[1];
    v[0] = (T)q0.x; v[1] = (T)q0.y; v[2] = (T)q1.x; v[3] = (T)q1.y;
  }
}


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

// rng (optional): only the entries [rng[0], rng[1]) of `blocks` are factored
// (device range: the double-precision pool of blocks whose single-precision
// factorisation failed or converged too slowly); bfail (optional): per-block
// failure flags, see factor_panel.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bandchol(const Block* __restrict__ blocks,
                                                       T* __restrict__ band,
                                                       T* __restrict__ invdiag, int32_t* status,
                                                       int ldP, const int* __restrict__ rng,
                                                       int* __restrict__ bfail) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* P = reinterpret_cast<T*>(smem);  // [NB][ldP]: P[t*ldP + i] = A[c0+i][c0+t]
  if (rng && ((int)blockIdx.x < rng[0] || (int)blockIdx.x >= rng[1])) return;
  const Block b = blocks[blockIdx.x];
  const int nb = b.nb, hb = b.hb, ld = hb + 1;
  T* AB = band + b.band_off;
  const int tid = threadIdx.x;
  for (int c0 = 0; c0 < nb; c0 += NB) {
    const int nbc = min(NB, nb - c0);
    const int rows = min(nbc + hb, nb - c0);
    load_panel(AB, ld, hb, c0, nbc, rows, P, ldP);
    __syncthreads();
    if (!factor_panel(P, ldP, nbc, rows, invdiag ? invdiag + b.row_off + c0 : nullptr, status,
                      bfail, b.id))
      return;  // uniform: every thread read the same pivot
    write_panel(AB, ld, hb, c0, nbc, rows, P, ldP);
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
        const bool vec = ((nbc & 3) == 0) && (i0 + 3 < rows) && (j0 + 3 < rows);
        for (int t = 0; t < nbc; ++t) {
          const T* Pt = P + t * ldP;
          T av[4], bv[4];
          if (vec) {
            lds4(Pt + i0, av);
            lds4(Pt + j0, bv);
          } else {
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = (i0 + a < rows) ? Pt[i0 + a] : T(0);
#pragma unroll
            for (int c = 0; c < 4; ++c) bv[c] = (j0 + c < rows) ? Pt[j0 + c] : T(0);
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
        }
        // read the 16 entries, then write them: the loads are independent, so
        // they are all in flight together
        T old[4][4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int jj = 4 * C + c;  // window-relative column
          const T* colp = AB + (int64_t)(c0 + nbc + jj) * ld;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int ii = 4 * I + a;
            old[a][c] = (jj < W && ii < W && ii >= jj) ? colp[ii - jj] : T(0);
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int jj = 4 * C + c;
          T* colp = AB + (int64_t)(c0 + nbc + jj) * ld;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int ii = 4 * I + a;
            if (jj < W && ii < W && ii >= jj) colp[ii - jj] = old[a][c] - acc[a][c];
          }
        }
      }
    }
    __syncthreads();
  }
}

// Solve L L^T X = B for members [m0, m0 + NMB) of one block.  The rows of B
// the current panel touches (NB + hb of them) live in a circular window of WR
// rows in shared memory (row i in slot i mod WR, WR a multiple of NB, so a
// panel's own rows are contiguous slots); finished rows go back to global
// memory and the next ones are read in their place.  The NB x NB diagonal
// triangles are solved one member per thread in registers.  T: the factor
// and the arithmetic; TR: the right-hand sides (single-precision rhs of a
// block factored in double).  pool (optional, the double-precision pool):
// `blocks` has pool[1] live entries; those in [pool[2], pool[3]) are solved,
// the others get a zero solution (a refinement step whose correction they do
// not need).  skip (optional): blocks with skip[id] set are left to the
// double-precision pool.
template <typename T, typename TR, int NMB>
__global__ void __launch_bounds__(kSolveThreads) k_bandsolve(const Block* __restrict__ blocks,
                                                        const T* __restrict__ band,
                                                        TR* __restrict__ rhs, int N, int ldP,
                                                        int WRmax, const int* __restrict__ pool,
                                                        const int* __restrict__ skip) {
  constexpr int NMP = NMB + 4;
  extern __shared__ __align__(16) unsigned char smem[];
  T* P = reinterpret_cast<T*>(smem);   // [NB][ldP]
  T* Wn = P + (size_t)NB * ldP;        // [WRmax][NMP]
  T* Red = Wn + (size_t)WRmax * NMP;   // [4][NB][NMB] partial sums
  T* invd = Red + 4 * NB * NMB;        // [NB]
  // the member chunks of one block are consecutive thread blocks, so they run
  // together and share the factor through L2
  if (pool && (int)blockIdx.y >= pool[1]) return;
  const Block b = blocks[blockIdx.y];
  if (skip && skip[b.id]) return;
  if (pool && ((int)blockIdx.y < pool[2] || (int)blockIdx.y >= pool[3])) {
    const int m0z = blockIdx.x * NMB, nmz = min(NMB, N - m0z);
    TR* Bz = rhs + b.row_off * N + (int64_t)m0z * b.nb;
    for (int64_t e = threadIdx.x; e < (int64_t)nmz * b.nb; e += blockDim.x) Bz[e] = TR(0);
    return;
  }
  const int m0 = blockIdx.x * NMB;
  const int nm = min(NMB, N - m0);
  const int nb = b.nb, hb = b.hb, ld = hb + 1;
  const int WR = ((NB + hb + NB - 1) / NB) * NB;
  const T* AB = band + b.band_off;
  TR* B = rhs + b.row_off * N + (int64_t)m0 * nb;  // B[m * nb + i], m relative to m0
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;

  // rows [r0, r0 + cnt) <-> slots starting at r0 mod WR (no wrap inside: cnt <= NB
  // and r0 a multiple of NB, or the initial fill starting at slot 0)
  auto load_rows = [&](int r0, int cnt) {
    const int sb = r0 % WR;
    for (int m = warp; m < nm; m += nw)
      for (int i = lane; i < cnt; i += 32) Wn[(sb + i) * NMP + m] = (T)B[(int64_t)m * nb + r0 + i];
  };
  auto store_rows = [&](int r0, int cnt) {
    const int sb = r0 % WR;
    for (int m = warp; m < nm; m += nw)
      for (int i = lane; i < cnt; i += 32) B[(int64_t)m * nb + r0 + i] = (TR)Wn[(sb + i) * NMP + m];
  };
  auto slot = [&](int base, int i) {
    const int sl = base + i;
    return sl >= WR ? sl - WR : sl;
  };

  // ---- forward: L Y = B ----
  load_rows(0, min(WR, nb));
  for (int c0 = 0; c0 < nb; c0 += NB) {
    const int nbc = min(NB, nb - c0);
    const int rows = min(nbc + hb, nb - c0);
    const int base = c0 % WR;
    load_panel(AB, ld, hb, c0, nbc, rows, P, ldP);
    __syncthreads();
    if (tid < NB) invd[tid] = tid < nbc ? T(1) / P[tid * ldP + tid] : T(0);
    __syncthreads();
    // forward triangle in blocks of 8 rows: one thread per member solves the
    // block in registers, then every thread updates the panel rows below it
#pragma unroll 1
    for (int B0 = 0; B0 < nbc; B0 += 8) {
      if (tid < nm) {
        T* w = Wn + base * NMP + tid;
        T yv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) yv[j] = (B0 + j < nbc) ? w[(B0 + j) * NMP] : T(0);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          T acc = yv[j];
#pragma unroll
          for (int i = 0; i < j; ++i) acc = fma(-P[(B0 + i) * ldP + B0 + j], yv[i], acc);
          yv[j] = acc * invd[B0 + j];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (B0 + j < nbc) w[(B0 + j) * NMP] = yv[j];
      }
      __syncthreads();
      const int rem = nbc - (B0 + 8);  // > 0 only when this sub-block is full
      for (int idx = tid; idx < rem * nm; idx += blockDim.x) {
        const int t = B0 + 8 + idx / nm, m = idx - (idx / nm) * nm;
        T* wt = Wn + (base + t) * NMP + m;
        const T* y8 = Wn + (base + B0) * NMP + m;
        T acc = *wt;
#pragma unroll
        for (int j = 0; j < 8; ++j) acc = fma(-P[(B0 + j) * ldP + t], y8[j * NMP], acc);
        *wt = acc;
      }
      __syncthreads();
    }
    const int Wr = rows - nbc;
    const int nTi = (Wr + 3) >> 2;
    constexpr int TMT = NMB / 8;
    for (int tile = tid; tile < nTi * TMT; tile += blockDim.x) {
      const int Ti = tile / TMT, Tm = tile - Ti * TMT;
      const int i0 = nbc + 4 * Ti, mm0 = 8 * Tm;
      if (mm0 >= nm) continue;
      T acc[4][8];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[a][c] = T(0);
      const bool vec = ((nbc & 3) == 0) && (i0 + 3 < rows);
      for (int t = 0; t < nbc; ++t) {
        T av[4], yv[8], y0[4], y1[4];
        if (vec) {
          lds4(P + t * ldP + i0, av);
        } else {
#pragma unroll
          for (int a = 0; a < 4; ++a) av[a] = (i0 + a < rows) ? P[t * ldP + i0 + a] : T(0);
        }
        const T* yr = Wn + (base + t) * NMP + mm0;
        lds4(yr, y0);
        lds4(yr + 4, y1);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          yv[c] = y0[c];
          yv[4 + c] = y1[c];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[a][c] = fma(av[a], yv[c], acc[a][c]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        if (i0 + a >= rows) break;
        T* wr = Wn + slot(base, i0 + a) * NMP + mm0;
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
    const int base = c0 % WR;
    load_rows(c0, nbc);  // Y of this panel (its slots held rows >= c0 + hb)
    load_panel(AB, ld, hb, c0, nbc, rows, P, ldP);
    __syncthreads();
    if (tid < NB) invd[tid] = tid < nbc ? T(1) / P[tid * ldP + tid] : T(0);
    // partial sums of L[c0+i][c0+t] X[c0+i][m] over i in [nbc, rows), 4 groups of i
    constexpr int TM4 = NMB / 4;
    for (int job = tid; job < (NB / 4) * TM4 * 4; job += blockDim.x) {
      const int tile = job % ((NB / 4) * TM4), kg = job / ((NB / 4) * TM4);
      const int t0 = 4 * (tile / TM4), mm0 = 4 * (tile % TM4);
      T acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = T(0);
      for (int i = nbc + kg; i < rows; i += 4) {
        T lv[4], xv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) lv[a] = (t0 + a < nbc) ? P[(t0 + a) * ldP + i] : T(0);
        lds4(Wn + slot(base, i) * NMP + mm0, xv);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][c] = fma(lv[a], xv[c], acc[a][c]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) Red[(kg * NB + t0 + a) * NMB + mm0 + c] = acc[a][c];
    }
    __syncthreads();
    for (int idx = tid; idx < nbc * nm; idx += blockDim.x) {
      const int t = idx / nm, m = idx - t * nm;
      Wn[(base + t) * NMP + m] -= Red[(0 * NB + t) * NMB + m] + Red[(1 * NB + t) * NMB + m] +
                                  Red[(2 * NB + t) * NMB + m] + Red[(3 * NB + t) * NMB + m];
    }
    __syncthreads();
    // backward triangle in blocks of 8 rows, last block first; the rows above a
    // solved block are updated by every thread
#pragma unroll 1
    for (int B0 = ((nbc - 1) / 8) * 8; B0 >= 0; B0 -= 8) {
      if (tid < nm) {
        T* w = Wn + base * NMP + tid;
        T yv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) yv[j] = (B0 + j < nbc) ? w[(B0 + j) * NMP] : T(0);
#pragma unroll
        for (int j = 7; j >= 0; --j) {
          T acc = yv[j];
#pragma unroll
          for (int i = j + 1; i < 8; ++i) acc = fma(-P[(B0 + j) * ldP + B0 + i], yv[i], acc);
          yv[j] = acc * invd[B0 + j];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (B0 + j < nbc) w[(B0 + j) * NMP] = yv[j];
      }
      __syncthreads();
      const int jn = min(8, nbc - B0);  // rows of this sub-block inside the panel
      for (int idx = tid; idx < B0 * nm; idx += blockDim.x) {
        const int t = idx / nm, m = idx - t * nm;
        T* wt = Wn + (base + t) * NMP + m;
        const T* y8 = Wn + (base + B0) * NMP + m;
        T acc = *wt;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (j < jn) acc = fma(-P[t * ldP + B0 + j], y8[j * NMP], acc);
        *wt = acc;
      }
      __syncthreads();
    }
    store_rows(c0, nbc);
    __syncthreads();
  }
}

// The double-precision pool: blocks in block order, their entries with
// band_off moved into `cap` slots of `stride` elements.  append = 0: rebuild
// from the blocks flagged 1 (non-positive pivot); append = 1: add the blocks
// flagged 2 (refinement converging too slowly) after the present ones and
// flag them 1.  meta holds three views {0, end, lo, hi} of the pool (end
// blocks) for k_bandsolve: meta[0..3] solves all of them, meta[4..7] the ones
// added by this call, meta[8..11] none; meta + 2 and meta + 6 are the
// {lo, hi} ranges of all and of the added blocks for the assembly and the
// factorisation.  More blocks than slots: ENOTSPD for the first block left
// out.  One thread (a few thousand flags at most).
__global__ void k_fallback_list(const Block* __restrict__ blocks, int nblock,
                                int* __restrict__ bfail, Block* __restrict__ pool,
                                int* __restrict__ meta, int cap, int64_t stride, int32_t* status,
                                int append) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int k = append ? meta[1] : 0;
  const int first = k;
  for (int i = 0; i < nblock; ++i) {
    if (bfail[i] != (append ? 2 : 1)) continue;
    if (k == cap) {
      record_error(status, ENKFMC_ENOTSPD, (int64_t)i);
      break;
    }
    Block b = blocks[i];
    b.band_off = (int64_t)k * stride;
    pool[k++] = b;
    bfail[i] = 1;
  }
  const int views[12] = {0, k, 0, k, 0, k, first, k, 0, k, 0, 0};
  for (int i = 0; i < 12; ++i) meta[i] = views[i];
}

// Convergence of the single-precision refinement per block (one CTA each):
// phase 0 stores max |c| of the first correction; phase 1, after the second
// correction c, flags the block 2 (double precision from here) when the
// corrections do not shrink (rho = max|c2| / max|c1| >= 1) or when the
// error they predict after two more steps, max|c2| rho^2, exceeds
// tau max|x|.  Blocks already in the pool are left alone.
__global__ void __launch_bounds__(256) k_ir_check(const Block* __restrict__ blocks, int N,
                                                  const float* __restrict__ c,
                                                  const float* __restrict__ x,
                                                  float* __restrict__ c1max,
                                                  int* __restrict__ bfail, float tau, int phase) {
  __shared__ float red[2][8];
  const Block b = blocks[blockIdx.x];
  if (bfail[b.id]) return;
  const int64_t cnt = (int64_t)b.nb * N, base = b.row_off * N;
  float mc = 0.f, mx = 0.f;
  for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) {
    mc = fmaxf(mc, fabsf(c[base + e]));
    if (phase) mx = fmaxf(mx, fabsf(x[base + e]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    mc = fmaxf(mc, __shfl_xor_sync(0xffffffffu, mc, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = mc;
    red[1][warp] = mx;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
    mc = fmaxf(mc, red[0][w]);
    mx = fmaxf(mx, red[1][w]);
  }
  if (phase == 0) {
    c1max[b.id] = mc;
    return;
  }
  const float c1 = c1max[b.id];
  const float rho = c1 > 0.f ? mc / c1 : 0.f;
  if (!(rho < 1.f) || !(mc * rho * rho <= tau * mx)) bfail[b.id] = 2;
}

}  // namespace

template <typename T>
cudaError_t launch_bandchol(const Block* blocks, int nblock, int hb_max, T* band, T* invdiag,
                            int32_t* status, cudaStream_t s, const int* rng, int* bfail) {
  const int ldP = (NB + hb_max + 1 + 3) / 4 * 4;
  const size_t smem = sizeof(T) * (size_t)NB * ldP;
  cudaError_t e = cudaFuncSetAttribute(k_bandchol<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_bandchol<T><<<nblock, kThreads, smem, s>>>(blocks, band, invdiag, status, ldP, rng, bfail);
  return cudaGetLastError();
}

template <typename T, typename TR, int NMB>
cudaError_t launch_bandsolve_nm(const Block* blocks, int nblock, int N, const T* band, TR* rhs,
                                cudaStream_t s, size_t smem, int ldP, int WRmax, const int* pool,
                                const int* skip) {
  cudaError_t e = cudaFuncSetAttribute(k_bandsolve<T, TR, NMB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((N + NMB - 1) / NMB, nblock);
  k_bandsolve<T, TR, NMB><<<grid, kSolveThreads, smem, s>>>(blocks, band, rhs, N, ldP, WRmax, pool,
                                                            skip);
  return cudaGetLastError();
}

// Shared memory of the CUDA-core band kernels for a half-bandwidth hb and
// elements of esize bytes (the launchers below size them the same way).
constexpr size_t kBandSmemLimit = 227 * 1024;
size_t bandchol_smem(int hb, size_t esize) {
  const int ldP = (NB + hb + 1 + 3) / 4 * 4;
  return esize * (size_t)NB * ldP;
}
size_t bandsolve_smem(int hb, size_t esize, int nmb) {
  const int ldP = (NB + hb + 1 + 3) / 4 * 4;
  const int WRmax = ((NB + hb + NB - 1) / NB) * NB;
  return esize * ((size_t)NB * ldP + (size_t)WRmax * (nmb + 4) + 4 * (size_t)NB * nmb + NB);
}

bool band_kernels_fit(int hb, size_t esize) {
  return bandchol_smem(hb, esize) <= kBandSmemLimit &&
         bandsolve_smem(hb, esize, 8) <= kBandSmemLimit;
}

template <typename T, typename TR>
cudaError_t launch_bandsolve(const Block* blocks, int nblock, int hb_max, int N, const T* band,
                             TR* rhs, cudaStream_t s, const int* pool, const int* skip) {
  const int ldP = (NB + hb_max + 1 + 3) / 4 * 4;
  const int WRmax = ((NB + hb_max + NB - 1) / NB) * NB;
  auto bytes = [&](int nmb) { return bandsolve_smem(hb_max, sizeof(T), nmb); };
  const size_t lim = kBandSmemLimit;
  if (bytes(32) <= lim)
    return launch_bandsolve_nm<T, TR, 32>(blocks, nblock, N, band, rhs, s, bytes(32), ldP, WRmax,
                                          pool, skip);
  if (bytes(16) <= lim)
    return launch_bandsolve_nm<T, TR, 16>(blocks, nblock, N, band, rhs, s, bytes(16), ldP, WRmax,
                                          pool, skip);
  if (bytes(8) <= lim)
    return launch_bandsolve_nm<T, TR, 8>(blocks, nblock, N, band, rhs, s, bytes(8), ldP, WRmax,
                                         pool, skip);
  return cudaErrorInvalidConfiguration;
}

cudaError_t launch_fallback_list(const Block* blocks, int nblock, int* bfail, Block* pool,
                                 int* meta, int cap, int64_t stride, int32_t* status, int append,
                                 cudaStream_t s) {
  k_fallback_list<<<1, 32, 0, s>>>(blocks, nblock, bfail, pool, meta, cap, stride, status,
                                   append);
  return cudaGetLastError();
}

cudaError_t launch_ir_check(const Block* blocks, int nblock, int N, const float* c,
                            const float* x, float* c1max, int* bfail, float tau, int phase,
                            cudaStream_t s) {
  k_ir_check<<<nblock, 256, 0, s>>>(blocks, N, c, x, c1max, bfail, tau, phase);
  return cudaGetLastError();
}

template cudaError_t launch_bandchol<float>(const Block*, int, int, float*, float*, int32_t*,
                                            cudaStream_t, const int*, int*);
template cudaError_t launch_bandchol<double>(const Block*, int, int, double*, double*, int32_t*,
                                             cudaStream_t, const int*, int*);
template cudaError_t launch_bandsolve<float, float>(const Block*, int, int, int, const float*,
                                                    float*, cudaStream_t, const int*, const int*);
template cudaError_t launch_bandsolve<double, double>(const Block*, int, int, int, const double*,
                                                      double*, cudaStream_t, const int*,
                                                      const int*);
template cudaError_t launch_bandsolve<double, float>(const Block*, int, int, int, const double*,
                                                     float*, cudaStream_t, const int*,
                                                     const int*);

}  // namespace enkfmc
