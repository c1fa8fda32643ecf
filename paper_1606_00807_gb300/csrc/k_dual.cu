// Dual form of the sub-domain analysis (Eq. 12-13).  With B = T^-1 D T^-T the
// inverse of T^T D^-1 T (Eq. 9), X~ = T^-1 D^1/2 (Eq. 13) and V = H X~, the
// increment of Eq. 12 is
//     dX = X~ V^T (R + V V^T)^-1 (Y^s - H X^b) = T^-1 D Z W,
// where Z = T^-T H^T (n_b x m_b) and W = (R + Z^T D Z)^-1 (Y^s - H X^b)
// (m_b x N): two unit-triangular solves with the block's T and one dense m_b x
// m_b system in observation space, instead of the band factor of A.  Per
// (sub-domain, variable) block, on the same T rows and D entries as the primal
// form (interior rows from the global estimate, boundary rows re-estimated
// from the local samples), and the same observations (those inside the
// extended set):
//   k_dual_z      Z = T^-T H^T, one warp per 32 observation columns;
//   k_dual_obs    S = R + Z^T D Z, S = L L^T, W = S^-1 (Y^s - H X^b), one CTA
//                 per block, in shared memory;
//   k_dual_q      Q = D (Z W) into the increment buffer, a tiled product;
//   k_dual_apply  dX = T^-1 Q in place, one warp per 32 members.
//
// Solve order.  T is unit lower triangular in label order (a predecessor has a
// smaller label).  Within a row segment of the block (one level, one
// latitude) the local index follows the longitude from the box's western edge,
// which passes the longitude seam when the box wraps; the solves therefore walk
// the rows in label order, position t: segment by segment, and inside a
// segment from the columns past the seam (x = 0, 1, ...) to those before it.
// A row and any of its predecessors lie less than W = (vr ey + r + 1) ex
// positions apart, so a solve keeps the last W rows of its columns in a ring
// in shared memory.
#include <algorithm>

#include "enkfmc_internal.h"

namespace enkfmc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// position t (label order) <-> local index of a block's row
struct SolveOrder {
  int ex, npre;  // npre: columns of a segment before the seam (all when none)
  __device__ __forceinline__ int loc_of(int t) const {
    const int seg = t / ex;
    int xx = t - seg * ex + npre;
    if (xx >= ex) xx -= ex;
    return seg * ex + xx;
  }
  __device__ __forceinline__ int pos_of(int loc) const {
    const int seg = loc / ex;
    int u = loc - seg * ex - npre;
    if (u < 0) u += ex;
    return seg * ex + u;
  }
};

__device__ __forceinline__ SolveOrder solve_order(const Block& b, int nlon) {
  return {b.ex, min(b.ex, nlon - b.lon_lo)};
}

// A position walked one step at a time (no divisions): segment, offset u in
// it, and the local index.
struct OrderCursor {
  int seg, u, ex, npre;
  __device__ __forceinline__ OrderCursor(const SolveOrder& o, int t)
      : seg(t / o.ex), u(t - (t / o.ex) * o.ex), ex(o.ex), npre(o.npre) {}
  __device__ __forceinline__ int loc() const {
    int xx = u + npre;
    if (xx >= ex) xx -= ex;
    return seg * ex + xx;
  }
  __device__ __forceinline__ void next() {
    if (++u == ex) {
      u = 0;
      ++seg;
    }
  }
  __device__ __forceinline__ void prev() {
    if (--u < 0) {
      u = ex - 1;
      --seg;
    }
  }
};

__device__ __forceinline__ void local_coords(const Block& b, int nlon, int loc, int& k, int& y,
                                             int& x) {
  const int plane = b.ey * b.ex;
  k = loc / plane;
  const int rem = loc - k * plane;
  const int yy = rem / b.ex;
  y = b.lat_lo + yy;
  x = imod(b.lon_lo + rem - yy * b.ex, nlon);
}

// Row of T for local row loc at (k, y, x): the global estimate inside the
// tile, the re-estimated boundary row otherwise (as in the primal assembly).
template <typename T>
__device__ __forceinline__ const T* block_trow(const Geom& g, const Block& b, int k, int y, int x,
                                               int loc, const T* Tg, const T* Te) {
  if (in_interior(b, y, x)) return Tg + coords_label(g, b.var, k, y, x) * g.pmax;
  return Te + (b.row_off + loc) * g.pmax;
}

template <typename T>
__device__ __forceinline__ T block_d(const Geom& g, const Block& b, int k, int y, int x, int loc,
                                     const T* Dg, const T* De) {
  if (in_interior(b, y, x)) return Dg[coords_label(g, b.var, k, y, x)];
  return De[b.row_off + loc];
}

__device__ __forceinline__ void load_slot_offsets(const Geom& g, signed char* so) {
  for (int s = threadIdx.x; s < g.pmax; s += blockDim.x) {
    int dk, dy, dx;
    slot_offset(s, g.r, g.vr, dk, dy, dx);
    so[s] = (signed char)dk;
    so[g.pmax + s] = (signed char)dy;
    so[2 * g.pmax + s] = (signed char)dx;
  }
}

__host__ __device__ inline int slot_bytes(int pmax) { return (3 * pmax + 15) / 16 * 16; }

// One term of a row's sum: the ring offset (slot x 32) of the row it reads and
// its coefficient.
template <typename T>
struct alignas(2 * sizeof(T) > 8 ? 16 : 8) Term {
  int at;
  T v;
};

// Entries per row of the term tables: pmax rounded up to even, so that every
// row starts on a 16-byte boundary (the solves copy rows in 16-byte pieces).
__host__ __device__ inline int term_stride(int pmax) { return (pmax + 1) & ~1; }

// Rows the solves stage ahead of the one they sum (cp.async pipeline depth).
constexpr int kStages = 8;

// Shared memory of a triangular solve (one warp): the ring [W][32], the
// current row's compacted terms [pmax], the staged table rows
// [kStages][term_stride] and (forward solve) the staged q values [kStages][32].
template <typename T>
size_t solve_smem(int W, int pmax) {
  return (size_t)W * 32 * sizeof(T) + (size_t)term_stride(pmax) * sizeof(Term<T>) +
         (size_t)kStages * term_stride(pmax) * sizeof(Term<T>) + (size_t)kStages * 32 * sizeof(T);
}

// x - sum of v ring[at + lane] over the terms: four partial sums, unrolled
// (a fixed order, so the same bits on every run).
template <typename T>
__device__ __forceinline__ T sub_terms(T x, const Term<T>* terms, int n, const T* ring,
                                       int lane) {
  T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
  int i = 0;
  for (; i + 4 <= n; i += 4) {
    const Term<T> e0 = terms[i], e1 = terms[i + 1], e2 = terms[i + 2], e3 = terms[i + 3];
    a0 = fma(e0.v, ring[e0.at + lane], a0);
    a1 = fma(e1.v, ring[e1.at + lane], a1);
    a2 = fma(e2.v, ring[e2.at + lane], a2);
    a3 = fma(e3.v, ring[e3.at + lane], a3);
  }
  for (; i < n; ++i) {
    const Term<T> e = terms[i];
    a0 = fma(e.v, ring[e.at + lane], a0);
  }
  return x - ((a0 + a1) + (a2 + a3));
}

// Slots of a row handled by one lane (s = lane + 32 q): pmax <= 32 kSlotQ.
constexpr int kSlotQ = kDualMaxSlots / 32;

// ---------------------------------------------------------------------------
// The two solves' term tables, per block in solve order [nb][pmax] at
// row_off pmax: for the row at position t and slot s,
//   pred[t][s] = {t - t_q, T[j][s]}   its predecessor in slot s (forward solve),
//   succ[t][s] = {t_i - t, T[i][s]}   the row i that holds it in slot s (the
//                                      solve with T^T),
// {0, 0} where there is none inside the extended set.  A thread per (row,
// slot); built once per analysis, so the serial solves read one contiguous
// row of terms per step instead of resolving the geometry (and the scattered
// coefficients of the successors) on their critical path.
// ---------------------------------------------------------------------------
template <typename TI, typename T>
__global__ void __launch_bounds__(256) k_dual_terms(const Geom g, const Block* __restrict__ blocks,
                                                    const TI* __restrict__ Tg,
                                                    const TI* __restrict__ Te,
                                                    Term<T>* __restrict__ pred,
                                                    Term<T>* __restrict__ succ) {
  __shared__ signed char so[3 * 128];
  const Block b = blocks[blockIdx.y];
  load_slot_offsets(g, so);
  __syncthreads();
  const int pmax = g.pmax;
  const int t = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (t >= b.nb) return;
  const SolveOrder ord = solve_order(b, g.nlon);
  const int j = ord.loc_of(t);
  int k, y, x;
  local_coords(b, g.nlon, j, k, y, x);
  const TI* trow = block_trow(g, b, k, y, x, j, Tg, Te);
  const int ts = term_stride(pmax);
  Term<T>* P = pred + (b.row_off + t) * ts;
  Term<T>* S = succ + (b.row_off + t) * ts;
  if ((threadIdx.x & 31) == 0 && ts > pmax) {
    P[pmax] = Term<T>{0, T(0)};
    S[pmax] = Term<T>{0, T(0)};
  }
  for (int s = threadIdx.x & 31; s < pmax; s += 32) {
    // predecessor of row j in slot s
    Term<T> e{0, T(0)};
    const T v = (T)trow[s];
    int kq, yq, xq, yyq, xxq;
    if (v != T(0) &&
        slot_pred_off(g, k, y, x, so[s], so[pmax + s], so[2 * pmax + s], kq, yq, xq) &&
        in_ext(b, g.nlon, yq, xq, yyq, xxq)) {
      const int tq = ord.pos_of((kq * b.ey + yyq) * b.ex + xxq);
      if (tq < t) e = Term<T>{t - tq, v};
    }
    P[s] = e;
    // the row i that holds j in slot s
    Term<T> f{0, T(0)};
    const int ki = k - so[s], yi = y - so[pmax + s];
    int xi = x - so[2 * pmax + s];
    bool ok = ki < b.nlev_b && yi >= 0 && yi < g.nlat;
    if (ok && (xi < 0 || xi >= g.nlon)) {
      if (g.periodic) xi = imod(xi, g.nlon);
      else ok = false;
    }
    int yyi, xxi;
    if (ok && in_ext(b, g.nlon, yi, xi, yyi, xxi)) {
      const int li = (ki * b.ey + yyi) * b.ex + xxi;
      const int ti = ord.pos_of(li);
      const T w = (T)block_trow(g, b, ki, yi, xi, li, Tg, Te)[s];
      if (ti > t && w != T(0)) f = Term<T>{ti - t, w};
    }
    S[s] = f;
  }
}

// Asynchronous global -> shared copies (cp.async), committed in one group per
// staged row and waited for kStages - 1 groups behind.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
template <int B>
__device__ __forceinline__ void cp_async_small(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(B)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_stages() {
  asm volatile("cp.async.wait_group %0;" ::"n"(kStages - 1) : "memory");
}

// One table row (ts entries, 16-byte aligned) into a stage, by the lanes.
template <typename T>
__device__ __forceinline__ void stage_row(Term<T>* dst, const Term<T>* src, int ts, int lane) {
  const int chunks = ts * (int)sizeof(Term<T>) / 16;
  for (int i = lane; i < chunks; i += 32)
    cp_async16(reinterpret_cast<char*>(dst) + 16 * i, reinterpret_cast<const char*>(src) + 16 * i);
}

// The terms of one staged row compacted into `terms` with their ring offsets
// (slot x 32; the row at distance d: sign +1 after t, -1 before; only
// distances below W and, with lim >= 0, rows at positions up to lim count).
// Returns the number of terms.
template <typename T>
__device__ __forceinline__ int load_terms(Term<T>* terms, const Term<T>* row, int pmax, int rt,
                                          int W, int sign, int t, int lim, int lane) {
  int n = 0;
#pragma unroll
  for (int q = 0; q < kSlotQ; ++q) {
    const int s = lane + 32 * q;
    Term<T> e{0, T(0)};
    if (s < pmax) e = row[s];
    const bool on = e.at > 0 && e.at < W && (lim < 0 || t + e.at <= lim);
    const unsigned mask = __ballot_sync(0xffffffffu, on);
    if (on) {
      int sl = rt + sign * e.at;
      if (sl >= W) sl -= W;
      if (sl < 0) sl += W;
      terms[n + __popc(mask & ((1u << lane) - 1u))] = Term<T>{sl * 32, e.v};
    }
    n += __popc(mask);
    if (32 * (q + 1) >= pmax) break;
  }
  return n;
}

// ---------------------------------------------------------------------------
// Z = T^-T H^T.  Column c of block b holds the observation dobs[dob_off[b] + c]
// = {t_c, o} (columns in increasing position t_c); T^T z = e_{t_c} is solved
// from the last row backwards: z_j = e_j - sum over the rows i that hold j in a
// slot s of T[i][s] z_i (i after j).  Rows after the warp's last t_c are zero
// in all its columns.  Z: [nb][mb] per block (local row index), at zoff[b].
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(32) k_dual_z(const Geom g, const Block* __restrict__ blocks,
                                               const int2* __restrict__ dobs,
                                               const int64_t* __restrict__ dob_off,
                                               const int64_t* __restrict__ zoff,
                                               const Term<T>* __restrict__ succ,
                                               T* __restrict__ Zb, int W) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int pmax = g.pmax, ts = term_stride(pmax);
  T* ring = reinterpret_cast<T*>(smem);
  Term<T>* terms = reinterpret_cast<Term<T>*>(ring + (size_t)W * 32);
  Term<T>* stage = terms + ts;  // [kStages][ts]
  const Block b = blocks[blockIdx.y];
  const int64_t o0 = dob_off[blockIdx.y];
  const int mb = (int)(dob_off[blockIdx.y + 1] - o0);
  const int c0 = blockIdx.x * 32;
  if (c0 >= mb) return;
  const int lane = threadIdx.x;
  const int c = c0 + lane;
  const bool act = c < mb;
  const int tc = act ? dobs[o0 + c].x : -1;
  const int tlast = __shfl_sync(kFull, tc, min(31, mb - 1 - c0));
  const SolveOrder ord = solve_order(b, g.nlon);
  T* Z = Zb + zoff[blockIdx.y];
  for (int t = tlast + 1; t < b.nb; ++t)
    if (act) Z[(int64_t)ord.loc_of(t) * mb + c] = T(0);
  const Term<T>* tab = succ + b.row_off * ts;
  // rows tlast, tlast - 1, ... staged kStages ahead (stage of row t: (tlast - t) % kStages)
  for (int d = 0; d < kStages; ++d) {
    if (tlast - d >= 0) stage_row(stage + d * ts, tab + (int64_t)(tlast - d) * ts, ts, lane);
    cp_async_commit();
  }
  int rt = tlast % W;  // ring slot of position t
  int st = 0;          // stage of row t
  OrderCursor cur(ord, tlast);
  for (int t = tlast; t >= 0; --t) {
    cp_async_wait_stages();
    __syncwarp();
    const int n = load_terms(terms, stage + st * ts, pmax, rt, W, 1, t, tlast, lane);
    __syncwarp();
    if (t - kStages >= 0) stage_row(stage + st * ts, tab + (int64_t)(t - kStages) * ts, ts, lane);
    cp_async_commit();
    st = st + 1 == kStages ? 0 : st + 1;
    const T z = sub_terms((t == tc) ? T(1) : T(0), terms, n, ring, lane);
    ring[rt * 32 + lane] = z;
    if (act) Z[(int64_t)cur.loc() * mb + c] = z;
    cur.prev();
    rt = rt == 0 ? W - 1 : rt - 1;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// S = R + Z^T D Z (lower triangle), S = L L^T, and W = S^-1 (Y^s - H X^b)
// for the block's observations; one CTA per block, all in shared memory.
// W: [mb][N] per block at N dob_off[b].  A non-positive or non-finite pivot
// records ENOTSPD (the block's W is then zero).
// ---------------------------------------------------------------------------
constexpr int kObsThreads = 256;
constexpr int kObsRows = 32;  // rows of Z staged per step of the product

__host__ __device__ inline int obs_zld(int mb) {  // row stride of the staged Z rows
  return (mb + 3) & ~3;
}

// Shared memory of k_dual_obs: S, lower triangle packed row by row, then one
// region that first stages Z rows with their D (the product) and then holds
// the innovations and W [mb][N].
template <typename T>
size_t obs_smem(int mb, int N) {
  const size_t tri = (size_t)mb * (mb + 1) / 2 + 1;
  const size_t stage = (size_t)kObsRows * obs_zld(mb) + kObsRows;
  return sizeof(T) * (tri + std::max((size_t)mb * N, stage)) + 16;
}

template <typename TI, typename T>
__global__ void __launch_bounds__(kObsThreads) k_dual_obs(
    const Geom g, const Block* __restrict__ blocks, const int2* __restrict__ dobs,
    const int64_t* __restrict__ dob_off, const int64_t* __restrict__ zoff,
    const int32_t* __restrict__ obs_idx, int64_t mobs, const TI* __restrict__ Xb,
    const TI* __restrict__ y, const TI* __restrict__ R, const TI* __restrict__ Zp,
    const TI* __restrict__ Dg, const TI* __restrict__ De, const T* __restrict__ Zb,
    T* __restrict__ Wb, int32_t* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Block b = blocks[blockIdx.x];
  const int64_t o0 = dob_off[blockIdx.x];
  const int mb = (int)(dob_off[blockIdx.x + 1] - o0);
  if (mb == 0) return;
  const int N = g.N, zld = obs_zld(mb);
  T* S = reinterpret_cast<T*>(smem);             // packed lower triangle, S(i, l) at tri(i) + l
  T* Wm = S + (size_t)mb * (mb + 1) / 2 + 1;     // [mb][N], after the product
  T* Zs = Wm;                                    // [kObsRows][zld] during the product
  T* Ds = Zs + (size_t)kObsRows * zld;           // [kObsRows]
  auto tri = [](int i) { return i * (i + 1) / 2; };
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  const T* Z = Zb + zoff[blockIdx.x];

  // S = Z^T D Z: 4 x 4 tiles of the lower triangle, one per thread per round
  const int nt = (mb + 3) / 4, npair = nt * (nt + 1) / 2;
  for (int base = 0; base < npair; base += kObsThreads) {
    const int pr = base + tid;
    int I = 0, J = 0;
    if (pr < npair) {
      I = (int)((sqrtf(8.f * pr + 1.f) - 1.f) * 0.5f);
      while ((I + 1) * (I + 2) / 2 <= pr) ++I;
      while (I * (I + 1) / 2 > pr) --I;
      J = pr - I * (I + 1) / 2;
    }
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[a][e] = T(0);
    for (int j0 = 0; j0 < b.nb; j0 += kObsRows) {
      __syncthreads();
      const int nr = min(kObsRows, b.nb - j0);
      for (int e = tid; e < kObsRows * zld; e += kObsThreads) {
        const int rr = e / zld, cc = e - rr * zld;
        Zs[e] = (rr < nr && cc < mb) ? Z[(int64_t)(j0 + rr) * mb + cc] : T(0);
      }
      if (tid < kObsRows) {
        T d = T(0);
        if (tid < nr) {
          int k, yy, xx;
          local_coords(b, g.nlon, j0 + tid, k, yy, xx);
          d = (T)block_d(g, b, k, yy, xx, j0 + tid, Dg, De);
        }
        Ds[tid] = d;
      }
      __syncthreads();
      if (pr < npair) {
        for (int rr = 0; rr < nr; ++rr) {
          const T d = Ds[rr];
          const T* zr = Zs + rr * zld;
          T a[4], e4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            a[q] = d * zr[4 * I + q];
            e4[q] = zr[4 * J + q];
          }
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[q][u] = fma(a[q], e4[u], acc[q][u]);
        }
      }
    }
    if (pr < npair) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = 4 * I + q, l = 4 * J + u;
          if (i < mb && l <= i) S[tri(i) + l] = acc[q][u];
        }
    }
  }
  __syncthreads();
  // + R on the diagonal; the innovations Y^s - H X^b into Wm
  for (int c = tid; c < mb; c += kObsThreads) S[tri(c) + c] += (T)R[dobs[o0 + c].y];
  for (int e = tid; e < mb * N; e += kObsThreads) {
    const int c = e / N, m = e - c * N;
    const int o = dobs[o0 + c].y;
    const T sq = sqrt((T)R[o]);
    Wm[e] = fma(sq, (T)Zp[(int64_t)m * mobs + o], (T)y[o]) -
            (T)Xb[(int64_t)m * g.n + obs_idx[o]];
  }
  __syncthreads();
  // Cholesky, right-looking: column k scaled, then the trailing lower triangle
  // (a warp per row, lanes over its columns)
  const int lane = tid & 31, warp = tid >> 5, nw = kObsThreads / 32;
  for (int k = 0; k < mb; ++k) {
    if (tid == 0) {
      const T d = S[tri(k) + k];
      if (!(d > T(0)) || !isfinite(d)) bad = 1;
      else S[tri(k) + k] = sqrt(d);
    }
    __syncthreads();
    if (bad) break;
    const T inv = T(1) / S[tri(k) + k];
    for (int i = k + 1 + tid; i < mb; i += kObsThreads) S[tri(i) + k] *= inv;
    __syncthreads();
    for (int i = k + 1 + warp; i < mb; i += nw) {
      T* Si = S + tri(i);
      const T sik = Si[k];
      for (int l = k + 1 + lane; l <= i; l += 32) Si[l] = fma(-sik, S[tri(l) + k], Si[l]);
    }
    __syncthreads();
  }
  T* Wout = Wb + o0 * N;
  if (bad) {
    if (tid == 0 && status) record_error(status, ENKFMC_ENOTSPD, b.id);
    for (int e = tid; e < mb * N; e += kObsThreads) Wout[e] = T(0);
    return;
  }
  // L L^T W = innovations, a thread per member
  for (int m = tid; m < N; m += kObsThreads) {
    for (int c = 0; c < mb; ++c) {
      const T* Sc = S + tri(c);
      T w = Wm[c * N + m];
      for (int l = 0; l < c; ++l) w = fma(-Sc[l], Wm[l * N + m], w);
      Wm[c * N + m] = w / Sc[c];
    }
    for (int c = mb - 1; c >= 0; --c) {
      T w = Wm[c * N + m];
      for (int l = c + 1; l < mb; ++l) w = fma(-S[tri(l) + c], Wm[l * N + m], w);
      Wm[c * N + m] = w / S[tri(c) + c];
    }
  }
  __syncthreads();
  for (int e = tid; e < mb * N; e += kObsThreads) Wout[e] = Wm[e];
}

// ---------------------------------------------------------------------------
// Q = D (Z W) for every row of every block into the increment buffer
// (dX[row_off N + m nb + loc], the primal solve's layout): a CTA computes 128
// rows x 32 members, a thread rows {tr + 32 a} x members {4 tm + e}, over
// chunks of kQK observation columns staged in shared memory.
// ---------------------------------------------------------------------------
constexpr int kQRows = 128, kQMem = 32, kQK = 16;

template <typename TI, typename T>
__global__ void __launch_bounds__(256) k_dual_q(const Geom g, const Block* __restrict__ blocks,
                                                const int64_t* __restrict__ dob_off,
                                                const int64_t* __restrict__ zoff,
                                                const T* __restrict__ Zb, const T* __restrict__ Wb,
                                                const TI* __restrict__ Dg,
                                                const TI* __restrict__ De, T* __restrict__ dX) {
  __shared__ T Zs[kQRows][kQK + 1];
  __shared__ T Ws[kQK][kQMem];
  const Block b = blocks[blockIdx.y];
  const int r0 = blockIdx.x * kQRows;
  if (r0 >= b.nb) return;
  const int m0 = blockIdx.z * kQMem;
  const int64_t o0 = dob_off[blockIdx.y];
  const int mb = (int)(dob_off[blockIdx.y + 1] - o0);
  const int N = g.N;
  const int tid = threadIdx.x, tr = tid & 31, tm = tid >> 5;  // tm: members 4 tm .. 4 tm + 3
  const T* Z = Zb + zoff[blockIdx.y];
  const T* Wv = Wb + o0 * N;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[a][e] = T(0);
  for (int k0 = 0; k0 < mb; k0 += kQK) {
    __syncthreads();
    for (int e = tid; e < kQRows * kQK; e += 256) {
      const int rr = e / kQK, cc = e - rr * kQK;
      const int j = r0 + rr, o = k0 + cc;
      Zs[rr][cc] = (j < b.nb && o < mb) ? Z[(int64_t)j * mb + o] : T(0);
    }
    for (int e = tid; e < kQK * kQMem; e += 256) {
      const int cc = e / kQMem, mm = e - cc * kQMem;
      const int o = k0 + cc, m = m0 + mm;
      Ws[cc][mm] = (o < mb && m < N) ? Wv[(int64_t)o * N + m] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kQK; ++kk) {
      T w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) w[e] = Ws[kk][4 * tm + e];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const T z = Zs[tr + 32 * a][kk];
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[a][e] = fma(z, w[e], acc[a][e]);
      }
    }
  }
  T* out = dX + b.row_off * N;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int j = r0 + tr + 32 * a;
    if (j >= b.nb) continue;
    int k, y, x;
    local_coords(b, g.nlon, j, k, y, x);
    const T d = (T)block_d(g, b, k, y, x, j, Dg, De);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int m = m0 + 4 * tm + e;
      if (m < N) out[(int64_t)m * b.nb + j] = d * acc[a][e];
    }
  }
}

// ---------------------------------------------------------------------------
// dX = T^-1 Q in place, forward in label order: x_j = q_j - sum_s T[j][s]
// x_{pred_s(j)}; a warp per 32 members of a block.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(32) k_dual_apply(const Geom g, const Block* __restrict__ blocks,
                                                   const Term<T>* __restrict__ pred,
                                                   const T* __restrict__ Q, T* __restrict__ dX,
                                                   int W) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int pmax = g.pmax, ts = term_stride(pmax);
  T* ring = reinterpret_cast<T*>(smem);
  Term<T>* terms = reinterpret_cast<Term<T>*>(ring + (size_t)W * 32);
  Term<T>* stage = terms + ts;                                // [kStages][ts]
  T* qst = reinterpret_cast<T*>(stage + (size_t)kStages * ts);  // [kStages][32]
  const Block b = blocks[blockIdx.y];
  const int lane = threadIdx.x;
  const int m = blockIdx.x * 32 + lane;
  const bool act = m < g.N;
  const SolveOrder ord = solve_order(b, g.nlon);
  const int64_t cofs = b.row_off * g.N + (int64_t)(act ? m : 0) * b.nb;
  const T* qcol = Q + cofs;
  T* col = dX + cofs;
  const Term<T>* tab = pred + b.row_off * ts;
  OrderCursor ahead(ord, 0);  // the row staged next
  auto stage_t = [&](int slot, int t) {
    stage_row(stage + slot * ts, tab + (int64_t)t * ts, ts, lane);
    if (act) cp_async_small<sizeof(T)>(qst + slot * 32 + lane, qcol + ahead.loc());
    ahead.next();
  };
  for (int d = 0; d < kStages; ++d) {
    if (d < b.nb) stage_t(d, d);
    cp_async_commit();
  }
  int rt = 0, st = 0;
  OrderCursor cur(ord, 0);
  for (int t = 0; t < b.nb; ++t) {
    cp_async_wait_stages();
    __syncwarp();
    const int n = load_terms(terms, stage + st * ts, pmax, rt, W, -1, t, -1, lane);
    const T qv = act ? qst[st * 32 + lane] : T(0);
    __syncwarp();
    if (t + kStages < b.nb) stage_t(st, t + kStages);
    cp_async_commit();
    st = st + 1 == kStages ? 0 : st + 1;
    const T xv = sub_terms(qv, terms, n, ring, lane);
    ring[rt * 32 + lane] = xv;
    if (act) col[cur.loc()] = xv;
    cur.next();
    rt = rt + 1 == W ? 0 : rt + 1;
    __syncwarp();
  }
}

}  // namespace

template <typename T>
size_t dual_solve_smem(int W, int pmax) {
  return solve_smem<T>(W, pmax);
}

template <typename T>
size_t dual_obs_smem(int mb, int N) {
  return obs_smem<T>(mb, N);
}

template <typename TI, typename TC>
cudaError_t launch_dual_z(const Geom& g, const Block* blocks, int nblock, int nb_max, int mb_max,
                          const int2* dobs, const int64_t* dob_off, const int64_t* zoff,
                          const TI* Tg, const TI* Te, void* pred, void* succ, TC* Zb, int W,
                          cudaStream_t s, int* nk) {
  const dim3 gt((nb_max + 7) / 8, nblock);
  k_dual_terms<TI, TC><<<gt, 256, 0, s>>>(g, blocks, Tg, Te, (Term<TC>*)pred, (Term<TC>*)succ);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ++*nk;
  if (mb_max <= 0) return cudaSuccess;
  const size_t smem = solve_smem<TC>(W, g.pmax);
  e = cudaFuncSetAttribute(k_dual_z<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((mb_max + 31) / 32, nblock);
  k_dual_z<TC><<<grid, 32, smem, s>>>(g, blocks, dobs, dob_off, zoff, (const Term<TC>*)succ, Zb,
                                      W);
  ++*nk;
  return cudaGetLastError();
}

template <typename TI, typename TC>
cudaError_t launch_dual_obs(const Geom& g, const Block* blocks, int nblock, int mb_max,
                            const int2* dobs, const int64_t* dob_off, const int64_t* zoff,
                            const int32_t* obs_idx, int64_t m, const TI* Xb, const TI* y,
                            const TI* R, const TI* Zp, const TI* Dg, const TI* De, const TC* Zb,
                            TC* Wb, int32_t* status, cudaStream_t s) {
  if (mb_max <= 0) return cudaSuccess;
  const size_t smem = obs_smem<TC>(mb_max, g.N);
  cudaError_t e = cudaFuncSetAttribute(k_dual_obs<TI, TC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_dual_obs<TI, TC><<<nblock, kObsThreads, smem, s>>>(g, blocks, dobs, dob_off, zoff, obs_idx,
                                                       m, Xb, y, R, Zp, Dg, De, Zb, Wb, status);
  return cudaGetLastError();
}

template <typename TI, typename TC>
cudaError_t launch_dual_apply(const Geom& g, const Block* blocks, int nblock, int nb_max,
                              const int64_t* dob_off, const int64_t* zoff, const TC* Zb,
                              const TC* Wb, const TI* Dg, const TI* De, const void* pred, TC* Q,
                              TC* dX, int W, cudaStream_t s, int* nk) {
  const dim3 gq((nb_max + kQRows - 1) / kQRows, nblock, (g.N + kQMem - 1) / kQMem);
  k_dual_q<TI, TC><<<gq, 256, 0, s>>>(g, blocks, dob_off, zoff, Zb, Wb, Dg, De, Q);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = solve_smem<TC>(W, g.pmax);
  e = cudaFuncSetAttribute(k_dual_apply<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 ga((g.N + 31) / 32, nblock);
  k_dual_apply<TC><<<ga, 32, smem, s>>>(g, blocks, (const Term<TC>*)pred, Q, dX, W);
  *nk += 2;
  return cudaGetLastError();
}

size_t dual_table_bytes(size_t esize, int pmax) {
  return (esize == 8 ? sizeof(Term<double>) : sizeof(Term<float>)) * (size_t)term_stride(pmax);
}

template size_t dual_solve_smem<float>(int, int);
template size_t dual_solve_smem<double>(int, int);
template size_t dual_obs_smem<float>(int, int);
template size_t dual_obs_smem<double>(int, int);

#define INST(TI, TC)                                                                           \
  template cudaError_t launch_dual_z<TI, TC>(const Geom&, const Block*, int, int, int,         \
                                             const int2*, const int64_t*, const int64_t*,      \
                                             const TI*, const TI*, void*, void*, TC*, int,     \
                                             cudaStream_t, int*);                              \
  template cudaError_t launch_dual_obs<TI, TC>(                                                \
      const Geom&, const Block*, int, int, const int2*, const int64_t*, const int64_t*,        \
      const int32_t*, int64_t, const TI*, const TI*, const TI*, const TI*, const TI*,          \
      const TI*, const TC*, TC*, int32_t*, cudaStream_t);                                      \
  template cudaError_t launch_dual_apply<TI, TC>(const Geom&, const Block*, int, int,          \
                                                 const int64_t*, const int64_t*, const TC*,    \
                                                 const TC*, const TI*, const TI*, const void*, \
                                                 TC*, TC*, int, cudaStream_t, int*);
INST(float, float)
INST(float, double)
INST(double, double)
#undef INST

}  // namespace enkfmc
