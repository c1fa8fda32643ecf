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
//   k_dual_terms  per row and slot, the solves' terms {distance, coefficient};
//   k_dual_z      Z = T^-T H^T, one warp per 32 observation columns;
//   k_dual_syrk   Z^T D Z, a CTA per tile of the packed lower triangle;
//   k_dual_obs    S = R + Z^T D Z = L L^T, W = S^-1 (Y^s - H X^b), one CTA per
//                 block, in shared memory;
//   k_dual_q      Q = D (Z W), a tiled product;
//   k_dual_apply  dX = T^-1 Q, one warp per 32 members;
//   k_dual_writeback  Xa = Xb + dX on the interiors (Q and dX members fastest).
//
// Solve order.  T is unit lower triangular in label order (a predecessor has a
// smaller label).  Within a row segment of the block (one level, one
// latitude) the local index follows the longitude from the box's western edge,
// which passes the longitude seam when the box wraps; the solves therefore walk
// the rows in label order, position t: segment by segment, and inside a
// segment from the columns past the seam (x = 0, 1, ...) to those before it.
// A row and any of its predecessors lie less than W = (vr ey + r + 1) ex
// positions apart; a solve keeps the rows its next steps read in shared memory
// (the two rings below).
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
constexpr int kStages = kDualStages;

// The solves' rows in shared memory: a row's terms reach rows less than W
// positions away; those less than Wn away (its own level) come from the near
// ring [Wn][32], written as the solve goes; those Df or more away (the levels
// below, or above for the solve with T^T) from the far ring [Wf][32], Wf =
// W - Df + kStages + 1, into which each row is copied back from global memory
// kStages + 1 steps before it is first read (the rows between Wn and Df away are
// needed by no row).  Without such a gap (Df < Wn) the near ring holds all W
// rows and the far ring is unused (Df = W).
using Rings = DualRings;

// Shared memory of a triangular solve (one warp): the near and far rings, the
// compacted terms of the current and the next row [2][term_stride], the staged
// table rows [kStages][term_stride] and (forward solve) the staged q values
// [kStages][32].
template <typename T>
size_t solve_smem(const Rings& rg, int pmax) {
  return (size_t)(rg.Wn + rg.Wf) * 32 * sizeof(T) +
         (size_t)2 * term_stride(pmax) * sizeof(Term<T>) +
         (size_t)kStages * term_stride(pmax) * sizeof(Term<T>) + (size_t)kStages * 32 * sizeof(T);
}

// x - sum of v ring[at + lane] over the terms: four partial sums, unrolled by
// four, the next four terms read while the current four are summed (a fixed
// order, so the same bits on every run).
template <typename T>
__device__ __forceinline__ T sub_terms(T x, const Term<T>* terms, int n, const T* ring,
                                       int lane) {
  T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
  int i = 0;
  if (n >= 4) {
    Term<T> e0 = terms[0], e1 = terms[1], e2 = terms[2], e3 = terms[3];
    for (; i + 8 <= n; i += 4) {
      const Term<T> f0 = terms[i + 4], f1 = terms[i + 5], f2 = terms[i + 6], f3 = terms[i + 7];
      const T r0 = ring[e0.at + lane], r1 = ring[e1.at + lane], r2 = ring[e2.at + lane],
              r3 = ring[e3.at + lane];
      a0 = fma(e0.v, r0, a0);
      a1 = fma(e1.v, r1, a1);
      a2 = fma(e2.v, r2, a2);
      a3 = fma(e3.v, r3, a3);
      e0 = f0;
      e1 = f1;
      e2 = f2;
      e3 = f3;
    }
    a0 = fma(e0.v, ring[e0.at + lane], a0);
    a1 = fma(e1.v, ring[e1.at + lane], a1);
    a2 = fma(e2.v, ring[e2.at + lane], a2);
    a3 = fma(e3.v, ring[e3.at + lane], a3);
    i += 4;
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
  __shared__ signed char so[3 * kDualMaxSlots];
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

// The terms of one staged row compacted into `terms` with their offsets in
// the rings (the near ring first, then the far ring; slot x 32).  The row at
// distance d (sign +1: after t, -1: before): near slot rn + sign d (mod Wn),
// or far slot rf + sign (d - Df) (mod Wf), rn and rf the slots of the rows t
// and t + sign Df.  Only distances below Wn or in [Df, W), and with lim >= 0
// rows at positions up to lim, count.  Returns the number of terms.
template <typename T>
__device__ __forceinline__ int load_terms(Term<T>* terms, const Term<T>* row, int pmax,
                                          const Rings& rg, int rn, int rf, int sign, int t,
                                          int lim, int lane) {
  int n = 0;
#pragma unroll
  for (int q = 0; q < kSlotQ; ++q) {
    const int s = lane + 32 * q;
    Term<T> e{0, T(0)};
    if (s < pmax) e = row[s];
    const int d = e.at;
    const bool near = d > 0 && d < rg.Wn, far = d >= rg.Df && d < rg.W;
    const bool on = (near || far) && (lim < 0 || t + d <= lim);
    const unsigned mask = __ballot_sync(0xffffffffu, on);
    if (on) {
      int at;
      if (near) {
        int sl = rn + sign * d;
        if (sl >= rg.Wn) sl -= rg.Wn;
        if (sl < 0) sl += rg.Wn;
        at = sl;
      } else {
        int sl = rf + sign * (d - rg.Df);
        if (sl >= rg.Wf) sl -= rg.Wf;
        if (sl < 0) sl += rg.Wf;
        at = rg.Wn + sl;
      }
      terms[n + __popc(mask & ((1u << lane) - 1u))] = Term<T>{at * 32, e.v};
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
                                               T* __restrict__ Zb, const Rings rg) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int pmax = g.pmax, ts = term_stride(pmax);
  T* ring = reinterpret_cast<T*>(smem);  // near ring [Wn][32], then far ring [Wf][32]
  T* ringf = ring + (size_t)rg.Wn * 32;
  Term<T>* terms = reinterpret_cast<Term<T>*>(ring + (size_t)(rg.Wn + rg.Wf) * 32);  // [2][ts]
  Term<T>* stage = terms + 2 * ts;  // [kStages][ts]
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
  const bool has_far = rg.Df < rg.W;
  // far ring: row p (> t) is copied back from Z while the row p - Df + 1 is
  // summed (kStages + 1 steps before its first use), into slot p mod Wf;
  // farc walks those rows downwards from the first one within the block
  const int pf_hi = b.nb - 1;
  int pf = tlast - 1 - kStages + rg.Df;  // the far row copied back at step tlast
  OrderCursor farc(ord, max(0, min(pf, pf_hi)));
  int rfs = max(0, min(pf, pf_hi)) % rg.Wf;
  auto stage_far = [&](int p) {
    if (has_far && p >= 0 && p <= pf_hi) {
      if (act) cp_async_small<sizeof(T)>(ringf + rfs * 32 + lane, Z + (int64_t)farc.loc() * mb + c);
      farc.prev();
      rfs = rfs == 0 ? rg.Wf - 1 : rfs - 1;
    }
  };
  // rows tlast, tlast - 1, ... staged kStages ahead (stage of row t: (tlast - t) % kStages)
  for (int d = 0; d < kStages; ++d) {
    if (tlast - d >= 0) stage_row(stage + d * ts, tab + (int64_t)(tlast - d) * ts, ts, lane);
    cp_async_commit();
  }
  int rn = tlast % rg.Wn;             // near slot of position t
  int rf = (tlast + rg.Df) % rg.Wf;   // far slot of position t + Df
  // the terms of row tlast, then its stage refilled with row tlast - kStages
  cp_async_wait_stages();
  __syncwarp();
  int ncur = load_terms(terms, stage, pmax, rg, rn, rf, 1, tlast, tlast, lane);
  __syncwarp();
  if (tlast - kStages >= 0) stage_row(stage, tab + (int64_t)(tlast - kStages) * ts, ts, lane);
  cp_async_commit();
  int st = kStages > 1 ? 1 : 0;  // stage of row t - 1
  int cur = 0;
  OrderCursor pos(ord, tlast);
  for (int t = tlast; t >= 0; --t) {
    const int rn1 = rn == 0 ? rg.Wn - 1 : rn - 1, rf1 = rf == 0 ? rg.Wf - 1 : rf - 1;
    int nnext = 0;
    if (t > 0) {  // the next row's terms while this one is summed
      cp_async_wait_stages();
      __syncwarp();
      nnext = load_terms(terms + (1 - cur) * ts, stage + st * ts, pmax, rg, rn1, rf1, 1, t - 1,
                         tlast, lane);
      __syncwarp();
      if (t - 1 - kStages >= 0)
        stage_row(stage + st * ts, tab + (int64_t)(t - 1 - kStages) * ts, ts, lane);
      stage_far(pf);
      --pf;
      st = st + 1 == kStages ? 0 : st + 1;
    }
    cp_async_commit();
    const T z = sub_terms((t == tc) ? T(1) : T(0), terms + cur * ts, ncur, ring, lane);
    ring[rn * 32 + lane] = z;
    if (act) Z[(int64_t)pos.loc() * mb + c] = z;
    pos.prev();
    rn = rn1;
    rf = rf1;
    ncur = nnext;
    cur = 1 - cur;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// S = Z^T D Z, the lower triangle of each block's m_b x m_b matrix (packed row
// by row at soff[b]): a CTA per TILE x TILE tile of the lower triangle (64, or
// 32 when the blocks hold few observations), a thread per (TILE/16)^2 outputs,
// over the block's rows in chunks of 32 staged in shared memory (the D of
// each row folded into the left operand).
// ---------------------------------------------------------------------------
constexpr int kSyRows = 32;

template <typename TI, typename T, int TILE>
__global__ void __launch_bounds__(256) k_dual_syrk(const Geom g, const Block* __restrict__ blocks,
                                                   const int64_t* __restrict__ dob_off,
                                                   const int64_t* __restrict__ zoff,
                                                   const int64_t* __restrict__ soff,
                                                   const TI* __restrict__ Dg,
                                                   const TI* __restrict__ De,
                                                   const T* __restrict__ Zb, T* __restrict__ Sb) {
  constexpr int P = TILE / 16;  // outputs per thread in each direction
  __shared__ T A[kSyRows][TILE + 1];   // D z of the tile's row columns
  __shared__ T Bm[kSyRows][TILE + 1];  // z of its column columns
  const Block b = blocks[blockIdx.y];
  const int64_t o0 = dob_off[blockIdx.y];
  const int mb = (int)(dob_off[blockIdx.y + 1] - o0);
  const int nt = (mb + TILE - 1) / TILE;
  const int pr = blockIdx.x;
  if (pr >= nt * (nt + 1) / 2) return;
  int I = (int)((sqrtf(8.f * pr + 1.f) - 1.f) * 0.5f);
  while ((I + 1) * (I + 2) / 2 <= pr) ++I;
  while (I * (I + 1) / 2 > pr) --I;
  const int J = pr - I * (I + 1) / 2;
  const int i0 = I * TILE, l0 = J * TILE;
  const T* Z = Zb + zoff[blockIdx.y];
  const int tid = threadIdx.x, ti = tid >> 4, tl = tid & 15;  // outputs (i0 + ti + 16 a, l0 + tl + 16 e)
  T acc[P][P];
#pragma unroll
  for (int a = 0; a < P; ++a)
#pragma unroll
    for (int e = 0; e < P; ++e) acc[a][e] = T(0);
  for (int j0 = 0; j0 < b.nb; j0 += kSyRows) {
    __syncthreads();
    for (int e = tid; e < kSyRows * TILE; e += 256) {
      const int rr = e / TILE, cc = e - rr * TILE;
      const int j = j0 + rr;
      T za = T(0), zb = T(0);
      if (j < b.nb) {
        const T* zr = Z + (int64_t)j * mb;
        if (i0 + cc < mb) za = zr[i0 + cc];
        if (l0 + cc < mb) zb = zr[l0 + cc];
      }
      A[rr][cc] = za;
      Bm[rr][cc] = zb;
    }
    __syncthreads();
    if (tid < kSyRows) {  // fold D into A
      const int j = j0 + tid;
      T d = T(0);
      if (j < b.nb) {
        int k, y, x;
        local_coords(b, g.nlon, j, k, y, x);
        d = (T)block_d(g, b, k, y, x, j, Dg, De);
      }
      for (int cc = 0; cc < TILE; ++cc) A[tid][cc] *= d;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < kSyRows; ++rr) {
      T av[P], bv[P];
#pragma unroll
      for (int a = 0; a < P; ++a) av[a] = A[rr][ti + 16 * a];
#pragma unroll
      for (int e = 0; e < P; ++e) bv[e] = Bm[rr][tl + 16 * e];
#pragma unroll
      for (int a = 0; a < P; ++a)
#pragma unroll
        for (int e = 0; e < P; ++e) acc[a][e] = fma(av[a], bv[e], acc[a][e]);
    }
  }
  T* S = Sb + soff[blockIdx.y];
#pragma unroll
  for (int a = 0; a < P; ++a)
#pragma unroll
    for (int e = 0; e < P; ++e) {
      const int i = i0 + ti + 16 * a, l = l0 + tl + 16 * e;
      if (i < mb && l <= i) S[(int64_t)i * (i + 1) / 2 + l] = acc[a][e];
    }
}

// ---------------------------------------------------------------------------
// S + R = L L^T and W = (S + R)^-1 (Y^s - H X^b) for the block's
// observations; one CTA per block, in shared memory (S packed, the
// innovations then W [mb][N]).  Right-looking factorisation and solves, the
// CTA's threads over the trailing rows x members.  W: [mb][N] per block at
// N dob_off[b].  A non-positive or non-finite pivot records ENOTSPD (the
// block's W is then zero).
// ---------------------------------------------------------------------------
constexpr int kObsThreads = 256;

// Shared memory of k_dual_obs: S packed, then W.
template <typename T>
size_t obs_smem(int mb, int N) {
  return sizeof(T) * ((size_t)mb * (mb + 1) / 2 + 1 + (size_t)mb * N) + 16;
}

template <typename TI, typename T>
__global__ void __launch_bounds__(kObsThreads) k_dual_obs(
    const Geom g, const Block* __restrict__ blocks, const int2* __restrict__ dobs,
    const int64_t* __restrict__ dob_off, const int64_t* __restrict__ soff,
    const int32_t* __restrict__ obs_idx, int64_t mobs, const TI* __restrict__ Xb,
    const TI* __restrict__ y, const TI* __restrict__ R, const TI* __restrict__ Zp,
    const T* __restrict__ Sb, T* __restrict__ Wb, int32_t* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Block b = blocks[blockIdx.x];
  const int64_t o0 = dob_off[blockIdx.x];
  const int mb = (int)(dob_off[blockIdx.x + 1] - o0);
  if (mb == 0) return;
  const int N = g.N;
  const int ntri = mb * (mb + 1) / 2;
  T* S = reinterpret_cast<T*>(smem);  // packed lower triangle, S(i, l) at tri(i) + l
  T* Wm = S + ntri + 1;               // [mb][N]
  auto tri = [](int i) { return i * (i + 1) / 2; };
  __shared__ int bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kObsThreads / 32;
  if (tid == 0) bad = 0;
  const T* Sg = Sb + soff[blockIdx.x];
  for (int e = tid; e < ntri; e += kObsThreads) S[e] = Sg[e];
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
  // Cholesky: column k scaled, then the trailing lower triangle (a warp per
  // row, lanes over its columns)
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
  // L w = innovations: row c final, then subtracted from the rows below
  for (int c = 0; c < mb; ++c) {
    const T inv = T(1) / S[tri(c) + c];
    for (int m = tid; m < N; m += kObsThreads) Wm[c * N + m] *= inv;
    __syncthreads();
    for (int i = c + 1 + warp; i < mb; i += nw) {
      const T lic = S[tri(i) + c];
      for (int m = lane; m < N; m += 32) Wm[i * N + m] = fma(-lic, Wm[c * N + m], Wm[i * N + m]);
    }
    __syncthreads();
  }
  // L^T W = w: row c final, then subtracted from the rows above
  for (int c = mb - 1; c >= 0; --c) {
    const T inv = T(1) / S[tri(c) + c];
    for (int m = tid; m < N; m += kObsThreads) Wm[c * N + m] *= inv;
    __syncthreads();
    for (int i = warp; i < c; i += nw) {
      const T lci = S[tri(c) + i];
      for (int m = lane; m < N; m += 32) Wm[i * N + m] = fma(-lci, Wm[c * N + m], Wm[i * N + m]);
    }
    __syncthreads();
  }
  for (int e = tid; e < mb * N; e += kObsThreads) Wout[e] = Wm[e];
}

// ---------------------------------------------------------------------------
// Q = D (Z W) for every row of every block, members fastest
// (Q[(row_off + loc) N + m]): a CTA computes 128 rows x 32 members, a thread
// rows {rg + 32 a} x members {4 mg + e} (eight threads cover a row's 32
// members), over chunks of kQK observation columns staged in shared memory.
// ---------------------------------------------------------------------------
constexpr int kQRows = 128, kQMem = 32, kQK = 16;

template <typename TI, typename T>
__global__ void __launch_bounds__(256) k_dual_q(const Geom g, const Block* __restrict__ blocks,
                                                const int64_t* __restrict__ dob_off,
                                                const int64_t* __restrict__ zoff,
                                                const T* __restrict__ Zb, const T* __restrict__ Wb,
                                                const TI* __restrict__ Dg,
                                                const TI* __restrict__ De, T* __restrict__ Q) {
  __shared__ T Zs[kQRows][kQK + 1];
  __shared__ __align__(16) T Ws[kQK][kQMem];
  const Block b = blocks[blockIdx.y];
  const int r0 = blockIdx.x * kQRows;
  if (r0 >= b.nb) return;
  const int m0 = blockIdx.z * kQMem;
  const int64_t o0 = dob_off[blockIdx.y];
  const int mb = (int)(dob_off[blockIdx.y + 1] - o0);
  const int N = g.N;
  const int tid = threadIdx.x, mg = tid & 7, rg = tid >> 3;
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
      for (int e = 0; e < 4; ++e) w[e] = Ws[kk][4 * mg + e];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const T z = Zs[rg + 32 * a][kk];
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[a][e] = fma(z, w[e], acc[a][e]);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int j = r0 + rg + 32 * a;
    if (j >= b.nb) continue;
    int k, y, x;
    local_coords(b, g.nlon, j, k, y, x);
    const T d = (T)block_d(g, b, k, y, x, j, Dg, De);
    T* out = Q + (b.row_off + j) * N;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int m = m0 + 4 * mg + e;
      if (m < N) out[m] = d * acc[a][e];
    }
  }
}

// ---------------------------------------------------------------------------
// Xa[m][l] = Xb[m][l] + dX[(row_off + loc) N + m] for the sub-domain whose
// interior holds l (Eq. 10): a CTA per 32 components x 32 members, read along
// the members and written along the components through a shared tile.
// ---------------------------------------------------------------------------
template <typename TI, typename T>
__global__ void __launch_bounds__(256) k_dual_writeback(const Geom g,
                                                        const Block* __restrict__ blocks,
                                                        int nsubx, int sub_lon, int sub_lat,
                                                        const TI* __restrict__ Xb,
                                                        const T* __restrict__ dX,
                                                        TI* __restrict__ Xa) {
  __shared__ T tile[32][33];
  const int64_t l0 = (int64_t)blockIdx.x * 32;
  const int m0 = blockIdx.y * 32;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int i = wp; i < 32; i += 8) {  // component l0 + i, member m0 + lane
    const int64_t l = l0 + i;
    T v = T(0);
    if (l < g.n && m0 + lane < g.N) {
      int var, k, y, x;
      label_coords(g, l, var, k, y, x);
      const int sub = (y / sub_lat) * nsubx + x / sub_lon;
      const Block& b = blocks[sub * g.nvar + var];
      const int loc = (k * b.ey + (y - b.lat_lo)) * b.ex + imod(x - b.lon_lo, g.nlon);
      v = dX[(b.row_off + loc) * g.N + m0 + lane];
    }
    tile[i][lane] = v;
  }
  __syncthreads();
  for (int i = wp; i < 32; i += 8) {  // member m0 + i, component l0 + lane
    const int m = m0 + i;
    const int64_t l = l0 + lane;
    if (m < g.N && l < g.n) {
      const int64_t e = (int64_t)m * g.n + l;
      Xa[e] = Xb[e] + (TI)tile[lane][i];
    }
  }
}

// ---------------------------------------------------------------------------
// dX = T^-1 Q, forward in label order: x_j = q_j - sum_s T[j][s]
// x_{pred_s(j)}; a warp per 32 members of a block (Q and dX members fastest).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(32) k_dual_apply(const Geom g, const Block* __restrict__ blocks,
                                                   const Term<T>* __restrict__ pred,
                                                   const T* __restrict__ Q, T* __restrict__ dX,
                                                   const Rings rg) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int pmax = g.pmax, ts = term_stride(pmax);
  T* ring = reinterpret_cast<T*>(smem);  // near ring [Wn][32], then far ring [Wf][32]
  T* ringf = ring + (size_t)rg.Wn * 32;
  Term<T>* terms = reinterpret_cast<Term<T>*>(ring + (size_t)(rg.Wn + rg.Wf) * 32);  // [2][ts]
  Term<T>* stage = terms + 2 * ts;                            // [kStages][ts]
  T* qst = reinterpret_cast<T*>(stage + (size_t)kStages * ts);  // [kStages][32]
  const Block b = blocks[blockIdx.y];
  const int lane = threadIdx.x;
  const int m = blockIdx.x * 32 + lane;
  const bool act = m < g.N;
  const SolveOrder ord = solve_order(b, g.nlon);
  // Q and dX: [(row_off + loc) N + m], the lanes' members side by side
  const int N = g.N, mm = act ? m : 0;
  const T* qcol = Q + b.row_off * N + mm;
  T* col = dX + b.row_off * N + mm;
  const Term<T>* tab = pred + b.row_off * ts;
  OrderCursor ahead(ord, 0);  // the row staged next
  auto stage_t = [&](int slot, int t) {
    stage_row(stage + slot * ts, tab + (int64_t)t * ts, ts, lane);
    if (act) cp_async_small<sizeof(T)>(qst + slot * 32 + lane, qcol + (int64_t)ahead.loc() * N);
    ahead.next();
  };
  for (int d = 0; d < kStages; ++d) {
    if (d < b.nb) stage_t(d, d);
    cp_async_commit();
  }
  // far ring: row p (< t) is copied back from dX while the row p + Df - 1 is
  // summed (kStages + 1 steps before its first use; rows are final there:
  // Df > kStages + 1), into slot p mod Wf
  const bool has_far = rg.Df < rg.W;
  int pf = kStages + 1 - rg.Df;  // the far row copied back at step 0
  OrderCursor farc(ord, 0);
  int rfs = 0;
  auto stage_far = [&](int p) {
    if (has_far && p >= 0) {
      if (act) cp_async_small<sizeof(T)>(ringf + rfs * 32 + lane, col + (int64_t)farc.loc() * N);
      farc.next();
      rfs = rfs + 1 == rg.Wf ? 0 : rfs + 1;
    }
  };
  int rn = 0, rf = (rg.Wf - rg.Df % rg.Wf) % rg.Wf;  // slots of positions t and t - Df
  // the terms and q of row 0, then its stage refilled with row kStages
  cp_async_wait_stages();
  __syncwarp();
  int ncur = load_terms(terms, stage, pmax, rg, rn, rf, -1, 0, -1, lane);
  T qcur = act ? qst[lane] : T(0);
  __syncwarp();
  if (kStages < b.nb) stage_t(0, kStages);
  cp_async_commit();
  int st = kStages > 1 ? 1 : 0;  // stage of row t + 1
  int cur = 0;
  OrderCursor pos(ord, 0);
  for (int t = 0; t < b.nb; ++t) {
    const int rn1 = rn + 1 == rg.Wn ? 0 : rn + 1, rf1 = rf + 1 == rg.Wf ? 0 : rf + 1;
    int nnext = 0;
    T qnext = T(0);
    if (t + 1 < b.nb) {  // the next row's terms while this one is summed
      cp_async_wait_stages();
      __syncwarp();
      nnext = load_terms(terms + (1 - cur) * ts, stage + st * ts, pmax, rg, rn1, rf1, -1, t + 1,
                         -1, lane);
      qnext = act ? qst[st * 32 + lane] : T(0);
      __syncwarp();
      if (t + 1 + kStages < b.nb) stage_t(st, t + 1 + kStages);
      stage_far(pf);
      ++pf;
      st = st + 1 == kStages ? 0 : st + 1;
    }
    cp_async_commit();
    const T xv = sub_terms(qcur, terms + cur * ts, ncur, ring, lane);
    ring[rn * 32 + lane] = xv;
    if (act) col[(int64_t)pos.loc() * N] = xv;
    pos.next();
    rn = rn1;
    rf = rf1;
    ncur = nnext;
    qcur = qnext;
    cur = 1 - cur;
    __syncwarp();
  }
}

}  // namespace

template <typename T>
size_t dual_solve_smem(const DualRings& rg, int pmax) {
  return solve_smem<T>(rg, pmax);
}

template <typename T>
size_t dual_obs_smem(int mb, int N) {
  return obs_smem<T>(mb, N);
}

template <typename TI, typename TC>
cudaError_t launch_dual_z(const Geom& g, const Block* blocks, int nblock, int nb_max, int mb_max,
                          const int2* dobs, const int64_t* dob_off, const int64_t* zoff,
                          const TI* Tg, const TI* Te, void* pred, void* succ, TC* Zb,
                          const DualRings& rg, cudaStream_t s, int* nk) {
  const dim3 gt((nb_max + 7) / 8, nblock);
  k_dual_terms<TI, TC><<<gt, 256, 0, s>>>(g, blocks, Tg, Te, (Term<TC>*)pred, (Term<TC>*)succ);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ++*nk;
  if (mb_max <= 0) return cudaSuccess;
  const size_t smem = solve_smem<TC>(rg, g.pmax);
  e = cudaFuncSetAttribute(k_dual_z<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((mb_max + 31) / 32, nblock);
  k_dual_z<TC><<<grid, 32, smem, s>>>(g, blocks, dobs, dob_off, zoff, (const Term<TC>*)succ, Zb,
                                      rg);
  ++*nk;
  return cudaGetLastError();
}

template <typename TI, typename TC>
cudaError_t launch_dual_obs(const Geom& g, const Block* blocks, int nblock, int mb_max,
                            const int2* dobs, const int64_t* dob_off, const int64_t* zoff,
                            const int64_t* soff, const int32_t* obs_idx, int64_t m, const TI* Xb,
                            const TI* y, const TI* R, const TI* Zp, const TI* Dg, const TI* De,
                            const TC* Zb, TC* Sb, TC* Wb, int32_t* status, cudaStream_t s,
                            int* nk) {
  if (mb_max <= 0) return cudaSuccess;
  if (mb_max <= 128) {
    const int nt = (mb_max + 31) / 32;
    k_dual_syrk<TI, TC, 32><<<dim3(nt * (nt + 1) / 2, nblock), 256, 0, s>>>(
        g, blocks, dob_off, zoff, soff, Dg, De, Zb, Sb);
  } else {
    const int nt = (mb_max + 63) / 64;
    k_dual_syrk<TI, TC, 64><<<dim3(nt * (nt + 1) / 2, nblock), 256, 0, s>>>(
        g, blocks, dob_off, zoff, soff, Dg, De, Zb, Sb);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = obs_smem<TC>(mb_max, g.N);
  e = cudaFuncSetAttribute(k_dual_obs<TI, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  k_dual_obs<TI, TC><<<nblock, kObsThreads, smem, s>>>(g, blocks, dobs, dob_off, soff, obs_idx,
                                                       m, Xb, y, R, Zp, Sb, Wb, status);
  *nk += 2;
  return cudaGetLastError();
}

template <typename TI, typename TC>
cudaError_t launch_dual_apply(const Geom& g, const Block* blocks, int nblock, int nb_max,
                              const int64_t* dob_off, const int64_t* zoff, const TC* Zb,
                              const TC* Wb, const TI* Dg, const TI* De, const void* pred, TC* Q,
                              TC* dX, const DualRings& rg, cudaStream_t s, int* nk) {
  const dim3 gq((nb_max + kQRows - 1) / kQRows, nblock, (g.N + kQMem - 1) / kQMem);
  k_dual_q<TI, TC><<<gq, 256, 0, s>>>(g, blocks, dob_off, zoff, Zb, Wb, Dg, De, Q);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = solve_smem<TC>(rg, g.pmax);
  e = cudaFuncSetAttribute(k_dual_apply<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 ga((g.N + 31) / 32, nblock);
  k_dual_apply<TC><<<ga, 32, smem, s>>>(g, blocks, (const Term<TC>*)pred, Q, dX, rg);
  *nk += 2;
  return cudaGetLastError();
}

template <typename TI, typename TC>
cudaError_t launch_dual_writeback(const Geom& g, const Block* blocks, int nsubx, int sub_lon,
                                  int sub_lat, const TI* Xb, const TC* dX, TI* Xa,
                                  cudaStream_t s) {
  const dim3 grid((unsigned)((g.n + 31) / 32), (g.N + 31) / 32);
  k_dual_writeback<TI, TC><<<grid, 256, 0, s>>>(g, blocks, nsubx, sub_lon, sub_lat, Xb, dX, Xa);
  return cudaGetLastError();
}

size_t dual_table_bytes(size_t esize, int pmax) {
  return (esize == 8 ? sizeof(Term<double>) : sizeof(Term<float>)) * (size_t)term_stride(pmax);
}

template size_t dual_solve_smem<float>(const DualRings&, int);
template size_t dual_solve_smem<double>(const DualRings&, int);
template size_t dual_obs_smem<float>(int, int);
template size_t dual_obs_smem<double>(int, int);

#define INST(TI, TC)                                                                           \
  template cudaError_t launch_dual_z<TI, TC>(const Geom&, const Block*, int, int, int,         \
                                             const int2*, const int64_t*, const int64_t*,      \
                                             const TI*, const TI*, void*, void*, TC*,          \
                                             const DualRings&, cudaStream_t, int*);            \
  template cudaError_t launch_dual_obs<TI, TC>(                                                \
      const Geom&, const Block*, int, int, const int2*, const int64_t*, const int64_t*,        \
      const int64_t*, const int32_t*, int64_t, const TI*, const TI*, const TI*, const TI*,     \
      const TI*, const TI*, const TC*, TC*, TC*, int32_t*, cudaStream_t, int*);                \
  template cudaError_t launch_dual_apply<TI, TC>(const Geom&, const Block*, int, int,          \
                                                 const int64_t*, const int64_t*, const TC*,    \
                                                 const TC*, const TI*, const TI*, const void*, \
                                                 TC*, TC*, const DualRings&, cudaStream_t,     \
                                                 int*);                                        \
  template cudaError_t launch_dual_writeback<TI, TC>(const Geom&, const Block*, int, int, int,  \
                                                     const TI*, const TC*, TI*, cudaStream_t);
INST(float, float)
INST(float, double)
INST(double, double)
#undef INST

}  // namespace enkfmc
