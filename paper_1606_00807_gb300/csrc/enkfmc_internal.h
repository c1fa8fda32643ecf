// Internal declarations of libenkfmc: geometry shared by host tables and
// kernels, the handle, and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "enkfmc.h"

namespace enkfmc {

constexpr int kMaxVar = 16;

// Grid and localisation parameters (Section 2.2-2.3).  Passed by value to
// kernels.
struct Geom {
  int32_t nlon, nlat, nlev, nvar3, nvar2, nvar;
  int32_t r, vr, periodic, N, ldN;  // vr: effective vertical reach
  int32_t pmax;
  int32_t sm_count;      // SMs of the device (launch shapes; host side only)
  int32_t regress_cap;   // CTAs per SM of the regressions' grid-stride launch
  int32_t regress_kernel; // regression kernels: 0/1 tiled, 2 register, 3 paired (k_estimate.cu)
  int32_t plain_fp32;     // single precision without double-precision rows or blocks
  int64_t n;
  int64_t var_off[kMaxVar + 1];
  int32_t var_lev[kMaxVar];
};

// One (sub-domain, variable) block of the extended set.  Local index of a
// component: loc = (k * ey + (lat - lat_lo)) * ex + ((lon - lon_lo) mod nlon).
struct Block {
  int32_t id;                      // index of the block in the handle's list
  int32_t sub, var, nlev_b;
  int32_t lat_lo, ey, lon_lo, ex;  // extended box (ex == nlon: the whole ring)
  int32_t lat0, lat1, lon0, lon1;  // interior tile (absolute, lon1 <= nlon)
  int32_t hb;                      // half-bandwidth of A in local order
  int32_t nb;                      // rows of the block
  int32_t pair_base, npair;        // slot-pair list of the block's shape (-1: none)
  int64_t band_off;                // offset of the band in the band array
  int64_t row_off;                 // offset of the block's rows (Te, De, rhs rows)
};

// Dual form (k_dual.cu): rows the triangular solves stage ahead (cp.async),
// and their rings: rows less than Wn positions away in the near ring, rows Df
// to W - 1 away in the far ring of Wf = W - Df + kDualStages + 1 rows (Df = W:
// none).
constexpr int kDualStages = 8;
struct DualRings {
  int Wn, Df, Wf, W;
};

// ---------------------------------------------------------------------------
// Stencil slots.  Slot s of a row of T is the neighbour at offset
// (dk, dy, dx): first the vr lower levels ((2r+1)^2 each), then the r earlier
// latitude rows of the same level, then the r neighbours to the left on the
// same row, then (ring only) the r neighbours to the right that precede the
// component across the longitude seam.
// ---------------------------------------------------------------------------
__host__ __device__ inline int slot_count(int r, int vr, int periodic) {
  const int w = 2 * r + 1;
  return vr * w * w + r * w + r + (periodic ? r : 0);
}

__host__ __device__ inline void slot_offset(int s, int r, int vr, int& dk, int& dy, int& dx) {
  const int w = 2 * r + 1, box = w * w;
  if (s < vr * box) {
    dk = -vr + s / box;
    const int t = s % box;
    dy = t / w - r;
    dx = t % w - r;
    return;
  }
  s -= vr * box;
  dk = 0;
  if (s < r * w) {
    dy = -r + s / w;
    dx = s % w - r;
    return;
  }
  s -= r * w;
  dy = 0;
  dx = (s < r) ? (-r + s) : (1 + (s - r));
}

// a mod m in [0, m); one step without a division when |a| < 2m (the usual
// case: a longitude plus or minus less than one circle)
__host__ __device__ inline int imod(int a, int m) {
  if (a >= 0 && a < m) return a;
  if (a < 0 && a >= -m) return a + m;
  if (a >= m && a - m < m) return a - m;
  int x = a % m;
  return x < 0 ? x + m : x;
}

__host__ __device__ inline int var_of_label(const Geom& g, int64_t l) {
  int v = 0;
  while (v + 1 < g.nvar && l >= g.var_off[v + 1]) ++v;
  return v;
}

__host__ __device__ inline void label_coords(const Geom& g, int64_t l, int& v, int& k, int& y,
                                             int& x) {
  v = var_of_label(g, l);
  // labels are below 2^31 (the handle refuses larger grids): 32-bit divisions
  int rem = (int)(l - g.var_off[v]);
  const int plane = g.nlat * g.nlon;
  k = rem / plane;
  rem -= k * plane;
  y = rem / g.nlon;
  x = rem - y * g.nlon;
}

__host__ __device__ inline int64_t coords_label(const Geom& g, int v, int k, int y, int x) {
  return g.var_off[v] + ((int64_t)k * g.nlat + y) * g.nlon + x;
}

// Is the neighbour of component (v, k, y, x) at the offsets (dk, dy, dx) of a
// stencil slot a predecessor?  On success returns the neighbour's (k, y, x)
// with x on [0, nlon).
__host__ __device__ inline bool slot_pred_off(const Geom& g, int k, int y, int x, int dk, int dy,
                                              int dx, int& kq, int& yq, int& xq) {
  kq = k + dk;
  if (kq < 0) return false;
  yq = y + dy;
  if (yq < 0 || yq >= g.nlat) return false;
  xq = x + dx;
  if (dk == 0 && dy == 0) {
    if (dx < 0) return xq >= 0;  // left neighbour on the same row, no wrap
    if (!g.periodic || xq < g.nlon) return false;
    xq -= g.nlon;                 // right neighbour across the seam
    return true;
  }
  if (xq < 0 || xq >= g.nlon) {
    if (!g.periodic) return false;
    xq = imod(xq, g.nlon);
  }
  return true;
}

// Same, the offsets of slot s computed here.
__host__ __device__ inline bool slot_pred(const Geom& g, int k, int y, int x, int s, int& kq,
                                          int& yq, int& xq) {
  int dk, dy, dx;
  slot_offset(s, g.r, g.vr, dk, dy, dx);
  return slot_pred_off(g, k, y, x, dk, dy, dx, kq, yq, xq);
}

// Pair table of the typical row, whose predecessors are exactly the stencil
// slots 0..pf-1 (pf = pmax minus the seam slots of a periodic grid): entry pi of
// the lower triangle of the augmented Gram matrix (row-major, index pf = the row
// itself) -> {i | l << 8 | sel << 16, column h of the covariance table}, the
// entry being C[(sel ? q[l] : q[i]) * nH + h] for the labels q of the
// predecessors (the table holds the offset b - a of a pair (a, b) at row a when
// it lies in the stored half box, else at row b with the opposite offset).
__host__ __device__ inline int2 pair_table_entry(const Geom& g, int pf, int pi) {
  const int w4 = 4 * g.r + 1;
  const int B = (2 * g.vr + 1) * w4 * w4;
  const int t0 = (B - 1) / 2;
  int i = (int)((sqrtf(8.f * pi + 1.f) - 1.f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= pi) ++i;
  while (i * (i + 1) / 2 > pi) --i;
  const int l = pi - i * (i + 1) / 2;
  int dki = 0, dyi = 0, dxi = 0, dkl = 0, dyl = 0, dxl = 0;
  if (i < pf) slot_offset(i, g.r, g.vr, dki, dyi, dxi);
  if (l < pf) slot_offset(l, g.r, g.vr, dkl, dyl, dxl);
  const int t = ((dkl - dki + g.vr) * w4 + (dyl - dyi + 2 * g.r)) * w4 + (dxl - dxi + 2 * g.r);
  return t >= t0 ? make_int2(i | (l << 8), t - t0)
                 : make_int2(i | (l << 8) | (1 << 16), B - 1 - t - t0);
}

// Entry pi of the regressions' gather tables over the indices 0..pmax of a
// row's augmented Gram matrix in slot terms (slot s, or pmax for the row
// itself), lower triangle stored row by row: tri = i | l << 8 for the entry
// (i, l), l <= i; ftab = where the covariance of the pair of slots (i, l)
// sits in the covariance table: column h, and bit 15 set when it is read at
// the row of the entry's column (l) instead of its row (i), as for the offset
// b - a = off(l) - off(i) of the pair (a, b).  (pmax + 1)(pmax + 2) / 2 entries.
__host__ __device__ inline void gather_table_entry(const Geom& g, int pmax, int pi,
                                                   uint16_t& tri, uint16_t& ftab) {
  const int w4 = 4 * g.r + 1;
  const int B = (2 * g.vr + 1) * w4 * w4;
  const int t0 = (B - 1) / 2;
  int i = (int)((sqrtf(8.f * pi + 1.f) - 1.f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= pi) ++i;
  while (i * (i + 1) / 2 > pi) --i;
  const int l = pi - i * (i + 1) / 2;
  int dki = 0, dyi = 0, dxi = 0, dkl = 0, dyl = 0, dxl = 0;
  if (i < pmax) slot_offset(i, g.r, g.vr, dki, dyi, dxi);
  if (l < pmax) slot_offset(l, g.r, g.vr, dkl, dyl, dxl);
  const int t = ((dkl - dki + g.vr) * w4 + (dyl - dyi + 2 * g.r)) * w4 + (dxl - dxi + 2 * g.r);
  tri = (uint16_t)(i | (l << 8));
  ftab = (uint16_t)(t >= t0 ? t - t0 : ((B - 1 - t - t0) | 0x8000));
}

// Local position of absolute (yq, xq) in a block's extended box.
__host__ __device__ inline bool in_ext(const Block& b, int nlon, int yq, int xq, int& yy, int& xx) {
  yy = yq - b.lat_lo;
  if (yy < 0 || yy >= b.ey) return false;
  xx = imod(xq - b.lon_lo, nlon);
  return xx < b.ex;
}

__host__ __device__ inline bool in_interior(const Block& b, int y, int x) {
  return y >= b.lat0 && y < b.lat1 && x >= b.lon0 && x < b.lon1;
}

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace enkfmc

struct enkfmc_handle {
  enkfmc_problem prob;
  enkfmc::Geom g;
  cudaStream_t stream = nullptr;
  int device = 0;
  size_t esize = 8;  // bytes per floating-point element

  int32_t nsubx = 0, nsuby = 0, nsub = 0, nblock = 0, hb_max = 0, nb_max = 0;
  int64_t ext_rows = 0, halo_rows = 0, band_elems = 0;
  std::vector<enkfmc::Block> blocks;

  // device tables
  enkfmc::Block* d_blocks = nullptr;
  int4* d_pairs = nullptr;       // slot pairs per block shape, sorted by band diagonal
  int32_t* d_srcrow = nullptr;   // per extended row: global label (>= 0) or ~boundary row
  int2* d_ptab = nullptr;        // pair table of the typical row (pair_table_entry)
  uint16_t* d_gtab = nullptr;    // gather tables: tri, then ftab (gather_table_entry)
  bool pair_assembly = false;    // every block can use the pair lists
  int32_t npair_max = 0;         // longest pair list of a shape
  int32_t box_sum = 0;           // largest nlev_b + ey + ex of a block
  int32_t* d_halo = nullptr;     // halo rows: (block, local index) pairs
  int32_t* d_obs_of = nullptr;   // [n]: observation index of a component or -1
  int32_t* d_status = nullptr;   // [4]: first error code, pad, 64-bit info
  int64_t m = -1;

  // device workspace (element type by precision)
  void* d_U = nullptr;     // anomalies, component-major [n][ldN]
  void* d_C = nullptr;     // covariance table [n][cov_offset_count]
  double* d_U64 = nullptr; // FP32 problems with rows where 2p > N: FP64 anomalies
  double* d_C64 = nullptr; //   and FP64 covariance table for those rows
  const void* U_src = nullptr;  // Xb the anomalies and table were computed from
  void* d_Te = nullptr;    // boundary rows of T per block [ext_rows][pmax]
  void* d_De = nullptr;    // their D [ext_rows]
  void* d_band = nullptr;  // band of A, then of L
  void* d_invdiag = nullptr;  // 1 / L[c][c] per block row [ext_rows]
  void* d_rhs = nullptr;   // per block [N][nb] right-hand sides / increments
  void* d_res = nullptr;   // refinement: residual, then correction (FP32 path)
  void* d_vhi = nullptr;   // refinement scratch: (T dX) / D as double-float
  void* d_vlo = nullptr;
  bool tc_solve = false;  // FP32 solves on the tensor cores
  bool tc_chol = false;   // FP32 band Cholesky updates on the tensor cores
  bool refine_solve = false;
  int refine_steps = 0;   // refinement steps of every sub-domain solve (FP32)
  // FP32: blocks whose single-precision factorisation meets a non-positive
  // pivot are assembled, factored and solved again in double precision
  int32_t* d_bfail = nullptr;         // [nblock] failure flags of the last factorisation
  int32_t* d_fb_cnt = nullptr;        // pool views and ranges (12 ints, k_fallback_list)
  float* d_c1max = nullptr;           // [nblock] first refinement correction per block
  enkfmc::Block* d_fb_blocks = nullptr;  // [fb_cap] their entries, band_off in the pool
  double* d_fb_band = nullptr;        // [fb_cap][fb_stride] their bands and factors
  int32_t fb_cap = 0;
  int64_t fb_stride = 0;
  const void* T_assembled = nullptr;  // global T/D used by the last assemble
  const void* D_assembled = nullptr;
  const void* R_assembled = nullptr;  // and its observation variances
  bool assembled = false;
  int64_t workspace_bytes = 0;

  // host-cycle staging (allocated on first enkfmc_cycle_host), and the copy
  // stream that brings y, R and Z over while the estimate runs
  void *d_Xb = nullptr, *d_y = nullptr, *d_R = nullptr, *d_Z = nullptr, *d_Xa = nullptr;
  cudaStream_t c_stream = nullptr;
  cudaEvent_t c_start = nullptr, c_done = nullptr;

  // dual form (enkfmc_analyze_dual): per block the observations inside the
  // extended set in solve order {position, observation}, the offsets of the
  // blocks' lists and of their Z = T^-T H^T, and the Z and W buffers; built on
  // the first call after enkfmc_set_observations
  std::vector<int32_t> obs_of_host;  // [n] host copy of d_obs_of
  std::vector<int> p_ext;            // predecessors per extended row (-p-1: boundary)
  bool dual_ready = false;
  bool dual_fp64 = false;        // single-precision problem, dual arithmetic in double
  int32_t dual_mb_max = 0;
  enkfmc::DualRings dual_rings{1, 1, 1, 1};
  double* d_dx64 = nullptr;      // its increments [ext_rows][N] in double
  void *d_dpred = nullptr, *d_dsucc = nullptr;  // the solves' term tables
  void* d_dq = nullptr;          // Q = D Z W [ext_rows][N] (arithmetic type)
  int2* d_dobs = nullptr;
  int64_t* d_dob_off = nullptr;  // [nblock + 1]
  int64_t* d_dzoff = nullptr;    // [nblock]
  int64_t* d_dsoff = nullptr;    // [nblock] offsets of the packed S = Z^T D Z
  void* d_ds = nullptr;
  int32_t* d_obs_idx = nullptr;  // [m] observed component of each observation
  void* d_dz = nullptr;
  void* d_dw = nullptr;
  void *d_T = nullptr, *d_D = nullptr;

  // inputs of the last enkfmc_analyze (the reverse pass reads them again)
  const void *last_Xb = nullptr, *last_y = nullptr, *last_R = nullptr, *last_Z = nullptr;
  bool analyzed = false;
  // reverse-pass buffers (allocated on the first enkfmc_analyze_adjoint)
  void *d_lam = nullptr, *d_aT = nullptr, *d_bT = nullptr, *d_dxT = nullptr, *d_lamT = nullptr;
  void* d_W = nullptr;    // the reverse pass's right-hand side W (refinement)
  void *d_Eo = nullptr, *d_Fo = nullptr, *d_Vo = nullptr, *d_Ko = nullptr;  // per extended
                          // row: the regression adjoint's e, f, v (slots), kappa
  // filter cycling: squared-error partial sums (kSqGrid), and the fixed
  // buffers of the captured cycle (observations, perturbations, reference
  // state, squared error) with the stream it is captured on
  double* d_sqp = nullptr;
  void *d_fy = nullptr, *d_fZ = nullptr, *d_fx = nullptr;
  double* d_fsq = nullptr;
  cudaStream_t f_stream = nullptr;

  // kernel timing (events bracket each launch while enabled)
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  int64_t calls[ENKFMC_NKERNEL] = {};     // launcher calls per kind (always counted)
  int64_t kernels[ENKFMC_NKERNEL] = {};   // CUDA kernels those calls launched
  bool prof = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;

  // algorithmic work per launch
  double work_flops[ENKFMC_NKERNEL] = {};
  double work_bytes[ENKFMC_NKERNEL] = {};
};

namespace enkfmc {

// status codes written by kernels (first one wins)
__device__ inline void record_error(int32_t* status, int code, int64_t info) {
  if (atomicCAS(status, 0, code) == 0) {
    *reinterpret_cast<long long*>(status + 2) = (long long)info;
  }
}

// Right-hand side entry of Eq. 11 for an observed component:
// (y_o + sqrt(R_o) z - x^b) / R_o, written once so that every kernel that needs
// it rounds it the same way.
template <typename T>
__device__ __forceinline__ T rhs_entry(T yo, T sq, T z, T xb, T rinv) {
  return (fma(sq, z, yo) - xb) * rinv;
}

// Kernel launchers (implemented per .cu file).  T is float or double.  Each
// adds the number of kernels it launched to *nk.

// Offsets in the half box |dk| <= vr, |dlat|, |dlon| <= 2r with (dk, dlat, dlon) >= 0
// lexicographically: the columns of the covariance table C[n][count].
int cov_offset_count(int r, int vr);

// Precision rule of the estimate: a single-precision problem regresses the rows
// with 2p > N (p/N > 0.5, nearly singular Gram matrices) in double precision
// from FP64 anomalies and an FP64 covariance table.  True when some row of the
// problem can have 2p > N.
bool has_fp64_rows(const Geom& g, bool single);
// The estimate kernels can run this geometry (gather-table index widths,
// members, shared memory of the covariance table and of the regressions, in
// the problem's precision and, with FP64 rows, in double).
bool estimate_supported(const Geom& g, bool single);

// Validate a problem description and fill its geometry (shared by the handle
// and the allocation-free estimate): EINVAL for out-of-range sizes, label
// counts of 2^31 or more, or a geometry the estimate kernels cannot run.
enkfmc_status problem_geom(const enkfmc_problem& p, Geom& g);

// Statistics of one ensemble: anomalies U [n][ldN] and covariance table
// C [n][cov_offset_count] in the problem's precision; U64, C64 their FP64
// counterparts (single-precision problems with FP64 rows), else null.
template <typename T>
struct EstStats {
  T* U;
  T* C;
  double* U64;
  double* C64;
};

template <typename T>
cudaError_t launch_stat_anomalies(const Geom& g, const T* Xb, const EstStats<T>& st,
                                  cudaStream_t s, int* nk);
template <typename T>
cudaError_t launch_stat_covtables(const Geom& g, const EstStats<T>& st, cudaStream_t s,
                                  int* nk);
// Regressions of the global rows (halo null, nitems = n) or of the boundary
// rows listed in halo; status may be null.
template <typename T>
cudaError_t launch_regressions(const Geom& g, const EstStats<T>& st, const int32_t* halo,
                               int64_t nitems, const Block* blocks, T* Tout, T* Dout,
                               double ridge_c, int32_t* status, cudaStream_t s, int* nk);

// General band assembly (any block); TB the band's type (double for the
// double-precision pool, rng its device range {lo, hi}).
template <typename T, typename TB = T>
cudaError_t launch_assemble(const Geom& g, const Block* blocks, int nblock, int nb_max,
                            const T* Tg, const T* Dg, const T* Te, const T* De,
                            const int32_t* obs_of, const T* R, TB* band, int32_t* status,
                            cudaStream_t s, int hb_max, const int* rng = nullptr);

// Band assembly from per-shape slot-pair lists (blocks whose extended box does
// not wrap onto itself in longitude).
template <typename T>
cudaError_t launch_assemble_pairs(const Geom& g, const Block* blocks, int nblock, int nb_max,
                                  int hb_max, int npair_max, const int4* pairs,
                                  const int32_t* srcrow, const T* Tg, const T* Dg, const T* Te,
                                  const T* De, const int32_t* obs_of, const T* R, T* band,
                                  int box_sum, cudaStream_t s);
// Shared memory of one pair-assembly tile (element size esize; box_sum the
// largest nlev + ey + ex of a block).
size_t assemble_pairs_smem(size_t esize, int pmax, int hb_max, int r, int npair_max,
                           int box_sum);

// Factor every block in place; invdiag[row_off + c] = 1 / L[c][c] (may be null).
// rng (may be null): only the entries [rng[0], rng[1]) of `blocks` (a device
// range); bfail (may be null): a finite non-positive pivot sets bfail[block
// id] instead of recording ENOTSPD.
template <typename T>
cudaError_t launch_bandchol(const Block* blocks, int nblock, int hb_max, T* band, T* invdiag,
                            int32_t* status, cudaStream_t s, const int* rng = nullptr,
                            int* bfail = nullptr);
// The double-precision pool (k_fallback_list in k_band.cu): blocks flagged 1
// (append = 0, rebuilt) or flagged 2 (append = 1, added) into `cap` slots of
// `stride` elements; meta (12 ints) receives its solve views and ranges.
cudaError_t launch_fallback_list(const Block* blocks, int nblock, int* bfail, Block* pool,
                                 int* meta, int cap, int64_t stride, int32_t* status, int append,
                                 cudaStream_t s);
// Refinement convergence per block: phase 0 stores max|c| in c1max; phase 1
// flags 2 the blocks whose corrections predict an error above tau max|x|.
cudaError_t launch_ir_check(const Block* blocks, int nblock, int N, const float* c,
                            const float* x, float* c1max, int* bfail, float tau, int phase,
                            cudaStream_t s);

template <typename T>
cudaError_t launch_rhs(const Geom& g, const Block* blocks, int nblock, int nb_max,
                       const int32_t* obs_of, int64_t m, const T* Xb, const T* y, const T* R,
                       const T* Z, T* rhs, cudaStream_t s);

// L L^T X = B for N members per block; T the factor's type, TR the rhs's.
// pool (may be null): a view {0, live, lo, hi} of the double-precision pool
// (solve [lo, hi), zero the other live blocks' solutions); skip (may be
// null): blocks with skip[id] set are left alone.
template <typename T, typename TR>
cudaError_t launch_bandsolve(const Block* blocks, int nblock, int hb_max, int N, const T* band,
                             TR* rhs, cudaStream_t s, const int* pool = nullptr,
                             const int* skip = nullptr);

// Single-precision band solves with the panel updates on the tensor cores
// (k_band_tc.cu); usable when N <= 128 and the staged panels of a band of
// half-width hb_max fit in shared memory and TMEM.
bool bandsolve_tc_supported(int hb_max, int N);
// Single-precision band Cholesky with the trailing updates on the tensor cores
// (k_band_tc.cu); usable when 32 + hb_max <= 384.
bool bandchol_tc_supported(int hb_max);
cudaError_t launch_bandchol_tc(const Block* blocks, int nblock, int hb_max, float* band,
                               float* invdiag, int32_t* status, cudaStream_t s,
                               int* bfail = nullptr);
cudaError_t launch_bandsolve_tc(const Block* blocks, int nblock, int hb_max, int N,
                                const float* band, const float* invdiag, float* rhs,
                                int32_t* status, cudaStream_t s, const int* skip = nullptr);

// Xa = Xb + dX (+ dX2 when not null) on sub-domain interiors; TD the
// increments' type (float with double increments, or the same as T).
template <typename T, typename TD = T>
cudaError_t launch_writeback(const Geom& g, const Block* blocks, int nsubx, int sub_lon,
                             int sub_lat, const T* Xb, const TD* dX, const TD* dX2, T* Xa,
                             cudaStream_t s);

// Reverse pass (k_adjoint.cu and k_adj_regress in k_estimate.cu).
template <typename T>
cudaError_t launch_adj_seed(const Geom& g, const Block* blocks, int nblock, int nb_max,
                            const T* Xa_bar, T* W, cudaStream_t s);
template <typename T>
cudaError_t launch_adj_ab(const Geom& g, const Block* blocks, int nblock, int nb_max,
                          const T* Tg, const T* Te, const T* lam, const T* dX, const T* dX2,
                          T* aT, T* bT, T* dxT, T* lamT, cudaStream_t s);
// Reverse pass through the regressions of every extended row: stores the
// row's e, f ([ext row][ldN]), v ([ext row][pmax], in its slots) and kappa.
template <typename T>
cudaError_t launch_adj_regressions(const Geom& g, const Block* blocks, int nblock, int nb_max,
                                   const EstStats<T>& st, const T* Tg, const T* Dg, const T* Te,
                                   const T* De, const T* aT, const T* bT, const T* dxT,
                                   const T* lamT, const int2* ptab, const uint16_t* gtab, T* Eo,
                                   T* Fo, T* Vo, T* Ko, double ridge_c, int32_t* status,
                                   cudaStream_t s, int* nk);
// Ubar of every extended row from the stored terms of the rows that hold it,
// in slot order: Ub[row][ldN] (k_adjoint.cu).
template <typename T>
cudaError_t launch_adj_gather(const Geom& g, const Block* blocks, int nblock, int nb_max,
                              const T* Tg, const T* Te, const T* U, const T* Eo, const T* Fo,
                              const T* Vo, const T* Ko, T* Ub, cudaStream_t s);
// dL/dX^b, dL/dy, dL/d diag(R) of every component and observation from the
// blocks that hold it, in block order: the anomaly projection of the summed
// Ubar, dL/dX^a, and the observation terms (k_adjoint.cu).
template <typename T>
cudaError_t launch_adj_owner(const Geom& g, const Block* blocks, int nsubx, int nsuby,
                             int sub_lon, int sub_lat, const int32_t* obs_of, int64_t m,
                             const T* Xb, const T* y, const T* R, const T* Z, const T* Ub,
                             const T* lamT, const T* dxT, const T* Xa_bar, T* Xb_bar, T* y_bar,
                             T* R_bar, cudaStream_t s);

// Single-precision refinement residual res = rhs - A dX (two passes; vhi, vlo
// are scratch of the size of dX).  rhs: Eq. 11's observation term formed from
// Xb, y, R, Z, or rhs_in (per block [N][nb]) when it is not null.
cudaError_t launch_refine_residual(const Geom& g, const Block* blocks, int nblock, int nb_max,
                                   const int32_t* obs_of, int64_t m, const float* Xb,
                                   const float* y, const float* R, const float* Z,
                                   const float* Tg, const float* Dg, const float* Te,
                                   const float* De, const float* dX, float* vhi, float* vlo,
                                   const float* rhs_in, float* res, cudaStream_t s);
// y += x over `count` elements.
cudaError_t launch_accumulate(float* y, const float* x, int64_t count, cudaStream_t s);

// Dual form of the sub-domain analysis (k_dual.cu, Eq. 12-13): Z = T^-T H^T,
// then W = (R + Z^T D Z)^-1 (Y^s - H X^b), then dX = T^-1 D Z W into the
// increment buffer (the primal solve's layout).  dobs: per block its
// observations {solve position, observation index} from dob_off[block]; Z of
// a block [nb][mb] at zoff[block]; W of a block [mb][N] at N dob_off[block];
// W: the solves' ring (rows).
constexpr int kDualMaxSlots = 128;  // stencil slots the dual solves handle (4 per lane)
template <typename T>
size_t dual_solve_smem(const DualRings& rg, int pmax);
template <typename T>
size_t dual_obs_smem(int mb, int N);
// TI: the type of the inputs (T, D, X^b, y, R, Z); TC: the arithmetic and
// the type of Z, W and dX (double for single-precision problems with rows
// where 2p > N, whose T^-1 and R + Z^T D Z need it, else TI).
// Bytes of one row of the solves' term tables ({distance, coefficient} of the
// arithmetic type, pmax entries padded to 16 bytes).
size_t dual_table_bytes(size_t esize, int pmax);
// The term tables pred and succ ([ext rows][pmax] each, in solve order), then
// Z = T^-T H^T.
template <typename TI, typename TC>
cudaError_t launch_dual_z(const Geom& g, const Block* blocks, int nblock, int nb_max, int mb_max,
                          const int2* dobs, const int64_t* dob_off, const int64_t* zoff,
                          const TI* Tg, const TI* Te, void* pred, void* succ, TC* Zb,
                          const DualRings& rg, cudaStream_t s, int* nk);
// S = Z^T D Z (packed lower triangles at soff[block]), then (S + R) W =
// Y^s - H X^b.
template <typename TI, typename TC>
cudaError_t launch_dual_obs(const Geom& g, const Block* blocks, int nblock, int mb_max,
                            const int2* dobs, const int64_t* dob_off, const int64_t* zoff,
                            const int64_t* soff, const int32_t* obs_idx, int64_t m, const TI* Xb,
                            const TI* y, const TI* R, const TI* Zp, const TI* Dg, const TI* De,
                            const TC* Zb, TC* Sb, TC* Wb, int32_t* status, cudaStream_t s,
                            int* nk);
// Q = D Z W, then dX = T^-1 Q (Q and dX: [ext rows][N], members fastest).
template <typename TI, typename TC>
cudaError_t launch_dual_apply(const Geom& g, const Block* blocks, int nblock, int nb_max,
                              const int64_t* dob_off, const int64_t* zoff, const TC* Zb,
                              const TC* Wb, const TI* Dg, const TI* De, const void* pred, TC* Q,
                              TC* dX, const DualRings& rg, cudaStream_t s, int* nk);
// Xa = Xb + dX on the sub-domain interiors, dX members fastest.
template <typename TI, typename TC>
cudaError_t launch_dual_writeback(const Geom& g, const Block* blocks, int nsubx, int sub_lon,
                                  int sub_lat, const TI* Xb, const TC* dX, TI* Xa,
                                  cudaStream_t s);

// True when the CUDA-core band Cholesky and solves (k_band.cu) can launch for
// half-bandwidth hb with elements of esize bytes.
bool band_kernels_fit(int hb, size_t esize);

// filter cycling (k_cycle.cu): forecast operator and Eq. 18's squared error
constexpr int kSqGrid = 1024;  // blocks of the squared-error reduction (fixed order)
template <typename T>
cudaError_t launch_shift(const Geom& g, const T* X, T* Y, int nvec, int shift, double rho,
                         cudaStream_t s);
template <typename T>
cudaError_t launch_sqerr(const Geom& g, const T* Xa, const T* xref, double* part, double* out,
                         cudaStream_t s);

}  // namespace enkfmc
