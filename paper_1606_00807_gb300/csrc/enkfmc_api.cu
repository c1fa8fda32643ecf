// Host side of the C ABI: problem validation, geometry tables (sub-domains,
// blocks, boundary rows, band widths), workspace, and the call sequence of
// one analysis (Algorithm 2: estimate, assemble, analyze).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "enkfmc_internal.h"

using namespace enkfmc;

namespace {

#define CUDA_TRY(expr)                                  \
  do {                                                  \
    cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) {                            \
      (void)cudaGetLastError();                         \
      return e_ == cudaErrorMemoryAllocation ? ENKFMC_ENOMEM : ENKFMC_ECUDA; \
    }                                                   \
  } while (0)

template <typename P>
enkfmc_status dalloc(enkfmc_handle* h, P** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    *ptr = nullptr;
    return e == cudaErrorMemoryAllocation ? ENKFMC_ENOMEM : ENKFMC_ECUDA;
  }
  h->workspace_bytes += (int64_t)bytes;
  return ENKFMC_OK;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

bool is_fp64(const enkfmc_handle* h) { return h->prob.precision == ENKFMC_FP64; }

// Half-bandwidth of A on one block: the widest spread, in local order, of a
// row of T together with its predecessors inside the extended box.
int block_bandwidth(const Geom& g, const Block& b) {
  int hb = 0;
  for (int loc = 0; loc < b.nb; ++loc) {
    const int plane = b.ey * b.ex;
    const int k = loc / plane;
    const int yy = (loc - k * plane) / b.ex;
    const int xx = loc - k * plane - yy * b.ex;
    const int y = b.lat_lo + yy, x = imod(b.lon_lo + xx, g.nlon);
    int lo = loc, hi = loc;
    for (int s = 0; s < g.pmax; ++s) {
      int kq, yq, xq, yyq, xxq;
      if (!slot_pred(g, k, y, x, s, kq, yq, xq)) continue;
      if (!in_ext(b, g.nlon, yq, xq, yyq, xxq)) continue;
      const int lq = (kq * b.ey + yyq) * b.ex + xxq;
      lo = std::min(lo, lq);
      hi = std::max(hi, lq);
    }
    hb = std::max(hb, hi - lo);
  }
  return hb;
}

void compute_work(enkfmc_handle* h, const std::vector<int>& p_global,
                  const std::vector<int>& p_ext);

}  // namespace

namespace enkfmc {

enkfmc_status problem_geom(const enkfmc_problem& p, Geom& g) {
  const int nvar = p.nvar_3d + p.nvar_2d;
  if (p.nlon < 1 || p.nlat < 1 || p.nlev < 1 || p.nvar_3d < 0 || p.nvar_2d < 0 || nvar < 1 ||
      nvar > kMaxVar || p.r < 0 || p.vert_reach < 0 || p.N < 2 || p.N > 128 || p.sub_lon < 1 ||
      p.sub_lat < 1 || !(p.ridge_c >= 0.0) || p.r > 16)
    return ENKFMC_EINVAL;
  if (p.precision != ENKFMC_FP64 && p.precision != ENKFMC_FP32) return ENKFMC_EINVAL;
  if (p.lon_periodic && p.nlon < 2 * p.r + 1) return ENKFMC_EINVAL;
  // every extent and product below 2^31 components before the label arithmetic
  // (32-bit labels in the kernels) and any buffer size is formed
  const int64_t lim = ((int64_t)1 << 31) - 1;
  if ((int64_t)p.nlon * p.nlat > lim || (int64_t)p.nlon * p.nlat * p.nlev > lim) return ENKFMC_EINVAL;
  std::memset(&g, 0, sizeof(g));
  g.nlon = p.nlon;
  g.nlat = p.nlat;
  g.nlev = p.nlev;
  g.nvar3 = p.nvar_3d;
  g.nvar2 = p.nvar_2d;
  g.nvar = nvar;
  g.r = p.r;
  g.vr = p.nvar_3d > 0 ? std::min(p.vert_reach, p.nlev - 1) : 0;
  g.periodic = p.lon_periodic ? 1 : 0;
  g.N = p.N;
  g.ldN = (p.N + 3) / 4 * 4;
  // at most 255 stencil slots (checked again by estimate_supported): bounds vr
  // before slot_count multiplies it
  if ((int64_t)g.vr * (2 * g.r + 1) * (2 * g.r + 1) > 255) return ENKFMC_EINVAL;
  g.pmax = slot_count(g.r, g.vr, g.periodic);
  int64_t off = 0;
  for (int v = 0; v < nvar; ++v) {
    g.var_off[v] = off;
    g.var_lev[v] = v < p.nvar_3d ? p.nlev : 1;
    off += (int64_t)g.var_lev[v] * p.nlat * p.nlon;
    if (off > lim) return ENKFMC_EINVAL;
  }
  g.var_off[nvar] = off;
  g.n = off;
  if (!estimate_supported(g, p.precision != ENKFMC_FP64)) return ENKFMC_EINVAL;
  g.sm_count = 0;  // filled where a device is at hand
  g.regress_cap = 0;
  g.regress_kernel = 0;
  g.plain_fp32 = (p.flags & ENKFMC_FLAG_PLAIN_FP32) ? 1 : 0;
  return ENKFMC_OK;
}

}  // namespace enkfmc

namespace {

enkfmc_status build(enkfmc_handle* h) {
  const enkfmc_problem& p = h->prob;
  if (p.flags & ~(ENKFMC_FLAG_NO_SOLVE_REFINEMENT | ENKFMC_FLAG_SIMT_BAND |
                  ENKFMC_FLAG_PLAIN_FP32 | ENKFMC_FLAG_REFINE_MASK))
    return ENKFMC_EINVAL;
  Geom& g = h->g;
  enkfmc_status gst = problem_geom(p, g);
  if (gst) return gst;
  if (cudaDeviceGetAttribute(&g.sm_count, cudaDevAttrMultiProcessorCount, h->device) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    g.sm_count = 0;
  }
  const int nvar = g.nvar;
  h->esize = is_fp64(h) ? sizeof(double) : sizeof(float);
  h->refine_solve = !is_fp64(h) && !(p.flags & ENKFMC_FLAG_NO_SOLVE_REFINEMENT);
  if (h->refine_solve) {
    // one step, or four where the regressions are nearly singular (2p > N): the
    // small residual variances D_j make A ill-conditioned there (condition
    // numbers near 1e8 at N = 40, r = 2), and each step gains about one digit
    const int req = (p.flags & ENKFMC_FLAG_REFINE_MASK) >> 8;
    h->refine_steps = req ? req : (has_fp64_rows(g, true) ? 4 : 1);
  }

  // sub-domains and blocks (Section 3, Fig. 3)
  h->nsuby = (p.nlat + p.sub_lat - 1) / p.sub_lat;
  h->nsubx = (p.nlon + p.sub_lon - 1) / p.sub_lon;
  h->nsub = h->nsubx * h->nsuby;
  h->nblock = h->nsub * nvar;
  h->blocks.clear();
  h->blocks.reserve(h->nblock);
  int64_t row_off = 0, band_off = 0;
  h->hb_max = 0;
  h->nb_max = 0;
  std::vector<int32_t> halo;
  for (int sy = 0; sy < h->nsuby; ++sy) {
    for (int sx = 0; sx < h->nsubx; ++sx) {
      Block b{};
      b.sub = sy * h->nsubx + sx;
      b.lat0 = sy * p.sub_lat;
      b.lat1 = std::min(p.nlat, b.lat0 + p.sub_lat);
      b.lon0 = sx * p.sub_lon;
      b.lon1 = std::min(p.nlon, b.lon0 + p.sub_lon);
      b.lat_lo = std::max(0, b.lat0 - p.r);
      b.ey = std::min(p.nlat, b.lat1 + p.r) - b.lat_lo;
      if (g.periodic) {
        b.ex = std::min(b.lon1 - b.lon0 + 2 * p.r, p.nlon);
        b.lon_lo = imod(b.lon0 - p.r, p.nlon);
      } else {
        b.lon_lo = std::max(0, b.lon0 - p.r);
        b.ex = std::min(p.nlon, b.lon1 + p.r) - b.lon_lo;
      }
      for (int v = 0; v < nvar; ++v) {
        Block bb = b;
        bb.var = v;
        bb.nlev_b = g.var_lev[v];
        bb.nb = bb.nlev_b * bb.ey * bb.ex;
        bb.hb = block_bandwidth(g, bb);
        bb.row_off = row_off;
        bb.band_off = band_off;
        const int blk = (int)h->blocks.size();
        bb.id = blk;
        for (int loc = 0; loc < bb.nb; ++loc) {
          const int plane = bb.ey * bb.ex;
          const int k = loc / plane;
          const int yy = (loc - k * plane) / bb.ex;
          const int xx = loc - k * plane - yy * bb.ex;
          (void)k;
          if (!in_interior(bb, bb.lat_lo + yy, imod(bb.lon_lo + xx, p.nlon))) {
            halo.push_back(blk);
            halo.push_back(loc);
          }
        }
        row_off += bb.nb;
        band_off += (int64_t)bb.nb * (bb.hb + 1);
        h->hb_max = std::max(h->hb_max, bb.hb);
        h->nb_max = std::max(h->nb_max, bb.nb);
        h->blocks.push_back(bb);
      }
    }
  }
  h->ext_rows = row_off;
  h->band_elems = band_off;
  h->halo_rows = (int64_t)halo.size() / 2;
  // within each block, the boundary rows in order of their predecessor count
  // (stable): rows are independent, and neighbouring items with the same count
  // let a warp run two of them in step (k_regress_pair)
  {
    std::vector<int> pcount(h->halo_rows);
    for (int64_t it = 0; it < h->halo_rows; ++it) {
      const Block& bb = h->blocks[halo[2 * it]];
      const int loc = halo[2 * it + 1];
      const int plane = bb.ey * bb.ex;
      const int k = loc / plane;
      const int yy = (loc - k * plane) / bb.ex;
      const int xx = loc - k * plane - yy * bb.ex;
      const int y = bb.lat_lo + yy, x = imod(bb.lon_lo + xx, g.nlon);
      int cnt = 0;
      for (int s = 0; s < g.pmax; ++s) {
        int dk, dy, dx, kq, yq, xq, yy2, xx2;
        slot_offset(s, g.r, g.vr, dk, dy, dx);
        if (slot_pred_off(g, k, y, x, dk, dy, dx, kq, yq, xq) &&
            in_ext(bb, g.nlon, yq, xq, yy2, xx2))
          ++cnt;
      }
      pcount[it] = cnt;
    }
    std::vector<int64_t> order(h->halo_rows);
    for (int64_t it = 0; it < h->halo_rows; ++it) order[it] = it;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t c) {
      const int ba = halo[2 * a], bc = halo[2 * c];
      return ba != bc ? ba < bc : pcount[a] < pcount[c];
    });
    std::vector<int32_t> sorted(halo.size());
    for (int64_t i = 0; i < h->halo_rows; ++i) {
      sorted[2 * i] = halo[2 * order[i]];
      sorted[2 * i + 1] = halo[2 * order[i] + 1];
    }
    halo.swap(sorted);
  }
  // the CUDA-core band kernels (FP64 problems, the single-precision path when
  // the tensor-core kernels do not apply, and the double-precision pool of an
  // FP32 problem) hold a panel and a window of the band in shared memory:
  // refuse bands too wide for them
  if (!band_kernels_fit(h->hb_max, h->esize)) return ENKFMC_EINVAL;
  if (!is_fp64(h) && !g.plain_fp32 && !band_kernels_fit(h->hb_max, sizeof(double)))
    return ENKFMC_EINVAL;
  h->tc_solve = !is_fp64(h) && !(p.flags & ENKFMC_FLAG_SIMT_BAND) &&
               bandsolve_tc_supported(h->hb_max, p.N);
  h->tc_chol = !is_fp64(h) && !(p.flags & ENKFMC_FLAG_SIMT_BAND) &&
               bandchol_tc_supported(h->hb_max);

  // slot-pair lists per block shape for the band assembly: pairs (s1, s2) of
  // stencil slots (index pmax = the row itself) with local offsets
  // o(s1) - o(s2) = d, 0 <= d <= hb, sorted by d.  Row j = c - o(s2) adds
  // T[j][s1] T[j][s2] / D[j] to A[c + d][c].  Each record is
  // {s1, s2, o(s2), d}.  Valid when the extended box does not wrap onto itself
  // (ex + r <= nlon), so local and geometric offsets agree.
  std::vector<int4> pairs;
  h->pair_assembly = true;
  for (const Block& b : h->blocks)
    if (g.periodic && b.ex + g.r > g.nlon) h->pair_assembly = false;
  {
    // staged rows, output tile and pair list of a 32-column tile in shared memory
    const size_t npairs = (size_t)(g.pmax + 1) * (g.pmax + 2) / 2;
    for (const Block& b : h->blocks) h->box_sum = std::max(h->box_sum, b.nlev_b + b.ey + b.ex);
    if (g.pmax > 63 ||
        assemble_pairs_smem(h->esize, g.pmax, h->hb_max, g.r, (int)npairs, h->box_sum) >
            227 * 1024)
      h->pair_assembly = false;
  }
  if (h->pair_assembly) {
    struct Shape {
      int nlev, ey, ex, hb, pair_base, npair;
    };
    std::vector<Shape> shapes;
    for (Block& b : h->blocks) {
      int id = -1;
      for (size_t i = 0; i < shapes.size(); ++i)
        if (shapes[i].nlev == b.nlev_b && shapes[i].ey == b.ey && shapes[i].ex == b.ex) id = (int)i;
      if (id < 0) {
        shapes.push_back({b.nlev_b, b.ey, b.ex, 0, 0, 0});
        id = (int)shapes.size() - 1;
      }
      shapes[id].hb = std::max(shapes[id].hb, b.hb);
      b.pair_base = id;  // temporarily the shape id
    }
    for (Shape& sh : shapes) {
      const int ns = g.pmax + 1;
      std::vector<int> dk(ns, 0), dy(ns, 0), dx(ns, 0), o(ns, 0);
      for (int s2 = 0; s2 < g.pmax; ++s2) slot_offset(s2, g.r, g.vr, dk[s2], dy[s2], dx[s2]);
      for (int s2 = 0; s2 < ns; ++s2) o[s2] = (dk[s2] * sh.ey + dy[s2]) * sh.ex + dx[s2];
      std::vector<std::vector<int4>> byd(sh.hb + 1);
      for (int a = 0; a < ns; ++a)
        for (int c = 0; c < ns; ++c) {
          const int d = o[a] - o[c];
          if (d < 0 || (d == 0 && a != c) || d > sh.hb) continue;
          byd[d].push_back(make_int4(a, c, o[c], d));
        }
      sh.pair_base = (int)pairs.size();
      for (int d = 0; d <= sh.hb; ++d)
        for (const int4& pr : byd[d]) pairs.push_back(pr);
      sh.npair = (int)pairs.size() - sh.pair_base;
      h->npair_max = std::max(h->npair_max, sh.npair);
    }
    for (Block& b : h->blocks) {
      const Shape& sh = shapes[b.pair_base];
      b.pair_base = sh.pair_base;
      b.npair = sh.npair;
    }
  } else {
    for (Block& b : h->blocks) b.pair_base = b.npair = -1;
  }

  // predecessor counts for the work model
  std::vector<int> p_global((size_t)g.n), p_ext;
  p_ext.reserve((size_t)h->ext_rows);
  for (int64_t l = 0; l < g.n; ++l) {
    int v, k, y, x;
    label_coords(g, l, v, k, y, x);
    int p = 0;
    for (int s = 0; s < g.pmax; ++s) {
      int kq, yq, xq;
      if (slot_pred(g, k, y, x, s, kq, yq, xq)) ++p;
    }
    p_global[(size_t)l] = p;
  }
  for (const Block& b : h->blocks) {
    const int plane = b.ey * b.ex;
    for (int loc = 0; loc < b.nb; ++loc) {
      const int k = loc / plane, yy = (loc - k * plane) / b.ex, xx = loc - k * plane - yy * b.ex;
      const int y = b.lat_lo + yy, x = imod(b.lon_lo + xx, g.nlon);
      int p = 0;
      for (int s = 0; s < g.pmax; ++s) {
        int kq, yq, xq, a, c;
        if (slot_pred(g, k, y, x, s, kq, yq, xq) && in_ext(b, g.nlon, yq, xq, a, c)) ++p;
      }
      p_ext.push_back(in_interior(b, y, x) ? p : -p - 1);
    }
  }
  compute_work(h, p_global, p_ext);
  h->p_ext = std::move(p_ext);

  enkfmc_status st;
  if ((st = dalloc(h, &h->d_blocks, sizeof(Block) * h->blocks.size()))) return st;
  if ((st = dalloc(h, &h->d_halo, sizeof(int32_t) * halo.size()))) return st;
  if ((st = dalloc(h, &h->d_status, 16))) return st;
  if ((st = dalloc(h, &h->d_obs_of, sizeof(int32_t) * g.n))) return st;
  if ((st = dalloc(h, &h->d_U, h->esize * g.n * g.ldN))) return st;
  if ((st = dalloc(h, &h->d_Te, h->esize * h->ext_rows * std::max(1, g.pmax)))) return st;
  if ((st = dalloc(h, &h->d_De, h->esize * h->ext_rows))) return st;
  if ((st = dalloc(h, &h->d_band, h->esize * h->band_elems))) return st;
  if ((st = dalloc(h, &h->d_invdiag, h->esize * h->ext_rows))) return st;
  if ((st = dalloc(h, &h->d_rhs, h->esize * h->ext_rows * g.N))) return st;
  if ((st = dalloc(h, &h->d_C, h->esize * (size_t)g.n * cov_offset_count(g.r, g.vr)))) return st;
  if (!is_fp64(h)) {  // double-precision pool for blocks whose FP32 factorisation fails
    // room for every block: ill-conditioned problems can need most (none in the
    // plain form)
    h->fb_cap = g.plain_fp32 ? 1 : h->nblock;
    h->fb_stride = (int64_t)h->nb_max * (h->hb_max + 1);
    if ((st = dalloc(h, &h->d_bfail, sizeof(int32_t) * h->nblock))) return st;
    if ((st = dalloc(h, &h->d_c1max, sizeof(float) * h->nblock))) return st;
    if ((st = dalloc(h, &h->d_fb_cnt, sizeof(int32_t) * 12))) return st;
    if ((st = dalloc(h, &h->d_fb_blocks, sizeof(Block) * h->fb_cap))) return st;
    if ((st = dalloc(h, &h->d_fb_band, sizeof(double) * h->fb_cap * h->fb_stride))) return st;
    CUDA_TRY(cudaMemset(h->d_fb_cnt, 0, sizeof(int32_t) * 12));
    CUDA_TRY(cudaMemset(h->d_bfail, 0, sizeof(int32_t) * h->nblock));
  }
  if (has_fp64_rows(g, !is_fp64(h))) {
    if ((st = dalloc(h, &h->d_U64, sizeof(double) * g.n * g.ldN))) return st;
    if ((st = dalloc(h, &h->d_C64, sizeof(double) * (size_t)g.n * cov_offset_count(g.r, g.vr))))
      return st;
  }
  if (h->refine_solve) {
    if ((st = dalloc(h, &h->d_res, h->esize * h->ext_rows * g.N))) return st;
    if ((st = dalloc(h, &h->d_vhi, h->esize * h->ext_rows * g.N))) return st;
    if ((st = dalloc(h, &h->d_vlo, h->esize * h->ext_rows * g.N))) return st;
  }
  CUDA_TRY(cudaMemcpy(h->d_blocks, h->blocks.data(), sizeof(Block) * h->blocks.size(),
                      cudaMemcpyHostToDevice));
  if (h->pair_assembly) {
    if ((st = dalloc(h, &h->d_pairs, sizeof(int4) * std::max<size_t>(1, pairs.size())))) return st;
    // source of every extended row: the global row of T (interior) or the
    // block's boundary row
    std::vector<int32_t> srcrow((size_t)h->ext_rows);
    for (const Block& b : h->blocks)
      for (int loc = 0; loc < b.nb; ++loc) {
        const int plane = b.ey * b.ex;
        const int k = loc / plane, yy = (loc - k * plane) / b.ex, xx = loc - k * plane - yy * b.ex;
        const int y = b.lat_lo + yy, x = imod(b.lon_lo + xx, g.nlon);
        srcrow[(size_t)(b.row_off + loc)] =
            in_interior(b, y, x) ? (int32_t)coords_label(g, b.var, k, y, x)
                                 : ~(int32_t)(b.row_off + loc);
      }
    if ((st = dalloc(h, &h->d_srcrow, sizeof(int32_t) * srcrow.size()))) return st;
    CUDA_TRY(cudaMemcpy(h->d_srcrow, srcrow.data(), sizeof(int32_t) * srcrow.size(),
                        cudaMemcpyHostToDevice));
    if (!pairs.empty())
      CUDA_TRY(cudaMemcpy(h->d_pairs, pairs.data(), sizeof(int4) * pairs.size(),
                          cudaMemcpyHostToDevice));
  }
  if (!halo.empty())
    CUDA_TRY(cudaMemcpy(h->d_halo, halo.data(), sizeof(int32_t) * halo.size(),
                        cudaMemcpyHostToDevice));
  {  // pair table of the typical row (gather of the regression Gram matrices)
    const int pf = g.pmax - (g.periodic ? g.r : 0);
    std::vector<int2> ptab((size_t)(pf + 1) * (pf + 2) / 2);
    for (size_t pi = 0; pi < ptab.size(); ++pi) ptab[pi] = pair_table_entry(g, pf, (int)pi);
    if ((st = dalloc(h, &h->d_ptab, sizeof(int2) * ptab.size()))) return st;
    CUDA_TRY(cudaMemcpy(h->d_ptab, ptab.data(), sizeof(int2) * ptab.size(),
                        cudaMemcpyHostToDevice));
    // gather tables of any row (gather_table_entry): tri, then ftab
    const size_t nfull = (size_t)(g.pmax + 1) * (g.pmax + 2) / 2;
    std::vector<uint16_t> gtab(2 * nfull);
    for (size_t pi = 0; pi < nfull; ++pi)
      gather_table_entry(g, g.pmax, (int)pi, gtab[pi], gtab[nfull + pi]);
    if ((st = dalloc(h, &h->d_gtab, sizeof(uint16_t) * gtab.size()))) return st;
    CUDA_TRY(cudaMemcpy(h->d_gtab, gtab.data(), sizeof(uint16_t) * gtab.size(),
                        cudaMemcpyHostToDevice));
  }
  CUDA_TRY(cudaMemset(h->d_status, 0, 16));
  return ENKFMC_OK;
}

void release(enkfmc_handle* h) {
  void* bufs[] = {h->d_pairs, h->d_srcrow, h->d_ptab,  h->d_gtab,    h->d_blocks, h->d_halo,
                  h->d_status, h->d_obs_of, h->d_U,   h->d_C,       h->d_Te,     h->d_De,
                  h->d_band,  h->d_invdiag, h->d_rhs, h->d_res,     h->d_vhi,    h->d_vlo,
                  h->d_Xb,    h->d_y,       h->d_R,   h->d_Z,       h->d_Xa,     h->d_T,
                  h->d_D,     h->d_lam,     h->d_aT,  h->d_bT,      h->d_dxT,    h->d_lamT,
                  h->d_Eo,    h->d_Fo,      h->d_Vo,  h->d_Ko,  h->d_U64,     h->d_C64, h->d_W,      h->d_bfail,  h->d_fb_cnt,
                  h->d_fb_blocks, h->d_fb_band, h->d_c1max, h->d_sqp, h->d_fy, h->d_fZ,
                  h->d_fx,    h->d_fsq,     h->d_dobs, h->d_dob_off, h->d_dzoff, h->d_obs_idx,
                  h->d_dz,    h->d_dw,      h->d_dx64, h->d_dpred, h->d_dsucc,
                  h->d_dq,    h->d_dsoff,   h->d_ds};
  for (void* b : bufs) dfree(b);
  if (h->f_stream) cudaStreamDestroy(h->f_stream);
  if (h->c_stream) cudaStreamDestroy(h->c_stream);
  if (h->c_start) cudaEventDestroy(h->c_start);
  if (h->c_done) cudaEventDestroy(h->c_done);
  for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
  h->pool.clear();
}

enkfmc_status check_launch(cudaError_t e) {
  if (e == cudaSuccess) return ENKFMC_OK;
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? ENKFMC_ENOMEM : ENKFMC_ECUDA;
}

cudaEvent_t pooled_event(enkfmc_handle* h) {
  if (h->pool_used == h->pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
    h->pool.push_back(e);
  }
  return h->pool[h->pool_used++];
}

// Run one launcher: a callable taking int* (it adds the kernels it launched)
// or a callable without arguments (one kernel).  The launches are counted per
// kind; while profiling they are bracketed with events on the stream.
template <class F>
enkfmc_status timed(enkfmc_handle* h, int kind, F&& launch) {
  int nk = 0;
  auto call = [&]() -> cudaError_t {
    if constexpr (std::is_invocable<F, int*>::value) {
      return launch(&nk);
    } else {
      nk = 1;
      return launch();
    }
  };
  if (!h->prof) {
    const enkfmc_status st = check_launch(call());
    h->calls[kind] += 1;
    h->kernels[kind] += nk;
    return st;
  }
  cudaEvent_t a = pooled_event(h), b = pooled_event(h);
  if (!a || !b) return ENKFMC_ECUDA;
  cudaEventRecord(a, h->stream);
  enkfmc_status st = check_launch(call());
  cudaEventRecord(b, h->stream);
  h->calls[kind] += 1;
  h->kernels[kind] += nk;
  h->recs.push_back({kind, a, b});
  return st;
}

template <typename T>
EstStats<T> stats_of(enkfmc_handle* h) {
  return {(T*)h->d_U, (T*)h->d_C, h->d_U64, h->d_C64};
}

// Anomalies and covariance table of Xb (skipped when already computed from it).
template <typename T>
enkfmc_status run_statistics(enkfmc_handle* h, const T* Xb) {
  if (h->U_src == Xb) return ENKFMC_OK;
  h->U_src = nullptr;
  const EstStats<T> sts = stats_of<T>(h);
  enkfmc_status st = timed(h, ENKFMC_K_ANOMALIES, [&](int* nk) {
    return launch_stat_anomalies<T>(h->g, Xb, sts, h->stream, nk);
  });
  if (st) return st;
  st = timed(h, ENKFMC_K_COVTABLE, [&](int* nk) {
    return launch_stat_covtables<T>(h->g, sts, h->stream, nk);
  });
  if (st) return st;
  h->U_src = Xb;
  return ENKFMC_OK;
}

template <typename T>
enkfmc_status run_estimate(enkfmc_handle* h, const T* Xb, T* Tv, T* D) {
  h->U_src = nullptr;  // a new estimate always recomputes the statistics
  enkfmc_status st = run_statistics<T>(h, Xb);
  if (st) return st;
  return timed(h, ENKFMC_K_REGRESS, [&](int* nk) {
    return launch_regressions<T>(h->g, stats_of<T>(h), nullptr, h->g.n, h->d_blocks, Tv, D,
                                 h->prob.ridge_c, h->d_status, h->stream, nk);
  });
}

// Predicted error (relative to the block's solution) above which a block's
// single-precision refinement hands over to double precision.
constexpr float kRefineTolerance = 1e-6f;

// Blocks of the double-precision pool (append = 0: those whose single-
// precision factorisation met a non-positive pivot, the pool rebuilt; 1: the
// ones flagged by the refinement check, added): assembled from the same
// single-precision T, D and R in double, then factored in double.
enkfmc_status fp64_pool(enkfmc_handle* h, const float* Tv, const float* D, const float* R,
                        int append) {
  if (h->g.plain_fp32) {  // no double-precision blocks: a failed block is reported
    return timed(h, ENKFMC_K_FP64_BLOCKS, [&]() {
      return launch_fallback_list(h->d_blocks, h->nblock, h->d_bfail, h->d_fb_blocks,
                                  h->d_fb_cnt, 0, h->fb_stride, h->d_status, append, h->stream);
    });
  }
  return timed(h, ENKFMC_K_FP64_BLOCKS, [&](int* nk) {
    *nk += 3;
    int* rng = h->d_fb_cnt + (append ? 6 : 2);  // {lo, hi} of the blocks to (re)factor
    cudaError_t e = launch_fallback_list(h->d_blocks, h->nblock, h->d_bfail, h->d_fb_blocks,
                                         h->d_fb_cnt, h->fb_cap, h->fb_stride, h->d_status,
                                         append, h->stream);
    if (e != cudaSuccess) return e;
    e = launch_assemble<float, double>(h->g, h->d_fb_blocks, h->fb_cap, h->nb_max, Tv, D,
                                       (const float*)h->d_Te, (const float*)h->d_De, h->d_obs_of,
                                       R, h->d_fb_band, h->d_status, h->stream, h->hb_max, rng);
    if (e != cudaSuccess) return e;
    return launch_bandchol<double>(h->d_fb_blocks, h->fb_cap, h->hb_max, h->d_fb_band, nullptr,
                                   h->d_status, h->stream, rng, nullptr);
  });
}

template <typename T>
enkfmc_status run_assemble(enkfmc_handle* h, const T* Tv, const T* D, const T* R) {
  enkfmc_status st = timed(h, ENKFMC_K_REGRESS_HALO, [&](int* nk) {
    return launch_regressions<T>(h->g, stats_of<T>(h), h->d_halo, h->halo_rows, h->d_blocks,
                                 (T*)h->d_Te, (T*)h->d_De, h->prob.ridge_c, h->d_status,
                                 h->stream, nk);
  });
  if (st) return st;
  st = timed(h, ENKFMC_K_ASSEMBLE, [&] {
    if (h->pair_assembly)
      return launch_assemble_pairs<T>(h->g, h->d_blocks, h->nblock, h->nb_max, h->hb_max,
                                      h->npair_max, h->d_pairs, h->d_srcrow, Tv, D,
                                      (const T*)h->d_Te, (const T*)h->d_De, h->d_obs_of, R,
                                      (T*)h->d_band, h->box_sum, h->stream);
    return launch_assemble<T>(h->g, h->d_blocks, h->nblock, h->nb_max, Tv, D, (const T*)h->d_Te,
                              (const T*)h->d_De, h->d_obs_of, R, (T*)h->d_band, h->d_status,
                              h->stream, h->hb_max);
  });
  if (st) return st;
  if constexpr (std::is_same<T, double>::value) {
    return timed(h, ENKFMC_K_BANDCHOL, [&] {
      return launch_bandchol<T>(h->d_blocks, h->nblock, h->hb_max, (T*)h->d_band,
                                (T*)h->d_invdiag, h->d_status, h->stream);
    });
  } else {
    // single precision: blocks whose factorisation meets a non-positive pivot
    // are flagged, assembled again from the same T and D in double precision,
    // and factored in double (their solves too)
    CUDA_TRY(cudaMemsetAsync(h->d_bfail, 0, sizeof(int32_t) * h->nblock, h->stream));
    st = timed(h, ENKFMC_K_BANDCHOL, [&] {
      if (h->tc_chol)
        return launch_bandchol_tc(h->d_blocks, h->nblock, h->hb_max, (float*)h->d_band,
                                  (float*)h->d_invdiag, h->d_status, h->stream, h->d_bfail);
      return launch_bandchol<float>(h->d_blocks, h->nblock, h->hb_max, (float*)h->d_band,
                                    (float*)h->d_invdiag, h->d_status, h->stream, nullptr,
                                    h->d_bfail);
    });
    if (st) return st;
    h->R_assembled = R;
    return fp64_pool(h, (const float*)Tv, (const float*)D, (const float*)R, 0);
  }
}

// Views of the double-precision pool for solve_band (offsets into its meta).
constexpr int kPoolAll = 0, kPoolNew = 4, kPoolNone = 8;

// L L^T X = B in place for every block, N members (Eq. 11).  Single
// precision: the blocks of the double-precision pool are solved in double
// (their rhs stays single precision) when the view includes them, else get a
// zero solution; the others are solved on the tensor or CUDA cores.
template <typename T>
cudaError_t solve_band(enkfmc_handle* h, T* rhs, int* nk, int view = kPoolAll) {
  ++*nk;
  if constexpr (std::is_same<T, double>::value) {
    return launch_bandsolve<double, double>(h->d_blocks, h->nblock, h->hb_max, h->g.N,
                                            (const double*)h->d_band, rhs, h->stream);
  } else {
    cudaError_t e;
    if (h->tc_solve)
      e = launch_bandsolve_tc(h->d_blocks, h->nblock, h->hb_max, h->g.N, (const float*)h->d_band,
                              (const float*)h->d_invdiag, rhs, h->d_status, h->stream,
                              h->d_bfail);
    else
      e = launch_bandsolve<float, float>(h->d_blocks, h->nblock, h->hb_max, h->g.N,
                                         (const float*)h->d_band, rhs, h->stream, nullptr,
                                         h->d_bfail);
    if (e != cudaSuccess) return e;
    ++*nk;
    return launch_bandsolve<double, float>(h->d_fb_blocks, h->fb_cap, h->hb_max, h->g.N,
                                           h->d_fb_band, rhs, h->stream, h->d_fb_cnt + view,
                                           nullptr);
  }
}

template <typename T>
enkfmc_status run_analyze(enkfmc_handle* h, const T* Xb, const T* y, const T* R, const T* Z,
                          T* Xa) {
  enkfmc_status st = timed(h, ENKFMC_K_RHS, [&] {
    return launch_rhs<T>(h->g, h->d_blocks, h->nblock, h->nb_max, h->d_obs_of, h->m, Xb, y, R, Z,
                         (T*)h->d_rhs, h->stream);
  });
  if (st) return st;
  st = timed(h, ENKFMC_K_BANDSOLVE, [&](int* nk) {
    return solve_band<T>(h, (T*)h->d_rhs, nk);
  });
  if (st) return st;
  const T* corr = nullptr;
  if (h->refine_solve && sizeof(T) == sizeof(float)) {
    // with three or more steps, blocks whose corrections shrink too slowly
    // after two steps join the double-precision pool for the third
    const bool check = h->refine_steps >= 3 && !h->g.plain_fp32;
    for (int step = 0; step < h->refine_steps; ++step) {
      st = timed(h, ENKFMC_K_RESIDUAL, [&](int* nk) {
        cudaError_t e = cudaSuccess;
        if (step > 0) {  // fold the previous correction into dX
          ++*nk;
          e = launch_accumulate((float*)h->d_rhs, (const float*)h->d_res,
                                h->ext_rows * (int64_t)h->g.N, h->stream);
          if (e != cudaSuccess) return e;
        }
        *nk += 2;  // k_whiten, k_residual
        return launch_refine_residual(
            h->g, h->d_blocks, h->nblock, h->nb_max, h->d_obs_of, h->m, (const float*)Xb,
            (const float*)y, (const float*)R, (const float*)Z, (const float*)h->T_assembled,
            (const float*)h->D_assembled, (const float*)h->d_Te, (const float*)h->d_De,
            (const float*)h->d_rhs, (float*)h->d_vhi, (float*)h->d_vlo, nullptr,
            (float*)h->d_res, h->stream);
      });
      if (st) return st;
      st = timed(h, ENKFMC_K_BANDSOLVE, [&](int* nk) {
        return solve_band<T>(h, (T*)h->d_res, nk, check && step == 2 ? kPoolNew : kPoolNone);
      });
      if (st) return st;
      if (check && step < 2) {
        st = timed(h, ENKFMC_K_FP64_BLOCKS, [&](int* nk) {
          ++*nk;
          return launch_ir_check(h->d_blocks, h->nblock, h->g.N, (const float*)h->d_res,
                                 (const float*)h->d_rhs, h->d_c1max, h->d_bfail,
                                 kRefineTolerance, step, h->stream);
        });
        if (st) return st;
        if (step == 1) {
          st = fp64_pool(h, (const float*)h->T_assembled, (const float*)h->D_assembled,
                         (const float*)h->R_assembled, 1);
          if (st) return st;
        }
      }
    }
    corr = (const T*)h->d_res;
  }
  return timed(h, ENKFMC_K_WRITEBACK, [&] {
    return launch_writeback<T>(h->g, h->d_blocks, h->nsubx, h->prob.sub_lon, h->prob.sub_lat, Xb,
                               (const T*)h->d_rhs, corr, Xa, h->stream);
  });
}

// Algorithmic work per launch (see enkfmc_work_per_launch).  Regression of a
// row with p predecessors: augmented Gram 2N((p+1)(p+2)/2), Cholesky p^3/3,
// two triangular solves 2p^2, residual 2Np.  Band factor: column c with
// w = min(hb, nb-1-c) entries below the diagonal costs w + w(w+1) flops.
// Band solves: 4N w per column plus 2N divisions.
void compute_work(enkfmc_handle* h, const std::vector<int>& p_global,
                  const std::vector<int>& p_ext) {
  const Geom& g = h->g;
  const double N = g.N, es = (double)h->esize;
  // per row: Cholesky p^3/3, two triangular solves 2p^2, residual 2Np (the Gram
  // entries come from the covariance table)
  auto reg = [&](double p) { return p * p * p / 3.0 + 2.0 * p * p + 2.0 * N * p; };
  double f_glob = 0, f_halo = 0, f_asm = 0, t_read = 0;
  for (int p : p_global) f_glob += reg(p);
  for (size_t i = 0; i < p_ext.size(); ++i) {
    const double p = p_ext[i] >= 0 ? p_ext[i] : -p_ext[i] - 1;
    if (p_ext[i] < 0) f_halo += reg(p);  // negative entries mark boundary rows
    f_asm += (p + 1) * (p + 2);
    t_read += p + 2;
  }
  double f_chol = 0, f_solve = 0;
  for (const Block& b : h->blocks) {
    for (int c = 0; c < b.nb; ++c) {
      const double w = std::min(b.hb, b.nb - 1 - c);
      f_chol += w + w * (w + 1);
      f_solve += 4.0 * N * w + 2.0 * N;
    }
  }
  const double n = (double)g.n, er = (double)h->ext_rows, hr = (double)h->halo_rows;
  h->work_flops[ENKFMC_K_ANOMALIES] = 2.0 * N * n;
  h->work_bytes[ENKFMC_K_ANOMALIES] = es * 2.0 * N * n;
  h->work_flops[ENKFMC_K_REGRESS] = f_glob;
  h->work_bytes[ENKFMC_K_REGRESS] = es * (N * n + n * (g.pmax + 1));
  h->work_flops[ENKFMC_K_REGRESS_HALO] = f_halo;
  h->work_bytes[ENKFMC_K_REGRESS_HALO] = es * (N * hr + hr * (g.pmax + 1));
  h->work_flops[ENKFMC_K_ASSEMBLE] = f_asm;
  h->work_bytes[ENKFMC_K_ASSEMBLE] = es * ((double)h->band_elems + t_read);
  h->work_flops[ENKFMC_K_BANDCHOL] = f_chol;
  h->work_bytes[ENKFMC_K_BANDCHOL] = es * 2.0 * (double)h->band_elems;
  h->work_flops[ENKFMC_K_RHS] = 0;
  h->work_bytes[ENKFMC_K_RHS] = es * N * er;
  h->work_flops[ENKFMC_K_BANDSOLVE] = f_solve;
  h->work_bytes[ENKFMC_K_BANDSOLVE] = es * (2.0 * (double)h->band_elems + 4.0 * N * er);
  h->work_flops[ENKFMC_K_WRITEBACK] = N * n;
  h->work_bytes[ENKFMC_K_WRITEBACK] = es * 3.0 * N * n;
  h->work_flops[ENKFMC_K_FORECAST] = 0;
  h->work_bytes[ENKFMC_K_FORECAST] = es * 2.0 * N * n;
  h->work_flops[ENKFMC_K_SQERR] = (N + 2.0) * n;
  h->work_bytes[ENKFMC_K_SQERR] = es * (N + 1.0) * n;
  // covariance table: 2N flops per valid pair (both components inside the grid)
  const int r = g.r, w4 = 4 * r + 1, nH = cov_offset_count(g.r, g.vr);
  double pairs = 0;
  for (int v = 0; v < g.nvar; ++v)
    for (int k = 0; k < g.var_lev[v]; ++k)
      for (int y = 0; y < g.nlat; ++y)
        for (int dk = 0; dk <= g.vr; ++dk)
          for (int dy = (dk == 0 ? 0 : -2 * r); dy <= 2 * r; ++dy) {
            if (k + dk >= g.var_lev[v] || y + dy < 0 || y + dy >= g.nlat) continue;
            const int ndx = (dk == 0 && dy == 0) ? 2 * r + 1 : w4;
            pairs += (double)g.nlon * (g.periodic ? ndx : ndx);
          }
  h->work_flops[ENKFMC_K_COVTABLE] = 2.0 * N * pairs;
  h->work_bytes[ENKFMC_K_COVTABLE] = es * (N * n + n * (double)nH);
  // refinement residual: T dX, T^T v and the observation term, 2N flops per entry
  h->work_flops[ENKFMC_K_RESIDUAL] = h->refine_solve ? 4.0 * N * (t_read - er) : 0.0;
  h->work_bytes[ENKFMC_K_RESIDUAL] = h->refine_solve ? es * 2.0 * N * er : 0.0;
}

// Observation-dependent terms: rhs reads Xb, Z for every observed ext row.
void compute_obs_work(enkfmc_handle* h, const std::vector<int32_t>& obs_of) {
  const Geom& g = h->g;
  double ext_obs = 0;
  for (const Block& b : h->blocks) {
    const int plane = b.ey * b.ex;
    for (int loc = 0; loc < b.nb; ++loc) {
      const int k = loc / plane, yy = (loc - k * plane) / b.ex, xx = loc - k * plane - yy * b.ex;
      if (obs_of[coords_label(g, b.var, k, b.lat_lo + yy, imod(b.lon_lo + xx, g.nlon))] >= 0)
        ext_obs += 1;
    }
  }
  const double N = g.N, es = (double)h->esize;
  h->work_flops[ENKFMC_K_RHS] = 4.0 * N * ext_obs;
  h->work_bytes[ENKFMC_K_RHS] = es * (N * (double)h->ext_rows + 2.0 * N * ext_obs);
}

template <typename T>
enkfmc_status run_adjoint(enkfmc_handle* h, const T* Xa_bar, T* y_bar, T* R_bar, T* Xb_bar) {
  const Geom& g = h->g;
  const size_t es = sizeof(T);
  enkfmc_status st;
  if (!h->d_lam) {
    const size_t rows = (size_t)h->ext_rows;
    if ((st = dalloc(h, &h->d_lam, es * rows * g.N))) return st;
    if ((st = dalloc(h, &h->d_aT, es * rows * g.ldN))) return st;
    if ((st = dalloc(h, &h->d_bT, es * rows * g.ldN))) return st;
    if ((st = dalloc(h, &h->d_dxT, es * rows * g.ldN))) return st;
    if ((st = dalloc(h, &h->d_lamT, es * rows * g.ldN))) return st;
    if ((st = dalloc(h, &h->d_Eo, es * rows * g.ldN))) return st;
    if ((st = dalloc(h, &h->d_Fo, es * rows * g.ldN))) return st;
    if ((st = dalloc(h, &h->d_Vo, es * rows * std::max(1, g.pmax)))) return st;
    if ((st = dalloc(h, &h->d_Ko, es * rows))) return st;
    if (h->refine_solve && sizeof(T) == sizeof(float)) {
      if ((st = dalloc(h, &h->d_W, es * rows * g.N * 2))) return st;  // W, then residuals
    }
  }
  const T* dX2 = (h->refine_solve && sizeof(T) == sizeof(float)) ? (const T*)h->d_res : nullptr;
  const T* Tg = (const T*)h->T_assembled;
  const T* Dg = (const T*)h->D_assembled;
  st = timed(h, ENKFMC_K_ADJOINT, [&] {
    return launch_adj_seed<T>(g, h->d_blocks, h->nblock, h->nb_max, Xa_bar, (T*)h->d_lam,
                              h->stream);
  });
  if (st) return st;
  const bool refine = h->refine_solve && sizeof(T) == sizeof(float);
  const int64_t nrhs = h->ext_rows * (int64_t)g.N;
  T* W = refine ? (T*)h->d_W : nullptr;
  T* Wres = refine ? (T*)h->d_W + nrhs : nullptr;
  if (refine)
    CUDA_TRY(cudaMemcpyAsync(W, h->d_lam, sizeof(T) * nrhs, cudaMemcpyDeviceToDevice, h->stream));
  st = timed(h, ENKFMC_K_BANDSOLVE, [&](int* nk) {
    return solve_band<T>(h, (T*)h->d_lam, nk, kPoolAll);
  });
  if (st) return st;
  // Lambda = A^-1 W refined with the forward solve's steps (A is the same)
  for (int step = 0; refine && step < h->refine_steps; ++step) {
    st = timed(h, ENKFMC_K_RESIDUAL, [&](int* nk) {
      *nk += 2;
      return launch_refine_residual(
          g, h->d_blocks, h->nblock, h->nb_max, h->d_obs_of, h->m, (const float*)h->last_Xb,
          (const float*)h->last_y, (const float*)h->last_R, (const float*)h->last_Z,
          (const float*)Tg, (const float*)Dg, (const float*)h->d_Te, (const float*)h->d_De,
          (const float*)h->d_lam, (float*)h->d_vhi, (float*)h->d_vlo, (const float*)W,
          (float*)Wres, h->stream);
    });
    if (st) return st;
    st = timed(h, ENKFMC_K_BANDSOLVE, [&](int* nk) {
      return solve_band<T>(h, Wres, nk, kPoolNone);
    });
    if (st) return st;
    st = timed(h, ENKFMC_K_RESIDUAL, [&] {
      return launch_accumulate((float*)h->d_lam, (const float*)Wres, nrhs, h->stream);
    });
    if (st) return st;
  }
  st = timed(h, ENKFMC_K_ADJOINT, [&] {
    return launch_adj_ab<T>(g, h->d_blocks, h->nblock, h->nb_max, Tg, (const T*)h->d_Te,
                            (const T*)h->d_lam, (const T*)h->d_rhs, dX2, (T*)h->d_aT,
                            (T*)h->d_bT, (T*)h->d_dxT, (T*)h->d_lamT, h->stream);
  });
  if (st) return st;
  st = timed(h, ENKFMC_K_ADJ_REGRESS, [&](int* nk) {
    return launch_adj_regressions<T>(g, h->d_blocks, h->nblock, h->nb_max, stats_of<T>(h), Tg, Dg,
                                     (const T*)h->d_Te, (const T*)h->d_De, (const T*)h->d_aT,
                                     (const T*)h->d_bT, (const T*)h->d_dxT, (const T*)h->d_lamT,
                                     h->d_ptab, h->d_gtab, (T*)h->d_Eo, (T*)h->d_Fo,
                                     (T*)h->d_Vo, (T*)h->d_Ko, h->prob.ridge_c, h->d_status,
                                     h->stream, nk);
  });
  if (st) return st;
  // Ubar per extended row (into aT, free once the regressions are done), then
  // every component and observation from the blocks holding it, in order
  st = timed(h, ENKFMC_K_ADJOINT, [&] {
    return launch_adj_gather<T>(g, h->d_blocks, h->nblock, h->nb_max, Tg, (const T*)h->d_Te,
                                (const T*)h->d_U, (const T*)h->d_Eo, (const T*)h->d_Fo,
                                (const T*)h->d_Vo, (const T*)h->d_Ko, (T*)h->d_aT, h->stream);
  });
  if (st) return st;
  return timed(h, ENKFMC_K_ADJOINT, [&] {
    return launch_adj_owner<T>(g, h->d_blocks, h->nsubx, h->nsuby, h->prob.sub_lon,
                               h->prob.sub_lat, h->d_obs_of, h->m, (const T*)h->last_Xb,
                               (const T*)h->last_y, (const T*)h->last_R, (const T*)h->last_Z,
                               (const T*)h->d_aT, (const T*)h->d_lamT, (const T*)h->d_dxT, Xa_bar,
                               Xb_bar, y_bar, R_bar, h->stream);
  });
}

// Dual form set-up for the current observations: per block the observations
// inside its extended set in solve order (label order: segment by segment,
// inside a segment from the columns past the longitude seam), the offsets of
// the blocks' lists and Z buffers, the solves' ring W (rows: a row and its
// predecessors lie less than (vr ey + r + 1) ex positions apart), the
// buffers, and the work model of the three dual kinds.  EINVAL (nothing
// queued) when the observation systems or the rings exceed shared memory.
enkfmc_status build_dual(enkfmc_handle* h) {
  const Geom& g = h->g;
  // the arithmetic: double for single-precision problems with rows where
  // 2p > N (the precision rule of the regressions; there T^-1 and R + Z^T D Z
  // need more than single precision), else the problem's
  const bool fp64 = !is_fp64(h) && has_fp64_rows(g, true);
  const size_t es = fp64 ? 8 : h->esize;
  std::vector<int2> dobs;
  std::vector<int64_t> off((size_t)h->nblock + 1, 0), zoff((size_t)h->nblock, 0),
      soff((size_t)h->nblock, 0);
  int64_t ssum = 0;
  int mb_max = 0, W = 1, Wn = 1, Df = 1 << 30;
  int64_t zsum = 0;
  size_t prow = 0;
  const double N = g.N;
  double fz = 0, fo = 0, fa = 0, bz = 0, bw = 0, pz = 0;
  for (int bi = 0; bi < h->nblock; ++bi) {
    const Block& b = h->blocks[bi];
    const int npre = std::min(b.ex, g.nlon - b.lon_lo), plane = b.ey * b.ex;
    double pre = 0;  // predecessors of the rows up to position t
    int mb = 0;
    for (int t = 0; t < b.nb; ++t) {
      const int seg = t / b.ex;
      int xx = t - seg * b.ex + npre;
      if (xx >= b.ex) xx -= b.ex;
      const int loc = seg * b.ex + xx, k = loc / plane, yy = (loc - k * plane) / b.ex;
      const int pe = h->p_ext[prow + (size_t)loc];
      pre += pe >= 0 ? pe : -pe - 1;
      const int o = h->obs_of_host[(size_t)coords_label(g, b.var, k, b.lat_lo + yy,
                                                        imod(b.lon_lo + xx, g.nlon))];
      if (o >= 0) {
        dobs.push_back(make_int2(t, o));
        fz += 2.0 * pre;  // column o: the rows up to its own position
        ++mb;
      }
    }
    prow += (size_t)b.nb;
    off[(size_t)bi + 1] = (int64_t)dobs.size();
    zoff[(size_t)bi] = zsum;
    zsum += (int64_t)b.nb * mb;
    soff[(size_t)bi] = ssum;
    ssum += (int64_t)mb * (mb + 1) / 2;
    mb_max = std::max(mb_max, mb);
    // positions apart of a row and its predecessor: below (vr ey + r + 1) ex;
    // on its own level below (r + 1) ex, on a level below at least
    // (ey - r - 1) ex + 1 (the segment of (level, latitude) and the column
    // in label order differ by at most r and ex - 1, resp. at least ey - r
    // and at most ex - 1)
    W = std::max(W, (g.vr * b.ey + g.r + 1) * b.ex);
    Wn = std::max(Wn, (g.r + 1) * b.ex);
    if (g.vr > 0 && b.nlev_b > 1) Df = std::min(Df, (b.ey - g.r - 1) * b.ex + 1);
    const double nb = b.nb, m = mb;
    fo += nb * m * (m + 1) + m * m * m / 3.0 + 2.0 * m * m * N;
    fa += 2.0 * nb * m * N + nb * N + 2.0 * N * pre;
    bz += nb * m;
    bw += m * N;
    pz += pre;
  }
  W = std::min(W, std::max(1, h->nb_max));
  DualRings rg{W, W, 1, W};  // one ring of W rows
  Wn = std::min(Wn, W);
  if (Df < W && Df >= Wn && Df > kDualStages + 1)
    rg = DualRings{Wn, Df, W - Df + kDualStages + 1, W};
  const size_t lim = 227 * 1024;
  const size_t ssolve = es == 8 ? dual_solve_smem<double>(rg, g.pmax)
                                : dual_solve_smem<float>(rg, g.pmax);
  const size_t sobs = mb_max == 0 ? 0
                      : es == 8   ? dual_obs_smem<double>(mb_max, g.N)
                                  : dual_obs_smem<float>(mb_max, g.N);
  if (ssolve > lim || sobs > lim || g.pmax > kDualMaxSlots) return ENKFMC_EINVAL;
  std::vector<int32_t> oidx((size_t)std::max<int64_t>(h->m, 0), 0);
  for (size_t l = 0; l < h->obs_of_host.size(); ++l)
    if (h->obs_of_host[l] >= 0) oidx[(size_t)h->obs_of_host[l]] = (int32_t)l;
  void* old[] = {h->d_dobs, h->d_dob_off, h->d_dzoff, h->d_obs_idx, h->d_dz, h->d_dw,
                 h->d_dsoff, h->d_ds};
  CUDA_TRY(cudaStreamSynchronize(h->stream));  // buffers of an earlier set may be in use
  for (void* p : old) dfree(p);
  h->d_dobs = nullptr;
  h->d_dob_off = h->d_dzoff = nullptr;
  h->d_obs_idx = nullptr;
  h->d_dz = h->d_dw = h->d_ds = nullptr;
  h->d_dsoff = nullptr;
  enkfmc_status st;
  if ((st = dalloc(h, &h->d_dobs, sizeof(int2) * dobs.size()))) return st;
  if ((st = dalloc(h, &h->d_dob_off, sizeof(int64_t) * off.size()))) return st;
  if ((st = dalloc(h, &h->d_dzoff, sizeof(int64_t) * zoff.size()))) return st;
  if ((st = dalloc(h, &h->d_obs_idx, sizeof(int32_t) * oidx.size()))) return st;
  if ((st = dalloc(h, &h->d_dz, es * (size_t)zsum))) return st;
  if ((st = dalloc(h, &h->d_dw, es * (size_t)dobs.size() * g.N))) return st;
  if ((st = dalloc(h, &h->d_dsoff, sizeof(int64_t) * soff.size()))) return st;
  if ((st = dalloc(h, &h->d_ds, es * (size_t)ssum))) return st;
  CUDA_TRY(cudaMemcpy(h->d_dsoff, soff.data(), sizeof(int64_t) * soff.size(),
                      cudaMemcpyHostToDevice));
  if (fp64 && !h->d_dx64 &&
      (st = dalloc(h, &h->d_dx64, sizeof(double) * (size_t)h->ext_rows * g.N)))
    return st;
  const size_t tab = dual_table_bytes(es, g.pmax) * (size_t)h->ext_rows;
  if (!h->d_dpred && (st = dalloc(h, &h->d_dpred, tab))) return st;
  if (!h->d_dsucc && (st = dalloc(h, &h->d_dsucc, tab))) return st;
  if (!h->d_dq && (st = dalloc(h, &h->d_dq, es * (size_t)h->ext_rows * g.N))) return st;
  h->dual_fp64 = fp64;
  if (!dobs.empty())
    CUDA_TRY(cudaMemcpy(h->d_dobs, dobs.data(), sizeof(int2) * dobs.size(),
                        cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(h->d_dob_off, off.data(), sizeof(int64_t) * off.size(),
                      cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(h->d_dzoff, zoff.data(), sizeof(int64_t) * zoff.size(),
                      cudaMemcpyHostToDevice));
  if (!oidx.empty())
    CUDA_TRY(cudaMemcpy(h->d_obs_idx, oidx.data(), sizeof(int32_t) * oidx.size(),
                        cudaMemcpyHostToDevice));
  h->dual_mb_max = mb_max;
  h->dual_rings = rg;
  h->work_flops[ENKFMC_K_DUAL_Z] = fz;
  h->work_bytes[ENKFMC_K_DUAL_Z] = (double)es * (bz + pz);
  h->work_flops[ENKFMC_K_DUAL_OBS] = fo;
  h->work_bytes[ENKFMC_K_DUAL_OBS] = (double)es * (bz + bw + 2.0 * bw);
  h->work_flops[ENKFMC_K_DUAL_APPLY] = fa;
  h->work_bytes[ENKFMC_K_DUAL_APPLY] =
      (double)es * (bz + bw + pz + 2.0 * N * (double)h->ext_rows);
  h->dual_ready = true;
  return ENKFMC_OK;
}

// The dual kernels with inputs TI and arithmetic TC; dX: the increments (TC).
template <typename TI, typename TC>
enkfmc_status run_dual_kernels(enkfmc_handle* h, const TI* Xb, const TI* Tv, const TI* D,
                               const TI* y, const TI* R, const TI* Z, TI* Xa, TC* dX) {
  const Geom& g = h->g;
  enkfmc_status st = timed(h, ENKFMC_K_DUAL_Z, [&](int* nk) {
    return launch_dual_z<TI, TC>(g, h->d_blocks, h->nblock, h->nb_max, h->dual_mb_max,
                                 h->d_dobs, h->d_dob_off, h->d_dzoff, Tv, (const TI*)h->d_Te,
                                 h->d_dpred, h->d_dsucc, (TC*)h->d_dz, h->dual_rings, h->stream,
                                 nk);
  });
  if (st) return st;
  st = timed(h, ENKFMC_K_DUAL_OBS, [&](int* nk) {
    return launch_dual_obs<TI, TC>(g, h->d_blocks, h->nblock, h->dual_mb_max, h->d_dobs,
                                   h->d_dob_off, h->d_dzoff, h->d_dsoff, h->d_obs_idx, h->m, Xb,
                                   y, R, Z, D, (const TI*)h->d_De, (const TC*)h->d_dz,
                                   (TC*)h->d_ds, (TC*)h->d_dw, h->d_status, h->stream, nk);
  });
  if (st) return st;
  st = timed(h, ENKFMC_K_DUAL_APPLY, [&](int* nk) {
    return launch_dual_apply<TI, TC>(g, h->d_blocks, h->nblock, h->nb_max, h->d_dob_off,
                                     h->d_dzoff, (const TC*)h->d_dz, (const TC*)h->d_dw, D,
                                     (const TI*)h->d_De, h->d_dpred, (TC*)h->d_dq, dX,
                                     h->dual_rings, h->stream, nk);
  });
  if (st) return st;
  return timed(h, ENKFMC_K_WRITEBACK, [&] {
    return launch_dual_writeback<TI, TC>(g, h->d_blocks, h->nsubx, h->prob.sub_lon,
                                         h->prob.sub_lat, Xb, (const TC*)dX, Xa, h->stream);
  });
}

template <typename T>
enkfmc_status run_analyze_dual(enkfmc_handle* h, const T* Xb, const T* Tv, const T* D,
                               const T* y, const T* R, const T* Z, T* Xa) {
  enkfmc_status st;
  if (!h->dual_ready && (st = build_dual(h))) return st;  // EINVAL: nothing changed
  // the boundary rows are re-estimated here: the band of the last assembly no
  // longer matches them, and the reverse pass follows the primal form only
  h->assembled = false;
  h->analyzed = false;
  const Geom& g = h->g;
  // boundary rows of every block from its local samples (Algorithm 3), as for
  // the primal assembly
  if ((st = run_statistics<T>(h, Xb))) return st;
  st = timed(h, ENKFMC_K_REGRESS_HALO, [&](int* nk) {
    return launch_regressions<T>(g, stats_of<T>(h), h->d_halo, h->halo_rows, h->d_blocks,
                                 (T*)h->d_Te, (T*)h->d_De, h->prob.ridge_c, h->d_status,
                                 h->stream, nk);
  });
  if (st) return st;
  if constexpr (std::is_same<T, float>::value) {
    if (h->dual_fp64)
      return run_dual_kernels<float, double>(h, Xb, Tv, D, y, R, Z, Xa, h->d_dx64);
  }
  return run_dual_kernels<T, T>(h, Xb, Tv, D, y, R, Z, Xa, (T*)h->d_rhs);
}

}  // namespace

extern "C" {

const char* enkfmc_strerror(enkfmc_status s) {
  switch (s) {
    case ENKFMC_OK: return "ok";
    case ENKFMC_EINVAL: return "invalid argument or unsupported geometry";
    case ENKFMC_ENOMEM: return "out of memory";
    case ENKFMC_ENOTSPD: return "sub-domain matrix not positive definite";
    case ENKFMC_EDNONPOS: return "singular Gram matrix or non-positive residual variance";
    case ENKFMC_ENONFINITE: return "non-finite value";
    case ENKFMC_ETIMEOUT: return "device wait timed out";
    case ENKFMC_ECUDA: return "CUDA runtime error";
    case ENKFMC_ENOTIMPL: return "not implemented";
    case ENKFMC_ESTATE: return "call out of order";
  }
  return "unknown status";
}

enkfmc_status enkfmc_check_problem(const enkfmc_problem* p) {
  if (!p) return ENKFMC_EINVAL;
  if (p->flags & ~(ENKFMC_FLAG_NO_SOLVE_REFINEMENT | ENKFMC_FLAG_SIMT_BAND |
                   ENKFMC_FLAG_PLAIN_FP32 | ENKFMC_FLAG_REFINE_MASK))
    return ENKFMC_EINVAL;
  Geom g;
  return problem_geom(*p, g);
}

enkfmc_status enkfmc_create(enkfmc_handle** out, const enkfmc_problem* p, void* stream) {
  if (!out || !p) return ENKFMC_EINVAL;
  *out = nullptr;
  enkfmc_handle* h = new (std::nothrow) enkfmc_handle();
  if (!h) return ENKFMC_ENOMEM;
  h->prob = *p;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    (void)cudaGetLastError();
    delete h;
    return ENKFMC_ECUDA;
  }
  enkfmc_status st = build(h);
  if (st != ENKFMC_OK) {
    release(h);
    delete h;
    return st;
  }
  *out = h;
  return ENKFMC_OK;
}

void enkfmc_destroy(enkfmc_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  release(h);
  delete h;
}

enkfmc_status enkfmc_query(const enkfmc_handle* h, enkfmc_info* info) {
  if (!h || !info) return ENKFMC_EINVAL;
  info->n = h->g.n;
  info->pmax = h->g.pmax;
  info->nsub = h->nsub;
  info->nblock = h->nblock;
  info->hb_max = h->hb_max;
  info->ext_rows = h->ext_rows;
  info->halo_rows = h->halo_rows;
  info->band_elems = h->band_elems;
  info->workspace_bytes = h->workspace_bytes;
  info->m = h->m;
  info->tc_chol = h->tc_chol ? 1 : 0;
  info->tc_solve = h->tc_solve ? 1 : 0;
  info->refine_steps = h->refine_solve ? h->refine_steps : 0;
  info->fp64_rows = h->d_C64 ? 1 : 0;
  return ENKFMC_OK;
}

enkfmc_status enkfmc_set_stream(enkfmc_handle* h, void* stream) {
  if (!h) return ENKFMC_EINVAL;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  return ENKFMC_OK;
}

enkfmc_status enkfmc_slot_offsets(const enkfmc_handle* h, int32_t* dk, int32_t* dlat,
                                  int32_t* dlon) {
  if (!h || !dk || !dlat || !dlon) return ENKFMC_EINVAL;
  for (int s = 0; s < h->g.pmax; ++s) {
    int a, b, c;
    slot_offset(s, h->g.r, h->g.vr, a, b, c);
    dk[s] = a;
    dlat[s] = b;
    dlon[s] = c;
  }
  return ENKFMC_OK;
}

enkfmc_status enkfmc_set_observations(enkfmc_handle* h, const int32_t* obs_idx, int64_t m) {
  if (!h || m < 0 || (m > 0 && !obs_idx) || m > h->g.n) return ENKFMC_EINVAL;
  std::vector<int32_t> of((size_t)h->g.n, -1);
  for (int64_t o = 0; o < m; ++o) {
    const int32_t c = obs_idx[o];
    if (c < 0 || c >= h->g.n) return ENKFMC_EINVAL;
    if (o > 0 && c <= obs_idx[o - 1]) return ENKFMC_EINVAL;
    of[c] = (int32_t)o;
  }
  CUDA_TRY(cudaMemcpy(h->d_obs_of, of.data(), sizeof(int32_t) * of.size(),
                      cudaMemcpyHostToDevice));
  h->m = m;
  h->assembled = false;
  h->dual_ready = false;
  h->obs_of_host = std::move(of);
  compute_obs_work(h, h->obs_of_host);
  return ENKFMC_OK;
}

enkfmc_status enkfmc_estimate(enkfmc_handle* h, const void* Xb, void* Tvals, void* D) {
  if (!h || !Xb || !Tvals || !D) return ENKFMC_EINVAL;
  if (is_fp64(h))
    return run_estimate<double>(h, (const double*)Xb, (double*)Tvals, (double*)D);
  return run_estimate<float>(h, (const float*)Xb, (float*)Tvals, (float*)D);
}

enkfmc_status enkfmc_assemble(enkfmc_handle* h, const void* Xb, const void* Tvals, const void* D,
                              const void* Rdiag) {
  if (!h || !Xb || !Tvals || !D || (h->m > 0 && !Rdiag)) return ENKFMC_EINVAL;
  if (h->m < 0) return ENKFMC_ESTATE;
  // anomalies and covariances of this Xb (the boundary regressions use them)
  enkfmc_status st;
  if (is_fp64(h)) {
    st = run_statistics<double>(h, (const double*)Xb);
    if (!st) st = run_assemble<double>(h, (const double*)Tvals, (const double*)D, (const double*)Rdiag);
  } else {
    st = run_statistics<float>(h, (const float*)Xb);
    if (!st) st = run_assemble<float>(h, (const float*)Tvals, (const float*)D, (const float*)Rdiag);
  }
  h->assembled = (st == ENKFMC_OK);
  h->analyzed = false;
  h->T_assembled = Tvals;
  h->D_assembled = D;
  return st;
}

enkfmc_status enkfmc_analyze(enkfmc_handle* h, const void* Xb, const void* y, const void* Rdiag,
                             const void* Z, void* Xa) {
  if (!h || !Xb || !Xa || Xa == Xb) return ENKFMC_EINVAL;
  if (h->m > 0 && (!y || !Rdiag || !Z)) return ENKFMC_EINVAL;
  if (!h->assembled) return ENKFMC_ESTATE;
  h->last_Xb = Xb;
  h->last_y = y;
  h->last_R = Rdiag;
  h->last_Z = Z;
  enkfmc_status st;
  if (is_fp64(h))
    st = run_analyze<double>(h, (const double*)Xb, (const double*)y, (const double*)Rdiag,
                             (const double*)Z, (double*)Xa);
  else
    st = run_analyze<float>(h, (const float*)Xb, (const float*)y, (const float*)Rdiag,
                            (const float*)Z, (float*)Xa);
  h->analyzed = (st == ENKFMC_OK);
  return st;
}

enkfmc_status enkfmc_cycle_host(enkfmc_handle* h, const void* Xb, const void* y, const void* Rdiag,
                                const void* Z, void* Xa) {
  if (!h || !Xb || !Xa) return ENKFMC_EINVAL;
  if (h->m < 0) return ENKFMC_ESTATE;
  if (h->m > 0 && (!y || !Rdiag || !Z)) return ENKFMC_EINVAL;
  const size_t es = h->esize;
  const size_t xbytes = es * (size_t)h->g.N * h->g.n;
  const size_t obytes = es * (size_t)h->m;
  const size_t zbytes = es * (size_t)h->g.N * h->m;
  enkfmc_status st;
  if (!h->d_Xb) {
    if ((st = dalloc(h, &h->d_Xb, xbytes))) return st;
    if ((st = dalloc(h, &h->d_Xa, xbytes))) return st;
    if ((st = dalloc(h, &h->d_y, obytes))) return st;
    if ((st = dalloc(h, &h->d_R, obytes))) return st;
    if ((st = dalloc(h, &h->d_Z, zbytes))) return st;
    if ((st = dalloc(h, &h->d_T, es * (size_t)h->g.n * std::max(1, h->g.pmax)))) return st;
    if ((st = dalloc(h, &h->d_D, es * (size_t)h->g.n))) return st;
  }
  if (h->m > 0 && !h->c_stream) {
    CUDA_TRY(cudaStreamCreateWithFlags(&h->c_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&h->c_start, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&h->c_done, cudaEventDisableTiming));
  }
  // X^b first on the handle's stream; y, R and Z follow on the copy stream
  // once it is in (the two directions of the link are shared, so running them
  // beside it would only delay the estimate), overlapping the estimate, which
  // reads X^b alone; assemble and analyze wait for them
  CUDA_TRY(cudaMemcpyAsync(h->d_Xb, Xb, xbytes, cudaMemcpyHostToDevice, h->stream));
  if (h->m > 0) {
    CUDA_TRY(cudaEventRecord(h->c_start, h->stream));
    CUDA_TRY(cudaStreamWaitEvent(h->c_stream, h->c_start, 0));
    CUDA_TRY(cudaMemcpyAsync(h->d_y, y, obytes, cudaMemcpyHostToDevice, h->c_stream));
    CUDA_TRY(cudaMemcpyAsync(h->d_R, Rdiag, obytes, cudaMemcpyHostToDevice, h->c_stream));
    CUDA_TRY(cudaMemcpyAsync(h->d_Z, Z, zbytes, cudaMemcpyHostToDevice, h->c_stream));
    CUDA_TRY(cudaEventRecord(h->c_done, h->c_stream));
  }
  st = enkfmc_estimate(h, h->d_Xb, h->d_T, h->d_D);
  if (h->m > 0) {
    const cudaError_t e = cudaStreamWaitEvent(h->stream, h->c_done, 0);
    if (st || e != cudaSuccess) {
      // the caller may release y, R and Z on return: no copy stays in flight
      (void)cudaStreamSynchronize(h->c_stream);
      if (!st) st = check_launch(e);
    }
  }
  if (st) return st;
  if ((st = enkfmc_assemble(h, h->d_Xb, h->d_T, h->d_D, h->d_R))) return st;
  if ((st = enkfmc_analyze(h, h->d_Xb, h->d_y, h->d_R, h->d_Z, h->d_Xa))) return st;
  CUDA_TRY(cudaMemcpyAsync(Xa, h->d_Xa, xbytes, cudaMemcpyDeviceToHost, h->stream));
  return enkfmc_get_status(h, nullptr);
}

enkfmc_status enkfmc_analyze_dual(enkfmc_handle* h, const void* Xb, const void* Tvals,
                                  const void* D, const void* y, const void* Rdiag,
                                  const void* Z, void* Xa) {
  if (!h || !Xb || !Tvals || !D || !Xa || Xa == Xb) return ENKFMC_EINVAL;
  if (h->m < 0) return ENKFMC_ESTATE;
  if (h->m > 0 && (!y || !Rdiag || !Z)) return ENKFMC_EINVAL;
  if (is_fp64(h))
    return run_analyze_dual<double>(h, (const double*)Xb, (const double*)Tvals,
                                    (const double*)D, (const double*)y, (const double*)Rdiag,
                                    (const double*)Z, (double*)Xa);
  return run_analyze_dual<float>(h, (const float*)Xb, (const float*)Tvals, (const float*)D,
                                 (const float*)y, (const float*)Rdiag, (const float*)Z,
                                 (float*)Xa);
}

enkfmc_status enkfmc_analyze_adjoint(enkfmc_handle* h, const void* Xa_bar, void* y_bar,
                                     void* Rdiag_bar, void* Xb_bar) {
  if (!h || !Xa_bar || !Xb_bar || Xb_bar == Xa_bar) return ENKFMC_EINVAL;
  if (h->m > 0 && (!y_bar || !Rdiag_bar)) return ENKFMC_EINVAL;
  if (!h->analyzed || !h->assembled) return ENKFMC_ESTATE;
  if (is_fp64(h))
    return run_adjoint<double>(h, (const double*)Xa_bar, (double*)y_bar, (double*)Rdiag_bar,
                               (double*)Xb_bar);
  return run_adjoint<float>(h, (const float*)Xa_bar, (float*)y_bar, (float*)Rdiag_bar,
                            (float*)Xb_bar);
}

enkfmc_status enkfmc_get_status(enkfmc_handle* h, int64_t* info) {
  if (!h) return ENKFMC_EINVAL;
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  int32_t st[4] = {0, 0, 0, 0};
  CUDA_TRY(cudaMemcpy(st, h->d_status, 16, cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(h->d_status, 0, 16));
  if (info) {
    int64_t v;
    std::memcpy(&v, st + 2, 8);
    *info = v;
  }
  return (enkfmc_status)st[0];
}

enkfmc_status enkfmc_fp64_blocks(enkfmc_handle* h, int32_t* count) {
  if (!h || !count) return ENKFMC_EINVAL;
  *count = 0;
  if (!h->d_fb_cnt) return ENKFMC_OK;
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  CUDA_TRY(cudaMemcpy(count, h->d_fb_cnt + 1, sizeof(int32_t), cudaMemcpyDeviceToHost));
  return ENKFMC_OK;
}

enkfmc_status enkfmc_export_T_pattern(const enkfmc_handle* h, int64_t* rowptr, int32_t* colidx) {
  if (!h || !rowptr) return ENKFMC_EINVAL;
  const Geom& g = h->g;
  std::vector<int64_t> row;
  int64_t nnz = 0;
  rowptr[0] = 0;
  for (int64_t l = 0; l < g.n; ++l) {
    int v, k, y, x;
    label_coords(g, l, v, k, y, x);
    row.clear();
    for (int s = 0; s < g.pmax; ++s) {
      int kq, yq, xq;
      if (slot_pred(g, k, y, x, s, kq, yq, xq)) row.push_back(coords_label(g, v, kq, yq, xq));
    }
    std::sort(row.begin(), row.end());
    if (colidx)
      for (size_t i = 0; i < row.size(); ++i) colidx[nnz + (int64_t)i] = (int32_t)row[i];
    nnz += (int64_t)row.size();
    rowptr[l + 1] = nnz;
  }
  return ENKFMC_OK;
}

enkfmc_status enkfmc_debug_block(enkfmc_handle* h, int32_t b, void* host, int64_t capacity,
                                 int64_t* nb, int32_t* hb) {
  if (!h || b < 0 || b >= h->nblock) return ENKFMC_EINVAL;
  const Block& bl = h->blocks[b];
  if (nb) *nb = bl.nb;
  if (hb) *hb = bl.hb;
  const int64_t cnt = (int64_t)bl.nb * (bl.hb + 1);
  if (!host) return ENKFMC_OK;
  if (capacity < cnt) return ENKFMC_EINVAL;
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  CUDA_TRY(cudaMemcpy(host, (char*)h->d_band + h->esize * bl.band_off, h->esize * cnt,
                      cudaMemcpyDeviceToHost));
  return ENKFMC_OK;
}

enkfmc_status enkfmc_forecast_shift(enkfmc_handle* h, const void* X, void* Xout, int32_t nvec,
                                    int32_t shift, double inflation) {
  if (!h || !X || !Xout || X == Xout || nvec < 1 || !(inflation > 0.0) || inflation > 1e3)
    return ENKFMC_EINVAL;
  const int nl = h->g.nlon;
  const int s = ((shift % nl) + nl) % nl;
  return timed(h, ENKFMC_K_FORECAST, [&]() -> cudaError_t {
    if (is_fp64(h))
      return launch_shift<double>(h->g, (const double*)X, (double*)Xout, nvec, s, inflation,
                                  h->stream);
    return launch_shift<float>(h->g, (const float*)X, (float*)Xout, nvec, s, inflation,
                               h->stream);
  });
}

enkfmc_status enkfmc_ensemble_sqerr(enkfmc_handle* h, const void* Xa, const void* xref,
                                    double* out) {
  if (!h || !Xa || !xref || !out) return ENKFMC_EINVAL;
  if (!h->d_sqp) {
    if (enkfmc_status st = dalloc(h, &h->d_sqp, sizeof(double) * kSqGrid)) return st;
  }
  return timed(h, ENKFMC_K_SQERR, [&](int* nk) -> cudaError_t {
    *nk += 2;
    if (is_fp64(h))
      return launch_sqerr<double>(h->g, (const double*)Xa, (const double*)xref, h->d_sqp, out,
                                  h->stream);
    return launch_sqerr<float>(h->g, (const float*)Xa, (const float*)xref, h->d_sqp, out,
                               h->stream);
  });
}

enkfmc_status enkfmc_profile(enkfmc_handle* h, int32_t enable) {
  if (!h) return ENKFMC_EINVAL;
  h->prof = enable != 0;
  return ENKFMC_OK;
}

enkfmc_status enkfmc_profile_read(enkfmc_handle* h, int64_t* calls, int64_t* kernels,
                                  double* ms) {
  if (!h || !calls || !kernels || !ms) return ENKFMC_EINVAL;
  for (int k = 0; k < ENKFMC_NKERNEL; ++k) {
    calls[k] = h->calls[k];
    kernels[k] = h->kernels[k];
    h->calls[k] = h->kernels[k] = 0;
    ms[k] = 0.0;
  }
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  for (const auto& r : h->recs) {
    float t = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
    ms[r.kind] += t;
  }
  h->recs.clear();
  h->pool_used = 0;
  return ENKFMC_OK;
}

const char* enkfmc_kernel_name(int32_t kind) {
  static const char* names[ENKFMC_NKERNEL] = {"anomalies", "regress",   "regress_halo",
                                              "assemble",  "bandchol",  "rhs",
                                              "bandsolve", "writeback", "covtable",
                                              "residual",  "adjoint",   "adj_regress",
                                              "fp64_blocks", "forecast", "sqerr",
                                              "dual_z",    "dual_obs",  "dual_apply"};
  return (kind >= 0 && kind < ENKFMC_NKERNEL) ? names[kind] : "unknown";
}

enkfmc_status enkfmc_work_per_launch(const enkfmc_handle* h, double* flops, double* bytes) {
  if (!h || !flops || !bytes) return ENKFMC_EINVAL;
  for (int k = 0; k < ENKFMC_NKERNEL; ++k) {
    flops[k] = h->work_flops[k];
    bytes[k] = h->work_bytes[k];
  }
  return ENKFMC_OK;
}

}  // extern "C"
