// Band solves L L^T X = B (Eq. 11) for all N <= 128 members of one block of
// A per CTA, with the panel updates on the tensor cores (single precision).
//
// Storage as in k_band.cu: the factor of a block is the column-major lower
// band band[c (hb + 1) + d] = L[c + d][c], which is the strided view
// L[i][c] = F[c hb + i] (c <= i <= c + hb) of the block's slice F.
//
// Forward, panel p of 32 rows [c0, c0 + 32):
//   Y_p = L_pp^-1 (B_p - S_p), S_p the sum of L[c0+t][j] Y_j over earlier rows,
// with S accumulated in TMEM: member m is TMEM lane m and row i of the block
// is TMEM column i mod WT, so the rows that a panel still has to update (its
// own 32 and the hb rows below) form a circular window of columns.  Once Y_p
// is known one group of tcgen05.mma adds Y_p^T L[rows below][panel]^T to the
// window (D = A B^T with A = Y_p^T, 128 x 32, and B = the hb x 32 block of L
// below the diagonal block); the group's first part covers the next panel's
// 32 columns and is committed to its own mbarrier, so the next triangle can
// start while the rest of the group runs.  Backward (L^T X = Y) runs the same
// schedule from the last panel, with B = L[panel][rows above]^T.
//
// Precision: every operand is split x = hi + lo (hi the nearest TF32 value)
// and each product is taken as hi*hi + hi*lo + lo*hi with FP32 accumulation
// (about 21 significant bits per product); the 32 x 32 triangles are solved
// in FP32 registers, one member per thread.
#include "band_panel.cuh"
#include "enkfmc_internal.h"
#include "tc_sm100.cuh"

namespace enkfmc {

namespace {

constexpr int kSolveWarps = 8;                  // 4 member warps + 4 staging warps
constexpr int kABytes = 128 * 32 * 4;           // one split of the member operand
constexpr uint64_t kWaitNs = 2000000000ull;     // bound of every mbarrier wait (2 s)

// Byte offset of element (row n, K index t) in a K-major tile of 32 K-values.
__device__ __forceinline__ int core_off(int n, int kc) {
  return ((n >> 3) * 8 + kc) * 128 + (n & 7) * 16;
}

__device__ __forceinline__ void put_split4(unsigned char* hi, unsigned char* lo, int off,
                                           const float (&v)[4]) {
  float4 h, l;
  tc::split_tf32(v[0], h.x, l.x);
  tc::split_tf32(v[1], h.y, l.y);
  tc::split_tf32(v[2], h.z, l.z);
  tc::split_tf32(v[3], h.w, l.w);
  *reinterpret_cast<float4*>(hi + off) = h;
  *reinterpret_cast<float4*>(lo + off) = l;
}

__device__ __forceinline__ void cp_async4(void* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(tc::smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}
// all but the most recently committed group complete
__device__ __forceinline__ void cp_async_wait_prev() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}
// x - (x with the 13 low mantissa bits cleared): the part of x that a TF32
// operand read drops, exact in FP32
__device__ __forceinline__ float tf32_rest(float x) {
  return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

// Producer warps' own barrier (named barrier 1, the 128 producer threads).
__device__ __forceinline__ void producer_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// 256 threads: warps 0-3 are the member warps (thread m = member m = TMEM lane
// m: TMEM columns, triangles, member operands, MMA issue by thread 0), warps
// 4-7 stage operands (band tiles, their TF32 remainders, diagonal blocks).
// One CTA-wide barrier per panel hands the staged operands over.
__global__ void __launch_bounds__(kSolveWarps * 32, 1)
    k_bandsolve_tc(const Block* __restrict__ blocks, const float* __restrict__ band,
                   const float* __restrict__ invdiag, float* __restrict__ rhs, int N, int NU,
                   int nbufB, int WT, int32_t* __restrict__ status,
                   const int* __restrict__ skip) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool member = warp < 4;
  const int m = tid;          // member warps: member index
  const int pt = tid - 128;   // staging warps: thread index
  const int pw = warp - 4;
  const Block b = blocks[blockIdx.x];
  // a block factored in double precision is solved by the double-precision
  // pass (uniform exit, before any TMEM or barrier is set up)
  if (skip && skip[b.id]) return;
  const int nb = b.nb, hb = b.hb;
  const float* F = band + b.band_off;
  const float* Fi = invdiag + b.row_off;
  float* X = rhs + b.row_off * N;
  const int NUb = min(NU, (hb + 15) & ~15);  // rows one panel reaches, multiple of 16
  const int bbytes = NU * 128;

  // [2 groups][hi, lo] member operands; [nbufB][raw, rest] band operands (the raw
  // FP32 tile is the TF32 "hi" operand as read by the tensor cores, the rest tile
  // holds what that read drops); [2 panels] diagonal triangles and 1/L[c][c]
  unsigned char* sA = smem;
  unsigned char* sB = smem + 4 * kABytes;
  float* Lpp = reinterpret_cast<float*>(sB + (size_t)nbufB * 2 * bbytes);  // [2][32][32]
  float* invd = Lpp + 2 * 32 * 32;                                     // [2][32]
  uint64_t* bars = reinterpret_cast<uint64_t*>(invd + 2 * 32);         // ready, done0, done1
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 3);

  if (warp == 0) tc::tmem_alloc(slot, (uint32_t)WT);
  if (tid == 0) {
    tc::mbar_init(&bars[0], 1);
    tc::mbar_init(&bars[1], 1);
    tc::mbar_init(&bars[2], 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *slot;
  const uint32_t tlane = tbase + ((uint32_t)((warp & 3) * 32) << 16);
  const uint32_t bar_ready = tc::smem_u32(&bars[0]);
  const uint32_t bar_done0 = tc::smem_u32(&bars[1]);
  const uint32_t bar_done1 = tc::smem_u32(&bars[2]);

  int ngroups = 0;  // MMA groups issued so far (same value in every thread)
  int pending = 0;  // this thread's outstanding timeout, folded into the next handoff
  // two band buffers: the staging warps copy the next group's tile one panel ahead
  const bool lookahead = nbufB == 2;
  bool aborted = false;

  auto wait_ready_local = [&](int g) {
    if (!tc::mbar_wait(bar_ready, (uint32_t)(g & 1), kWaitNs)) pending = 1;
  };
  auto wait_done_local = [&](int g) {
    if (!tc::mbar_wait((g & 1) ? bar_done1 : bar_done0, (uint32_t)((g >> 1) & 1), kWaitNs))
      pending = 1;
  };
  // the per-panel handoff: staged operands published, aborts agreed
  auto handoff = [&]() -> bool {
    tc::fence_before_sync();
    const int bad = __syncthreads_or(pending);
    pending = 0;
    if (bad && tid == 0) record_error(status, ENKFMC_ETIMEOUT, (int64_t)blockIdx.x);
    return bad != 0;
  };

  // D columns [col0, col0 + len) (rows of the block, mod WT) += A B^T with B
  // rows [brow0, brow0 + len) of buffer bbuf; len and col0 multiples of 16.
  auto issue = [&](int abuf, int bbuf, int col0, int len, int brow0) {
    const uint32_t a_hi = tc::smem_u32(sA + (abuf * 2 + 0) * kABytes);
    const uint32_t a_lo = tc::smem_u32(sA + (abuf * 2 + 1) * kABytes);
    const uint32_t b_hi = tc::smem_u32(sB + (size_t)(bbuf * 2 + 0) * bbytes);
    const uint32_t b_lo = tc::smem_u32(sB + (size_t)(bbuf * 2 + 1) * bbytes);
    // the start-address field is (address >> 4): a byte offset o adds o >> 4
    const uint64_t ah0 = tc::desc_kmajor(a_hi, 128, 1024);
    const uint64_t al0 = tc::desc_kmajor(a_lo, 128, 1024);
    const uint64_t bh0 = tc::desc_kmajor(b_hi, 128, 1024);
    const uint64_t bl0 = tc::desc_kmajor(b_lo, 128, 1024);
    while (len > 0) {
      const int c = col0 % WT;
      const int n = min(min(len, WT - c), 256);
      const uint32_t id = tc::idesc_tf32(128, n);
      const uint64_t boff = (uint64_t)(brow0 >> 3) * 64u;  // 1024-byte row groups
      const uint32_t d = tbase + (uint32_t)c;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint64_t k16 = (uint64_t)ks * 16u;  // 256 bytes per K step
        tc::mma_tf32(d, ah0 + k16, bl0 + boff + k16, id, 1);
        tc::mma_tf32(d, al0 + k16, bh0 + boff + k16, id, 1);
        tc::mma_tf32(d, ah0 + k16, bh0 + boff + k16, id, 1);
      }
      col0 += n;
      brow0 += n;
      len -= n;
    }
  };

  // ---- member warps ----
  // 32 rows [c0, c0 + 32) of this member (zero beyond the block or member count)
  auto load_rows = [&](int c0, float (&z)[32]) {
    if (m < N) {
      const float* src = X + (int64_t)m * nb + c0;
      if (c0 + 32 <= nb && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 v = reinterpret_cast<const float4*>(src)[q];
          z[4 * q] = v.x; z[4 * q + 1] = v.y; z[4 * q + 2] = v.z; z[4 * q + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int t = 0; t < 32; ++t) z[t] = (c0 + t < nb) ? src[t] : 0.f;
      }
    } else {
#pragma unroll
      for (int t = 0; t < 32; ++t) z[t] = 0.f;
    }
  };
  auto store_rows = [&](int c0, const float (&z)[32]) {
    if (m < N) {
      float* dst = X + (int64_t)m * nb + c0;
      if (c0 + 32 <= nb && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          reinterpret_cast<float4*>(dst)[q] =
              make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
      } else {
#pragma unroll
        for (int t = 0; t < 32; ++t)
          if (c0 + t < nb) dst[t] = z[t];
      }
    }
  };
  // member operand of the next group: row m, K index t
  auto put_member = [&](int abuf, const float (&z)[32]) {
    unsigned char* hi = sA + (abuf * 2 + 0) * kABytes;
    unsigned char* lo = sA + (abuf * 2 + 1) * kABytes;
#pragma unroll
    for (int kc = 0; kc < 8; ++kc) {
      const float v[4] = {z[4 * kc], z[4 * kc + 1], z[4 * kc + 2], z[4 * kc + 3]};
      put_split4(hi, lo, core_off(m, kc), v);
    }
  };

  // ---- staging warps ----
  // Lpp[u][t] = L[c0+t][c0+u] (forward, t >= u) or L[c0+u][c0+t] (backward, t <= u),
  // invd[t] = 1 / L[c0+t][c0+t]; asynchronous copies, zeros stored directly
  auto prefetch_diag = [&](int c0, bool fwd, int buf) {
    const int nbc = min(32, nb - c0);
    float* Lq = Lpp + buf * 1024;
    for (int e = pt; e < 1024; e += 128) {
      const int u = e >> 5, t = e & 31;
      const float* src = nullptr;
      if (u < nbc && t < nbc) {
        if (fwd) {
          if (t >= u && t - u <= hb) src = F + (int64_t)(c0 + u) * hb + c0 + t;
        } else {
          if (t <= u && u - t <= hb) src = F + (int64_t)(c0 + t) * hb + c0 + u;
        }
      }
      if (src) cp_async4(Lq + e, src);
      else Lq[e] = 0.f;
    }
    if (pt < 32) {
      if (pt < nbc) cp_async4(invd + buf * 32 + pt, Fi + c0 + pt);
      else invd[buf * 32 + pt] = 0.f;
    }
  };
  // Raw tiles: lane (n mod 8, t mod 4) of a warp, warps over 8-row groups, the
  // 8 K chunks unrolled; every shared-memory word of a warp's store is distinct.
  const int nl = lane >> 2, tl = lane & 3;
  // forward group of panel c0: B rows n <-> block rows c0 + 32 + n, K index t <->
  // column c0 + t (per chunk: 4 columns x 8 consecutive rows)
  auto prefetch_fwd = [&](int c0, int len, int bbuf) {
    unsigned char* raw = sB + (size_t)(bbuf * 2 + 0) * bbytes;
    for (int ng = pw; ng < (len >> 3); ng += 4) {
      const int i = c0 + 32 + ng * 8 + nl;
      float* d = reinterpret_cast<float*>(raw + ng * 1024 + nl * 16 + tl * 4);
      const float* src = F + (int64_t)(c0 + tl) * hb + i;
#pragma unroll
      for (int kc = 0; kc < 8; ++kc) {
        const int c = c0 + 4 * kc + tl;
        float* dst = d + kc * 32;
        if (i < nb && c < nb && i - c <= hb) cp_async4(dst, src + (int64_t)(4 * kc) * hb);
        else *dst = 0.f;
      }
    }
  };
  // backward group of panel c0: B rows n <-> block rows jlo + n, K index t <-> row
  // c0 + t (per chunk: 8 rows x 4 consecutive t)
  auto prefetch_bwd = [&](int c0, int jlo, int len, int bbuf) {
    unsigned char* raw = sB + (size_t)(bbuf * 2 + 0) * bbytes;
    for (int ng = pw; ng < (len >> 3); ng += 4) {
      const int j = jlo + ng * 8 + nl;
      float* d = reinterpret_cast<float*>(raw + ng * 1024 + nl * 16 + tl * 4);
      const float* src = F + (int64_t)j * hb + c0 + tl;
#pragma unroll
      for (int kc = 0; kc < 8; ++kc) {
        const int r = c0 + 4 * kc + tl;
        float* dst = d + kc * 32;
        if (r < nb && r - j <= hb) cp_async4(dst, src + 4 * kc);
        else *dst = 0.f;
      }
    }
  };
  // rest tile from the raw tile (len rows = len * 128 contiguous bytes)
  auto make_rest = [&](int len, int bbuf) {
    const float4* raw = reinterpret_cast<const float4*>(sB + (size_t)(bbuf * 2 + 0) * bbytes);
    float4* rest = reinterpret_cast<float4*>(sB + (size_t)(bbuf * 2 + 1) * bbytes);
    for (int e = pt; e < len * 8; e += 128) {
      const float4 v = raw[e];
      rest[e] = make_float4(tf32_rest(v.x), tf32_rest(v.y), tf32_rest(v.z), tf32_rest(v.w));
    }
  };
  auto fwd_len = [&](int c0) {  // B rows of the forward group of panel c0
    return min(NUb, (nb - (c0 + 32) + 15) & ~15);
  };
  auto bwd_jlo = [&](int c0) { return max(0, c0 - NUb); };

  const int np = (nb + 31) / 32;
  float z[32];

  // ---------------- forward: L Y = B ----------------
  if (member) {
    for (int c = 0; c < WT; c += 32) tc::tmem_zero32(tlane + (uint32_t)c);
    tc::tmem_wait_st();
    load_rows(0, z);
  } else {
    // diagonal block 0 and, with two band buffers, the tile of group 0
    prefetch_diag(0, true, 0);
    if (lookahead && 32 < nb) prefetch_fwd(0, fwd_len(0), 0);
    cp_async_commit();
    cp_async_wait_all();
    producer_sync();
    if (lookahead && 32 < nb) {
      make_rest(fwd_len(0), 0);
      tc::fence_async_smem();
    }
  }
  aborted = handoff();
  for (int p = 0; p < np && !aborted; ++p) {
    const int c0 = p * 32;
    const bool below = c0 + 32 < nb;
    if (member) {
      if (p > 0) {
        wait_ready_local(ngroups - 1);
        tc::fence_after_sync();
        float d[32];
        tc::tmem_ld32(tlane + (uint32_t)(c0 % WT), d);
#pragma unroll
        for (int t = 0; t < 32; ++t) z[t] -= d[t];
      }
      if (32 * warp < N) {  // triangle: right-looking over the columns u of L_pp
        const float* Lq = Lpp + (p & 1) * 1024;
        const float* iv = invd + (p & 1) * 32;
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const float yu = z[u] * iv[u];
          z[u] = yu;
          const float4* col = reinterpret_cast<const float4*>(Lq + u * 32);
#pragma unroll
          for (int g = (u + 1) >> 2; g < 8; ++g) {
            const float4 q = col[g];
            const float lv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
              if (4 * g + k > u) z[4 * g + k] = fmaf(-lv[k], yu, z[4 * g + k]);
          }
        }
      }
      store_rows(c0, z);
      if (below) put_member(ngroups & 1, z);
      tc::tmem_zero32(tlane + (uint32_t)(c0 % WT));
      tc::tmem_wait_st();
      tc::fence_async_smem();
      if (p + 1 < np) load_rows(c0 + 32, z);
    } else if (lookahead) {
      // interval p: the next diagonal block; the rest tile of this panel's group
      // (raw tile copied during the previous interval); the raw tile of the next
      // panel's group once the group that last read its buffer is done
      if (p + 1 < np) prefetch_diag(c0 + 32, true, (p + 1) & 1);
      cp_async_commit();
      if (below && p > 0) {
        cp_async_wait_prev();
        producer_sync();
        make_rest(fwd_len(c0), ngroups % 2);
        tc::fence_async_smem();
      }
      if (c0 + 64 < nb) {
        if (ngroups >= 1) wait_done_local(ngroups - 1);
        prefetch_fwd(c0 + 32, fwd_len(c0 + 32), (ngroups + 1) % 2);
      }
      cp_async_commit();
      cp_async_wait_prev();
    } else {
      if (below) {
        const int H = ngroups - nbufB;  // last group that read the buffer to refill
        if (H >= 0) wait_done_local(H);
        prefetch_fwd(c0, fwd_len(c0), ngroups % nbufB);
      }
      if (p + 1 < np) prefetch_diag(c0 + 32, true, (p + 1) & 1);
      cp_async_commit();
      cp_async_wait_all();
      producer_sync();
      if (below) {
        make_rest(fwd_len(c0), ngroups % nbufB);
        tc::fence_async_smem();
      }
    }
    if (handoff()) {
      aborted = true;
      break;
    }
    if (below) {
      if (tid == 0) {
        const int len = fwd_len(c0);
        const int len1 = min(32, len);
        tc::fence_after_sync();
        issue(ngroups & 1, ngroups % nbufB, c0 + 32, len1, 0);
        tc::commit(bar_ready);
        issue(ngroups & 1, ngroups % nbufB, c0 + 32 + len1, len - len1, len1);
        tc::commit((ngroups & 1) ? bar_done1 : bar_done0);
      }
      ++ngroups;
    }
  }
  if (!aborted && ngroups > 0) {
    wait_done_local(ngroups - 1);
    aborted = handoff();
  }

  // ---------------- backward: L^T X = Y ----------------
  if (!aborted) {
    const int cl = (np - 1) * 32;
    if (member) {
      for (int c = 0; c < WT; c += 32) tc::tmem_zero32(tlane + (uint32_t)c);
      tc::tmem_wait_st();
      load_rows(cl, z);
    } else {
      cp_async_wait_all();
      prefetch_diag(cl, false, 0);
      if (lookahead && cl >= 32) prefetch_bwd(cl, bwd_jlo(cl), cl - bwd_jlo(cl), ngroups % 2);
      cp_async_commit();
      cp_async_wait_all();
      producer_sync();
      if (lookahead && cl >= 32) {
        make_rest(cl - bwd_jlo(cl), ngroups % 2);
        tc::fence_async_smem();
      }
    }
    aborted = handoff();
    int q = 0;  // panels done (selects the diagonal buffer)
    for (int p = np - 1; p >= 0 && !aborted; --p, ++q) {
      const int c0 = p * 32;
      const bool above = p >= 1;
      if (member) {
        if (p < np - 1) {
          wait_ready_local(ngroups - 1);
          tc::fence_after_sync();
          float d[32];
          tc::tmem_ld32(tlane + (uint32_t)(c0 % WT), d);
#pragma unroll
          for (int t = 0; t < 32; ++t) z[t] -= d[t];
        }
        if (32 * warp < N) {  // triangle: right-looking from the last row, rows u of L_pp
          const float* Lq = Lpp + (q & 1) * 1024;
          const float* iv = invd + (q & 1) * 32;
#pragma unroll
          for (int u = 31; u >= 0; --u) {
            const float xu = z[u] * iv[u];
            z[u] = xu;
            const float4* row = reinterpret_cast<const float4*>(Lq + u * 32);
#pragma unroll
            for (int g = 0; g < 8; ++g) {
              if (4 * g >= u) break;
              const float4 qv = row[g];
              const float lv[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
              for (int k = 0; k < 4; ++k)
                if (4 * g + k < u) z[4 * g + k] = fmaf(-lv[k], xu, z[4 * g + k]);
            }
          }
        }
        store_rows(c0, z);
        if (above) put_member(ngroups & 1, z);
        tc::tmem_zero32(tlane + (uint32_t)(c0 % WT));
        tc::tmem_wait_st();
        tc::fence_async_smem();
        if (above) load_rows(c0 - 32, z);
      } else if (lookahead) {
        if (above) prefetch_diag(c0 - 32, false, (q + 1) & 1);
        cp_async_commit();
        if (above && p < np - 1) {
          cp_async_wait_prev();
          producer_sync();
          make_rest(c0 - bwd_jlo(c0), ngroups % 2);
          tc::fence_async_smem();
        }
        if (p >= 2) {
          const int c1 = c0 - 32;
          if (ngroups >= 1) wait_done_local(ngroups - 1);
          prefetch_bwd(c1, bwd_jlo(c1), c1 - bwd_jlo(c1), (ngroups + 1) % 2);
        }
        cp_async_commit();
        cp_async_wait_prev();
      } else {
        if (above) {
          const int H = ngroups - nbufB;
          if (H >= 0) wait_done_local(H);
          prefetch_bwd(c0, bwd_jlo(c0), c0 - bwd_jlo(c0), ngroups % nbufB);
          prefetch_diag(c0 - 32, false, (q + 1) & 1);
        }
        cp_async_commit();
        cp_async_wait_all();
        producer_sync();
        if (above) {
          make_rest(c0 - bwd_jlo(c0), ngroups % nbufB);
          tc::fence_async_smem();
        }
      }
      if (handoff()) {
        aborted = true;
        break;
      }
      if (above) {
        if (tid == 0) {
          const int jlo = bwd_jlo(c0);
          const int len = c0 - jlo;
          const int len1 = min(32, len);
          tc::fence_after_sync();
          issue(ngroups & 1, ngroups % nbufB, c0 - len1, len1, len - len1);
          tc::commit(bar_ready);
          issue(ngroups & 1, ngroups % nbufB, jlo, len - len1, 0);
          tc::commit((ngroups & 1) ? bar_done1 : bar_done0);
        }
        ++ngroups;
      }
    }
    if (!aborted && ngroups > 0) {
      wait_done_local(ngroups - 1);
      aborted = handoff();
    }
  }
  if (aborted && ngroups > 0) {
    // let the groups in flight finish (bounded) before the columns are released
    (void)tc::mbar_wait(((ngroups - 1) & 1) ? bar_done1 : bar_done0,
                        (uint32_t)(((ngroups - 1) >> 1) & 1), kWaitNs);
  }
  cp_async_wait_all();
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, (uint32_t)WT);
  }
}

// ---------------------------------------------------------------------------
// Band Cholesky with the trailing updates on the tensor cores.  Thread r owns
// row c0 + r of panel c0 (32 columns, rows [c0, c0 + 32 + hb)) in registers:
//  * warp 0 factors the 32 x 32 diagonal block right-looking (lane t = row
//    t, each column broadcast through shared memory) and leaves L11
//    column-major there;
//  * rows r >= 32 solve l_r L11^T = a_r in registers (right-looking over the
//    columns of L11, broadcast reads);
//  * every row writes its part of the factor to the band, and the rows below
//    the diagonal block write L21 (W x 32, W <= hb) as TF32 hi + lo tiles
//    (K-major);
//  * D = L21 L21^T is formed by tcgen05.mma as the 128 x 128 tiles (mi, nj),
//    nj <= mi, of its lower block triangle (hi*hi + hi*lo + lo*hi, FP32
//    accumulation in TMEM); thread (tile, row) reads its row of D and
//    subtracts it from the band, the lanes of a warp on consecutive rows of
//    one band column (coalesced), 64 entries read before any is written;
//  * batch 0 forms the tiles (mi, 0), whose first 32 columns are the next
//    panel: thread t handles window row t there, which is row t of the next
//    panel, so those updated entries go to the thread's own column of sA
//    (shared memory) instead of the band, together with the entries of the
//    rows that enter the band with the next panel; batch 1 forms the tiles
//    (mi, nj >= 1).  The next panel starts from sA, not from the band.
constexpr int kCholThreads = 384;  // 12 warps: rows of the panel; 3 tiles x 4 lane quarters
constexpr int kOpRows = 384;       // L21 rows staged (3 tiles of 128)

// Tile k of a panel whose window spans nt row tiles: k < nt -> (k, 0) (batch
// 0); then (1,1), (2,1), (2,2) (batch 1).
__device__ __forceinline__ void syrk_tile(int k, int nt, int& mi, int& nj) {
  if (k < nt) {
    mi = k;
    nj = 0;
    return;
  }
  const int k1 = k - nt;
  mi = k1 < 1 ? 1 : 2;
  nj = k1 - (mi * (mi - 1)) / 2 + 1;
}

__global__ void __launch_bounds__(kCholThreads, 1)
    k_bandchol_tc(const Block* __restrict__ blocks, float* __restrict__ band,
                  float* __restrict__ invdiag, int32_t* __restrict__ status, int WT,
                  int* __restrict__ bfail) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sHi = smem;                               // [384 rows][32] K-major
  unsigned char* sLo = smem + kOpRows * 128;
  float* Lc = reinterpret_cast<float*>(smem + 2 * kOpRows * 128);  // [32][32] column-major L11
  float* invs = Lc + 32 * 32;                                       // [32]
  float* sA = invs + 32;  // [32][kCholThreads]: next panel, column t of row r at t * 384 + r
  uint64_t* bar = reinterpret_cast<uint64_t*>(sA + 32 * kCholThreads);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  int* fail = reinterpret_cast<int*>(slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Block b = blocks[blockIdx.x];
  const int nb = b.nb, hb = b.hb;
  float* F = band + b.band_off;  // A[i][c] = F[c hb + i], c <= i <= c + hb

  if (warp == 0) tc::tmem_alloc(slot, (uint32_t)WT);
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
    *fail = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *slot;
  const uint32_t bar_a = tc::smem_u32(bar);
  const uint32_t hi0 = tc::smem_u32(sHi), lo0 = tc::smem_u32(sLo);
  uint32_t phase = 0;
  bool inflight = false;
  int covered = 0;  // rows of this panel whose entries batch 0 left in sA

  for (int c0 = 0; c0 < nb; c0 += 32) {
    const int nbc = min(32, nb - c0);
    const int rows = min(nbc + hb, nb - c0);
    const int W = rows - nbc;
    const int r = tid;
    const bool own = r < rows;
    // row c0 + r of the panel: A[c0+r][c0+t], inside the band for 0 <= r - t <= hb
    float a[32];
    if (r < covered) {  // warp-uniform (covered is a multiple of 128)
#pragma unroll
      for (int t = 0; t < 32; ++t) a[t] = sA[t * kCholThreads + r];
    } else {
#pragma unroll
      for (int t = 0; t < 32; ++t)
        a[t] = (own && t < nbc && r - t >= 0 && r - t <= hb)
                   ? F[(int64_t)(c0 + t) * hb + c0 + r]
                   : 0.f;
    }
    if (warp == 0) {  // diagonal block, right-looking, lane t = row t
      // column u of L11 goes to Lc (zeros above the diagonal), and every lane
      // reads it back with 16-byte broadcast loads for its update: one
      // shuffle per column (the pivot) instead of one per entry.  Entries of
      // a lane above the diagonal take harmless updates and are zeroed when
      // their column is reached.  1 / L[u][u] is Newton's iteration for the
      // reciprocal square root started from rsqrtf.
      bool ok = true;
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        if (u < nbc && ok) {
          const float piv = __shfl_sync(0xffffffffu, a[u], u);
          if (!isfinite(piv) || !(piv > 0.f)) {
            // a finite pivot that is not positive: with bfail the block is
            // factored again in double precision, else ENOTSPD
            if (lane == 0) {
              if (bfail && isfinite(piv)) bfail[b.id] = 1;
              else record_error(status, isfinite(piv) ? ENKFMC_ENOTSPD : ENKFMC_ENONFINITE,
                                (int64_t)b.id);
            }
            ok = false;
          } else {
            float inv = rsqrtf(piv);
            inv = inv * fmaf(-0.5f * piv * inv, inv, 1.5f);
            const float lu = lane == u ? piv * inv : (lane > u ? a[u] * inv : 0.f);
            a[u] = lu;
            Lc[u * 32 + lane] = lu;
            if (lane == u) {
              invs[u] = inv;
              invdiag[b.row_off + c0 + u] = inv;
            }
            __syncwarp();
            const float4* col = reinterpret_cast<const float4*>(Lc + u * 32);
#pragma unroll
            for (int g = (u + 1) >> 2; g < 8; ++g) {
              const float4 q = col[g];
              const float lv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
              for (int k = 0; k < 4; ++k)
                if (4 * g + k > u) a[4 * g + k] = fmaf(-lu, lv[k], a[4 * g + k]);
            }
          }
        }
      }
      for (int u = nbc; u < 32; ++u) Lc[u * 32 + lane] = 0.f;
      if (!ok && lane == 0) *fail = 1;
    }
    __syncthreads();
    if (*fail) break;  // uniform
    if (warp > 0 && own) {  // l_r L11^T = a_r
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        if (u < nbc) {
          const float xu = a[u] * invs[u];
          a[u] = xu;
          const float4* col = reinterpret_cast<const float4*>(Lc + u * 32);
#pragma unroll
          for (int g = (u + 1) >> 2; g < 8; ++g) {
            const float4 q = col[g];
            const float lv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
              if (4 * g + k > u) a[4 * g + k] = fmaf(-lv[k], xu, a[4 * g + k]);
          }
        }
      }
    }
    // factor entries of this row to the band
#pragma unroll
    for (int t = 0; t < 32; ++t)
      if (own && t < nbc && r - t >= 0 && r - t <= hb) F[(int64_t)(c0 + t) * hb + c0 + r] = a[t];
    if (W <= 0) {
      __syncthreads();
      covered = 0;
      continue;
    }
    const int nt = (W + 127) >> 7;
    const int Wp = nt * 128;
    // L21 tiles: tile row rr = r - 32 <-> block row c0 + 32 + rr (zero beyond W)
    if (warp > 0 && r - 32 < Wp) {
#pragma unroll
      for (int kc = 0; kc < 8; ++kc) {
        const float v[4] = {own ? a[4 * kc] : 0.f, own ? a[4 * kc + 1] : 0.f,
                            own ? a[4 * kc + 2] : 0.f, own ? a[4 * kc + 3] : 0.f};
        put_split4(sHi, sLo, core_off(r - 32, kc), v);
      }
    }
    if (warp == 0 && 352 + lane < Wp) {  // tile rows past the last thread
      const float z[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kc = 0; kc < 8; ++kc) put_split4(sHi, sLo, core_off(352 + lane, kc), z);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    const int ntiles = nt * (nt + 1) / 2;
    // next panel: rows [0, rows_next), columns [0, nbc_next) of this window
    const int rows_next = min(32 + hb, nb - c0 - 32);
    const int nbc_next = min(32, nb - c0 - 32);
    bool bad = false;
    for (int rd = 0; rd < 2; ++rd) {
      const int t0 = rd ? nt : 0;
      const int nr = rd ? ntiles - nt : nt;
      if (nr == 0) break;
      if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t id = tc::idesc_tf32(128, 128);
        // the start-address field is (address >> 4): a byte offset o adds o >> 4
        const uint64_t dh0 = tc::desc_kmajor(hi0, 128, 1024);
        const uint64_t dl0 = tc::desc_kmajor(lo0, 128, 1024);
        for (int k = 0; k < nr; ++k) {
          int mi, nj;
          syrk_tile(t0 + k, nt, mi, nj);
          const uint32_t d = tbase + (uint32_t)(128 * k);
          const uint64_t ao = (uint64_t)mi * 1024u, bo = (uint64_t)nj * 1024u;  // 16 KB tiles
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t k16 = (uint64_t)ks * 16u;  // 256 bytes per K step
            tc::mma_tf32(d, dh0 + ao + k16, dl0 + bo + k16, id, ks > 0 ? 1u : 0u);
            tc::mma_tf32(d, dl0 + ao + k16, dh0 + bo + k16, id, 1);
            tc::mma_tf32(d, dh0 + ao + k16, dh0 + bo + k16, id, 1);
          }
        }
        tc::commit(bar_a);
      }
      inflight = true;
      int to = !tc::mbar_wait(bar_a, phase, kWaitNs);
      to = __syncthreads_or(to);
      if (to) {
        if (tid == 0) record_error(status, ENKFMC_ETIMEOUT, (int64_t)blockIdx.x);
        bad = true;
        break;
      }
      inflight = false;
      phase ^= 1;
      tc::fence_after_sync();
      if (warp / 4 < nr) {  // warp-uniform: tile warp / 4, lane quarter warp % 4
        int mi, nj;
        syrk_tile(t0 + warp / 4, nt, mi, nj);
        const int q = warp & 3;
        const int rr = 128 * mi + 32 * q + lane;  // row of L21 / of the window
        // A[c0+32+rr][c0+32+cc] = F[(c0+32+cc) hb + c0+32+rr] = base[cc hb]
        float* base = F + (int64_t)(c0 + 32) * hb + c0 + 32 + rr;
        const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(128 * (warp / 4));
#pragma unroll 1
        for (int h2 = 0; h2 < 4; h2 += 2) {
          const int cb = 128 * nj + 32 * h2;
          // columns [0, 32) of batch 0 are the next panel (rr == tid there):
          // the rows entering the band with it are read as well
          const bool nxt = rd == 0 && h2 == 0;
          float o[64];
#pragma unroll
          for (int n = 0; n < 64; ++n) {
            bool in = cb + n <= rr && rr < W;
            if (nxt && n < 32)
              in = n <= rr && (rr < W || (rr < rows_next && rr - n <= hb && n < nbc_next));
            o[n] = in ? base[(cb + n) * hb] : 0.f;
          }
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            float dv[32];
            tc::tmem_ld32(ta + (uint32_t)(32 * (h2 + hh)), dv);
            if (nxt && hh == 0) {
#pragma unroll
              for (int n = 0; n < 32; ++n)
                sA[n * kCholThreads + tid] = n <= rr ? o[n] - dv[n] : 0.f;
            } else {
#pragma unroll
              for (int n = 0; n < 32; ++n) {
                const int cc = cb + 32 * hh + n;
                if (cc <= rr && rr < W) base[cc * hb] = o[32 * hh + n] - dv[n];
              }
            }
          }
        }
      }
      tc::fence_before_sync();
      __syncthreads();
    }
    covered = 128 * nt;
    if (bad) break;
  }
  if (inflight) (void)tc::mbar_wait(bar_a, phase, kWaitNs);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, (uint32_t)WT);
  }
}

struct TcPlan {
  int NU = 0, nbufB = 0, WT = 0;
  size_t smem = 0;
};

TcPlan plan_tc(int hb_max, int N) {
  TcPlan pl;
  if (N < 1 || N > 128) return pl;
  const int NU = (max(hb_max, 16) + 15) & ~15;
  int WT = 32;
  while (WT < 32 + NU) WT *= 2;
  if (WT > 512) return pl;
  const size_t lim = 227 * 1024;
  for (int nbuf = 2; nbuf >= 1; --nbuf) {
    const size_t bytes =
        4 * (size_t)kABytes + (size_t)nbuf * 2 * NU * 128 + 2 * 32 * 32 * 4 + 2 * 32 * 4 + 3 * 8 + 8;
    if (bytes <= lim) {
      pl.NU = NU;
      pl.nbufB = nbuf;
      pl.WT = WT;
      pl.smem = bytes;
      return pl;
    }
  }
  return pl;
}

}  // namespace

bool bandsolve_tc_supported(int hb_max, int N) { return plan_tc(hb_max, N).nbufB > 0; }

bool bandchol_tc_supported(int hb_max) {
  return hb_max >= 1 && 32 + hb_max <= kCholThreads;  // one thread per panel row
}

cudaError_t launch_bandchol_tc(const Block* blocks, int nblock, int hb_max, float* band,
                               float* invdiag, int32_t* status, cudaStream_t s, int* bfail) {
  if (!bandchol_tc_supported(hb_max)) return cudaErrorInvalidConfiguration;
  const size_t smem =
      2 * (size_t)kOpRows * 128 + sizeof(float) * (32 * 32 + 32 + 32 * kCholThreads) + 32;
  const int WT = hb_max <= 128 ? 128 : 512;  // one tile, or batches of three
  cudaError_t e = cudaFuncSetAttribute(k_bandchol_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_bandchol_tc<<<nblock, kCholThreads, smem, s>>>(blocks, band, invdiag, status, WT, bfail);
  return cudaGetLastError();
}

cudaError_t launch_bandsolve_tc(const Block* blocks, int nblock, int hb_max, int N,
                                const float* band, const float* invdiag, float* rhs,
                                int32_t* status, cudaStream_t s, const int* skip) {
  const TcPlan pl = plan_tc(hb_max, N);
  if (pl.nbufB == 0) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_bandsolve_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)pl.smem);
  if (e != cudaSuccess) return e;
  k_bandsolve_tc<<<nblock, kSolveWarps * 32, pl.smem, s>>>(blocks, band, invdiag, rhs, N, pl.NU,
                                                     pl.nbufB, pl.WT, status, skip);
  return cudaGetLastError();
}

}  // namespace enkfmc
