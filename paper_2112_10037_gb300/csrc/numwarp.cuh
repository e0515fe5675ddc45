// Numeric pass, dense-window accumulator owned by one warp.
//
// Row i of C is the sum over A(i,k) of A(i,k) * B(k,:) (Sec. 2.2).  A warp
// owns a window of W consecutive columns in shared memory: a dense value
// array and an "owner" byte per column (nonzero = the column is present).
// Rows of B are sorted, so the part of B(k,:) inside a window is one
// contiguous segment, found from a per-nonzero cursor.  Each product is
// accumulated with one fused multiply-add, acc[j] = fma(A(i,k), B(k,j), acc[j]),
// with no atomics: only this warp touches the window, lanes that walk one
// segment hit distinct columns, and when lanes carry products of different
// segments a lane first claims its column by writing its id into the owner
// byte; the lanes that read their own id back update, the rest retry.  The
// window is emitted in column order by a popcount prefix over the owner
// bytes, so no sort is needed, and cleared on the way out.
//
// Work items, handed out largest first through a global counter:
//  * split rows (heavy rows, product count above a threshold): one item per
//    tile of W columns aligned to multiples of W.  The item finds each
//    nonzero's segment by binary search inside a coarse tile of the B-row
//    tile-boundary table, and writes at the offset given by the per-tile
//    output counts of the symbolic pass.
//  * other rows: one item per row, swept window by window from its smallest
//    column; the next window starts at the smallest unread column.  Cursors
//    live in registers (up to 32 * SLOTS nonzeros per row) or in global
//    arrays parallel to A's nonzeros.
#pragma once

#include "internal.cuh"

namespace sg {

struct NumSplit {
  int heavy_bin;          // rows in bins >= heavy_bin are split (within capacity)
  int hcap;               // capacity of the per-tile count table (rows)
  int ntf;                // fine tiles (of W columns) per row
  int ntc;                // coarse tiles per row
  int tc_shift;           // log2 of the coarse tile width
  const int32_t* bnd;     // B-row coarse tile boundaries, nrows(B) x (ntc + 1)
  const int32_t* hcnt;    // output counts per (split row, fine tile)
  unsigned* counter;      // work counter, zero before the launch
};

constexpr int NW_SLOTS = 8;  // register cursors: up to 256 nonzeros of A per row

__device__ __forceinline__ unsigned byte_mask16(const uint4 q) {
  auto m4 = [](unsigned w) -> unsigned {
    const unsigned nz = __vcmpne4(w, 0u) & 0x01010101u;
    return (nz * 0x01020408u) >> 24;
  };
  return m4(q.x) | (m4(q.y) << 4) | (m4(q.z) << 8) | (m4(q.w) << 12);
}

template <int W, typename T>
struct WarpWin {
  T* acc;
  uint8_t* own;
  uint32_t* err;

  // Lanes carry products of one segment: distinct columns, no claim needed.
  __device__ __forceinline__ void add_distinct(int j, T a, T b, bool act) {
    if (act) {
      if ((unsigned)j < (unsigned)W) {
        own[j] = 1;
        acc[j] = fma(a, b, acc[j]);
      } else {
        atomicOr(err, EB_UNSORTED);
      }
    }
  }

  // Lanes may carry equal columns: claim, check, update, retry.
  __device__ __forceinline__ void add_claimed(int j, T a, T b, bool act) {
    const int lane = lane_id();
    if (act && (unsigned)j >= (unsigned)W) {
      atomicOr(err, EB_UNSORTED);
      act = false;
    }
    bool pending = act;
    const uint8_t me = (uint8_t)(lane + 1);
    while (__any_sync(FULL, pending)) {
      if (pending) own[j] = me;
      __syncwarp();
      if (pending && own[j] == me) {
        acc[j] = fma(a, b, acc[j]);
        pending = false;
      }
      __syncwarp();
    }
  }

  // Products of segments [s, s+len) of B with multiplier a (one segment per
  // lane), columns relative to base.  Long segments are walked by the whole
  // warp; short ones are flattened so each lane takes one product.
  __device__ __forceinline__ void segments(const Csr& B, const T* __restrict__ bv, int s, int len, T a,
                                           int base) {
    const int lane = lane_id();
    unsigned lm = __ballot_sync(FULL, len >= 32);
    while (lm) {
      const int L = __ffs(lm) - 1;
      lm &= lm - 1;
      const int ls = __shfl_sync(FULL, s, L), ln = __shfl_sync(FULL, len, L);
      const T la = __shfl_sync(FULL, a, L);
      int t = lane;
      for (; t + 96 < ln; t += 128) {
        const int c0 = B.ci[ls + t], c1 = B.ci[ls + t + 32], c2 = B.ci[ls + t + 64], c3 = B.ci[ls + t + 96];
        const T b0 = bv[ls + t], b1 = bv[ls + t + 32], b2 = bv[ls + t + 64], b3 = bv[ls + t + 96];
        add_distinct(c0 - base, la, b0, true);
        add_distinct(c1 - base, la, b1, true);
        add_distinct(c2 - base, la, b2, true);
        add_distinct(c3 - base, la, b3, true);
      }
      for (; t < ln; t += 32) add_distinct(B.ci[ls + t] - base, la, bv[ls + t], true);
      __syncwarp();
    }
    const int sl = len < 32 ? len : 0;
    const int incl = warp_incl_scan(sl);
    const int tot = __shfl_sync(FULL, incl, 31);
    const int excl = incl - sl;
    for (int p0 = 0; p0 < tot; p0 += 64) {
      const int p = p0 + lane, p2 = p + 32;
      const int o = warp_owner(incl, p), o2 = warp_owner(incl, p2);
      const int os = __shfl_sync(FULL, s, o), oex = __shfl_sync(FULL, excl, o);
      const T oa = __shfl_sync(FULL, a, o);
      const int os2 = __shfl_sync(FULL, s, o2), oex2 = __shfl_sync(FULL, excl, o2);
      const T oa2 = __shfl_sync(FULL, a, o2);
      int j = 0, j2 = 0;
      T b = T(0), b2 = T(0);
      if (p < tot) {
        const int bi = os + p - oex;
        j = B.ci[bi] - base;
        b = bv[bi];
      }
      if (p2 < tot) {
        const int bi = os2 + p2 - oex2;
        j2 = B.ci[bi] - base;
        b2 = bv[bi];
      }
      add_claimed(j, oa, b, p < tot);
      add_claimed(j2, oa2, b2, p2 < tot);
    }
  }

  // Emits the window [base, base + ncols) in column order at out (checked
  // against out_end), clears it, returns the number of entries.
  __device__ __forceinline__ long long emit(int base, int ncols, long long out, long long out_end,
                                            int32_t* __restrict__ c_ci, T* __restrict__ c_v) {
    const int lane = lane_id();
    const long long start = out;
    __syncwarp();
    for (int cb = 0; cb < ncols; cb += 512) {
      uint4* qp = reinterpret_cast<uint4*>(own + cb + lane * 16);
      const uint4 q = *qp;
      unsigned m = byte_mask16(q);
      const int cnt = __popc(m);
      const int inc = warp_incl_scan(cnt);
      long long pos = out + inc - cnt;
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const int jj = cb + lane * 16 + b;
        if (pos < out_end) {
          c_ci[pos] = base + jj;
          c_v[pos] = acc[jj];
        } else {
          atomicOr(err, EB_INTERNAL);
        }
        acc[jj] = T(0);
        ++pos;
      }
      if (cnt) *qp = make_uint4(0u, 0u, 0u, 0u);
      out += __shfl_sync(FULL, inc, 31);
    }
    __syncwarp();
    return out - start;
  }
};

// Binary search: first index in [lo, hi) with B.ci[idx] >= c (hi if none).
__device__ __forceinline__ int lower_bound_col(const int32_t* __restrict__ ci, int lo, int hi, int c) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (ci[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

template <int W, int NWARP, typename T>
__global__ void __launch_bounds__(NWARP * 32)
k_num_warp(Csr A, Csr B, const T* __restrict__ av, const T* __restrict__ bv, RowInfo ri, const DevStats* st,
           int bin_lo, int bin_hi, NumSplit sp, int32_t* __restrict__ gcur, int32_t* __restrict__ gnxt,
           const int32_t* __restrict__ c_rp, int32_t* __restrict__ c_ci, T* __restrict__ c_v, uint32_t* err) {
  static_assert(W % 512 == 0, "window must be a multiple of 512 columns");
  constexpr size_t WB = (size_t)W * sizeof(T) + W;  // per-warp bytes
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_lb, s_le, s_nh;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  WarpWin<W, T> win;
  win.acc = reinterpret_cast<T*>(smem_raw + (size_t)warp * WB);
  win.own = reinterpret_cast<uint8_t*>(smem_raw + (size_t)warp * WB + (size_t)W * sizeof(T));
  win.err = err;
  for (int t = lane; t < W; t += 32) win.acc[t] = T(0);
  for (int t = lane; t < W / 16; t += 32) reinterpret_cast<uint4*>(win.own)[t] = make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) {
    int b, e;
    bin_range(st, bin_lo, bin_hi, &b, &e);
    s_lb = b;
    s_le = e;
    int hb, he;  // split rows: the leading rows of bins >= heavy_bin, within capacity
    bin_range(st, sp.heavy_bin > bin_lo ? sp.heavy_bin : bin_lo, bin_hi, &hb, &he);
    int nh = (sp.heavy_bin <= bin_hi && hb == b) ? he - hb : 0;
    s_nh = nh < sp.hcap ? nh : sp.hcap;
  }
  if (block_skip(st)) return;
  const int lb = s_lb, le = s_le, nh = s_nh;
  const long long nsplit_items = (long long)nh * sp.ntf;
  const long long total = nsplit_items + (le - lb - nh);
  const int wshift = 31 - __clz(W);

  while (true) {
    long long item = 0;
    if (lane == 0) item = atomicAdd(sp.counter, 1u);
    item = __shfl_sync(FULL, item, 0);
    if (item >= total) break;
    if (item < nsplit_items) {
      // ---- one W-column tile of a split row
      const int h = (int)(item / sp.ntf), tf = (int)(item % sp.ntf);
      const int r = ri.rows[lb + h];
      const int cmn = ri.cmin[r], cmx = ri.cmax[r];
      const int tbase = tf << wshift;
      if (tbase + W - 1 < cmn || tbase > cmx) continue;
      // output offset: row start + counts of the row's earlier tiles
      const int32_t* hc = sp.hcnt + (size_t)h * sp.ntf;
      int before = 0;
      for (int t = lane; t < tf; t += 32) before += hc[t];
      before = warp_sum(before);
      const long long out0 = (long long)c_rp[r] + before;
      const long long out_end = out0 + hc[tf];
      if (before < 0 || hc[tf] < 0 || out_end > (long long)c_rp[r + 1]) {  // inconsistent counts
        if (lane == 0) atomicOr(err, EB_INTERNAL);
        continue;
      }
      const long long i = ri.row_begin + r;
      const int a0 = A.rp[i], a1 = A.rp[i + 1];
      const int tc = tbase >> sp.tc_shift;
      const int tend = tbase + W;
      for (int e0 = a0; e0 < a1; e0 += 32) {
        const int e = e0 + lane;
        int s = 0, len = 0;
        T a = T(0);
        if (e < a1) {
          const int k = A.ci[e];
          a = av[e];
          const int32_t* bk = sp.bnd + (size_t)k * (sp.ntc + 1) + tc;
          const int cs = bk[0], ce = bk[1];
          if (cs < ce) {
            const int lo = lower_bound_col(B.ci, cs, ce, tbase);
            const int hi = lower_bound_col(B.ci, lo, ce, tend);
            s = lo;
            len = hi - lo;
          }
        }
        win.segments(B, bv, s, len, a, tbase);
      }
      const int ncols = min(W, cmx - tbase + 1);
      const long long n = win.emit(tbase, (ncols + 511) & ~511, out0, out_end, c_ci, c_v);
      if (lane == 0 && out0 + n != out_end) atomicOr(err, EB_INTERNAL);
      continue;
    }
    // ---- a whole row, swept window by window
    const long long idx = lb + nh + (item - nsplit_items);
    const int r = ri.rows[idx];
    const long long i = ri.row_begin + r;
    const int a0 = A.rp[i], a1 = A.rp[i + 1], nA = a1 - a0;
    const int cmx = ri.cmax[r];
    const long long out_beg = c_rp[r], out_end = c_rp[r + 1];
    long long out = out_beg;
    if (nA <= 32 * NW_SLOTS) {
      const int nslots = (nA + 31) >> 5;
      int cur[NW_SLOTS], end[NW_SLOTS], nx[NW_SLOTS];
      T a[NW_SLOTS];
      int mn = INT_MAX;
#pragma unroll
      for (int q = 0; q < NW_SLOTS; ++q) {
        cur[q] = 0; end[q] = 0; nx[q] = INT_MAX; a[q] = T(0);
        if (q < nslots) {
          const int e = a0 + q * 32 + lane;
          if (e < a1) {
            const int k = A.ci[e];
            a[q] = av[e];
            cur[q] = B.rp[k];
            end[q] = B.rp[k + 1];
            nx[q] = cur[q] < end[q] ? B.ci[cur[q]] : INT_MAX;
          }
          mn = min(mn, nx[q]);
        }
      }
      int base = warp_min(mn);
      while (base != INT_MAX) {
        const int wend = (int)min((long long)base + W, (long long)INT_MAX);
        mn = INT_MAX;
#pragma unroll
        for (int q = 0; q < NW_SLOTS; ++q) {
          if (q < nslots) {
            int s = cur[q], len = 0;
            if (nx[q] < wend) {
              int seg = end[q], nn = INT_MAX;
              if (B.ci[end[q] - 1] >= wend) {
                seg = lower_bound_col(B.ci, cur[q] + 1, end[q] - 1, wend);
                nn = B.ci[seg];
              }
              len = seg - cur[q];
              cur[q] = seg;
              nx[q] = nn;
            }
            win.segments(B, bv, s, len, a[q], base);
            mn = min(mn, nx[q]);
          }
        }
        const int ncols = min(W, cmx - base + 1);
        out += win.emit(base, (ncols + 511) & ~511, out, out_end, c_ci, c_v);
        base = warp_min(mn);
      }
    } else {
      // cursors in global arrays parallel to A's nonzeros (one warp per row)
      int mn = INT_MAX;
      for (int e = a0 + lane; e < a1; e += 32) {
        const int k = A.ci[e];
        const int c0 = B.rp[k], c1 = B.rp[k + 1];
        gcur[e] = c0;
        const int v = c0 < c1 ? B.ci[c0] : INT_MAX;
        gnxt[e] = v;
        mn = min(mn, v);
      }
      int base = warp_min(mn);
      while (base != INT_MAX) {
        const int wend = (int)min((long long)base + W, (long long)INT_MAX);
        mn = INT_MAX;
        for (int e0 = a0; e0 < a1; e0 += 32) {
          const int e = e0 + lane;
          int s = 0, len = 0;
          T av_e = T(0);
          if (e < a1) {
            const int nxe = gnxt[e];
            if (nxe < wend) {
              const int k = A.ci[e];
              const int c1 = B.rp[k + 1];
              const int c0 = gcur[e];
              av_e = av[e];
              int seg = c1, nn = INT_MAX;
              if (B.ci[c1 - 1] >= wend) {
                seg = lower_bound_col(B.ci, c0 + 1, c1 - 1, wend);
                nn = B.ci[seg];
              }
              s = c0;
              len = seg - c0;
              gcur[e] = seg;
              gnxt[e] = nn;
              mn = min(mn, nn);
            } else {
              mn = min(mn, nxe);
            }
          }
          win.segments(B, bv, s, len, av_e, base);
        }
        const int ncols = min(W, cmx - base + 1);
        out += win.emit(base, (ncols + 511) & ~511, out, out_end, c_ci, c_v);
        base = warp_min(mn);
      }
    }
    if (lane == 0 && out != out_end) atomicOr(err, EB_INTERNAL);
  }
}

}  // namespace sg
