// Numeric pass, dense-window accumulator owned by one warp.
//
// Row i of C is the sum over A(i,k) of A(i,k) * B(k,:) (Sec. 2.2).  A warp
// owns a window of W consecutive columns in shared memory: a dense value
// array and a presence bit per column.
// Rows of B are sorted, so the part of B(k,:) inside a window is one
// contiguous segment.  Only this warp touches the window.  When the warp
// walks one long segment its lanes hit distinct columns, so each product is
// one fused multiply-add, acc[j] = fma(A(i,k), B(k,j), acc[j]), without
// atomics.  Products of several short segments are spread over the lanes
// and may share columns; those go through shared-memory atomic adds.  The
// window is emitted in column order by a popcount prefix over a presence
// bitmap, so no sort is needed, and cleared on the way out.
//
// Windows are aligned to multiples of W, and B comes with its window-run
// list (runs of entries of one row inside one window, see SplitInfo), so the
// segment of B(k,:) in a window is exactly one run: [start_j, start_{j+1}).
//
// Work items, handed out largest first through a global counter:
//  * split rows (heavy rows, product count above a threshold): one item per
//    window of the row.  Each nonzero finds its run for the window by binary
//    search over the runs of its B row; the item writes at the offset given
//    by the per-window output counts of the symbolic pass.
//  * other rows: one item per row, swept window by window; the next window
//    is the smallest window id among the nonzeros' current runs.  Each
//    nonzero's run cursor lives in registers (up to 32 * SLOTS nonzeros per
//    row) or in global arrays parallel to A's nonzeros.
#pragma once

#include "internal.cuh"
#include "semiring.cuh"

namespace sg {

struct NumSplit {
  int heavy_bin;          // rows in bins [heavy_bin, hi_bin] are split (within capacity)
  int hi_bin;
  int hcap;               // capacity of the per-window count table (rows)
  int ntf;                // windows (of W columns) per row
  const int32_t* rr;      // B's run pointers (nrows(B) + 1)
  const int2* runs;       // B's runs: (window id, start), sentinel per row
  const int32_t* hcnt;    // output counts per (split row, window)
  unsigned* counter;      // work counter, zero before the launch
};

constexpr int NW_SLOTS = 8;  // register cursors: up to 256 nonzeros of A per row

template <int W, typename T, int SR = SPGEMM_PLUS_TIMES>
struct WarpWin {
  using Ops = SrOps<T, SR>;
  T* acc;
  uint32_t* bits;   // presence bitmap, W / 32 words
  uint32_t* err;

  __device__ __forceinline__ void mark(int j) { atomicOr(&bits[j >> 5], 1u << (j & 31)); }

  // Lanes carry products of one segment: distinct columns, no claim needed.
  // The column is marked present on its first update (the word still +0.0,
  // its cleared state).
  __device__ __forceinline__ void add_distinct(int j, T a, T b, bool act) {
    if (act) {
      if ((unsigned)j < (unsigned)W) {
        const T old = acc[j];
        acc[j] = Ops::madd(a, b, old);
        if (Ops::cleared(old)) mark(j);
      } else {
        atomicOr(err, EB_UNSORTED);
      }
    }
  }

  // Lanes may carry equal columns (short segments of different B rows often
  // share the hub columns): shared-memory atomic add, which resolves equal
  // addresses in hardware.  (The compare-and-swap of fma_shared saves an FP64
  // operation per product, but its round trip lengthens this latency-bound
  // loop: measured 7 % slower here.)
  __device__ __forceinline__ void add_atomic(int j, T a, T b, bool act) {
    if (act) {
      if ((unsigned)j < (unsigned)W) {
        mark(j);
        Ops::red_shared(&acc[j], a, b, err);
      } else {
        atomicOr(err, EB_UNSORTED);
      }
    }
  }

  // Products of long segments (at least 32 entries; one segment per lane,
  // the others skipped): the whole warp walks one segment at a time.
  __device__ __forceinline__ void long_segments(const Csr& B, const T* __restrict__ bv, int s, int len, T a,
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
  }

  // Short segments (fewer than 32 entries) are flattened so every lane takes
  // one product.  flat_gather places the first 64 products and issues their
  // loads; flat_apply adds them (and any further products).  Splitting the
  // two lets a caller issue a later window's loads before it emits this one.
  struct Flat {
    int tot, incl, excl, j0, j1;
    T b0, b1, a0, a1;
  };

  __device__ __forceinline__ void flat_gather(const Csr& B, const T* __restrict__ bv, int s, int len, T a, int base,
                                              Flat& f) {
    const int lane = lane_id();
    const int sl = len < 32 ? len : 0;
    f.incl = warp_incl_scan(sl);
    f.tot = __shfl_sync(FULL, f.incl, 31);
    f.excl = f.incl - sl;
    f.j0 = f.j1 = 0;
    f.b0 = f.b1 = f.a0 = f.a1 = T(0);
    if (f.tot == 0) return;
    const int p = lane, p2 = lane + 32;
    const int o = warp_owner(f.incl, p), o2 = warp_owner(f.incl, p2);
    const int os = __shfl_sync(FULL, s, o), oex = __shfl_sync(FULL, f.excl, o);
    f.a0 = __shfl_sync(FULL, a, o);
    const int os2 = __shfl_sync(FULL, s, o2), oex2 = __shfl_sync(FULL, f.excl, o2);
    f.a1 = __shfl_sync(FULL, a, o2);
    if (p < f.tot) {
      const int bi = os + p - oex;
      f.j0 = B.ci[bi] - base;
      f.b0 = bv[bi];
    }
    if (p2 < f.tot) {
      const int bi = os2 + p2 - oex2;
      f.j1 = B.ci[bi] - base;
      f.b1 = bv[bi];
    }
  }

  // s, a: the same lane values flat_gather had.
  __device__ __forceinline__ void flat_apply(const Csr& B, const T* __restrict__ bv, int s, T a, int base,
                                             const Flat& f) {
    const int lane = lane_id();
    if (f.tot == 0) return;
    add_atomic(f.j0, f.a0, f.b0, lane < f.tot);
    add_atomic(f.j1, f.a1, f.b1, lane + 32 < f.tot);
    for (int p0 = 64; p0 < f.tot; p0 += 64) {
      const int p = p0 + lane, p2 = p + 32;
      const int o = warp_owner(f.incl, p), o2 = warp_owner(f.incl, p2);
      const int os = __shfl_sync(FULL, s, o), oex = __shfl_sync(FULL, f.excl, o);
      const T oa = __shfl_sync(FULL, a, o);
      const int os2 = __shfl_sync(FULL, s, o2), oex2 = __shfl_sync(FULL, f.excl, o2);
      const T oa2 = __shfl_sync(FULL, a, o2);
      int j = 0, j2 = 0;
      T b = T(0), b2 = T(0);
      if (p < f.tot) {
        const int bi = os + p - oex;
        j = B.ci[bi] - base;
        b = bv[bi];
      }
      if (p2 < f.tot) {
        const int bi = os2 + p2 - oex2;
        j2 = B.ci[bi] - base;
        b2 = bv[bi];
      }
      add_atomic(j, oa, b, p < f.tot);
      add_atomic(j2, oa2, b2, p2 < f.tot);
    }
    __syncwarp();
  }

  // Products of segments [s, s+len) of B with multiplier a (one segment per
  // lane), columns relative to base.
  __device__ __forceinline__ void segments(const Csr& B, const T* __restrict__ bv, int s, int len, T a,
                                           int base) {
    if (!__any_sync(FULL, len > 0)) return;
    long_segments(B, bv, s, len, a, base);
    Flat f;
    flat_gather(B, bv, s, len, a, base, f);
    flat_apply(B, bv, s, a, base, f);
  }

  // Emits the window [base, base + ncols) in column order at c_ci/c_v + out
  // (offsets relative to the row's first entry, checked against out_end),
  // clears it, returns the number of entries.  Lanes take consecutive outputs
  // (the word of an output from a warp search over the words' popcount
  // prefix, its bit from a binary search on popcounts inside the word), so a
  // window takes ceil(entries / 32) steps and the stores of C are coalesced.
  __device__ __forceinline__ int emit(int base, int ncols, int out, int out_end,
                                                int32_t* __restrict__ c_ci, T* __restrict__ c_v) {
    const int lane = lane_id();
    const int nw = (ncols + 31) >> 5;
    __syncwarp();
    int total = 0;
    for (int wb = 0; wb < nw; wb += 32) {
      const int wi = wb + lane;
      const uint32_t m = wi < nw ? bits[wi] : 0u;
      const int c = __popc(m);
      const int inc = warp_incl_scan(c);
      const int tot = __shfl_sync(FULL, inc, 31);
      const int exc = inc - c;
      for (int t0 = 0; t0 < tot; t0 += 32) {
        const int t = t0 + lane;
        const int o = warp_owner(inc, t);
        const uint32_t mo = __shfl_sync(FULL, m, o & 31);
        const int eo = __shfl_sync(FULL, exc, o & 31);
        if (t < tot) {
          uint32_t x = mo;
          int rank = t - eo, bit = 0;
#pragma unroll
          for (int sh = 16; sh >= 1; sh >>= 1) {
            const int lowc = __popc(x & ((1u << sh) - 1u));
            if (rank >= lowc) {
              rank -= lowc;
              x >>= sh;
              bit += sh;
            }
          }
          const int jj = ((wb + o) << 5) + bit;
          const T v = acc[jj];
          acc[jj] = Ops::zero();
          const int pos = out + total + t;
          if (pos < out_end) {
            __stcs(c_ci + pos, base + jj);
            __stcs(c_v + pos, v);
          } else {
            atomicOr(err, EB_INTERNAL);
          }
        }
      }
      if (m) bits[wi] = 0u;  // each lane clears the word it read; others used a shuffled copy
      total += tot;
    }
    __syncwarp();
    return total;
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

// First run of [lo, hi) whose window id is >= w (hi if none).
__device__ __forceinline__ int lower_bound_run(const int2* __restrict__ runs, int lo, int hi, int w) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (runs[mid].x < w) lo = mid + 1; else hi = mid;
  }
  return lo;
}

template <int W, int NWARP, typename T, int SR = SPGEMM_PLUS_TIMES>
__global__ void __launch_bounds__(NWARP * 32)
k_num_warp(Csr A, Csr B, const T* __restrict__ av, const T* __restrict__ bv, RowInfo ri, const DevStats* st,
           int bin_lo, int bin_hi, NumSplit sp, int32_t* __restrict__ gcur, int32_t* __restrict__ gnxt,
           const int32_t* __restrict__ c_rp, int32_t* __restrict__ c_ci, T* __restrict__ c_v, uint32_t* err,
           int skip_small) {
  static_assert(W % 512 == 0, "window must be a multiple of 512 columns");
  constexpr size_t WB = (size_t)W * sizeof(T) + W / 8;  // per-warp bytes
  constexpr int WSHIFT = (W == 512) ? 9 : (W == 1024) ? 10 : (W == 2048) ? 11 : (W == 4096) ? 12 : 13;
  static_assert((1 << WSHIFT) == W, "window must be a power of two");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_lb, s_le, s_nh;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  WarpWin<W, T, SR> win;
  win.acc = reinterpret_cast<T*>(smem_raw + (size_t)warp * WB);
  win.bits = reinterpret_cast<uint32_t*>(smem_raw + (size_t)warp * WB + (size_t)W * sizeof(T));
  win.err = err;
  for (int t = lane; t < W; t += 32) win.acc[t] = SrOps<T, SR>::zero();
  for (int t = lane; t < W / 32; t += 32) win.bits[t] = 0u;
  if (threadIdx.x == 0) {
    int b, e;
    bin_range(st, bin_lo, bin_hi, &b, &e);
    s_lb = b;
    s_le = e;
    // split rows (bins [heavy_bin, hi_bin], the symbolic pass's numbering):
    // only when they are the leading rows of this launch's range
    int nh = 0, hb = 0, he = 0;
    if (sp.heavy_bin < NBINS && sp.hi_bin >= sp.heavy_bin && sp.heavy_bin >= bin_lo && sp.hi_bin == bin_hi) {
      bin_range(st, sp.heavy_bin, sp.hi_bin, &hb, &he);
      if (hb == b) nh = he - hb;
    }
    s_nh = nh < sp.hcap ? nh : sp.hcap;
  }
  if (block_skip(st)) return;
  const int lb = s_lb, le = s_le, nh = s_nh;
  const long long nsplit_items = (long long)nh * sp.ntf;
  const long long total = nsplit_items + (le - lb - nh);

  while (true) {
    long long item = 0;
    if (lane == 0) item = atomicAdd(sp.counter, 1u);
    item = __shfl_sync(FULL, item, 0);
    if (item >= total) break;
    if (item < nsplit_items) {
      // ---- one window of a split row
      const int h = (int)(item / sp.ntf), tw = (int)(item % sp.ntf);
      const int r = ri.rows[lb + h];
      const int cmn = ri.cmin[r], cmx = ri.cmax[r];
      const int tbase = tw << WSHIFT;
      if (tbase + W - 1 < cmn || tbase > cmx) continue;
      const int32_t* hc = sp.hcnt + (size_t)h * sp.ntf;
      int before = 0;
      for (int t = lane; t < tw; t += 32) before += hc[t];
      before = warp_sum(before);
      const long long rbeg = c_rp[r];
      const int out0 = before;
      const int out_end = out0 + hc[tw];
      if (before < 0 || hc[tw] < 0 || rbeg + out_end > (long long)c_rp[r + 1]) {  // inconsistent counts
        if (lane == 0) atomicOr(err, EB_INTERNAL);
        continue;
      }
      const long long i = ri.row_begin + r;
      const int a0 = A.rp[i], a1 = A.rp[i + 1];
      for (int e0 = a0; e0 < a1; e0 += 32) {
        const int e = e0 + lane;
        int s = 0, len = 0;
        T a = T(0);
        if (e < a1) {
          const int k = A.ci[e];
          a = av[e];
          const int r0 = sp.rr[k], r1 = sp.rr[k + 1] - 1;  // runs without the sentinel
          const int j = lower_bound_run(sp.runs, r0, r1, tw);
          if (j < r1) {
            const int2 cur = sp.runs[j];
            if (cur.x == tw) {
              s = cur.y;
              len = sp.runs[j + 1].y - cur.y;
            }
          }
        }
        win.segments(B, bv, s, len, a, tbase);
      }
      const int ncols = min(W, cmx - tbase + 1);
      const int n = win.emit(tbase, ncols, out0, out_end, c_ci + rbeg, c_v + rbeg);
      if (lane == 0 && out0 + n != out_end) atomicOr(err, EB_INTERNAL);
      continue;
    }
    // ---- a whole row, swept window by window
    const long long idx = lb + nh + (item - nsplit_items);
    const int r = ri.rows[idx];
    const long long i = ri.row_begin + r;
    const int a0 = A.rp[i], a1 = A.rp[i + 1], nA = a1 - a0;
    if (skip_small && nA <= 32) continue;  // k_num_warp1 takes the row
    const int cmx = ri.cmax[r];
    const long long rbeg = c_rp[r];
    const int out_end = (int)(c_rp[r + 1] - rbeg);
    int32_t* const rci = c_ci + rbeg;
    T* const rcv = c_v + rbeg;
    int out = 0;
    if (nA <= 32 * NW_SLOTS) {
      // cursor per nonzero: run index j, its window id and segment [s0, s1)
      const int nslots = (nA + 31) >> 5;
      int rj[NW_SLOTS], wid[NW_SLOTS], s0[NW_SLOTS], s1[NW_SLOTS];
      T a[NW_SLOTS];
      int mn = INT_MAX;
#pragma unroll
      for (int q = 0; q < NW_SLOTS; ++q) {
        rj[q] = 0; wid[q] = INT_MAX; s0[q] = 0; s1[q] = 0; a[q] = T(0);
        if (q < nslots) {
          const int e = a0 + q * 32 + lane;
          if (e < a1) {
            const int k = A.ci[e];
            a[q] = av[e];
            rj[q] = sp.rr[k];
            const int2 c0 = sp.runs[rj[q]];
            wid[q] = c0.x;
            s0[q] = c0.y;
            if (c0.x != INT_MAX) s1[q] = sp.runs[rj[q] + 1].y;  // empty rows hold only the sentinel
          }
          mn = min(mn, wid[q]);
        }
      }
      int w = warp_min(mn);
      while (w != INT_MAX) {
        const int base = w << WSHIFT;
        mn = INT_MAX;
#pragma unroll
        for (int q = 0; q < NW_SLOTS; ++q) {
          if (q < nslots) {
            const bool act = wid[q] == w;
            // issue the loads of the next run before this window's products,
            // so their latency overlaps the accumulation
            int2 nx = make_int2(wid[q], s0[q]);
            int nend = s1[q];
            if (act) {
              nx = sp.runs[rj[q] + 1];
              if (nx.x != INT_MAX) nend = sp.runs[rj[q] + 2].y;
            }
            win.segments(B, bv, s0[q], act ? s1[q] - s0[q] : 0, a[q], base);
            if (act) {  // advance to the next run of this B row
              ++rj[q];
              wid[q] = nx.x;
              s0[q] = nx.y;
              s1[q] = nend;
            }
            mn = min(mn, wid[q]);
          }
        }
        const int ncols = min(W, cmx - base + 1);
        out += win.emit(base, ncols, out, out_end, rci, rcv);
        w = warp_min(mn);
      }
    } else {
      // run cursors in global arrays parallel to A's nonzeros (one warp per row)
      int mn = INT_MAX;
      for (int e = a0 + lane; e < a1; e += 32) {
        const int k = A.ci[e];
        const int j = sp.rr[k];
        gcur[e] = j;
        const int v = sp.runs[j].x;
        gnxt[e] = v;
        mn = min(mn, v);
      }
      int w = warp_min(mn);
      while (w != INT_MAX) {
        const int base = w << WSHIFT;
        mn = INT_MAX;
        for (int e0 = a0; e0 < a1; e0 += 32) {
          const int e = e0 + lane;
          int s = 0, len = 0;
          T av_e = T(0);
          if (e < a1) {
            const int we = gnxt[e];
            if (we == w) {
              const int j = gcur[e];
              const int2 c0 = sp.runs[j], c1 = sp.runs[j + 1];
              av_e = av[e];
              s = c0.y;
              len = c1.y - c0.y;
              gcur[e] = j + 1;
              gnxt[e] = c1.x;
              mn = min(mn, c1.x);
            } else {
              mn = min(mn, we);
            }
          }
          win.segments(B, bv, s, len, av_e, base);
        }
        const int ncols = min(W, cmx - base + 1);
        out += win.emit(base, ncols, out, out_end, rci, rcv);
        w = warp_min(mn);
      }
    }
    if (lane == 0 && out != out_end) atomicOr(err, EB_INTERNAL);
  }
}

// Rows of at most 32 nonzeros of A (not split): one cursor per lane.  Each
// lane holds its current run and the next one, and loads the run after
// that one window ahead, so the next window is known at the top of a
// window: its short-segment products are placed and their loads issued
// before this window's products are accumulated and emitted, which hide
// their latency.  Same accumulator, emission and result as k_num_warp.
template <int W, int NWARP, typename T, int SR = SPGEMM_PLUS_TIMES>
__global__ void __launch_bounds__(NWARP * 32, W <= 1024 ? 3 : 1)
k_num_warp1(Csr A, Csr B, const T* __restrict__ av, const T* __restrict__ bv, RowInfo ri, const DevStats* st,
            int bin_lo, int bin_hi, NumSplit sp, const int32_t* __restrict__ c_rp, int32_t* __restrict__ c_ci,
            T* __restrict__ c_v, unsigned* counter, uint32_t* err) {
  constexpr size_t WB = (size_t)W * sizeof(T) + W / 8;  // per-warp bytes
  constexpr int WSHIFT = (W == 512) ? 9 : (W == 1024) ? 10 : (W == 2048) ? 11 : (W == 4096) ? 12 : 13;
  static_assert((1 << WSHIFT) == W, "window must be a power of two");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_lb, s_le, s_nh;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  WarpWin<W, T, SR> win;
  win.acc = reinterpret_cast<T*>(smem_raw + (size_t)warp * WB);
  win.bits = reinterpret_cast<uint32_t*>(smem_raw + (size_t)warp * WB + (size_t)W * sizeof(T));
  win.err = err;
  for (int t = lane; t < W; t += 32) win.acc[t] = SrOps<T, SR>::zero();
  for (int t = lane; t < W / 32; t += 32) win.bits[t] = 0u;
  if (threadIdx.x == 0) {
    int b, e;
    bin_range(st, bin_lo, bin_hi, &b, &e);
    s_lb = b;
    s_le = e;
    // split rows are the leading rows of the range (k_num_warp takes them)
    int nh = 0, hb = 0, he = 0;
    if (sp.heavy_bin < NBINS && sp.hi_bin >= sp.heavy_bin && sp.heavy_bin >= bin_lo && sp.hi_bin == bin_hi) {
      bin_range(st, sp.heavy_bin, sp.hi_bin, &hb, &he);
      if (hb == b) nh = he - hb;
    }
    s_nh = nh < sp.hcap ? nh : sp.hcap;
  }
  if (block_skip(st)) return;
  const int lb = s_lb, le = s_le, nh = s_nh;
  while (true) {
    long long item = 0;
    if (lane == 0) item = atomicAdd(counter, 1u);
    item = __shfl_sync(FULL, item, 0);
    const long long idx = (long long)lb + nh + item;
    if (idx >= le) break;
    const int r = ri.rows[idx];
    const long long i = ri.row_begin + r;
    const int a0 = A.rp[i], a1 = A.rp[i + 1];
    if (a1 - a0 > 32) continue;  // k_num_warp takes the row
    const int cmx = ri.cmax[r];
    const long long rbeg = c_rp[r];
    const int out_end = (int)(c_rp[r + 1] - rbeg);
    int32_t* const rci = c_ci + rbeg;
    T* const rcv = c_v + rbeg;
    // this lane's nonzero: its current run (window wid, segment [s0, s1))
    // and the next one (nwid, [ns0, ns1)); entries read past a row's
    // sentinel are padding and never used
    int rj = 0, wid = INT_MAX, s0 = 0, s1 = 0, nwid = INT_MAX, ns0 = 0, ns1 = 0;
    T a = T(0);
    const int e = a0 + lane;
    if (e < a1) {
      const int k = A.ci[e];
      a = av[e];
      rj = sp.rr[k];
      const int2 c0 = sp.runs[rj], c1 = sp.runs[rj + 1];
      const int y2 = sp.runs[rj + 2].y;
      if (c0.x != INT_MAX) {  // empty rows hold only the sentinel
        wid = c0.x;
        s0 = c0.y;
        s1 = c1.y;
        nwid = c1.x;
        ns0 = c1.y;
        ns1 = y2;
      }
    }
    int w = warp_min(wid);
    typename WarpWin<W, T, SR>::Flat f;
    if (w != INT_MAX) win.flat_gather(B, bv, s0, wid == w ? s1 - s0 : 0, a, w << WSHIFT, f);
    int out = 0;
    while (w != INT_MAX) {
      const int base = w << WSHIFT;
      const bool act = wid == w;
      // the run after the next one, for the window after the next
      int2 n2 = make_int2(INT_MAX, 0);
      int n2end = 0;
      if (act && nwid != INT_MAX) {
        n2 = sp.runs[rj + 2];
        n2end = sp.runs[rj + 3].y;
      }
      // the next window and its short-segment products, their loads in
      // flight while this window is accumulated and emitted
      const int wid1 = act ? nwid : wid, s01 = act ? ns0 : s0, s11 = act ? ns1 : s1;
      const int wn = warp_min(wid1);
      typename WarpWin<W, T, SR>::Flat fn;
      if (wn != INT_MAX) win.flat_gather(B, bv, s01, wid1 == wn ? s11 - s01 : 0, a, wn << WSHIFT, fn);
      const int len = act ? s1 - s0 : 0;
      win.long_segments(B, bv, s0, len, a, base);
      win.flat_apply(B, bv, s0, a, base, f);
      const int ncols = min(W, cmx - base + 1);
      out += win.emit(base, ncols, out, out_end, rci, rcv);
      if (act) {
        ++rj;
        wid = nwid;
        s0 = ns0;
        s1 = ns1;
        nwid = n2.x;
        ns0 = n2.y;
        ns1 = n2end;
      }
      f = fn;
      w = wn;
    }
    if (lane == 0 && out != out_end) atomicOr(err, EB_INTERNAL);
  }
}

}  // namespace sg
