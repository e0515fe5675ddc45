// Row kernels shared by the symbolic pass (sizes of C's rows) and the
// numeric pass (C's columns and values).  Both follow the row-wise Gustavson
// method (Sec. 2.2): row i of C accumulates A(i,k) * B(k,:) over the nonzeros
// of A's row i, and equal columns are merged by adding their values
// (Sec. 2.2, Algorithm 1), leaving the row's columns ascending and unique.
//
// Two accumulators are used, chosen per row by its product count P:
//
//  * register sort (P <= 32): a group of G lanes holds one product per lane,
//    sorts the (column, value) pairs with a bitonic network over shuffles
//    and adds runs of equal columns with a segmented suffix sum.  The sorted
//    order is the output order, so nothing is written to shared memory.
//
//  * dense column window: a warp (or a block) owns a window of W
//    consecutive columns held as a presence bitmap plus, for the numeric
//    pass, a dense value array in shared memory.  Every B row touched by the
//    row is read from a per-nonzero cursor up to the window's end (rows of
//    B are sorted, so that is one contiguous segment), products are added
//    with shared-memory atomics, and the window is emitted in column order
//    by a popcount prefix over the bitmap -- no sort is needed.  The next
//    window starts at the smallest column still unread, so windows skip
//    column ranges the row does not touch.
#pragma once

#include "internal.cuh"

namespace sg {

// ---------------------------------------------------------------- tiny path
// One row per group of G lanes (G in 8/16/32), P <= G products.
template <int G, bool NUM, typename T>
__global__ void __launch_bounds__(256)
k_tiny(Csr A, Csr B, const T* __restrict__ av, const T* __restrict__ bv, RowInfo ri,
       const DevStats* st, int bin_lo, int bin_hi, int32_t* __restrict__ c_cnt,
       const int32_t* __restrict__ c_rp, int32_t* __restrict__ c_ci, T* __restrict__ c_v,
       uint32_t* err) {
  __shared__ int s_lb, s_le;
  if (threadIdx.x == 0) bin_range(st, bin_lo, bin_hi, &s_lb, &s_le);
  if (block_skip(st)) return;
  const int lb = s_lb, le = s_le;
  const int lane = lane_id();
  const int gl = lane & (G - 1);
  const int gi = lane / G;
  constexpr int GPW = 32 / G;
  const unsigned gmask = (G == 32) ? FULL : (((1u << G) - 1u) << (gi * G));
  const long long warp_g = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = (gridDim.x * (long long)blockDim.x) >> 5;
  for (long long wb = lb + warp_g * GPW; wb < le; wb += nwarps * GPW) {
    const long long idx = wb + gi;
    const bool vrow = idx < le;
    int r = 0, a0 = 0, a1 = 0;
    if (vrow) {
      r = ri.rows[idx];
      const long long i = ri.row_begin + r;
      a0 = A.rp[i];
      a1 = A.rp[i + 1];
    }
    // Gather: lane gl of the group takes the row's gl-th product.
    int col = INT_MAX;
    T val = T(0);
    int done = 0;
    for (int e0 = a0; __any_sync(FULL, e0 < a1); e0 += G) {
      const int e = e0 + gl;
      int s = 0, len = 0;
      T a = T(0);
      if (e < a1) {
        const int k = A.ci[e];
        s = B.rp[k];
        len = B.rp[k + 1] - s;
        if (NUM) a = av[e];
      }
      int incl = len;
#pragma unroll
      for (int d = 1; d < G; d <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, d, G);
        if (gl >= d) incl += t;
      }
      const int tot = __shfl_sync(FULL, incl, G - 1, G);
      const int q = gl - done;
      int o = 0;
#pragma unroll
      for (int sp = G / 2; sp >= 1; sp >>= 1) {
        const int t = __shfl_sync(FULL, incl, o + sp - 1, G);
        if (t <= q) o += sp;
      }
      const int os = __shfl_sync(FULL, s, o, G);
      const int oex = __shfl_sync(FULL, incl - len, o, G);
      const T oa = __shfl_sync(FULL, a, o, G);
      if (q >= 0 && q < tot) {
        const int bi = os + q - oex;
        col = B.ci[bi];
        if (NUM) val = oa * bv[bi];
      }
      done += tot;
    }
    if (!NUM) {
      // Distinct columns: one leader per run of equal keys inside the group.
      const unsigned long long key = ((unsigned long long)(unsigned)gi << 32) | (unsigned)col;
      const unsigned m = __match_any_sync(FULL, key);
      const bool leader = col != INT_MAX && (__ffs(m) - 1) == lane;
      const int cnt = __popc(__ballot_sync(FULL, leader) & gmask);
      if (vrow && gl == 0) c_cnt[r] = cnt;
    } else {
      // Bitonic sort of (col, val) by col inside the group.
#pragma unroll
      for (int k = 2; k <= G; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
          const int pc = __shfl_xor_sync(FULL, col, j);
          const T pv = __shfl_xor_sync(FULL, val, j);
          const bool up = (gl & k) == 0;
          const bool lower = (gl & j) == 0;
          const bool take = (lower == up) ? (pc < col) : (pc > col);
          if (take) {
            col = pc;
            val = pv;
          }
        }
      }
      // Segmented suffix sum over runs of equal columns.
      T acc = val;
#pragma unroll
      for (int d = 1; d < G; d <<= 1) {
        const T t = __shfl_down_sync(FULL, acc, d, G);
        const int tc = __shfl_down_sync(FULL, col, d, G);
        if (gl + d < G && tc == col) acc += t;
      }
      const int prevc = __shfl_up_sync(FULL, col, 1, G);
      const bool head = col != INT_MAX && (gl == 0 || prevc != col);
      const unsigned hb = __ballot_sync(FULL, head) & gmask;
      if (vrow) {
        const long long ob = c_rp[r], oe = c_rp[r + 1];
        if (head) {
          const long long o = ob + __popc(hb & lanemask_lt());
          if (o < oe) {
            c_ci[o] = col;
            c_v[o] = acc;
          }
        }
        if (gl == 0 && ob + __popc(hb) != oe) atomicOr(err, EB_INTERNAL);
      }
    }
  }
}

// ------------------------------------------------------- dense-window path
template <int GW>
__device__ __forceinline__ void group_sync(int g) {
  if (GW == 1) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(GW * 32) : "memory");
  }
}

template <int W, bool NUM, typename T>
__device__ __forceinline__ void win_insert(T* acc, uint32_t* bits, int j, T v, uint32_t* err) {
  if ((unsigned)j >= (unsigned)W) {  // only reachable with unsorted input
    atomicOr(err, EB_UNSORTED);
    return;
  }
  const uint32_t m = 1u << (j & 31);
  if (NUM) {
    atomicAdd(&acc[j], v);
    atomicOr(&bits[j >> 5], m);
  } else {
    if (!(bits[j >> 5] & m)) atomicOr(&bits[j >> 5], m);
  }
}

template <int W, bool NUM, typename T>
constexpr size_t window_group_bytes(int gw) {
  return (((NUM ? (size_t)W * sizeof(T) : 0) + (size_t)(W / 32) * 4 + (size_t)gw * 8) + 15) & ~(size_t)15;
}

// GW warps per row (group), CW warps per block, W columns per window.
template <int GW, int CW, int W, bool NUM, typename T>
__global__ void __launch_bounds__(CW * 32)
k_window(Csr A, Csr B, const T* __restrict__ av, const T* __restrict__ bv, RowInfo ri,
         const DevStats* st, int bin_lo, int bin_hi, int32_t* __restrict__ cursor,
         int32_t* __restrict__ c_cnt, const int32_t* __restrict__ c_rp, int32_t* __restrict__ c_ci,
         T* __restrict__ c_v, uint32_t* err) {
  static_assert(CW % GW == 0 && W % 32 == 0, "bad shape");
  constexpr int NWORDS = W / 32;
  constexpr int NG = CW / GW;
  constexpr size_t ACC_BYTES = NUM ? (size_t)W * sizeof(T) : 0;
  constexpr size_t GB = window_group_bytes<W, NUM, T>(GW);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_lb, s_le;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const int g = warp / GW, wig = warp % GW;
  unsigned char* gbase = smem_raw + (size_t)g * GB;
  T* acc = reinterpret_cast<T*>(gbase);
  uint32_t* bits = reinterpret_cast<uint32_t*>(gbase + ACC_BYTES);
  int* wcnt = reinterpret_cast<int*>(bits + NWORDS);
  int* wnext = wcnt + GW;
  for (int t = wig * 32 + lane; t < NWORDS; t += GW * 32) bits[t] = 0u;
  if (NUM)
    for (int t = wig * 32 + lane; t < W; t += GW * 32) acc[t] = T(0);
  if (threadIdx.x == 0) bin_range(st, bin_lo, bin_hi, &s_lb, &s_le);
  if (block_skip(st)) return;
  const int lb = s_lb, le = s_le;

  for (long long idx = lb + (long long)blockIdx.x * NG + g; idx < le; idx += (long long)gridDim.x * NG) {
    const int r = ri.rows[idx];
    const long long i = ri.row_begin + r;
    const int a0 = A.rp[i], a1 = A.rp[i + 1], nA = a1 - a0;
    int base = ri.cmin[r];
    const int last = ri.cmax[r];
    const int CS = min(32, max(1, (nA + GW - 1) / GW));  // nonzeros per chunk
    const int nch = (nA + CS - 1) / CS;
    const bool regcur = nch <= GW;  // one chunk per warp: cursor stays in a register
    int rcur = 0;
    long long obeg = 0, oend = 0;
    if (NUM) {
      obeg = c_rp[r];
      oend = c_rp[r + 1];
    }
    long long rowcount = 0;
    bool first = true;
    while (true) {
      const int wend = (int)min((long long)base + W, (long long)INT_MAX);
      int mynext = INT_MAX;
      for (int c = wig; c < nch; c += GW) {
        const int e = a0 + c * CS + lane;
        const bool ve = lane < CS && e < a1;
        int s = 0, len = 0;
        T a = T(0);
        if (ve) {
          const int k = A.ci[e];
          if (NUM) a = av[e];
          const int rs = B.rp[k], re = B.rp[k + 1];
          const int cur = first ? rs : (regcur ? rcur : cursor[e]);
          int seg = cur, nx = INT_MAX;
          if (cur < re) {
            if (B.ci[re - 1] < wend) {
              seg = re;
            } else {
              int lo = cur, hi = re - 1;  // B.ci[hi] >= wend
              while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (B.ci[mid] >= wend) hi = mid; else lo = mid + 1;
              }
              seg = lo;
              nx = B.ci[lo];
            }
          }
          s = cur;
          len = seg - cur;
          if (regcur) rcur = seg; else cursor[e] = seg;
          mynext = min(mynext, nx);
        }
        // Long segments: the whole warp walks one B row segment, coalesced.
        unsigned lm = __ballot_sync(FULL, len >= 32);
        while (lm) {
          const int L = __ffs(lm) - 1;
          lm &= lm - 1;
          const int ls = __shfl_sync(FULL, s, L), ln = __shfl_sync(FULL, len, L);
          const T la = __shfl_sync(FULL, a, L);
          for (int t = lane; t < ln; t += 32) {
            const int bi = ls + t;
            win_insert<W, NUM, T>(acc, bits, B.ci[bi] - base, NUM ? la * bv[bi] : T(0), err);
          }
        }
        // Short segments: flattened so every lane takes one product.
        const int sl = len < 32 ? len : 0;
        const int incl = warp_incl_scan(sl);
        const int tot = __shfl_sync(FULL, incl, 31);
        for (int p0 = 0; p0 < tot; p0 += 32) {
          const int p = p0 + lane;
          const int o = warp_owner(incl, p);
          const int os = __shfl_sync(FULL, s, o);
          const int oex = __shfl_sync(FULL, incl - sl, o);
          const T oa = __shfl_sync(FULL, a, o);
          if (p < tot) {
            const int bi = os + p - oex;
            win_insert<W, NUM, T>(acc, bits, B.ci[bi] - base, NUM ? oa * bv[bi] : T(0), err);
          }
        }
      }
      mynext = warp_min(mynext);
      const int hic = min(wend - 1, last);
      const int nw = hic >= base ? ((hic - base) >> 5) + 1 : 0;
      group_sync<GW>(g);
      const int wpw = (nw + GW - 1) / GW;
      const int w0 = min(nw, wig * wpw), w1 = min(nw, w0 + wpw);
      int cnt = 0;
      for (int j = w0 + lane; j < w1; j += 32) {
        cnt += __popc(bits[j]);
        if (!NUM) bits[j] = 0u;
      }
      cnt = warp_sum(cnt);
      if (lane == 0) {
        wcnt[wig] = cnt;
        wnext[wig] = mynext;
      }
      group_sync<GW>(g);
      int before = 0, total = 0, nb = INT_MAX;
      for (int w = 0; w < GW; ++w) {
        const int cw = wcnt[w];
        if (w < wig) before += cw;
        total += cw;
        nb = min(nb, wnext[w]);
      }
      if (NUM) {
        long long off = obeg + rowcount + before;
        if (cnt * 4 >= (w1 - w0) * 32) {
          // dense words: lanes take bits, so each store is contiguous
          for (int j = w0; j < w1; ++j) {
            const uint32_t wd = bits[j];
            if (wd == 0u) continue;
            if ((wd >> lane) & 1u) {
              const long long o = off + __popc(wd & lanemask_lt());
              const int jj = j * 32 + lane;
              if (o < oend) {
                c_ci[o] = base + jj;
                c_v[o] = acc[jj];
              }
              acc[jj] = T(0);
            }
            off += __popc(wd);
          }
          __syncwarp();
          for (int j = w0 + lane; j < w1; j += 32) bits[j] = 0u;
        } else {
          // sparse words: lanes take words and walk their set bits
          for (int jb = w0; jb < w1; jb += 32) {
            const int j = jb + lane;
            uint32_t wd = j < w1 ? bits[j] : 0u;
            const int c = __popc(wd);
            const int inc = warp_incl_scan(c);
            long long o = off + inc - c;
            while (wd) {
              const int b = __ffs(wd) - 1;
              wd &= wd - 1;
              const int jj = j * 32 + b;
              if (o < oend) {
                c_ci[o] = base + jj;
                c_v[o] = acc[jj];
              }
              acc[jj] = T(0);
              ++o;
            }
            if (j < w1) bits[j] = 0u;
            off += __shfl_sync(FULL, inc, 31);
          }
        }
      }
      rowcount += total;
      group_sync<GW>(g);
      first = false;
      if (nb == INT_MAX) break;
      base = nb;
    }
    if (wig == 0 && lane == 0) {
      if (!NUM) c_cnt[r] = (int)rowcount;
      else if (obeg + rowcount != oend) atomicOr(err, EB_INTERNAL);
    }
  }
}

}  // namespace sg
