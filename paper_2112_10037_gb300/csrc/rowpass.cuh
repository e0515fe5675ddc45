// Row kernels shared by the symbolic pass (sizes of C's rows) and the
// numeric pass (C's columns and values).  Both follow the row-wise Gustavson
// method (Sec. 2.2): row i of C accumulates A(i,k) * B(k,:) over the nonzeros
// of A's row i, and equal columns are merged by adding their values
// (Sec. 2.2, Algorithm 1), leaving the row's columns ascending and unique.
//
// Two accumulators are used, chosen per row by its product count P:
//
//  * register sort (P <= 128): a group of G lanes holds up to E products per
//    lane, sorts the (column, value) pairs with a bitonic network over
//    shuffles and registers, and adds runs of equal columns with a segmented
//    suffix sum.  The sorted order is the output order, so nothing is
//    written to shared memory.
//
//  * bitmap window (symbolic pass, larger rows): a warp or a block owns a
//    presence bitmap of W consecutive columns in shared memory.  Every B
//    row touched by the row is read from a per-nonzero cursor up to the
//    window's end (rows of B are sorted, so that is one contiguous segment)
//    and sets one bit per product; the row size is the popcount.  The next
//    window starts at the smallest column still unread, so windows skip
//    column ranges the row does not touch.  The numeric counterpart (a dense
//    value window per warp) is in numwarp.cuh.
#pragma once

#include "internal.cuh"
#include "semiring.cuh"

namespace sg {

// ---------------------------------------------------------------- tiny path
// One row per group of G lanes holding E products per lane (G*E >= P).
// Element x of the row's product sequence lives in slot x / G of lane x % G,
// so every slot is a run of G consecutive elements after the sort; the
// bitonic network exchanges through shuffles (partner distance < G) or
// between a lane's own slots (distance >= G).
template <int G, int E, bool NUM, typename T, int SR = SPGEMM_PLUS_TIMES>
__global__ void __launch_bounds__(256)
k_tiny(Csr A, Csr B, const T* __restrict__ av, const T* __restrict__ bv, RowInfo ri,
       const DevStats* st, int bin_lo, int bin_hi, int32_t* __restrict__ c_cnt,
       const int32_t* __restrict__ c_rp, int32_t* __restrict__ c_ci, T* __restrict__ c_v,
       uint32_t* err) {
  static_assert(E == 1 || G == 32, "multi-slot rows use whole warps");
  constexpr int N = G * E;
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
    // Gather: slot s of lane gl takes the row's (s*G + gl)-th product.
    int col[E];
    T val[E];
#pragma unroll
    for (int s = 0; s < E; ++s) { col[s] = INT_MAX; val[s] = T(0); }
    int done = 0;
    for (int e0 = a0; __any_sync(FULL, e0 < a1); e0 += G) {
      const int e = e0 + gl;
      int sb = 0, len = 0;
      T a = T(0);
      if (e < a1) {
        const int k = A.ci[e];
        sb = B.rp[k];
        len = B.rp[k + 1] - sb;
        if (NUM) a = av[e];
      }
      int incl = len;
#pragma unroll
      for (int d = 1; d < G; d <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, d, G);
        if (gl >= d) incl += t;
      }
      const int tot = __shfl_sync(FULL, incl, G - 1, G);
      const int excl = incl - len;
#pragma unroll
      for (int s = 0; s < E; ++s) {
        const int q = s * G + gl - done;
        int o = 0;
#pragma unroll
        for (int sp = G / 2; sp >= 1; sp >>= 1) {
          const int t = __shfl_sync(FULL, incl, o + sp - 1, G);
          if (t <= q) o += sp;
        }
        const int os = __shfl_sync(FULL, sb, o, G);
        const int oex = __shfl_sync(FULL, excl, o, G);
        const T oa = __shfl_sync(FULL, a, o, G);
        if (q >= 0 && q < tot) {
          const int bi = os + q - oex;
          col[s] = B.ci[bi];
          if (NUM) val[s] = SrOps<T, SR>::mul(oa, bv[bi]);
        }
      }
      done += tot;
    }
    if (!NUM && E == 1) {
      // Distinct columns: one leader per run of equal keys inside the group.
      const unsigned long long key = ((unsigned long long)(unsigned)gi << 32) | (unsigned)col[0];
      const unsigned m = __match_any_sync(FULL, key);
      const bool leader = col[0] != INT_MAX && (__ffs(m) - 1) == lane;
      const int cnt = __popc(__ballot_sync(FULL, leader) & gmask);
      if (vrow && gl == 0) c_cnt[r] = cnt;
      continue;
    }
    // Bitonic sort of the N = G*E elements by column.
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        if (j >= G) {
#pragma unroll
          for (int s = 0; s < E; ++s) {
            const int s2 = s ^ (j / G);
            if (s < s2) {
              const bool up = ((s * G + gl) & k) == 0;
              if (up ? (col[s] > col[s2]) : (col[s] < col[s2])) {
                const int tc = col[s]; col[s] = col[s2]; col[s2] = tc;
                if (NUM) { const T tv = val[s]; val[s] = val[s2]; val[s2] = tv; }
              }
            }
          }
        } else {
#pragma unroll
          for (int s = 0; s < E; ++s) {
            const int pc = __shfl_xor_sync(FULL, col[s], j);
            T pv = T(0);
            if (NUM) pv = __shfl_xor_sync(FULL, val[s], j);
            const bool up = ((s * G + gl) & k) == 0;
            const bool lower = (gl & j) == 0;
            const bool take = (lower == up) ? (pc < col[s]) : (pc > col[s]);
            if (take) {
              col[s] = pc;
              if (NUM) val[s] = pv;
            }
          }
        }
      }
    }
    // Heads of runs of equal columns, in element order.
    bool head[E];
    int nheads = 0;
    unsigned hb[E];
#pragma unroll
    for (int s = 0; s < E; ++s) {
      // every lane executes both shuffles (s is a compile-time constant)
      const int up1 = __shfl_up_sync(FULL, col[s], 1, G);
      const int prevlast = (s > 0) ? __shfl_sync(FULL, col[s > 0 ? s - 1 : 0], G - 1, G) : -1;
      const int prev = (gl == 0) ? prevlast : up1;
      head[s] = col[s] != INT_MAX && prev != col[s];
      hb[s] = __ballot_sync(FULL, head[s]) & gmask;
      nheads += __popc(hb[s]);
    }
    if (!NUM) {
      if (vrow && gl == 0) c_cnt[r] = nheads;
      continue;
    }
    // Segmented suffix sums, last slot first, carrying runs across slots.
    T acc[E];
#pragma unroll
    for (int s = E - 1; s >= 0; --s) {
      T a = val[s];
#pragma unroll
      for (int d = 1; d < G; d <<= 1) {
        const T t = __shfl_down_sync(FULL, a, d, G);
        const int tc = __shfl_down_sync(FULL, col[s], d, G);
        if (gl + d < G && tc == col[s]) a = SrOps<T, SR>::add(a, t);
      }
      if (s < E - 1) {
        const int lastc = __shfl_sync(FULL, col[s], G - 1, G);
        const int nextc = __shfl_sync(FULL, col[s < E - 1 ? s + 1 : s], 0, G);
        const T nexta = __shfl_sync(FULL, acc[s < E - 1 ? s + 1 : s], 0, G);
        if (nextc == lastc && col[s] == lastc) a = SrOps<T, SR>::add(a, nexta);
      }
      acc[s] = a;
    }
    if (vrow) {
      const long long ob = c_rp[r], oe = c_rp[r + 1];
      long long before = 0;
#pragma unroll
      for (int s = 0; s < E; ++s) {
        if (head[s]) {
          const long long o = ob + before + __popc(hb[s] & lanemask_lt());
          if (o < oe) {
            c_ci[o] = col[s];
            c_v[o] = acc[s];
          }
        }
        before += __popc(hb[s]);
      }
      if (gl == 0 && ob + nheads != oe) atomicOr(err, EB_INTERNAL);
    }
  }
}

// ------------------------------------------------------- bitmap-window path
// Symbolic pass for rows above the register-sort limit: a group of GW warps
// owns a presence bitmap of W columns; each product sets its column's bit
// (shared-memory atomicOr after a plain test), and the row size is the
// popcount of the window.  Windows start at a multiple of 32 at or below the
// smallest unread column.  For split rows the popcounts are also added up
// per fine tile into hcnt, which fixes where each tile's entries go.
template <int GW>
__device__ __forceinline__ void group_sync(int g) {
  if (GW == 1) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(GW * 32) : "memory");
  }
}

__device__ __forceinline__ void bit_insert(uint32_t* bits, int j, int W, uint32_t* err) {
  if ((unsigned)j >= (unsigned)W) {  // only reachable with unsorted input
    atomicOr(err, EB_UNSORTED);
    return;
  }
  const uint32_t m = 1u << (j & 31);
  if (!(bits[j >> 5] & m)) atomicOr(&bits[j >> 5], m);
}

// Smallest fine-tile width the symbolic kernel sizes its tile counters for.
constexpr int SYM_MIN_FINE = 1024;

template <int W, int GW, int WF = SYM_MIN_FINE>
__host__ __device__ constexpr size_t sym_group_bytes() {
  return (((size_t)(W / 32) * 4 + (size_t)GW * 8 + (size_t)(W / WF + 2) * 4) + 15) & ~(size_t)15;
}

// GW warps per row (group), CW warps per block, W columns per window; the
// fine tile width is 2^sp.wf_shift >= SYM_MIN_FINE columns.
template <int GW, int CW, int W>
__global__ void __launch_bounds__(CW * 32)
k_sym_window(Csr A, Csr B, RowInfo ri, const DevStats* st, int bin_lo, int bin_hi, SplitInfo sp,
             int32_t* __restrict__ cursor, int32_t* __restrict__ c_cnt, uint32_t* err) {
  static_assert(CW % GW == 0 && W % 32 == 0, "bad shape");
  constexpr int NWORDS = W / 32;
  constexpr int NG = CW / GW;
  constexpr int NTW = W / SYM_MIN_FINE + 2;  // fine tiles a window can touch
  constexpr size_t GB = sym_group_bytes<W, GW>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_lb, s_le, s_nh, s_hs;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const int g = warp / GW, wig = warp % GW;
  unsigned char* gbase = smem_raw + (size_t)g * GB;
  uint32_t* bits = reinterpret_cast<uint32_t*>(gbase);
  int* wcnt = reinterpret_cast<int*>(bits + NWORDS);
  int* wnext = wcnt + GW;
  int* tcnt = wnext + GW;
  for (int t = wig * 32 + lane; t < NWORDS; t += GW * 32) bits[t] = 0u;
  for (int t = wig * 32 + lane; t < NTW; t += GW * 32) tcnt[t] = 0;
  if (threadIdx.x == 0) {
    bin_range(st, bin_lo, bin_hi, &s_lb, &s_le);
    s_nh = split_rows(st, sp, &s_hs);
  }
  if (block_skip(st)) return;
  const int lb = s_lb, le = s_le, nh = s_nh, hs = s_hs;
  const int wf_shift = sp.wf_shift;

  for (long long idx = lb + (long long)blockIdx.x * NG + g; idx < le; idx += (long long)gridDim.x * NG) {
    const int r = ri.rows[idx];
    const bool split = idx >= hs && idx < hs + nh;
    const long long hrow = idx - hs;  // row of the per-window count table
    const long long i = ri.row_begin + r;
    const int a0 = A.rp[i], a1 = A.rp[i + 1], nA = a1 - a0;
    int base = ri.cmin[r] & ~31;
    const int last = ri.cmax[r];
    const int CS = min(32, max(1, (nA + GW - 1) / GW));  // nonzeros per chunk
    const int nch = (nA + CS - 1) / CS;
    const bool regcur = nch <= GW;  // one chunk per warp: cursor stays in a register
    int rcur = 0;
    long long rowcount = 0;
    bool first = true;
    if (split) {
      for (int t = wig * 32 + lane; t < sp.ntf; t += GW * 32) sp.hcnt[(size_t)hrow * sp.ntf + t] = 0;
      group_sync<GW>(g);
    }
    while (true) {
      const int wend = (int)min((long long)base + W, (long long)INT_MAX);
      int mynext = INT_MAX;
      for (int c = wig; c < nch; c += GW) {
        const int e = a0 + c * CS + lane;
        const bool ve = lane < CS && e < a1;
        int s = 0, len = 0;
        if (ve) {
          const int k = A.ci[e];
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
          int t = lane;
          for (; t + 96 < ln; t += 128) {
            const int c0 = B.ci[ls + t], c1 = B.ci[ls + t + 32], c2 = B.ci[ls + t + 64], c3 = B.ci[ls + t + 96];
            bit_insert(bits, c0 - base, W, err);
            bit_insert(bits, c1 - base, W, err);
            bit_insert(bits, c2 - base, W, err);
            bit_insert(bits, c3 - base, W, err);
          }
          for (; t < ln; t += 32) bit_insert(bits, B.ci[ls + t] - base, W, err);
        }
        // Short segments: flattened so every lane takes one product.
        const int sl = len < 32 ? len : 0;
        const int incl = warp_incl_scan(sl);
        const int tot = __shfl_sync(FULL, incl, 31);
        const int excl = incl - sl;
        for (int p0 = 0; p0 < tot; p0 += 64) {
          const int p = p0 + lane, p2 = p + 32;
          const int o = warp_owner(incl, p), o2 = warp_owner(incl, p2);
          const int os = __shfl_sync(FULL, s, o), oex = __shfl_sync(FULL, excl, o);
          const int os2 = __shfl_sync(FULL, s, o2), oex2 = __shfl_sync(FULL, excl, o2);
          const int c0 = p < tot ? B.ci[os + p - oex] : 0;
          const int c1 = p2 < tot ? B.ci[os2 + p2 - oex2] : 0;
          if (p < tot) bit_insert(bits, c0 - base, W, err);
          if (p2 < tot) bit_insert(bits, c1 - base, W, err);
        }
      }
      mynext = warp_min(mynext);
      const int hic = min(wend - 1, last);
      const int nw = hic >= base ? ((hic - base) >> 5) + 1 : 0;
      group_sync<GW>(g);
      const int wpw = (nw + GW - 1) / GW;
      const int w0 = min(nw, wig * wpw), w1 = min(nw, w0 + wpw);
      const int tile0 = base >> wf_shift;
      int cnt = 0;
      for (int j = w0 + lane; j < w1; j += 32) {
        const int pc = __popc(bits[j]);
        bits[j] = 0u;
        cnt += pc;
        if (split && pc) atomicAdd(&tcnt[((base + 32 * j) >> wf_shift) - tile0], pc);
      }
      cnt = warp_sum(cnt);
      if (lane == 0) {
        wcnt[wig] = cnt;
        wnext[wig] = mynext;
      }
      group_sync<GW>(g);
      int total = 0, nb = INT_MAX;
      for (int w = 0; w < GW; ++w) {
        total += wcnt[w];
        nb = min(nb, wnext[w]);
      }
      if (split) {
        const int ntw = min(NTW, sp.ntf - tile0);
        for (int t = wig * 32 + lane; t < ntw; t += GW * 32) {
          const int v = tcnt[t];
          if (v) {
            atomicAdd(&sp.hcnt[(size_t)hrow * sp.ntf + tile0 + t], v);
            tcnt[t] = 0;
          }
        }
      }
      rowcount += total;
      group_sync<GW>(g);
      first = false;
      if (nb == INT_MAX) break;
      base = nb & ~31;
    }
    if (wig == 0 && lane == 0) c_cnt[r] = (int)rowcount;
  }
}

}  // namespace sg
