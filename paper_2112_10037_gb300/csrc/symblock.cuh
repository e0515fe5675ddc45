// Symbolic pass for large rows: a presence bitmap of W columns shared by a
// block of NW warps, one row at a time (rows handed out by a work counter).
//
// The size of row i of C is the number of distinct columns among the B rows
// that A's row i touches (Sec. 2.2).  For each window, the segments of those
// B rows inside the window are listed in shared memory with their offsets in
// the window's product stream; the warps then take equal contiguous shares
// of the stream in whole 32-lane batches, so a hub row of B is spread over
// the block instead of keeping one warp busy.  Every product sets its
// column's bit (shared-memory atomicOr after a plain test); the window's
// count is the popcount of the bitmap, taken by all threads over equal word
// ranges, which also clears it.  A segment's end inside a window comes from a
// binary search on B's sorted columns (a single search when a window spans
// the row).  For split rows the popcounts are also added up per fine tile
// into hcnt, which fixes where each tile's entries go.
#pragma once

#include "rowpass.cuh"
#include "segstream.cuh"

namespace sg {

template <int NW>
__host__ __device__ constexpr int sb_segcap() {
  return 1024;
}

template <int W, int NW>
__host__ __device__ constexpr size_t symblock_smem_bytes() {
  return (size_t)(W / 32) * 4                           // bitmap
         + (size_t)sb_segcap<NW>() * 8                  // segment stream offsets and starts in B
         + (size_t)NW * 8                               // per-warp counts and next columns
         + (size_t)(W / SYM_MIN_FINE + 2) * 4;          // per fine tile counts (split rows)
}

// Marks the columns of products [lo, hi) of the window's stream (tot
// products, nseg segments).  While at least 32 products of the current
// segment are left, lanes walk the segment directly (four loads in flight
// per lane); batches that straddle segments find each lane's segment from
// the segment ends.  Every lane must call it.
__device__ __forceinline__ void sb_range(const Csr& B, const int* off, const int* sstart, int nseg, int tot, int lo,
                                         int hi, int base, int W, uint32_t* bits, uint32_t* err) {
  const int lane = lane_id();
  int f = seg_find(off, nseg, lo);
  int p = lo;
  while (p < hi) {
    const int sb = off[f];
    const int se = f + 1 < nseg ? off[f + 1] : tot;
    const int run = min(se, hi) - p;
    if (run >= 32) {  // whole batches inside segment f
      const int n = run & ~31;
      const int* ci = B.ci + sstart[f] + (p - sb);
      int t = lane;
      for (; t + 96 < n; t += 128) {
        const int c0 = ci[t], c1 = ci[t + 32], c2 = ci[t + 64], c3 = ci[t + 96];
        bit_insert(bits, c0 - base, W, err);
        bit_insert(bits, c1 - base, W, err);
        bit_insert(bits, c2 - base, W, err);
        bit_insert(bits, c3 - base, W, err);
      }
      for (; t < n; t += 32) bit_insert(bits, ci[t] - base, W, err);
      p += n;
      if (p == se) ++f;
      continue;
    }
    // one batch across segments: lane j holds the end of segment f + j
    const int nx = f + lane + 1;
    const int end = nx < nseg ? off[nx] : (nx == nseg ? tot : INT_MAX);
    const int d = end == INT_MAX ? INT_MAX : end - p;
    const unsigned m = __reduce_or_sync(FULL, d <= 31 ? (1u << d) : 0u);
    const int k = f + __popc(m & (lane == 31 ? FULL : ((2u << lane) - 1u)));
    const int q = p + lane;
    if (q < hi) bit_insert(bits, B.ci[sstart[k] + (q - off[k])] - base, W, err);
    const int pn = p + 32;
    if (pn < hi) {  // segment of the next product
      const int c = __popc(__ballot_sync(FULL, end <= pn));
      f = c < 32 ? f + c : seg_find(off, nseg, pn);
    }
    p = pn;
  }
}

// cursor: per nonzero of A, the first entry of its B row not yet counted.
template <int W, int NW>
__global__ void __launch_bounds__(NW * 32)
k_sym_block(Csr A, Csr B, RowInfo ri, const DevStats* st, int bin_lo, int bin_hi, SplitInfo sp,
            int32_t* __restrict__ cursor, int32_t* __restrict__ c_cnt, unsigned* counter, uint32_t* err) {
  static_assert(W % 32 == 0 && W >= SYM_MIN_FINE, "bad window");
  constexpr int NWORDS = W / 32;
  constexpr int SEGCAP = sb_segcap<NW>();
  constexpr int NTW = W / SYM_MIN_FINE + 2;  // fine tiles a window can touch
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t* bits = reinterpret_cast<uint32_t*>(smem_raw);
  int* seg_off = reinterpret_cast<int*>(bits + NWORDS);
  int* seg_s = seg_off + SEGCAP;
  int* wcnt = seg_s + SEGCAP;
  int* wnext = wcnt + NW;
  int* tcnt = wnext + NW;
  __shared__ int s_lb, s_le, s_nh, s_hs, s_item;
  __shared__ unsigned long long s_pack[2];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  for (int t = threadIdx.x; t < NWORDS; t += NW * 32) bits[t] = 0u;
  for (int t = threadIdx.x; t < NTW; t += NW * 32) tcnt[t] = 0;
  if (threadIdx.x == 0) {
    bin_range(st, bin_lo, bin_hi, &s_lb, &s_le);
    s_nh = split_rows(st, sp, &s_hs);
    s_pack[0] = 0ull;
    s_pack[1] = 0ull;
  }
  if (block_skip(st)) return;
  const int lb = s_lb, le = s_le, nh = s_nh, hs = s_hs;
  const int wf_shift = sp.wf_shift;
  int parity = 0;

  while (true) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const long long idx = (long long)lb + s_item;
    __syncthreads();  // s_item is reused by the next iteration
    if (idx >= le) break;
    const int r = ri.rows[idx];
    const bool split = idx >= hs && idx < hs + nh;
    const long long hrow = idx - hs;  // row of the per-window count table
    const long long i = ri.row_begin + r;
    const int a0 = A.rp[i], a1 = A.rp[i + 1];
    int base = ri.cmin[r] & ~31;
    const int last = ri.cmax[r];
    long long rowcount = 0;
    bool first = true;
    if (split) {
      for (int t = threadIdx.x; t < sp.ntf; t += NW * 32) sp.hcnt[(size_t)hrow * sp.ntf + t] = 0;
      __syncthreads();
    }
    while (true) {
      const int wend = (int)min((long long)base + W, (long long)INT_MAX);
      int mynext = INT_MAX;
      for (int r0 = a0; r0 < a1; r0 += SEGCAP) {
        const int r1 = min(a1, r0 + SEGCAP);
        unsigned long long* pk = &s_pack[parity];
        for (int e0 = r0 + warp * 32; e0 < r1; e0 += NW * 32) {
          const int e = e0 + lane;
          int s = 0, len = 0;
          if (e < r1) {
            const int k = A.ci[e];
            const int rs = B.rp[k], re = B.rp[k + 1];
            const int cur = first ? rs : cursor[e];
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
            cursor[e] = seg;
            mynext = min(mynext, nx);
          }
          seg_append(pk, s, len, seg_off, seg_s);
        }
        __syncthreads();  // the list is complete
        const unsigned long long pv = *pk;
        const int nseg = (int)(pv >> 32), tot = (int)(unsigned)(pv & 0xffffffffull);
        if (threadIdx.x == 0) s_pack[parity ^ 1] = 0ull;  // for the next round
        {
          const int share = ((tot + NW * 32 - 1) / (NW * 32)) * 32;
          const int lo = warp * share, hi = min(tot, lo + share);
          if (lo < hi) sb_range(B, seg_off, seg_s, nseg, tot, lo, hi, base, W, bits, err);
        }
        __syncthreads();  // all bits set; the list may be refilled
        parity ^= 1;
      }
      // count (and clear) the window's words, equal ranges per thread
      const int hic = min(wend - 1, last);
      const int nw = hic >= base ? ((hic - base) >> 5) + 1 : 0;
      const int tile0 = base >> wf_shift;
      int cnt = 0;
      for (int j = threadIdx.x; j < nw; j += NW * 32) {
        const int pc = __popc(bits[j]);
        bits[j] = 0u;
        cnt += pc;
        if (split && pc) atomicAdd(&tcnt[((base + 32 * j) >> wf_shift) - tile0], pc);
      }
      cnt = warp_sum(cnt);
      mynext = warp_min(mynext);
      if (lane == 0) {
        wcnt[warp] = cnt;
        wnext[warp] = mynext;
      }
      __syncthreads();
      int total = 0, nb = INT_MAX;
      for (int w = 0; w < NW; ++w) {
        total += wcnt[w];
        nb = min(nb, wnext[w]);
      }
      if (split) {
        const int ntw = min(NTW, sp.ntf - tile0);
        for (int t = threadIdx.x; t < ntw; t += NW * 32) {
          const int v = tcnt[t];
          if (v) {
            atomicAdd(&sp.hcnt[(size_t)hrow * sp.ntf + tile0 + t], v);
            tcnt[t] = 0;
          }
        }
      }
      rowcount += total;
      __syncthreads();  // counts read and tile counts flushed before the next window
      first = false;
      if (nb == INT_MAX) break;
      base = nb & ~31;
    }
    if (threadIdx.x == 0) c_cnt[r] = (int)rowcount;
  }
}

}  // namespace sg
