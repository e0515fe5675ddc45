// Numeric pass for large rows: a dense column window shared by a block.
//
// Row i of C is the sum over A(i,k) of A(i,k) * B(k,:) (Sec. 2.2).  One block
// of NW warps owns one row at a time and a window of W consecutive columns
// (a multiple of the run width of B's window-run list, aligned to W): a
// dense value array and a presence bitmap in shared memory.  For each
// window, a nonzero's segment of B(k,:) is the union of its consecutive runs
// whose window ids fall in the block window, so it is found by reading a few
// run entries, with no search.
//
// The segments of a window are first collected into a list in shared memory
// together with their offsets in the window's product stream (the
// concatenation of all segments).  The warps then take the stream in batches
// of 32 consecutive products, whatever segments they come from: every lane of
// every batch carries one product, so the FP64 pipe -- which spends the same
// time on a warp instruction whatever the number of active lanes -- is used
// at full width, and a long segment spreads over all warps by itself.
// Products from all warps land in the shared window, so they are added with
// shared-memory atomics (the hardware resolves equal addresses).
//
// The window is emitted in column order: every warp popcounts its share of
// the bitmap, a block prefix places the shares, lanes write their bits.
// Compared with one warp per row, a block window is W/1024 times wider, so a
// wide sparse row needs that many times fewer windows.
#pragma once

#include "segstream.cuh"
#include "semiring.cuh"

namespace sg {

// Nonzeros of A whose segments are collected per round: a nonzero has at most
// one segment in a block window, so the list never holds more entries.  Small
// blocks get a short list, so that more of them fit on an SM.
template <int NW>
__host__ __device__ constexpr int nb_segcap() {
  return NW >= 16 ? 1024 : 64 * NW;
}

template <int W, int NW, typename T>
__host__ __device__ constexpr size_t numblock_smem_bytes() {
  return (size_t)W * sizeof(T)                 // window values
         + (size_t)nb_segcap<NW>() * sizeof(T)  // segment multipliers A(i,k)
         + (size_t)(W / 32) * 8                // two presence bitmaps (alternate windows)
         + (size_t)nb_segcap<NW>() * 8         // segment stream offsets and starts in B
         + (size_t)NW * 8                      // per-warp counts and next windows
         + (size_t)(W / 32) * 2;               // per-word output offsets inside a warp's share
}

// Loads of one step of U batches of 32 products from pb on: column, B value
// and multiplier of every lane's product.  f is the segment of product pb on
// entry and of product pb + 32U on return.  The batches' segment lookups do
// not depend on each other (one shared load of 32 segment ends usually
// places every batch start), so their latencies overlap.  Every lane must
// call it.
template <int U, typename T>
struct NbStep {
  int col[U];
  T b[U], a[U];
};

template <int U, typename T>
__device__ __forceinline__ void nb_load(const Csr& B, const T* __restrict__ bv, const int* off, const int* sstart,
                                        const T* sa, int nseg, int tot, int hi, int pb, int& f, NbStep<U, T>& st) {
  const int lane = lane_id();
  auto end_of = [&](int g) {  // end of segment g + lane = start of the next one
    const int nx = g + lane + 1;
    return nx < nseg ? off[nx] : (nx == nseg ? tot : INT_MAX);
  };
  const int e0 = end_of(f);
  int fu[U + 1];
  fu[0] = f;
#pragma unroll
  for (int u = 1; u <= U; ++u) {
    const int t = pb + 32 * u;
    const int c = __popc(__ballot_sync(FULL, e0 <= t));
    // more than 32 segments ahead: search (t < tot keeps the search valid)
    fu[u] = c < 32 ? f + c : (t < tot ? seg_find(off, nseg, t) : nseg);
  }
  f = fu[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int p0 = pb + 32 * u;
    st.col[u] = 0;
    st.b[u] = T(0);
    st.a[u] = T(0);
    if (p0 < hi) {  // warp-uniform
      const int end = u == 0 ? e0 : end_of(fu[u]);
      const int d = end == INT_MAX ? INT_MAX : end - p0;
      const unsigned m = __reduce_or_sync(FULL, d <= 31 ? (1u << d) : 0u);
      const int k = fu[u] + __popc(m & (lane == 31 ? FULL : ((2u << lane) - 1u)));
      const int p = p0 + lane;
      if (p < hi) {
        const int q = sstart[k] + (p - off[k]);
        st.col[u] = B.ci[q];
        st.b[u] = bv[q];
        st.a[u] = sa[k];
      }
    }
  }
}

// One product: acc[col - base] += a * b, the column marked present on its
// first update.
template <int W, typename T, int SR>
__device__ __forceinline__ void nb_add(int col, T a, T b, int base, T* acc, uint32_t* bits, uint32_t* err) {
  const int j = col - base;
  if ((unsigned)j < (unsigned)W) {
    if (SrOps<T, SR>::madd_shared(&acc[j], a, b, err)) atomicOr(&bits[j >> 5], 1u << (j & 31));
  } else {
    atomicOr(err, EB_UNSORTED);
  }
}

// The products [lo, hi) of the window's stream (tot products, nseg
// segments), software-pipelined U batches at a time: the loads of the next
// step are in flight while this step's products are accumulated (three steps
// measured 2.4 % faster than two on R-MAT 18; walking long segments directly
// instead of through the stream mapping was 4 % slower).  hi - lo is a
// multiple of 32 unless hi == tot.  Every lane must call it.
template <int W, typename T, int U = 3, int SR = SPGEMM_PLUS_TIMES>
__device__ __forceinline__ void nb_range(const Csr& B, const T* __restrict__ bv, const int* off, const int* sstart,
                                         const T* sa, int nseg, int tot, int lo, int hi, int base, T* acc,
                                         uint32_t* bits, uint32_t* err) {
  const int lane = lane_id();
  int f = seg_find(off, nseg, lo);
  NbStep<U, T> cur;
  nb_load<U, T>(B, bv, off, sstart, sa, nseg, tot, hi, lo, f, cur);
  for (int p0 = lo; p0 < hi; p0 += 32 * U) {
    NbStep<U, T> nxt;
    if (p0 + 32 * U < hi) nb_load<U, T>(B, bv, off, sstart, sa, nseg, tot, hi, p0 + 32 * U, f, nxt);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (p0 + 32 * u + lane < hi) nb_add<W, T, SR>(cur.col[u], cur.a[u], cur.b[u], base, acc, bits, err);
    cur = nxt;
  }
}

// Emission of a window in column order, balanced over the block's warps by
// output count.  Bitmap words are grouped in NW chunks of WPW words (chunk w
// was popcounted by warp w: wpre holds each word's exclusive offset inside its
// chunk, wcnt the chunk totals).  The window's outputs are cut into NW equal
// contiguous shares; lanes take consecutive outputs, so the stores of C are
// coalesced.  An output's chunk comes from a warp search over the chunk
// offsets, its word from a binary search over the chunk's offsets, its bit
// from a binary search on popcounts inside the word.  Every lane must call it.
template <int NW, int WPW, typename T, int SR>
__device__ __forceinline__ void nb_emit(const uint32_t* bits, const uint16_t* wpre, const int* wcnt, T* acc, int base,
                                        int out, int out_end, int32_t* __restrict__ rci, T* __restrict__ rcv,
                                        uint32_t* err) {
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  const int cnt = lane < NW ? wcnt[lane] : 0;
  const int cinc = warp_incl_scan(cnt);  // chunk ends (lanes >= NW repeat the total)
  const int total = __shfl_sync(FULL, cinc, 31);
  const int share = ((total + NW * 32 - 1) / (NW * 32)) * 32;
  const int lo = warp * share, hi = min(total, lo + share);
  for (int t0 = lo; t0 < hi; t0 += 32) {
    const int t = t0 + lane;
    const int c = warp_owner(cinc, t);  // chunk of output t
    const int coff = __shfl_sync(FULL, cinc - cnt, c & 31);
    if (t < hi) {
      const int rel = t - coff;
      const uint16_t* pre = wpre + c * WPW;
      int wj = 0;  // last word of the chunk whose offset is <= rel
#pragma unroll
      for (int sh = 16; sh >= 1; sh >>= 1)
        if (sh < WPW && wj + sh < WPW && pre[wj + sh] <= rel) wj += sh;
      const int word = c * WPW + wj;
      uint32_t x = bits[word];
      int rank = rel - pre[wj], bit = 0;
#pragma unroll
      for (int sh = 16; sh >= 1; sh >>= 1) {
        const int lowc = __popc(x & ((1u << sh) - 1u));
        if (rank >= lowc) {
          rank -= lowc;
          x >>= sh;
          bit += sh;
        }
      }
      const int jj = (word << 5) + bit;
      const int pos = out + t;
      const T v = acc[jj];
      acc[jj] = SrOps<T, SR>::zero();
      if (pos < out_end) {
        __stcs(rci + pos, base + jj);
        __stcs(rcv + pos, v);
      } else {
        atomicOr(err, EB_INTERNAL);
      }
    }
  }
}

// Blocks of this geometry that share an SM's 228 KB of shared memory, but no
// more than leave each thread 64 registers (at least one block): the
// register budget the compiler may use follows from it.
template <int W, int NW, typename T>
__host__ __device__ constexpr int nb_blocks_per_sm() {
  constexpr int by_smem = (int)(228 * 1024 / (numblock_smem_bytes<W, NW, T>() + 1024));
  constexpr int by_regs = 65536 / (NW * 32 * 64);
  constexpr int b = by_smem < by_regs ? by_smem : by_regs;
  return b > 0 ? b : 1;
}

// rrb/runsb: B's run list at the block window's granularity (log2 W), so the
// segment of B(k,:) in a block window is exactly one run.
template <int W, int NW, typename T, int SR = SPGEMM_PLUS_TIMES>
__global__ void __launch_bounds__(NW * 32, nb_blocks_per_sm<W, NW, T>())
k_num_block(Csr A, Csr B, const T* __restrict__ av, const T* __restrict__ bv, RowInfo ri, const DevStats* st,
            int bin_lo, int bin_hi, const int32_t* __restrict__ rrb, const int2* __restrict__ runsb,
            int32_t* __restrict__ gcur, const int32_t* __restrict__ c_rp, int32_t* __restrict__ c_ci,
            T* __restrict__ c_v, unsigned* counter, uint32_t* err) {
  static_assert(W % 1024 == 0, "window must be a multiple of 1024 columns");
  constexpr int NWORDS = W / 32;
  constexpr int WPW = NWORDS / NW;  // bitmap words emitted per warp
  static_assert(WPW >= 1 && WPW <= 32, "one bitmap word per lane at most");
  constexpr int SEGCAP = nb_segcap<NW>();
  static_assert(SEGCAP <= 1024, "the segment search covers 32 x 32 entries");
  static_assert(SEGCAP >= NW * 32, "a row with register cursors fits one round");
  constexpr int WSHIFT = (W == 2048) ? 11 : (W == 4096) ? 12 : (W == 8192) ? 13 : 14;
  static_assert((1 << WSHIFT) == W, "window must be 2048, 4096, 8192 or 16384 columns");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* acc = reinterpret_cast<T*>(smem_raw);
  T* seg_a = acc + W;
  // presence bitmaps of alternate windows: a window's bitmap is cleared
  // during the next window, so the emission needs no closing barrier
  uint32_t* bits0 = reinterpret_cast<uint32_t*>(seg_a + SEGCAP);
  uint32_t* bits1 = bits0 + NWORDS;
  int* seg_off = reinterpret_cast<int*>(bits1 + NWORDS);
  int* seg_s = seg_off + SEGCAP;
  int* wcnt = seg_s + SEGCAP;
  int* wnext = wcnt + NW;
  uint16_t* wpre = reinterpret_cast<uint16_t*>(wnext + NW);  // word offsets inside a chunk (< 1024)
  __shared__ int s_lb, s_le, s_item;
  // (segments << 32) | products collected so far in a round; two of them, so
  // one can be cleared while the other is read
  __shared__ unsigned long long s_pack[2];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  for (int t = threadIdx.x; t < W; t += NW * 32) acc[t] = SrOps<T, SR>::zero();
  for (int t = threadIdx.x; t < 2 * NWORDS; t += NW * 32) bits0[t] = 0u;
  if (threadIdx.x == 0) {
    bin_range(st, bin_lo, bin_hi, &s_lb, &s_le);
    s_pack[0] = 0ull;
    s_pack[1] = 0ull;
  }
  if (block_skip(st)) return;
  const int lb = s_lb, le = s_le;
  int parity = 0;  // which s_pack the current round uses
  int bsel = 0;    // bitmap of the current window
  // this warp's non-empty words of the previous window's bitmap, cleared
  // once every warp has finished that window's emission
  uint32_t prev_w = 0u;
  int prev_i = 0;

  while (true) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const long long idx = (long long)lb + s_item;
    __syncthreads();  // s_item is reused by the next iteration
    if (idx >= le) break;
    const int r = ri.rows[idx];
    const long long i = ri.row_begin + r;
    const int a0 = A.rp[i], a1 = A.rp[i + 1];
    const int cmx = ri.cmax[r];
    const long long rbeg = c_rp[r];
    const int out_end = (int)(c_rp[r + 1] - rbeg);
    int32_t* const rci = c_ci + rbeg;
    T* const rcv = c_v + rbeg;
    // Cursor of a nonzero: index of its current run in the block-granular run
    // list.  Up to 32 * NW nonzeros keep it in registers (thread t owns
    // nonzero a0 + t) together with the run after it, loaded one window
    // ahead; longer rows keep the index in gcur (parallel to A's nonzeros)
    // and walk in rounds of SEGCAP nonzeros.
    const bool regc = a1 - a0 <= NW * 32;  // block-uniform
    int rj = 0;
    int2 rcur = make_int2(INT_MAX, 0), rnxt = make_int2(INT_MAX, 0);
    T ra = T(0);
    int mn = INT_MAX;
    if (regc) {
      const int e = a0 + threadIdx.x;
      if (e < a1) {
        rj = rrb[A.ci[e]];
        rcur = runsb[rj];
        rnxt = runsb[rj + 1];  // past a row's sentinel: padding or the next row, never used
        ra = av[e];
        mn = rcur.x;
      }
    } else {
      for (int e = a0 + threadIdx.x; e < a1; e += NW * 32) {
        const int j = rrb[A.ci[e]];
        gcur[e] = j;
        mn = min(mn, runsb[j].x);
      }
    }
    mn = warp_min(mn);
    if (lane == 0) wnext[warp] = mn;
    __syncthreads();
    int wb = INT_MAX;  // block window index (the run list's window id)
    for (int w = 0; w < NW; ++w) wb = min(wb, wnext[w]);
    int out = 0;
    while (wb != INT_MAX) {
      const int base = wb << WSHIFT;
      uint32_t* const bits = bsel ? bits1 : bits0;
      mn = INT_MAX;
      bool first_round = true;
      for (int r0 = a0; r0 < a1; r0 += SEGCAP) {  // one round with register cursors
        const int r1 = min(a1, r0 + SEGCAP);
        unsigned long long* pk = &s_pack[parity];
        if (regc) {
          int s = 0, len = 0;
          if (rcur.x == wb) {
            s = rcur.y;
            len = rnxt.y - s;
            ++rj;
            rcur = rnxt;
            rnxt = runsb[rj + 1];  // in flight until a later window needs it
          }
          mn = min(mn, rcur.x);
          seg_append<T>(pk, s, len, ra, seg_off, seg_s, seg_a);
        } else {
          for (int e0 = r0 + warp * 32; e0 < r1; e0 += NW * 32) {
            const int e = e0 + lane;
            int s = 0, len = 0;
            T a = T(0);
            if (e < r1) {
              const int j = gcur[e];
              const int2 c0 = runsb[j], c1 = runsb[j + 1];
              if (c0.x == wb) {
                s = c0.y;
                len = c1.y - s;
                a = av[e];
                gcur[e] = j + 1;
                mn = min(mn, c1.x);
              } else {
                mn = min(mn, c0.x);
              }
            }
            seg_append<T>(pk, s, len, a, seg_off, seg_s, seg_a);
          }
        }
        __syncthreads();  // the list is complete (and the previous window emitted)
        if (first_round) {
          if (prev_w) (bsel ? bits0 : bits1)[prev_i] = 0u;
          prev_w = 0u;
          first_round = false;
        }
        const unsigned long long pv = *pk;
        const int nseg = (int)(pv >> 32), tot = (int)(unsigned)(pv & 0xffffffffull);
        if (threadIdx.x == 0) s_pack[parity ^ 1] = 0ull;  // for the next round
        {  // each warp takes a contiguous share of the stream, whole batches
          const int share = ((tot + NW * 32 - 1) / (NW * 32)) * 32;
          const int lo = warp * share, hi = min(tot, lo + share);
          if (lo < hi) nb_range<W, T, 3, SR>(B, bv, seg_off, seg_s, seg_a, nseg, tot, lo, hi, base, acc, bits, err);
        }
        __syncthreads();  // all products in; the list may be refilled
        parity ^= 1;
      }
      // emission: warp w popcounts bitmap words [w * WPW, (w + 1) * WPW), then
      // all warps emit equal shares of the window's outputs
      mn = warp_min(mn);
      const int ncols = min(W, cmx - base + 1);
      const int nwd = (ncols + 31) >> 5;
      const int w0 = warp * WPW;
      const int wi = w0 + lane;
      const uint32_t myw = (lane < WPW && wi < nwd) ? bits[wi] : 0u;
      const int c = __popc(myw);
      const int inc = warp_incl_scan(c);
      if (lane < WPW) wpre[wi] = (uint16_t)(inc - c);
      if (lane == 31) {
        wcnt[warp] = inc;
        wnext[warp] = mn;
      }
      __syncthreads();
      int total = 0, nb = INT_MAX;
      for (int w = 0; w < NW; ++w) {
        total += wcnt[w];
        nb = min(nb, wnext[w]);
      }
      nb_emit<NW, WPW, T, SR>(bits, wpre, wcnt, acc, base, out, out_end, rci, rcv, err);
      out += total;
      // no barrier: the next window's list barrier orders this emission
      // before its products (which use the other bitmap, and find the
      // emitted accumulator entries zeroed) and before this bitmap's clear
      prev_w = myw;
      prev_i = wi;
      bsel ^= 1;
      wb = nb;
    }
    if (threadIdx.x == 0 && out != out_end) atomicOr(err, EB_INTERNAL);
  }
}

}  // namespace sg
