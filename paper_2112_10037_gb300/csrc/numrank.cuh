// Numeric pass for mid-size rows: a rank-compacted accumulator shared by a
// block.
//
// Row i of C is the sum over A(i,k) of A(i,k) * B(k,:) (Sec. 2.2), written
// with its columns ascending.  Rows of a few thousand to tens of thousands
// of products in a power-law product reach most of B's columns with little
// overlap between their B rows (one to two products per output column), so
// a dense value window is mostly empty: a warp window of 1024 columns holds
// a few dozen products, and a row sweeps hundreds of such windows, each
// paying its set-up and its bitmap emission.
//
// Here one block owns one row and a window of up to 2^18 columns (usually the
// row's whole column span), in two passes over the row's products:
//  1. mark: every product sets its column's bit in a presence bitmap of the
//     window (one shared-memory OR, no values);
//  2. a block prefix over the bitmap words gives every present column its
//     rank, i.e. its position in the output row; the columns are emitted in
//     order from the bitmap;
//  3. accumulate: each product adds A(i,k) * B(k,j) into a compact value
//     array at its column's rank (rank = prefix of its word + popcount of the
//     lower bits), as one fused multiply-add under a shared-memory
//     compare-and-swap; the array is then stored to C in order, coalesced.
// Value storage is proportional to the outputs, not to the window width.  A
// window with more than CAP outputs accumulates in chunks of CAP ranks, one
// pass over the products per chunk (products outside the chunk are skipped
// after their rank is known).
//
// The row's products are handed out as in the block window kernel: the
// nonzeros' B segments are listed in shared memory with their offsets in the
// window's product stream, and the warps take equal shares of the stream in
// full 32-lane batches, whatever the segment lengths.  When the row's column
// span fits one window, a nonzero's segment is its whole B row; otherwise the
// window's part of it is found by binary search.
#pragma once

#include "numblock.cuh"
#include "numwarp.cuh"  // lower_bound_col

namespace sg {

constexpr int RANK_SPAN_SHIFT = 18;
constexpr int RANK_SPAN = 1 << RANK_SPAN_SHIFT;     // columns per window
constexpr int RANK_WORDS = RANK_SPAN / 32;           // bitmap words per window
constexpr int RANK_GROUP_SHIFT = 11;                 // word offsets are kept per group of 2048 words,
constexpr int RANK_GROUPS = RANK_WORDS >> RANK_GROUP_SHIFT;  // so they fit 16 bits

template <int NW, int CAP, typename T>
__host__ __device__ constexpr size_t numrank_smem_bytes() {
  return (size_t)CAP * sizeof(T)                     // compact values of one rank chunk (none
                                                     // when CAP == 0: values accumulate in C)
         + (size_t)nb_segcap<NW>() * sizeof(T)       // segment multipliers A(i,k)
         + (size_t)RANK_WORDS * 4                    // presence bitmap
         + (size_t)nb_segcap<NW>() * 8               // segment stream offsets and starts in B
         + (size_t)RANK_WORDS * 2;                   // word offsets inside their group
}

// Loads of U batches of 32 products of the stream from pb on (see nb_load):
// columns always, B values and multipliers when VALS.
template <int U, bool VALS, typename T>
__device__ __forceinline__ void rk_load(const Csr& B, const T* __restrict__ bv, const int* off, const int* sstart,
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
    fu[u] = c < 32 ? f + c : (t < tot ? seg_find(off, nseg, t) : nseg);
  }
  f = fu[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int p0 = pb + 32 * u;
    st.col[u] = -1;
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
        if (VALS) {
          st.b[u] = bv[q];
          st.a[u] = sa[k];
        }
      }
    }
  }
}

// Rank of window column j (present in the bitmap): offset of its word's group
// (the four group offsets held in registers), of its word inside the group,
// and the set bits below it in the word.
static_assert(RANK_GROUPS == 4, "group offsets travel as an int4");
__device__ __forceinline__ int rk_rank(const uint32_t* bits, const uint16_t* wpre, int4 gp, int j) {
  const int w = j >> 5;
  const int g = w >> RANK_GROUP_SHIFT;
  const int base = g < 2 ? (g == 0 ? gp.x : gp.y) : (g == 2 ? gp.z : gp.w);
  return base + (int)wpre[w] + __popc(bits[w] & ((1u << (j & 31)) - 1u));
}

// acc += v on a global-memory word, result unused: the addition happens in
// the L2 cache's atomic units, not in the SM's FP64 pipe.
__device__ __forceinline__ void red_add_global(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void red_add_global(float* p, float v) { atomicAdd(p, v); }

// Stream products [lo, hi) of the list (tot products, nseg segments), software
// pipelined as in nb_range.  MARK: set the columns' bits.  Otherwise: add the
// products whose rank lies in [t0, t0 + chunk) into vals (a shared-memory
// array of chunk values), or with GLOBAL every product into vals[rank] (the
// row's values in C, global memory).  Every lane must call it.
template <bool MARK, typename T, bool GLOBAL = false>
__device__ __forceinline__ void rk_range(const Csr& B, const T* __restrict__ bv, const int* off, const int* sstart,
                                         const T* sa, int nseg, int tot, int lo, int hi, int wbase, int wlen,
                                         uint32_t* bits, const uint16_t* wpre, int4 gp, T* vals, int t0,
                                         int chunk, uint32_t* err) {
  constexpr int U = 2;
  const int lane = lane_id();
  int f = seg_find(off, nseg, lo);
  NbStep<U, T> cur;
  rk_load<U, !MARK, T>(B, bv, off, sstart, sa, nseg, tot, hi, lo, f, cur);
  for (int p0 = lo; p0 < hi; p0 += 32 * U) {
    NbStep<U, T> nxt;
    if (p0 + 32 * U < hi) rk_load<U, !MARK, T>(B, bv, off, sstart, sa, nseg, tot, hi, p0 + 32 * U, f, nxt);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (p0 + 32 * u + lane < hi) {
        const int j = cur.col[u] - wbase;
        if ((unsigned)j < (unsigned)wlen) {
          if (MARK) {
            atomicOr(&bits[j >> 5], 1u << (j & 31));
          } else if (GLOBAL) {
            red_add_global(&vals[rk_rank(bits, wpre, gp, j)], cur.a[u] * cur.b[u]);
          } else {
            const int rel = rk_rank(bits, wpre, gp, j) - t0;
            if ((unsigned)rel < (unsigned)chunk) fma_shared(&vals[rel], cur.a[u], cur.b[u], err);
          }
        } else {
          atomicOr(err, EB_UNSORTED);
        }
      }
    }
    cur = nxt;
  }
}

// Segment list of nonzeros [r0, r1) of a row for window [wbase, wend) (whole:
// every nonzero's whole B row), built by the whole block; returns the list's
// (segments << 32 | products).  Contains two block barriers.
template <int NW, typename T>
__device__ __forceinline__ unsigned long long rk_list(const Csr& A, const Csr& B, const T* __restrict__ av, int r0,
                                                      int r1, bool whole, int wbase, int wend,
                                                      unsigned long long* pack, int* seg_off, int* seg_s, T* seg_a) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
  if (tid == 0) *pack = 0ull;
  __syncthreads();
  for (int e0 = r0 + warp * 32; e0 < r1; e0 += NW * 32) {
    const int e = e0 + lane;
    int s = 0, len = 0;
    T a = T(0);
    if (e < r1) {
      const int k = A.ci[e];
      const int b0 = B.rp[k], b1 = B.rp[k + 1];
      if (whole) {
        s = b0;
        len = b1 - b0;
      } else {
        s = lower_bound_col(B.ci, b0, b1, wbase);
        len = lower_bound_col(B.ci, s, b1, wend) - s;  // wend <= ncols(B) < 2^31
      }
      a = av[e];
    }
    seg_append<T>(pack, s, len, a, seg_off, seg_s, seg_a);
  }
  __syncthreads();
  return *pack;
}

template <int NW, int CAP, typename T>
__global__ void __launch_bounds__(NW * 32, CAP == 0 ? 3 : 2)
k_num_rank(Csr A, Csr B, const T* __restrict__ av, const T* __restrict__ bv, RowInfo ri, const DevStats* st,
           int bin_lo, int bin_hi, const int32_t* __restrict__ c_rp, int32_t* __restrict__ c_ci,
           T* __restrict__ c_v, unsigned* counter, uint32_t* err) {
  constexpr int NT = NW * 32;
  constexpr int SEGCAP = nb_segcap<NW>();
  static_assert(SEGCAP <= 1024, "the segment search covers 32 x 32 entries");
  constexpr int WPT = RANK_WORDS / NT;  // bitmap words per thread in the prefix
  static_assert(WPT >= 1 && RANK_WORDS % NT == 0 && (1 << RANK_GROUP_SHIFT) % WPT == 0,
                "a thread's words lie inside one group");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* vals = reinterpret_cast<T*>(smem_raw);
  T* seg_a = vals + CAP;
  uint32_t* bits = reinterpret_cast<uint32_t*>(seg_a + SEGCAP);
  int* seg_off = reinterpret_cast<int*>(bits + RANK_WORDS);
  int* seg_s = seg_off + SEGCAP;
  uint16_t* wpre = reinterpret_cast<uint16_t*>(seg_s + SEGCAP);
  __shared__ int s_lb, s_le, s_item;
  __shared__ int s_gpre[RANK_GROUPS];
  __shared__ int s_wsum[NW];
  __shared__ unsigned long long s_pack;
  const int tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
  if (tid == 0) bin_range(st, bin_lo, bin_hi, &s_lb, &s_le);
  if (block_skip(st)) return;
  const int lb = s_lb, le = s_le;

  while (true) {
    if (tid == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const long long idx = (long long)lb + s_item;
    __syncthreads();  // s_item is reused by the next iteration
    if (idx >= le) break;
    const int r = ri.rows[idx];
    const long long i = ri.row_begin + r;
    const int a0 = A.rp[i], a1 = A.rp[i + 1];
    const int cmn = ri.cmin[r], cmx = ri.cmax[r];
    const long long rbeg = c_rp[r];
    const int out_end = (int)(c_rp[r + 1] - rbeg);
    int32_t* const rci = c_ci + rbeg;
    T* const rcv = c_v + rbeg;
    const bool one_round = a1 - a0 <= SEGCAP;
    int out = 0;
    for (long long wbase = cmn; wbase <= cmx; wbase += RANK_SPAN) {  // block-uniform
      const long long wend = wbase + RANK_SPAN < (long long)cmx + 1 ? wbase + RANK_SPAN : (long long)cmx + 1;
      const bool whole = wbase == cmn && wend == (long long)cmx + 1;
      const int wlen = (int)(wend - wbase);
      const int nwords = (wlen + 31) >> 5;
      for (int t = tid; t < nwords; t += NT) bits[t] = 0u;
      // 1. mark
      unsigned long long pk = 0ull;
      for (int r0 = a0; r0 < a1; r0 += SEGCAP) {
        pk = rk_list<NW, T>(A, B, av, r0, min(a1, r0 + SEGCAP), whole, (int)wbase, (int)wend, &s_pack, seg_off, seg_s,
                            seg_a);  // its first barrier orders the clear
        const int nseg = (int)(pk >> 32), tot = (int)(unsigned)(pk & 0xffffffffull);
        const int share = ((tot + NT - 1) / NT) * 32;  // whole 32-product batches per warp
        const int lo = warp * share, hi = min(tot, lo + share);
        if (lo < hi)
          rk_range<true, T>(B, bv, seg_off, seg_s, seg_a, nseg, tot, lo, hi, (int)wbase, wlen, bits, wpre,
                            make_int4(0, 0, 0, 0), vals, 0, 0, err);
        __syncthreads();
      }
      // 2. ranks: a block prefix of the words' popcounts, kept as 16-bit
      // offsets inside groups of 2048 words plus the groups' offsets
      int sum = 0;
#pragma unroll 4
      for (int q = 0; q < WPT; ++q) {
        const int w = tid * WPT + q;
        if (w < nwords) sum += __popc(bits[w]);
      }
      const int incl = warp_incl_scan(sum);
      if (lane == 31) s_wsum[warp] = incl;
      __syncthreads();
      int woff = 0, total = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const int v = s_wsum[w];
        woff += w < warp ? v : 0;
        total += v;
      }
      const int excl = woff + incl - sum;
      if (((tid * WPT) & ((1 << RANK_GROUP_SHIFT) - 1)) == 0) s_gpre[(tid * WPT) >> RANK_GROUP_SHIFT] = excl;
      __syncthreads();
      {
        int run = excl - s_gpre[(tid * WPT) >> RANK_GROUP_SHIFT];
#pragma unroll 4
        for (int q = 0; q < WPT; ++q) {
          const int w = tid * WPT + q;
          if (w < nwords) {
            wpre[w] = (uint16_t)run;
            run += __popc(bits[w]);
          }
        }
      }
      if (out + total > out_end && tid == 0) atomicOr(err, EB_INTERNAL);
      __syncthreads();  // word offsets complete
      // columns in order: warp w takes slabs of 32 words (a slab lies inside
      // one group); lanes take consecutive outputs of a slab (owner word by
      // a warp search, bit by a binary search on popcounts), so the stores
      // are coalesced
      for (int sb = warp * 32; sb < nwords; sb += NT) {
        const int wi = sb + lane;
        const uint32_t m = wi < nwords ? bits[wi] : 0u;
        const int cnt = __popc(m);
        const int inc = warp_incl_scan(cnt);
        const int stot = __shfl_sync(FULL, inc, 31);
        const int first = out + s_gpre[sb >> RANK_GROUP_SHIFT] + (int)wpre[sb];  // rank of the slab's first output
        for (int q0 = 0; q0 < stot; q0 += 32) {
          const int q = q0 + lane;
          const int o = warp_owner(inc, q);
          const uint32_t mo = __shfl_sync(FULL, m, o & 31);
          const int eo = __shfl_sync(FULL, inc - cnt, o & 31);
          if (q < stot) {
            uint32_t x = mo;
            int rank = q - eo, bit = 0;
#pragma unroll
            for (int sh = 16; sh >= 1; sh >>= 1) {
              const int lowc = __popc(x & ((1u << sh) - 1u));
              if (rank >= lowc) {
                rank -= lowc;
                x >>= sh;
                bit += sh;
              }
            }
            const int p = first + q;
            if (p < out_end) __stcs(rci + p, (int)(wbase + (long long)((sb + o) << 5) + bit));
          }
        }
      }
      const int4 gp = make_int4(s_gpre[0], s_gpre[1], s_gpre[2], s_gpre[3]);
      if constexpr (CAP == 0) {
        // 3. values added in global memory: the row's entries of C are
        // zeroed (made visible before any reduction), then every product is
        // reduced into its rank's entry in the L2 cache
        const int nz = min(total, out_end - out);
        for (int t = tid; t < nz; t += NT) rcv[out + t] = T(0);
        __threadfence();
        if (one_round) {
          __syncthreads();
          const int nseg = (int)(pk >> 32), tot = (int)(unsigned)(pk & 0xffffffffull);
          const int share = ((tot + NT - 1) / NT) * 32;  // whole 32-product batches per warp
          const int lo = warp * share, hi = min(tot, lo + share);
          if (lo < hi && out + total <= out_end)
            rk_range<false, T, true>(B, bv, seg_off, seg_s, seg_a, nseg, tot, lo, hi, (int)wbase, wlen, bits, wpre,
                                     gp, rcv + out, 0, 0, err);
        } else {
          for (int r0 = a0; r0 < a1; r0 += SEGCAP) {
            const unsigned long long pr = rk_list<NW, T>(A, B, av, r0, min(a1, r0 + SEGCAP), whole, (int)wbase,
                                                         (int)wend, &s_pack, seg_off, seg_s, seg_a);
            const int nseg = (int)(pr >> 32), tot = (int)(unsigned)(pr & 0xffffffffull);
            const int share = ((tot + NT - 1) / NT) * 32;  // whole 32-product batches per warp
            const int lo = warp * share, hi = min(tot, lo + share);
            if (lo < hi && out + total <= out_end)
              rk_range<false, T, true>(B, bv, seg_off, seg_s, seg_a, nseg, tot, lo, hi, (int)wbase, wlen, bits,
                                       wpre, gp, rcv + out, 0, 0, err);
            __syncthreads();
          }
        }
      } else {
      // 3. values, CAP ranks at a time
      for (int t0 = 0; t0 < total; t0 += CAP) {
        const int chunk = min(CAP, total - t0);
        for (int t = tid; t < chunk; t += NT) vals[t] = T(0);
        if (one_round) {
          __syncthreads();
          const int nseg = (int)(pk >> 32), tot = (int)(unsigned)(pk & 0xffffffffull);
          const int share = ((tot + NT - 1) / NT) * 32;  // whole 32-product batches per warp
          const int lo = warp * share, hi = min(tot, lo + share);
          if (lo < hi)
            rk_range<false, T>(B, bv, seg_off, seg_s, seg_a, nseg, tot, lo, hi, (int)wbase, wlen, bits, wpre,
                               gp, vals, t0, chunk, err);
        } else {
          for (int r0 = a0; r0 < a1; r0 += SEGCAP) {
            const unsigned long long pr = rk_list<NW, T>(A, B, av, r0, min(a1, r0 + SEGCAP), whole, (int)wbase,
                                                         (int)wend, &s_pack, seg_off, seg_s, seg_a);
            const int nseg = (int)(pr >> 32), tot = (int)(unsigned)(pr & 0xffffffffull);
            const int share = ((tot + NT - 1) / NT) * 32;  // whole 32-product batches per warp
            const int lo = warp * share, hi = min(tot, lo + share);
            if (lo < hi)
              rk_range<false, T>(B, bv, seg_off, seg_s, seg_a, nseg, tot, lo, hi, (int)wbase, wlen, bits, wpre,
                                 gp, vals, t0, chunk, err);
            __syncthreads();
          }
        }
        __syncthreads();
        for (int t = tid; t < chunk; t += NT) {
          const int p = out + t0 + t;
          if (p < out_end) __stcs(rcv + p, vals[t]);
        }
        __syncthreads();  // vals is cleared again by the next chunk
      }
      }
      out += total;
      __syncthreads();  // the bitmap and offsets are rebuilt by the next window or row
    }
    if (tid == 0 && out != out_end) atomicOr(err, EB_INTERNAL);
  }
}

}  // namespace sg
