// Numeric pass for large rows: a dense column window shared by a block.
//
// Row i of C is the sum over A(i,k) of A(i,k) * B(k,:) (Sec. 2.2).  One block
// of NW warps owns one row at a time and a window of W consecutive columns
// (a multiple of the run width of B's window-run list, aligned to W): a
// dense value array and a presence bitmap in shared memory.  The row's
// nonzeros are dealt to the warps in chunks; for each window, a nonzero's
// segment of B(k,:) is the union of its consecutive runs whose window ids
// fall in the block window, so it is found by reading a few run entries, with
// no search.  Products from all warps land in the shared window, so they are
// added with shared-memory atomics (the hardware resolves equal addresses).
// The window is emitted in column order: every warp popcounts its share of
// the bitmap, a block prefix places the shares, lanes write their bits.
// Compared with one warp per row, a block window is W/1024 times wider, so a
// wide sparse row needs that many times fewer windows.
#pragma once

#include "internal.cuh"

namespace sg {

// Long segments (at least NB_LONG entries) are cut into pieces of
// NB_PIECE products and queued in shared memory; after the warps have read
// their nonzeros' segments, all warps take pieces from the queue, so one hub
// row of B no longer keeps a single warp busy while the others wait.
constexpr int NB_LONG = 128;
constexpr int NB_PIECE = 256;
constexpr int NB_QCAP = 512;

template <typename T>
struct NbPiece {
  int s;    // first position in B
  int len;  // products in this piece
  T a;      // A(i,k)
};

template <int W, int NW, typename T>
__host__ __device__ constexpr size_t numblock_smem_bytes() {
  return (size_t)W * sizeof(T) + (size_t)(W / 32) * 4 + (size_t)NW * 8 + 16 +
         (size_t)NB_QCAP * sizeof(NbPiece<T>) + 16;
}

// Products of one segment piece by the whole warp (distinct columns inside
// the piece; other warps may hit the same columns, hence atomics).
template <int W, typename T>
__device__ __forceinline__ void nb_piece(const Csr& B, const T* __restrict__ bv, int s, int len, T a, int base,
                                         T* acc, uint32_t* bits, uint32_t* err) {
  const int lane = lane_id();
  int t = lane;
  for (; t + 96 < len; t += 128) {
    const int q = s + t;
    const int j0 = B.ci[q] - base, j1 = B.ci[q + 32] - base, j2 = B.ci[q + 64] - base, j3 = B.ci[q + 96] - base;
    const T b0 = bv[q], b1 = bv[q + 32], b2 = bv[q + 64], b3 = bv[q + 96];
    if (((unsigned)j0 | (unsigned)j1 | (unsigned)j2 | (unsigned)j3) < (unsigned)W) {
      atomicOr(&bits[j0 >> 5], 1u << (j0 & 31));
      atomicAdd(&acc[j0], a * b0);
      atomicOr(&bits[j1 >> 5], 1u << (j1 & 31));
      atomicAdd(&acc[j1], a * b1);
      atomicOr(&bits[j2 >> 5], 1u << (j2 & 31));
      atomicAdd(&acc[j2], a * b2);
      atomicOr(&bits[j3 >> 5], 1u << (j3 & 31));
      atomicAdd(&acc[j3], a * b3);
    } else {
      atomicOr(err, EB_UNSORTED);
    }
  }
  for (; t < len; t += 32) {
    const int q = s + t;
    const int jj = B.ci[q] - base;
    if ((unsigned)jj < (unsigned)W) {
      atomicOr(&bits[jj >> 5], 1u << (jj & 31));
      atomicAdd(&acc[jj], a * bv[q]);
    } else {
      atomicOr(err, EB_UNSORTED);
    }
  }
}

template <int W, int NW, typename T>
__global__ void __launch_bounds__(NW * 32)
k_num_block(Csr A, Csr B, const T* __restrict__ av, const T* __restrict__ bv, RowInfo ri, const DevStats* st,
            int bin_lo, int bin_hi, const int32_t* __restrict__ rr, const int2* __restrict__ runs, int run_shift,
            int32_t* __restrict__ gcur, int32_t* __restrict__ gnxt, const int32_t* __restrict__ c_rp,
            int32_t* __restrict__ c_ci, T* __restrict__ c_v, unsigned* counter, uint32_t* err) {
  static_assert(W % 1024 == 0, "window must be a multiple of 1024 columns");
  constexpr int NWORDS = W / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* acc = reinterpret_cast<T*>(smem_raw);
  uint32_t* bits = reinterpret_cast<uint32_t*>(smem_raw + (size_t)W * sizeof(T));
  int* wcnt = reinterpret_cast<int*>(bits + NWORDS);
  int* wnext = wcnt + NW;
  NbPiece<T>* queue = reinterpret_cast<NbPiece<T>*>(
      smem_raw + (((size_t)W * sizeof(T) + (size_t)NWORDS * 4 + (size_t)NW * 8 + 16 + 15) & ~(size_t)15));
  __shared__ int s_lb, s_le, s_item, s_qn, s_qtake;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  for (int t = threadIdx.x; t < W; t += NW * 32) acc[t] = T(0);
  for (int t = threadIdx.x; t < NWORDS; t += NW * 32) bits[t] = 0u;
  if (threadIdx.x == 0) {
    bin_range(st, bin_lo, bin_hi, &s_lb, &s_le);
    s_qn = 0;
    s_qtake = 0;
  }
  if (block_skip(st)) return;
  const int lb = s_lb, le = s_le;
  const int wshift = 31 - __clz(W);      // block window width
  const int rper = W >> run_shift;       // run windows of B per block window

  while (true) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const long long idx = (long long)lb + s_item;
    __syncthreads();  // s_item is reused by the next iteration
    if (idx >= le) break;
    const int r = ri.rows[idx];
    const long long i = ri.row_begin + r;
    const int a0 = A.rp[i], a1 = A.rp[i + 1], nA = a1 - a0;
    const int cmx = ri.cmax[r];
    const long long rbeg = c_rp[r];
    const int out_end = (int)(c_rp[r + 1] - rbeg);
    int32_t* const rci = c_ci + rbeg;
    T* const rcv = c_v + rbeg;
    const int CS = min(32, max(1, (nA + NW - 1) / NW));  // nonzeros per chunk
    const int nch = (nA + CS - 1) / CS;
    // cursor of every nonzero: index of its current run in B's run list;
    // gnxt holds that run's window id (INT_MAX when the B row is done)
    int mn = INT_MAX;
    for (int c = warp; c < nch; c += NW) {
      const int e = a0 + c * CS + lane;
      if (lane < CS && e < a1) {
        const int j = rr[A.ci[e]];
        const int wid = runs[j].x;
        gcur[e] = j;
        gnxt[e] = wid;
        mn = min(mn, wid);
      }
    }
    mn = warp_min(mn);
    if (lane == 0) wnext[warp] = mn;
    __syncthreads();
    const int dshift = wshift - run_shift;  // run windows per block window = 2^dshift
    int wb = INT_MAX;  // block window index
    for (int w = 0; w < NW; ++w) wb = min(wb, wnext[w]);
    if (wb != INT_MAX) wb >>= dshift;
    int out = 0;
    while (wb != INT_MAX) {
      const int base = wb << wshift;
      const int wlim = (wb + 1) * rper;  // first run window id past this block window
      mn = INT_MAX;
      for (int c = warp; c < nch; c += NW) {
        const int e = a0 + c * CS + lane;
        int s = 0, len = 0;
        T a = T(0);
        if (lane < CS && e < a1) {
          int wid = gnxt[e];
          if (wid < wlim) {
            int j = gcur[e];
            s = runs[j].y;
            do {  // consecutive runs of this B row inside the block window
              ++j;
              wid = runs[j].x;
            } while (wid < wlim);
            len = runs[j].y - s;
            gcur[e] = j;
            gnxt[e] = wid;
            a = av[e];
          }
          mn = min(mn, wid);
        }
        // very long segments: queue their pieces for all warps (warp-aggregated
        // reservation); if the queue is full the warp keeps the segment
        bool keep = len >= 32;
        if (len >= NB_LONG) {
          const int np = (len + NB_PIECE - 1) / NB_PIECE;
          const int at = atomicAdd(&s_qn, np);  // reserve np slots
          if (at + np <= NB_QCAP) {
            for (int p = 0; p < np; ++p) {
              NbPiece<T> pc;
              pc.s = s + p * NB_PIECE;
              pc.len = min(NB_PIECE, len - p * NB_PIECE);
              pc.a = a;
              queue[at + p] = pc;
            }
            keep = false;
          } else {
            // queue full: the slots reserved below the capacity stay empty
            for (int p = at; p < NB_QCAP && p < at + np; ++p) {
              NbPiece<T> pc;
              pc.s = 0;
              pc.len = 0;
              pc.a = T(0);
              queue[p] = pc;
            }
          }
        }
        // remaining long segments by the whole warp, short ones flattened
        unsigned lm = __ballot_sync(FULL, keep);
        while (lm) {
          const int L = __ffs(lm) - 1;
          lm &= lm - 1;
          const int ls = __shfl_sync(FULL, s, L), ln = __shfl_sync(FULL, len, L);
          const T la = __shfl_sync(FULL, a, L);
          nb_piece<W, T>(B, bv, ls, ln, la, base, acc, bits, err);
        }
        const int sl = len < 32 ? len : 0;
        const int incl = warp_incl_scan(sl);
        const int tot = __shfl_sync(FULL, incl, 31);
        const int excl = incl - sl;
        for (int p0 = 0; p0 < tot; p0 += 32) {
          const int p = p0 + lane;
          const int o = warp_owner(incl, p);
          const int os = __shfl_sync(FULL, s, o), oex = __shfl_sync(FULL, excl, o);
          const T oa = __shfl_sync(FULL, a, o);
          if (p < tot) {
            const int q = os + p - oex;
            const int jj = B.ci[q] - base;
            if ((unsigned)jj < (unsigned)W) {
              atomicOr(&bits[jj >> 5], 1u << (jj & 31));
              atomicAdd(&acc[jj], oa * bv[q]);
            } else {
              atomicOr(err, EB_UNSORTED);
            }
          }
        }
      }
      mn = warp_min(mn);
      __syncthreads();  // the queue is complete
      {
        const int qn = min(s_qn, NB_QCAP);
        while (true) {
          int pi = 0;
          if (lane == 0) pi = atomicAdd(&s_qtake, 1);
          pi = __shfl_sync(FULL, pi, 0);
          if (pi >= qn) break;
          const NbPiece<T> pc = queue[pi];
          nb_piece<W, T>(B, bv, pc.s, pc.len, pc.a, base, acc, bits, err);
        }
      }
      // emission: each warp takes NWORDS / NW consecutive words of the bitmap
      const int ncols = min(W, cmx - base + 1);
      const int nwd = (ncols + 31) >> 5;
      constexpr int WPW = NWORDS / NW;
      __syncthreads();  // all products are in
      const int w0 = warp * WPW;
      int cnt = 0;
      for (int j = w0 + lane; j < w0 + WPW && j < nwd; j += 32) cnt += __popc(bits[j]);
      cnt = warp_sum(cnt);
      if (lane == 0) {
        wcnt[warp] = cnt;
        wnext[warp] = mn;
      }
      if (threadIdx.x == 0) {  // queue drained by everyone (all past the barrier above)
        s_qn = 0;
        s_qtake = 0;
      }
      __syncthreads();
      int before = 0, total = 0, nb = INT_MAX;
      for (int w = 0; w < NW; ++w) {
        const int v = wcnt[w];
        if (w < warp) before += v;
        total += v;
        nb = min(nb, wnext[w]);
      }
      int pos0 = out + before;
      for (int jb = w0; jb < w0 + WPW && jb < nwd; jb += 32) {
        const int j = jb + lane;
        uint32_t m = (j < w0 + WPW && j < nwd) ? bits[j] : 0u;
        const int c = __popc(m);
        const int inc = warp_incl_scan(c);
        int pos = pos0 + inc - c;
        if (m) bits[j] = 0u;
        while (m) {
          const int b = __ffs(m) - 1;
          m &= m - 1;
          const int jj = (j << 5) + b;
          if (pos < out_end) {
            __stcs(rci + pos, base + jj);
            __stcs(rcv + pos, acc[jj]);
          } else {
            atomicOr(err, EB_INTERNAL);
          }
          acc[jj] = T(0);
          ++pos;
        }
        pos0 += __shfl_sync(FULL, inc, 31);
      }
      out += total;
      __syncthreads();  // window cleared before the next one fills it
      wb = nb == INT_MAX ? INT_MAX : (nb >> dshift);
    }
    if (threadIdx.x == 0 && out != out_end) atomicOr(err, EB_INTERNAL);
  }
}

}  // namespace sg
