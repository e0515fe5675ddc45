// Numeric pass: columns (ascending) and values of every row of C, per path
// of the row bins; templated on the value type and on the semiring (Sec. 2.2's
// sum and product, or min-plus, max-plus, or-and: those skip the rank path,
// register sorts above 128 products and the non-default window sizes).
#pragma once

#include <cstddef>

#include "launch_util.cuh"
#include "numblock.cuh"
#include "numrank.cuh"
#include "numwarp.cuh"
#include "rowhash.cuh"
#include "rowlane.cuh"
#include "rowpass.cuh"

namespace sg {

constexpr int NUM_WARPS_CTA = 4;  // warps per block on the window path
// k_num_warp1's warps per block: 9 warps of 1024-column FP64 windows
// (74.9 KB) let 3 blocks, 27 warps, share an SM's 228 KB of shared memory
// (4-warp blocks fit 24); wider windows take fewer warps per block.
template <int W>
constexpr int num_warps_cta1() {
  return W <= 1024 ? 9 : (W <= 2048 ? 4 : 2);
}

static long long rows_in(const int* path_rows, int p) { return path_rows ? path_rows[p] : -1; }

template <typename T, int G, int E, int SR>
static cudaError_t tiny_num(const LaunchCtx& c, const Csr& A, const Csr& B, const T* av, const T* bv,
                            const RowInfo& ri, int lo, int hi, const int32_t* c_rp, int32_t* c_ci, T* c_v,
                            long long rows) {
  auto k = k_tiny<G, E, true, T, SR>;
  const int occ = kernel_blocks_per_sm(k, 256, 0);
  const int grid = persistent_grid(rows, 8 * (32 / G), c.nsm, occ);
  k<<<grid, 256, 0, c.stream>>>(A, B, av, bv, ri, c.st, lo, hi, nullptr, c_rp, c_ci, c_v, c.err);
  count_launch(c);
  return cudaGetLastError();
}

template <typename T, int E, int SR>
static cudaError_t hash_num(const LaunchCtx& c, const Csr& A, const Csr& B, const T* av, const T* bv,
                            const RowInfo& ri, int lo, int hi, const int32_t* c_rp, int32_t* c_ci, T* c_v,
                            long long rows) {
  auto k = k_hash_num<E, T, SR>;
  const int occ = kernel_blocks_per_sm(k, HASH_WARPS * 32, 0);
  const int grid = persistent_grid(rows, HASH_WARPS, c.nsm, occ);
  k<<<grid, HASH_WARPS * 32, 0, c.stream>>>(A, B, av, bv, ri, c.st, lo, hi, c_rp, c_ci, c_v, c.err);
  count_launch(c);
  return cudaGetLastError();
}

// Whether bins lo..hi hold no row (hist: rows per bin on the host, as the
// symbolic pass read them; null: unknown, never empty).
static bool empty_bins(const int* hist, int lo, int hi) {
  if (!hist) return false;
  for (int b = lo; b <= hi; ++b)
    if (hist[b]) return false;
  return true;
}

// Hash bins: 6 -> 1 product per lane (P <= 32), 7 -> 2 (P <= 64), 8 -> 4 (P <= 128).
template <typename F1, typename F2, typename F4>
static cudaError_t hash_dispatch(const int* hist, int lo, int hi, F1 f1, F2 f2, F4 f4) {
  cudaError_t e = cudaSuccess;
  auto clip = [&](int a, int b, auto f) -> cudaError_t {
    const int l = lo > a ? lo : a, h = hi < b ? hi : b;
    return (l <= h && !empty_bins(hist, l, h)) ? f(l, h) : cudaSuccess;
  };
  if ((e = clip(1, 6, f1))) return e;
  if ((e = clip(7, 7, f2))) return e;
  if ((e = clip(8, 8, f4))) return e;
  return cudaSuccess;
}

template <typename T, int W, int SR>
static cudaError_t warp_num(const LaunchCtx& c, const Csr& A, const Csr& B, const T* av, const T* bv,
                            const RowInfo& ri, int lo, int hi, const SplitInfo& sp, int32_t* cur, int32_t* nxt,
                            const int32_t* c_rp, int32_t* c_ci, T* c_v, long long rows_wide) {
  auto k = k_num_warp<W, NUM_WARPS_CTA, T, SR>;
  const size_t smem = (size_t)NUM_WARPS_CTA * ((size_t)W * sizeof(T) + W / 8);
  const int occ = kernel_blocks_per_sm(k, NUM_WARPS_CTA * 32, smem);
  if (occ <= 0) return cudaErrorInvalidConfiguration;
  NumSplit ns;
  ns.heavy_bin = sp.heavy_bin;
  ns.hi_bin = sp.hi_bin;
  ns.hcap = sp.hcap;
  ns.ntf = sp.ntf;
  ns.rr = sp.rr;
  ns.runs = sp.runs;
  ns.hcnt = sp.hcnt;
  ns.counter = &c.st->work[0];
  // rows of at most 32 nonzeros first (one cursor per lane, next window's
  // loads overlapped with this window's emission), then the others
  constexpr int NW1 = num_warps_cta1<W>();
  auto k1 = k_num_warp1<W, NW1, T, SR>;
  const size_t smem1 = (size_t)NW1 * ((size_t)W * sizeof(T) + W / 8);
  const int occ1 = kernel_blocks_per_sm(k1, NW1 * 32, smem1);
  if (occ1 <= 0) return cudaErrorInvalidConfiguration;
  unsigned* counter1 = &c.st->work[3];
  // the general kernel has work only for split rows and rows of more than
  // 32 nonzeros (a stencil or Galerkin product has neither)
  const bool general = rows_wide != 0 || (sp.heavy_bin < NBINS && sp.hcap > 0);
  cudaError_t e = cudaMemsetAsync(counter1, 0, sizeof(unsigned), c.stream);
  if (e == cudaSuccess && general) e = cudaMemsetAsync(ns.counter, 0, sizeof(unsigned), c.stream);
  if (e != cudaSuccess) return e;
  k1<<<c.nsm * occ1, NW1 * 32, smem1, c.stream>>>(A, B, av, bv, ri, c.st, lo, hi, ns, c_rp, c_ci, c_v,
                                                           counter1, c.err);
  count_launch(c);
  if ((e = cudaGetLastError()) != cudaSuccess || !general) return e;
  const int grid = c.nsm * occ;
  k<<<grid, NUM_WARPS_CTA * 32, smem, c.stream>>>(A, B, av, bv, ri, c.st, lo, hi, ns, cur, nxt, c_rp, c_ci, c_v,
                                                  c.err, 1);
  count_launch(c);
  return cudaGetLastError();
}

template <typename T, int W, int NUM_BLOCK_WARPS, int SR>
static cudaError_t block_num(const LaunchCtx& c, const Csr& A, const Csr& B, const T* av, const T* bv,
                             const RowInfo& ri, int lo, int hi, const SplitInfo& sp, int32_t* cur, int32_t* nxt,
                             const int32_t* c_rp, int32_t* c_ci, T* c_v) {
  auto k = k_num_block<W, NUM_BLOCK_WARPS, T, SR>;
  const size_t smem = numblock_smem_bytes<W, NUM_BLOCK_WARPS, T>();
  const int occ = kernel_blocks_per_sm(k, NUM_BLOCK_WARPS * 32, smem);
  if (occ <= 0) return cudaErrorInvalidConfiguration;
  unsigned* counter = &c.st->work[1];
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), c.stream);
  if (e != cudaSuccess) return e;
  if (!sp.rrb || !sp.runsb || (1 << sp.wb_shift) != W) return cudaErrorInvalidValue;  // block-granular runs
  k<<<c.nsm * occ, NUM_BLOCK_WARPS * 32, smem, c.stream>>>(A, B, av, bv, ri, c.st, lo, hi, sp.rrb, sp.runsb, cur,
                                                          c_rp, c_ci, c_v, counter, c.err);
  count_launch(c);
  return cudaGetLastError();
}

// Rank-compacted accumulator: 8 warps per block; values either reduced into
// C in global memory (the default, 56 KB of shared memory per block, four
// blocks per SM) or summed in shared memory 6144 ranks at a time (104 KB in
// FP64, two blocks per SM).
constexpr int RANK_WARPS = 8;
constexpr int RANK_CAP = 6144;

template <typename T, int CAP>
static cudaError_t rank_num(const LaunchCtx& c, const Csr& A, const Csr& B, const T* av, const T* bv,
                            const RowInfo& ri, int lo, int hi, const int32_t* c_rp, int32_t* c_ci, T* c_v) {
  auto k = k_num_rank<RANK_WARPS, CAP, T>;
  const size_t smem = numrank_smem_bytes<RANK_WARPS, CAP, T>();
  const int occ = kernel_blocks_per_sm(k, RANK_WARPS * 32, smem);
  if (occ <= 0) return cudaErrorInvalidConfiguration;
  unsigned* counter = &c.st->work[2];
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), c.stream);
  if (e != cudaSuccess) return e;
  k<<<c.nsm * occ, RANK_WARPS * 32, smem, c.stream>>>(A, B, av, bv, ri, c.st, lo, hi, c_rp, c_ci, c_v, counter,
                                                      c.err);
  count_launch(c);
  return cudaGetLastError();
}

// The rank-compacted path and register sorts of more than 128 products
// exist for the ordinary sum and product only; other semirings never route
// rows to them.
template <typename T, int G, int E, int SR>
static cudaError_t tiny_num_wide(const LaunchCtx& c, const Csr& A, const Csr& B, const T* av, const T* bv,
                                 const RowInfo& ri, int lo, int hi, const int32_t* c_rp, int32_t* c_ci, T* c_v,
                                 long long rows) {
  if constexpr (SR == SPGEMM_PLUS_TIMES) return tiny_num<T, G, E, SR>(c, A, B, av, bv, ri, lo, hi, c_rp, c_ci, c_v, rows);
  else return cudaErrorInvalidValue;
}
template <typename T, int CAP, int SR>
static cudaError_t rank_num_plus(const LaunchCtx& c, const Csr& A, const Csr& B, const T* av, const T* bv,
                                 const RowInfo& ri, int lo, int hi, const int32_t* c_rp, int32_t* c_ci, T* c_v) {
  if constexpr (SR == SPGEMM_PLUS_TIMES) return rank_num<T, CAP>(c, A, B, av, bv, ri, lo, hi, c_rp, c_ci, c_v);
  else return cudaErrorInvalidValue;
}

template <typename F8, typename F16, typename F32, typename F64, typename F128, typename F256, typename F512>
static cudaError_t tiny_dispatch(const int* hist, int lo, int hi, F8 f8, F16 f16, F32 f32, F64 f64, F128 f128,
                                 F256 f256, F512 f512) {
  cudaError_t e = cudaSuccess;
  auto clip = [&](int a, int b, auto f) -> cudaError_t {
    const int l = lo > a ? lo : a, h = hi < b ? hi : b;
    return (l <= h && !empty_bins(hist, l, h)) ? f(l, h) : cudaSuccess;
  };
  if ((e = clip(1, 4, f8))) return e;
  if ((e = clip(5, 5, f16))) return e;
  if ((e = clip(6, 6, f32))) return e;
  if ((e = clip(7, 7, f64))) return e;
  if ((e = clip(8, 8, f128))) return e;
  if ((e = clip(9, 9, f256))) return e;
  if ((e = clip(10, 10, f512))) return e;
  return cudaSuccess;
}

template <typename T, int SR>
static cudaError_t numeric_t(const LaunchCtx& c, const Csr& A, const Csr& B, const RowInfo& ri,
                             const PathBins& pb, const Tuning& tu, const SplitInfo& sp, const T* av,
                             const T* bv, int32_t* cur, int32_t* nxt, const int32_t* c_rp, int32_t* c_ci,
                             T* c_v, const int* path_rows, long long rows_wide, const int* hist) {
  cudaError_t e = cudaSuccess;
  if (pb.hi[PATH_TINY] >= pb.lo[PATH_TINY]) {
    const long long rows = rows_in(path_rows, PATH_TINY);
    timer_mark(c, T_NUM_TINY, 0);
    e = tiny_dispatch(hist, pb.lo[PATH_TINY], pb.hi[PATH_TINY],
        [&](int l, int h) { return tiny_num<T, 8, 1, SR>(c, A, B, av, bv, ri, l, h, c_rp, c_ci, c_v, rows); },
        [&](int l, int h) { return tiny_num<T, 16, 1, SR>(c, A, B, av, bv, ri, l, h, c_rp, c_ci, c_v, rows); },
        [&](int l, int h) { return tiny_num<T, 32, 1, SR>(c, A, B, av, bv, ri, l, h, c_rp, c_ci, c_v, rows); },
        [&](int l, int h) { return tiny_num<T, 32, 2, SR>(c, A, B, av, bv, ri, l, h, c_rp, c_ci, c_v, rows); },
        [&](int l, int h) { return tiny_num<T, 32, 4, SR>(c, A, B, av, bv, ri, l, h, c_rp, c_ci, c_v, rows); },
        [&](int l, int h) { return tiny_num_wide<T, 32, 8, SR>(c, A, B, av, bv, ri, l, h, c_rp, c_ci, c_v, rows); },
        [&](int l, int h) { return tiny_num_wide<T, 32, 16, SR>(c, A, B, av, bv, ri, l, h, c_rp, c_ci, c_v, rows); });
    timer_mark(c, T_NUM_TINY, 1);
    if (e) return e;
  }
  if (pb.hi[PATH_HASH] >= pb.lo[PATH_HASH]) {
    const long long rows = rows_in(path_rows, PATH_HASH);
    timer_mark(c, T_NUM_HASH, 0);
    // When the hash rows are most of the product's rows (stencil and
    // Galerkin products, where every row lands here), rows of at most 64
    // products take one lane per row: throughput over many similar rows.
    // A few such rows among larger ones (a power-law product) keep the warp
    // per row, whose latency per row is lower.
    long long all_rows = 0;
    if (path_rows)
      for (int q = 0; q < NPATHS; ++q) all_rows += path_rows[q];
    const bool lanes = path_rows && 2 * (long long)path_rows[PATH_HASH] >= all_rows;
    const int llo = pb.lo[PATH_HASH], lhi = lanes ? (pb.hi[PATH_HASH] < 7 ? pb.hi[PATH_HASH] : 7) : 0;
    if (llo <= lhi && !empty_bins(hist, llo, lhi))
      e = lane_rows<true, T, SR>(c, A, B, av, bv, ri, llo, lhi, nullptr, c_rp, c_ci, c_v, rows);
    const int wlo = lhi >= llo ? lhi + 1 : llo;
    if (!e && pb.hi[PATH_HASH] >= wlo)
      e = hash_dispatch(hist, wlo, pb.hi[PATH_HASH],
          [&](int l, int h) { return hash_num<T, 1, SR>(c, A, B, av, bv, ri, l, h, c_rp, c_ci, c_v, rows); },
          [&](int l, int h) { return hash_num<T, 2, SR>(c, A, B, av, bv, ri, l, h, c_rp, c_ci, c_v, rows); },
          [&](int l, int h) { return hash_num<T, 4, SR>(c, A, B, av, bv, ri, l, h, c_rp, c_ci, c_v, rows); });
    timer_mark(c, T_NUM_HASH, 1);
    if (e) return e;
  }
  // every other row: the warp-owned dense window up to tu.num_lo_block,
  // the block-wide window from there on (rows of the symbolic warp and block
  // paths both land here)
  int lo = NBINS, hi = 0;
  for (int p : {PATH_WARP, PATH_BLOCK})
    if (pb.hi[p] >= pb.lo[p]) {
      lo = pb.lo[p] < lo ? pb.lo[p] : lo;
      hi = pb.hi[p] > hi ? pb.hi[p] : hi;
    }
  const int blo = tu.num_lo_block > lo ? tu.num_lo_block : lo;
  if (hi >= blo && !empty_bins(hist, blo, hi)) {
    timer_mark(c, T_NUM_BLOCK, 0);
#define SG_BLOCK_NUM(WW, NWW) e = block_num<T, WW, NWW, SR>(c, A, B, av, bv, ri, blo, hi, sp, cur, nxt, c_rp, c_ci, c_v)
    // supported geometries (window columns, warps); others fall back to 8192 x 8
    const int wbk = tu.window_block, nwk = tu.block_warps;
    if (SR != SPGEMM_PLUS_TIMES) SG_BLOCK_NUM(8192, 8);
    else if (wbk == 2048 && nwk == 4) SG_BLOCK_NUM(2048, 4);
    else if (wbk == 2048 && nwk == 8) SG_BLOCK_NUM(2048, 8);
    else if (wbk == 4096 && nwk == 4) SG_BLOCK_NUM(4096, 4);
    else if (wbk == 4096 && nwk == 8) SG_BLOCK_NUM(4096, 8);
    else if (wbk == 4096 && nwk == 16) SG_BLOCK_NUM(4096, 16);
    else if (wbk == 16384 && nwk == 16) SG_BLOCK_NUM(16384, 16);
    else if (wbk == 8192 && nwk == 16) SG_BLOCK_NUM(8192, 16);
    else SG_BLOCK_NUM(8192, 8);
#undef SG_BLOCK_NUM
    timer_mark(c, T_NUM_BLOCK, 1);
    if (e) return e;
  }
  if (hi >= blo) hi = blo - 1;
  // rows of the rank bins (below the block window) take the rank-compacted
  // accumulator, unless heavy rows are split (the warp kernel owns those)
  const bool split = sp.heavy_bin < NBINS && sp.hcap > 0;
  const int rlo = tu.num_lo_rank > lo ? tu.num_lo_rank : lo;
  if (SR == SPGEMM_PLUS_TIMES && !split && hi >= rlo) {
    if (!empty_bins(hist, rlo, hi)) {
      timer_mark(c, T_NUM_RANK, 0);
      e = tu.rank_accum == 1 ? rank_num_plus<T, RANK_CAP, SR>(c, A, B, av, bv, ri, rlo, hi, c_rp, c_ci, c_v)
                             : rank_num_plus<T, 0, SR>(c, A, B, av, bv, ri, rlo, hi, c_rp, c_ci, c_v);
      timer_mark(c, T_NUM_RANK, 1);
      if (e) return e;
    }
    hi = rlo - 1;
  }
  if (hi >= lo && !empty_bins(hist, lo, hi)) {
    timer_mark(c, T_NUM_WARP, 0);
    switch (SR == SPGEMM_PLUS_TIMES ? tu.window_warp : 1024) {
      case 2048: e = warp_num<T, 2048, SR>(c, A, B, av, bv, ri, lo, hi, sp, cur, nxt, c_rp, c_ci, c_v, rows_wide); break;
      case 4096: e = warp_num<T, 4096, SR>(c, A, B, av, bv, ri, lo, hi, sp, cur, nxt, c_rp, c_ci, c_v, rows_wide); break;
      default: e = warp_num<T, 1024, SR>(c, A, B, av, bv, ri, lo, hi, sp, cur, nxt, c_rp, c_ci, c_v, rows_wide); break;
    }
    timer_mark(c, T_NUM_WARP, 1);
    if (e) return e;
  }
  return cudaSuccess;
}


// Entry of the numeric pass for one semiring, both value types.
template <int SR>
static cudaError_t launch_numeric_sr(const LaunchCtx& c, const Csr& A, const Csr& B, const RowInfo& ri,
                                     const PathBins& pb, const Tuning& tu, const SplitInfo& sp, int dtype,
                                     const void* av, const void* bv, int32_t* cur, int32_t* nxt,
                                     const int32_t* c_rp, int32_t* c_ci, void* c_v, const int* path_rows,
                                     long long rows_wide, const int* hist) {
  if (dtype == SPGEMM_F32)
    return numeric_t<float, SR>(c, A, B, ri, pb, tu, sp, (const float*)av, (const float*)bv, cur, nxt, c_rp, c_ci,
                                (float*)c_v, path_rows, rows_wide, hist);
  return numeric_t<double, SR>(c, A, B, ri, pb, tu, sp, (const double*)av, (const double*)bv, cur, nxt, c_rp, c_ci,
                               (double*)c_v, path_rows, rows_wide, hist);
}

}  // namespace sg
