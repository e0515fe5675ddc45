// Numeric pass: columns (ascending) and values of every row of C.
#include "launch_util.cuh"
#include "rowpass.cuh"

namespace sg {

constexpr int NUM_WARP_CTA = 8;     // warps (rows) per block on the warp path
constexpr int NUM_BLOCK_WARPS = 16; // warps per row on the block path

static long long rows_in(const int* path_rows, int p) { return path_rows ? path_rows[p] : -1; }

template <typename T, int G>
static cudaError_t tiny_launch(const LaunchCtx& c, const Csr& A, const Csr& B, const T* av, const T* bv,
                               const RowInfo& ri, int lo, int hi, const int32_t* c_rp, int32_t* c_ci,
                               T* c_v, long long rows) {
  auto k = k_tiny<G, true, T>;
  const int occ = kernel_blocks_per_sm(k, 256, 0);
  const int grid = persistent_grid(rows, 8 * (32 / G), c.nsm, occ);
  k<<<grid, 256, 0, c.stream>>>(A, B, av, bv, ri, c.st, lo, hi, nullptr, c_rp, c_ci, c_v, c.err);
  count_launch(c);
  return cudaGetLastError();
}

template <typename T, int GW, int CW, int W>
static cudaError_t window_launch(const LaunchCtx& c, const Csr& A, const Csr& B, const T* av, const T* bv,
                                 const RowInfo& ri, int lo, int hi, int32_t* cursor, const int32_t* c_rp,
                                 int32_t* c_ci, T* c_v, long long rows) {
  auto k = k_window<GW, CW, W, true, T>;
  const size_t smem = (size_t)(CW / GW) * window_group_bytes<W, true, T>(GW);
  const int occ = kernel_blocks_per_sm(k, CW * 32, smem);
  if (occ <= 0) return cudaErrorInvalidConfiguration;
  const int grid = persistent_grid(rows, CW / GW, c.nsm, occ);
  k<<<grid, CW * 32, smem, c.stream>>>(A, B, av, bv, ri, c.st, lo, hi, cursor, nullptr, c_rp, c_ci, c_v, c.err);
  count_launch(c);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t numeric_t(const LaunchCtx& c, const Csr& A, const Csr& B, const RowInfo& ri,
                             const PathBins& pb, const Tuning& tu, const T* av, const T* bv,
                             int32_t* cursor, const int32_t* c_rp, int32_t* c_ci, T* c_v,
                             const int* path_rows) {
  cudaError_t e = cudaSuccess;
  if (pb.hi[PATH_TINY] >= pb.lo[PATH_TINY]) {
    const int lo = pb.lo[PATH_TINY], hi = pb.hi[PATH_TINY];
    const long long rows = rows_in(path_rows, PATH_TINY);
    timer_mark(c, T_NUM_TINY, 0);
    if (lo <= 4 && (e = tiny_launch<T, 8>(c, A, B, av, bv, ri, lo, hi < 4 ? hi : 4, c_rp, c_ci, c_v, rows))) return e;
    if (lo <= 5 && hi >= 5 && (e = tiny_launch<T, 16>(c, A, B, av, bv, ri, 5, 5, c_rp, c_ci, c_v, rows))) return e;
    if (hi >= 6 && (e = tiny_launch<T, 32>(c, A, B, av, bv, ri, 6 > lo ? 6 : lo, hi, c_rp, c_ci, c_v, rows))) return e;
    timer_mark(c, T_NUM_TINY, 1);
  }
  if (pb.hi[PATH_WARP] >= pb.lo[PATH_WARP]) {
    const int lo = pb.lo[PATH_WARP], hi = pb.hi[PATH_WARP];
    const long long rows = rows_in(path_rows, PATH_WARP);
    timer_mark(c, T_NUM_WARP, 0);
    switch (tu.window_warp) {
      case 512: e = window_launch<T, 1, NUM_WARP_CTA, 512>(c, A, B, av, bv, ri, lo, hi, cursor, c_rp, c_ci, c_v, rows); break;
      case 2048: e = window_launch<T, 1, NUM_WARP_CTA, 2048>(c, A, B, av, bv, ri, lo, hi, cursor, c_rp, c_ci, c_v, rows); break;
      default: e = window_launch<T, 1, NUM_WARP_CTA, 1024>(c, A, B, av, bv, ri, lo, hi, cursor, c_rp, c_ci, c_v, rows); break;
    }
    timer_mark(c, T_NUM_WARP, 1);
    if (e) return e;
  }
  if (pb.hi[PATH_BLOCK] >= pb.lo[PATH_BLOCK]) {
    const int lo = pb.lo[PATH_BLOCK], hi = pb.hi[PATH_BLOCK];
    const long long rows = rows_in(path_rows, PATH_BLOCK);
    timer_mark(c, T_NUM_BLOCK, 0);
    switch (tu.window_block) {
      case 4096: e = window_launch<T, NUM_BLOCK_WARPS, NUM_BLOCK_WARPS, 4096>(c, A, B, av, bv, ri, lo, hi, cursor, c_rp, c_ci, c_v, rows); break;
      case 16384: e = window_launch<T, NUM_BLOCK_WARPS, NUM_BLOCK_WARPS, 16384>(c, A, B, av, bv, ri, lo, hi, cursor, c_rp, c_ci, c_v, rows); break;
      default: e = window_launch<T, NUM_BLOCK_WARPS, NUM_BLOCK_WARPS, 8192>(c, A, B, av, bv, ri, lo, hi, cursor, c_rp, c_ci, c_v, rows); break;
    }
    timer_mark(c, T_NUM_BLOCK, 1);
    if (e) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_numeric(const LaunchCtx& c, const Csr& A, const Csr& B, const RowInfo& ri,
                           const PathBins& pb, const Tuning& tu, int dtype, const void* av,
                           const void* bv, int32_t* cursor, const int32_t* c_rp, int32_t* c_ci,
                           void* c_v, const int* path_rows) {
  if (dtype == SPGEMM_F32)
    return numeric_t<float>(c, A, B, ri, pb, tu, (const float*)av, (const float*)bv, cursor, c_rp, c_ci,
                            (float*)c_v, path_rows);
  return numeric_t<double>(c, A, B, ri, pb, tu, (const double*)av, (const double*)bv, cursor, c_rp, c_ci,
                           (double*)c_v, path_rows);
}

}  // namespace sg
