// Symbolic pass: the number of distinct columns of every row of C
// (Sec. 2.2: the union of the columns of the B rows a row of A touches).
#include "launch_util.cuh"
#include "rowpass.cuh"

namespace sg {

// Symbolic windows hold only a presence bitmap, so they are wide.
constexpr int SYM_WARP_W = 32768;    // 4 KB of bits per warp
constexpr int SYM_BLOCK_W = 262144;  // 32 KB of bits per block
constexpr int SYM_BLOCK_WARPS = 16;

static long long rows_in(const int* path_rows, int p) { return path_rows ? path_rows[p] : -1; }

cudaError_t launch_symbolic(const LaunchCtx& c, const Csr& A, const Csr& B, const RowInfo& ri,
                            const PathBins& pb, const Tuning& tu, int32_t* cursor, int32_t* c_cnt,
                            const int* path_rows) {
  (void)tu;
  const double* nv = nullptr;
  double* nvo = nullptr;
  // register-sort path: bins 1..4 -> 8 lanes, 5 -> 16 lanes, 6 -> 32 lanes
  if (pb.hi[PATH_TINY] >= pb.lo[PATH_TINY]) {
    timer_mark(c, T_SYM_TINY, 0);
    const int lo = pb.lo[PATH_TINY], hi = pb.hi[PATH_TINY];
    const int ranges[3][2] = {{lo, hi < 4 ? hi : 4}, {5 > lo ? 5 : lo, hi < 5 ? hi : 5}, {6 > lo ? 6 : lo, hi}};
    for (int t = 0; t < 3; ++t) {
      if (ranges[t][1] < ranges[t][0]) continue;
      const int G = 8 << t;
      int occ = 0;
      int grid;
      if (G == 8) {
        occ = kernel_blocks_per_sm(k_tiny<8, false, double>, 256, 0);
        grid = persistent_grid(rows_in(path_rows, PATH_TINY), 8 * 4, c.nsm, occ);
        k_tiny<8, false, double><<<grid, 256, 0, c.stream>>>(A, B, nv, nv, ri, c.st, ranges[t][0], ranges[t][1], c_cnt, nullptr, nullptr, nvo, c.err);
      } else if (G == 16) {
        occ = kernel_blocks_per_sm(k_tiny<16, false, double>, 256, 0);
        grid = persistent_grid(rows_in(path_rows, PATH_TINY), 8 * 2, c.nsm, occ);
        k_tiny<16, false, double><<<grid, 256, 0, c.stream>>>(A, B, nv, nv, ri, c.st, ranges[t][0], ranges[t][1], c_cnt, nullptr, nullptr, nvo, c.err);
      } else {
        occ = kernel_blocks_per_sm(k_tiny<32, false, double>, 256, 0);
        grid = persistent_grid(rows_in(path_rows, PATH_TINY), 8, c.nsm, occ);
        k_tiny<32, false, double><<<grid, 256, 0, c.stream>>>(A, B, nv, nv, ri, c.st, ranges[t][0], ranges[t][1], c_cnt, nullptr, nullptr, nvo, c.err);
      }
      count_launch(c);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    timer_mark(c, T_SYM_TINY, 1);
  }
  if (pb.hi[PATH_WARP] >= pb.lo[PATH_WARP]) {
    timer_mark(c, T_SYM_WARP, 0);
    auto k = k_window<1, 8, SYM_WARP_W, false, double>;
    const size_t smem = 8 * window_group_bytes<SYM_WARP_W, false, double>(1);
    const int occ = kernel_blocks_per_sm(k, 256, smem);
    if (occ <= 0) return cudaErrorInvalidConfiguration;
    const int grid = persistent_grid(rows_in(path_rows, PATH_WARP), 8, c.nsm, occ);
    k<<<grid, 256, smem, c.stream>>>(A, B, nv, nv, ri, c.st, pb.lo[PATH_WARP], pb.hi[PATH_WARP], cursor, c_cnt, nullptr, nullptr, nvo, c.err);
    count_launch(c);
    timer_mark(c, T_SYM_WARP, 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (pb.hi[PATH_BLOCK] >= pb.lo[PATH_BLOCK]) {
    timer_mark(c, T_SYM_BLOCK, 0);
    auto k = k_window<SYM_BLOCK_WARPS, SYM_BLOCK_WARPS, SYM_BLOCK_W, false, double>;
    const size_t smem = window_group_bytes<SYM_BLOCK_W, false, double>(SYM_BLOCK_WARPS);
    const int occ = kernel_blocks_per_sm(k, SYM_BLOCK_WARPS * 32, smem);
    if (occ <= 0) return cudaErrorInvalidConfiguration;
    const int grid = persistent_grid(rows_in(path_rows, PATH_BLOCK), 1, c.nsm, occ);
    k<<<grid, SYM_BLOCK_WARPS * 32, smem, c.stream>>>(A, B, nv, nv, ri, c.st, pb.lo[PATH_BLOCK], pb.hi[PATH_BLOCK], cursor, c_cnt, nullptr, nullptr, nvo, c.err);
    count_launch(c);
    timer_mark(c, T_SYM_BLOCK, 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sg
