// Symbolic pass: the number of distinct columns of every row of C
// (Sec. 2.2: the union of the columns of the B rows a row of A touches).
#include "launch_util.cuh"
#include "rowhash.cuh"
#include "rowlane.cuh"
#include "rowpass.cuh"
#include "symblock.cuh"

namespace sg {

// Symbolic windows hold only a presence bitmap, so they are wide.
constexpr int SYM_WARP_W = 32768;    // 4 KB of bits per warp
constexpr int SYM_BLOCK_W = 262144;  // 32 KB of bits per block
constexpr int SYM_BLOCK_WARPS = 8;

static long long rows_in(const int* path_rows, int p) { return path_rows ? path_rows[p] : -1; }

template <int G, int E>
static cudaError_t tiny_sym(const LaunchCtx& c, const Csr& A, const Csr& B, const RowInfo& ri, int lo, int hi,
                            int32_t* c_cnt, long long rows) {
  const double* nv = nullptr;
  double* nvo = nullptr;
  auto k = k_tiny<G, E, false, double>;
  const int occ = kernel_blocks_per_sm(k, 256, 0);
  const int grid = persistent_grid(rows, 8 * (32 / G), c.nsm, occ);
  k<<<grid, 256, 0, c.stream>>>(A, B, nv, nv, ri, c.st, lo, hi, c_cnt, nullptr, nullptr, nvo, c.err);
  count_launch(c);
  return cudaGetLastError();
}

// Register-sort bins: 1..4 -> 8 lanes, 5 -> 16 lanes, 6 -> 32 lanes,
// 7 -> 32 lanes x 2 slots, 8 -> x 4, 9 -> x 8, 10 -> x 16 slots (P <= 512).
template <typename F8, typename F16, typename F32, typename F64, typename F128, typename F256, typename F512>
static cudaError_t tiny_dispatch(int lo, int hi, F8 f8, F16 f16, F32 f32, F64 f64, F128 f128, F256 f256,
                                 F512 f512) {
  cudaError_t e = cudaSuccess;
  auto clip = [&](int a, int b, auto f) -> cudaError_t {
    const int l = lo > a ? lo : a, h = hi < b ? hi : b;
    return l <= h ? f(l, h) : cudaSuccess;
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

template <int E>
static cudaError_t hash_sym(const LaunchCtx& c, const Csr& A, const Csr& B, const RowInfo& ri, int lo, int hi,
                            int32_t* c_cnt, long long rows) {
  auto k = k_hash_sym<E>;
  const int occ = kernel_blocks_per_sm(k, HASH_WARPS * 32, 0);
  const int grid = persistent_grid(rows, HASH_WARPS, c.nsm, occ);
  k<<<grid, HASH_WARPS * 32, 0, c.stream>>>(A, B, ri, c.st, lo, hi, c_cnt, c.err);
  count_launch(c);
  return cudaGetLastError();
}

// Hash bins: 6 -> 1 product per lane (P <= 32), 7 -> 2 (P <= 64), 8 -> 4 (P <= 128).
template <typename F1, typename F2, typename F4>
static cudaError_t hash_dispatch(int lo, int hi, F1 f1, F2 f2, F4 f4) {
  cudaError_t e = cudaSuccess;
  auto clip = [&](int a, int b, auto f) -> cudaError_t {
    const int l = lo > a ? lo : a, h = hi < b ? hi : b;
    return l <= h ? f(l, h) : cudaSuccess;
  };
  if ((e = clip(1, 6, f1))) return e;
  if ((e = clip(7, 7, f2))) return e;
  if ((e = clip(8, 8, f4))) return e;
  return cudaSuccess;
}

template <int GW, int CW, int W>
static cudaError_t window_sym(const LaunchCtx& c, const Csr& A, const Csr& B, const RowInfo& ri, int lo, int hi,
                              const SplitInfo& sp, int32_t* cursor, int32_t* c_cnt, long long rows) {
  auto k = k_sym_window<GW, CW, W>;
  const size_t smem = (size_t)(CW / GW) * sym_group_bytes<W, GW>();
  const int occ = kernel_blocks_per_sm(k, CW * 32, smem);
  if (occ <= 0) return cudaErrorInvalidConfiguration;
  const int grid = persistent_grid(rows, CW / GW, c.nsm, occ);
  k<<<grid, CW * 32, smem, c.stream>>>(A, B, ri, c.st, lo, hi, sp, cursor, c_cnt, c.err);
  count_launch(c);
  return cudaGetLastError();
}

template <int W, int NW>
static cudaError_t block_sym(const LaunchCtx& c, const Csr& A, const Csr& B, const RowInfo& ri, int lo, int hi,
                             const SplitInfo& sp, int32_t* cursor, int32_t* c_cnt) {
  auto k = k_sym_block<W, NW>;
  const size_t smem = symblock_smem_bytes<W, NW>();
  const int occ = kernel_blocks_per_sm(k, NW * 32, smem);
  if (occ <= 0) return cudaErrorInvalidConfiguration;
  unsigned* counter = &c.st->work[2];
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), c.stream);
  if (e != cudaSuccess) return e;
  k<<<c.nsm * occ, NW * 32, smem, c.stream>>>(A, B, ri, c.st, lo, hi, sp, cursor, c_cnt, counter, c.err);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_symbolic(const LaunchCtx& c, const Csr& A, const Csr& B, const RowInfo& ri,
                            const PathBins& pb, const Tuning& tu, const SplitInfo& sp, int32_t* cursor,
                            int32_t* c_cnt, const int* path_rows) {
  (void)tu;
  cudaError_t e = cudaSuccess;
  if (pb.hi[PATH_TINY] >= pb.lo[PATH_TINY]) {
    timer_mark(c, T_SYM_TINY, 0);
    const long long rows = rows_in(path_rows, PATH_TINY);
    e = tiny_dispatch(pb.lo[PATH_TINY], pb.hi[PATH_TINY],
        [&](int l, int h) { return tiny_sym<8, 1>(c, A, B, ri, l, h, c_cnt, rows); },
        [&](int l, int h) { return tiny_sym<16, 1>(c, A, B, ri, l, h, c_cnt, rows); },
        [&](int l, int h) { return tiny_sym<32, 1>(c, A, B, ri, l, h, c_cnt, rows); },
        [&](int l, int h) { return tiny_sym<32, 2>(c, A, B, ri, l, h, c_cnt, rows); },
        [&](int l, int h) { return tiny_sym<32, 4>(c, A, B, ri, l, h, c_cnt, rows); },
        [&](int l, int h) { return tiny_sym<32, 8>(c, A, B, ri, l, h, c_cnt, rows); },
        [&](int l, int h) { return tiny_sym<32, 16>(c, A, B, ri, l, h, c_cnt, rows); });
    timer_mark(c, T_SYM_TINY, 1);
    if (e) return e;
  }
  if (pb.hi[PATH_HASH] >= pb.lo[PATH_HASH]) {
    timer_mark(c, T_SYM_HASH, 0);
    const long long rows = rows_in(path_rows, PATH_HASH);
    // rows of at most 64 products: one lane per row; 65..128: a warp per row
    const int llo = pb.lo[PATH_HASH], lhi = pb.hi[PATH_HASH] < 7 ? pb.hi[PATH_HASH] : 7;
    if (llo <= lhi)
      e = lane_rows<false, double>(c, A, B, nullptr, nullptr, ri, llo, lhi, c_cnt, nullptr, nullptr, nullptr, rows);
    if (!e && pb.hi[PATH_HASH] >= 8)
      e = hash_dispatch(8, pb.hi[PATH_HASH],
          [&](int l, int h) { return hash_sym<1>(c, A, B, ri, l, h, c_cnt, rows); },
          [&](int l, int h) { return hash_sym<2>(c, A, B, ri, l, h, c_cnt, rows); },
          [&](int l, int h) { return hash_sym<4>(c, A, B, ri, l, h, c_cnt, rows); });
    timer_mark(c, T_SYM_HASH, 1);
    if (e) return e;
  }
  if (pb.hi[PATH_WARP] >= pb.lo[PATH_WARP]) {
    timer_mark(c, T_SYM_WARP, 0);
    e = window_sym<1, 8, SYM_WARP_W>(c, A, B, ri, pb.lo[PATH_WARP], pb.hi[PATH_WARP], sp, cursor, c_cnt,
                                      rows_in(path_rows, PATH_WARP));
    timer_mark(c, T_SYM_WARP, 1);
    if (e) return e;
  }
  if (pb.hi[PATH_BLOCK] >= pb.lo[PATH_BLOCK]) {
    timer_mark(c, T_SYM_BLOCK, 0);
    e = block_sym<SYM_BLOCK_W, SYM_BLOCK_WARPS>(c, A, B, ri, pb.lo[PATH_BLOCK], pb.hi[PATH_BLOCK], sp, cursor, c_cnt);
    timer_mark(c, T_SYM_BLOCK, 1);
    if (e) return e;
  }
  return cudaSuccess;
}

}  // namespace sg
