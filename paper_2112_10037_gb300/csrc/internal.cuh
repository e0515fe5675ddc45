// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (include/spgemm.h is).
#pragma once

#include <cuda_runtime.h>
#include <climits>
#include <cstddef>
#include <cstdint>

#include "spgemm.h"  // include/ is on the include path (see build.py)

namespace sg {

// Rows are binned by their product count P (Sec. 2.2: the number of
// scalar-times-row products that build row i; Table 1's B_NUM_VEC summed
// over the row).  bin 0 holds P = 0; bin b >= 1 holds P in (2^(b-2), 2^(b-1)],
// i.e. bin 1: P = 1, bin 2: P = 2, bin 3: P in [3,4], ... ; the last bin takes
// everything larger.
constexpr int NBINS = 48;

__host__ __device__ inline int bin_of(long long p) {
  if (p <= 0) return 0;
  int b;
#ifdef __CUDA_ARCH__
  b = (p == 1) ? 1 : (64 - __clzll(p - 1)) + 1;
#else
  b = (p == 1) ? 1 : (64 - __builtin_clzll((unsigned long long)(p - 1))) + 1;
#endif
  return b < NBINS ? b : NBINS - 1;
}

// Error bits of the device error word.
enum : uint32_t {
  EB_UNSORTED = 1u,   // column index out of range / not ascending / row_ptr broken
  EB_OVERFLOW = 2u,   // nnz(C) >= 2^31
  EB_TABLE = 4u,      // a bounded probe or loop gave up
  EB_INTERNAL = 8u,   // symbolic and numeric disagree, or an output bound was hit
};

// Small device-resident statistics block at the start of the workspace.
struct DevStats {
  unsigned long long total_products;
  unsigned long long max_products;
  long long nnz_c;
  long long nruns;   // entries of B's window-run list
  long long nruns_b;  // entries of its block-window-granular copy
  long long scratch_total;  // total of the transpose's prefix sum
  uint32_t err;
  uint32_t rows_wide;  // rows of the plan with more than 32 nonzeros of A
  int hist[NBINS];   // rows per bin
  int fill[NBINS];   // scatter cursors
  unsigned int work[8];  // dynamic work counters (reset before each use)
};

// Paths a non-empty row can take.
enum Path : int { PATH_TINY = 0, PATH_HASH = 1, PATH_WARP = 2, PATH_BLOCK = 3, NPATHS = 4 };

struct Csr {
  const int32_t* rp;
  const int32_t* ci;
  long long nrows;
  long long ncols;
  long long nnz;
};

// Per-row analysis arrays (all of length mloc, indexed by the local row r).
struct RowInfo {
  long long row_begin;   // global row of A = row_begin + r
  long long mloc;
  const long long* prod; // products per row
  const int* cmin;       // smallest column any product reaches
  const int* cmax;       // largest column any product reaches
  const int* rows;       // local rows ordered by descending bin
};

// Bin ranges of each path, computed on the host from the options.
struct PathBins {
  int lo[NPATHS];
  int hi[NPATHS];  // inclusive; hi < lo means the path is unused
};

// Tuning of the paths, fixed when the plan is made.
struct Tuning {
  int window_warp;     // numeric window width (columns) of the warp accumulator
  int window_block;    // numeric window width (columns) of the block accumulator
  int hash_max;        // largest P of the hash path (0: path disabled)
  int warp_max;        // largest P of the symbolic warp path
  int num_lo_block;    // numeric bins >= this use the block kernel (NBINS: never)
  int num_lo_rank;     // numeric bins >= this (below num_lo_block) use the rank kernel (NBINS: never)
  int rank_accum;      // 0: rank kernel values reduced in global memory; 1: in shared-memory chunks
  int block_warps;     // warps per numeric block window
};

// Window-run list of B: the numeric pass uses windows of 2^wf_shift columns
// aligned to multiples of their width.  Each row k of B is cut into runs of
// consecutive entries that fall in the same window; run j of the list holds
// (window id, first position in B), rows own runs [rr[k], rr[k+1]), and the
// last run of each row is a sentinel (INT_MAX, end of row) so run j covers
// positions [start_j, start_{j+1}).
//
// Splitting of heavy rows into window tiles (numeric pass): heavy rows are
// the leading rows of the descending-bin list whose bin is >= heavy_bin, at
// most hcap of them; row h of the list owns hcnt[h * ntf .. h * ntf + ntf).
struct SplitInfo {
  int heavy_bin;      // NBINS disables splitting
  int hi_bin;         // split rows are the rows of bins [heavy_bin, hi_bin]
  int hcap;
  int wf_shift;       // log2 of the window (= fine tile) width
  int ntf;            // windows per row: ceil(ncols(B) / width)
  int32_t* rr;        // nrows(B) + 1 run pointers
  int2* runs;         // (window id, start) per run, sentinel-terminated rows
  int32_t* hcnt;      // hcap x ntf output counts
  // the same run list at the numeric block window's granularity (log2 of its
  // width in wb_shift); null when the plan has no block window
  int wb_shift;
  int32_t* rrb;
  int2* runsb;
};

// Entries allocated past the last run, so that a kernel may read the few
// runs after a row's current one in parallel without a bounds check (it
// stops at the row's sentinel; what lies beyond is never used).
constexpr int RUNS_PAD = 4;

// ---------------------------------------------------------------- warp utils
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename V>
__device__ __forceinline__ V warp_incl_scan(V v) {
  const int lane = lane_id();
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    V t = __shfl_up_sync(FULL, v, d);
    if (lane >= d) v += t;
  }
  return v;
}

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
  return v;
}

// 32-bit integer reductions are single warp instructions (redux.sync).
__device__ __forceinline__ int warp_sum(int v) { return __reduce_add_sync(FULL, v); }
__device__ __forceinline__ unsigned warp_sum(unsigned v) { return __reduce_add_sync(FULL, v); }
__device__ __forceinline__ int warp_min(int v) { return __reduce_min_sync(FULL, v); }
__device__ __forceinline__ int warp_max(int v) { return __reduce_max_sync(FULL, v); }

// acc += v on a shared-memory word, result unused (a reduction, not a fetch).
__device__ __forceinline__ void red_add_shared(double* p, double v) {
  asm volatile("red.shared.add.f64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "d"(v) : "memory");
}
__device__ __forceinline__ void red_add_shared(float* p, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "f"(v) : "memory");
}

// acc += a * b on a shared-memory word, for FP64 as one fused multiply-add
// under a compare-and-swap: GB300 runs FP64 at two lane-operations per SM per
// clock, and a multiply followed by a shared-memory FP64 add costs two of
// them; the swap itself runs on the shared-memory unit.  Equal addresses,
// in one warp or in several, retry with the value that won.  Returns whether
// the word still held +0.0, the cleared state, before this update: the first
// update of a column sees it, so the caller marks the column present then
// and skips the bitmap atomic on every later update.  FP32 adds in hardware
// (red.shared.add.f32) and always reports a first update.
constexpr int CAS_RETRY_LIMIT = 1 << 16;

__device__ __forceinline__ bool is_cleared(double v) { return __double_as_longlong(v) == 0ll; }
__device__ __forceinline__ bool is_cleared(float v) { return __float_as_uint(v) == 0u; }

__device__ __forceinline__ bool fma_shared(double* p, double a, double b, uint32_t* err) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  unsigned long long old;
  asm volatile("ld.shared.u64 %0, [%1];" : "=l"(old) : "r"(s) : "memory");
  for (int it = 0; it < CAS_RETRY_LIMIT; ++it) {
    const unsigned long long nv = (unsigned long long)__double_as_longlong(fma(a, b, __longlong_as_double((long long)old)));
    unsigned long long prev;
    asm volatile("atom.shared.cas.b64 %0, [%1], %2, %3;" : "=l"(prev) : "r"(s), "l"(old), "l"(nv) : "memory");
    if (prev == old) return old == 0ull;
    old = prev;
  }
  atomicOr(err, EB_INTERNAL);  // never expected: each failed swap is another update's success
  return false;
}
__device__ __forceinline__ bool fma_shared(float* p, float a, float b, uint32_t*) {
  red_add_shared(p, a * b);
  return true;
}

// Index of the first lane whose inclusive prefix `incl` exceeds p (incl is
// non-decreasing over the 32 lanes).  Every lane must call it.
__device__ __forceinline__ int warp_owner(int incl, int p) {
  int lo = 0;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    int t = __shfl_sync(FULL, incl, lo + s - 1);
    if (t <= p) lo += s;
  }
  return lo;
}

// Block-uniform check of the error word (one read by thread 0, shared with
// the block through a barrier), so a block never splits around a barrier.
// Kernels call it first and return when the input was rejected.
__device__ __forceinline__ bool block_skip(const DevStats* st) {
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = (*(volatile const uint32_t*)&st->err & EB_UNSORTED) != 0;
  __syncthreads();
  return s_skip != 0;
}

// [begin, end) of the rows of bins [lo, hi] inside the descending-bin list.
__device__ __forceinline__ void bin_range(const DevStats* st, int lo, int hi, int* begin, int* end) {
  int b = 0, e = 0;
  for (int k = NBINS - 1; k >= 1; --k) {
    int h = st->hist[k];
    if (k > hi) b += h;
    else if (k >= lo) e += h;
  }
  *begin = b;
  *end = b + e;
}

// ------------------------------------------------------------ host launchers
struct LaunchCtx {
  cudaStream_t stream;
  int nsm;
  DevStats* st;
  uint32_t* err;
  cudaEvent_t* timers;   // 2 events per timer group, or null (profiling off)
  int* timer_used;       // set to 1 for each group recorded by this call
  long long* launches;   // kernel launch counter (host)
};

// Timer groups (the order of spgemm_plan_kernel_times).
enum Timer : int {
  T_ANALYSE = 0, T_SYM_TINY = 1, T_SYM_HASH = 2, T_SYM_WARP = 3, T_SYM_BLOCK = 4, T_SCAN = 5,
  T_NUM_TINY = 6, T_NUM_HASH = 7, T_NUM_WARP = 8, T_NUM_BLOCK = 9, T_NUM_RANK = 10, NTIMERS = 11
};

inline void timer_mark(const LaunchCtx& c, int t, int end) {
  if (c.timers) {
    cudaEventRecord(c.timers[2 * t + end], c.stream);
    if (c.timer_used) c.timer_used[t] = 1;
  }
}

inline void count_launch(const LaunchCtx& c) {
  if (c.launches) ++*c.launches;
}

cudaError_t launch_validate(const LaunchCtx& c, const Csr& M);
cudaError_t launch_analyse(const LaunchCtx& c, const Csr& A, const Csr& B, long long row_begin,
                           long long mloc, long long* prod, int* cmin, int* cmax, int* rows);
// win_lo > 0: skip building the lists when the analysis put no row in bins
// win_lo and above (only valid when no other plan reads this plan's lists
// for rows outside it).
cudaError_t launch_runs(const LaunchCtx& c, const Csr& B, const SplitInfo& sp, long long* partials, int win_lo);
cudaError_t launch_symbolic(const LaunchCtx& c, const Csr& A, const Csr& B, const RowInfo& ri,
                            const PathBins& pb, const Tuning& tu, const SplitInfo& sp, int32_t* cursor,
                            int32_t* c_rp, const int* path_rows /* host, may be null */);
cudaError_t launch_scan(const LaunchCtx& c, int32_t* c_rp, long long mloc, long long* partials,
                        long long* total_out = nullptr);
size_t scan_partials_count(long long mloc);
cudaError_t launch_numeric(const LaunchCtx& c, const Csr& A, const Csr& B, const RowInfo& ri,
                           const PathBins& pb, const Tuning& tu, const SplitInfo& sp, int dtype,
                           const void* av, const void* bv, int32_t* cursor, int32_t* nxt,
                           const int32_t* c_rp, int32_t* c_ci, void* c_v,
                           const int* path_rows /* host, may be null */,
                           long long rows_wide /* rows with more than 32 nonzeros, -1: unknown */,
                           const int* hist /* host rows per bin, may be null: bins without rows
                                              are not launched */,
                           int semiring /* spgemm_semiring_kind */);
// The numeric pass over the min-plus, max-plus and or-and semirings.
#define SG_NUMERIC_SR_DECL(NAME)                                                                              \
  cudaError_t NAME(const LaunchCtx& c, const Csr& A, const Csr& B, const RowInfo& ri, const PathBins& pb,     \
                   const Tuning& tu, const SplitInfo& sp, int dtype, const void* av, const void* bv,          \
                   int32_t* cur, int32_t* nxt, const int32_t* c_rp, int32_t* c_ci, void* c_v,                 \
                   const int* path_rows, long long rows_wide, const int* hist)
SG_NUMERIC_SR_DECL(launch_numeric_min_plus);
SG_NUMERIC_SR_DECL(launch_numeric_max_plus);
SG_NUMERIC_SR_DECL(launch_numeric_or_and);

// Scratch of a transpose of a matrix with n columns and nnz entries whose
// values have vbytes bytes (0: structure only): tmp (int32), the digit table
// (int32) and the scan partials (int64).
struct TransposeScratch {
  size_t tmp_ints, table_ints, part_count;
};
TransposeScratch transpose_scratch(long long n, long long nnz, int vbytes);
// M^T: t_rp (n+1), t_ci and t_src (nnz, required), and with vbytes 4 or 8
// and both value pointers, t_vals[q] = vals[t_src[q]].
cudaError_t launch_transpose(const LaunchCtx& c, long long m, long long n, long long nnz, const int32_t* rp,
                             const int32_t* ci, int32_t* t_rp, int32_t* t_ci, int32_t* t_src, int vbytes,
                             const void* vals, void* t_vals, int32_t* tmp, int32_t* table, long long* partials);
// Masked product on M's pattern over a semiring (spgemm_semiring; 0 is
// C<M> = (A*B) .* M, mv null for the pattern only; mv is unused otherwise).
cudaError_t launch_masked(const LaunchCtx& c, int dtype, int semiring, const Csr& A, const Csr& B, const Csr& M,
                          const void* av, const void* bv, const void* mv, void* out);
// out[q] = row of entry q of a CSR with row pointer rp (nrows rows).
cudaError_t launch_row_index(const LaunchCtx& c, const int32_t* rp, long long nrows, int32_t* out);
cudaError_t launch_backward(const LaunchCtx& c, int dtype, const Csr& A, const Csr& B, long long row_begin,
                            long long mloc, const void* av, const void* bv, const int32_t* a_row,
                            const int32_t* b_row, const int32_t* t_rp, const int32_t* t_ci, const int32_t* t_src,
                            const int32_t* c_rp, const int32_t* c_ci, const void* dc, void* da, void* db);

// One instance of a batched product (see batch.cu).
struct BatchDesc {
  const int32_t* a_rp;
  const int32_t* a_ci;
  const void* a_v;
  const int32_t* b_rp;
  const int32_t* b_ci;
  const void* b_v;
  long long m, k, n;     // A_i is m x k, B_i is k x n
  long long a_nnz, b_nnz;
  long long roff, koff, noff, aoff, boff;  // offsets in the stacked arrays
};
cudaError_t launch_stack_structure(const LaunchCtx& c, int n, const BatchDesc* d, long long total_rows,
                                   long long total_k, int32_t* a_rp, int32_t* a_ci, int32_t* b_rp, int32_t* b_ci,
                                   long long total_a_nnz, long long total_b_nnz);
cudaError_t launch_stack_values(const LaunchCtx& c, int n, int dtype, const BatchDesc* d, void* a_v, void* b_v);
cudaError_t launch_unstack_columns(const LaunchCtx& c, int n, const BatchDesc* d, const int32_t* c_rp, int32_t* c_ci);
cudaError_t launch_batch_bounds(const LaunchCtx& c, int n, const BatchDesc* d, const int32_t* c_rp, long long total_rows,
                                int32_t* out);
cudaError_t launch_batch_products(const LaunchCtx& c, int n, const BatchDesc* d, long long* products);

// Split (heavy) rows: list positions [*hs, *hs + return value) -- the rows of
// bins [heavy_bin, hi_bin], at most hcap of them; split row h of both passes
// is list position *hs + h.
__device__ __forceinline__ int split_rows(const DevStats* st, const SplitInfo& sp, int* hs) {
  *hs = 0;
  if (sp.heavy_bin >= NBINS || sp.hi_bin < sp.heavy_bin) return 0;
  int he = 0;
  bin_range(st, sp.heavy_bin, sp.hi_bin, hs, &he);
  const int n = he - *hs;
  return n < sp.hcap ? n : sp.hcap;
}


}  // namespace sg
