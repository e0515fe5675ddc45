/*
 * spgemm.h -- C ABI of the GB300 (sm_103a) Gustavson SpGEMM library.
 *
 * C = A * B for sparse matrices in CSR form (Sec. 2.1: values, column
 * indices, row pointers), computed row by row with the row-wise Gustavson
 * method (Sec. 2.2): row i of C is the sum, over the nonzeros A(i,k), of the
 * scaled rows A(i,k) * B(k,:).  Adding sparse rows merges them by column and
 * adds the values of equal columns (Sec. 2.2, Algorithm 1), so every output
 * row holds each reached column once, in ascending order.  Entries whose
 * products cancel to 0.0 are kept: the pattern of C is structural.
 *
 * Conventions for every call below
 *   - Indices are int32.  Row pointers of inputs and of C are int32, so
 *     nnz(A), nnz(B), nnz(C) must each stay below 2^31; the number of
 *     products may exceed that (it is counted in int64).
 *   - Column indices of A and B must be ascending and unique within each
 *     row, and inside [0, ncols).  With opts.validate set the library checks
 *     this on the device and reports SPGEMM_ERR_UNSORTED_INPUT.
 *   - Every pointer to matrix data or workspace is a DEVICE pointer on the
 *     current CUDA device; c_nnz of spgemm_symbolic is a host pointer.
 *   - All matrix buffers and the workspace belong to the caller; the library
 *     never allocates device memory, never frees caller memory and never
 *     calls cudaDeviceSynchronize.  The plan is library-owned host memory.
 *   - Work is issued asynchronously on the given stream (a cudaStream_t;
 *     NULL is the legacy default stream).  Only spgemm_symbolic and
 *     spgemm_plan_check block, on that stream only.
 *   - Errors are returned as spgemm_status; nothing aborts and no C++
 *     exception crosses this boundary.  Faults detected on the device (bad
 *     input with validate, index overflow, an exhausted probe bound) are
 *     recorded in a device error word and reported by the next blocking call.
 */
#ifndef SPGEMM_GB300_H
#define SPGEMM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st* spgemm_stream_t;

typedef enum spgemm_status {
  SPGEMM_OK = 0,
  SPGEMM_ERR_INVALID_ARG = 1,     /* NULL pointer, negative size, bad option */
  SPGEMM_ERR_DIM_MISMATCH = 2,    /* A.ncols != B.nrows, or row range outside A */
  SPGEMM_ERR_UNSORTED_INPUT = 3,  /* a column index out of range, repeated or descending */
  SPGEMM_ERR_INDEX_OVERFLOW = 4,  /* nnz(C) (or an input nnz) does not fit int32 */
  SPGEMM_ERR_WORKSPACE = 5,       /* workspace NULL or smaller than spgemm_workspace_size */
  SPGEMM_ERR_TABLE_OVERFLOW = 6,  /* a shared-memory hash table found no free slot (the
                                     tables are sized at twice a row's products, so this
                                     means broken input or a library fault) */
  SPGEMM_ERR_CUDA = 7,            /* a CUDA runtime call failed */
  SPGEMM_ERR_INTERNAL = 8,
  SPGEMM_ERR_NOT_READY = 9        /* calls out of order (numeric before symbolic) */
} spgemm_status;

typedef enum spgemm_dtype { SPGEMM_F64 = 0, SPGEMM_F32 = 1 } spgemm_dtype;

/* A CSR matrix (Sec. 2.1).  row_ptr has nrows+1 entries with row_ptr[0] = 0
 * and row_ptr[nrows] = nnz; col_idx and vals have nnz entries.  vals may be
 * NULL where a call reads only the structure. */
typedef struct spgemm_csr {
  int64_t nrows;
  int64_t ncols;
  int64_t nnz;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const void* vals;
} spgemm_csr;

/* Tuning and behaviour.  Fill with spgemm_opts_default, then override. */
typedef struct spgemm_opts {
  int32_t dtype;       /* spgemm_dtype of A, B and C values */
  int32_t validate;    /* nonzero: check the column-index preconditions on the device */
  int64_t row_begin;   /* multiply rows [row_begin, row_end) of A only; C then has */
  int64_t row_end;     /*   row_end - row_begin rows.  row_end < 0 means A.nrows */
  int32_t warp_max;    /* rows with at most this many products use one warp per row;
                          more use a whole block (0: library default) */
  int32_t force_path;  /* -1: automatic.  Testing overrides: 1 (2) sends every row
                          above the register-sort limit to the warp (block) path;
                          3 (4) sends every non-empty row to the warp (block) path */
  int32_t hash_max;    /* rows of 17 .. hash_max products use the warp hash accumulator
                          (a shared-memory table of twice the row's products, ranked
                          into column order); 0: 128, otherwise rounded up to 32, 64 or
                          128; -1: off (register sort up to sort_max).  Off as well when
                          force_path >= 0 or sort_max is 256 or 512.  Rows of at most
                          16 products always use the register sort */
  int32_t window_warp; /* columns of the numeric dense window (one per warp):
                          1024, 2048 or 4096 (0: default 1024) */
  int32_t window_block;/* columns of the numeric block window, with block_warps one of
                          the pairs (2048, 4), (2048, 8), (4096, 4), (4096, 8),
                          (4096, 16), (8192, 8), (8192, 16), (16384, 16); 0 or any
                          other pair: (8192, 8) */
  int32_t split_min;   /* rows with more products than this are split into column
                          tiles of window_warp columns, processed independently
                          (0: default 131072; -1: never split); used only for rows
                          the block-window numeric kernel does not take */
  int32_t backward;    /* nonzero: the plan also keeps the transpose of A's structure,
                          which spgemm_backward needs (more workspace) */
  int32_t num_block_min;/* rows with more products than this run the numeric pass
                          with a block-wide window (0: default 65536; -1: never, then
                          heavy rows are split as split_min says) */
  int32_t block_warps; /* warps sharing a numeric block window (see window_block) */
  int32_t sort_max;    /* rows of at most this many products are merged by a sort in
                          registers: 128, 256 or 512 (0: 128); rows of 17 or more
                          products take the hash path instead unless it is off
                          (see hash_max) */
  int32_t rank_min;    /* > 0: rows with more products than this (and not above
                          num_block_min) run the numeric pass with the rank-compacted
                          accumulator: a presence bitmap over up to 2^18 columns gives
                          each output column its position in the row, and values
                          accumulate in an array of the row's outputs.  0 or -1: off
                          (the default), those rows use the warp window.  Off as well
                          with force_path >= 0 or when heavy rows are split (split_min) */
  int32_t rank_accum;  /* where the rank-compacted accumulator sums its values: 0 (default)
                          in C itself, zeroed first, by reductions in the L2 cache's atomic
                          units; 1 in shared memory, 6144 ranks per pass over the row's
                          products */
  int32_t semiring;    /* sum and product of the numeric pass (spgemm_semiring_kind below):
                          SPGEMM_PLUS_TIMES (0, the default) or min-plus, max-plus, or-and,
                          each row of C then the semiring sum over A(i,k) of the products
                          A(i,k) (x) B(k,:) on the same pattern (Sec. 2.2 with + and *
                          replaced; min, max and or do not depend on the order of the sums,
                          so those values are exact).  With another semiring sort_max,
                          rank_min, split_min, window_warp, window_block and block_warps
                          are ignored (defaults; no rank-compacted accumulator, no split
                          rows), and backward must be 0 */
} spgemm_opts;

typedef struct spgemm_plan spgemm_plan;

/* Fills *o with defaults: F64, no validation, all rows, automatic paths. */
void spgemm_opts_default(spgemm_opts* o);

/* Text for a status code (static storage). */
const char* spgemm_status_string(spgemm_status s);

/* Library version string, e.g. "0.1.0". */
const char* spgemm_version(void);

/* Bytes of device workspace a plan for this A, B and options needs.  Host
 * only, no device work.  The size depends on A.nrows (or the row range) and
 * A.nnz, not on the values. */
spgemm_status spgemm_workspace_size(const spgemm_csr* A, const spgemm_csr* B,
                                    const spgemm_opts* opts, size_t* bytes);

/* Structure analysis of C = A*B (Sec. 2.2; the per-row product count is the
 * row sum of the per-nonzero B_NUM_VEC of Table 1).  Checks shapes on the
 * host, then issues on `stream`: per-row product counts and column spans,
 * the binning of rows by product count, and (with validate) the index
 * checks.  Creates *plan, which keeps the pointers of A's and B's structure
 * and of the workspace: they must stay valid and unchanged until
 * spgemm_plan_destroy.  Does not block. */
spgemm_status spgemm_analyse(const spgemm_csr* A, const spgemm_csr* B,
                             const spgemm_opts* opts, void* workspace,
                             size_t workspace_bytes, spgemm_stream_t stream,
                             spgemm_plan** plan);

/* Row-range plans sharing one preprocessing of B.  Rows of C are independent
 * (Sec. 2.2: row i of C depends only on row i of A), so C can be produced in
 * row ranges, for example to copy one range to the host while the next is
 * computed.  spgemm_analyse_rows creates a plan for rows [row_begin, row_end)
 * of base's product (C then has row_end - row_begin rows) that reads base's
 * window-run lists of B instead of building its own; its options are base's
 * (validate and backward off).  base must have been analysed on `stream`
 * (or work ordered before it) and must outlive the new plan; A, B and base's
 * workspace must stay unchanged.  spgemm_rows_workspace_size gives the
 * workspace the new plan needs.  SPGEMM_ERR_DIM_MISMATCH for a range outside
 * [0, nrows(A)].  Does not block. */
spgemm_status spgemm_rows_workspace_size(const spgemm_plan* base, int64_t row_begin,
                                         int64_t row_end, size_t* bytes);
spgemm_status spgemm_analyse_rows(const spgemm_plan* base, int64_t row_begin, int64_t row_end,
                                  void* workspace, size_t workspace_bytes,
                                  spgemm_stream_t stream, spgemm_plan** plan);

/* Sizes a plan without its symbolic pass, from row sizes computed elsewhere
 * (for a row-range plan: the whole product's symbolic pass).  The c_row_ptr
 * later given to spgemm_numeric must then hold, for each of the plan's rows,
 * the offset of the row's first entry in the caller's c_col_idx / c_vals
 * (for example a slice of the whole product's row pointer, so that ranges are
 * written in place), and nnz is the number of entries of the plan's rows.
 * Rows whose sizes disagree with their products are written only inside
 * their given extent and reported as SPGEMM_ERR_INTERNAL.  Plans with split
 * rows (split_min) need the symbolic pass: SPGEMM_ERR_NOT_READY.  BLOCKS on
 * `stream` to read the analysis results. */
spgemm_status spgemm_plan_adopt_row_ptr(spgemm_plan* plan, int64_t nnz, spgemm_stream_t stream);

/* Symbolic pass: sizes every row of C (the number of distinct columns the
 * row's products reach, Sec. 2.2) and writes C's row pointer to c_row_ptr
 * (device, int32, nrows(C)+1 entries) by an exclusive prefix sum.  BLOCKS on
 * `stream` to return nnz(C) in *c_nnz (host) and to report any device error
 * recorded so far.  SPGEMM_ERR_INDEX_OVERFLOW if nnz(C) >= 2^31. */
spgemm_status spgemm_symbolic(spgemm_plan* plan, int32_t* c_row_ptr, int64_t* c_nnz,
                              spgemm_stream_t stream);

/* Numeric pass: C's column indices (ascending in each row) and values, for
 * the values a_vals / b_vals (device, plan dtype, aligned with A's and B's
 * col_idx).  c_row_ptr is the array spgemm_symbolic wrote; c_col_idx and
 * c_vals have nnz(C) entries.  Repeatable with new values of the same
 * structure.  Does not block and allocates nothing, so it may be captured
 * in a CUDA graph. */
spgemm_status spgemm_numeric(spgemm_plan* plan, const void* a_vals, const void* b_vals,
                             const int32_t* c_row_ptr, int32_t* c_col_idx, void* c_vals,
                             spgemm_stream_t stream);

/* Work statistics of an analysed plan (blocks on `stream` to read them):
 * total and largest per-row product count, and the number of rows sent to
 * the register-sort, hash, warp and block paths of
 * the symbolic pass.  Any output may be NULL. */
spgemm_status spgemm_plan_stats(spgemm_plan* plan, spgemm_stream_t stream,
                                int64_t* total_products, int64_t* max_row_products,
                                int64_t* rows_per_path /* 4 entries */);

/* Per-kernel timing for measurement.  With on != 0 the plan records a pair of
 * CUDA events (on the launching stream) around each group of kernels it
 * issues; spgemm_plan_kernel_times then blocks on the last recorded event
 * and returns the elapsed milliseconds of the most recent call of each group
 * in ms[0..n-1], in this order: analyse, symbolic register-sort, symbolic
 * hash, symbolic warp, symbolic block, scan, numeric register-sort, numeric
 * hash, numeric warp, numeric block (SPGEMM_TIMER_COUNT entries; groups
 * the plan never ran read as 0), and numeric rank (the rank-compacted
 * accumulator, opts.rank_min).  Creating the events is the only resource
 * this allocates (host-side event handles). */
#define SPGEMM_TIMER_COUNT 11
spgemm_status spgemm_plan_set_profiling(spgemm_plan* plan, int on);
spgemm_status spgemm_plan_kernel_times(spgemm_plan* plan, float* ms, int n);

/* Number of kernel launches this plan has issued since it was created. */
spgemm_status spgemm_plan_launches(spgemm_plan* plan, int64_t* launches);

/* Blocks on `stream` and returns the device error word as a status. */
spgemm_status spgemm_plan_check(spgemm_plan* plan, spgemm_stream_t stream);

/* Adjoint of C = A*B for a scalar loss with gradient dC on C's pattern
 * (for L = sum W .* C, dC = W):
 *   dA(i,k) = sum_j dC(i,j) * B(k,j)  on pattern(A)   -- (dC * B^T) sampled on A
 *   dB(k,j) = sum_i A(i,k) * dC(i,j)  on pattern(B)   -- (A^T * dC) sampled on B
 * The plan must have been made with opts.backward set and spgemm_symbolic
 * called; c_row_ptr / c_col_idx are C's structure from this plan, dc_vals
 * its gradient values (plan dtype).  da_vals (aligned with A's col_idx, all
 * of A's nonzeros; entries of rows outside the plan's row range are left
 * untouched) and db_vals (aligned with B's col_idx; sums over the plan's
 * rows only) are overwritten; either may be NULL to skip it.  Each output is
 * summed in a fixed order -- one fused multiply-add chain when it has at most
 * 128 terms, otherwise 32 lane chains added by a fixed shuffle tree -- so the
 * result is deterministic (the same bits on every call).
 * Does not block, allocates nothing. */
spgemm_status spgemm_backward(spgemm_plan* plan, const void* a_vals, const void* b_vals,
                              const int32_t* c_row_ptr, const int32_t* c_col_idx,
                              const void* dc_vals, void* da_vals, void* db_vals,
                              spgemm_stream_t stream);

/* Device workspace bytes for spgemm_transpose of an nrows x ncols matrix
 * with nnz entries (host only). */
spgemm_status spgemm_transpose_workspace_size(int64_t nrows, int64_t ncols, int64_t nnz, size_t* bytes);

/* M^T in CSR (Sec. 2.1: M's CSC form): t_row_ptr (ncols+1 entries),
 * t_col_idx (nnz; each row ascending), t_vals (nnz values of `dtype`, or NULL
 * for structure only), t_src (nnz source positions in M, or NULL), so that
 * t_vals[q] = M.vals[t_src[q]].  Column indices of M must be in range; the
 * transpose does not rely on their order within a row (it is a stable sort
 * of M's entries by column, so every row of M^T is ascending by source row;
 * a column repeated in a row of M gives that source row twice, adjacent).
 * Does not block; spgemm_transpose_check reads the error word:
 * SPGEMM_ERR_UNSORTED_INPUT for a column index out of range. */
spgemm_status spgemm_transpose(const spgemm_csr* M, int32_t dtype, int32_t* t_row_ptr, int32_t* t_col_idx,
                               void* t_vals, int32_t* t_src, void* workspace, size_t workspace_bytes,
                               spgemm_stream_t stream);

/* Blocks on `stream` and reports an error recorded by spgemm_transpose in
 * this workspace (a column index out of range). */
spgemm_status spgemm_transpose_check(void* workspace, spgemm_stream_t stream);

/* The same transpose as spgemm_transpose, for callers that cannot allocate
 * device memory when they need it (for example code inside an allocator's
 * out-of-memory path, code holding a lock the allocator also takes, or a
 * service whose device memory is fixed at start-up): it takes no workspace
 * and allocates nothing.  The paper has no counterpart; this is a library
 * convenience.
 *
 * Its scratch is one fixed 8 MiB device array inside this library, present
 * on every GPU that loads the library until the process exits.  Inputs whose
 * scratch would exceed it are rejected with SPGEMM_ERR_WORKSPACE: the need
 * is, for 513 to 262,144 columns, 12*nnz bytes plus 8*nnz (FP64) or 4*nnz
 * (FP32) when t_vals is given (none of this for at most 512 columns; 4*nnz
 * more above 262,144 columns), plus 4*nnz when t_src is NULL (the source
 * positions then need scratch too), plus the digit counts (4 bytes per
 * digit value and 4096 entries: at most nnz/2 bytes) and their scan partials
 * (8 bytes per 4096 counts or columns), plus about 2 KB of bookkeeping and
 * alignment; so about 400 K entries fit with t_src and FP64 t_vals given.
 * The inputs follow
 * spgemm_transpose's preconditions.  The first call on a device looks
 * up the array's device address; make that first call before any stream
 * capture.  All calls on a device share the array (each call clears what
 * must start at zero), so calls whose GPU work can overlap -- on different
 * streams without ordering -- race and must not be issued.  Errors found on
 * the device are not reported by this call. */
spgemm_status spgemm_transpose_noalloc(const spgemm_csr* M, int32_t dtype, int32_t* t_row_ptr,
                                       int32_t* t_col_idx, void* t_vals, int32_t* t_src,
                                       spgemm_stream_t stream);

/* Masked product C<M> = (A*B) .* M, the sampled SpGEMM of triangle counting
 * and Markov clustering (two of the applications Sec. 1 lists), computed on
 * the pattern of M with the row-wise Gustavson order of Sec. 2.2.  For entry
 * p = (i,j) of M:
 *   c_vals[p] = M(i,j) * sum_k A(i,k) * B(k,j),
 * the sum over the k with A(i,k) and B(k,j) both stored; an entry of M that
 * no product reaches gets 0 (the output keeps all of M's pattern).  With
 * use_mask_values == 0 the factor M(i,j) is 1 and M.vals is not read.
 *   A: m x k, B: k x n, M: m x n (device CSR; M's columns ascending in each
 *   row, A's columns below k).  c_vals: nnz(M) values of `dtype`, aligned
 *   with M's col_idx, caller-allocated, overwritten.
 * c_vals is zeroed by the call, then each product is rounded and added to
 * its entry's sum (shared-memory and global FP64 reductions), and the
 * finished sums are multiplied by M's values.  The order of the additions
 * is not fixed, so real-valued sums may differ from a sequential sum in the
 * last bits (integer-valued inputs are exact).
 * Errors: SPGEMM_ERR_DIM_MISMATCH for inconsistent shapes,
 * SPGEMM_ERR_INVALID_ARG for missing arrays or a bad dtype.  Does not
 * block, allocates nothing, keeps no state. */
spgemm_status spgemm_masked(const spgemm_csr* A, const spgemm_csr* B, const spgemm_csr* M, int32_t dtype,
                            int32_t use_mask_values, void* c_vals, spgemm_stream_t stream);

/* Semirings of spgemm_semiring: the "sum" that merges the products of one
 * entry, the "product" of A(i,k) and B(k,j), and the zero an entry keeps when
 * no product reaches it. */
typedef enum spgemm_semiring_kind {
  SPGEMM_PLUS_TIMES = 0, /* sum +,   product a*b,                       zero 0     */
  SPGEMM_MIN_PLUS = 1,   /* sum min, product a+b,                       zero +inf  */
  SPGEMM_MAX_PLUS = 2,   /* sum max, product a+b,                       zero -inf  */
  SPGEMM_OR_AND = 3      /* sum or,  product (a != 0 and b != 0) as 1/0, zero 0     */
} spgemm_semiring_kind;

/* The masked product of spgemm_masked over another semiring (all-pairs
 * shortest paths by repeated min-plus squaring, longest paths, reachability;
 * Sec. 1 lists shortest paths among SpGEMM's applications), on the pattern
 * of M with the row-wise Gustavson order of Sec. 2.2:
 *   c_vals[p] = sum over k of product(A(i,k), B(k,j))  for entry p = (i,j) of M,
 * over the k with A(i,k) and B(k,j) both stored, and the semiring's zero where
 * there is none.  M's values are not read.  With M the pattern of A*B (from
 * spgemm_symbolic and spgemm_numeric) this is the full semiring product.
 * Min-plus, max-plus and or-and results do not depend on the order of the
 * sums, so they are exact; plus-times is spgemm_masked without M's values.
 * Shapes, arrays and errors as spgemm_masked; SPGEMM_ERR_INVALID_ARG for an
 * unknown semiring.  Does not block, allocates nothing, keeps no state. */
spgemm_status spgemm_semiring(const spgemm_csr* A, const spgemm_csr* B, const spgemm_csr* M, int32_t dtype,
                              int32_t semiring, void* c_vals, spgemm_stream_t stream);

/* ------------------------------------------------------- host buffers
 * The whole product from host memory to host memory.  A and B are CSR with
 * HOST pointers (pinned memory lets the copies overlap); C arrives in host
 * arrays the caller allocates once nnz(C) is known.  Rows of C are
 * independent (Sec. 2.2), so after one symbolic pass the numeric pass runs
 * in row ranges of about equal output, each copied to the host on a second
 * stream while the later ranges compute. */
typedef struct spgemm_host_product spgemm_host_product;

/* Device workspace of spgemm_host_product_begin: copies of A and B (one copy
 * when B is A), C's row pointer and the plan of the whole product.  Host
 * only. */
spgemm_status spgemm_host_product_workspace_size(const spgemm_csr* A, const spgemm_csr* B,
                                                 const spgemm_opts* opts, size_t* bytes);

/* Copies A and B (host CSR, values of opts->dtype) into the workspace on
 * `stream`, analyses the product, runs the symbolic pass and cuts the rows
 * into at most `chunks` ranges by output (the last rows' range about
 * 1/(2 chunks) of nnz(C), the others equal).  BLOCKS on `stream` to
 * return nnz(C).  The workspace (device, 16-byte aligned) must stay valid
 * until spgemm_host_product_destroy; the host inputs may be released on
 * return.  opts: row_begin/row_end, backward and validate are ignored. */
spgemm_status spgemm_host_product_begin(const spgemm_csr* A, const spgemm_csr* B, const spgemm_opts* opts,
                                        int32_t chunks, void* workspace, size_t workspace_bytes,
                                        spgemm_stream_t stream, spgemm_host_product** product, int64_t* nnz_c);

/* Device staging bytes spgemm_host_product_finish needs: C's columns and
 * values, and the workspaces of the row-range plans. */
spgemm_status spgemm_host_product_staging_size(const spgemm_host_product* product, size_t* bytes);

/* Numeric pass of every row range on `stream` into the staging buffer
 * (device, 16-byte aligned), from the last range to the first (the small
 * last-rows range first, so the copies start early), each range copied into
 * c_col_idx / c_vals (host, nnz(C) entries) on copy_stream as soon as it is
 * done (NULL: `stream`, no overlap); c_row_ptr (host, nrows(A) + 1 entries) receives C's
 * row pointer.  BLOCKS until C is complete in host memory; reports any
 * device error of the range plans.  Repeatable (the inputs' values are those
 * copied by begin). */
spgemm_status spgemm_host_product_finish(spgemm_host_product* product, int32_t* c_row_ptr, int32_t* c_col_idx,
                                         void* c_vals, void* staging, size_t staging_bytes, spgemm_stream_t stream,
                                         spgemm_stream_t copy_stream);

/* Number of row ranges, and the device timeline of the last finish: for
 * range r, ms[4r .. 4r+3] = its numeric pass's start and end and its copy's
 * start and end, in milliseconds from the start of the first range (entries
 * past the ranges read 0). */
spgemm_status spgemm_host_product_ranges(const spgemm_host_product* product, int32_t* nranges);
spgemm_status spgemm_host_product_timeline(const spgemm_host_product* product, float* ms, int32_t n);

/* Frees the handle and its plan (host memory only).  NULL is allowed. */
void spgemm_host_product_destroy(spgemm_host_product* product);

/* Frees the plan (host memory only).  NULL is allowed. */
void spgemm_plan_destroy(spgemm_plan* plan);

/* ------------------------------------------------------------------ batch
 * Many independent products C_i = A_i * B_i (i < n) computed together: the
 * instances are stacked into one block-diagonal product, so each pass is one
 * persistent launch per path over a global work list of all instances' rows
 * (largest rows first).  The stacked C is returned in one CSR: instance i
 * owns the rows [r_i, r_i + A_i.nrows) with r_i = sum of the earlier
 * A_j.nrows, and its column indices are its own (0 .. B_i.ncols-1).
 * Counts over all instances (rows, nnz of A, nnz of B, nnz of C) must each
 * fit int32 (split a larger batch into waves). */
typedef struct spgemm_batch spgemm_batch;

/* Device workspace bytes for a batch (host only). */
spgemm_status spgemm_batch_workspace_size(int32_t n, const spgemm_csr* As, const spgemm_csr* Bs,
                                          const spgemm_opts* opts, size_t* bytes);

/* Creates the batch from n host descriptors whose pointers are device
 * pointers; As[i].vals / Bs[i].vals are the value buffers that every later
 * spgemm_batch_numeric reads (update them in place for new values).  Stacks
 * the structure and analyses the stacked product on `stream`; does not block.
 * All buffers must stay valid until spgemm_batch_destroy. */
spgemm_status spgemm_batched(int32_t n, const spgemm_csr* As, const spgemm_csr* Bs, const spgemm_opts* opts,
                             void* workspace, size_t workspace_bytes, spgemm_stream_t stream,
                             spgemm_batch** batch);

/* Rows of the stacked C (the length of c_row_ptr minus one). */
spgemm_status spgemm_batch_rows(spgemm_batch* batch, int64_t* total_rows);

/* Symbolic pass of all instances: writes the stacked row pointer and BLOCKS
 * to return c_nnz[i] for each instance and c_nnz[n] = total (host array of
 * n+1 entries). */
spgemm_status spgemm_batch_symbolic(spgemm_batch* batch, int32_t* c_row_ptr, int64_t* c_nnz,
                                    spgemm_stream_t stream);

/* Numeric pass of all instances: gathers the instances' values, runs the
 * stacked numeric pass, writes C's columns (per-instance numbering) and
 * values.  Does not block and allocates nothing: capturable in a CUDA graph. */
spgemm_status spgemm_batch_numeric(spgemm_batch* batch, const int32_t* c_row_ptr, int32_t* c_col_idx,
                                   void* c_vals, spgemm_stream_t stream);

/* Same types as cudaGraph_t and cudaGraphExec_t. */
typedef struct CUgraph_st* spgemm_graph_t;
typedef struct CUgraphExec_st* spgemm_graph_exec_t;

/* Records the batch numeric pass (spgemm_batch_numeric with these output
 * arrays) into a new CUDA graph, which *graph receives and the caller owns
 * (spgemm_graph_destroy or cudaGraphDestroy).  The batched launch of the
 * spec workloads is meant to run this way: instantiate once, then
 * launch the graph for every new set of values written in place into the
 * instances' value buffers.  The graph reads the value buffers given to
 * spgemm_batched and writes c_col_idx / c_vals; all of them must stay valid
 * while the graph can run.  spgemm_batch_symbolic must have run
 * (SPGEMM_ERR_NOT_READY otherwise).  `stream` is used for the capture only:
 * it must be a stream the caller created (not the legacy default stream,
 * SPGEMM_ERR_INVALID_ARG) that is not already capturing; the capture is in
 * thread-local mode and issues no GPU work.  Does not block. */
spgemm_status spgemm_batch_capture(spgemm_batch* batch, const int32_t* c_row_ptr, int32_t* c_col_idx,
                                   void* c_vals, spgemm_stream_t stream, spgemm_graph_t* graph);

/* Graph helpers for callers without the CUDA runtime API at hand (thin
 * wrappers of cudaGraphInstantiate, cudaGraphLaunch, cudaGraphExecDestroy
 * and cudaGraphDestroy).  spgemm_graph_launch is asynchronous on `stream`;
 * spgemm_graph_destroy accepts NULL for either argument. */
spgemm_status spgemm_graph_instantiate(spgemm_graph_t graph, spgemm_graph_exec_t* exec);
spgemm_status spgemm_graph_launch(spgemm_graph_exec_t exec, spgemm_stream_t stream);
void spgemm_graph_destroy(spgemm_graph_t graph, spgemm_graph_exec_t exec);

/* Waves.  One spgemm_batched call stacks its instances into one CSR, so the
 * stacked counts above and nnz of the stacked C must each stay below 2^31.
 * A larger batch (for example 512 instances whose products add up to about
 * 10^10) runs as several waves, each one spgemm_batched call on a run of
 * consecutive instances with its own C.  The number of scalar products of
 * C_i = A_i * B_i (Sec. 2.2: each nonzero A_i(r,k) scales the nnz(B_i(k,:))
 * entries of row k of B_i) bounds nnz(C_i) from above, so waves are cut by
 * product counts. */

/* Device workspace bytes of spgemm_batch_products for n instances (host only). */
spgemm_status spgemm_batch_products_workspace_size(int32_t n, size_t* bytes);

/* products[i] (device, n int64 entries, overwritten) = the number of scalar
 * products of C_i = A_i * B_i, i.e. the sum over the nonzeros A_i(r,k) of
 * nnz(B_i(k,:)).  Reads only the structure of A_i and B_i (device CSR).  One
 * launch over all instances on `stream`; does not block (the descriptors are
 * staged from host memory before it returns).  workspace: device, at least
 * spgemm_batch_products_workspace_size bytes, 16-byte aligned, in use until
 * the launch has run.  SPGEMM_ERR_DIM_MISMATCH if A_i.ncols != B_i.nrows. */
spgemm_status spgemm_batch_products(int32_t n, const spgemm_csr* As, const spgemm_csr* Bs, int64_t* products,
                                    void* workspace, size_t workspace_bytes, spgemm_stream_t stream);

/* Splits n instances into waves of consecutive instances: wave w holds
 * instances [wave_first[w], wave_first[w+1]), *nwaves waves in all
 * (wave_first: host, n+1 entries).  A wave takes instances in order while
 * its stacked rows, columns, nnz(A) and nnz(B) stay below 2^31 - 1 and the
 * sum of its products (host array, from spgemm_batch_products) stays at or
 * below max_products (<= 0: 2^31 - 1, which keeps every wave's nnz(C) inside
 * int32), and the sum of its nnz(B_i) at or below max_b_nnz (<= 0: no bound
 * beyond int32; a bound sized to the L2 cache keeps each wave's B operands,
 * which every row of the wave re-reads, resident there).  An instance that
 * alone exceeds a bound forms a wave of its own (its nnz(C) may still fit;
 * spgemm_batch_symbolic reports SPGEMM_ERR_INDEX_OVERFLOW if not).  Host
 * only; reads only the sizes of the descriptors.  SPGEMM_ERR_INDEX_OVERFLOW
 * if one instance alone breaks a count limit. */
spgemm_status spgemm_batch_waves(int32_t n, const spgemm_csr* As, const spgemm_csr* Bs, const int64_t* products,
                                 int64_t max_products, int64_t max_b_nnz, int32_t* wave_first, int32_t* nwaves);

/* The plan of the stacked product (statistics, timers, error word). */
spgemm_plan* spgemm_batch_plan(spgemm_batch* batch);

void spgemm_batch_destroy(spgemm_batch* batch);

#ifdef __cplusplus
}
#endif

#endif /* SPGEMM_GB300_H */
