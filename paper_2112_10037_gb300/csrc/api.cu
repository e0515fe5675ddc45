// C ABI of the library (declared in include/spgemm.h): argument checks,
// workspace carving, plan state and the order of the passes.
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "internal.cuh"

struct spgemm_plan {
  int device = 0;
  int nsm = 0;
  sg::Csr A{}, B{};
  spgemm_opts opts{};
  long long row_begin = 0, mloc = 0;
  // carved workspace
  unsigned char* ws = nullptr;
  size_t ws_bytes = 0;
  sg::DevStats* st = nullptr;
  long long* prod = nullptr;
  int* cmin = nullptr;
  int* cmax = nullptr;
  int* rows = nullptr;
  int32_t* cursor = nullptr;
  int32_t* nxt = nullptr;
  long long* scan_part = nullptr;
  long long* runs_part = nullptr;
  // transpose of A's structure (backward pass)
  int32_t* at_rp = nullptr;
  int32_t* at_ci = nullptr;
  int32_t* at_src = nullptr;
  int32_t* a_row = nullptr;  // row of every nonzero of A (backward)
  int32_t* b_row = nullptr;  // row of every entry of B (backward)
  // host state
  sg::PathBins pb{};
  sg::Tuning tu{};
  sg::SplitInfo sp{};
  bool symbolic_done = false;
  long long nnz_c = -1;
  int path_rows[sg::NPATHS] = {0, 0, 0, 0};
  sg::DevStats host_st{};
  // measurement
  bool profiling = false;
  cudaEvent_t timers[2 * sg::NTIMERS] = {};
  int timer_used[sg::NTIMERS] = {};
  long long launches = 0;

  ~spgemm_plan() {
    for (auto& ev : timers)
      if (ev) cudaEventDestroy(ev);
  }
};

namespace {

constexpr size_t ALIGN = 256;
inline size_t align_up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }

struct Layout {
  size_t st, prod, cmin, cmax, rows, cursor, nxt, scan, rr, runs, runs_part, hcnt, rrb, runsb;
  size_t at_rp, at_ci, at_src, at_tmp, at_table, at_part, a_row, b_row;  // opts.backward only
  size_t total;
};

// Workspace of a transpose of an m x n matrix with nnz entries, at offset
// `off`; returns the end offset.
size_t transpose_layout(size_t off, long long n, long long nnz, int vbytes, size_t* tmp, size_t* table,
                        size_t* part) {
  const sg::TransposeScratch s = sg::transpose_scratch(n, nnz, vbytes);
  *tmp = off; off = align_up(off + sizeof(int32_t) * s.tmp_ints);
  *table = off; off = align_up(off + sizeof(int32_t) * s.table_ints);
  *part = off; off = align_up(off + sizeof(long long) * s.part_count);
  return off;
}

int numeric_block_bin(const spgemm_opts& o);

// Last bin of the register-sort path: rows of at most 128, 256 or 512
// products (opts.sort_max; bin b holds products in (2^(b-2), 2^(b-1)]).
int tiny_hi_bin(const spgemm_opts& o) {
  const int m = o.sort_max > 0 ? o.sort_max : 128;
  return m >= 512 ? 10 : (m >= 256 ? 9 : 8);
}

// First bin of the hash path (rows of 17 or more products; smaller rows keep
// the register sort, whose network is then at most 16 elements wide).
constexpr int HASH_LO_BIN = 6;

// Last bin of the hash path, 0 when it is off: rows of 17..opts.hash_max
// products (0: 128; rounded up to 32, 64 or 128).  Off with hash_max < 0,
// with a forced path, or when a register sort above 128 products is asked
// for (sort_max 256 or 512).
int hash_hi_bin(const spgemm_opts& o) {
  if (o.hash_max < 0 || o.force_path >= 0 || o.sort_max > 128) return 0;
  int m = o.hash_max > 0 ? o.hash_max : 128;
  if (m < 17) m = 17;
  if (m > 128) m = 128;
  return sg::bin_of(m);
}

// Last bin of the rows that need no column window (register sort or hash).
int small_hi_bin(const spgemm_opts& o) {
  const int h = hash_hi_bin(o);
  return h > 0 ? h : tiny_hi_bin(o);
}

// Window geometry and split capacity from the options and B's width (see
// sg::SplitInfo).  *hcnt_entries is 0 when no row is split.
void split_geometry(const spgemm_opts& o, int window, long long mloc, long long ncols_b, sg::SplitInfo* sp,
                    size_t* hcnt_entries) {
  sp->heavy_bin = sg::NBINS;
  sp->hi_bin = numeric_block_bin(o) - 1;  // the warp kernel's last bin
  if (sp->hi_bin > sg::NBINS - 1) sp->hi_bin = sg::NBINS - 1;
  sp->hcap = 0;
  sp->wf_shift = 0;
  while ((1 << sp->wf_shift) < window) ++sp->wf_shift;
  sp->ntf = (int)((ncols_b + window - 1) / window);
  *hcnt_entries = 0;
  if (o.split_min < 0 || o.force_path >= 0 || mloc <= 0 || sp->ntf < 2) return;
  const long long smin = o.split_min > 0 ? o.split_min : 131072;
  if (sg::bin_of(smin) + 1 >= numeric_block_bin(o)) return;  // those rows use the block window
  long long cap = mloc < 16384 ? mloc : 16384;
  const long long lim = ((long long)1 << 24) / sp->ntf;
  if (cap > lim) cap = lim;
  if (cap <= 0) return;
  // split rows always lie above the register-sort bins (1..8), so their
  // sizes come from the bitmap-window kernel, which records per-window counts
  sp->heavy_bin = sg::bin_of(smin) + 1;
  if (sp->heavy_bin < small_hi_bin(o) + 1) sp->heavy_bin = small_hi_bin(o) + 1;
  if (sp->heavy_bin >= sg::NBINS) { sp->heavy_bin = sg::NBINS; return; }
  sp->hcap = (int)cap;
  *hcnt_entries = (size_t)cap * (size_t)sp->ntf;
}

// First bin of rows whose numeric pass uses the block-wide window.
int numeric_block_bin(const spgemm_opts& o) {
  if (o.force_path == 1 || o.force_path == 3) return sg::NBINS;  // warp window only
  if (o.force_path == 2) return tiny_hi_bin(o) + 1;                 // every row above the register sort
  if (o.force_path == 4) return 1;                                 // every non-empty row
  if (o.num_block_min < 0) return sg::NBINS;
  const long long m = o.num_block_min > 0 ? o.num_block_min : 65536;
  const int b = sg::bin_of(m) + 1;
  return b < small_hi_bin(o) + 1 ? small_hi_bin(o) + 1 : b;
}

// First bin of rows whose numeric pass uses the rank-compacted block
// accumulator: rows of more than opts.rank_min products below the block
// window's bins; NBINS when off (rank_min <= 0, the default).
int numeric_rank_bin(const spgemm_opts& o) {
  if (o.force_path >= 0 || o.rank_min <= 0) return sg::NBINS;
  const long long m = o.rank_min;
  const int b = sg::bin_of(m) + 1;
  return b < small_hi_bin(o) + 1 ? small_hi_bin(o) + 1 : b;
}

int numeric_window(const spgemm_opts& o) {
  return (o.window_warp == 2048 || o.window_warp == 4096) ? o.window_warp : 1024;
}

// own_b: the plan builds its own window-run lists of B (false: it reads
// another plan's).
Layout layout_for(const spgemm_opts& o, long long mloc, long long nnz_a, long long nrows_b, long long ncols_b,
                  long long nnz_b, bool own_b = true) {
  sg::SplitInfo sp;
  size_t nh = 0;
  split_geometry(o, numeric_window(o), mloc, ncols_b, &sp, &nh);
  Layout L{};
  size_t off = 0;
  L.st = off; off = align_up(off + sizeof(sg::DevStats));
  L.prod = off; off = align_up(off + sizeof(long long) * (size_t)mloc);
  L.cmin = off; off = align_up(off + sizeof(int) * (size_t)mloc);
  L.cmax = off; off = align_up(off + sizeof(int) * (size_t)mloc);
  L.rows = off; off = align_up(off + sizeof(int) * (size_t)mloc);
  L.cursor = off; off = align_up(off + sizeof(int32_t) * (size_t)nnz_a);
  L.nxt = off; off = align_up(off + sizeof(int32_t) * (size_t)nnz_a);
  L.scan = off; off = align_up(off + sizeof(long long) * sg::scan_partials_count(mloc));
  L.rr = L.runs = L.runs_part = 0;
  if (own_b) {
    L.rr = off; off = align_up(off + sizeof(int32_t) * (size_t)(nrows_b + 1));
    L.runs = off; off = align_up(off + sizeof(int2) * (size_t)(nnz_b + nrows_b + sg::RUNS_PAD));
    L.runs_part = off; off = align_up(off + sizeof(long long) * sg::scan_partials_count(nrows_b));
  }
  L.hcnt = off; off = align_up(off + sizeof(int32_t) * nh);
  L.rrb = L.runsb = 0;
  if (own_b && numeric_block_bin(o) < sg::NBINS) {  // run list at the block window's width
    L.rrb = off; off = align_up(off + sizeof(int32_t) * (size_t)(nrows_b + 1));
    L.runsb = off; off = align_up(off + sizeof(int2) * (size_t)(nnz_b + nrows_b + sg::RUNS_PAD));
  }
  if (o.backward) {
    L.at_rp = off; off = align_up(off + sizeof(int32_t) * (size_t)(nrows_b + 1));
    L.at_ci = off; off = align_up(off + sizeof(int32_t) * (size_t)nnz_a);
    L.at_src = off; off = align_up(off + sizeof(int32_t) * (size_t)nnz_a);
    L.a_row = off; off = align_up(off + sizeof(int32_t) * (size_t)nnz_a);
    L.b_row = off; off = align_up(off + sizeof(int32_t) * (size_t)nnz_b);
    off = transpose_layout(off, nrows_b, nnz_a, 0, &L.at_tmp, &L.at_table, &L.at_part);
  }
  L.total = off;
  return L;
}

int sm_count_for(int dev) {
  static std::mutex mu;
  static int cache[64] = {0};
  if (dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> g(mu);
  if (!cache[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) cache[dev] = n;
  }
  return cache[dev];
}

spgemm_status check_csr(const spgemm_csr* M) {
  if (!M) return SPGEMM_ERR_INVALID_ARG;
  if (M->nrows < 0 || M->ncols < 0 || M->nnz < 0) return SPGEMM_ERR_INVALID_ARG;
  if (M->nrows >= (1ll << 31) - 1 || M->ncols >= (1ll << 31) - 1 || M->nnz >= (1ll << 31))
    return SPGEMM_ERR_INDEX_OVERFLOW;
  if (!M->row_ptr) return SPGEMM_ERR_INVALID_ARG;
  if (M->nnz > 0 && !M->col_idx) return SPGEMM_ERR_INVALID_ARG;
  return SPGEMM_OK;
}

// Window columns and warps of the numeric block kernel: one of the compiled
// pairs, the default where the options name none or an unsupported one.
static void block_geometry(const spgemm_opts& o, int* w, int* nw) {
  static const int pairs[][2] = {{2048, 4}, {2048, 8}, {4096, 4}, {4096, 8}, {4096, 16}, {8192, 8}, {8192, 16},
                                 {16384, 16}};
  const int dw = 8192, dn = 8;  // default geometry
  const int ww = o.window_block > 0 ? o.window_block : dw, nn = o.block_warps > 0 ? o.block_warps : dn;
  *w = dw;
  *nw = dn;
  for (const auto& p : pairs)
    if (p[0] == ww && p[1] == nn) {
      *w = ww;
      *nw = nn;
    }
}

// Bin ranges of the paths from the options (see sg::bin_of for the bins).
void choose_paths(const spgemm_opts& o, sg::PathBins* pb, sg::Tuning* tu) {
  const int last = sg::NBINS - 1;
  tu->warp_max = o.warp_max > 0 ? o.warp_max : 8192;
  tu->window_warp = numeric_window(o);
  block_geometry(o, &tu->window_block, &tu->block_warps);
  const int HASH_HI = hash_hi_bin(o);
  tu->hash_max = HASH_HI > 0 ? 1 << (HASH_HI - 1) : 0;
  tu->num_lo_block = numeric_block_bin(o);
  tu->num_lo_rank = numeric_rank_bin(o);
  tu->rank_accum = o.rank_accum == 1 ? 1 : 0;
  const int TINY_HI = tiny_hi_bin(o);  // register sort up to opts.sort_max products
  const int SMALL_HI = small_hi_bin(o);
  const int wb = sg::bin_of(tu->warp_max) < SMALL_HI + 1 ? SMALL_HI + 1 : sg::bin_of(tu->warp_max);
  for (int p = 0; p < sg::NPATHS; ++p) { pb->lo[p] = 1; pb->hi[p] = 0; }
  switch (o.force_path) {
    case 1: pb->lo[sg::PATH_TINY] = 1; pb->hi[sg::PATH_TINY] = TINY_HI; pb->lo[sg::PATH_WARP] = TINY_HI + 1; pb->hi[sg::PATH_WARP] = last; break;
    case 2: pb->lo[sg::PATH_TINY] = 1; pb->hi[sg::PATH_TINY] = TINY_HI; pb->lo[sg::PATH_BLOCK] = TINY_HI + 1; pb->hi[sg::PATH_BLOCK] = last; break;
    case 3: pb->lo[sg::PATH_WARP] = 1; pb->hi[sg::PATH_WARP] = last; break;
    case 4: pb->lo[sg::PATH_BLOCK] = 1; pb->hi[sg::PATH_BLOCK] = last; break;
    default:
      pb->lo[sg::PATH_TINY] = 1; pb->hi[sg::PATH_TINY] = HASH_HI > 0 ? HASH_LO_BIN - 1 : TINY_HI;
      if (HASH_HI > 0) { pb->lo[sg::PATH_HASH] = HASH_LO_BIN; pb->hi[sg::PATH_HASH] = HASH_HI; }
      pb->lo[sg::PATH_WARP] = SMALL_HI + 1; pb->hi[sg::PATH_WARP] = wb;
      pb->lo[sg::PATH_BLOCK] = wb + 1; pb->hi[sg::PATH_BLOCK] = last;
      break;
  }
}

spgemm_status from_err_word(uint32_t w) {
  if (w & sg::EB_UNSORTED) return SPGEMM_ERR_UNSORTED_INPUT;
  if (w & sg::EB_OVERFLOW) return SPGEMM_ERR_INDEX_OVERFLOW;
  if (w & sg::EB_TABLE) return SPGEMM_ERR_TABLE_OVERFLOW;
  if (w & sg::EB_INTERNAL) return SPGEMM_ERR_INTERNAL;
  return SPGEMM_OK;
}

sg::LaunchCtx ctx_of(spgemm_plan* p, spgemm_stream_t s) {
  sg::LaunchCtx c;
  c.stream = (cudaStream_t)s;
  c.nsm = p->nsm;
  c.st = p->st;
  c.err = &p->st->err;
  c.timers = p->profiling ? p->timers : nullptr;
  c.timer_used = p->timer_used;
  c.launches = &p->launches;
  return c;
}

sg::RowInfo rowinfo_of(const spgemm_plan* p) {
  sg::RowInfo ri;
  ri.row_begin = p->row_begin;
  ri.mloc = p->mloc;
  ri.prod = p->prod;
  ri.cmin = p->cmin;
  ri.cmax = p->cmax;
  ri.rows = p->rows;
  return ri;
}

spgemm_status read_stats(spgemm_plan* p, cudaStream_t s) {
  if (cudaMemcpyAsync(&p->host_st, p->st, sizeof(sg::DevStats), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return SPGEMM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SPGEMM_ERR_CUDA;
  for (int q = 0; q < sg::NPATHS; ++q) {
    int n = 0;
    for (int b = p->pb.lo[q]; b <= p->pb.hi[q]; ++b) n += p->host_st.hist[b];
    p->path_rows[q] = n;
  }
  return SPGEMM_OK;
}

}  // namespace

// Other semirings than plus-times skip the rank-compacted accumulator,
// register sorts above 128 products, split rows and the non-default window
// sizes: their options are reset here, for the workspace size and the plan
// alike.
static void semiring_defaults(spgemm_opts* o) {
  if (o->semiring == SPGEMM_PLUS_TIMES) return;
  o->sort_max = 0;
  o->rank_min = -1;
  o->split_min = -1;
  o->window_warp = 0;
  o->window_block = 0;
  o->block_warps = 0;
}

// base: another plan of the same product whose window-run lists of B this
// plan reads instead of building its own (null: build them).
static spgemm_status analyse_impl(const spgemm_csr* A, const spgemm_csr* B, const spgemm_opts* opts,
                                  void* workspace, size_t workspace_bytes, spgemm_stream_t stream,
                                  const spgemm_plan* base, spgemm_plan** plan) {
  if (!plan) return SPGEMM_ERR_INVALID_ARG;
  *plan = nullptr;
  spgemm_status s;
  if ((s = check_csr(A)) != SPGEMM_OK) return s;
  if ((s = check_csr(B)) != SPGEMM_OK) return s;
  if (A->ncols != B->nrows) return SPGEMM_ERR_DIM_MISMATCH;
  spgemm_opts o;
  if (opts) o = *opts; else spgemm_opts_default(&o);
  if (o.dtype != SPGEMM_F64 && o.dtype != SPGEMM_F32) return SPGEMM_ERR_INVALID_ARG;
  if (o.force_path < -1 || o.force_path > 4) return SPGEMM_ERR_INVALID_ARG;
  if (o.semiring < SPGEMM_PLUS_TIMES || o.semiring > SPGEMM_OR_AND) return SPGEMM_ERR_INVALID_ARG;
  if (o.semiring != SPGEMM_PLUS_TIMES && o.backward) return SPGEMM_ERR_INVALID_ARG;
  semiring_defaults(&o);
  const long long rb = o.row_begin, re = o.row_end < 0 ? A->nrows : o.row_end;
  if (rb < 0 || re < rb || re > A->nrows) return SPGEMM_ERR_DIM_MISMATCH;
  const Layout L = layout_for(o, re - rb, A->nnz, B->nrows, B->ncols, B->nnz, base == nullptr);
  if (!workspace || workspace_bytes < L.total) return SPGEMM_ERR_WORKSPACE;
  if (((uintptr_t)workspace) % 16) return SPGEMM_ERR_WORKSPACE;

  spgemm_plan* p = new (std::nothrow) spgemm_plan();
  if (!p) return SPGEMM_ERR_INTERNAL;
  if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return SPGEMM_ERR_CUDA; }
  p->nsm = sm_count_for(p->device);
  if (p->nsm <= 0) { delete p; return SPGEMM_ERR_CUDA; }
  p->A = sg::Csr{A->row_ptr, A->col_idx, A->nrows, A->ncols, A->nnz};
  p->B = sg::Csr{B->row_ptr, B->col_idx, B->nrows, B->ncols, B->nnz};
  p->opts = o;
  p->row_begin = rb;
  p->mloc = re - rb;
  p->ws = (unsigned char*)workspace;
  p->ws_bytes = workspace_bytes;
  p->st = (sg::DevStats*)(p->ws + L.st);
  p->prod = (long long*)(p->ws + L.prod);
  p->cmin = (int*)(p->ws + L.cmin);
  p->cmax = (int*)(p->ws + L.cmax);
  p->rows = (int*)(p->ws + L.rows);
  p->cursor = (int32_t*)(p->ws + L.cursor);
  p->nxt = (int32_t*)(p->ws + L.nxt);
  p->scan_part = (long long*)(p->ws + L.scan);
  choose_paths(o, &p->pb, &p->tu);
  {
    size_t nh = 0;
    split_geometry(o, p->tu.window_warp, p->mloc, B->ncols, &p->sp, &nh);
    p->sp.hcnt = nh ? (int32_t*)(p->ws + L.hcnt) : nullptr;
    p->sp.wb_shift = 0;
    while ((1 << p->sp.wb_shift) < p->tu.window_block) ++p->sp.wb_shift;
    if (base) {
      p->sp.rr = base->sp.rr;
      p->sp.runs = base->sp.runs;
      p->sp.rrb = base->sp.rrb;
      p->sp.runsb = base->sp.runsb;
      p->runs_part = nullptr;
    } else {
      p->sp.rr = (int32_t*)(p->ws + L.rr);
      p->sp.runs = (int2*)(p->ws + L.runs);
      p->sp.rrb = L.rrb ? (int32_t*)(p->ws + L.rrb) : nullptr;
      p->sp.runsb = L.runsb ? (int2*)(p->ws + L.runsb) : nullptr;
      p->runs_part = (long long*)(p->ws + L.runs_part);
    }
  }

  cudaStream_t st = (cudaStream_t)stream;
  sg::LaunchCtx c = ctx_of(p, stream);
  cudaError_t e = cudaMemsetAsync(p->st, 0, sizeof(sg::DevStats), st);
  if (e == cudaSuccess && o.validate) {
    e = sg::launch_validate(c, p->A);
    if (e == cudaSuccess) e = sg::launch_validate(c, p->B);
  }
  if (e == cudaSuccess) e = sg::launch_analyse(c, p->A, p->B, p->row_begin, p->mloc, p->prod, p->cmin, p->cmax, p->rows);
  if (e == cudaSuccess && !base) {
    // Only the numeric window paths read the run lists.  A plan of every row
    // of A may leave them unbuilt when none of its rows takes such a path:
    // plans derived from it cover subsets of those rows.
    int win_lo = sg::NBINS;
    for (int q : {sg::PATH_WARP, sg::PATH_BLOCK})
      if (p->pb.hi[q] >= p->pb.lo[q] && p->pb.lo[q] < win_lo) win_lo = p->pb.lo[q];
    if (rb != 0 || re != A->nrows) win_lo = 0;
    e = sg::launch_runs(c, p->B, p->sp, p->runs_part, win_lo);
  }
  if (e == cudaSuccess && o.backward) {
    p->at_rp = (int32_t*)(p->ws + L.at_rp);
    p->at_ci = (int32_t*)(p->ws + L.at_ci);
    p->at_src = (int32_t*)(p->ws + L.at_src);
    e = sg::launch_transpose(c, A->nrows, A->ncols, A->nnz, A->row_ptr, A->col_idx, p->at_rp, p->at_ci, p->at_src,
                             0, nullptr, nullptr, (int32_t*)(p->ws + L.at_tmp), (int32_t*)(p->ws + L.at_table),
                             (long long*)(p->ws + L.at_part));
    p->a_row = (int32_t*)(p->ws + L.a_row);
    p->b_row = (int32_t*)(p->ws + L.b_row);
    if (e == cudaSuccess) e = sg::launch_row_index(c, A->row_ptr, A->nrows, p->a_row);
    if (e == cudaSuccess) e = sg::launch_row_index(c, B->row_ptr, B->nrows, p->b_row);
  }
  if (e != cudaSuccess) { delete p; return SPGEMM_ERR_CUDA; }
  *plan = p;
  return SPGEMM_OK;
}

extern "C" {

void spgemm_opts_default(spgemm_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->dtype = SPGEMM_F64;
  o->validate = 0;
  o->row_begin = 0;
  o->row_end = -1;
  o->warp_max = 0;
  o->force_path = -1;
  o->hash_max = 0;
  o->window_warp = 0;
  o->window_block = 0;
  o->split_min = 0;
  o->backward = 0;
  o->num_block_min = 0;
  o->block_warps = 0;
  o->sort_max = 0;
  o->rank_min = 0;
  o->rank_accum = 0;
}

const char* spgemm_status_string(spgemm_status s) {
  switch (s) {
    case SPGEMM_OK: return "ok";
    case SPGEMM_ERR_INVALID_ARG: return "invalid argument";
    case SPGEMM_ERR_DIM_MISMATCH: return "dimension mismatch";
    case SPGEMM_ERR_UNSORTED_INPUT: return "column indices out of range, repeated or not ascending";
    case SPGEMM_ERR_INDEX_OVERFLOW: return "index overflow (a count does not fit int32)";
    case SPGEMM_ERR_WORKSPACE: return "workspace missing or too small";
    case SPGEMM_ERR_TABLE_OVERFLOW: return "reserved status";
    case SPGEMM_ERR_CUDA: return "CUDA runtime error";
    case SPGEMM_ERR_INTERNAL: return "internal error";
    case SPGEMM_ERR_NOT_READY: return "call out of order";
  }
  return "unknown status";
}

const char* spgemm_version(void) { return "0.1.0"; }

spgemm_status spgemm_workspace_size(const spgemm_csr* A, const spgemm_csr* B, const spgemm_opts* opts,
                                    size_t* bytes) {
  if (!bytes) return SPGEMM_ERR_INVALID_ARG;
  spgemm_status s;
  if ((s = check_csr(A)) != SPGEMM_OK) return s;
  if ((s = check_csr(B)) != SPGEMM_OK) return s;
  spgemm_opts o;
  if (opts) o = *opts; else spgemm_opts_default(&o);
  semiring_defaults(&o);  // the options spgemm_analyse will use
  const long long rb = o.row_begin, re = o.row_end < 0 ? A->nrows : o.row_end;
  if (rb < 0 || re < rb || re > A->nrows) return SPGEMM_ERR_DIM_MISMATCH;
  *bytes = layout_for(o, re - rb, A->nnz, B->nrows, B->ncols, B->nnz).total;
  return SPGEMM_OK;
}

spgemm_status spgemm_analyse(const spgemm_csr* A, const spgemm_csr* B, const spgemm_opts* opts,
                             void* workspace, size_t workspace_bytes, spgemm_stream_t stream,
                             spgemm_plan** plan) {
  return analyse_impl(A, B, opts, workspace, workspace_bytes, stream, nullptr, plan);
}

// Options, A and B of a row-range plan derived from base.
static void rows_args(const spgemm_plan* base, int64_t rb, int64_t re, spgemm_csr* A, spgemm_csr* B,
                      spgemm_opts* o) {
  *A = spgemm_csr{base->A.nrows, base->A.ncols, base->A.nnz, base->A.rp, base->A.ci, nullptr};
  *B = spgemm_csr{base->B.nrows, base->B.ncols, base->B.nnz, base->B.rp, base->B.ci, nullptr};
  *o = base->opts;
  o->row_begin = rb;
  o->row_end = re;
  o->backward = 0;
  o->validate = 0;
}

spgemm_status spgemm_rows_workspace_size(const spgemm_plan* base, int64_t row_begin, int64_t row_end,
                                         size_t* bytes) {
  if (!base || !bytes) return SPGEMM_ERR_INVALID_ARG;
  if (!base->sp.rr || !base->sp.runs) return SPGEMM_ERR_NOT_READY;
  if (row_begin < 0 || row_end < row_begin || row_end > base->A.nrows) return SPGEMM_ERR_DIM_MISMATCH;
  spgemm_csr A, B;
  spgemm_opts o;
  rows_args(base, row_begin, row_end, &A, &B, &o);
  *bytes = layout_for(o, row_end - row_begin, A.nnz, B.nrows, B.ncols, B.nnz, false).total;
  return SPGEMM_OK;
}

spgemm_status spgemm_analyse_rows(const spgemm_plan* base, int64_t row_begin, int64_t row_end, void* workspace,
                                  size_t workspace_bytes, spgemm_stream_t stream, spgemm_plan** plan) {
  if (!plan) return SPGEMM_ERR_INVALID_ARG;
  *plan = nullptr;
  if (!base) return SPGEMM_ERR_INVALID_ARG;
  if (!base->sp.rr || !base->sp.runs) return SPGEMM_ERR_NOT_READY;
  if (row_begin < 0 || row_end < row_begin || row_end > base->A.nrows) return SPGEMM_ERR_DIM_MISMATCH;
  spgemm_csr A, B;
  spgemm_opts o;
  rows_args(base, row_begin, row_end, &A, &B, &o);
  return analyse_impl(&A, &B, &o, workspace, workspace_bytes, stream, base, plan);
}

spgemm_status spgemm_symbolic(spgemm_plan* p, int32_t* c_row_ptr, int64_t* c_nnz, spgemm_stream_t stream) {
  if (!p || !c_row_ptr || !c_nnz) return SPGEMM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  sg::LaunchCtx c = ctx_of(p, stream);
  const sg::RowInfo ri = rowinfo_of(p);
  cudaError_t e = cudaMemsetAsync(c_row_ptr, 0, sizeof(int32_t) * (size_t)(p->mloc + 1), st);
  if (e == cudaSuccess && p->mloc > 0)
    e = sg::launch_symbolic(c, p->A, p->B, ri, p->pb, p->tu, p->sp, p->cursor, c_row_ptr, nullptr);
  if (e == cudaSuccess) e = sg::launch_scan(c, c_row_ptr, p->mloc, p->scan_part);
  if (e != cudaSuccess) return SPGEMM_ERR_CUDA;
  spgemm_status s = read_stats(p, st);
  if (s != SPGEMM_OK) return s;
  s = from_err_word(p->host_st.err);
  if (s != SPGEMM_OK) return s;
  p->nnz_c = p->host_st.nnz_c;
  *c_nnz = p->nnz_c;
  p->symbolic_done = true;
  return SPGEMM_OK;
}

spgemm_status spgemm_plan_adopt_row_ptr(spgemm_plan* p, int64_t nnz, spgemm_stream_t stream) {
  if (!p || nnz < 0) return SPGEMM_ERR_INVALID_ARG;
  if (nnz >= (1ll << 31)) return SPGEMM_ERR_INDEX_OVERFLOW;
  // split rows take their per-window offsets from the symbolic pass
  if (p->sp.heavy_bin < sg::NBINS && p->sp.hcap > 0) return SPGEMM_ERR_NOT_READY;
  cudaStream_t st = (cudaStream_t)stream;
  spgemm_status s = read_stats(p, st);  // rows per path, and any error of the analysis
  if (s != SPGEMM_OK) return s;
  s = from_err_word(p->host_st.err);
  if (s != SPGEMM_OK) return s;
  p->nnz_c = nnz;
  p->symbolic_done = true;
  return SPGEMM_OK;
}

spgemm_status spgemm_numeric(spgemm_plan* p, const void* a_vals, const void* b_vals, const int32_t* c_row_ptr,
                             int32_t* c_col_idx, void* c_vals, spgemm_stream_t stream) {
  if (!p) return SPGEMM_ERR_INVALID_ARG;
  if (!p->symbolic_done) return SPGEMM_ERR_NOT_READY;
  if (!c_row_ptr) return SPGEMM_ERR_INVALID_ARG;
  if (p->nnz_c == 0) return SPGEMM_OK;
  if (!a_vals || !b_vals || !c_col_idx || !c_vals) return SPGEMM_ERR_INVALID_ARG;
  sg::LaunchCtx c = ctx_of(p, stream);
  const sg::RowInfo ri = rowinfo_of(p);
  cudaError_t e = sg::launch_numeric(c, p->A, p->B, ri, p->pb, p->tu, p->sp, p->opts.dtype, a_vals, b_vals,
                                     p->cursor, p->nxt, c_row_ptr, c_col_idx, c_vals, p->path_rows,
                                     (long long)p->host_st.rows_wide, p->host_st.hist, p->opts.semiring);
  return e == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

spgemm_status spgemm_plan_stats(spgemm_plan* p, spgemm_stream_t stream, int64_t* total_products,
                                int64_t* max_row_products, int64_t* rows_per_path) {
  if (!p) return SPGEMM_ERR_INVALID_ARG;
  spgemm_status s = read_stats(p, (cudaStream_t)stream);
  if (s != SPGEMM_OK) return s;
  if (total_products) *total_products = (int64_t)p->host_st.total_products;
  if (max_row_products) *max_row_products = (int64_t)p->host_st.max_products;
  if (rows_per_path)
    for (int q = 0; q < sg::NPATHS; ++q) rows_per_path[q] = p->path_rows[q];
  return SPGEMM_OK;
}

spgemm_status spgemm_plan_check(spgemm_plan* p, spgemm_stream_t stream) {
  if (!p) return SPGEMM_ERR_INVALID_ARG;
  uint32_t w = 0;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&w, &p->st->err, sizeof(w), cudaMemcpyDeviceToHost, st) != cudaSuccess) return SPGEMM_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SPGEMM_ERR_CUDA;
  return from_err_word(w);
}

spgemm_status spgemm_plan_set_profiling(spgemm_plan* p, int on) {
  if (!p) return SPGEMM_ERR_INVALID_ARG;
  if (on && !p->timers[0]) {
    for (auto& ev : p->timers)
      if (cudaEventCreate(&ev) != cudaSuccess) return SPGEMM_ERR_CUDA;
  }
  p->profiling = on != 0;
  return SPGEMM_OK;
}

spgemm_status spgemm_plan_kernel_times(spgemm_plan* p, float* ms, int n) {
  if (!p || !ms || n < 0) return SPGEMM_ERR_INVALID_ARG;
  for (int t = 0; t < n; ++t) {
    ms[t] = 0.0f;
    if (t >= sg::NTIMERS || !p->timer_used[t] || !p->timers[0]) continue;
    if (cudaEventSynchronize(p->timers[2 * t + 1]) != cudaSuccess) return SPGEMM_ERR_CUDA;
    if (cudaEventElapsedTime(&ms[t], p->timers[2 * t], p->timers[2 * t + 1]) != cudaSuccess) return SPGEMM_ERR_CUDA;
  }
  return SPGEMM_OK;
}

spgemm_status spgemm_plan_launches(spgemm_plan* p, int64_t* launches) {
  if (!p || !launches) return SPGEMM_ERR_INVALID_ARG;
  *launches = p->launches;
  return SPGEMM_OK;
}

spgemm_status spgemm_backward(spgemm_plan* p, const void* a_vals, const void* b_vals, const int32_t* c_row_ptr,
                              const int32_t* c_col_idx, const void* dc_vals, void* da_vals, void* db_vals,
                              spgemm_stream_t stream) {
  if (!p) return SPGEMM_ERR_INVALID_ARG;
  if (!p->symbolic_done || !p->at_rp) return SPGEMM_ERR_NOT_READY;
  if (!da_vals && !db_vals) return SPGEMM_OK;
  if (!c_row_ptr || (p->nnz_c > 0 && (!c_col_idx || !dc_vals))) return SPGEMM_ERR_INVALID_ARG;
  if ((da_vals && p->B.nnz > 0 && !b_vals) || (db_vals && p->A.nnz > 0 && !a_vals)) return SPGEMM_ERR_INVALID_ARG;
  sg::LaunchCtx c = ctx_of(p, stream);
  cudaError_t e = cudaSuccess;
  // rows outside the plan's range keep their dA; zero nothing else
  if (db_vals && p->B.nnz > 0)
    e = cudaMemsetAsync(db_vals, 0, (size_t)p->B.nnz * (p->opts.dtype == SPGEMM_F32 ? 4 : 8), c.stream);
  if (e == cudaSuccess)
    e = sg::launch_backward(c, p->opts.dtype, p->A, p->B, p->row_begin, p->mloc, a_vals, b_vals, p->a_row, p->b_row,
                            p->at_rp, p->at_ci, p->at_src, c_row_ptr, c_col_idx, dc_vals, da_vals, db_vals);
  return e == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

spgemm_status spgemm_transpose_workspace_size(int64_t nrows, int64_t ncols, int64_t nnz, size_t* bytes) {
  if (!bytes || nrows < 0 || ncols < 0 || nnz < 0) return SPGEMM_ERR_INVALID_ARG;
  if (nnz >= (1ll << 31) || ncols >= (1ll << 31) - 1) return SPGEMM_ERR_INDEX_OVERFLOW;
  size_t tmp, table, part;
  size_t off = align_up(sizeof(sg::DevStats));
  off = align_up(off + sizeof(int32_t) * (size_t)nnz);  // source positions if the caller wants none
  *bytes = transpose_layout(off, ncols, nnz, 8, &tmp, &table, &part);  // room for FP64 values
  return SPGEMM_OK;
}

spgemm_status spgemm_transpose(const spgemm_csr* M, int32_t dtype, int32_t* t_row_ptr, int32_t* t_col_idx,
                               void* t_vals, int32_t* t_src, void* workspace, size_t workspace_bytes,
                               spgemm_stream_t stream) {
  spgemm_status s;
  if ((s = check_csr(M)) != SPGEMM_OK) return s;
  if (!t_row_ptr || (M->nnz > 0 && !t_col_idx)) return SPGEMM_ERR_INVALID_ARG;
  if (dtype != SPGEMM_F64 && dtype != SPGEMM_F32) return SPGEMM_ERR_INVALID_ARG;
  if (t_vals && M->nnz > 0 && !M->vals) return SPGEMM_ERR_INVALID_ARG;
  size_t need = 0;
  if ((s = spgemm_transpose_workspace_size(M->nrows, M->ncols, M->nnz, &need)) != SPGEMM_OK) return s;
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace) % 16) return SPGEMM_ERR_WORKSPACE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPGEMM_ERR_CUDA;
  unsigned char* ws = (unsigned char*)workspace;
  sg::LaunchCtx c{};
  c.stream = (cudaStream_t)stream;
  c.nsm = sm_count_for(dev);
  c.st = (sg::DevStats*)ws;
  c.err = &c.st->err;
  size_t off = align_up(sizeof(sg::DevStats));
  int32_t* own_src = (int32_t*)(ws + off);
  off = align_up(off + sizeof(int32_t) * (size_t)M->nnz);
  size_t tmp, table, part;
  transpose_layout(off, M->ncols, M->nnz, 8, &tmp, &table, &part);
  int32_t* src = t_src ? t_src : own_src;
  const int vbytes = t_vals ? (dtype == SPGEMM_F32 ? 4 : 8) : 0;
  cudaError_t e = cudaMemsetAsync(c.st, 0, sizeof(sg::DevStats), c.stream);
  if (e == cudaSuccess)
    e = sg::launch_transpose(c, M->nrows, M->ncols, M->nnz, M->row_ptr, M->col_idx, t_row_ptr, t_col_idx, src,
                             vbytes, M->vals, t_vals, (int32_t*)(ws + tmp), (int32_t*)(ws + table),
                             (long long*)(ws + part));
  return e == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

static spgemm_status masked_impl(const spgemm_csr* A, const spgemm_csr* B, const spgemm_csr* M, int32_t dtype,
                                 int32_t semiring, bool use_mask_values, void* c_vals, spgemm_stream_t stream) {
  spgemm_status s;
  if ((s = check_csr(A)) != SPGEMM_OK) return s;
  if ((s = check_csr(B)) != SPGEMM_OK) return s;
  if ((s = check_csr(M)) != SPGEMM_OK) return s;
  if (A->ncols != B->nrows || M->nrows != A->nrows || M->ncols != B->ncols) return SPGEMM_ERR_DIM_MISMATCH;
  if (dtype != SPGEMM_F64 && dtype != SPGEMM_F32) return SPGEMM_ERR_INVALID_ARG;
  if (semiring < SPGEMM_PLUS_TIMES || semiring > SPGEMM_OR_AND) return SPGEMM_ERR_INVALID_ARG;
  if (M->nnz == 0) return SPGEMM_OK;
  if (!c_vals) return SPGEMM_ERR_INVALID_ARG;
  if ((A->nnz > 0 && !A->vals) || (B->nnz > 0 && !B->vals)) return SPGEMM_ERR_INVALID_ARG;
  if (use_mask_values && !M->vals) return SPGEMM_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPGEMM_ERR_CUDA;
  sg::LaunchCtx c{};
  c.stream = (cudaStream_t)stream;
  c.nsm = sm_count_for(dev);
  if (c.nsm <= 0) return SPGEMM_ERR_CUDA;
  const sg::Csr a{A->row_ptr, A->col_idx, A->nrows, A->ncols, A->nnz};
  const sg::Csr b{B->row_ptr, B->col_idx, B->nrows, B->ncols, B->nnz};
  const sg::Csr m{M->row_ptr, M->col_idx, M->nrows, M->ncols, M->nnz};
  const cudaError_t e = sg::launch_masked(c, dtype, semiring, a, b, m, A->vals, B->vals,
                                          use_mask_values ? M->vals : nullptr, c_vals);
  return e == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

spgemm_status spgemm_masked(const spgemm_csr* A, const spgemm_csr* B, const spgemm_csr* M, int32_t dtype,
                            int32_t use_mask_values, void* c_vals, spgemm_stream_t stream) {
  return masked_impl(A, B, M, dtype, SPGEMM_PLUS_TIMES, use_mask_values != 0, c_vals, stream);
}

spgemm_status spgemm_semiring(const spgemm_csr* A, const spgemm_csr* B, const spgemm_csr* M, int32_t dtype,
                              int32_t semiring, void* c_vals, spgemm_stream_t stream) {
  return masked_impl(A, B, M, dtype, semiring, false, c_vals, stream);
}

spgemm_status spgemm_transpose_check(void* workspace, spgemm_stream_t stream) {
  if (!workspace) return SPGEMM_ERR_INVALID_ARG;
  uint32_t w = 0;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&w, &((sg::DevStats*)workspace)->err, sizeof(w), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SPGEMM_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SPGEMM_ERR_CUDA;
  return from_err_word(w);
}

void spgemm_plan_destroy(spgemm_plan* p) { delete p; }

}  // extern "C"

struct spgemm_batch {
  int n = 0;
  int dtype = SPGEMM_F64;
  long long rows = 0, ks = 0, ncols = 0, a_nnz = 0, b_nnz = 0;
  std::vector<sg::BatchDesc> desc;
  sg::BatchDesc* d_desc = nullptr;
  int32_t *a_rp = nullptr, *a_ci = nullptr, *b_rp = nullptr, *b_ci = nullptr, *bounds = nullptr;
  void *a_v = nullptr, *b_v = nullptr;
  spgemm_plan* plan = nullptr;
  std::vector<int32_t> host_bounds;
  ~spgemm_batch() { spgemm_plan_destroy(plan); }
};

namespace {

struct BatchLayout {
  size_t desc, a_rp, a_ci, a_v, b_rp, b_ci, b_v, bounds, plan, total;
  spgemm_csr A, B;  // stacked shapes (pointers unset)
};

spgemm_status batch_layout(int n, const spgemm_csr* As, const spgemm_csr* Bs, const spgemm_opts& o,
                           BatchLayout* L, std::vector<sg::BatchDesc>* desc) {
  if (n < 0 || (n > 0 && (!As || !Bs))) return SPGEMM_ERR_INVALID_ARG;
  long long rows = 0, ks = 0, ncols = 0, an = 0, bn = 0;
  if (desc) desc->resize((size_t)n);
  for (int i = 0; i < n; ++i) {
    spgemm_status s;
    if ((s = check_csr(&As[i])) != SPGEMM_OK) return s;
    if ((s = check_csr(&Bs[i])) != SPGEMM_OK) return s;
    if (As[i].ncols != Bs[i].nrows) return SPGEMM_ERR_DIM_MISMATCH;
    if (desc) {
      sg::BatchDesc& D = (*desc)[(size_t)i];
      D.a_rp = As[i].row_ptr; D.a_ci = As[i].col_idx; D.a_v = As[i].vals;
      D.b_rp = Bs[i].row_ptr; D.b_ci = Bs[i].col_idx; D.b_v = Bs[i].vals;
      D.m = As[i].nrows; D.k = As[i].ncols; D.n = Bs[i].ncols;
      D.a_nnz = As[i].nnz; D.b_nnz = Bs[i].nnz;
      D.roff = rows; D.koff = ks; D.noff = ncols; D.aoff = an; D.boff = bn;
    }
    rows += As[i].nrows; ks += As[i].ncols; ncols += Bs[i].ncols; an += As[i].nnz; bn += Bs[i].nnz;
  }
  const long long lim = (1ll << 31) - 1;
  if (rows >= lim || ks >= lim || ncols >= lim || an >= lim || bn >= lim) return SPGEMM_ERR_INDEX_OVERFLOW;
  const size_t vb = o.dtype == SPGEMM_F32 ? 4 : 8;
  size_t off = 0;
  L->desc = off; off = align_up(off + sizeof(sg::BatchDesc) * (size_t)(n > 0 ? n : 1));
  L->a_rp = off; off = align_up(off + sizeof(int32_t) * (size_t)(rows + 1));
  L->a_ci = off; off = align_up(off + sizeof(int32_t) * (size_t)an);
  L->a_v = off; off = align_up(off + vb * (size_t)an);
  L->b_rp = off; off = align_up(off + sizeof(int32_t) * (size_t)(ks + 1));
  L->b_ci = off; off = align_up(off + sizeof(int32_t) * (size_t)bn);
  L->b_v = off; off = align_up(off + vb * (size_t)bn);
  L->bounds = off; off = align_up(off + sizeof(int32_t) * (size_t)(n + 1));
  L->plan = off;
  L->A = spgemm_csr{rows, ks, an, nullptr, nullptr, nullptr};
  L->B = spgemm_csr{ks, ncols, bn, nullptr, nullptr, nullptr};
  // the inner plan's size depends only on the stacked shapes
  L->A.row_ptr = (const int32_t*)16;
  L->B.row_ptr = (const int32_t*)16;
  if (an) L->A.col_idx = (const int32_t*)16;
  if (bn) L->B.col_idx = (const int32_t*)16;
  size_t pw = 0;
  spgemm_status s = spgemm_workspace_size(&L->A, &L->B, &o, &pw);
  if (s != SPGEMM_OK) return s;
  L->total = align_up(off + pw);
  return SPGEMM_OK;
}

}  // namespace

extern "C" {

spgemm_status spgemm_batch_workspace_size(int32_t n, const spgemm_csr* As, const spgemm_csr* Bs,
                                          const spgemm_opts* opts, size_t* bytes) {
  if (!bytes) return SPGEMM_ERR_INVALID_ARG;
  spgemm_opts o;
  if (opts) o = *opts; else spgemm_opts_default(&o);
  o.row_begin = 0;
  o.row_end = -1;
  BatchLayout L;
  spgemm_status s = batch_layout(n, As, Bs, o, &L, nullptr);
  if (s == SPGEMM_OK) *bytes = L.total;
  return s;
}

spgemm_status spgemm_batched(int32_t n, const spgemm_csr* As, const spgemm_csr* Bs, const spgemm_opts* opts,
                             void* workspace, size_t workspace_bytes, spgemm_stream_t stream,
                             spgemm_batch** batch) {
  if (!batch) return SPGEMM_ERR_INVALID_ARG;
  *batch = nullptr;
  spgemm_opts o;
  if (opts) o = *opts; else spgemm_opts_default(&o);
  if (o.dtype != SPGEMM_F64 && o.dtype != SPGEMM_F32) return SPGEMM_ERR_INVALID_ARG;
  o.row_begin = 0;
  o.row_end = -1;
  o.backward = 0;
  spgemm_batch* b = new (std::nothrow) spgemm_batch();
  if (!b) return SPGEMM_ERR_INTERNAL;
  BatchLayout L;
  spgemm_status s = batch_layout(n, As, Bs, o, &L, &b->desc);
  if (s != SPGEMM_OK) { delete b; return s; }
  if (!workspace || workspace_bytes < L.total || ((uintptr_t)workspace) % 16) { delete b; return SPGEMM_ERR_WORKSPACE; }
  for (int i = 0; i < n; ++i)
    if ((As[i].nnz > 0 && !As[i].vals) || (Bs[i].nnz > 0 && !Bs[i].vals)) { delete b; return SPGEMM_ERR_INVALID_ARG; }
  unsigned char* ws = (unsigned char*)workspace;
  b->n = n;
  b->dtype = o.dtype;
  b->rows = L.A.nrows; b->ks = L.A.ncols; b->ncols = L.B.ncols; b->a_nnz = L.A.nnz; b->b_nnz = L.B.nnz;
  b->d_desc = (sg::BatchDesc*)(ws + L.desc);
  b->a_rp = (int32_t*)(ws + L.a_rp); b->a_ci = (int32_t*)(ws + L.a_ci); b->a_v = ws + L.a_v;
  b->b_rp = (int32_t*)(ws + L.b_rp); b->b_ci = (int32_t*)(ws + L.b_ci); b->b_v = ws + L.b_v;
  b->bounds = (int32_t*)(ws + L.bounds);
  b->host_bounds.resize((size_t)n + 1);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { delete b; return SPGEMM_ERR_CUDA; }
  sg::LaunchCtx c{};
  c.stream = (cudaStream_t)stream;
  c.nsm = sm_count_for(dev);
  cudaError_t e = cudaSuccess;
  if (n > 0)
    e = cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(sg::BatchDesc) * (size_t)n, cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess)
    e = sg::launch_stack_structure(c, n, b->d_desc, b->rows, b->ks, b->a_rp, b->a_ci, b->b_rp, b->b_ci, b->a_nnz,
                                   b->b_nnz);
  if (n == 0 && e == cudaSuccess) {
    e = cudaMemsetAsync(b->a_rp, 0, sizeof(int32_t), c.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->b_rp, 0, sizeof(int32_t), c.stream);
  }
  if (e != cudaSuccess) { delete b; return SPGEMM_ERR_CUDA; }
  spgemm_csr A = L.A, B = L.B;
  A.row_ptr = b->a_rp; A.col_idx = b->a_nnz ? b->a_ci : nullptr; A.vals = b->a_v;
  B.row_ptr = b->b_rp; B.col_idx = b->b_nnz ? b->b_ci : nullptr; B.vals = b->b_v;
  s = spgemm_analyse(&A, &B, &o, ws + L.plan, workspace_bytes - L.plan, stream, &b->plan);
  if (s != SPGEMM_OK) { delete b; return s; }
  *batch = b;
  return SPGEMM_OK;
}

spgemm_status spgemm_batch_rows(spgemm_batch* b, int64_t* total_rows) {
  if (!b || !total_rows) return SPGEMM_ERR_INVALID_ARG;
  *total_rows = b->rows;
  return SPGEMM_OK;
}

spgemm_status spgemm_batch_symbolic(spgemm_batch* b, int32_t* c_row_ptr, int64_t* c_nnz, spgemm_stream_t stream) {
  if (!b || !c_row_ptr || !c_nnz) return SPGEMM_ERR_INVALID_ARG;
  int64_t total = 0;
  spgemm_status s = spgemm_symbolic(b->plan, c_row_ptr, &total, stream);
  if (s != SPGEMM_OK) return s;
  if (b->n > 0) {
    sg::LaunchCtx c = ctx_of(b->plan, stream);
    if (sg::launch_batch_bounds(c, b->n, b->d_desc, c_row_ptr, b->rows, b->bounds) != cudaSuccess) return SPGEMM_ERR_CUDA;
    if (cudaMemcpyAsync(b->host_bounds.data(), b->bounds, sizeof(int32_t) * (size_t)(b->n + 1), cudaMemcpyDeviceToHost,
                        c.stream) != cudaSuccess)
      return SPGEMM_ERR_CUDA;
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return SPGEMM_ERR_CUDA;
    for (int i = 0; i < b->n; ++i) c_nnz[i] = (int64_t)b->host_bounds[(size_t)i + 1] - b->host_bounds[(size_t)i];
  }
  c_nnz[b->n] = total;
  return SPGEMM_OK;
}

spgemm_status spgemm_batch_numeric(spgemm_batch* b, const int32_t* c_row_ptr, int32_t* c_col_idx, void* c_vals,
                                   spgemm_stream_t stream) {
  if (!b || !c_row_ptr) return SPGEMM_ERR_INVALID_ARG;
  if (!b->plan->symbolic_done) return SPGEMM_ERR_NOT_READY;
  if (b->plan->nnz_c == 0) return SPGEMM_OK;
  if (!c_col_idx || !c_vals) return SPGEMM_ERR_INVALID_ARG;
  sg::LaunchCtx c = ctx_of(b->plan, stream);
  if (sg::launch_stack_values(c, b->n, b->dtype, b->d_desc, b->a_v, b->b_v) != cudaSuccess) return SPGEMM_ERR_CUDA;
  spgemm_status s = spgemm_numeric(b->plan, b->a_v, b->b_v, c_row_ptr, c_col_idx, c_vals, stream);
  if (s != SPGEMM_OK) return s;
  if (sg::launch_unstack_columns(c, b->n, b->d_desc, c_row_ptr, c_col_idx) != cudaSuccess) return SPGEMM_ERR_CUDA;
  return SPGEMM_OK;
}

spgemm_status spgemm_batch_capture(spgemm_batch* b, const int32_t* c_row_ptr, int32_t* c_col_idx, void* c_vals,
                                   spgemm_stream_t stream, spgemm_graph_t* graph) {
  if (!b || !c_row_ptr || !graph || !stream) return SPGEMM_ERR_INVALID_ARG;
  *graph = nullptr;
  if (!b->plan->symbolic_done) return SPGEMM_ERR_NOT_READY;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return SPGEMM_ERR_CUDA;
  if (cs != cudaStreamCaptureStatusNone) return SPGEMM_ERR_INVALID_ARG;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SPGEMM_ERR_CUDA;
  spgemm_status s = spgemm_batch_numeric(b, c_row_ptr, c_col_idx, c_vals, stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (s != SPGEMM_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return s != SPGEMM_OK ? s : SPGEMM_ERR_CUDA;
  }
  *graph = (spgemm_graph_t)g;
  return SPGEMM_OK;
}

spgemm_status spgemm_graph_instantiate(spgemm_graph_t graph, spgemm_graph_exec_t* exec) {
  if (!graph || !exec) return SPGEMM_ERR_INVALID_ARG;
  cudaGraphExec_t ge = nullptr;
  if (cudaGraphInstantiate(&ge, (cudaGraph_t)graph, 0) != cudaSuccess) {
    *exec = nullptr;
    return SPGEMM_ERR_CUDA;
  }
  *exec = (spgemm_graph_exec_t)ge;
  return SPGEMM_OK;
}

spgemm_status spgemm_graph_launch(spgemm_graph_exec_t exec, spgemm_stream_t stream) {
  if (!exec) return SPGEMM_ERR_INVALID_ARG;
  return cudaGraphLaunch((cudaGraphExec_t)exec, (cudaStream_t)stream) == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

void spgemm_graph_destroy(spgemm_graph_t graph, spgemm_graph_exec_t exec) {
  if (exec) cudaGraphExecDestroy((cudaGraphExec_t)exec);
  if (graph) cudaGraphDestroy((cudaGraph_t)graph);
}

spgemm_status spgemm_batch_products_workspace_size(int32_t n, size_t* bytes) {
  if (!bytes || n < 0) return SPGEMM_ERR_INVALID_ARG;
  *bytes = align_up(sizeof(sg::BatchDesc) * (size_t)(n > 0 ? n : 1));
  return SPGEMM_OK;
}

spgemm_status spgemm_batch_products(int32_t n, const spgemm_csr* As, const spgemm_csr* Bs, int64_t* products,
                                    void* workspace, size_t workspace_bytes, spgemm_stream_t stream) {
  if (n < 0 || (n > 0 && (!As || !Bs || !products))) return SPGEMM_ERR_INVALID_ARG;
  if (n == 0) return SPGEMM_OK;
  size_t need = 0;
  spgemm_batch_products_workspace_size(n, &need);
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace) % 16) return SPGEMM_ERR_WORKSPACE;
  std::vector<sg::BatchDesc> desc((size_t)n);
  for (int i = 0; i < n; ++i) {
    spgemm_status s;
    if ((s = check_csr(&As[i])) != SPGEMM_OK) return s;
    if ((s = check_csr(&Bs[i])) != SPGEMM_OK) return s;
    if (As[i].ncols != Bs[i].nrows) return SPGEMM_ERR_DIM_MISMATCH;
    sg::BatchDesc& D = desc[(size_t)i];
    D = sg::BatchDesc{};
    D.a_rp = As[i].row_ptr; D.a_ci = As[i].col_idx; D.b_rp = Bs[i].row_ptr; D.b_ci = Bs[i].col_idx;
    D.m = As[i].nrows; D.k = As[i].ncols; D.n = Bs[i].ncols; D.a_nnz = As[i].nnz; D.b_nnz = Bs[i].nnz;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPGEMM_ERR_CUDA;
  sg::LaunchCtx c{};
  c.stream = (cudaStream_t)stream;
  c.nsm = sm_count_for(dev);
  // pageable source: the call returns once the descriptors are staged
  if (cudaMemcpyAsync(workspace, desc.data(), sizeof(sg::BatchDesc) * (size_t)n, cudaMemcpyHostToDevice,
                      c.stream) != cudaSuccess)
    return SPGEMM_ERR_CUDA;
  if (sg::launch_batch_products(c, n, (const sg::BatchDesc*)workspace, (long long*)products) != cudaSuccess)
    return SPGEMM_ERR_CUDA;
  return SPGEMM_OK;
}

spgemm_status spgemm_batch_waves(int32_t n, const spgemm_csr* As, const spgemm_csr* Bs, const int64_t* products,
                                 int64_t max_products, int64_t max_b_nnz, int32_t* wave_first, int32_t* nwaves) {
  if (n < 0 || !wave_first || !nwaves || (n > 0 && (!As || !Bs || !products))) return SPGEMM_ERR_INVALID_ARG;
  const long long lim = (1ll << 31) - 1;  // stacked counts must stay below this (int32 indices)
  const long long pmax = (max_products > 0 && max_products < lim) ? max_products : lim;
  const long long bmax = (max_b_nnz > 0 && max_b_nnz < lim) ? max_b_nnz : lim;
  long long rows = 0, ks = 0, ncols = 0, an = 0, bn = 0, pr = 0;
  int w = 0, count = 0;  // waves so far, instances in the open wave
  wave_first[0] = 0;
  for (int i = 0; i < n; ++i) {
    spgemm_status s;
    if ((s = check_csr(&As[i])) != SPGEMM_OK) return s;
    if ((s = check_csr(&Bs[i])) != SPGEMM_OK) return s;
    if (As[i].ncols != Bs[i].nrows) return SPGEMM_ERR_DIM_MISMATCH;
    if (products[i] < 0) return SPGEMM_ERR_INVALID_ARG;
    const bool fits = rows + As[i].nrows < lim && ks + As[i].ncols < lim && ncols + Bs[i].ncols < lim &&
                      an + As[i].nnz < lim && bn + Bs[i].nnz < lim && bn + Bs[i].nnz <= bmax &&
                      pr + products[i] <= pmax;
    if (!fits && count > 0) {  // close the open wave
      wave_first[++w] = i;
      rows = ks = ncols = an = bn = pr = 0;
      count = 0;
    }
    rows += As[i].nrows; ks += As[i].ncols; ncols += Bs[i].ncols; an += As[i].nnz; bn += Bs[i].nnz;
    pr += products[i];
    ++count;
    if (rows >= lim || ks >= lim || ncols >= lim || an >= lim || bn >= lim) return SPGEMM_ERR_INDEX_OVERFLOW;
  }
  if (count > 0) ++w;
  wave_first[w] = n;
  *nwaves = w;
  return SPGEMM_OK;
}

spgemm_plan* spgemm_batch_plan(spgemm_batch* b) { return b ? b->plan : nullptr; }

void spgemm_batch_destroy(spgemm_batch* b) { delete b; }

}  // extern "C"
