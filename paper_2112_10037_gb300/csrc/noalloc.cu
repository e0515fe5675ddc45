// CSR transpose that allocates nothing: its scratch memory is a fixed,
// file-scope device array instead of a caller-provided workspace.
//
// Why: some callers cannot obtain device memory at the point where they need
// a transpose -- for example code running inside an allocator's own
// out-of-memory handling, code that must not call into the CUDA allocator
// (or PyTorch's caching allocator) because it runs under a lock that
// allocator also takes, or a long-running service that fixes its memory
// footprint at start-up and may not allocate afterwards.  Such callers pass
// only their inputs and outputs; the scratch comes from the array below.
//
// Limits and sharing: the array holds NOALLOC_SCRATCH_BYTES (8 MiB) on every
// GPU that loads this library, for the life of the process.  A call whose
// scratch would not fit is rejected with SPGEMM_ERR_WORKSPACE before any work
// is issued.  All calls on a device share the one array and it keeps the
// previous call's contents, so the parts that must start at zero are cleared
// at the start of every call; two calls whose GPU work overlaps (for example
// on two streams without ordering between them) race on the array.
#include <mutex>

#include "internal.cuh"

namespace sg {

constexpr size_t NOALLOC_SCRATCH_BYTES = 8u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

constexpr size_t NA_ALIGN = 256;
inline size_t na_align(size_t x) { return (x + NA_ALIGN - 1) & ~(NA_ALIGN - 1); }

struct NaLayout {
  size_t st, src, tmp, table, part, total;
};

// The source positions get scratch only when the caller passes no t_src;
// values (vbytes each, 0 without t_vals) travel through the scratch.
NaLayout na_layout(long long ncols, long long nnz, bool need_src, int vbytes) {
  const TransposeScratch s = transpose_scratch(ncols, nnz, vbytes);
  NaLayout L{};
  size_t off = 0;
  L.st = off; off = na_align(off + sizeof(DevStats));
  L.src = off;
  if (need_src) off = na_align(off + sizeof(int32_t) * (size_t)nnz);
  L.tmp = off; off = na_align(off + sizeof(int32_t) * s.tmp_ints);
  L.table = off; off = na_align(off + sizeof(int32_t) * s.table_ints);
  L.part = off; off = na_align(off + sizeof(long long) * s.part_count);
  L.total = off;
  return L;
}

// Device address of the scratch array, looked up once per device with that
// device current (in host code the array's name is only a stand-in).
std::mutex g_na_mu;
unsigned char* g_na_ptr[64] = {nullptr};
int g_na_sms[64] = {0};

cudaError_t na_setup(int dev, unsigned char** ptr, int* nsm) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = (unsigned char*)p;
    g_na_sms[dev] = n;
  }
  *ptr = g_na_ptr[dev];
  *nsm = g_na_sms[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace sg

extern "C" spgemm_status spgemm_transpose_noalloc(const spgemm_csr* M, int32_t dtype, int32_t* t_row_ptr,
                                                  int32_t* t_col_idx, void* t_vals, int32_t* t_src,
                                                  spgemm_stream_t stream) {
  using namespace sg;
  if (!M) return SPGEMM_ERR_INVALID_ARG;
  if (M->nrows < 0 || M->ncols < 0 || M->nnz < 0) return SPGEMM_ERR_INVALID_ARG;
  if (M->nrows >= (1ll << 31) - 1 || M->ncols >= (1ll << 31) - 1 || M->nnz >= (1ll << 31))
    return SPGEMM_ERR_INDEX_OVERFLOW;
  if (!M->row_ptr || (M->nnz > 0 && !M->col_idx)) return SPGEMM_ERR_INVALID_ARG;
  if (!t_row_ptr || (M->nnz > 0 && !t_col_idx)) return SPGEMM_ERR_INVALID_ARG;
  if (dtype != SPGEMM_F64 && dtype != SPGEMM_F32) return SPGEMM_ERR_INVALID_ARG;
  if (t_vals && M->nnz > 0 && !M->vals) return SPGEMM_ERR_INVALID_ARG;
  const int vbytes = t_vals ? (dtype == SPGEMM_F32 ? 4 : 8) : 0;
  const NaLayout L = na_layout(M->ncols, M->nnz, t_src == nullptr, vbytes);
  if (L.total > NOALLOC_SCRATCH_BYTES) return SPGEMM_ERR_WORKSPACE;  // does not fit the fixed scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPGEMM_ERR_CUDA;
  unsigned char* ws = nullptr;
  int nsm = 0;
  if (na_setup(dev, &ws, &nsm) != cudaSuccess) return SPGEMM_ERR_CUDA;
  LaunchCtx c{};
  c.stream = (cudaStream_t)stream;
  c.nsm = nsm;
  c.st = (DevStats*)(ws + L.st);
  c.err = &c.st->err;
  int32_t* src = t_src ? t_src : (int32_t*)(ws + L.src);
  // the stats word (error bits, scan total) must start at zero every call
  cudaError_t e = cudaMemsetAsync(c.st, 0, sizeof(DevStats), c.stream);
  if (e == cudaSuccess)
    e = launch_transpose(c, M->nrows, M->ncols, M->nnz, M->row_ptr, M->col_idx, t_row_ptr, t_col_idx, src,
                         vbytes, M->vals, t_vals, (int32_t*)(ws + L.tmp), (int32_t*)(ws + L.table),
                         (long long*)(ws + L.part));
  return e == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}
