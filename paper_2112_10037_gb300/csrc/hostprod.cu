// End-to-end product with host buffers: A and B in host memory in, C in host
// memory out, through the device.  Built on the library's own entry points:
// the inputs are copied into the caller's workspace, one plan analyses the
// whole product and sizes C (one symbolic pass); rows of C are independent
// (Sec. 2.2), so the numeric pass then runs in row ranges of about equal
// output -- plans derived with spgemm_analyse_rows that write their rows in
// place of the whole C staged on the device -- and each finished range is
// copied to the host on a second stream while the next ones compute.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"

struct spgemm_host_product {
  spgemm_opts opts{};
  long long m = 0, k = 0, n = 0, a_nnz = 0, b_nnz = 0;
  int32_t *a_rp = nullptr, *a_ci = nullptr, *b_rp = nullptr, *b_ci = nullptr, *c_rp = nullptr;
  void *a_v = nullptr, *b_v = nullptr;
  spgemm_plan* plan = nullptr;
  long long nnz_c = 0;
  std::vector<int32_t> host_rp;               // C's row pointer
  std::vector<long long> bounds;              // row ranges [bounds[r], bounds[r+1])
  std::vector<size_t> ws_off;                 // staging offsets of the range plans' workspaces
  size_t staging = 0;                         // staging bytes needed
  std::vector<float> timeline;                // 4 per range: numeric start/end, copy start/end (ms)
  ~spgemm_host_product() { spgemm_plan_destroy(plan); }
};

namespace {

constexpr size_t HP_ALIGN = 256;
inline size_t hp_align(size_t x) { return (x + HP_ALIGN - 1) & ~(HP_ALIGN - 1); }

struct HpLayout {
  size_t a_rp, a_ci, a_v, b_rp, b_ci, b_v, c_rp, plan, total;
};

bool hp_aliased(const spgemm_csr* A, const spgemm_csr* B) {
  return A == B || (A->row_ptr == B->row_ptr && A->col_idx == B->col_idx && A->vals == B->vals &&
                    A->nrows == B->nrows && A->ncols == B->ncols && A->nnz == B->nnz);
}

spgemm_status hp_check(const spgemm_csr* M) {
  if (!M || M->nrows < 0 || M->ncols < 0 || M->nnz < 0) return SPGEMM_ERR_INVALID_ARG;
  if (M->nrows >= (1ll << 31) - 1 || M->ncols >= (1ll << 31) - 1 || M->nnz >= (1ll << 31))
    return SPGEMM_ERR_INDEX_OVERFLOW;
  if (!M->row_ptr || (M->nnz > 0 && (!M->col_idx || !M->vals))) return SPGEMM_ERR_INVALID_ARG;
  return SPGEMM_OK;
}

spgemm_status hp_layout(const spgemm_csr* A, const spgemm_csr* B, const spgemm_opts& o, HpLayout* L) {
  spgemm_status s;
  if ((s = hp_check(A)) != SPGEMM_OK) return s;
  if ((s = hp_check(B)) != SPGEMM_OK) return s;
  if (A->ncols != B->nrows) return SPGEMM_ERR_DIM_MISMATCH;
  const size_t vb = o.dtype == SPGEMM_F32 ? 4 : 8;
  const bool al = hp_aliased(A, B);
  size_t off = 0;
  L->a_rp = off; off = hp_align(off + 4 * (size_t)(A->nrows + 1));
  L->a_ci = off; off = hp_align(off + 4 * (size_t)A->nnz);
  L->a_v = off; off = hp_align(off + vb * (size_t)A->nnz);
  if (al) {
    L->b_rp = L->a_rp; L->b_ci = L->a_ci; L->b_v = L->a_v;
  } else {
    L->b_rp = off; off = hp_align(off + 4 * (size_t)(B->nrows + 1));
    L->b_ci = off; off = hp_align(off + 4 * (size_t)B->nnz);
    L->b_v = off; off = hp_align(off + vb * (size_t)B->nnz);
  }
  L->c_rp = off; off = hp_align(off + 4 * (size_t)(A->nrows + 1));
  L->plan = off;
  // the plan's size depends only on the shapes (device pointers unset here)
  spgemm_csr dA{A->nrows, A->ncols, A->nnz, (const int32_t*)16, A->nnz ? (const int32_t*)16 : nullptr, nullptr};
  spgemm_csr dB{B->nrows, B->ncols, B->nnz, (const int32_t*)16, B->nnz ? (const int32_t*)16 : nullptr, nullptr};
  size_t pw = 0;
  if ((s = spgemm_workspace_size(&dA, &dB, &o, &pw)) != SPGEMM_OK) return s;
  L->total = hp_align(off + pw);
  return SPGEMM_OK;
}

spgemm_opts hp_opts(const spgemm_opts* opts) {
  spgemm_opts o;
  if (opts) o = *opts; else spgemm_opts_default(&o);
  o.row_begin = 0;
  o.row_end = -1;
  o.backward = 0;
  o.validate = 0;
  return o;
}

}  // namespace

extern "C" {

spgemm_status spgemm_host_product_workspace_size(const spgemm_csr* A, const spgemm_csr* B, const spgemm_opts* opts,
                                                 size_t* bytes) {
  if (!bytes) return SPGEMM_ERR_INVALID_ARG;
  const spgemm_opts o = hp_opts(opts);
  HpLayout L;
  spgemm_status s = hp_layout(A, B, o, &L);
  if (s == SPGEMM_OK) *bytes = L.total;
  return s;
}

spgemm_status spgemm_host_product_begin(const spgemm_csr* A, const spgemm_csr* B, const spgemm_opts* opts,
                                        int32_t chunks, void* workspace, size_t workspace_bytes,
                                        spgemm_stream_t stream, spgemm_host_product** product, int64_t* nnz_c) {
  if (!product || !nnz_c || chunks < 1) return SPGEMM_ERR_INVALID_ARG;
  *product = nullptr;
  const spgemm_opts o = hp_opts(opts);
  if (o.dtype != SPGEMM_F64 && o.dtype != SPGEMM_F32) return SPGEMM_ERR_INVALID_ARG;
  HpLayout L;
  spgemm_status s = hp_layout(A, B, o, &L);
  if (s != SPGEMM_OK) return s;
  if (!workspace || workspace_bytes < L.total || ((uintptr_t)workspace) % 16) return SPGEMM_ERR_WORKSPACE;
  spgemm_host_product* h = new (std::nothrow) spgemm_host_product();
  if (!h) return SPGEMM_ERR_INTERNAL;
  unsigned char* ws = (unsigned char*)workspace;
  const size_t vb = o.dtype == SPGEMM_F32 ? 4 : 8;
  h->opts = o;
  h->m = A->nrows; h->k = A->ncols; h->n = B->ncols; h->a_nnz = A->nnz; h->b_nnz = B->nnz;
  h->a_rp = (int32_t*)(ws + L.a_rp); h->a_ci = (int32_t*)(ws + L.a_ci); h->a_v = ws + L.a_v;
  h->b_rp = (int32_t*)(ws + L.b_rp); h->b_ci = (int32_t*)(ws + L.b_ci); h->b_v = ws + L.b_v;
  h->c_rp = (int32_t*)(ws + L.c_rp);
  cudaStream_t st = (cudaStream_t)stream;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return bytes == 0 || cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  bool ok = up(h->a_rp, A->row_ptr, 4 * (size_t)(A->nrows + 1)) && up(h->a_ci, A->col_idx, 4 * (size_t)A->nnz) &&
            up(h->a_v, A->vals, vb * (size_t)A->nnz);
  if (ok && !hp_aliased(A, B))
    ok = up(h->b_rp, B->row_ptr, 4 * (size_t)(B->nrows + 1)) && up(h->b_ci, B->col_idx, 4 * (size_t)B->nnz) &&
         up(h->b_v, B->vals, vb * (size_t)B->nnz);
  if (!ok) { delete h; return SPGEMM_ERR_CUDA; }
  const spgemm_csr dA{h->m, h->k, h->a_nnz, h->a_rp, h->a_nnz ? h->a_ci : nullptr, h->a_v};
  const spgemm_csr dB{h->k, h->n, h->b_nnz, h->b_rp, h->b_nnz ? h->b_ci : nullptr, h->b_v};
  s = spgemm_analyse(&dA, &dB, &o, ws + L.plan, workspace_bytes - L.plan, stream, &h->plan);
  if (s == SPGEMM_OK) s = spgemm_symbolic(h->plan, h->c_rp, nnz_c, stream);  // blocks
  if (s != SPGEMM_OK) { delete h; return s; }
  h->nnz_c = *nnz_c;
  h->host_rp.resize((size_t)h->m + 1);
  if (cudaMemcpyAsync(h->host_rp.data(), h->c_rp, 4 * (size_t)(h->m + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    delete h;
    return SPGEMM_ERR_CUDA;
  }
  // row ranges cut by output.  The copies run back to back once the first
  // range computed is done, so only that range's numeric pass is not hidden
  // under a copy: it is the last rows' range, about 1/(2 chunks) of nnz(C)
  // (the heaviest rows, whose numeric time per output is highest, sit at
  // the top of a power-law matrix), and finish computes the ranges from the
  // last to the first.  The other ranges share the rest of C equally; range r
  // ends at the first row whose row pointer reaches its target.
  const long long m = h->m, total = h->nnz_c;
  const long long nr = std::max(1ll, std::min((long long)chunks, m));
  const long long last = nr > 1 ? total / (2 * nr) : 0;
  h->bounds.push_back(0);
  for (long long r = 1; r < nr; ++r) {
    const long long target = (total - last) * r / (nr - 1);
    const long long cut = std::lower_bound(h->host_rp.begin(), h->host_rp.end(), (int32_t)target) - h->host_rp.begin();
    if (cut > h->bounds.back() && cut < m) h->bounds.push_back(cut);
  }
  if (m > h->bounds.back() || m == 0) h->bounds.push_back(m);
  // staging: C's columns and values, then the range plans' workspaces
  size_t off = hp_align(4 * (size_t)total);
  off = hp_align(off + vb * (size_t)total);
  for (size_t r = 0; r + 1 < h->bounds.size(); ++r) {
    size_t b = 0;
    s = spgemm_rows_workspace_size(h->plan, h->bounds[r], h->bounds[r + 1], &b);
    if (s != SPGEMM_OK) { delete h; return s; }
    h->ws_off.push_back(off);
    off = hp_align(off + b);
  }
  h->staging = off;
  *product = h;
  return SPGEMM_OK;
}

spgemm_status spgemm_host_product_staging_size(const spgemm_host_product* h, size_t* bytes) {
  if (!h || !bytes) return SPGEMM_ERR_INVALID_ARG;
  *bytes = h->staging;
  return SPGEMM_OK;
}

spgemm_status spgemm_host_product_finish(spgemm_host_product* h, int32_t* c_row_ptr, int32_t* c_col_idx,
                                         void* c_vals, void* staging, size_t staging_bytes, spgemm_stream_t stream,
                                         spgemm_stream_t copy_stream) {
  if (!h || !c_row_ptr || (h->nnz_c > 0 && (!c_col_idx || !c_vals))) return SPGEMM_ERR_INVALID_ARG;
  if (!staging || staging_bytes < h->staging || ((uintptr_t)staging) % 16) return SPGEMM_ERR_WORKSPACE;
  std::memcpy(c_row_ptr, h->host_rp.data(), 4 * h->host_rp.size());
  const size_t vb = h->opts.dtype == SPGEMM_F32 ? 4 : 8;
  unsigned char* sg_base = (unsigned char*)staging;
  int32_t* ci = (int32_t*)sg_base;
  unsigned char* v = sg_base + hp_align(4 * (size_t)h->nnz_c);
  cudaStream_t st = (cudaStream_t)stream;
  cudaStream_t cp = copy_stream ? (cudaStream_t)copy_stream : st;
  const size_t nr = h->bounds.size() - 1;
  h->timeline.assign(4 * nr, 0.0f);
  if (h->nnz_c == 0) return SPGEMM_OK;
  // range plans first (each sizes itself from the whole row pointer and
  // blocks once), then the numeric passes, each followed by its copy
  std::vector<spgemm_plan*> plans(nr, nullptr);
  std::vector<cudaEvent_t> ev(4 * nr + 1, nullptr);
  spgemm_status s = SPGEMM_OK;
  auto cleanup = [&]() {
    for (auto* p : plans) spgemm_plan_destroy(p);
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
  };
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) { cleanup(); return SPGEMM_ERR_CUDA; }
  for (size_t r = 0; r < nr && s == SPGEMM_OK; ++r) {
    size_t b = 0;
    s = spgemm_rows_workspace_size(h->plan, h->bounds[r], h->bounds[r + 1], &b);
    if (s == SPGEMM_OK)
      s = spgemm_analyse_rows(h->plan, h->bounds[r], h->bounds[r + 1], sg_base + h->ws_off[r], b, stream, &plans[r]);
    if (s == SPGEMM_OK) {
      const long long n = (long long)h->host_rp[h->bounds[r + 1]] - h->host_rp[h->bounds[r]];
      s = spgemm_plan_adopt_row_ptr(plans[r], n, stream);
    }
  }
  if (s != SPGEMM_OK) { cleanup(); return s; }
  cudaError_t e = cudaEventRecord(ev[4 * nr], st);  // origin of the timeline
  if (e == cudaSuccess && cp != st) e = cudaStreamWaitEvent(cp, ev[4 * nr], 0);
  for (size_t q = 0; q < nr && e == cudaSuccess && s == SPGEMM_OK; ++q) {
    const size_t r = nr - 1 - q;  // last range first
    const long long rb = h->bounds[r];
    const long long o = h->host_rp[rb], n = (long long)h->host_rp[h->bounds[r + 1]] - o;
    e = cudaEventRecord(ev[4 * r], st);
    if (e != cudaSuccess) break;
    s = spgemm_numeric(plans[r], h->a_v, h->b_v, h->c_rp + rb, ci, v, stream);
    if (s != SPGEMM_OK) break;
    if ((e = cudaEventRecord(ev[4 * r + 1], st)) != cudaSuccess) break;
    if (cp != st && (e = cudaStreamWaitEvent(cp, ev[4 * r + 1], 0)) != cudaSuccess) break;
    if ((e = cudaEventRecord(ev[4 * r + 2], cp)) != cudaSuccess) break;
    if (n > 0) {
      e = cudaMemcpyAsync(c_col_idx + o, ci + o, 4 * (size_t)n, cudaMemcpyDeviceToHost, cp);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync((unsigned char*)c_vals + vb * (size_t)o, v + vb * (size_t)o, vb * (size_t)n,
                            cudaMemcpyDeviceToHost, cp);
      if (e != cudaSuccess) break;
    }
    e = cudaEventRecord(ev[4 * r + 3], cp);
  }
  if (e == cudaSuccess && cp != st) e = cudaStreamSynchronize(cp);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && s == SPGEMM_OK) {
    for (size_t r = 0; r < nr && s == SPGEMM_OK; ++r) s = spgemm_plan_check(plans[r], stream);
    for (size_t q = 0; q < 4 * nr; ++q) cudaEventElapsedTime(&h->timeline[q], ev[4 * nr], ev[q]);
  }
  cleanup();
  if (e != cudaSuccess) return SPGEMM_ERR_CUDA;
  return s;
}

spgemm_status spgemm_host_product_timeline(const spgemm_host_product* h, float* ms, int32_t n) {
  if (!h || (!ms && n > 0) || n < 0) return SPGEMM_ERR_INVALID_ARG;
  for (int32_t q = 0; q < n; ++q) ms[q] = (size_t)q < h->timeline.size() ? h->timeline[(size_t)q] : 0.0f;
  return SPGEMM_OK;
}

spgemm_status spgemm_host_product_ranges(const spgemm_host_product* h, int32_t* nranges) {
  if (!h || !nranges) return SPGEMM_ERR_INVALID_ARG;
  *nranges = (int32_t)(h->bounds.size() - 1);
  return SPGEMM_OK;
}

void spgemm_host_product_destroy(spgemm_host_product* h) { delete h; }

}  // extern "C"
