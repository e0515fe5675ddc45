// Batched products C_i = A_i * B_i.
//
// The instances are stacked into one block-diagonal product
//   diag(A_1, ..., A_n) * diag(B_1, ..., B_n) = diag(A_1 B_1, ..., A_n B_n),
// so a single analysis bins the rows of all instances together and each pass
// (symbolic, numeric) is one persistent launch per path over that global
// (instance, row) work list, largest rows first.  Instance i's rows of A sit
// at row offset roff_i, its columns (rows of B) at koff_i, its columns of C at
// noff_i.  These kernels build the stacked index arrays once, gather the
// instances' values before each numeric pass, and map C's stacked column
// indices back to each instance's own.
#include "launch_util.cuh"

namespace sg {


// grid.y = instance; blocks along x stride over the instance's entries.
__global__ void __launch_bounds__(256) k_stack_structure(const BatchDesc* __restrict__ d, int32_t* __restrict__ a_rp,
                                                         int32_t* __restrict__ a_ci, int32_t* __restrict__ b_rp,
                                                         int32_t* __restrict__ b_ci, long long total_rows,
                                                         long long total_a_nnz, long long total_k,
                                                         long long total_b_nnz) {
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {  // closing row pointers
    a_rp[total_rows] = (int32_t)total_a_nnz;
    b_rp[total_k] = (int32_t)total_b_nnz;
  }
  const BatchDesc D = d[blockIdx.y];
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long st = (long long)gridDim.x * blockDim.x;
  for (long long r = t0; r < D.m; r += st) a_rp[D.roff + r] = (int32_t)(D.aoff + D.a_rp[r]);
  for (long long p = t0; p < D.a_nnz; p += st) a_ci[D.aoff + p] = (int32_t)(D.koff + D.a_ci[p]);
  for (long long r = t0; r < D.k; r += st) b_rp[D.koff + r] = (int32_t)(D.boff + D.b_rp[r]);
  for (long long q = t0; q < D.b_nnz; q += st) b_ci[D.boff + q] = (int32_t)(D.noff + D.b_ci[q]);
}

template <typename T>
__global__ void __launch_bounds__(256) k_stack_values(const BatchDesc* __restrict__ d, T* __restrict__ a_v,
                                                      T* __restrict__ b_v) {
  const BatchDesc D = d[blockIdx.y];
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long st = (long long)gridDim.x * blockDim.x;
  const T* av = (const T*)D.a_v;
  const T* bv = (const T*)D.b_v;
  for (long long p = t0; p < D.a_nnz; p += st) a_v[D.aoff + p] = av[p];
  for (long long q = t0; q < D.b_nnz; q += st) b_v[D.boff + q] = bv[q];
}

// C's rows of instance i hold stacked columns noff_i + j; give back j.
__global__ void __launch_bounds__(256) k_unstack_columns(const BatchDesc* __restrict__ d, const int32_t* __restrict__ c_rp,
                                                         int32_t* __restrict__ c_ci) {
  const BatchDesc D = d[blockIdx.y];
  const long long lo = c_rp[D.roff], hi = c_rp[D.roff + D.m];
  const int off = (int)D.noff;
  for (long long t = lo + blockIdx.x * (long long)blockDim.x + threadIdx.x; t < hi; t += (long long)gridDim.x * blockDim.x)
    c_ci[t] -= off;
}

static dim3 batch_grid(int n, int nsm) {
  int x = (nsm * 4 + n - 1) / (n > 0 ? n : 1);
  if (x < 1) x = 1;
  if (x > 256) x = 256;
  return dim3((unsigned)x, (unsigned)n, 1);
}

cudaError_t launch_stack_structure(const LaunchCtx& c, int n, const BatchDesc* d, long long total_rows,
                                   long long total_k, int32_t* a_rp, int32_t* a_ci, int32_t* b_rp, int32_t* b_ci,
                                   long long total_a_nnz, long long total_b_nnz) {
  if (n <= 0) return cudaSuccess;
  k_stack_structure<<<batch_grid(n, c.nsm), 256, 0, c.stream>>>(d, a_rp, a_ci, b_rp, b_ci, total_rows, total_a_nnz,
                                                                 total_k, total_b_nnz);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_stack_values(const LaunchCtx& c, int n, int dtype, const BatchDesc* d, void* a_v, void* b_v) {
  if (n <= 0) return cudaSuccess;
  if (dtype == SPGEMM_F32)
    k_stack_values<float><<<batch_grid(n, c.nsm), 256, 0, c.stream>>>(d, (float*)a_v, (float*)b_v);
  else
    k_stack_values<double><<<batch_grid(n, c.nsm), 256, 0, c.stream>>>(d, (double*)a_v, (double*)b_v);
  count_launch(c);
  return cudaGetLastError();
}

// c_rp at each instance's first row (and the end): per-instance nnz on the host.
__global__ void k_batch_bounds(const BatchDesc* __restrict__ d, int n, const int32_t* __restrict__ c_rp,
                               long long total_rows, int32_t* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x)
    out[i] = c_rp[i < n ? d[i].roff : total_rows];
}

cudaError_t launch_batch_bounds(const LaunchCtx& c, int n, const BatchDesc* d, const int32_t* c_rp, long long total_rows,
                                int32_t* out) {
  k_batch_bounds<<<(n + 256) / 256, 256, 0, c.stream>>>(d, n, c_rp, total_rows, out);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_unstack_columns(const LaunchCtx& c, int n, const BatchDesc* d, const int32_t* c_rp, int32_t* c_ci) {
  if (n <= 0) return cudaSuccess;
  k_unstack_columns<<<batch_grid(n, c.nsm), 256, 0, c.stream>>>(d, c_rp, c_ci);
  count_launch(c);
  return cudaGetLastError();
}

// Per-instance product counts: products[i] = sum over A_i's nonzeros (r,k)
// of nnz(B_i(k,:)).  grid.y = instance; blocks along x stride over A_i's
// nonzeros, reduce in the block and add once to products[i] (zeroed first).
__global__ void __launch_bounds__(256) k_batch_products(const BatchDesc* __restrict__ d,
                                                        unsigned long long* __restrict__ products) {
  __shared__ unsigned long long s_part[8];
  const BatchDesc D = d[blockIdx.y];
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long st = (long long)gridDim.x * blockDim.x;
  unsigned long long sum = 0;
  for (long long p = t0; p < D.a_nnz; p += st) {
    const int k = D.a_ci[p];
    sum += (unsigned long long)(D.b_rp[k + 1] - D.b_rp[k]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(FULL, sum, o);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_part[w];
    if (tot) atomicAdd(&products[blockIdx.y], tot);
  }
}

cudaError_t launch_batch_products(const LaunchCtx& c, int n, const BatchDesc* d, long long* products) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(products, 0, sizeof(long long) * (size_t)n, c.stream);
  if (e != cudaSuccess) return e;
  k_batch_products<<<batch_grid(n, c.nsm), 256, 0, c.stream>>>(d, (unsigned long long*)products);
  count_launch(c);
  return cudaGetLastError();
}

}  // namespace sg
