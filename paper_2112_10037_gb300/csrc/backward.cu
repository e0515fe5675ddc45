// Adjoint of C = A*B for a scalar loss L with dL/dC = dC given on C's
// pattern (the loss L = sum W .* C has dC = W):
//   dA(i,k) = sum_j dC(i,j) * B(k,j)   on the pattern of A   (dC * B^T sampled)
//   dB(k,j) = sum_i A(i,k) * dC(i,j)   on the pattern of B   (A^T * dC sampled)
// Every (i,k,j) with A(i,k), B(k,j) nonzero has C(i,j) in C's pattern, so
// each lookup of dC(i,j) succeeds; it is a binary search in the sorted row i
// of C.  Both kernels give each lane one output and run its sum as a chain of
// fused multiply-adds, so nothing is accumulated atomically and the result
// is deterministic.
#include "launch_util.cuh"

namespace sg {

__device__ __forceinline__ int find_col(const int32_t* __restrict__ ci, int lo, int hi, int c) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (ci[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// dA: one lane per nonzero (i,k) of A, walking B(k,:).
template <typename T>
__global__ void __launch_bounds__(256) k_grad_a(Csr A, Csr B, const T* __restrict__ bv, long long row_begin,
                                                long long mloc, const int32_t* __restrict__ c_rp,
                                                const int32_t* __restrict__ c_ci, const T* __restrict__ dc,
                                                T* __restrict__ da, uint32_t* err) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
  const int lane = lane_id();
  for (long long r = w; r < mloc; r += nw) {
    const long long i = row_begin + r;
    const int a0 = A.rp[i], a1 = A.rp[i + 1];
    const int c0 = c_rp[r], c1 = c_rp[r + 1];
    for (int e = a0 + lane; e < a1; e += 32) {
      const int k = A.ci[e];
      T acc = T(0);
      int lo = c0;
      for (int q = B.rp[k]; q < B.rp[k + 1]; ++q) {
        const int j = B.ci[q];
        const int pos = find_col(c_ci, lo, c1, j);  // B(k,:) ascends, so the search narrows
        if (pos < c1 && c_ci[pos] == j) {
          acc = fma(dc[pos], bv[q], acc);
          lo = pos + 1;
        } else {
          atomicOr(err, EB_INTERNAL);
        }
      }
      da[e] = acc;
    }
  }
}

// dB: one lane per entry (k,j) of B, walking A^T(k,:) = {(i, A(i,k))}.
template <typename T>
__global__ void __launch_bounds__(256) k_grad_b(Csr B, const T* __restrict__ av, const int32_t* __restrict__ t_rp,
                                                const int32_t* __restrict__ t_ci, const int32_t* __restrict__ t_src,
                                                long long row_begin, long long row_end,
                                                const int32_t* __restrict__ c_rp, const int32_t* __restrict__ c_ci,
                                                const T* __restrict__ dc, T* __restrict__ db, uint32_t* err) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
  const int lane = lane_id();
  for (long long k = w; k < B.nrows; k += nw) {
    const int b0 = B.rp[k], b1 = B.rp[k + 1];
    const int t0 = t_rp[k], t1 = t_rp[k + 1];
    for (int q = b0 + lane; q < b1; q += 32) {
      const int j = B.ci[q];
      T acc = T(0);
      for (int t = t0; t < t1; ++t) {
        const long long i = t_ci[t];
        if (i < row_begin || i >= row_end) continue;  // rows outside the plan's range
        const int r = (int)(i - row_begin);
        const int c0 = c_rp[r], c1 = c_rp[r + 1];
        const int pos = find_col(c_ci, c0, c1, j);
        if (pos < c1 && c_ci[pos] == j) acc = fma(av[t_src[t]], dc[pos], acc);
        else atomicOr(err, EB_INTERNAL);
      }
      db[q] = acc;
    }
  }
}

static int grid_for(long long warps, int nsm) {
  long long g = (warps + 7) / 8;
  const long long cap = (long long)nsm * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_backward(const LaunchCtx& c, int dtype, const Csr& A, const Csr& B, long long row_begin,
                            long long mloc, const void* av, const void* bv, const int32_t* t_rp,
                            const int32_t* t_ci, const int32_t* t_src, const int32_t* c_rp,
                            const int32_t* c_ci, const void* dc, void* da, void* db) {
  if (da && mloc > 0) {
    if (dtype == SPGEMM_F32)
      k_grad_a<float><<<grid_for(mloc, c.nsm), 256, 0, c.stream>>>(A, B, (const float*)bv, row_begin, mloc, c_rp,
                                                                   c_ci, (const float*)dc, (float*)da, c.err);
    else
      k_grad_a<double><<<grid_for(mloc, c.nsm), 256, 0, c.stream>>>(A, B, (const double*)bv, row_begin, mloc, c_rp,
                                                                    c_ci, (const double*)dc, (double*)da, c.err);
    count_launch(c);
  }
  if (db && B.nrows > 0) {
    if (dtype == SPGEMM_F32)
      k_grad_b<float><<<grid_for(B.nrows, c.nsm), 256, 0, c.stream>>>(B, (const float*)av, t_rp, t_ci, t_src, row_begin,
                                                                      row_begin + mloc, c_rp, c_ci, (const float*)dc,
                                                                      (float*)db, c.err);
    else
      k_grad_b<double><<<grid_for(B.nrows, c.nsm), 256, 0, c.stream>>>(B, (const double*)av, t_rp, t_ci, t_src,
                                                                       row_begin, row_begin + mloc, c_rp, c_ci,
                                                                       (const double*)dc, (double*)db, c.err);
    count_launch(c);
  }
  return cudaGetLastError();
}

}  // namespace sg
