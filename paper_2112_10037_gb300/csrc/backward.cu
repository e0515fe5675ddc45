// Adjoint of C = A*B for a scalar loss L with dL/dC = dC given on C's
// pattern (the loss L = sum W .* C has dC = W):
//   dA(i,k) = sum_j dC(i,j) * B(k,j)   on the pattern of A   (dC * B^T sampled)
//   dB(k,j) = sum_i A(i,k) * dC(i,j)   on the pattern of B   (A^T * dC sampled)
// Every (i,k,j) with A(i,k), B(k,j) nonzero has C(i,j) in C's pattern, so
// each lookup of dC(i,j) succeeds; it is a binary search in the sorted row i
// of C.
//
// Work is cut into slabs of 32 consecutive outputs (nonzeros of A for dA,
// of B for dB), one warp per slab, so a power-law input spreads its long
// rows over many warps.  An output whose sum has few terms (at most 128) is
// summed by its own lane as a chain of fused multiply-adds; an output with
// more terms is summed by the whole warp -- lane l takes terms l, l+32, ...,
// each lane chains its own terms, and a fixed shuffle tree adds the 32
// partial sums.  Both orders are fixed, so the result is deterministic (the
// same bits on every run), and nothing is accumulated atomically.
#include "launch_util.cuh"

namespace sg {

// Sums of at most this many terms stay in one lane: with lanes of a slab
// summing up to this many terms each, their chains run side by side; a sum
// far longer than its neighbours' (a hub row) would hold the warp alone.
constexpr int GRAD_LANE_MAX = 128;

__device__ __forceinline__ int find_col(const int32_t* __restrict__ ci, int lo, int hi, int c) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (ci[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// out[q] = the row holding entry q (one warp per row), so the gradient
// kernels find an output's row with one load.
__global__ void __launch_bounds__(256) k_row_index(const int32_t* __restrict__ rp, long long nrows,
                                                   int32_t* __restrict__ out) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
  const int lane = lane_id();
  for (long long r = w; r < nrows; r += nw)
    for (int q = rp[r] + lane; q < rp[r + 1]; q += 32) out[q] = (int32_t)r;
}

// Sum of the 32 lanes' partial sums in a fixed order (a butterfly tree).
template <typename T>
__device__ __forceinline__ T warp_sum_fixed(T v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
  return v;
}

// dA over the plan's rows [row_begin, row_begin + mloc): output e = (i,k) is
// the dot product of B(k,:) with dC(i,:).
template <typename T>
__global__ void __launch_bounds__(256) k_grad_a(Csr A, Csr B, const T* __restrict__ bv, long long row_begin,
                                                long long mloc, const int32_t* __restrict__ a_row,
                                                const int32_t* __restrict__ c_rp,
                                                const int32_t* __restrict__ c_ci, const T* __restrict__ dc,
                                                T* __restrict__ da, uint32_t* err) {
  const int lane = lane_id();
  const long long e_lo = A.rp[row_begin], e_hi = A.rp[row_begin + mloc];
  const long long nslab = (e_hi - e_lo + 31) >> 5;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
  for (long long s = w0; s < nslab; s += nw) {
    const long long e = e_lo + (s << 5) + lane;
    const bool have = e < e_hi;
    int k = 0, b0 = 0, b1 = 0, c0 = 0, c1 = 0;
    if (have) {
      const long long r = (long long)a_row[e] - row_begin;
      k = A.ci[e];
      b0 = B.rp[k];
      b1 = B.rp[k + 1];
      c0 = c_rp[r];
      c1 = c_rp[r + 1];
    }
    const bool wide = have && b1 - b0 > GRAD_LANE_MAX;
    // short sums: the lane's own chain, walking B(k,:) (ascending, so the
    // search range narrows)
    T acc = T(0);
    if (have && !wide) {
      int lo = c0;
      for (int q = b0; q < b1; ++q) {
        const int j = B.ci[q];
        const int pos = find_col(c_ci, lo, c1, j);
        if (pos < c1 && c_ci[pos] == j) {
          acc = fma(dc[pos], bv[q], acc);
          lo = pos + 1;
        } else {
          atomicOr(err, EB_INTERNAL);
        }
      }
    }
    // long sums: the whole warp on one output at a time
    unsigned wm = __ballot_sync(FULL, wide);
    while (wm) {
      const int L = __ffs(wm) - 1;
      wm &= wm - 1;
      const int lb0 = __shfl_sync(FULL, b0, L), lb1 = __shfl_sync(FULL, b1, L);
      const int lc0 = __shfl_sync(FULL, c0, L), lc1 = __shfl_sync(FULL, c1, L);
      T part = T(0);
      for (int q = lb0 + lane; q < lb1; q += 32) {
        const int j = B.ci[q];
        const int pos = find_col(c_ci, lc0, lc1, j);
        if (pos < lc1 && c_ci[pos] == j) part = fma(dc[pos], bv[q], part);
        else atomicOr(err, EB_INTERNAL);
      }
      const T tot = warp_sum_fixed(part);
      if (lane == L) acc = tot;
    }
    if (have) da[e] = acc;
  }
}

// dB: output q = (k,j) of B sums A(i,k) * dC(i,j) over the rows i of A (in
// the plan's range) with a nonzero in column k, i.e. over A^T(k,:), whose
// entries (t_ci: row i, t_src: position of A(i,k)) the plan keeps.
template <typename T>
__global__ void __launch_bounds__(256) k_grad_b(Csr B, const T* __restrict__ av, const int32_t* __restrict__ b_row,
                                                const int32_t* __restrict__ t_rp,
                                                const int32_t* __restrict__ t_ci, const int32_t* __restrict__ t_src,
                                                long long row_begin, long long row_end,
                                                const int32_t* __restrict__ c_rp, const int32_t* __restrict__ c_ci,
                                                const T* __restrict__ dc, T* __restrict__ db, uint32_t* err) {
  const int lane = lane_id();
  const long long nslab = (B.nnz + 31) >> 5;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
  for (long long s = w0; s < nslab; s += nw) {
    const long long q = (s << 5) + lane;
    const bool have = q < B.nnz;
    int j = 0, t0 = 0, t1 = 0;
    if (have) {
      const int k = b_row[q];
      j = B.ci[q];
      t0 = t_rp[k];
      t1 = t_rp[k + 1];
    }
    const bool wide = have && t1 - t0 > GRAD_LANE_MAX;
    T acc = T(0);
    if (have && !wide) {
      for (int t = t0; t < t1; ++t) {
        const long long i = t_ci[t];
        if (i < row_begin || i >= row_end) continue;  // rows outside the plan's range
        const int r = (int)(i - row_begin);
        const int c0 = c_rp[r], c1 = c_rp[r + 1];
        const int pos = find_col(c_ci, c0, c1, j);
        if (pos < c1 && c_ci[pos] == j) acc = fma(av[t_src[t]], dc[pos], acc);
        else atomicOr(err, EB_INTERNAL);
      }
    }
    unsigned wm = __ballot_sync(FULL, wide);
    while (wm) {
      const int L = __ffs(wm) - 1;
      wm &= wm - 1;
      const int lj = __shfl_sync(FULL, j, L);
      const int lt0 = __shfl_sync(FULL, t0, L), lt1 = __shfl_sync(FULL, t1, L);
      T part = T(0);
      for (int t = lt0 + lane; t < lt1; t += 32) {
        const long long i = t_ci[t];
        if (i < row_begin || i >= row_end) continue;
        const int r = (int)(i - row_begin);
        const int c0 = c_rp[r], c1 = c_rp[r + 1];
        const int pos = find_col(c_ci, c0, c1, lj);
        if (pos < c1 && c_ci[pos] == lj) part = fma(av[t_src[t]], dc[pos], part);
        else atomicOr(err, EB_INTERNAL);
      }
      const T tot = warp_sum_fixed(part);
      if (lane == L) acc = tot;
    }
    if (have) db[q] = acc;
  }
}

static int grid_for(long long slabs, int nsm) {
  long long g = (slabs + 7) / 8;  // 8 warps (slabs in flight) per block
  const long long cap = (long long)nsm * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_row_index(const LaunchCtx& c, const int32_t* rp, long long nrows, int32_t* out) {
  if (nrows <= 0) return cudaSuccess;
  k_row_index<<<grid_for(nrows / 8 + 1, c.nsm), 256, 0, c.stream>>>(rp, nrows, out);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_backward(const LaunchCtx& c, int dtype, const Csr& A, const Csr& B, long long row_begin,
                            long long mloc, const void* av, const void* bv, const int32_t* a_row,
                            const int32_t* b_row, const int32_t* t_rp, const int32_t* t_ci, const int32_t* t_src,
                            const int32_t* c_rp, const int32_t* c_ci, const void* dc, void* da, void* db) {
  if (da && mloc > 0) {
    const long long slabs = A.nnz / 32 + 1;  // an upper bound; the kernel reads the range's own extent
    if (dtype == SPGEMM_F32)
      k_grad_a<float><<<grid_for(slabs, c.nsm), 256, 0, c.stream>>>(A, B, (const float*)bv, row_begin, mloc, a_row, c_rp,
                                                                    c_ci, (const float*)dc, (float*)da, c.err);
    else
      k_grad_a<double><<<grid_for(slabs, c.nsm), 256, 0, c.stream>>>(A, B, (const double*)bv, row_begin, mloc, a_row,
                                                                     c_rp,
                                                                     c_ci, (const double*)dc, (double*)da, c.err);
    count_launch(c);
  }
  if (db && B.nnz > 0) {
    const long long slabs = (B.nnz + 31) / 32;
    if (dtype == SPGEMM_F32)
      k_grad_b<float><<<grid_for(slabs, c.nsm), 256, 0, c.stream>>>(B, (const float*)av, b_row, t_rp, t_ci, t_src,
                                                                     row_begin,
                                                                     row_begin + mloc, c_rp, c_ci, (const float*)dc,
                                                                     (float*)db, c.err);
    else
      k_grad_b<double><<<grid_for(slabs, c.nsm), 256, 0, c.stream>>>(B, (const double*)av, b_row, t_rp, t_ci,
                                                                      t_src,
                                                                      row_begin, row_begin + mloc, c_rp, c_ci,
                                                                      (const double*)dc, (double*)db, c.err);
    count_launch(c);
  }
  return cudaGetLastError();
}

}  // namespace sg
