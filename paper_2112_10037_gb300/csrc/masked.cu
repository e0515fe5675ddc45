// Masked product C<M> = (A*B) .* M on the pattern of M: the sampled product
// behind triangle counting and Markov clustering, two of the SpGEMM
// applications Sec. 1 lists.  For entry p = (i,j) of M,
//   C[p] = M(i,j) * sum_k A(i,k) * B(k,j)     (factor 1 without M's values),
// 0 when no product reaches (i,j).  Every row runs the row-wise Gustavson
// order of Sec. 2.2 (A's entries of the row, each with its row of B) and
// keeps only the products whose column lies in M's row.
//
// Work is cut into units of 32 consecutive nonzeros of A (so rows of any
// length spread over many warps and the dense core of a power-law graph
// does not hold one warp for long); each lane finds its entry's row by a
// binary search over A's row pointer.  The unit's products are formed in
// full 32-lane batches (a prefix sum over the lanes' B row lengths, then a
// search for each lane's owner).  A product whose column lies in its row of
// M adds its rounded value A(i,k)*B(k,j) to that entry:
//  * when the whole unit lies in one row and that row of M has at most
//    MASK_CAP columns, the row's mask columns and one accumulator each are
//    staged in shared memory, each product's column is found there by binary
//    search, hits add with a shared-memory reduction, and the unit ends by
//    adding its nonzero accumulators to the output with global FP64
//    reductions (other units of the row add to the same entries);
//  * otherwise each product searches its row of M in global memory and a hit
//    adds straight to the output with a global FP64 reduction.
// The output is zeroed before and, with M's values, scaled by them after
// (the sum is finished before the factor, as in the definition).
#include <type_traits>

#include "launch_util.cuh"

namespace sg {

constexpr int MASK_WARPS = 8;
constexpr int MASK_CAP = 512;   // mask columns staged per warp

// Largest r with rp[r] <= e (the row holding position e), over rows [0, m).
__device__ __forceinline__ int row_of(const int32_t* __restrict__ rp, int m, int e) {
  int lo = 0, hi = m - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rp[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Position of column j in the ascending ci[lo, end), or -1.
__device__ __forceinline__ int find_in(const int32_t* __restrict__ ci, int lo, int end, int j) {
  int hi = end;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (ci[mid] < j) lo = mid + 1; else hi = mid;
  }
  return (lo < end && ci[lo] == j) ? lo : -1;
}

template <typename T>
__global__ void __launch_bounds__(MASK_WARPS * 32)
k_masked(Csr A, Csr B, Csr M, const T* __restrict__ av, const T* __restrict__ bv, T* __restrict__ out) {
  __shared__ __align__(16) int s_col[MASK_WARPS][MASK_CAP];
  __shared__ __align__(16) T s_acc[MASK_WARPS][MASK_CAP];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  int* mc = s_col[warp];
  T* acc = s_acc[warp];
  const long long units = (A.nnz + 31) / 32;
  const long long w = (long long)blockIdx.x * MASK_WARPS + warp;
  const long long nw = (long long)gridDim.x * MASK_WARPS;
  for (long long u = w; u < units; u += nw) {
    const int e = (int)(32 * u) + lane;
    const bool ve = e < A.nnz;
    int i = 0, sb = 0, len = 0;
    T a = T(0);
    if (ve) {
      i = row_of(A.rp, (int)A.nrows, e);
      const int k = A.ci[e];
      if (k >= 0 && (long long)k < B.nrows) {  // a column of A out of range names no row of B
        sb = B.rp[k];
        len = B.rp[k + 1] - sb;
        a = av[e];
      }
    }
    const int last = min(31, (int)(A.nnz - 32 * u) - 1);  // last valid lane
    const int i0 = __shfl_sync(FULL, i, 0), i1 = __shfl_sync(FULL, i, last);
    const int m0 = M.rp[i0], m1 = M.rp[i0 + 1];
    const bool staged = i0 == i1 && m1 - m0 <= MASK_CAP;  // warp-uniform
    if (staged) {
      for (int t = lane; t < m1 - m0; t += 32) {
        mc[t] = M.ci[m0 + t];
        acc[t] = T(0);
      }
      __syncwarp();
    }
    // per lane: its row's mask range (the owner's is read by shuffle)
    int mr0 = 0, mr1 = 0;
    if (ve && !staged) {
      mr0 = M.rp[i];
      mr1 = M.rp[i + 1];
    }
    const int incl = warp_incl_scan(len);
    const int tot = __shfl_sync(FULL, incl, 31);
    const int excl = incl - len;
    for (int q0 = 0; q0 < tot; q0 += 32) {
      const int q = q0 + lane;
      const int o = warp_owner(incl, q);
      const int os = __shfl_sync(FULL, sb, o);
      const int oex = __shfl_sync(FULL, excl, o);
      const T oa = __shfl_sync(FULL, a, o);
      const int olo = __shfl_sync(FULL, mr0, o), ohi = __shfl_sync(FULL, mr1, o);
      if (q < tot) {
        const int bi = os + q - oex;
        const int j = B.ci[bi];
        if (staged) {
          const int p = (m1 > m0) ? find_in(mc, 0, m1 - m0, j) : -1;
          if (p >= 0) red_add_shared(&acc[p], oa * bv[bi]);
        } else if (ohi > olo) {
          const int p = find_in(M.ci, olo, ohi, j);
          if (p >= 0) atomicAdd(&out[p], oa * bv[bi]);
        }
      }
    }
    if (staged) {
      __syncwarp();
      for (int t = lane; t < m1 - m0; t += 32) {
        const T v = acc[t];
        if (v != T(0)) atomicAdd(&out[m0 + t], v);
      }
      __syncwarp();
    }
  }
}

// out[p] *= mv[p] for the nnz(M) entries.
template <typename T>
__global__ void __launch_bounds__(256) k_scale(T* __restrict__ out, const T* __restrict__ mv, long long n) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
    out[p] = out[p] * mv[p];
}

cudaError_t launch_masked(const LaunchCtx& c, int dtype, const Csr& A, const Csr& B, const Csr& M, const void* av,
                          const void* bv, const void* mv, void* out) {
  if (M.nrows <= 0 || M.nnz <= 0) return cudaSuccess;
  auto run = [&](auto* tag) -> cudaError_t {
    using T = std::remove_pointer_t<decltype(tag)>;
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(T) * (size_t)M.nnz, c.stream);
    if (e != cudaSuccess || A.nnz <= 0) return e;
    auto k = k_masked<T>;
    const int occ = kernel_blocks_per_sm(k, MASK_WARPS * 32, 0);
    const int grid = persistent_grid((A.nnz + 31) / 32, MASK_WARPS, c.nsm, occ);
    k<<<grid, MASK_WARPS * 32, 0, c.stream>>>(A, B, M, (const T*)av, (const T*)bv, (T*)out);
    count_launch(c);
    if ((e = cudaGetLastError()) != cudaSuccess || !mv) return e;
    const long long blocks = (M.nnz + 255) / 256;
    k_scale<T><<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, c.stream>>>((T*)out, (const T*)mv, M.nnz);
    count_launch(c);
    return cudaGetLastError();
  };
  return dtype == SPGEMM_F32 ? run((float*)nullptr) : run((double*)nullptr);
}

}  // namespace sg
