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

// Semirings (sum, product, zero): 0 plus-times (+, *, 0); 1 min-plus (min,
// +, +inf); 2 max-plus (max, +, -inf); 3 or-and (or, both nonzero, 0 with
// true written as 1).
template <int SR, typename T>
__device__ __forceinline__ T sr_zero() {
  if (SR == 1) return T(INFINITY);
  if (SR == 2) return T(-INFINITY);
  return T(0);
}

template <int SR, typename T>
__device__ __forceinline__ T sr_product(T a, T b) {
  if (SR == 0) return a * b;
  if (SR == 3) return (a != T(0) && b != T(0)) ? T(1) : T(0);
  return a + b;
}

__device__ __forceinline__ unsigned long long to_bits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ unsigned to_bits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ double from_bits(unsigned long long u) { return __longlong_as_double((long long)u); }
__device__ __forceinline__ float from_bits(unsigned u) { return __uint_as_float(u); }

// *p = min(*p, v) (MIN) or max(*p, v), shared or global memory, by
// compare-and-swap on the bit pattern (no FP64 min/max atomics exist).  A
// failed swap means another update improved the value first, so the loop
// ends after at most as many rounds as there are updates of *p; the bound
// is a guard that no input reaches.
template <bool MIN, typename T>
__device__ __forceinline__ void atomic_minmax(T* p, T v) {
  using U = decltype(to_bits(v));
  U* up = reinterpret_cast<U*>(p);
  U old = *reinterpret_cast<volatile U*>(up);
  for (int it = 0; it < CAS_RETRY_LIMIT; ++it) {
    const T cur = from_bits(old);
    if (MIN ? !(v < cur) : !(v > cur)) return;
    const U prev = atomicCAS(up, old, to_bits(v));
    if (prev == old) return;
    old = prev;
  }
}

// acc (+)= v in shared memory for semiring SR.
template <int SR, typename T>
__device__ __forceinline__ void sr_reduce_shared(T* p, T v) {
  if (SR == 0) red_add_shared(p, v);
  else if (SR == 1) atomic_minmax<true>(p, v);
  else if (SR == 2) atomic_minmax<false>(p, v);
  else if (v != T(0)) *p = T(1);  // every writer writes the same value
}

// out (+)= v in global memory for semiring SR; v equal to the zero is skipped.
template <int SR, typename T>
__device__ __forceinline__ void sr_reduce_global(T* p, T v) {
  if (v == sr_zero<SR, T>()) return;
  if (SR == 0) atomicAdd(p, v);
  else if (SR == 1) atomic_minmax<true>(p, v);
  else if (SR == 2) atomic_minmax<false>(p, v);
  else *p = T(1);
}

template <typename T, int SR>
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
        acc[t] = sr_zero<SR, T>();
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
          if (p >= 0) sr_reduce_shared<SR>(&acc[p], sr_product<SR>(oa, bv[bi]));
        } else if (ohi > olo) {
          const int p = find_in(M.ci, olo, ohi, j);
          if (p >= 0) sr_reduce_global<SR>(&out[p], sr_product<SR>(oa, bv[bi]));
        }
      }
    }
    if (staged) {
      __syncwarp();
      for (int t = lane; t < m1 - m0; t += 32) sr_reduce_global<SR>(&out[m0 + t], acc[t]);
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

// out[p] = the semiring's zero (+inf or -inf) for the nnz(M) entries.
template <typename T, int SR>
__global__ void __launch_bounds__(256) k_fill_zero(T* __restrict__ out, long long n) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
    out[p] = sr_zero<SR, T>();
}

template <typename T, int SR>
static cudaError_t masked_t(const LaunchCtx& c, const Csr& A, const Csr& B, const Csr& M, const T* av, const T* bv,
                            const T* mv, T* out) {
  const long long blocks = (M.nnz + 255) / 256;
  const int eg = (int)(blocks < 4096 ? blocks : 4096);
  cudaError_t e;
  if (SR == 1 || SR == 2) {
    k_fill_zero<T, SR><<<eg, 256, 0, c.stream>>>(out, M.nnz);
    count_launch(c);
    e = cudaGetLastError();
  } else {
    e = cudaMemsetAsync(out, 0, sizeof(T) * (size_t)M.nnz, c.stream);
  }
  if (e != cudaSuccess || A.nnz <= 0) return e;
  auto k = k_masked<T, SR>;
  const int occ = kernel_blocks_per_sm(k, MASK_WARPS * 32, 0);
  const int grid = persistent_grid((A.nnz + 31) / 32, MASK_WARPS, c.nsm, occ);
  k<<<grid, MASK_WARPS * 32, 0, c.stream>>>(A, B, M, av, bv, out);
  count_launch(c);
  if ((e = cudaGetLastError()) != cudaSuccess || SR != 0 || !mv) return e;
  k_scale<T><<<eg, 256, 0, c.stream>>>(out, mv, M.nnz);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_masked(const LaunchCtx& c, int dtype, int semiring, const Csr& A, const Csr& B, const Csr& M,
                          const void* av, const void* bv, const void* mv, void* out) {
  if (M.nrows <= 0 || M.nnz <= 0) return cudaSuccess;
  auto run = [&](auto* tag) -> cudaError_t {
    using T = std::remove_pointer_t<decltype(tag)>;
    const T* a = (const T*)av;
    const T* b = (const T*)bv;
    T* o = (T*)out;
    switch (semiring) {
      case 1: return masked_t<T, 1>(c, A, B, M, a, b, nullptr, o);
      case 2: return masked_t<T, 2>(c, A, B, M, a, b, nullptr, o);
      case 3: return masked_t<T, 3>(c, A, B, M, a, b, nullptr, o);
      default: return masked_t<T, 0>(c, A, B, M, a, b, (const T*)mv, o);
    }
  };
  return dtype == SPGEMM_F32 ? run((float*)nullptr) : run((double*)nullptr);
}

}  // namespace sg
