// Masked product C<M> = (A*B) .* M on the pattern of M: the sampled product
// behind triangle counting and Markov clustering, two of the SpGEMM
// applications Sec. 1 lists.  For entry p = (i,j) of M,
//   C[p] = M(i,j) * sum_k A(i,k) * B(k,j)     (factor 1 without M's values),
// 0 when no product reaches (i,j).  Every row runs the row-wise Gustavson
// order of Sec. 2.2 (A's entries of the row, each with its row of B) and
// keeps only the products whose column lies in M's row.
//
// One warp per row of M.  Up to MASK_CAP of the row's mask columns sit in
// shared memory with one accumulator each (longer rows of M are taken in
// slices of MASK_CAP columns, each slice re-reading the row's products).
// The row's products are formed in full 32-lane batches (a prefix sum over
// the B row lengths of each chunk of 32 A entries, then a search for each
// lane's owner), each product's column is searched in the slice (binary
// search in shared memory, after a range test), and a hit adds its rounded
// product A(i,k)*B(k,j) with a shared-memory reduction.  Output values are
// written once per slice, coalesced.
#include <type_traits>

#include "launch_util.cuh"

namespace sg {

constexpr int MASK_WARPS = 8;
constexpr int MASK_CAP = 512;   // mask columns per warp slice

template <typename T>
__global__ void __launch_bounds__(MASK_WARPS * 32)
k_masked(Csr A, Csr B, Csr M, const T* __restrict__ av, const T* __restrict__ bv, const T* __restrict__ mv,
         T* __restrict__ out) {
  __shared__ __align__(16) int s_col[MASK_WARPS][MASK_CAP];
  __shared__ __align__(16) T s_acc[MASK_WARPS][MASK_CAP];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  int* mc = s_col[warp];
  T* acc = s_acc[warp];
  const long long w = (long long)blockIdx.x * MASK_WARPS + warp;
  const long long nw = (long long)gridDim.x * MASK_WARPS;
  for (long long i = w; i < M.nrows; i += nw) {
    const int m0 = M.rp[i], m1 = M.rp[i + 1];
    if (m0 >= m1) continue;
    const int a0 = A.rp[i], a1 = A.rp[i + 1];
    for (int s0 = m0; s0 < m1; s0 += MASK_CAP) {
      const int ns = min(MASK_CAP, m1 - s0);
      for (int t = lane; t < ns; t += 32) {
        mc[t] = M.ci[s0 + t];
        acc[t] = T(0);
      }
      __syncwarp();
      const int jlo = mc[0], jhi = mc[ns - 1];
      for (int e0 = a0; e0 < a1; e0 += 32) {
        const int e = e0 + lane;
        int sb = 0, len = 0;
        T a = T(0);
        if (e < a1) {
          const int k = A.ci[e];
          if (k >= 0 && (long long)k < B.nrows) {  // a column of A out of range names no row of B
            sb = B.rp[k];
            len = B.rp[k + 1] - sb;
            a = av[e];
          }
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
          if (q < tot) {
            const int bi = os + q - oex;
            const int j = B.ci[bi];
            if (j >= jlo && j <= jhi) {
              int lo = 0, hi = ns - 1;  // mc[hi] >= j
              while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (mc[mid] < j) lo = mid + 1; else hi = mid;
              }
              if (mc[lo] == j) red_add_shared(&acc[lo], oa * bv[bi]);
            }
          }
        }
      }
      __syncwarp();
      for (int t = lane; t < ns; t += 32) {
        T v = acc[t];
        if (mv) v = v * mv[s0 + t];
        out[s0 + t] = v;
      }
      __syncwarp();
    }
  }
}

cudaError_t launch_masked(const LaunchCtx& c, int dtype, const Csr& A, const Csr& B, const Csr& M, const void* av,
                          const void* bv, const void* mv, void* out) {
  if (M.nrows <= 0 || M.nnz <= 0) return cudaSuccess;
  auto run = [&](auto* tag) -> cudaError_t {
    using T = std::remove_pointer_t<decltype(tag)>;
    auto k = k_masked<T>;
    const int occ = kernel_blocks_per_sm(k, MASK_WARPS * 32, 0);
    const int grid = persistent_grid(M.nrows, MASK_WARPS, c.nsm, occ);
    k<<<grid, MASK_WARPS * 32, 0, c.stream>>>(A, B, M, (const T*)av, (const T*)bv, (const T*)mv, (T*)out);
    count_launch(c);
    return cudaGetLastError();
  };
  return dtype == SPGEMM_F32 ? run((float*)nullptr) : run((double*)nullptr);
}

}  // namespace sg
