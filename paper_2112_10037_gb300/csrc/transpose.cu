// CSR transpose: the m x n matrix M in CSR becomes M^T (n x m) in CSR, which
// is M's CSC form (Sec. 2.1).  Entries of each output row are ordered by
// source row, so the result satisfies the sorted-columns precondition.
//
//  1. count the entries of every column (global atomics),
//  2. exclusive prefix sum of the counts -> row pointer of M^T,
//  3. scatter every entry to its column's range in arrival order, carrying
//     its source row (the new column index) and its source position,
//  4. sort each output row by source row (unique within a column): up to 32
//     entries in registers, up to 8192 entries by a block in shared memory,
//     longer rows through a shared-memory bitmap over their key range,
//  5. optionally gather the values through the source positions.
// The source positions let a caller move new values of the same structure
// (t_v[q] = v[t_src[q]]) without transposing again.
#include "launch_util.cuh"

namespace sg {

__global__ void __launch_bounds__(256) k_t_count(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                 long long m, long long n, int32_t* __restrict__ cnt, uint32_t* err) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
  const int lane = lane_id();
  for (long long i = w; i < m; i += nw) {
    for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
      const int c = ci[p];
      if (c < 0 || (long long)c >= n) { atomicOr(err, EB_UNSORTED); continue; }
      atomicAdd(&cnt[c], 1);
    }
  }
}

__global__ void __launch_bounds__(256) k_t_copy(const int32_t* __restrict__ a, int32_t* __restrict__ b, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    b[t] = a[t];
}

// fill[c] starts as t_rp[c]; each entry takes the next slot of its column.
__global__ void __launch_bounds__(256) k_t_scatter(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                   long long m, long long n, int32_t* __restrict__ fill,
                                                   int32_t* __restrict__ t_ci, int32_t* __restrict__ t_src) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
  const int lane = lane_id();
  for (long long i = w; i < m; i += nw) {
    for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
      const int c = ci[p];
      if (c < 0 || (long long)c >= n) continue;
      const int dst = atomicAdd(&fill[c], 1);
      t_ci[dst] = (int32_t)i;
      t_src[dst] = p;
    }
  }
}

// Rows of at most 32 entries: one warp per row, bitonic sort in registers.
__global__ void __launch_bounds__(256) k_t_sort_short(const int32_t* __restrict__ t_rp, long long n,
                                                      int32_t* __restrict__ t_ci, int32_t* __restrict__ t_src) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
  const int lane = lane_id();
  for (long long r = w; r < n; r += nw) {
    const int b = t_rp[r], len = t_rp[r + 1] - b;
    if (len <= 1 || len > 32) continue;
    int key = lane < len ? t_ci[b + lane] : INT_MAX;
    int src = lane < len ? t_src[b + lane] : 0;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        const int pk = __shfl_xor_sync(FULL, key, j);
        const int ps = __shfl_xor_sync(FULL, src, j);
        const bool up = (lane & k) == 0;
        const bool lower = (lane & j) == 0;
        if ((lower == up) ? (pk < key) : (pk > key)) {
          key = pk;
          src = ps;
        }
      }
    }
    if (lane < len) {
      t_ci[b + lane] = key;
      t_src[b + lane] = src;
    }
  }
}

constexpr int T_SMEM_SORT = 8192;

// Rows of 33..8192 entries: one block per row, bitonic sort of the row
// padded with +inf keys to a power of two in shared memory.
__global__ void __launch_bounds__(1024) k_t_sort_mid(const int32_t* __restrict__ t_rp, long long n,
                                                     int32_t* __restrict__ t_ci, int32_t* __restrict__ t_src) {
  extern __shared__ int t_smem[];  // 2 * T_SMEM_SORT ints
  int* sk = t_smem;
  int* ss = t_smem + T_SMEM_SORT;
  for (long long r = blockIdx.x; r < n; r += gridDim.x) {
    const int b = t_rp[r], len = t_rp[r + 1] - b;
    if (len <= 32 || len > T_SMEM_SORT) continue;
    int np2 = 64;
    while (np2 < len) np2 <<= 1;
    for (int x = threadIdx.x; x < np2; x += blockDim.x) {
      sk[x] = x < len ? t_ci[b + x] : INT_MAX;
      ss[x] = x < len ? t_src[b + x] : 0;
    }
    __syncthreads();
    for (int k = 2; k <= np2; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int x = threadIdx.x; x < np2; x += blockDim.x) {
          const int y = x ^ j;
          if (y > x) {
            const bool up = (x & k) == 0;
            const int kx = sk[x], ky = sk[y];
            if (up ? (kx > ky) : (kx < ky)) {
              sk[x] = ky;
              sk[y] = kx;
              const int t = ss[x];
              ss[x] = ss[y];
              ss[y] = t;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int x = threadIdx.x; x < len; x += blockDim.x) {
      t_ci[b + x] = sk[x];
      t_src[b + x] = ss[x];
    }
    __syncthreads();
  }
}

// Rows longer than 8192 entries (long columns of M): the row's keys (its
// source rows, distinct) are marked in a shared-memory bitmap, one window of
// T_BITS_WORDS * 32 keys at a time over the row's key range; a block-wide
// prefix sum of the window's per-word popcounts gives every marked key its
// rank, and the keys are written in ascending order to the scratch copy.
// Each key's source position is found again by a binary search for this
// column in the key's row of M (M's rows are sorted).  The scratch copy is
// then copied back.  Work per row: its entries, each with one binary search,
// plus its key span / 32 bitmap words.  This needs M's rows ascending and
// without repeated columns (the library's input precondition); a repeated
// column leaves fewer keys than entries and is reported as unsorted input.
constexpr int T_BITS_WORDS = 8192;   // 262,144 keys per window (32 KB)
constexpr int T_LONG_THREADS = 1024;

__global__ void __launch_bounds__(T_LONG_THREADS) k_t_sort_long(const int32_t* __restrict__ rp,
                                                                const int32_t* __restrict__ ci,
                                                                const int32_t* __restrict__ t_rp, long long n,
                                                                int32_t* __restrict__ t_ci, int32_t* __restrict__ t_src,
                                                                int32_t* __restrict__ tmp_ci,
                                                                int32_t* __restrict__ tmp_src, uint32_t* err) {
  constexpr int WPT = T_BITS_WORDS / T_LONG_THREADS;  // bitmap words per thread
  constexpr int NWARP = T_LONG_THREADS / 32;
  static_assert(NWARP == 32, "one warp scans the warp totals");
  __shared__ uint32_t bits[T_BITS_WORDS];
  __shared__ int s_warp[NWARP];
  __shared__ int s_kmin, s_kmax;
  const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  for (long long r = blockIdx.x; r < n; r += gridDim.x) {
    const int b = t_rp[r], len = t_rp[r + 1] - b;
    if (len <= T_SMEM_SORT) continue;  // the same for the whole block
    int mn = INT_MAX, mx = -1;
    for (int x = tid; x < len; x += T_LONG_THREADS) {
      const int k = t_ci[b + x];
      mn = min(mn, k);
      mx = max(mx, k);
    }
    mn = warp_min(mn);
    mx = warp_max(mx);
    if (tid == 0) {
      s_kmin = INT_MAX;
      s_kmax = -1;
    }
    __syncthreads();
    if (lane == 0) {
      atomicMin(&s_kmin, mn);
      atomicMax(&s_kmax, mx);
    }
    __syncthreads();
    const int kmin = s_kmin, kmax = s_kmax;
    int done = 0;  // keys placed by earlier windows
    for (long long w0 = kmin & ~31; w0 <= kmax; w0 += 32LL * T_BITS_WORDS) {
      for (int t = tid; t < T_BITS_WORDS; t += T_LONG_THREADS) bits[t] = 0u;
      __syncthreads();
      for (int x = tid; x < len; x += T_LONG_THREADS) {
        const long long d = (long long)t_ci[b + x] - w0;
        if (d >= 0 && d < 32LL * T_BITS_WORDS) atomicOr(&bits[d >> 5], 1u << (d & 31));
      }
      __syncthreads();
      uint32_t wv[WPT];
      int cnt = 0;
#pragma unroll
      for (int u = 0; u < WPT; ++u) {
        wv[u] = bits[tid * WPT + u];
        cnt += __popc(wv[u]);
      }
      const int incl = warp_incl_scan(cnt);
      if (lane == 31) s_warp[warp] = incl;
      __syncthreads();
      if (warp == 0) s_warp[lane] = warp_incl_scan(s_warp[lane]);
      __syncthreads();
      int pos = done + (warp > 0 ? s_warp[warp - 1] : 0) + incl - cnt;
      const int total = s_warp[NWARP - 1];
#pragma unroll
      for (int u = 0; u < WPT; ++u) {
        uint32_t v = wv[u];
        while (v) {
          const int bit = __ffs(v) - 1;
          v &= v - 1;
          const int key = (int)(w0 + 32LL * (tid * WPT + u) + bit);
          int lo = rp[key], hi = rp[key + 1];  // column r lies in row `key` of M
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (ci[mid] < (int)r) lo = mid + 1; else hi = mid;
          }
          tmp_ci[b + pos] = key;
          tmp_src[b + pos] = lo;
          ++pos;
        }
      }
      done += total;
      __syncthreads();  // bits and s_warp are reused by the next window
    }
    // a repeated column in a row of M marks one bit for two entries, so fewer
    // keys than entries were placed (the rest of the row was not written)
    if (tid == 0 && done != len) atomicOr(err, EB_UNSORTED);
    for (int x = tid; x < len; x += T_LONG_THREADS) {
      t_ci[b + x] = tmp_ci[b + x];
      t_src[b + x] = tmp_src[b + x];
    }
    __syncthreads();
  }
}

template <typename V>
__global__ void __launch_bounds__(256) k_gather(const V* __restrict__ v, const int32_t* __restrict__ src,
                                                V* __restrict__ out, long long nnz) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nnz; t += (long long)gridDim.x * blockDim.x)
    out[t] = v[src[t]];
}

static int grid_cap(long long units, int per_block, int nsm, int per_sm = 8) {
  long long g = (units + per_block - 1) / per_block;
  const long long cap = (long long)nsm * per_sm;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_transpose(const LaunchCtx& c, long long m, long long n, long long nnz, const int32_t* rp,
                             const int32_t* ci, int32_t* t_rp, int32_t* t_ci, int32_t* t_src, int32_t* fill,
                             int32_t* tmp_ci, int32_t* tmp_src, long long* partials) {
  cudaError_t e = cudaMemsetAsync(t_rp, 0, sizeof(int32_t) * (size_t)(n + 1), c.stream);
  if (e != cudaSuccess) return e;
  if (m > 0 && nnz > 0) {
    k_t_count<<<grid_cap(m, 8, c.nsm), 256, 0, c.stream>>>(rp, ci, m, n, t_rp, c.err);
    count_launch(c);
  }
  if ((e = launch_scan(c, t_rp, n, partials, &c.st->scratch_total)) != cudaSuccess) return e;
  if (nnz == 0 || n == 0) return cudaGetLastError();
  k_t_copy<<<grid_cap(n, 256, c.nsm), 256, 0, c.stream>>>(t_rp, fill, n);
  count_launch(c);
  k_t_scatter<<<grid_cap(m, 8, c.nsm), 256, 0, c.stream>>>(rp, ci, m, n, fill, t_ci, t_src);
  count_launch(c);
  k_t_sort_short<<<grid_cap(n, 8, c.nsm), 256, 0, c.stream>>>(t_rp, n, t_ci, t_src);
  count_launch(c);
  const size_t mid_smem = 2 * T_SMEM_SORT * sizeof(int);
  if (kernel_blocks_per_sm(k_t_sort_mid, 1024, mid_smem) <= 0) return cudaErrorInvalidConfiguration;
  k_t_sort_mid<<<grid_cap(n, 1, c.nsm, 2), 1024, mid_smem, c.stream>>>(t_rp, n, t_ci, t_src);
  count_launch(c);
  k_t_sort_long<<<grid_cap(n, 1, c.nsm, 2), T_LONG_THREADS, 0, c.stream>>>(rp, ci, t_rp, n, t_ci, t_src, tmp_ci,
                                                                            tmp_src, c.err);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_gather(const LaunchCtx& c, int dtype, const void* v, const int32_t* src, void* out, long long nnz) {
  if (nnz <= 0) return cudaSuccess;
  const int g = grid_cap(nnz, 256, c.nsm, 16);
  if (dtype == SPGEMM_F32)
    k_gather<float><<<g, 256, 0, c.stream>>>((const float*)v, src, (float*)out, nnz);
  else
    k_gather<double><<<g, 256, 0, c.stream>>>((const double*)v, src, (double*)out, nnz);
  count_launch(c);
  return cudaGetLastError();
}

}  // namespace sg
