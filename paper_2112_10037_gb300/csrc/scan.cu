// Exclusive prefix sum of the per-row sizes of C into C's row pointer.
//
// Three phases, no inter-block waiting: (1) each block reduces one tile,
// (2) one block scans the tile sums, (3) each block scans its tile again and
// adds its offset.  The sums are carried in int64; a total of 2^31 or more
// sets the overflow bit (row pointers are int32).  In place: c_rp[0..m-1]
// holds the row sizes on entry and the row starts on exit, c_rp[m] = nnz(C).
#include "internal.cuh"

namespace sg {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_PER_THREAD = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;  // 4096 rows per tile

size_t scan_partials_count(long long mloc) {
  return (size_t)((mloc + SCAN_TILE - 1) / SCAN_TILE) + 1;
}

// Block-wide exclusive scan of one int64 per thread; returns the block total.
__device__ __forceinline__ long long block_excl_scan(long long v, long long* total) {
  __shared__ long long s_warp[SCAN_THREADS / 32];
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  long long incl = warp_incl_scan(v);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    long long w = lane < SCAN_THREADS / 32 ? s_warp[lane] : 0;
    long long wi = warp_incl_scan(w);
    if (lane < SCAN_THREADS / 32) s_warp[lane] = wi - w;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  long long r = incl - v + s_warp[warp];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const int32_t* __restrict__ cnt, long long m,
                                                             long long* __restrict__ part) {
  const long long base = (long long)blockIdx.x * SCAN_TILE;
  long long v = 0;
#pragma unroll
  for (int j = 0; j < SCAN_PER_THREAD; ++j) {
    long long r = base + (long long)j * SCAN_THREADS + threadIdx.x;
    if (r < m) v += cnt[r];
  }
  v = warp_sum(v);
  __shared__ long long s_w[SCAN_THREADS / 32];
  if (lane_id() == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < SCAN_THREADS / 32; ++w) t += s_w[w];
    part[blockIdx.x] = t;
  }
}

// One block: exclusive scan of the tile sums in place, total to nnz_c.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_partials(long long* __restrict__ part, long long ntiles,
                                                               DevStats* st, int32_t* c_rp, long long m,
                                                               long long* total_out) {
  __shared__ long long s_carry;
  __shared__ long long s_tot;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (long long b = 0; b < ntiles; b += SCAN_THREADS) {
    long long i = b + threadIdx.x;
    long long v = i < ntiles ? part[i] : 0;
    long long ex = block_excl_scan(v, &s_tot);
    if (i < ntiles) part[i] = ex + s_carry;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += s_tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const long long total = s_carry;
    *total_out = total;
    if (total >= (1ll << 31)) atomicOr(&st->err, EB_OVERFLOW);
    c_rp[m] = (int32_t)(total < (1ll << 31) ? total : 0);
  }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(int32_t* __restrict__ c_rp, long long m,
                                                           const long long* __restrict__ part) {
  __shared__ long long s_tot;
  const long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_PER_THREAD;
  int32_t v[SCAN_PER_THREAD];
  long long sum = 0;
#pragma unroll
  for (int j = 0; j < SCAN_PER_THREAD; ++j) {
    long long r = base + j;
    v[j] = r < m ? c_rp[r] : 0;
    sum += v[j];
  }
  long long ex = block_excl_scan(sum, &s_tot) + part[blockIdx.x];
#pragma unroll
  for (int j = 0; j < SCAN_PER_THREAD; ++j) {
    long long r = base + j;
    if (r < m) c_rp[r] = (int32_t)ex;  // wraps only when the overflow bit is set
    ex += v[j];
  }
}

cudaError_t launch_scan(const LaunchCtx& c, int32_t* c_rp, long long m, long long* part, long long* total_out) {
  if (!total_out) total_out = &c.st->nnz_c;
  const long long ntiles = (m + SCAN_TILE - 1) / SCAN_TILE;
  timer_mark(c, T_SCAN, 0);
  if (ntiles > 0) {
    k_scan_reduce<<<(unsigned)ntiles, SCAN_THREADS, 0, c.stream>>>(c_rp, m, part);
    count_launch(c);
  }
  k_scan_partials<<<1, SCAN_THREADS, 0, c.stream>>>(part, ntiles, c.st, c_rp, m, total_out);
  count_launch(c);
  if (ntiles > 0) {
    k_scan_down<<<(unsigned)ntiles, SCAN_THREADS, 0, c.stream>>>(c_rp, m, part);
    count_launch(c);
  }
  timer_mark(c, T_SCAN, 1);
  return cudaGetLastError();
}

}  // namespace sg
