// Structure analysis: input validation, per-row product counts and column
// spans, and the counting sort of rows into bins by product count.
//
// The product count of row i is P_i = sum over the nonzeros A(i,k) of
// nnz(B(k,:)) -- the number of scalar-times-row products the row-wise
// Gustavson method (Sec. 2.2) forms for that row (the per-nonzero
// B_NUM_VEC of Table 1, summed).  Rows are later dispatched by P_i.
#include "internal.cuh"

namespace sg {

// One warp per row: column indices inside [0, ncols), strictly ascending;
// row_ptr non-decreasing and ending at nnz.
__global__ void k_validate(Csr M, uint32_t* err) {
  const int lane = lane_id();
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
  bool bad = false;
  if (w == 0 && lane == 0) {
    if (M.rp[0] != 0 || (long long)M.rp[M.nrows] != M.nnz) bad = true;
  }
  for (long long i = w; i < M.nrows; i += nw) {
    const int a0 = M.rp[i], a1 = M.rp[i + 1];
    if (a1 < a0 || a0 < 0 || (long long)a1 > M.nnz) { bad = true; continue; }
    for (int e = a0 + lane; e < a1; e += 32) {
      const int c = M.ci[e];
      if (c < 0 || (long long)c >= M.ncols) bad = true;
      if (e > a0 && M.ci[e - 1] >= c) bad = true;
    }
  }
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(err, EB_UNSORTED);
}

// Sum, minimum and maximum over aligned groups of G lanes (every lane of the
// warp calls them; G = 32 uses the single-instruction warp reductions).
template <int G, typename V>
__device__ __forceinline__ V group_sum(V v) {
  if constexpr (G == 32) {
    return warp_sum(v);
  } else {
#pragma unroll
    for (int d = G / 2; d >= 1; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
    return v;
  }
}
template <int G>
__device__ __forceinline__ int group_min(int v) {
  if constexpr (G == 32) {
    return warp_min(v);
  } else {
#pragma unroll
    for (int d = G / 2; d >= 1; d >>= 1) v = min(v, __shfl_xor_sync(FULL, v, d));
    return v;
  }
}
template <int G>
__device__ __forceinline__ int group_max(int v) {
  if constexpr (G == 32) {
    return warp_max(v);
  } else {
#pragma unroll
    for (int d = G / 2; d >= 1; d >>= 1) v = max(v, __shfl_xor_sync(FULL, v, d));
    return v;
  }
}

// G lanes per row of A (32: one warp; 8: four rows per warp, for matrices
// of short rows, where a warp per row leaves most lanes idle and each
// warp's rows form one long chain of dependent loads): P_i, the smallest and
// largest column any product of the row reaches (first and last column of
// each touched B row, since B's rows are sorted), histogram of bins, total
// and maximum P.
template <int G>
__global__ void __launch_bounds__(256) k_analyse(Csr A, Csr B, long long row_begin, long long mloc,
                                                 long long* __restrict__ prod, int* __restrict__ cmin,
                                                 int* __restrict__ cmax, DevStats* st) {
  static_assert(G == 8 || G == 16 || G == 32, "lanes per row");
  constexpr int RPW = 32 / G;  // rows per warp step
  __shared__ int s_hist[NBINS];
  __shared__ unsigned long long s_total, s_max;
  __shared__ unsigned s_wide;
  if (threadIdx.x < NBINS) s_hist[threadIdx.x] = 0;
  if (threadIdx.x == 0) { s_total = 0; s_max = 0; s_wide = 0; }
  if (block_skip(st)) return;  // validated input was rejected
  const int lane = lane_id();
  const int gl = lane & (G - 1), g = lane / G;
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
  unsigned long long my_total = 0, my_max = 0;
  unsigned my_wide = 0;
  bool bad = false;
  for (long long r0 = w * RPW; r0 < mloc; r0 += nw * RPW) {
    const long long r = r0 + g;
    const bool vr = r < mloc;
    const long long i = row_begin + r;
    int a0 = 0, a1 = 0;
    if (vr) {
      a0 = A.rp[i];
      a1 = A.rp[i + 1];
    }
    long long p = 0;
    int mn = INT_MAX, mx = -1;
    // four entries per lane per step, their dependent loads in flight
    // together (long rows of power-law matrices otherwise form the tail)
    for (int e0 = a0 + gl; e0 < a1; e0 += 4 * G) {
      int kk[4], ss[4], tt[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + G * u;
        kk[u] = e < a1 ? A.ci[e] : -1;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + G * u;
        ss[u] = tt[u] = 0;
        if (e < a1) {
          if (kk[u] < 0 || (long long)kk[u] >= B.nrows) {
            bad = true;
          } else {
            ss[u] = B.rp[kk[u]];
            tt[u] = B.rp[kk[u] + 1];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (tt[u] > ss[u]) {
          p += tt[u] - ss[u];
          mn = min(mn, B.ci[ss[u]]);
          mx = max(mx, B.ci[tt[u] - 1]);
        }
      }
    }
    p = group_sum<G>(p);
    mn = group_min<G>(mn);
    mx = group_max<G>(mx);
    if (vr && gl == 0) {
      my_wide += a1 - a0 > 32 ? 1u : 0u;
      prod[r] = p;
      cmin[r] = mn;
      cmax[r] = mx;
      atomicAdd(&s_hist[bin_of(p)], 1);
      my_total += (unsigned long long)p;
      my_max = my_max > (unsigned long long)p ? my_max : (unsigned long long)p;
    }
  }
  if (gl == 0 && my_total) {
    atomicAdd(&s_total, my_total);
    atomicMax(&s_max, my_max);
  }
  if (gl == 0 && my_wide) atomicAdd(&s_wide, my_wide);
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(&st->err, EB_UNSORTED);
  __syncthreads();
  if (threadIdx.x < NBINS && s_hist[threadIdx.x]) atomicAdd(&st->hist[threadIdx.x], s_hist[threadIdx.x]);
  if (threadIdx.x == 0 && s_total) {
    atomicAdd(&st->total_products, s_total);
    atomicMax(&st->max_products, s_max);
  }
  if (threadIdx.x == 0 && s_wide) atomicAdd(&st->rows_wide, s_wide);
}

// Counting sort of the non-empty rows by bin, largest bin first.  Each block
// takes a contiguous chunk of rows: counts per bin in shared memory, reserves
// one range per bin with a single global atomic, then places its rows.
constexpr int SCATTER_ROWS = 4096;

__global__ void __launch_bounds__(256) k_bin_scatter(const long long* __restrict__ prod, long long mloc,
                                                     DevStats* st, int* __restrict__ rows) {
  __shared__ int s_start[NBINS];
  __shared__ int s_cnt[NBINS];
  __shared__ int s_base[NBINS];
  if (block_skip(st)) return;
  if (threadIdx.x < NBINS) {
    int b = threadIdx.x, acc = 0;
    for (int k = NBINS - 1; k > b; --k) acc += st->hist[k];
    s_start[b] = acc;
    s_cnt[b] = 0;
  }
  __syncthreads();
  const long long r0 = (long long)blockIdx.x * SCATTER_ROWS;
  const long long r1 = min(mloc, r0 + SCATTER_ROWS);
  for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const int b = bin_of(prod[r]);
    if (b) atomicAdd(&s_cnt[b], 1);
  }
  __syncthreads();
  if (threadIdx.x < NBINS) {
    const int b = threadIdx.x;
    s_base[b] = s_cnt[b] ? s_start[b] + atomicAdd(&st->fill[b], s_cnt[b]) : 0;
    s_cnt[b] = 0;
  }
  __syncthreads();
  for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const int b = bin_of(prod[r]);
    if (b) rows[s_base[b] + atomicAdd(&s_cnt[b], 1)] = (int)r;
  }
}

static int grid_for_warps(long long nwarps, int warps_per_block, int nsm);

// True (for the whole block) when win_lo > 0 and the analysis put no row in
// bins win_lo and above, i.e. no row takes a numeric window path and the
// window-run lists will never be read.
__device__ __forceinline__ bool no_window_rows(const DevStats* st, int win_lo) {
  __shared__ int s_none;
  if (threadIdx.x == 0) {
    int n = 0;
    for (int b = win_lo > 0 ? win_lo : NBINS; b < NBINS; ++b) n += st->hist[b];
    s_none = win_lo > 0 && n == 0;
  }
  __syncthreads();
  return s_none != 0;
}

// Window-run lists of B (see SplitInfo), at two window widths (shifts s1
// and s2) from one read of B: pass 1 counts the runs of each row (plus its
// sentinel), an exclusive scan turns counts into run pointers, pass 2 writes
// (window id, first position) of every run.  One warp per row; a run starts
// where the window id differs from the previous entry's.  A null second list
// is skipped.  With no row in a window bin (win_lo, see no_window_rows) the
// counts are written as zeros and the lists stay unbuilt.
__global__ void __launch_bounds__(256) k_runs_count(Csr B, int s1, int32_t* __restrict__ rr1, int s2,
                                                    int32_t* __restrict__ rr2, const DevStats* st, int win_lo) {
  if (block_skip(st)) return;
  if (no_window_rows(st, win_lo)) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < B.nrows;
         k += (long long)gridDim.x * blockDim.x) {
      rr1[k] = 0;
      if (rr2) rr2[k] = 0;
    }
    return;
  }
  const int lane = lane_id();
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
  for (long long k = w; k < B.nrows; k += nw) {
    const int rs = B.rp[k], re = B.rp[k + 1];
    int n1 = 0, n2 = 0;
    for (int base = rs; base < re; base += 128) {  // 4 chunks of loads in flight per step
      int c[4], pc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = base + 32 * u + lane;
        c[u] = idx < re ? B.ci[idx] : 0;
        pc[u] = (idx < re && idx > rs) ? B.ci[idx - 1] : -1;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = base + 32 * u + lane;
        const bool in = idx < re;
        const bool b1 = in && (idx == rs || (pc[u] >> s1) != (c[u] >> s1));
        const bool b2 = in && (idx == rs || (pc[u] >> s2) != (c[u] >> s2));
        n1 += __popc(__ballot_sync(FULL, b1));
        n2 += __popc(__ballot_sync(FULL, b2));
      }
    }
    if (lane == 0) {
      rr1[k] = n1 + 1;
      if (rr2) rr2[k] = n2 + 1;
    }
  }
}

__device__ __forceinline__ void runs_fill_row(const Csr& B, int k, int shift, const int32_t* __restrict__ rr,
                                              int2* __restrict__ runs) {
  const int lane = lane_id();
  const int rs = B.rp[k], re = B.rp[k + 1];
  int pos = rr[k];
  for (int base = rs; base < re; base += 128) {  // 4 chunks of loads in flight per step
    int c[4], pc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + 32 * u + lane;
      c[u] = idx < re ? B.ci[idx] : 0;
      pc[u] = (idx < re && idx > rs) ? B.ci[idx - 1] : -1;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + 32 * u + lane;
      const int wid = c[u] >> shift;
      const bool start = idx < re && (idx == rs || (pc[u] >> shift) != wid);
      const unsigned m = __ballot_sync(FULL, start);
      if (start) runs[pos + __popc(m & lanemask_lt())] = make_int2(wid, idx);
      pos += __popc(m);
    }
  }
  if (lane == 0) runs[rr[k + 1] - 1] = make_int2(INT_MAX, re);
}

__global__ void __launch_bounds__(256) k_runs_fill(Csr B, int s1, const int32_t* __restrict__ rr1,
                                                   int2* __restrict__ runs1, int s2, const int32_t* __restrict__ rr2,
                                                   int2* __restrict__ runs2, const DevStats* st, int win_lo) {
  if (block_skip(st)) return;
  if (no_window_rows(st, win_lo)) return;
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
  for (long long k = w; k < B.nrows; k += nw) {
    runs_fill_row(B, (int)k, s1, rr1, runs1);
    if (runs2) runs_fill_row(B, (int)k, s2, rr2, runs2);
  }
}

cudaError_t launch_runs(const LaunchCtx& c, const Csr& B, const SplitInfo& sp, long long* partials, int win_lo) {
  if (!sp.rr || !sp.runs) return cudaSuccess;
  const bool two = sp.rrb && sp.runsb;
  if (B.nrows <= 0) {
    cudaError_t e = cudaMemsetAsync(sp.rr, 0, sizeof(int32_t), c.stream);
    if (e == cudaSuccess && two) e = cudaMemsetAsync(sp.rrb, 0, sizeof(int32_t), c.stream);
    return e;
  }
  const int grid = grid_for_warps(B.nrows, 8, c.nsm);
  k_runs_count<<<grid, 256, 0, c.stream>>>(B, sp.wf_shift, sp.rr, sp.wb_shift, two ? sp.rrb : nullptr, c.st,
                                           win_lo);
  count_launch(c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_scan(c, sp.rr, B.nrows, partials, &c.st->nruns);
  if (e == cudaSuccess && two) e = launch_scan(c, sp.rrb, B.nrows, partials, &c.st->nruns_b);
  if (e != cudaSuccess) return e;
  k_runs_fill<<<grid, 256, 0, c.stream>>>(B, sp.wf_shift, sp.rr, sp.runs, sp.wb_shift, two ? sp.rrb : nullptr,
                                          two ? sp.runsb : nullptr, c.st, win_lo);
  count_launch(c);
  return cudaGetLastError();
}

static int grid_for_warps(long long nwarps, int warps_per_block, int nsm) {
  long long blocks = (nwarps + warps_per_block - 1) / warps_per_block;
  long long cap = (long long)nsm * 8;
  if (blocks > cap) blocks = cap;
  return (int)(blocks < 1 ? 1 : blocks);
}

cudaError_t launch_validate(const LaunchCtx& c, const Csr& M) {
  k_validate<<<grid_for_warps(M.nrows > 0 ? M.nrows : 1, 8, c.nsm), 256, 0, c.stream>>>(M, c.err);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_analyse(const LaunchCtx& c, const Csr& A, const Csr& B, long long row_begin,
                           long long mloc, long long* prod, int* cmin, int* cmax, int* rows) {
  if (mloc <= 0) return cudaSuccess;
  timer_mark(c, T_ANALYSE, 0);
  // short rows on average (stencils, aggregation operators): 8 lanes per row
  if (A.nrows > 0 && A.nnz <= 12 * A.nrows)
    k_analyse<8><<<grid_for_warps((mloc + 3) / 4, 8, c.nsm), 256, 0, c.stream>>>(A, B, row_begin, mloc, prod,
                                                                                 cmin, cmax, c.st);
  else
    k_analyse<32><<<grid_for_warps(mloc, 8, c.nsm), 256, 0, c.stream>>>(A, B, row_begin, mloc, prod, cmin,
                                                                       cmax, c.st);
  count_launch(c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long blocks = (mloc + SCATTER_ROWS - 1) / SCATTER_ROWS;
  k_bin_scatter<<<(unsigned)blocks, 256, 0, c.stream>>>(prod, mloc, c.st, rows);
  count_launch(c);
  timer_mark(c, T_ANALYSE, 1);
  return cudaGetLastError();
}

}  // namespace sg
