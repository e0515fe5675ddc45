// Lane-per-row hash accumulator for rows of 17..64 products (bins 6..7):
// every row of a 3D 7-point stencil product (49 products, 25 columns) and of
// the Galerkin coarse product lands here.
//
// Row-wise Gustavson (Sec. 2.2): row i of C is the sum of the scaled rows
// A(i,k) * B(k,:), equal columns merged by adding their values (Algorithm
// 1), the row emitted with ascending columns.
//
// A warp takes 32 rows at once, one per lane.  Each lane owns a private
// open-addressing table of 64 slots in shared memory, laid out slot-major
// ([slot][lane]), so whatever slots the 32 lanes touch, each lane stays in
// its own bank: no bank conflicts and no atomics.  A lane walks its row's
// products one by one -- the first product of a column stores A(i,k)*B(k,j),
// later ones add with one fused multiply-add -- then compacts its occupied
// slots into a list (clearing the table for its next row) and writes each
// listed column at the position given by the number of smaller listed
// columns.  A warp-per-row table instead pays a shared-memory atomic per
// product, an FP64 reduction per repeated column (the FP64 pipe runs one
// such instruction per conflicting lane), and warp-wide gather and ranking
// work per row; here the FP64 pipe does one operation per product with all
// 32 lanes busy.
//
// A row of P <= 64 products has at most 64 distinct columns, so its table
// never overflows (the probe loop is bounded by the table size).
//
// In the numeric pass, rows with at most 8 nonzeros of A (the 7-point
// stencil's) skip the table: k_lane_merge stages the row's B rows in the
// same shared memory and merges them in column order.
#pragma once

#include "launch_util.cuh"
#include "semiring.cuh"

namespace sg {

constexpr int LANE_SLOTS = 64;     // table slots per lane (rows of at most 64 products)
constexpr int LANE_WARPS = 4;      // warps per block
constexpr int LANE_EMPTY = -1;

__device__ __forceinline__ unsigned lane_hash(int c) { return ((unsigned)c * 0x9E3779B1u) >> 26; }

// Slot of column j in the lane's table (claimed if absent; *fresh tells).
// keys: this warp's table base, slot-major.  -1 if the table is full of
// other columns (ruled out by the row's product count).
__device__ __forceinline__ int lane_probe(int* keys, int lane, int j, bool* fresh) {
  unsigned h = lane_hash(j);
  *fresh = false;
  for (int it = 0; it < LANE_SLOTS; ++it) {
    int* kp = &keys[h * 32 + lane];
    const int k = *kp;
    if (k == j) return (int)h;
    if (k == LANE_EMPTY) {
      *kp = j;
      *fresh = true;
      return (int)h;
    }
    h = (h + 1u) & (LANE_SLOTS - 1);
  }
  return -1;
}

// NUM = false: c_cnt[r] = distinct columns of row r.  NUM = true: C's
// columns and values at [c_rp[r], c_rp[r+1]).
template <bool NUM, typename T, int SR = SPGEMM_PLUS_TIMES>
__global__ void __launch_bounds__(LANE_WARPS * 32)
k_lane_rows(Csr A, Csr B, const T* __restrict__ av, const T* __restrict__ bv, RowInfo ri, const DevStats* st,
            int bin_lo, int bin_hi, int32_t* __restrict__ c_cnt, const int32_t* __restrict__ c_rp,
            int32_t* __restrict__ c_ci, T* __restrict__ c_v, uint32_t* err, int skip_upto) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_lb, s_le;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  // per warp: keys [64][32] int32, then (numeric) values [64][32] T
  const size_t per_warp = (size_t)LANE_SLOTS * 32 * (sizeof(int) + (NUM ? sizeof(T) : 0));
  int* keys = reinterpret_cast<int*>(smem_raw + warp * per_warp);
  T* vals = reinterpret_cast<T*>(smem_raw + warp * per_warp + (size_t)LANE_SLOTS * 32 * sizeof(int));
  for (int h = 0; h < LANE_SLOTS; ++h) keys[h * 32 + lane] = LANE_EMPTY;
  if (threadIdx.x == 0) bin_range(st, bin_lo, bin_hi, &s_lb, &s_le);
  if (block_skip(st)) return;
  const long long lb = s_lb, le = s_le;
  const long long gw = (long long)blockIdx.x * LANE_WARPS + warp;
  const long long nw = (long long)gridDim.x * LANE_WARPS;
  for (long long base = lb + gw * 32; base < le; base += nw * 32) {
    const long long idx = base + lane;
    if (idx < le) {
      const int r = ri.rows[idx];
      const long long i = ri.row_begin + r;
      const int a0 = A.rp[i], a1 = A.rp[i + 1];
      if (a1 - a0 <= skip_upto) continue;  // k_lane_merge took the row
      int nd = 0;     // distinct columns so far
      int np = 0;     // products so far
      bool over = false;
      for (int e = a0; e < a1; ++e) {
        const int k = A.ci[e];
        const T a = NUM ? av[e] : T(0);
        const int q0 = B.rp[k], q1 = B.rp[k + 1];
        // B(k,:) in groups of 8 entries whose loads are all issued before
        // the group's table updates (the updates depend on each other
        // through the table, the loads do not)
        for (int g = q0; g < q1; g += 8) {
          int jj[8];
          T bb[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            jj[u] = g + u < q1 ? B.ci[g + u] : -1;
            if (NUM) bb[u] = g + u < q1 ? bv[g + u] : T(0);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (jj[u] < 0) continue;
            bool fresh;
            const int h = lane_probe(keys, lane, jj[u], &fresh);
            ++np;
            if (h < 0) {
              over = true;
              continue;
            }
            if (fresh) ++nd;
            if (NUM) {
              T* vp = &vals[h * 32 + lane];
              *vp = fresh ? SrOps<T, SR>::mul(a, bb[u]) : SrOps<T, SR>::madd(a, bb[u], *vp);
            }
          }
        }
      }
      if (over || np > LANE_SLOTS) atomicOr(err, EB_INTERNAL);  // the row's bin rules this out
      if (!NUM) {
        c_cnt[r] = nd;
        for (int h = 0; h < LANE_SLOTS; ++h) keys[h * 32 + lane] = LANE_EMPTY;
      } else {
        // compact the occupied slots into slots [0, nd) of a list kept in
        // the same columns (read slot h before writing entry d <= h), and
        // clear the rest of the table
        int d = 0;
        for (int h = 0; h < LANE_SLOTS; ++h) {
          const int k = keys[h * 32 + lane];
          if (k != LANE_EMPTY) {
            const T v = vals[h * 32 + lane];
            keys[h * 32 + lane] = LANE_EMPTY;
            keys[d * 32 + lane] = k;  // d <= h
            vals[d * 32 + lane] = v;
            ++d;
          }
        }
        const int ob = c_rp[r], oe = c_rp[r + 1];
        if (ob + d != oe) atomicOr(err, EB_INTERNAL);
        // output position of a column: the listed columns smaller than it
        for (int x = 0; x < d; ++x) {
          const int kx = keys[x * 32 + lane];
          int r0 = 0, r1 = 0, r2 = 0, r3 = 0;  // four independent counts, so the loads overlap
          int y = 0;
          for (; y + 4 <= d; y += 4) {
            r0 += keys[y * 32 + lane] < kx;
            r1 += keys[(y + 1) * 32 + lane] < kx;
            r2 += keys[(y + 2) * 32 + lane] < kx;
            r3 += keys[(y + 3) * 32 + lane] < kx;
          }
          for (; y < d; ++y) r0 += keys[y * 32 + lane] < kx;
          const int rank = r0 + r1 + r2 + r3;
          const int o = ob + rank;
          if (o < oe) {
            c_ci[o] = kx;
            c_v[o] = vals[x * 32 + lane];
          }
        }
        for (int x = 0; x < d; ++x) keys[x * 32 + lane] = LANE_EMPTY;
      }
    }
  }
}

// Rows with at most LANE_MERGE_K nonzeros of A (every row of a 7-point
// stencil product): one lane per row stages its B rows (each sorted, at most
// 64 products in all: columns and values) in its slot-major shared-memory
// column, then merges them -- the next output column is the smallest head column, its
// value the products of the heads that hold it, each head advanced past it
// -- so the row comes out in column order with no table and no ranking.  The
// sums run in A's order, every product fused into the running sum from the
// semiring's identity (for plus-times the first product is a*b rounded,
// +0 where that product is exactly -0).
// (Measured on the 96^3 stencil: staging only the columns, for more warps
// per SM, and reading B's values from global memory was 13 % slower; one
// product per inner round, to issue fewer FP64 warp instructions, 14 %.)
constexpr int LANE_MERGE_K = 8;

template <typename T, int SR>
__global__ void __launch_bounds__(LANE_WARPS * 32)
k_lane_merge(Csr A, Csr B, const T* __restrict__ av, const T* __restrict__ bv, RowInfo ri, const DevStats* st,
             int bin_lo, int bin_hi, const int32_t* __restrict__ c_rp, int32_t* __restrict__ c_ci,
             T* __restrict__ c_v, uint32_t* err) {
  using Ops = SrOps<T, SR>;
  constexpr int K = LANE_MERGE_K;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_lb, s_le;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const size_t per_warp = (size_t)LANE_SLOTS * 32 * (sizeof(int) + sizeof(T));
  int* scol = reinterpret_cast<int*>(smem_raw + warp * per_warp);  // [slot][lane]
  T* sval = reinterpret_cast<T*>(smem_raw + warp * per_warp + (size_t)LANE_SLOTS * 32 * sizeof(int));
  if (threadIdx.x == 0) bin_range(st, bin_lo, bin_hi, &s_lb, &s_le);
  if (block_skip(st)) return;
  const long long lb = s_lb, le = s_le;
  const long long gw = (long long)blockIdx.x * LANE_WARPS + warp;
  const long long nw = (long long)gridDim.x * LANE_WARPS;
  for (long long base = lb + gw * 32; base < le; base += nw * 32) {
    const long long idx = base + lane;
    if (idx >= le) continue;
    const int r = ri.rows[idx];
    const long long i = ri.row_begin + r;
    const int a0 = A.rp[i], a1 = A.rp[i + 1];
    if (a1 - a0 > K) continue;  // k_lane_rows takes the row
    // stage B(k,:), the row's k-th nonzero, into slots [hs[k], he[k])
    int hs[K], he[K];
    T a[K];
    int q = 0;
    bool over = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      hs[k] = q;
      he[k] = q;
      a[k] = T(0);
      if (a0 + k < a1) {
        const int kk = A.ci[a0 + k];
        a[k] = av[a0 + k];
        const int s0 = B.rp[kk];
        int len = B.rp[kk + 1] - s0;
        if (q + len > LANE_SLOTS) {
          over = true;
          len = LANE_SLOTS - q;
        }
        for (int g = 0; g < len; g += 4) {
          int cc[4];
          T vv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            cc[u] = g + u < len ? B.ci[s0 + g + u] : 0;
            vv[u] = g + u < len ? bv[s0 + g + u] : T(0);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (g + u < len) {
              scol[(q + g + u) * 32 + lane] = cc[u];
              sval[(q + g + u) * 32 + lane] = vv[u];
            }
        }
        q += len;
        he[k] = q;
      }
    }
    int hc[K];  // head column of each staged row (INT_MAX when exhausted)
#pragma unroll
    for (int k = 0; k < K; ++k) hc[k] = hs[k] < he[k] ? scol[hs[k] * 32 + lane] : INT_MAX;
    const int ob = c_rp[r], oe = c_rp[r + 1];
    int o = ob;
    while (true) {
      int m = hc[0];
#pragma unroll
      for (int k = 1; k < K; ++k) m = min(m, hc[k]);
      if (m == INT_MAX) break;
      T acc = Ops::zero();
      bool any = false;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (hc[k] == m) {
          const T b = sval[hs[k] * 32 + lane];
          acc = Ops::madd(a[k], b, any ? acc : Ops::zero());  // one FP64 instruction per head test
          any = true;
          ++hs[k];
          hc[k] = hs[k] < he[k] ? scol[hs[k] * 32 + lane] : INT_MAX;
        }
      }
      if (o < oe) {
        c_ci[o] = m;
        c_v[o] = acc;
      }
      ++o;
    }
    if (over || o != oe) atomicOr(err, EB_INTERNAL);  // the row's bin and the symbolic count rule both out
  }
}

template <bool NUM, typename T>
constexpr size_t lane_rows_smem() {
  return (size_t)LANE_WARPS * LANE_SLOTS * 32 * (sizeof(int) + (NUM ? sizeof(T) : 0));
}

// Launch over the rows of bins [lo, hi] (rows: their number, -1 unknown).
// The numeric pass merges rows of at most LANE_MERGE_K nonzeros of A
// (k_lane_merge) and hashes the others; the symbolic pass hashes all.
template <bool NUM, typename T, int SR = SPGEMM_PLUS_TIMES>
static cudaError_t lane_rows(const LaunchCtx& c, const Csr& A, const Csr& B, const T* av, const T* bv,
                             const RowInfo& ri, int lo, int hi, int32_t* c_cnt, const int32_t* c_rp,
                             int32_t* c_ci, T* c_v, long long rows) {
  const size_t smem = lane_rows_smem<NUM, T>();
  if constexpr (NUM) {
    auto km = k_lane_merge<T, SR>;
    const size_t smem_m = smem;  // columns and values of 64 staged products per lane
    const int occm = kernel_blocks_per_sm(km, LANE_WARPS * 32, smem_m);
    if (occm <= 0) return cudaErrorInvalidConfiguration;
    const int gridm = persistent_grid(rows, LANE_WARPS * 32, c.nsm, occm);
    km<<<gridm, LANE_WARPS * 32, smem_m, c.stream>>>(A, B, av, bv, ri, c.st, lo, hi, c_rp, c_ci, c_v, c.err);
    count_launch(c);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  auto k = k_lane_rows<NUM, T, SR>;
  const int occ = kernel_blocks_per_sm(k, LANE_WARPS * 32, smem);
  if (occ <= 0) return cudaErrorInvalidConfiguration;
  const int grid = persistent_grid(rows, LANE_WARPS * 32, c.nsm, occ);
  k<<<grid, LANE_WARPS * 32, smem, c.stream>>>(A, B, av, bv, ri, c.st, lo, hi, c_cnt, c_rp, c_ci, c_v, c.err,
                                               NUM ? LANE_MERGE_K : -1);
  count_launch(c);
  return cudaGetLastError();
}

}  // namespace sg
