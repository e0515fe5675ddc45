// Hash-accumulator path for rows of 17..128 products (bins 6..8).
//
// Row-wise Gustavson (Sec. 2.2): row i of C is the sum of the scaled rows
// A(i,k) * B(k,:); two entries of equal column merge by adding their values
// (Algorithm 1), and the row comes out with its columns ascending.
//
// One warp owns one row at a time and a table of H = 64*E slots in shared
// memory (E = ceil(P / 32) products per lane, so the table is at most half
// full).  Each product claims or finds its column's slot by linear probing
// with a 32-bit compare-and-swap on the key (multiplicative hash), and the
// numeric pass adds A(i,k) * B(k,j) into the slot's value.  The occupied
// slots are then compacted into a list of the row's distinct columns; the
// position of each in the sorted output row is the number of listed columns
// smaller than it, counted by every lane over the whole list (broadcast
// 128-bit shared-memory reads), so no sort network is needed.  The lane that
// reads a slot during compaction also clears it, leaving the table empty for
// the warp's next row.
//
// Compared with the register sort (rowpass.cuh), which moves every product
// through a bitonic network of shuffles, a product here costs one hash
// insertion and one shared-memory update, and the ranking works on the
// distinct columns only.
#pragma once

#include "internal.cuh"
#include "semiring.cuh"

namespace sg {

constexpr int HASH_EMPTY = -1;   // free slot (columns are >= 0)
constexpr int HASH_WARPS = 8;    // warps (rows in flight) per block

// Slot of column c in a table of 2^lg slots: Fibonacci hashing of the column.
template <int LG>
__device__ __forceinline__ unsigned hash_slot(int c) {
  return ((unsigned)c * 0x9E3779B1u) >> (32 - LG);
}

// Claims or finds column c's slot.  Keys never change while a row is in
// flight (a slot is claimed once and cleared only after the row), so a plain
// read that sees another column can move on.  *fresh tells whether this call
// claimed the slot.  Returns -1 (and flags EB_TABLE) only if every slot holds
// another column, which the table's size rules out.
template <int LG>
__device__ __forceinline__ int hash_insert(int* key, int c, bool* fresh, uint32_t* err) {
  constexpr unsigned M = (1u << LG) - 1u;
  unsigned h = hash_slot<LG>(c);
  *fresh = false;
  for (int it = 0; it <= (int)M; ++it) {
    int k = *(volatile int*)&key[h];
    if (k == HASH_EMPTY) {
      k = atomicCAS(&key[h], HASH_EMPTY, c);
      if (k == HASH_EMPTY) {
        *fresh = true;
        return (int)h;
      }
    }
    if (k == c) return (int)h;
    h = (h + 1u) & M;
  }
  atomicOr(err, EB_TABLE);
  return -1;
}

// Per-lane operands of a row's first chunk of A entries (positions a0 ..
// a0+31): the B row bounds of the lane's entry and its A value.  Loaded one
// row ahead of the row's products (see the kernels' row loops).
template <typename T>
struct Chunk0 {
  int sb = 0, len = 0;
  T a = T(0);
};

// B row bounds of a lane's A entry e (its column k = A(i,e) already loaded).
__device__ __forceinline__ void b_bounds(const Csr& B, int k, int* sb, int* len) {
  const int s0 = B.rp[k];
  *sb = s0;
  *len = B.rp[k + 1] - s0;
}

// Gathers the row's products (A positions a0..a1) into E slots per lane:
// product q of the row (A's entries in order, each B row in order) goes to
// slot q / 32 of lane q % 32.  A prefix sum over each chunk of 32 A entries
// gives every entry's first product, and each lane finds the entry owning
// its product by a search over those sums.  The first chunk's operands come
// preloaded in c0; later chunks (rows of more than 32 nonzeros) load their
// own.  NUM: pv = A(i,k) * B(k,j), one rounded multiply per product.  Empty
// slots hold column INT_MAX.  Returns the row's product count.
template <int E, bool NUM, typename T, int SR = SPGEMM_PLUS_TIMES>
__device__ __forceinline__ int hash_gather(const Csr& A, const Csr& B, const T* __restrict__ av,
                                           const T* __restrict__ bv, int a0, int a1, const Chunk0<T>& c0,
                                           int (&col)[E], T (&pv)[E]) {
  const int lane = lane_id();
#pragma unroll
  for (int s = 0; s < E; ++s) {
    col[s] = INT_MAX;
    pv[s] = T(0);
  }
  int done = 0;
  for (int e0 = a0; e0 < a1; e0 += 32) {
    int sb = c0.sb, len = c0.len;
    T a = c0.a;
    if (e0 != a0) {
      const int e = e0 + lane;
      sb = len = 0;
      a = T(0);
      if (e < a1) {
        b_bounds(B, A.ci[e], &sb, &len);
        if (NUM) a = av[e];
      }
    }
    const int incl = warp_incl_scan(len);
    const int tot = __shfl_sync(FULL, incl, 31);
    const int excl = incl - len;
#pragma unroll
    for (int s = 0; s < E; ++s) {
      // products q = 32 s + lane - done of this chunk; warp-uniform test
      if (32 * s + 31 - done < 0 || 32 * s - done >= tot) continue;
      const int q = 32 * s + lane - done;
      const int o = warp_owner(incl, q);
      const int os = __shfl_sync(FULL, sb, o);
      const int oex = __shfl_sync(FULL, excl, o);
      T oa = T(0);
      if (NUM) oa = __shfl_sync(FULL, a, o);
      if (q >= 0 && q < tot) {
        const int bi = os + q - oex;
        col[s] = B.ci[bi];
        if (NUM) pv[s] = SrOps<T, SR>::mul(oa, bv[bi]);
      }
    }
    done += tot;
  }
  return done;
}

// The row loop shared by both kernels.  Warp w takes list positions
// idx = w, w + nw, ...; while row t's products are gathered and merged, the
// loads for the next rows are in flight: row t+1's first chunk of A entries
// (issued before row t's gather, its B row bounds after row t's hash
// insertions) and row t+2's bounds in A (row list read one more row ahead).
// body(r, a0, a1, c0, between) processes row t and calls between() once, after
// its hash insertions, to issue the later loads.
template <bool NUM, typename T, typename Body>
__device__ __forceinline__ void hash_row_loop(const Csr& A, const Csr& B, const T* __restrict__ av,
                                              const RowInfo& ri, long long lb, long long le, long long w,
                                              long long nw, Body body) {
  const int lane = lane_id();
  long long idx = lb + w;
  int r = 0, a0 = 0, a1 = 0, rn = 0, a0n = 0, a1n = 0;
  Chunk0<T> c0;
  if (idx < le) {
    r = ri.rows[idx];
    a0 = A.rp[ri.row_begin + r];
    a1 = A.rp[ri.row_begin + r + 1];
    if (a0 + lane < a1) {
      b_bounds(B, A.ci[a0 + lane], &c0.sb, &c0.len);
      if (NUM) c0.a = av[a0 + lane];
    }
  }
  if (idx + nw < le) {
    rn = ri.rows[idx + nw];
    a0n = A.rp[ri.row_begin + rn];
    a1n = A.rp[ri.row_begin + rn + 1];
  }
  for (; idx < le; idx += nw) {
    const bool has2 = idx + 2 * nw < le;
    const int rnn = has2 ? ri.rows[idx + 2 * nw] : 0;
    int kn = -1;
    Chunk0<T> c0n;
    if (a0n + lane < a1n) {  // row t+1 (a0n = a1n = 0 past the end)
      kn = A.ci[a0n + lane];
      if (NUM) c0n.a = av[a0n + lane];
    }
    int a0nn = 0, a1nn = 0;
    auto between = [&]() {
      if (kn >= 0) b_bounds(B, kn, &c0n.sb, &c0n.len);
      if (has2) {
        a0nn = A.rp[ri.row_begin + rnn];
        a1nn = A.rp[ri.row_begin + rnn + 1];
      }
    };
    body(r, a0, a1, c0, between);
    r = rn;
    a0 = a0n;
    a1 = a1n;
    c0 = c0n;
    rn = rnn;
    a0n = a0nn;
    a1n = a1nn;
  }
}

// Symbolic pass: the number of distinct columns of each row (the count of
// slots its products claimed).
template <int E>
__global__ void __launch_bounds__(HASH_WARPS * 32)
k_hash_sym(Csr A, Csr B, RowInfo ri, const DevStats* st, int bin_lo, int bin_hi, int32_t* __restrict__ c_cnt,
           uint32_t* err) {
  constexpr int LG = 6 + (E >= 4 ? 2 : (E >= 2 ? 1 : 0));
  constexpr int H = 1 << LG;
  static_assert(H == 64 * E, "table of twice the slots");
  __shared__ int s_lb, s_le;
  __shared__ __align__(16) int s_key[HASH_WARPS][H];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  int* key = s_key[warp];
  for (int t = lane; t < H; t += 32) key[t] = HASH_EMPTY;
  if (threadIdx.x == 0) bin_range(st, bin_lo, bin_hi, &s_lb, &s_le);
  if (block_skip(st)) return;
  const long long nw = (long long)gridDim.x * HASH_WARPS;
  hash_row_loop<false, float>(A, B, nullptr, ri, s_lb, s_le, (long long)blockIdx.x * HASH_WARPS + warp, nw,
                              [&](int r, int a0, int a1, const Chunk0<float>& c0, auto& between) {
    int col[E];
    float pv[E];
    const int P = hash_gather<E, false, float>(A, B, nullptr, nullptr, a0, a1, c0, col, pv);
    if (P > 32 * E && lane == 0) atomicOr(err, EB_INTERNAL);  // the row's bin rules this out
    int slot[E];
    int cnt = 0;
#pragma unroll
    for (int s = 0; s < E; ++s) {
      bool fresh = false;
      slot[s] = col[s] != INT_MAX ? hash_insert<LG>(key, col[s], &fresh, err) : -1;
      if (!fresh) slot[s] = -1;  // only the claiming lane clears the slot
      cnt += __popc(__ballot_sync(FULL, fresh));
    }
    between();
    if (lane == 0) c_cnt[r] = cnt;
    __syncwarp();
#pragma unroll
    for (int s = 0; s < E; ++s)
      if (slot[s] >= 0) key[slot[s]] = HASH_EMPTY;
    __syncwarp();
  });
}

// Numeric pass: C's columns (ascending) and values for each row, at the
// positions [c_rp[r], c_rp[r+1]) the symbolic pass and the scan fixed.
// The product that claims a column's slot stores its value there; the
// others add theirs with a shared-memory reduction after a warp barrier.
template <int E, typename T, int SR = SPGEMM_PLUS_TIMES>
__global__ void __launch_bounds__(HASH_WARPS * 32)
k_hash_num(Csr A, Csr B, const T* __restrict__ av, const T* __restrict__ bv, RowInfo ri, const DevStats* st,
           int bin_lo, int bin_hi, const int32_t* __restrict__ c_rp, int32_t* __restrict__ c_ci,
           T* __restrict__ c_v, uint32_t* err) {
  constexpr int LG = 6 + (E >= 4 ? 2 : (E >= 2 ? 1 : 0));
  constexpr int H = 1 << LG;
  constexpr int D = 32 * E;  // distinct columns of a row: at most its products
  static_assert(H == 64 * E, "table of twice the slots");
  __shared__ int s_lb, s_le;
  __shared__ __align__(16) int s_key[HASH_WARPS][H];
  __shared__ __align__(16) T s_val[HASH_WARPS][H];
  __shared__ __align__(16) int s_dk[HASH_WARPS][D + 4];  // +4: INT_MAX padding of the ranking reads
  __shared__ __align__(16) T s_dv[HASH_WARPS][D];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  int* key = s_key[warp];
  T* val = s_val[warp];
  int* dk = s_dk[warp];
  T* dv = s_dv[warp];
  for (int t = lane; t < H; t += 32) key[t] = HASH_EMPTY;
  if (threadIdx.x == 0) bin_range(st, bin_lo, bin_hi, &s_lb, &s_le);
  if (block_skip(st)) return;
  const long long nw = (long long)gridDim.x * HASH_WARPS;
  hash_row_loop<true, T>(A, B, av, ri, s_lb, s_le, (long long)blockIdx.x * HASH_WARPS + warp, nw,
                         [&](int r, int a0, int a1, const Chunk0<T>& c0, auto& between) {
    const int ob = c_rp[r], oe = c_rp[r + 1];
    int col[E];
    T pv[E];
    const int P = hash_gather<E, true, T, SR>(A, B, av, bv, a0, a1, c0, col, pv);
    if (P > 32 * E && lane == 0) atomicOr(err, EB_INTERNAL);  // the row's bin rules this out
    int slot[E];
    bool fresh[E];
#pragma unroll
    for (int s = 0; s < E; ++s) {
      fresh[s] = false;
      slot[s] = col[s] != INT_MAX ? hash_insert<LG>(key, col[s], &fresh[s], err) : -1;
    }
    between();
#pragma unroll
    for (int s = 0; s < E; ++s)
      if (fresh[s]) val[slot[s]] = pv[s];
    __syncwarp();
#pragma unroll
    for (int s = 0; s < E; ++s)
      if (!fresh[s] && slot[s] >= 0) SrOps<T, SR>::red_value(&val[slot[s]], pv[s], err);
    __syncwarp();
    // Compaction: the occupied slots, in slot order, into the list dk/dv;
    // each slot's key is cleared by the lane that read it.
    int nd = 0;
#pragma unroll
    for (int t = 0; t < H / 32; ++t) {
      const int h = 32 * t + lane;
      const int k = key[h];
      const bool occ = k != HASH_EMPTY;
      const unsigned m = __ballot_sync(FULL, occ);
      if (occ) {
        const int p = nd + __popc(m & lanemask_lt());
        if (p < D) {
          dk[p] = k;
          dv[p] = val[h];
        }
        key[h] = HASH_EMPTY;
      }
      nd += __popc(m);
    }
    if (nd > D) {  // more distinct columns than products: never expected
      if (lane == 0) atomicOr(err, EB_INTERNAL);
      nd = D;
    }
    if (lane < 4) dk[nd + lane] = INT_MAX;
    __syncwarp();
    // Ranking: output position of a column = listed columns smaller than it.
    int mk[E], rank[E];
    T mv[E];
#pragma unroll
    for (int u = 0; u < E; ++u) {
      const int d = 32 * u + lane;
      mk[u] = d < nd ? dk[d] : INT_MAX;
      mv[u] = d < nd ? dv[d] : T(0);
      rank[u] = 0;
    }
    for (int e = 0; e < nd; e += 4) {
      const int4 q = *reinterpret_cast<const int4*>(&dk[e]);
#pragma unroll
      for (int u = 0; u < E; ++u) {
        if (32 * u >= nd) break;  // warp-uniform
        rank[u] += (q.x < mk[u]) + (q.y < mk[u]) + (q.z < mk[u]) + (q.w < mk[u]);
      }
    }
    if (lane == 0 && ob + nd != oe) atomicOr(err, EB_INTERNAL);
#pragma unroll
    for (int u = 0; u < E; ++u) {
      const int d = 32 * u + lane;
      if (d < nd) {
        const int o = ob + rank[u];
        if (o < oe) {
          c_ci[o] = mk[u];
          c_v[o] = mv[u];
        }
      }
    }
    __syncwarp();  // the list is read before the next row's compaction overwrites it
  });
}

}  // namespace sg
