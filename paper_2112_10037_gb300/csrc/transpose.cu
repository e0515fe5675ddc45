// CSR transpose: the m x n matrix M in CSR becomes M^T (n x m) in CSR, which
// is M's CSC form (Sec. 2.1).  Entries of each output row are ordered by
// source row, so the result satisfies the sorted-columns precondition.
//
// M's entries, taken in CSR order, are already ascending by source row, so
// M^T is a STABLE sort of them by column: a least-significant-digit radix
// sort on the column index with digits of at most 9 bits (one pass for up
// to 512 columns, two for up to 262,144, three for up to 2^27, four above),
// every pass a stable counting scatter.  No output row is sorted afterwards
// and no source position is searched for, whatever the column lengths.
//
//  1. histogram pass per digit: per tile of TR_TILE consecutive entries the
//     count of every digit value, stored digit-major (table[d*T + t]); the
//     first pass also counts the entries of every column (M^T's row sizes)
//     and checks the column range,
//  2. exclusive prefix sums of the table and of the row sizes,
//  3. scatter pass per digit: a block takes a tile; each warp ranks its 512
//     consecutive entries among the equal digits of its earlier entries
//     (lanes of equal digit found by a warp match, one running count per
//     digit and warp in shared memory), the block turns the
//     per-warp counts into offsets, reorders the tile by digit in shared
//     memory and writes every digit's entries as one run from its table
//     offset.  The first pass reads M itself (source row by a search over
//     the row pointer, source position = entry index); the last writes the
//     source row (M^T's column index) and the source position.  Values,
//     when wanted, travel with the entries (read and written in order, no
//     gather through the source positions).
// The source positions let a caller move new values of the same structure
// (t_v[q] = v[t_src[q]]) without transposing again.
#include "launch_util.cuh"

namespace sg {

constexpr int TR_WARPS = 8;                         // warps of a scatter block
constexpr int TR_ITEMS = 16;                        // entries per lane and tile
constexpr int TR_TILE = TR_WARPS * 32 * TR_ITEMS;   // 4096 entries per tile
constexpr int TR_DIGIT = 9;                         // at most 512 digit values per pass
constexpr int TR_HIST_THREADS = 256;
static_assert(TR_WARPS * 32 >= (1 << TR_DIGIT) / 2, "two digits per thread at most");

struct TrPasses {
  int passes;
  int shift[4];
  int bits[4];
};

// Digits for columns in [0, n): the bits of n-1 (at least one) split into as
// few passes of at most TR_DIGIT bits as possible, as evenly as possible.
static TrPasses tr_passes(long long n) {
  int b = 1;
  while (b < 31 && (1ll << b) < n) ++b;
  TrPasses p{};
  p.passes = (b + TR_DIGIT - 1) / TR_DIGIT;
  int s = 0;
  for (int i = 0; i < p.passes; ++i) {
    const int left = p.passes - i;
    const int d = (b - s + left - 1) / left;
    p.shift[i] = s;
    p.bits[i] = d;
    s += d;
  }
  return p;
}

TransposeScratch transpose_scratch(long long n, long long nnz, int vbytes) {
  TransposeScratch s{};
  const TrPasses p = tr_passes(n);
  const long long tiles = (nnz + TR_TILE - 1) / TR_TILE;
  // pass outputs: X = (values, key, source row, source position) feeds the
  // last pass; Y, the one before it, keeps its rows, positions and values in
  // the outputs and needs only one more key array
  const size_t vints = (size_t)((vbytes + 3) / 4) * (size_t)nnz;
  s.tmp_ints = (p.passes >= 2 ? vints + 3 * (size_t)nnz : 0) + (p.passes >= 3 ? (size_t)nnz : 0);
  s.table_ints = (size_t)(tiles << p.bits[0]) + 1;
  const long long scan_len = (long long)s.table_ints > n ? (long long)s.table_ints : n;
  s.part_count = scan_partials_count(scan_len);
  return s;
}

__device__ __forceinline__ int tr_digit(int32_t key, int shift, int bits) {
  return (int)(((uint32_t)key >> shift) & ((1u << bits) - 1u));
}

// Digit counts of every tile; with cnt, also the entries of every column.
__global__ void __launch_bounds__(TR_HIST_THREADS) k_tr_hist(const int32_t* __restrict__ key, long long nnz,
                                                             int shift, int bits, long long tiles,
                                                             int32_t* __restrict__ table, int32_t* __restrict__ cnt,
                                                             long long n, uint32_t* err) {
  __shared__ int h[1 << TR_DIGIT];
  const int nb = 1 << bits;
  for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    for (int d = threadIdx.x; d < nb; d += TR_HIST_THREADS) h[d] = 0;
    __syncthreads();
    const long long e0 = t * TR_TILE;
    const long long e1 = e0 + TR_TILE < nnz ? e0 + TR_TILE : nnz;
    for (long long e = e0 + threadIdx.x; e < e1; e += TR_HIST_THREADS) {
      const int32_t c = key[e];
      if (cnt) {
        if (c < 0 || (long long)c >= n) atomicOr(err, EB_UNSORTED);
        else atomicAdd(&cnt[c], 1);
      }
      atomicAdd(&h[tr_digit(c, shift, bits)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nb; d += TR_HIST_THREADS) table[(long long)d * tiles + t] = h[d];
    __syncthreads();
  }
}

// Row of M holding entry e (rp[row] <= e < rp[row + 1]), searched upward
// from `row` (whose start is at most e): one step, then galloping and a
// binary search.  Stays within [row, m - 1] whatever rp holds.
__device__ __forceinline__ int tr_row_from(const int32_t* __restrict__ rp, int m, int row, long long e) {
  if (row + 1 >= m || rp[row + 1] > e) return row;
  int lo = row + 1;  // rp[lo] <= e
  long long step = 1;
  while (lo + step < m && rp[lo + step] <= e) {
    lo += (int)step;
    step <<= 1;
  }
  int hi = lo + step < m ? (int)(lo + step) : m;  // rp[hi] > e, or hi == m
  while (hi - lo > 1) {
    const int mid = lo + ((hi - lo) >> 1);
    if (rp[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

// Warp-wide search for the row holding entry e (the same e on every lane):
// 32 probes per step narrow [lo, hi) 32-fold.
__device__ __forceinline__ int tr_warp_row(const int32_t* __restrict__ rp, int m, long long e) {
  const int lane = lane_id();
  int lo = 0, hi = m;  // rp[lo] <= e, and rp[hi] > e unless hi == m
  while (hi - lo > 1) {
    const int step = (hi - lo + 31) >> 5;
    const long long q = (long long)lo + (long long)lane * step;
    const bool le = q < hi && rp[q] <= e;
    const unsigned b = __ballot_sync(FULL, le);
    const int last = b ? 31 - __clz(b) : 0;
    lo += last * step;
    hi = lo + step < hi ? lo + step : hi;
  }
  return lo;
}

template <int VB> struct TrVal { using type = unsigned int; };
template <> struct TrVal<8> { using type = unsigned long long; };

static size_t tr_scatter_smem(int bits, int vbytes) {
  return sizeof(int) * ((size_t)(TR_WARPS + 2) << bits) + (sizeof(int) * 3 + (size_t)vbytes) * (size_t)TR_TILE;
}

// One counting-scatter pass over one digit.  FIRST: the entries are M's
// (key = column, source row searched, source position = index, value =
// M's); otherwise (kin, rin, pin, vin).  LAST: writes the source row to rout
// (t_col_idx), the position to pout (t_src) and the value to vout (t_vals);
// otherwise the whole entry to (kout, rout, pout, vout).  VB: bytes per
// value (0: no values).  The tile is first reordered by digit in shared
// memory, so the global stores go out as runs of consecutive positions (one
// run per digit value).
template <bool FIRST, bool LAST, int VB>
__global__ void __launch_bounds__(TR_WARPS * 32) k_tr_scatter(const int32_t* __restrict__ rp, int m,
                                                              const int32_t* __restrict__ kin,
                                                              const int32_t* __restrict__ rin,
                                                              const int32_t* __restrict__ pin,
                                                              const void* __restrict__ vin_, long long nnz,
                                                              int shift, int bits, long long tiles,
                                                              const int32_t* __restrict__ table,
                                                              int32_t* __restrict__ kout, int32_t* __restrict__ rout,
                                                              int32_t* __restrict__ pout, void* __restrict__ vout_) {
  using V = typename TrVal<VB>::type;
  constexpr int NT = TR_WARPS * 32;
  const V* __restrict__ vin = (const V*)vin_;
  V* __restrict__ vout = (V*)vout_;
  extern __shared__ __align__(16) int tr_smem[];
  const int nb = 1 << bits;
  V* const sv = reinterpret_cast<V*>(tr_smem);  // the tile in digit order: values first (8-byte aligned),
  int* const sk = reinterpret_cast<int*>(sv + (VB ? TR_TILE : 0));  // keys, rows, positions
  int* const sr = sk + TR_TILE;
  int* const sp = sr + TR_TILE;
  int* const whist = sp + TR_TILE;            // [warp][digit]: running counts, then offsets in the digit
  int* const s_toff = whist + TR_WARPS * nb;  // [digit]: first position of the digit in the tile
  int* const s_goff = s_toff + nb;            // [digit]: global position minus tile position
  __shared__ int s_wsum[2 * TR_WARPS];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const unsigned lt = lanemask_lt();
  int* const wh = whist + warp * nb;
  for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    for (int x = threadIdx.x; x < TR_WARPS * nb; x += NT) whist[x] = 0;
    __syncthreads();
    const long long tbase = t * TR_TILE;
    const int tlen = (int)(nnz - tbase < TR_TILE ? nnz - tbase : TR_TILE);
    const long long wbase = tbase + (long long)warp * (32 * TR_ITEMS);
    int k[TR_ITEMS], r[TR_ITEMS], p[TR_ITEMS], loc[TR_ITEMS];
    V v[TR_ITEMS];
    if (FIRST) {
      int row = wbase < nnz ? tr_warp_row(rp, m, wbase) : 0;
#pragma unroll
      for (int j = 0; j < TR_ITEMS; ++j) {
        const long long e = wbase + 32 * j + lane;
        k[j] = 0; r[j] = 0; p[j] = 0; v[j] = 0;  // p is the entry index, formed when staged
        if (e < nnz) {
          row = tr_row_from(rp, m, row, e);
          k[j] = kin[e];
          r[j] = row;
          if (VB) v[j] = vin[e];
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < TR_ITEMS; ++j) {
        const long long e = wbase + 32 * j + lane;
        k[j] = 0; r[j] = 0; p[j] = 0; v[j] = 0;
        if (e < nnz) {
          k[j] = kin[e];
          r[j] = rin[e];
          p[j] = pin[e];
          if (VB) v[j] = vin[e];
        }
      }
    }
    // rank of each entry among the earlier entries of this warp with its digit
#pragma unroll
    for (int j = 0; j < TR_ITEMS; ++j) {
      const bool act = wbase + 32 * j + lane < nnz;
      const int d = act ? tr_digit(k[j], shift, bits) : nb;
      const unsigned peers = __match_any_sync(FULL, d);
      const int leader = __ffs(peers) - 1;
      int before = 0;
      if (act && lane == leader) {
        before = wh[d];
        wh[d] = before + __popc(peers);
      }
      before = __shfl_sync(FULL, before, leader);
      loc[j] = before + __popc(peers & lt);
      __syncwarp();
    }
    __syncthreads();
    // per digit (two per thread at most): offsets of the warps within the
    // digit and the digit's count, then a block scan of the counts for the
    // digit's place in the tile
    const int da = 2 * threadIdx.x, db = da + 1;
    int ca = 0, cb = 0;
    if (da < nb) {
#pragma unroll
      for (int w = 0; w < TR_WARPS; ++w) {
        const int x = whist[w * nb + da];
        whist[w * nb + da] = ca;
        ca += x;
      }
    }
    if (db < nb) {
#pragma unroll
      for (int w = 0; w < TR_WARPS; ++w) {
        const int x = whist[w * nb + db];
        whist[w * nb + db] = cb;
        cb += x;
      }
    }
    const int pair = ca + cb;
    const int incl = warp_incl_scan(pair);
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const int x = lane < TR_WARPS ? s_wsum[lane] : 0;
      const int xi = warp_incl_scan(x);
      if (lane < TR_WARPS) s_wsum[TR_WARPS + lane] = xi - x;
    }
    __syncthreads();
    const int ex = s_wsum[TR_WARPS + warp] + incl - pair;
    if (da < nb) {
      s_toff[da] = ex;
      s_goff[da] = table[(long long)da * tiles + t] - ex;
    }
    if (db < nb) {
      s_toff[db] = ex + ca;
      s_goff[db] = table[(long long)db * tiles + t] - ex - ca;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < TR_ITEMS; ++j) {
      const int q = warp * (32 * TR_ITEMS) + 32 * j + lane;
      if (q < tlen) {
        const int d = tr_digit(k[j], shift, bits);
        const int pos = s_toff[d] + wh[d] + loc[j];
        sk[pos] = k[j];
        sr[pos] = r[j];
        sp[pos] = FIRST ? (int)(tbase + q) : p[j];
        if (VB) sv[pos] = v[j];
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < tlen; q += NT) {
      const int kk = sk[q];
      const int dst = s_goff[tr_digit(kk, shift, bits)] + q;
      if (!LAST) kout[dst] = kk;
      rout[dst] = sr[q];
      pout[dst] = sp[q];
      if (VB) vout[dst] = sv[q];
    }
    __syncthreads();  // shared memory is reused by the next tile
  }
}

static int grid_cap(long long units, int per_block, int nsm, int per_sm = 8) {
  long long g = (units + per_block - 1) / per_block;
  const long long cap = (long long)nsm * per_sm;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

template <int VB>
static cudaError_t tr_scatter_launch(const LaunchCtx& c, bool first, bool last, const int32_t* rp, int m,
                                     const int32_t* kin, const int32_t* rin, const int32_t* pin, const void* vin,
                                     long long nnz, int shift, int bits, long long tiles, const int32_t* table,
                                     int32_t* ko, int32_t* ro, int32_t* po, void* vo) {
  const size_t smem = tr_scatter_smem(bits, VB);
  const size_t smem_max = tr_scatter_smem(TR_DIGIT, VB);
  auto k = first ? (last ? k_tr_scatter<true, true, VB> : k_tr_scatter<true, false, VB>)
                 : (last ? k_tr_scatter<false, true, VB> : k_tr_scatter<false, false, VB>);
  const int per_sm = kernel_blocks_per_sm(k, TR_WARPS * 32, smem_max);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  k<<<grid_cap(tiles, 1, c.nsm, per_sm), TR_WARPS * 32, smem, c.stream>>>(rp, m, kin, rin, pin, vin, nnz, shift,
                                                                        bits, tiles, table, ko, ro, po, vo);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_transpose(const LaunchCtx& c, long long m, long long n, long long nnz, const int32_t* rp,
                             const int32_t* ci, int32_t* t_rp, int32_t* t_ci, int32_t* t_src, int vbytes,
                             const void* vals, void* t_vals, int32_t* tmp, int32_t* table, long long* partials) {
  cudaError_t e = cudaMemsetAsync(t_rp, 0, sizeof(int32_t) * (size_t)(n + 1), c.stream);
  if (e != cudaSuccess) return e;
  if (m <= 0 || nnz <= 0) return launch_scan(c, t_rp, n, partials, &c.st->scratch_total);
  if (vbytes != 0 && vbytes != 4 && vbytes != 8) return cudaErrorInvalidValue;
  if (!t_vals || !vals) vbytes = 0;
  const TrPasses ps = tr_passes(n);
  const long long tiles = (nnz + TR_TILE - 1) / TR_TILE;
  if (n <= 0) {  // no column exists: every entry is out of range (reported), M^T is empty
    k_tr_hist<<<grid_cap(tiles, 1, c.nsm, 8), TR_HIST_THREADS, 0, c.stream>>>(ci, nnz, 0, 1, tiles, table, t_rp, n,
                                                                             c.err);
    count_launch(c);
    return launch_scan(c, t_rp, n, partials, &c.st->scratch_total);
  }
  // pass outputs: X = (values, key, row, position) feeds the last pass; Y,
  // the one before it, keeps its rows, positions and values in the outputs
  const size_t vints = (size_t)((vbytes + 3) / 4) * (size_t)nnz;
  void* xv = tmp;
  int32_t *xk = tmp + vints, *xr = xk + nnz, *xp = xr + nnz, *yk = xp + nnz;
  const int32_t *kin = ci, *rin = nullptr, *pin = nullptr;
  const void* vin = vals;
  for (int i = 0; i < ps.passes; ++i) {
    const bool first = i == 0, last = i == ps.passes - 1;
    k_tr_hist<<<grid_cap(tiles, 1, c.nsm, 8), TR_HIST_THREADS, 0, c.stream>>>(
        kin, nnz, ps.shift[i], ps.bits[i], tiles, table, first ? t_rp : nullptr, n, c.err);
    count_launch(c);
    if (first && (e = launch_scan(c, t_rp, n, partials, &c.st->scratch_total)) != cudaSuccess) return e;
    if ((e = launch_scan(c, table, tiles << ps.bits[i], partials, &c.st->scratch_total)) != cudaSuccess) return e;
    int32_t *ko, *ro, *po;
    void* vo;
    if (last) {
      ko = nullptr; ro = t_ci; po = t_src; vo = t_vals;
    } else if ((ps.passes - 2 - i) % 2 == 0) {
      ko = xk; ro = xr; po = xp; vo = xv;
    } else {
      ko = yk; ro = t_ci; po = t_src; vo = t_vals;
    }
    const int mm = (int)m;
    if (vbytes == 8)
      e = tr_scatter_launch<8>(c, first, last, rp, mm, kin, rin, pin, vin, nnz, ps.shift[i], ps.bits[i], tiles,
                               table, ko, ro, po, vo);
    else if (vbytes == 4)
      e = tr_scatter_launch<4>(c, first, last, rp, mm, kin, rin, pin, vin, nnz, ps.shift[i], ps.bits[i], tiles,
                               table, ko, ro, po, vo);
    else
      e = tr_scatter_launch<0>(c, first, last, rp, mm, kin, rin, pin, nullptr, nnz, ps.shift[i], ps.bits[i], tiles,
                               table, ko, ro, po, nullptr);
    if (e != cudaSuccess) return e;
    kin = ko; rin = ro; pin = po; vin = vo;
  }
  return cudaGetLastError();
}

}  // namespace sg
