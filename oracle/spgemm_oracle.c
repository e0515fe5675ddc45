/*
 * CPU oracle for the Gustavson SpGEMM path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load this file's library.  The product path (the CUDA library) never
 * calls it and shares no code, header, table or helper with it.
 *
 * Plain, single-threaded, deliberately unoptimised C.  Compiled with
 * -O2 -ffp-contract=off so every multiply and add is rounded separately and
 * the summation order is exactly the loop order written below.
 *
 * What it computes (Sec. 2.2, row-wise Gustavson): row i of C = A*B is the
 * sum over the nonzeros A(i,k) of the scaled rows A(i,k)*B(k,:).  Adding two
 * sparse rows means merging them by column index and adding the values of
 * equal columns (Sec. 2.2; Algorithm 1 is that merge).  The result row holds
 * every column reached by some product, ascending, each once.  Entries that
 * cancel to 0.0 are kept (the pattern is structural).
 *
 * The accumulation uses a dense value array and a marker array of length
 * ncols(B) (the textbook "sparse accumulator"): for each product the marker
 * says whether column j is already in the row; the touched columns are then
 * sorted ascending with the C library's qsort and emitted.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int cmp_i32(const void* x, const void* y) {
  int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  return (a > b) - (a < b);
}

/* Sizes of the rows of C = A*B.  c_row_ptr gets m+1 entries (int64).
 * Returns 0, or -1 on allocation failure. */
int oracle_spgemm_rowptr(int64_t m, int64_t n,
                         const int32_t* a_rp, const int32_t* a_ci,
                         const int32_t* b_rp, const int32_t* b_ci,
                         int64_t* c_rp) {
  int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!mark) return -1;
  for (int64_t j = 0; j < n; ++j) mark[j] = -1;
  c_rp[0] = 0;
  for (int64_t i = 0; i < m; ++i) {
    int64_t count = 0;
    for (int32_t p = a_rp[i]; p < a_rp[i + 1]; ++p) {
      int32_t k = a_ci[p];
      for (int32_t q = b_rp[k]; q < b_rp[k + 1]; ++q) {
        int32_t j = b_ci[q];
        if (mark[j] != i) { mark[j] = i; ++count; }
      }
    }
    c_rp[i + 1] = c_rp[i] + count;
  }
  free(mark);
  return 0;
}

/* C = A*B given the row pointer from oracle_spgemm_rowptr.  Fills c_ci (int32)
 * and c_v (double).  For each row: products in A's stored order, then B's
 * stored order; the first product of column j initialises acc[j], later ones
 * add to it; the touched columns are sorted ascending before they are
 * written.  Returns 0, or -1 on allocation failure. */
int oracle_spgemm(int64_t m, int64_t n,
                  const int32_t* a_rp, const int32_t* a_ci, const double* a_v,
                  const int32_t* b_rp, const int32_t* b_ci, const double* b_v,
                  const int64_t* c_rp, int32_t* c_ci, double* c_v) {
  size_t nn = (size_t)(n > 0 ? n : 1);
  int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * nn);
  double* acc = (double*)malloc(sizeof(double) * nn);
  int32_t* list = (int32_t*)malloc(sizeof(int32_t) * nn);
  if (!mark || !acc || !list) { free(mark); free(acc); free(list); return -1; }
  for (int64_t j = 0; j < n; ++j) { mark[j] = -1; acc[j] = 0.0; }
  for (int64_t i = 0; i < m; ++i) {
    int64_t len = 0;
    for (int32_t p = a_rp[i]; p < a_rp[i + 1]; ++p) {
      int32_t k = a_ci[p];
      double a = a_v[p];
      for (int32_t q = b_rp[k]; q < b_rp[k + 1]; ++q) {
        int32_t j = b_ci[q];
        double prod = a * b_v[q];
        if (mark[j] != i) {
          mark[j] = i;
          acc[j] = prod;
          list[len++] = j;
        } else {
          acc[j] = acc[j] + prod;
        }
      }
    }
    qsort(list, (size_t)len, sizeof(int32_t), cmp_i32);
    int64_t out = c_rp[i];
    for (int64_t t = 0; t < len; ++t) {
      c_ci[out + t] = list[t];
      c_v[out + t] = acc[list[t]];
    }
  }
  free(mark); free(acc); free(list);
  return 0;
}

/* Gradient of L = sum_{(i,j) in pattern(C)} W(i,j) * C(i,j) with C = A*B,
 * where dC = W is given on C's pattern (c_rp, c_ci, dc_v).
 *   dA(i,k) = sum_j dC(i,j) * B(k,j)   on pattern(A)
 *   dB(k,j) = sum_i A(i,k) * dC(i,j)   on pattern(B)
 * Row i of dC is scattered into a dense array w (with a marker), then every
 * product pair (A(i,k), B(k,j)) contributes once to each gradient, in A's
 * then B's stored order.  da / db may be NULL to skip.  Returns 0 or -1. */
int oracle_spgemm_backward(int64_t m, int64_t n,
                           const int32_t* a_rp, const int32_t* a_ci, const double* a_v,
                           const int32_t* b_rp, const int32_t* b_ci, const double* b_v,
                           int64_t b_nnz,
                           const int64_t* c_rp, const int32_t* c_ci, const double* dc_v,
                           double* da, double* db) {
  size_t nn = (size_t)(n > 0 ? n : 1);
  double* w = (double*)malloc(sizeof(double) * nn);
  int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * nn);
  if (!w || !mark) { free(w); free(mark); return -1; }
  for (int64_t j = 0; j < n; ++j) { mark[j] = -1; w[j] = 0.0; }
  if (da) memset(da, 0, sizeof(double) * (size_t)(m > 0 ? a_rp[m] : 0));
  if (db) memset(db, 0, sizeof(double) * (size_t)b_nnz);
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t t = c_rp[i]; t < c_rp[i + 1]; ++t) {
      mark[c_ci[t]] = i;
      w[c_ci[t]] = dc_v[t];
    }
    for (int32_t p = a_rp[i]; p < a_rp[i + 1]; ++p) {
      int32_t k = a_ci[p];
      for (int32_t q = b_rp[k]; q < b_rp[k + 1]; ++q) {
        int32_t j = b_ci[q];
        double g = (mark[j] == i) ? w[j] : 0.0;
        if (da) da[p] = da[p] + g * b_v[q];
        if (db) db[q] = db[q] + a_v[p] * g;
      }
    }
  }
  free(w); free(mark);
  return 0;
}

/* Transpose of an m x n CSR matrix into CSR of n x m (equivalently, the CSC
 * form of Sec. 2.1).  Entries of each output row appear in increasing
 * source-row order.  t_rp gets n+1 entries. */
int oracle_transpose(int64_t m, int64_t n,
                     const int32_t* rp, const int32_t* ci, const double* v,
                     int64_t* t_rp, int32_t* t_ci, double* t_v) {
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!fill) return -1;
  for (int64_t j = 0; j <= n; ++j) t_rp[j] = 0;
  for (int64_t i = 0; i < m; ++i)
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) t_rp[ci[p] + 1] += 1;
  for (int64_t j = 0; j < n; ++j) t_rp[j + 1] += t_rp[j];
  for (int64_t j = 0; j < n; ++j) fill[j] = t_rp[j];
  for (int64_t i = 0; i < m; ++i)
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t dst = fill[ci[p]]++;
      t_ci[dst] = (int32_t)i;
      if (v && t_v) t_v[dst] = v[p];
    }
  free(fill);
  return 0;
}

/* y = A*x (sparse matrix times dense vector), row by row in stored order. */
void oracle_spmv(int64_t m, const int32_t* rp, const int32_t* ci, const double* v,
                 const double* x, double* y) {
  for (int64_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) s = s + v[p] * x[ci[p]];
    y[i] = s;
  }
}

/* Number of products of each row: prod[i] = sum over A(i,k) of nnz(B(k,:)).
 * (The work count that A_DS.B_NUM_VEC carries per nonzero, Table 1.) */
void oracle_row_products(int64_t m, const int32_t* a_rp, const int32_t* a_ci,
                         const int32_t* b_rp, int64_t* prod) {
  for (int64_t i = 0; i < m; ++i) {
    int64_t s = 0;
    for (int32_t p = a_rp[i]; p < a_rp[i + 1]; ++p)
      s += (int64_t)(b_rp[a_ci[p] + 1] - b_rp[a_ci[p]]);
    prod[i] = s;
  }
}

/* Masked product C<M> = (A*B) .* M on M's pattern (the sampled product that
 * triangle counting and Markov clustering use; Sec. 1 names both as SpGEMM
 * applications).  c_v gets nnz(M) entries aligned with M's entries:
 *   c_v[p] = m_v[p] * sum_k A(i,k) * B(k,j)   for entry p = (i,j) of M,
 * the sum over the k with A(i,k) and B(k,j) both stored (0 when there is
 * none: the output keeps all of M's pattern); without m_v (NULL) the factor
 * is 1.  For each row: M's columns are scattered into a dense position array
 * (pos[j] = p, -1 elsewhere), then the row's products are formed in A's
 * stored order and, within each, B's stored order (the Gustavson order of
 * Sec. 2.2), and each product whose column is in M's row is added to that
 * entry's sum; the sums start at 0.0.  Returns 0, or -1 on allocation
 * failure. */
int oracle_masked(int64_t m, int64_t n,
                  const int32_t* a_rp, const int32_t* a_ci, const double* a_v,
                  const int32_t* b_rp, const int32_t* b_ci, const double* b_v,
                  const int32_t* m_rp, const int32_t* m_ci, const double* m_v,
                  double* c_v) {
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!pos) return -1;
  for (int64_t j = 0; j < n; ++j) pos[j] = -1;
  for (int64_t i = 0; i < m; ++i) {
    for (int32_t p = m_rp[i]; p < m_rp[i + 1]; ++p) {
      pos[m_ci[p]] = p;
      c_v[p] = 0.0;
    }
    for (int32_t e = a_rp[i]; e < a_rp[i + 1]; ++e) {
      int32_t k = a_ci[e];
      for (int32_t q = b_rp[k]; q < b_rp[k + 1]; ++q) {
        int64_t p = pos[b_ci[q]];
        if (p >= 0) c_v[p] = c_v[p] + a_v[e] * b_v[q];
      }
    }
    for (int32_t p = m_rp[i]; p < m_rp[i + 1]; ++p) {
      if (m_v) c_v[p] = c_v[p] * m_v[p];
      pos[m_ci[p]] = -1;
    }
  }
  free(pos);
  return 0;
}

/* Semiring versions of the masked product (the same row-wise Gustavson
 * order, products kept where M's row has their column; M's values are not
 * read).  For entry p = (i,j) of M, c_v[p] = the "sum" over the k with A(i,k)
 * and B(k,j) both stored of the "product" of A(i,k) and B(k,j), starting
 * from the semiring's zero (what an entry no product reaches keeps):
 *   semiring 1, min-plus: sum = min, product = a + b, zero = +infinity;
 *   semiring 2, max-plus: sum = max, product = a + b, zero = -infinity;
 *   semiring 3, or-and:   sum = or, product = (a != 0 and b != 0), values
 *                         1.0 (true) and 0.0 (false), zero = 0.0;
 * semiring 0 is the ordinary (plus, times) masked product of oracle_masked
 * without M's values.  Sec. 1 lists all-pairs shortest paths (min-plus)
 * among SpGEMM's applications.  Returns 0, -1 on allocation failure, -2 for
 * an unknown semiring. */
int oracle_masked_semiring(int64_t m, int64_t n, int32_t semiring,
                           const int32_t* a_rp, const int32_t* a_ci, const double* a_v,
                           const int32_t* b_rp, const int32_t* b_ci, const double* b_v,
                           const int32_t* m_rp, const int32_t* m_ci, double* c_v) {
  if (semiring < 0 || semiring > 3) return -2;
  const double inf = 1.0 / 0.0;
  const double zero = semiring == 1 ? inf : (semiring == 2 ? -inf : 0.0);
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!pos) return -1;
  for (int64_t j = 0; j < n; ++j) pos[j] = -1;
  for (int64_t i = 0; i < m; ++i) {
    for (int32_t p = m_rp[i]; p < m_rp[i + 1]; ++p) {
      pos[m_ci[p]] = p;
      c_v[p] = zero;
    }
    for (int32_t e = a_rp[i]; e < a_rp[i + 1]; ++e) {
      int32_t k = a_ci[e];
      for (int32_t q = b_rp[k]; q < b_rp[k + 1]; ++q) {
        int64_t p = pos[b_ci[q]];
        if (p < 0) continue;
        double a = a_v[e], b = b_v[q];
        switch (semiring) {
          case 0: c_v[p] = c_v[p] + a * b; break;
          case 1: if (a + b < c_v[p]) c_v[p] = a + b; break;
          case 2: if (a + b > c_v[p]) c_v[p] = a + b; break;
          default: if (a != 0.0 && b != 0.0) c_v[p] = 1.0; break;
        }
      }
    }
    for (int32_t p = m_rp[i]; p < m_rp[i + 1]; ++p) pos[m_ci[p]] = -1;
  }
  free(pos);
  return 0;
}
