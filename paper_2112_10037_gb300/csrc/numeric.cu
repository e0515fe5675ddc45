// Numeric pass with the ordinary sum and product; the other semirings'
// instantiations sit in numeric_minplus.cu, numeric_maxplus.cu and
// numeric_orand.cu (compiled in parallel).
#include "numdispatch.cuh"

namespace sg {

cudaError_t launch_numeric(const LaunchCtx& c, const Csr& A, const Csr& B, const RowInfo& ri,
                           const PathBins& pb, const Tuning& tu, const SplitInfo& sp, int dtype,
                           const void* av, const void* bv, int32_t* cur, int32_t* nxt, const int32_t* c_rp,
                           int32_t* c_ci, void* c_v, const int* path_rows, long long rows_wide,
                           const int* hist, int semiring) {
  switch (semiring) {
    case SPGEMM_PLUS_TIMES:
      return launch_numeric_sr<SPGEMM_PLUS_TIMES>(c, A, B, ri, pb, tu, sp, dtype, av, bv, cur, nxt, c_rp, c_ci, c_v,
                                                  path_rows, rows_wide, hist);
    case SPGEMM_MIN_PLUS:
      return launch_numeric_min_plus(c, A, B, ri, pb, tu, sp, dtype, av, bv, cur, nxt, c_rp, c_ci, c_v, path_rows,
                                     rows_wide, hist);
    case SPGEMM_MAX_PLUS:
      return launch_numeric_max_plus(c, A, B, ri, pb, tu, sp, dtype, av, bv, cur, nxt, c_rp, c_ci, c_v, path_rows,
                                     rows_wide, hist);
    case SPGEMM_OR_AND:
      return launch_numeric_or_and(c, A, B, ri, pb, tu, sp, dtype, av, bv, cur, nxt, c_rp, c_ci, c_v, path_rows,
                                   rows_wide, hist);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace sg
