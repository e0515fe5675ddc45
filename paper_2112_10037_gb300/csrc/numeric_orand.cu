// Numeric pass over the or-and (reachability) semiring: the row-wise
// accumulation of Sec. 2.2 with that semiring's sum and product.
#include "numdispatch.cuh"

namespace sg {

SG_NUMERIC_SR_DECL(launch_numeric_or_and) {
  return launch_numeric_sr<SPGEMM_OR_AND>(c, A, B, ri, pb, tu, sp, dtype, av, bv, cur, nxt, c_rp, c_ci, c_v,
                                       path_rows, rows_wide, hist);
}

}  // namespace sg
