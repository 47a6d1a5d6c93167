// Double-word apply bodies of order P = 8, non-collocated rules (see
// apply_dw.cu).
// the double-word sums by ordered Fast2Sum (dw.cuh: faster at this order)
#define FEM_DW_ADD_ORDERED 1
#include "apply_dispatch.cuh"

template <int P>
int fem_apply_dw_p(fem_op *op, const fem_apply::ApplyParams<dw> &prm, int choice, int bps) {
  return fem_apply::dispatch_q<dw, P, 1>(op, prm, choice, bps);   // the collocated rules: apply_dw_p8c.cu
}
template int fem_apply_dw_p<8>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
