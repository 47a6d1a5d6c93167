// Double-word apply bodies of order P = 3, collocated Gauss-Lobatto
// diffusion (BP5/BP6; see apply_dw.cu).  A translation unit of their own:
// they keep the TwoSum double-word sums (dw.cuh), which measured at least as
// fast for them as the ordered Fast2Sum of the non-collocated bodies.
#include "apply_dispatch.cuh"

template <int P>
int fem_apply_dw_pc(fem_op *op, const fem_apply::ApplyParams<dw> &prm, int choice, int bps) {
  return fem_apply::dispatch_q<dw, P, 2>(op, prm, choice, bps);
}
template int fem_apply_dw_pc<3>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
