// FP64 instantiations of the fused apply (see apply_kernel.cuh).
#include "apply_dispatch.cuh"

int fem_launch_apply_f64_shape(fem_op *op, const double *x, double *y, const int32_t *list,
                               int64_t nsel, double *dot_out, int choice, int bps,
                               const int *skip) {
  if (choice == FEM_CHOICE_DW_STENCIL) {
    if (!list && nsel == op->E && op->ncomp == 1 && op->d_stencil)
      return fem_launch_apply_stencil(op, x, y, dot_out, skip);
    choice = FEM_CHOICE_DW_ELMAT;   // element lists: the element-matrix body
  }
  if (fem_choice_is_dw(choice))
    return fem_launch_apply_dw_shape(op, x, y, list, nsel, dot_out, choice, bps, skip);
  fem_apply::ApplyParams<double> prm;
  prm.x = x; prm.y = y;
  prm.elem_nodes = op->mesh->d_elem_nodes;
  prm.list = list; prm.nsel = nsel;
  prm.N = op->N; prm.ncomp = op->ncomp;
  prm.qdata = op->d_qdata; prm.B = op->d_B; prm.Dq = op->d_Dq;
  prm.partials = op->d_partials; prm.counter = op->d_counter; prm.dot_out = dot_out;
  prm.skip = skip;
  if (nsel == 0) return FEM_OK;
  return fem_apply::dispatch<double>(op, prm, choice, bps);
}

int fem_launch_apply_f64(fem_op *op, const double *x, double *y, const int32_t *list,
                         int64_t nsel, double *dot_out, const int *skip) {
  return fem_launch_apply_f64_shape(op, x, y, list, nsel, dot_out, op->tune_epb[FEM_F64],
                                    op->tune_bps[FEM_F64], skip);
}
