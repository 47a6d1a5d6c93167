// FP32 instantiations of the fused apply (see apply_kernel.cuh): FP32 qdata,
// tables and arithmetic; the fused x.y is accumulated in FP64.
#include "apply_dispatch.cuh"

int fem_launch_apply_f32_shape(fem_op *op, const float *x, float *y, const int32_t *list,
                               int64_t nsel, double *dot_out, int choice, int bps,
                               const int *skip) {
  if (choice == FEM_CHOICE_DW_STENCIL) {
    if (!list && nsel == op->E && op->ncomp == 1 && op->d_stencil32)
      return fem_launch_apply_stencil_f32(op, x, y, dot_out, skip);
    choice = 7;   // element lists: the element-matrix body
  }
  if (!op->d_qdata32) {
    fem_set_error("apply_f32: operator was not created with FEM_F32");
    return FEM_EINVAL;
  }
  fem_apply::ApplyParams<float> prm;
  prm.x = x; prm.y = y;
  prm.elem_nodes = op->mesh->d_elem_nodes;
  prm.list = list; prm.nsel = nsel;
  prm.N = op->N; prm.ncomp = op->ncomp;
  prm.qdata = op->d_qdata32; prm.B = op->d_B32; prm.Dq = op->d_Dq32;
  prm.partials = op->d_partials; prm.counter = op->d_counter; prm.dot_out = dot_out;
  prm.skip = skip;
  if (nsel == 0) return FEM_OK;
  return fem_apply::dispatch<float>(op, prm, choice, bps);
}

int fem_launch_apply_f32(fem_op *op, const float *x, float *y, const int32_t *list,
                         int64_t nsel, double *dot_out, const int *skip) {
  return fem_launch_apply_f32_shape(op, x, y, list, nsel, dot_out, op->tune_epb[FEM_F32],
                                    op->tune_bps[FEM_F32], skip);
}
