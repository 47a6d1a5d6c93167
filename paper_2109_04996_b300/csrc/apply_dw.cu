// Double-word instantiations of the fused apply (launch choices 8..23 of an
// FP64 operator; see dw.cuh): the gathered FP64 x values are split into
// double words, the qdata (or element matrices) are read from the
// operator's double-word copy, the contractions and the pointwise products
// run in double-word arithmetic on the FP32 pipe, and the element results
// are rounded back to FP64 for the atomic scatter-add.
#include "apply_kernel.cuh"

// One order per translation unit (apply_dw_p2.cu .. apply_dw_p9.cu), so that
// the instantiations compile in parallel.
template <int P>
int fem_apply_dw_p(fem_op *op, const fem_apply::ApplyParams<dw> &prm, int choice, int bps);
extern template int fem_apply_dw_p<2>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
extern template int fem_apply_dw_p<3>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
extern template int fem_apply_dw_p<4>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
extern template int fem_apply_dw_p<5>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
extern template int fem_apply_dw_p<6>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
extern template int fem_apply_dw_p<7>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
extern template int fem_apply_dw_p<8>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
extern template int fem_apply_dw_p<9>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
// the collocated diffusion rules (apply_dw_p2c.cu .. apply_dw_p9c.cu)
template <int P>
int fem_apply_dw_pc(fem_op *op, const fem_apply::ApplyParams<dw> &prm, int choice, int bps);
extern template int fem_apply_dw_pc<2>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
extern template int fem_apply_dw_pc<3>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
extern template int fem_apply_dw_pc<4>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
extern template int fem_apply_dw_pc<5>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
extern template int fem_apply_dw_pc<6>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
extern template int fem_apply_dw_pc<7>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
extern template int fem_apply_dw_pc<8>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);
extern template int fem_apply_dw_pc<9>(fem_op *, const fem_apply::ApplyParams<dw> &, int, int);

int fem_launch_apply_dw_shape(fem_op *op, const double *x, double *y, const int32_t *list,
                              int64_t nsel, double *dot_out, int choice, int bps,
                              const int *skip) {
  if (choice == FEM_CHOICE_DW_ELMAT && !op->d_keldw) {
    fem_set_error("apply: the double-word element-matrix body needs the operator's split "
                  "element matrices");
    return FEM_EINVAL;
  }
  if (choice != FEM_CHOICE_DW_ELMAT && !op->d_qdw) {
    fem_set_error("apply: the double-word line body needs the operator's split qdata");
    return FEM_EINVAL;
  }
  fem_apply::ApplyParams<dw> prm;
  prm.x = x; prm.y = y;
  prm.elem_nodes = op->mesh->d_elem_nodes;
  prm.list = list; prm.nsel = nsel;
  prm.N = op->N; prm.ncomp = op->ncomp;
  prm.qdata = op->d_qdw; prm.B = nullptr; prm.Dq = nullptr;
  prm.partials = op->d_partials; prm.counter = op->d_counter; prm.dot_out = dot_out;
  prm.skip = skip;
  if (nsel == 0) return FEM_OK;
  if (op->colloc) {
    switch (op->P) {
      case 2: return fem_apply_dw_pc<2>(op, prm, choice, bps);
      case 3: return fem_apply_dw_pc<3>(op, prm, choice, bps);
      case 4: return fem_apply_dw_pc<4>(op, prm, choice, bps);
      case 5: return fem_apply_dw_pc<5>(op, prm, choice, bps);
      case 6: return fem_apply_dw_pc<6>(op, prm, choice, bps);
      case 7: return fem_apply_dw_pc<7>(op, prm, choice, bps);
      case 8: return fem_apply_dw_pc<8>(op, prm, choice, bps);
      case 9: return fem_apply_dw_pc<9>(op, prm, choice, bps);
    }
  }
  switch (op->P) {
    case 2: return fem_apply_dw_p<2>(op, prm, choice, bps);
    case 3: return fem_apply_dw_p<3>(op, prm, choice, bps);
    case 4: return fem_apply_dw_p<4>(op, prm, choice, bps);
    case 5: return fem_apply_dw_p<5>(op, prm, choice, bps);
    case 6: return fem_apply_dw_p<6>(op, prm, choice, bps);
    case 7: return fem_apply_dw_p<7>(op, prm, choice, bps);
    case 8: return fem_apply_dw_p<8>(op, prm, choice, bps);
    case 9: return fem_apply_dw_p<9>(op, prm, choice, bps);
  }
  fem_set_error("apply: unsupported P = %d", op->P);
  return FEM_EINVAL;
}
