// Launch and dispatch of the fused apply over (P, q, kind) and the launch
// shape: EPB (elements per block) and blocks per SM, the two parameters the
// autotuner picks.  Included once per arithmetic type (apply_f64.cu,
// apply_f32.cu).
#pragma once
#include "apply_lines.cuh"
#include "apply_trilinear.cuh"
#include "apply_elmat.cuh"

namespace fem_apply {

// Elements-per-block candidates: index 0 = default (about 256 threads),
// 1 = half of it, 2 = twice it.  Only shapes with <= 1024 threads and
// <= 200 KB of shared memory are valid.
template <int Q, int CHOICE>
struct EpbChoice {
  static constexpr int D = DefaultEpb<Q>::value;
  static constexpr int value = CHOICE == 0 ? D : (CHOICE == 1 ? (D / 2 > 0 ? D / 2 : 1) : 2 * D);
};

template <typename T, int P, int Q, int KIND, bool COLLOC, int EPB>
int launch_shape(fem_op *op, const ApplyParams<T> &prm, int bps) {
  constexpr int NT = ApplyShape<Q, EPB>::NT;
  constexpr size_t smem = apply_smem_bytes<T, Q, P, KIND, EPB, COLLOC>();
  if constexpr (NT > 1024 || smem > 200 * 1024) {
    fem_set_error("apply: launch shape EPB=%d not valid for P=%d q=%d", EPB, P, Q);
    return FEM_EINVAL;
  } else {
    auto kern = fem_apply_kernel<T, P, Q, KIND, COLLOC, EPB>;
    static FemKernelCache cache;
    int &max_bps = cache.here();
    if (max_bps < 0) {
      FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int per_sm = 0;
      FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
      max_bps = per_sm < 1 ? 1 : per_sm;
    }
    const int use = (bps <= 0 || bps > max_bps) ? max_bps : bps;
    const int64_t ngroups = (prm.nsel + EPB - 1) / EPB;
    int64_t grid = (int64_t)op->nsm * use;
    if (grid > ngroups) grid = ngroups;
    if (grid > FEM_MAX_BLOCKS) grid = FEM_MAX_BLOCKS;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, NT, smem, op->stream()>>>(prm);
    FEM_CHECK_LAUNCH();
    return FEM_OK;
  }
}

// Diffusion: the line-based, even-odd element body (apply_lines.cuh).
template <typename T, int P, int Q, bool COLLOC, int EPB, bool PIPE, int KIND, bool PK = false,
          bool PF = false>
int launch_lines_kernel(fem_op *op, const LineParams<T, P, Q> &lp, int bps) {
  constexpr int NT = ApplyShape<Q, EPB>::NT;
  constexpr size_t smem = lines_smem_bytes<T, Q, EPB>();
  auto kern = [] {
    constexpr int MINB = LinesMinBlocks<T, Q, EPB, PIPE, KIND, PK, PF>::value;
    if constexpr (MINB > 0) return fem_apply_lines_kernel_mb<MINB, T, P, Q, COLLOC, EPB, PIPE, KIND, PK, PF>;
    else return fem_apply_lines_kernel<T, P, Q, COLLOC, EPB, PIPE, KIND, PK, PF>;
  }();
  static FemKernelCache cache;
  int &max_bps = cache.here();
  if (max_bps < 0) {
    FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    max_bps = per_sm < 1 ? 1 : per_sm;
  }
  const int use = (bps <= 0 || bps > max_bps) ? max_bps : bps;
  const int64_t ngroups = (lp.a.nsel + EPB - 1) / EPB;
  int64_t grid = (int64_t)op->nsm * use;
  if (grid > ngroups) grid = ngroups;
  if (grid > FEM_MAX_BLOCKS) grid = FEM_MAX_BLOCKS;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, NT, smem, op->stream()>>>(lp);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

// pipe: carry the next group's x gather one group ahead (double words; the
// FP32 body always does for scalar whole-mesh launches)
// packed: the f32x2 form of the double-word contractions
// pf: L2 bulk prefetch of the next group's qdata and node ids (double words,
// packed only)
template <typename T, int P, int Q, bool COLLOC, int EPB, int KIND>
int launch_lines(fem_op *op, const ApplyParams<T> &prm, int bps, bool pipe = false,
                 bool packed = false, bool pf = false) {
  constexpr int NT = ApplyShape<Q, EPB>::NT;
  constexpr size_t smem = lines_smem_bytes<T, Q, EPB>();
  if constexpr (NT > 1024 || smem > 200 * 1024) {
    fem_set_error("apply: launch shape EPB=%d not valid for P=%d q=%d", EPB, P, Q);
    return FEM_EINVAL;
  } else {
    LineParams<T, P, Q> lp;
    lp.a = prm;
    double Bt[FEM_MAX_P * FEM_MAX_Q], Dt[FEM_MAX_Q * FEM_MAX_Q];
    for (int k = 0; k < Q; k++)
      for (int a = 0; a < P; a++) Bt[a * Q + k] = op->tab.B[k * P + a];
    for (int k = 0; k < Q; k++)
      for (int m = 0; m < Q; m++) Dt[m * Q + k] = op->tab.Dq[k * Q + m];
    make_symtab<T, P, Q>(op->tab.B, lp.t.Bf);
    make_symtab<T, Q, P>(Bt, lp.t.Bt);
    make_symtab<T, Q, Q>(op->tab.Dq, lp.t.Df);
    make_symtab<T, Q, Q>(Dt, lp.t.Dt);
    if constexpr (std::is_same<T, dw>::value) {
      if (packed && pf) {
        if (pipe && prm.ncomp == 1 && !prm.list)
          return launch_lines_kernel<T, P, Q, COLLOC, EPB, true, KIND, true, true>(op, lp, bps);
        return launch_lines_kernel<T, P, Q, COLLOC, EPB, false, KIND, true, true>(op, lp, bps);
      }
      if (packed) return launch_lines_kernel<T, P, Q, COLLOC, EPB, false, KIND, true>(op, lp, bps);
    }
    if constexpr (sizeof(T) == 4 || std::is_same<T, dw>::value) {
      if (prm.ncomp == 1 && !prm.list && (sizeof(T) == 4 || pipe))
        return launch_lines_kernel<T, P, Q, COLLOC, EPB, true, KIND>(op, lp, bps);
    }
    return launch_lines_kernel<T, P, Q, COLLOC, EPB, false, KIND>(op, lp, bps);
  }
}

// Trilinear diffusion (p = 1, Gauss): one thread per element.
template <typename T, int Q>
int launch_trilinear(fem_op *op, const ApplyParams<T> &prm, int bps) {
  TrilinearParams<T, Q> tp;
  tp.a = prm;
  if constexpr (sizeof(T) == 8) tp.qsum = reinterpret_cast<const T *>(op->d_qsum);
  else tp.qsum = reinterpret_cast<const T *>(op->d_qsum32);
  if (!tp.qsum) {
    fem_set_error("apply: the trilinear body needs the operator's qdata line sums");
    return FEM_EINVAL;
  }
  for (int k = 0; k < Q; k++)
    for (int a = 0; a < 2; a++) {
      tp.t.B[k][a] = (T)op->tab.B[k * 2 + a];
      tp.t.H[k][a] = (T)(0.5 * op->tab.B[k * 2 + a]);
    }
  constexpr int NT = kTrilinearThreads;
  auto kern = fem_apply_trilinear_kernel<T, Q>;
  static FemKernelCache cache;
  int &max_bps = cache.here();
  if (max_bps < 0) {
    int per_sm = 0;
    FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, 0));
    max_bps = per_sm < 1 ? 1 : per_sm;
  }
  const int use = (bps <= 0 || bps > max_bps) ? max_bps : bps;
  const int64_t nblk = (prm.nsel + NT - 1) / NT;
  int64_t grid = (int64_t)op->nsm * use;
  if (grid > nblk) grid = nblk;
  if (grid > FEM_MAX_BLOCKS) grid = FEM_MAX_BLOCKS;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, NT, 0, op->stream()>>>(tp);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

// Assembled element matrices (Gauss diffusion, P = 2 and 3): one thread per
// element.
template <typename T, int P>
int launch_elmat(fem_op *op, const ApplyParams<T> &prm, int bps) {
  ElmatParams<T> ep;
  ep.a = prm;
  ep.E = op->E;
  if constexpr (std::is_same<T, dw>::value) ep.K = op->d_keldw;
  else if constexpr (sizeof(T) == 8) ep.K = reinterpret_cast<const T *>(op->d_kel);
  else ep.K = reinterpret_cast<const T *>(op->d_kel32);
  if (!ep.K) {
    fem_set_error("apply: the element-matrix body needs the operator's element matrices");
    return FEM_EINVAL;
  }
  // double words at P = 3: the layered body (three warps per 32 elements)
  constexpr bool LAYERS = std::is_same<T, dw>::value && P == 3;
  constexpr int NT = LAYERS ? kLayerThreads : kElmatThreads;
  constexpr int PER_BLOCK = LAYERS ? 32 * kLayerGroups : kElmatThreads;
  constexpr size_t smem = 0;
  auto kern = [] {
    if constexpr (LAYERS) return fem_apply_elmat_layers_kernel<P>;
    else return fem_apply_elmat_kernel<T, P>;
  }();
  static FemKernelCache cache;
  int &max_bps = cache.here();
  if (max_bps < 0) {
    if (smem > 0) FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    max_bps = per_sm < 1 ? 1 : per_sm;
  }
  const int use = (bps <= 0 || bps > max_bps) ? max_bps : bps;
  const int64_t nblk = (prm.nsel + PER_BLOCK - 1) / PER_BLOCK;
  int64_t grid = (int64_t)op->nsm * use;
  if (grid > nblk) grid = nblk;
  if (grid > FEM_MAX_BLOCKS) grid = FEM_MAX_BLOCKS;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, NT, smem, op->stream()>>>(ep);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

// Launch shape choice: 0..2 the line-based body with the three EPB
// candidates, 3..5 the slab body, 6 the trilinear body (Gauss diffusion at
// p = 1 only; the slab body's default elsewhere), 7 the element-matrix body
// (Gauss diffusion at p = 1, 2); the collocated mass operator (pointwise)
// has only the slab body.
// Double words (FP64 operators, choices 8..23): the line body and the
// element-matrix body.
template <int P, int Q, int KIND, bool COLLOC>
int launch_epb_dw(fem_op *op, const ApplyParams<dw> &prm, int choice, int bps) {
  if constexpr ((P == 2 || P == 3) && KIND == FEM_DIFFUSION && !COLLOC) {
    if (choice == FEM_CHOICE_DW_ELMAT) return launch_elmat<dw, P>(op, prm, bps);
  }
  if constexpr (KIND == FEM_DIFFUSION || !COLLOC) {
    switch (choice) {
      case 8: return launch_lines<dw, P, Q, COLLOC, EpbChoice<Q, 0>::value, KIND>(op, prm, bps);
      case 9: return launch_lines<dw, P, Q, COLLOC, EpbChoice<Q, 1>::value, KIND>(op, prm, bps);
      case 10: return launch_lines<dw, P, Q, COLLOC, EpbChoice<Q, 2>::value, KIND>(op, prm, bps);
      case 12: return launch_lines<dw, P, Q, COLLOC, EpbChoice<Q, 0>::value, KIND>(op, prm, bps, true);
      case 13: return launch_lines<dw, P, Q, COLLOC, EpbChoice<Q, 1>::value, KIND>(op, prm, bps, true);
      case 14: return launch_lines<dw, P, Q, COLLOC, EpbChoice<Q, 2>::value, KIND>(op, prm, bps, true);
      case 15: return launch_lines<dw, P, Q, COLLOC, EpbChoice<Q, 0>::value, KIND>(op, prm, bps, false, true);
      case 16: return launch_lines<dw, P, Q, COLLOC, EpbChoice<Q, 1>::value, KIND>(op, prm, bps, false, true);
      case 17: return launch_lines<dw, P, Q, COLLOC, EpbChoice<Q, 2>::value, KIND>(op, prm, bps, false, true);
      case 18: return launch_lines<dw, P, Q, COLLOC, EpbChoice<Q, 0>::value, KIND>(op, prm, bps, false, true, true);
      case 19: return launch_lines<dw, P, Q, COLLOC, EpbChoice<Q, 1>::value, KIND>(op, prm, bps, false, true, true);
      case 20: return launch_lines<dw, P, Q, COLLOC, EpbChoice<Q, 2>::value, KIND>(op, prm, bps, false, true, true);
      case 21: return launch_lines<dw, P, Q, COLLOC, EpbChoice<Q, 0>::value, KIND>(op, prm, bps, true, true, true);
      case 22: return launch_lines<dw, P, Q, COLLOC, EpbChoice<Q, 1>::value, KIND>(op, prm, bps, true, true, true);
      case 23: return launch_lines<dw, P, Q, COLLOC, EpbChoice<Q, 2>::value, KIND>(op, prm, bps, true, true, true);
      default: break;
    }
  }
  fem_set_error("apply: launch choice %d has no double-word body for this operator", choice);
  return FEM_EINVAL;
}

template <typename T, int P, int Q, int KIND, bool COLLOC>
int launch_epb(fem_op *op, const ApplyParams<T> &prm, int choice, int bps) {
  if constexpr (std::is_same<T, dw>::value) {
    return launch_epb_dw<P, Q, KIND, COLLOC>(op, prm, choice, bps);
  } else {
  if constexpr (P == 2 && KIND == FEM_DIFFUSION && !COLLOC) {
    if (choice == 6) return launch_trilinear<T, Q>(op, prm, bps);
  }
  if constexpr ((P == 2 || P == 3) && KIND == FEM_DIFFUSION && !COLLOC) {
    if (choice == 7) return launch_elmat<T, P>(op, prm, bps);
  }
  if constexpr (KIND == FEM_DIFFUSION || !COLLOC) {
    switch (choice) {
      case 0: return launch_lines<T, P, Q, COLLOC, EpbChoice<Q, 0>::value, KIND>(op, prm, bps);
      case 1: return launch_lines<T, P, Q, COLLOC, EpbChoice<Q, 1>::value, KIND>(op, prm, bps);
      case 2: return launch_lines<T, P, Q, COLLOC, EpbChoice<Q, 2>::value, KIND>(op, prm, bps);
      case 4: return launch_shape<T, P, Q, KIND, COLLOC, EpbChoice<Q, 1>::value>(op, prm, bps);
      case 5: return launch_shape<T, P, Q, KIND, COLLOC, EpbChoice<Q, 2>::value>(op, prm, bps);
      default: return launch_shape<T, P, Q, KIND, COLLOC, EpbChoice<Q, 0>::value>(op, prm, bps);
    }
  }
  switch (choice) {
    case 1: return launch_shape<T, P, Q, KIND, COLLOC, EpbChoice<Q, 1>::value>(op, prm, bps);
    case 2: return launch_shape<T, P, Q, KIND, COLLOC, EpbChoice<Q, 2>::value>(op, prm, bps);
    default: return launch_shape<T, P, Q, KIND, COLLOC, EpbChoice<Q, 0>::value>(op, prm, bps);
  }
  }
}

// Launch shapes are tunable (epb_choices) except for the collocated mass
// operator, which is pointwise.
// PART: 0 every rule, 1 the non-collocated ones only, 2 the collocated ones
// only (the double-word bodies compile the two groups in separate
// translation units, with different double-word sums: dw.cuh)
template <typename T, int P, int PART = 0>
int dispatch_q(fem_op *op, const ApplyParams<T> &prm, int choice, int bps) {
  constexpr int QG = (P + 1 <= FEM_MAX_Q) ? P + 1 : P;
  const bool diff = op->kind == FEM_DIFFUSION;
  if constexpr (PART == 2) {
    if (op->Q == P && op->colloc && diff) return launch_epb<T, P, P, FEM_DIFFUSION, true>(op, prm, choice, bps);
    fem_set_error(diff ? "apply: not a collocated operator"
                       : "apply: the collocated mass operator has no double-word body");
    return FEM_EINVAL;
  } else {
  if (op->Q == P) {
    if (op->colloc) {
      if constexpr (PART == 1) {
        fem_set_error("apply: collocated operators take the other dispatch");
        return FEM_EINVAL;
      } else if (diff) return launch_epb<T, P, P, FEM_DIFFUSION, true>(op, prm, choice, bps);
      if constexpr (std::is_same<T, dw>::value) {
        fem_set_error("apply: the collocated mass operator has no double-word body");
        return FEM_EINVAL;
      } else {
        return launch_shape<T, P, P, FEM_MASS, true, EpbChoice<P, 0>::value>(op, prm, bps);
      }
    }
    return diff ? launch_epb<T, P, P, FEM_DIFFUSION, false>(op, prm, choice, bps)
                : launch_epb<T, P, P, FEM_MASS, false>(op, prm, choice, bps);
  }
  if (op->Q == P + 1 && QG == P + 1)
    return diff ? launch_epb<T, P, QG, FEM_DIFFUSION, false>(op, prm, choice, bps)
                : launch_epb<T, P, QG, FEM_MASS, false>(op, prm, choice, bps);
  fem_set_error("apply: unsupported (P, q) = (%d, %d)", P, op->Q);
  return FEM_EINVAL;
  }
}

template <typename T>
int dispatch(fem_op *op, const ApplyParams<T> &prm, int choice, int bps) {
  switch (op->P) {
    case 2: return dispatch_q<T, 2>(op, prm, choice, bps);
    case 3: return dispatch_q<T, 3>(op, prm, choice, bps);
    case 4: return dispatch_q<T, 4>(op, prm, choice, bps);
    case 5: return dispatch_q<T, 5>(op, prm, choice, bps);
    case 6: return dispatch_q<T, 6>(op, prm, choice, bps);
    case 7: return dispatch_q<T, 7>(op, prm, choice, bps);
    case 8: return dispatch_q<T, 8>(op, prm, choice, bps);
    case 9: return dispatch_q<T, 9>(op, prm, choice, bps);
  }
  fem_set_error("apply: unsupported P = %d", op->P);
  return FEM_EINVAL;
}


}  // namespace fem_apply
