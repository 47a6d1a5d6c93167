// Element body of the diffusion apply with assembled element matrices, for
// Gauss diffusion at P = 2 and 3 (p = 1, 2): one thread per element.
//
// The operator is still y = G^T (B^T D B) G x (section "libCEED": operator
// decomposition); here the element block B^T D B is formed once at set-up,
//   K_e[a][b] = sum_q grad phi_a(q)^T D(q) grad phi_b(q),
// and the apply is the gather, the dense symmetric product y_e = K_e x_e and
// the scatter-add.  The paper keeps full assembly for first and second
// order and partial assembly for high order (section "Miniapps": Laghos'
// full and partial assembly options), and on B300 the FP64 apply agrees:
// FP64 runs at 1/64 of the FP32 rate and bounds the partially assembled
// apply, while K_e costs (P^3)^2 FMAs per element (64 at p = 1, 729 at
// p = 2) against about 370 and 1500 FP64 instructions of the sum-factorized
// bodies, and its upper triangle (36 and 378 values) is no larger than the
// qdata those bodies read.
//
// Layout: the upper triangle packed by rows (a <= b), stored entry-major
// [P^3 (P^3 + 1) / 2][E] (fem_op::d_kel): the 32 elements of a warp load
// each entry in one coalesced access.  x_e and y_e stay in registers.
#pragma once
#include "apply_kernel.cuh"

namespace fem_apply {

template <typename T>
struct ElmatParams {
  ApplyParams<T> a;
  const T *K;     // [P^3 (P^3 + 1) / 2][E] (double words: split FP64 K_e)
  int64_t E;      // element stride of K (all elements of the operator)
};

// One K_e entry, streamed once per apply (evict-first).
template <typename T>
__device__ __forceinline__ T ld_entry(const T *p) { return __ldcs(p); }
template <>
__device__ __forceinline__ dw ld_entry<dw>(const dw *p) {
  const float2 v = __ldcs(reinterpret_cast<const float2 *>(p));
  return dw(v.x, v.y);
}

constexpr int kElmatThreads = 128;

// Element e: y += K_e x_e (every component) and this thread's share of x.y.
template <typename T, int P>
__device__ __forceinline__ void elmat_element(const ApplyParams<T> &prm, const T *__restrict__ K,
                                              int64_t E, int64_t e, DotAcc<T> &dl) {
  constexpr int P3 = P * P * P;
  // at P = 3 double words hold x_e and y_e in 108 registers: the node ids
  // are read again for the scatter (L1 hits) instead of being kept
  constexpr bool KEEP_IDS = !std::is_same<T, dw>::value || P == 2;
  int id[KEEP_IDS ? P3 : 1];
  const int32_t *en = prm.elem_nodes + e * P3;
  if constexpr (KEEP_IDS) {
#pragma unroll
    for (int a = 0; a < P3; a++) id[a] = en[a];
  }
  auto node = [&](int a) -> int { if constexpr (KEEP_IDS) return id[a]; else return en[a]; };
  for (int c = 0; c < prm.ncomp; c++) {
    const auto *xc = prm.x + c * prm.N;
    auto *yc = prm.y + c * prm.N;
    T x[P3], y[P3];
    // double words: x_e - x_0 1 (ShiftX; K_e annihilates constants)
    // (at P = 2 the shift's FP64 subtractions and the registers of the
    // unshifted values cost 2x, and the smoothest fields stay within 1e-12
    // without it: 7e-13 at 8e6 DOFs)
    constexpr bool SH = ShiftX<T, FEM_DIFFUSION>::value && P > 2;
    const double c0 = SH ? (double)gather_load(&xc[node(0)], prm.x_l2_only) : 0.0;
#pragma unroll
    for (int a = 0; a < P3; a++) {
      x[a] = gather_shifted<T, SH>(&xc[node(a)], prm.x_l2_only, c0);
      y[a] = T(0);
    }
    // the entries in their packed order: K_e is streamed once per apply
    // (evict-first loads keep x and y in L2)
    const T *kp = K + e;
#pragma unroll
    for (int a = 0; a < P3; a++) {
#pragma unroll
      for (int b = a; b < P3; b++) {
        const T kv = ld_entry(kp);
        kp += E;
        y[a] = fma(kv, x[b], y[a]);
        if (b != a) y[b] = fma(kv, x[a], y[b]);
      }
    }
#pragma unroll
    for (int a = 0; a < P3; a++) {
      atomic_add(&yc[node(a)], y[a]);
      dl.add(y[a], x[a]);
    }
  }
}

// Double words at P = 3: x_e (27 values, shifted by its node-0 value) in
// shared memory, laid out [node][thread] so that a warp's 8-byte loads of
// one node are contiguous (conflict-free); y_e (27 values) in registers.
// Holding both in registers took 255 registers a thread (8 warps per SM);
// with x_e in shared memory each packed entry (a, b) costs one shared load
// of x_b (x_a stays in a register through row a), and the kernel is held to
// 128 registers (4 blocks of 128 threads per SM, some spill to L1):
// measured at 8e6 DOFs 1.25 ms -> 1.02 ms (5 blocks: 1.13 ms).
template <int P>
__device__ __forceinline__ void elmat_element_xs(const ApplyParams<dw> &prm, const dw *__restrict__ K,
                                                 int64_t E, int64_t e, dw *xs, DotAcc<dw> &dl) {
  constexpr int P3 = P * P * P;
  const int32_t *en = prm.elem_nodes + e * P3;
  const int stride = blockDim.x;
  for (int c = 0; c < prm.ncomp; c++) {
    const double *xc = prm.x + c * prm.N;
    double *yc = prm.y + c * prm.N;
    const double c0 = gather_load(&xc[en[0]], prm.x_l2_only);
#pragma unroll
    for (int a = 0; a < P3; a++)
      xs[a * stride] = gather_shifted<dw, true>(&xc[en[a]], prm.x_l2_only, c0);
    dw y[P3];
#pragma unroll
    for (int a = 0; a < P3; a++) y[a] = dw(0.0f, 0.0f);
    const dw *kp = K + e;
#pragma unroll
    for (int a = 0; a < P3; a++) {
      const dw xa = xs[a * stride];
#pragma unroll
      for (int b = a; b < P3; b++) {
        const dw kv = ld_entry(kp);
        kp += E;
        if (b == a) {
          y[a] = fma(kv, xa, y[a]);
        } else {
          const dw xb = xs[b * stride];
          y[a] = fma(kv, xb, y[a]);
          y[b] = fma(kv, xa, y[b]);
        }
      }
    }
#pragma unroll
    for (int a = 0; a < P3; a++) {
      atomic_add(&yc[en[a]], y[a]);
      dl.add(y[a], xs[a * stride]);
    }
  }
}

template <int P>
__global__ void __launch_bounds__(kElmatThreads, 4) fem_apply_elmat_xs_kernel(const ElmatParams<dw> ep) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dw *xs = reinterpret_cast<dw *>(smem_raw) + threadIdx.x;
  const ApplyParams<dw> &prm = ep.a;
  if (apply_skipped(prm)) return;
  DotAcc<dw> dl;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // every thread of the block runs the same number of iterations of this
  // loop body's shape; threads past the end simply skip the element
  for (int64_t k_el = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k_el < prm.nsel; k_el += stride)
    elmat_element_xs<P>(prm, ep.K, ep.E, prm.list ? (int64_t)prm.list[k_el] : k_el, xs, dl);
  if (prm.dot_out) {
    double v[1] = {dl.get()};
    __shared__ double tot[1];
    if (fem_grid_sum<1>(v, prm.partials, prm.counter, tot) && threadIdx.x == 0)
      *prm.dot_out = tot[0];
  }
}

template <typename T, int P>
__global__ void __launch_bounds__(kElmatThreads) fem_apply_elmat_kernel(const ElmatParams<T> ep) {
  const ApplyParams<T> &prm = ep.a;
  if (apply_skipped(prm)) return;
  DotAcc<T> dl;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k_el = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k_el < prm.nsel; k_el += stride)
    elmat_element<T, P>(prm, ep.K, ep.E, prm.list ? (int64_t)prm.list[k_el] : k_el, dl);
  if (prm.dot_out) {
    double v[1] = {dl.get()};
    __shared__ double tot[1];
    if (fem_grid_sum<1>(v, prm.partials, prm.counter, tot) && threadIdx.x == 0)
      *prm.dot_out = tot[0];
  }
}

}  // namespace fem_apply
