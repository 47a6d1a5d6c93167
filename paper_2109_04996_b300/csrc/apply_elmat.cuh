// Element body of the diffusion apply with assembled element matrices, for
// Gauss diffusion at P = 2 and 3 (p = 1, 2): one thread per element (the
// double-word body at P = 3: three warps per 32 elements, by layers).
//
// The operator is still y = G^T (B^T D B) G x (section "libCEED": operator
// decomposition); here the element block B^T D B is formed once at set-up,
//   K_e[a][b] = sum_q grad phi_a(q)^T D(q) grad phi_b(q),
// and the apply is the gather, the dense symmetric product y_e = K_e x_e and
// the scatter-add.  The paper keeps full assembly for first and second
// order and partial assembly for high order (section "Miniapps": Laghos'
// full and partial assembly options), and on B300 the FP64 apply agrees:
// FP64 runs at about 1/73 of the FP32 rate and bounds the partially assembled
// apply, while K_e costs (P^3)^2 FMAs per element (64 at p = 1, 729 at
// p = 2) against about 370 and 1500 FP64 instructions of the sum-factorized
// bodies, and its upper triangle (36 and 378 values) is no larger than the
// qdata those bodies read.
//
// Layout: the upper triangle packed by rows (a <= b), stored entry-major
// [P^3 (P^3 + 1) / 2][E] (fem_op::d_kel): the 32 elements of a warp load
// each entry in one coalesced access.  x_e and y_e stay in registers.  The
// double-word copy at P = 3 is in the layered body's order (below).
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

// Double words at P = 3, layered: the element's 27 nodes form NL = 3 layers
// of L = 9 (the z-planes), and K_e splits into the 3 diagonal blocks K_tt
// and the 3 off-diagonal blocks K_{t,t+1 mod 3} (t = 0, 1, 2 covers each
// pair of distinct layers once).  Warp t of a triple owns layer t of 32
// elements (one element per lane): it applies K_tt symmetrically (upper
// triangle), then K_{t,t+1} both ways -- y_t += K x_{t+1} and
// w = K^T x_t, the contribution to layer t+1 -- and hands w over in shared
// memory.  Every entry is read once and used twice, the three warps run the
// same 243 double-word FMAs per element, and a thread holds 9 rows of y
// instead of 27.  Measured at 5e7 DOFs (BP3 p = 2): 7.64 ms with one thread
// per element (x_e in shared memory, y_e in registers, 128 registers and
// 16 warps per SM), 5.03 ms layered (64 registers, x_t read back from
// shared memory after the diagonal block, 30 warps per SM).  K layout
// ("layer order", [378][E]): the three diagonal blocks' upper triangles (45
// entries each, row-major, i <= j), then the three off-diagonal blocks (81
// entries each, row-major, rows in layer t, columns in layer t+1 mod 3;
// fem_elmat_layer_src).
constexpr int kLayerGroups = 2;                         // element groups of 32 per block
constexpr int kLayerThreads = 96 * kLayerGroups;        // three warps per group

template <int P>
__global__ void __launch_bounds__(kLayerThreads, 5) fem_apply_elmat_layers_kernel(const ElmatParams<dw> ep) {
  static_assert(P == 3, "the layered body is written for P = 3");
  constexpr int P3 = 27, L = 9, NL = 3, TRI = L * (L + 1) / 2;
  // x_e and the handed-over w, [group][layer][row][lane]
  __shared__ dw xs[kLayerGroups][NL][L][32];
  __shared__ dw ws[kLayerGroups][NL][L][32];
  const ApplyParams<dw> &prm = ep.a;
  if (apply_skipped(prm)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp / NL, t = warp - grp * NL, tn = (t + 1) % NL;
  const int64_t E = ep.E;
  DotAcc<dw> dl;
  const int64_t per_block = 32 * kLayerGroups, step = (int64_t)gridDim.x * per_block;
  // the trip count is uniform over the block (barriers inside)
  for (int64_t base = (int64_t)blockIdx.x * per_block; base < prm.nsel; base += step) {
    const int64_t k_el = base + grp * 32 + lane;
    const bool valid = k_el < prm.nsel;
    const int64_t e = valid ? (prm.list ? (int64_t)prm.list[k_el] : k_el) : 0;
    const int32_t *en = prm.elem_nodes + e * P3;
    const dw *Kd = ep.K + (int64_t)(t * TRI) * E + e;
    const dw *Ko = ep.K + (int64_t)(NL * TRI + t * L * L) * E + e;
    for (int c = 0; c < prm.ncomp; c++) {
      const double *xc = prm.x + c * prm.N;
      double *yc = prm.y + c * prm.N;
      dw xt[L], y[L];
      const double c0 = valid ? gather_load(&xc[en[0]], prm.x_l2_only) : 0.0;
#pragma unroll
      for (int r = 0; r < L; r++) {
        xt[r] = valid ? gather_shifted<dw, true>(&xc[en[L * t + r]], prm.x_l2_only, c0) : dw(0.0f, 0.0f);
        xs[grp][t][r][lane] = xt[r];
        y[r] = dw(0.0f, 0.0f);
      }
      // K_tt, upper triangle
      const dw *kp = Kd;
#pragma unroll
      for (int i = 0; i < L; i++) {
#pragma unroll
        for (int j = i; j < L; j++) {
          const dw kv = ld_entry(kp);
          kp += E;
          y[i] = fma(kv, xt[j], y[i]);
          if (j != i) y[j] = fma(kv, xt[i], y[j]);
        }
      }
      __syncthreads();
      // K_{t,t+1}: y_t += K x_{t+1}, w = K^T x_t
      dw xn[L], w[L];
#pragma unroll
      for (int j = 0; j < L; j++) {
        xn[j] = xs[grp][tn][j][lane];
        w[j] = dw(0.0f, 0.0f);
      }
      // (x_t is read back from shared memory from here on: its registers
      // are free for w)
      kp = Ko;
#pragma unroll
      for (int i = 0; i < L; i++) {
        const dw xi = xs[grp][t][i][lane];
#pragma unroll
        for (int j = 0; j < L; j++) {
          const dw kv = ld_entry(kp);
          kp += E;
          y[i] = fma(kv, xn[j], y[i]);
          w[j] = fma(kv, xi, w[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < L; j++) ws[grp][tn][j][lane] = w[j];
      __syncthreads();
#pragma unroll
      for (int r = 0; r < L; r++) {
        y[r] += ws[grp][t][r][lane];
        if (valid) {
          atomic_add(&yc[en[L * t + r]], y[r]);
          dl.add(y[r], xs[grp][t][r][lane]);
        }
      }
    }
  }
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
