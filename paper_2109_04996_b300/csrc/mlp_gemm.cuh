// Arguments of the per-element MLP's dense products and the FP32 GEMM of
// its debug mode (mode 1):
//   C = epilogue( op(A) op(B)^T ),  op(A) [M x K], op(B) [N x K]
// A stored row-major [M][K] (AT = false) or [K][M] (AT = true); B stored
// [N][K] (BT = false) or [K][N] (BT = true).  Epilogue: + bias[col], ReLU,
// times (mask > 0) (ReLU backward), store fp32, or atomic-add fp32 (split-K
// over grid.z).  64 x 64 x 16 tiles, 4 x 4 outputs per thread, FFMA.  The
// bf16 products of mode 0 run on the tensor cores (mlp_tc.cuh).
// Requirements: K (per split) and the leading dimensions are multiples of 8;
// rows / columns beyond M / N are masked.
#pragma once
#include <cuda_bf16.h>

#include "fem_internal.h"

namespace fem_mlp_k {

struct GemmArgs {
  const void *A, *B;
  int64_t lda, ldb;
  int64_t M;
  int N, K;             // K of the whole product
  int ksplit;           // grid.z splits of K (each a multiple of 32)
  void *C;
  int64_t ldc;
  int out_bf16;         // 1: store bf16, 0: fp32
  int accumulate;       // 1: atomicAdd into fp32 C
  const float *bias;    // [N] or null
  int relu;
  const void *mask;     // same type as inputs, [M][ldm], multiply by (mask > 0)
  int64_t ldm;
};

// FP32 reference path (debug mode).
template <bool AT, bool BT>
__global__ void __launch_bounds__(256) gemm_f32_kernel(const GemmArgs g) {
  constexpr int TB = 64, TK = 16;
  __shared__ float As[TK][TB + 1], Bs[TK][TB + 1];
  const float *A = (const float *)g.A, *B = (const float *)g.B;
  const int64_t m0 = (int64_t)blockIdx.x * TB;
  const int n0 = blockIdx.y * TB;
  const int kper = g.K / g.ksplit;
  const int kbeg = blockIdx.z * kper, kend = kbeg + kper;
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  float acc[4][4] = {};
  for (int k0 = kbeg; k0 < kend; k0 += TK) {
    for (int i = threadIdx.x; i < TB * TK; i += 256) {
      const int r = i / TK, k = i % TK;
      const int64_t gr = m0 + r;
      const int64_t gn = n0 + r;
      float av = 0.0f, bv = 0.0f;
      if (gr < g.M && k0 + k < kend) av = AT ? A[(int64_t)(k0 + k) * g.lda + gr] : A[gr * g.lda + k0 + k];
      if (gn < g.N && k0 + k < kend) bv = BT ? B[(int64_t)(k0 + k) * g.ldb + gn] : B[gn * g.ldb + k0 + k];
      As[k][r] = av;
      Bs[k][r] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; k++)
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] += As[k][tr * 4 + i] * Bs[k][tc * 4 + j];
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int64_t r = m0 + tr * 4 + i;
      const int c = n0 + tc * 4 + j;
      if (r >= g.M || c >= g.N) continue;
      float v = acc[i][j];
      if (g.bias) v += g.bias[c];
      if (g.relu) v = v > 0.0f ? v : 0.0f;
      if (g.mask && !(((const float *)g.mask)[r * g.ldm + c] > 0.0f)) v = 0.0f;
      if (g.accumulate) atomicAdd((float *)g.C + r * g.ldc + c, v);
      else ((float *)g.C)[r * g.ldc + c] = v;
    }
}

}  // namespace fem_mlp_k
