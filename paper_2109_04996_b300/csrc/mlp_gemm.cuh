// Dense GEMM kernels of the per-element MLP (learned preconditioner):
//   C = epilogue( op(A) op(B)^T ),  op(A) [M x K], op(B) [N x K]
// A stored row-major [M][K] (AT = false) or [K][M] (AT = true); B stored
// [N][K] (BT = false) or [K][N] (BT = true).  Epilogue: + bias[col], ReLU,
// times (mask > 0) (ReLU backward), store bf16 / fp32, or atomic-add fp32
// (split-K over grid.z).
//
// bf16 path: 128 x 128 x 32 block tiles, 8 warps of 64 x 32, mma.sync
// m16n8k16 (bf16 in, fp32 accumulate) fed by ldmatrix from padded shared
// tiles (pitch 40 elements: conflict-free ldmatrix rows), next K tile
// prefetched into registers while the current one is multiplied.
// fp32 path (debug mode, exact-ish reference): 64 x 64 x 16 tiles, 4 x 4
// outputs per thread, FFMA.
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

constexpr int BM = 128, BN = 128, BK = 32, PITCH = BK + 8, GT = 256;

__device__ __forceinline__ void ldsm_x4(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3,
                                        const void *p) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Load one operand tile [ROWS x BK] (rows of the logical [rows x K] matrix)
// into registers: 2 chunks of 8 bf16 per thread.
template <bool T_STORED, int ROWS>
struct TileLoader {
  uint4 v[ROWS * BK / 8 / GT];
  __device__ void load(const __nv_bfloat16 *P, int64_t ld, int64_t rows_total, int64_t r0,
                       int k0) {
#pragma unroll
    for (int i = 0; i < ROWS * BK / 8 / GT; i++) {
      const int idx = threadIdx.x + i * GT;
      if (!T_STORED) {
        const int r = idx / (BK / 8), ch = idx % (BK / 8);
        const int64_t gr = r0 + r;
        if (gr < rows_total)
          v[i] = *reinterpret_cast<const uint4 *>(P + gr * ld + k0 + ch * 8);
        else
          v[i] = make_uint4(0, 0, 0, 0);
      } else {
        // storage [K][rows]: chunk of 8 consecutive rows at one k
        const int kk = idx / (ROWS / 8), ch = idx % (ROWS / 8);
        const int64_t gr = r0 + ch * 8;
        const __nv_bfloat16 *src = P + (int64_t)(k0 + kk) * ld + gr;
        if (gr + 8 <= rows_total) {
          v[i] = *reinterpret_cast<const uint4 *>(src);
        } else {
          __nv_bfloat16 t[8];
#pragma unroll
          for (int j = 0; j < 8; j++) t[j] = (gr + j < rows_total) ? src[j] : __float2bfloat16(0.0f);
          v[i] = *reinterpret_cast<uint4 *>(t);
        }
      }
    }
  }
  __device__ void store(__nv_bfloat16 *S) const {
#pragma unroll
    for (int i = 0; i < ROWS * BK / 8 / GT; i++) {
      const int idx = threadIdx.x + i * GT;
      if (!T_STORED) {
        const int r = idx / (BK / 8), ch = idx % (BK / 8);
        *reinterpret_cast<uint4 *>(S + r * PITCH + ch * 8) = v[i];
      } else {
        const int kk = idx / (ROWS / 8), ch = idx % (ROWS / 8);
        const __nv_bfloat16 *t = reinterpret_cast<const __nv_bfloat16 *>(&v[i]);
#pragma unroll
        for (int j = 0; j < 8; j++) S[(ch * 8 + j) * PITCH + kk] = t[j];
      }
    }
  }
};

template <bool AT, bool BT>
__global__ void __launch_bounds__(GT) gemm_bf16_kernel(const GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 As[BM * PITCH];
  __shared__ __align__(16) __nv_bfloat16 Bs[BN * PITCH];
  const __nv_bfloat16 *A = (const __nv_bfloat16 *)g.A, *B = (const __nv_bfloat16 *)g.B;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  const int kper = g.K / g.ksplit;
  const int kbeg = blockIdx.z * kper, kend = kbeg + kper;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int q = 0; q < 4; q++) acc[i][j][q] = 0.0f;
  TileLoader<AT, BM> la;
  TileLoader<BT, BN> lb;
  la.load(A, g.lda, g.M, m0, kbeg);
  lb.load(B, g.ldb, g.N, n0, kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    __syncthreads();
    la.store(As);
    lb.store(Bs);
    __syncthreads();
    if (k0 + BK < kend) {
      la.load(A, g.lda, g.M, m0, k0 + BK);
      lb.load(B, g.ldb, g.N, n0, k0 + BK);
    }
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      unsigned af[4][4], bfr[4][2];
#pragma unroll
      for (int mi = 0; mi < 4; mi++) {
        const __nv_bfloat16 *p = As + (wm + mi * 16 + (lane & 15)) * PITCH + kk + (lane >> 4) * 8;
        ldsm_x4(af[mi][0], af[mi][1], af[mi][2], af[mi][3], p);
      }
#pragma unroll
      for (int nj = 0; nj < 2; nj++) {
        const __nv_bfloat16 *p =
            Bs + (wn + nj * 16 + (lane & 7) + (lane >> 4) * 8) * PITCH + kk + ((lane >> 3) & 1) * 8;
        ldsm_x4(bfr[2 * nj][0], bfr[2 * nj][1], bfr[2 * nj + 1][0], bfr[2 * nj + 1][1], p);
      }
#pragma unroll
      for (int mi = 0; mi < 4; mi++)
#pragma unroll
        for (int ni = 0; ni < 4; ni++)
          mma_bf16(acc[mi][ni], af[mi][0], af[mi][1], af[mi][2], af[mi][3], bfr[ni][0], bfr[ni][1]);
    }
  }
  // epilogue
#pragma unroll
  for (int mi = 0; mi < 4; mi++)
#pragma unroll
    for (int ni = 0; ni < 4; ni++)
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int64_t r = m0 + wm + mi * 16 + (lane >> 2) + h * 8;
        const int c = n0 + wn + ni * 8 + (lane & 3) * 2;
        if (r >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 2; j++) {
          if (c + j >= g.N) continue;
          float v = acc[mi][ni][h * 2 + j];
          if (g.bias) v += g.bias[c + j];
          if (g.relu) v = v > 0.0f ? v : 0.0f;
          if (g.mask) {
            const float mk = __bfloat162float(((const __nv_bfloat16 *)g.mask)[r * g.ldm + c + j]);
            if (!(mk > 0.0f)) v = 0.0f;
          }
          if (g.accumulate) atomicAdd((float *)g.C + r * g.ldc + c + j, v);
          else if (g.out_bf16) ((__nv_bfloat16 *)g.C)[r * g.ldc + c + j] = __float2bfloat16(v);
          else ((float *)g.C)[r * g.ldc + c + j] = v;
        }
      }
}

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
