// Forward GEMMs of the per-element MLP on the 5th-generation tensor cores:
//   C = epilogue(A B^T), A [M][K] and B [N][K] bf16, row-major (K-major),
//   FP32 accumulation in tensor memory, epilogue + bias[col], ReLU, store
//   bf16 or fp32 to C [M][ldc].
//
// One CTA of 4 warps per 128 x 128 output tile.  K is staged 64 at a time:
// every thread copies 16-byte row segments of A and B (cp.async, zero-filled
// beyond M / N) into shared memory in the canonical no-swizzle K-major
// layout -- 8-row x 16-byte core matrices, consecutive along K (leading
// byte offset 128) and then along the rows (stride byte offset 1024) -- then
// one thread issues four tcgen05.mma (kind::f16, M=128, N=128, K=16 each)
// and a tcgen05.commit that arrives on an mbarrier.  The 128 x 128 FP32
// accumulator lives in 128 TMEM columns (allocated per CTA); the epilogue
// reads it with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows).
// Every mbarrier wait is bounded: on expiry the CTA records an error, waits
// (bounded) for its own MMAs, frees its TMEM and returns.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace fem_mlp_tc {

constexpr int TM = 128, TN = 128, TK = 64, NT = 128;
constexpr int kTileBytes = TM * TK * 2;           // 16 KB per operand stage
constexpr int kSmemBytes = 56 * 1024;             // caps residency at 4 CTAs / SM (TMEM: 4 x 128 columns)
constexpr unsigned long long kWaitLimit = 1ull << 22;   // try_wait polls before giving up

struct TcArgs {
  const __nv_bfloat16 *A, *B;
  int64_t lda, ldb, M;
  int N, K;
  void *C;
  int64_t ldc;
  int out_bf16;
  const float *bias;
  int relu;
  int *error;           // set to 1 if a wait ran out
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start >> 4, leading byte offset >> 4 at
// bit 16, stride byte offset >> 4 at bit 32, descriptor version 1 at bit 46,
// no swizzle (layout type 0 at bits 61-63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B bf16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
  const int n = valid ? 16 : 0;   // 0: zero-fill, nothing read
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n) : "memory");
}

// Bounded wait for the mbarrier's phase `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (unsigned long long it = 0; it < kWaitLimit; it++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(NT) gemm_tc_kernel(const TcArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  unsigned char *sA = smem, *sB = smem + kTileBytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (int64_t)blockIdx.x * TM;
  const int col0 = blockIdx.y * TN;
  const uint32_t bar = smem_u32(&mbar);
  if (threadIdx.x == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TN) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const int nstages = (g.K + TK - 1) / TK;   // K segments past K are zero-filled
  uint32_t phase = 0;
  for (int st = 0; st < nstages; st++) {
    // ---- stage K columns [st*TK, st*TK + TK) of A and B into shared memory
    const int kbase = st * TK;
#pragma unroll
    for (int c = 0; c < (TM * TK / 8) / NT; c++) {
      const int chunk = threadIdx.x + c * NT;          // 0 .. 1023
      const int r = chunk >> 3, k8 = chunk & 7;          // row, 8-element segment
      const uint32_t off = (uint32_t)(((r >> 3) * (TK / 8) + k8) * 128 + (r & 7) * 16);
      const int kc = kbase + k8 * 8;
      const bool vk = kc < g.K;
      const int64_t ra = row0 + r;
      const bool va = vk && ra < g.M;
      cp_async16(smem_u32(sA + off), g.A + (va ? ra * g.lda + kc : 0), va);
      const int rb = col0 + r;
      const bool vb = vk && rb < g.N;
      cp_async16(smem_u32(sB + off), g.B + (vb ? (int64_t)rb * g.ldb + kc : 0), vb);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    // generic-proxy writes of shared memory -> visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < TK / 16; kk++) {
        // K = 16 per instruction: two core matrices along K (256 bytes)
        const uint64_t ad = smem_desc(smem_u32(sA) + kk * 256, 128, (TK / 8) * 128);
        const uint64_t bd = smem_desc(smem_u32(sB) + kk * 256, 128, (TK / 8) * 128);
        const uint32_t acc = (st > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                   : "memory");
    }
    // the stage buffers are reused: wait for these MMAs to finish; if the
    // wait runs out, record it and give the MMAs in flight a second bounded
    // wait before the TMEM they write is freed
    if (!mbar_wait(bar, phase)) {
      if (threadIdx.x == 0) { s_fail = 1; atomicExch(g.error, 1); }
      mbar_wait(bar, phase);
    }
    phase ^= 1;
    __syncthreads();
    if (s_fail) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (!s_fail) {
    // ---- epilogue: warp w reads tile rows 32w + lane, 32 columns at a time
    const int64_t row = row0 + warp * 32 + lane;
#pragma unroll 1
    for (int cb = 0; cb < TN; cb += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
            "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
            "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
            "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (row < g.M) {
#pragma unroll
        for (int j = 0; j < 32; j++) {
          const int col = col0 + cb + j;
          if (col < g.N) {
            float x = __uint_as_float(v[j]);
            if (g.bias) x += g.bias[col];
            if (g.relu) x = x > 0.0f ? x : 0.0f;
            if (g.out_bf16)
              reinterpret_cast<__nv_bfloat16 *>(g.C)[row * g.ldc + col] = __float2bfloat16(x);
            else
              reinterpret_cast<float *>(g.C)[row * g.ldc + col] = x;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TN) : "memory");
}

}  // namespace fem_mlp_tc
