// Forward GEMMs of the per-element MLP on the 5th-generation tensor cores:
//   C = epilogue(A B^T), A [M][K] and B [N][K] bf16, row-major (K-major),
//   FP32 accumulation in tensor memory, epilogue + bias[col], ReLU, store
//   bf16 or fp32 to C [M][ldc].
//
// One CTA of 4 warps per 128 x 128 output tile.  K is cut into 32-wide
// stages held in a ring of NS shared-memory buffers: every thread copies
// 16-byte row segments of A and B (cp.async, zero-filled beyond M, N or K)
// into the canonical no-swizzle K-major layout -- 8-row x 16-byte core
// matrices, consecutive along K (leading byte offset 128) and then along the
// rows (stride byte offset 512) -- and the copies of the next NS-1 stages
// stay in flight while one thread issues the current stage's two
// tcgen05.mma (kind::f16, M=128, N=128, K=16 each) and a tcgen05.commit
// that arrives on the stage buffer's mbarrier; a buffer is refilled once
// that mbarrier shows its MMAs done.  The 128 x 128 FP32 accumulator lives
// in 128 TMEM columns (allocated per CTA); the epilogue reads it with
// tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows).  Every
// mbarrier wait is bounded: on expiry the CTA records an error, waits
// (bounded) for its own MMAs, frees its TMEM and returns.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace fem_mlp_tc {

constexpr int TM = 128, TN = 128, TK = 32, NT = 128, NS = 3;
constexpr int kTileBytes = TM * TK * 2;           // 8 KB per operand and stage
constexpr int kStageBytes = 2 * kTileBytes;       // A and B
constexpr int kSmemBytes = NS * kStageBytes + 1024;   // 49 KB: 4 CTAs / SM (TMEM: 4 x 128 columns)
constexpr unsigned long long kWaitLimit = 1ull << 22;   // try_wait polls before giving up

struct TcArgs {
  const __nv_bfloat16 *A, *B;
  int64_t lda, ldb, M;
  int N, K;
  int kchunk;           // K columns per blockIdx.z (split-K; multiple of TK)
  void *C;
  int64_t ldc;
  int out_bf16;
  int accumulate;       // 1: atomic-add into fp32 C (split-K), no bias / ReLU
  const float *bias;
  int relu;
  const __nv_bfloat16 *mask;   // times (mask[row][col] > 0), or null
  int64_t ldm;
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

// cp.async.wait_group with a run-time count of groups allowed to stay pending
__device__ __forceinline__ void cp_async_wait_pending(int n) {
  if (n <= 0) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  else if (n == 1) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  else if (n == 2) asm volatile("cp.async.wait_group 2;\n" ::: "memory");
  else asm volatile("cp.async.wait_group 3;\n" ::: "memory");
}

// Two FP32 values as packed bf16 (round to nearest even), lo at the lower
// address.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&h);
}

// Copies of K stage `st` (columns [k0 + st*TK, k0 + st*TK + TK), below
// kend) into stage buffer b.
__device__ __forceinline__ void load_stage(const TcArgs &g, unsigned char *buf, int st, int64_t row0,
                                           int col0, int k0, int kend) {
  unsigned char *sA = buf, *sB = buf + kTileBytes;
  const int kbase = k0 + st * TK;
#pragma unroll
  for (int c = 0; c < (TM * TK / 8) / NT; c++) {
    const int chunk = threadIdx.x + c * NT;          // 0 .. 511
    const int r = chunk / (TK / 8), k8 = chunk % (TK / 8);   // row, 8-element segment
    const uint32_t off = (uint32_t)(((r >> 3) * (TK / 8) + k8) * 128 + (r & 7) * 16);
    const int kc = kbase + k8 * 8;
    const bool vk = kc < kend;
    const int64_t ra = row0 + r;
    const bool va = vk && ra < g.M;
    cp_async16(smem_u32(sA + off), g.A + (va ? ra * g.lda + kc : 0), va);
    const int rb = col0 + r;
    const bool vb = vk && rb < g.N;
    cp_async16(smem_u32(sB + off), g.B + (vb ? (int64_t)rb * g.ldb + kc : 0), vb);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__global__ void __launch_bounds__(NT) gemm_tc_kernel(const TcArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[NS];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // blockIdx.x runs over the output tiles with the column tiles of a row
  // block adjacent: they read the same rows of A, which the later ones find
  // in L2
  const int ntn = (g.N + TN - 1) / TN;
  const int64_t row0 = (int64_t)(blockIdx.x / ntn) * TM;
  const int col0 = (int)(blockIdx.x % ntn) * TN;
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int b = 0; b < NS; b++)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[b])) : "memory");
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
  const int k0 = blockIdx.z * g.kchunk;
  const int kend = k0 + g.kchunk < g.K ? k0 + g.kchunk : g.K;
  const int nst = kend > k0 ? (kend - k0 + TK - 1) / TK : 0;   // segments past kend are zero-filled
  // prologue: the first NS stages in flight
  int issued = 0;
  int committed = -1;   // the stage whose MMAs were committed last
  for (; issued < NS && issued < nst; issued++) load_stage(g, smem + issued * kStageBytes, issued, row0, col0, k0, kend);
  for (int st = 0; st < nst; st++) {
    const int b = st % NS;
    // stage st's copies done (later groups may stay pending)
    cp_async_wait_pending(issued - st - 1);
    // generic-proxy writes of shared memory -> visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t base = smem_u32(smem + b * kStageBytes);
#pragma unroll
      for (int kk = 0; kk < TK / 16; kk++) {
        // K = 16 per instruction: two core matrices along K (256 bytes)
        const uint64_t ad = smem_desc(base + kk * 256, 128, (TK / 8) * 128);
        const uint64_t bd = smem_desc(base + kTileBytes + kk * 256, 128, (TK / 8) * 128);
        const uint32_t acc = (st > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&mbar[b]))
                   : "memory");
    }
    committed = st;
    // refill the buffer of stage st - 1 (its MMAs were issued one step ago)
    // with stage st - 1 + NS, once those MMAs are done
    const int sp = st - 1;
    if (sp >= 0 && sp + NS < nst) {
      const int bp = sp % NS;
      if (!mbar_wait(smem_u32(&mbar[bp]), (uint32_t)((sp / NS) & 1))) {
        if (threadIdx.x == 0) { s_fail = 1; atomicExch(g.error, 1); }
      }
      __syncthreads();
      if (s_fail) break;
      load_stage(g, smem + bp * kStageBytes, sp + NS, row0, col0, k0, kend);
      issued++;
    }
  }
  // the last commit covers every MMA issued before it; after a failed wait
  // it is the MMAs' second (bounded) wait before their TMEM is freed
  if (committed >= 0) {
    const uint32_t bl = smem_u32(&mbar[committed % NS]), par = (uint32_t)((committed / NS) & 1);
    if (!mbar_wait(bl, par)) {
      if (threadIdx.x == 0) { s_fail = 1; atomicExch(g.error, 1); }
      mbar_wait(bl, par);
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (!s_fail && nst > 0) {
    // ---- epilogue.  After tcgen05.ld a lane holds 32 consecutive columns
    // of its own row.  Plain stores (vec): the lane writes them as 16-byte
    // vectors (bf16: 4, fp32: 8), one 64- or 128-byte row segment.  Atomic
    // adds (split K) or unaligned C: each 32-column chunk is staged in the
    // free stage buffers so that a warp adds its 32 rows with the lanes
    // along the columns.  The tile's bias is staged there in both cases.
    const bool vec = !g.accumulate && g.ldc % 8 == 0 && (reinterpret_cast<uintptr_t>(g.C) & 15) == 0 &&
                     (!g.mask || (g.ldm % 8 == 0 && (reinterpret_cast<uintptr_t>(g.mask) & 15) == 0));
    float *stile = reinterpret_cast<float *>(smem);        // [128][33]
    float *sbias = stile + TM * 33;                          // [TN]
    for (int i = threadIdx.x; i < TN; i += NT)
      sbias[i] = (g.bias && col0 + i < g.N) ? g.bias[col0 + i] : 0.0f;
    __syncthreads();
    const int rloc = warp * 32 + lane;                      // this thread's TMEM lane = tile row
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
      if (vec) {
        const int64_t row = row0 + rloc;
        const int cbase = col0 + cb;
        if (row < g.M) {
          float x[32];
#pragma unroll
          for (int j = 0; j < 32; j++) {
            x[j] = __uint_as_float(v[j]) + sbias[cb + j];
            if (g.relu) x[j] = x[j] > 0.0f ? x[j] : 0.0f;
          }
          if (cbase + 32 <= g.N) {
            if (g.mask) {
              const uint4 *mp = reinterpret_cast<const uint4 *>(g.mask + row * g.ldm + cbase);
#pragma unroll
              for (int q = 0; q < 4; q++) {
                const uint4 m = mp[q];
                const uint32_t w[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
                for (int t = 0; t < 4; t++) {
                  if (!(__uint_as_float(w[t] << 16) > 0.0f)) x[8 * q + 2 * t] = 0.0f;
                  if (!(__uint_as_float(w[t] & 0xffff0000u) > 0.0f)) x[8 * q + 2 * t + 1] = 0.0f;
                }
              }
            }
            if (g.out_bf16) {
              uint4 *cp = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(g.C) + row * g.ldc + cbase);
#pragma unroll
              for (int q = 0; q < 4; q++)
                cp[q] = make_uint4(pack_bf16x2(x[8 * q], x[8 * q + 1]), pack_bf16x2(x[8 * q + 2], x[8 * q + 3]),
                                   pack_bf16x2(x[8 * q + 4], x[8 * q + 5]), pack_bf16x2(x[8 * q + 6], x[8 * q + 7]));
            } else {
              float4 *cp = reinterpret_cast<float4 *>(reinterpret_cast<float *>(g.C) + row * g.ldc + cbase);
#pragma unroll
              for (int q = 0; q < 8; q++) cp[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
            }
          } else {
            // the ragged last chunk of N
#pragma unroll
            for (int j = 0; j < 32; j++) {
              const int col = cbase + j;
              if (col < g.N) {
                float y = x[j];
                if (g.mask && !(__bfloat162float(g.mask[row * g.ldm + col]) > 0.0f)) y = 0.0f;
                if (g.out_bf16)
                  reinterpret_cast<__nv_bfloat16 *>(g.C)[row * g.ldc + col] = __float2bfloat16(y);
                else
                  reinterpret_cast<float *>(g.C)[row * g.ldc + col] = y;
              }
            }
          }
        }
        continue;
      }
#pragma unroll
      for (int j = 0; j < 32; j++) stile[rloc * 33 + j] = __uint_as_float(v[j]);
      __syncwarp();
      const int col = col0 + cb + lane;
      const float bcol = sbias[cb + lane];
#pragma unroll 4
      for (int rr = 0; rr < 32; rr++) {
        const int64_t row = row0 + warp * 32 + rr;
        if (row < g.M && col < g.N) {
          float x = stile[(warp * 32 + rr) * 33 + lane];
          if (g.accumulate) {
            atomicAdd(&reinterpret_cast<float *>(g.C)[row * g.ldc + col], x);
            continue;
          }
          x += bcol;
          if (g.relu) x = x > 0.0f ? x : 0.0f;
          if (g.mask && !(__bfloat162float(g.mask[row * g.ldm + col]) > 0.0f)) x = 0.0f;
          if (g.out_bf16)
            reinterpret_cast<__nv_bfloat16 *>(g.C)[row * g.ldc + col] = __float2bfloat16(x);
          else
            reinterpret_cast<float *>(g.C)[row * g.ldc + col] = x;
        }
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TN) : "memory");
}

// out [C][R] = in [R][C]^T (bf16, row-major; leading dimensions ldi, ldo),
// through 32 x 32 shared-memory tiles.
__global__ void transpose_bf16_kernel(const __nv_bfloat16 *in, int64_t R, int C, int64_t ldi,
                                      __nv_bfloat16 *out, int64_t ldo) {
  __shared__ __nv_bfloat16 t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i;
    const int c = c0 + threadIdx.x;
    t[i][threadIdx.x] = (r < R && c < C) ? in[r * ldi + c] : __float2bfloat16(0.0f);
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i;
    const int64_t r = r0 + threadIdx.x;
    if (c < C && r < R) out[(int64_t)c * ldo + r] = t[threadIdx.x][i];
  }
}

}  // namespace fem_mlp_tc
