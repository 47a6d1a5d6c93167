// Grid-wide barrier for persistent kernels whose blocks are all resident
// (cooperative launches): a counter / generation pair in global memory and a
// wall-clock limit on every wait (the batched solve, batch.cu).
#pragma once
#include "fem_internal.h"

struct FemGridSync {
  unsigned count, gen;
  int error;   // FEM_ETIMEOUT once a wait ran out (every block then returns)
  int pad;
};

__device__ __forceinline__ unsigned long long fem_global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Returns false (every block) once any block has recorded an error.  Memory
// written before the barrier by any block is visible to ordinary loads after
// it: thread 0 fences (fence.sc at GPU scope) before arriving and after
// seeing the release, and the block's bar.sync orders its other threads after
// thread 0.  extra: arrivals that never come (a test hook that makes the wait
// run out); 0 in normal use.
static __device__ bool fem_grid_barrier(FemGridSync *s, unsigned extra,
                                        unsigned long long timeout_ns) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = &s->gen;
    volatile int *verr = &s->error;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&s->count, 1u);
    if (arrived == gridDim.x + extra - 1) {
      atomicExch(&s->count, 0u);
      __threadfence();
      atomicAdd(&s->gen, 1u);
    } else {
      const unsigned long long t0 = fem_global_ns();
      while (*vgen == g) {
        if (*verr) break;
        if (fem_global_ns() - t0 > timeout_ns) {
          atomicCAS(&s->error, 0, (int)FEM_ETIMEOUT);
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    s_ok = (*verr == 0);
  }
  __syncthreads();
  return s_ok != 0;
}
