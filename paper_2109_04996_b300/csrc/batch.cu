// Batched solve: many independent BP3-type problems (scalar or vector
// diffusion, Gauss-Legendre q = p+2, any order 1..8, any size) solved
// together.  Each problem runs the mixed-precision method of refine.cu (FP64
// iterative refinement around an FP32 inner Jacobi-PCG with FP64 dot products
// and scalars); the inner iterations of ALL problems run in one persistent
// cooperative kernel per outer step.  The paper batches small dense products
// across elements (section "Ecosystem", batched BLAS); here whole solves are
// batched so that small problems share the GPU instead of each paying launch
// and reduction latency.
//
// Persistent kernel, global iteration k (all active problems advance
// together; a problem leaves when its inner test is met):
//   apply phase     work items (problem, element group): y = A_32 p and the
//                   problem's p^T A p, accumulated into pAp[k&1];
//   barrier
//   update phase    work items (problem, vector chunk): alpha, d, r, z and
//                   r^T z, ||r||^2 into rz[k&1], rr[k&1];
//   barrier
//   direction phase beta = rz[k&1] / rz[(k+1)&1]; p = z + beta p; y = 0; block 0
//                   decides each problem's inner convergence;
//   barrier
// The ping-pong slots are cleared one phase after their last reader (see the
// comments at each clear).  Grid barriers are counter/generation barriers on
// global memory with a wall-clock limit: on expiry the kernel records
// FEM_ETIMEOUT and every block returns.
#include <limits.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <type_traits>
#include <vector>

#include "apply_lines.cuh"
#include "grid_sync.cuh"

using fem_apply::ApplyParams;
using fem_apply::LineTables;
using fem_apply::apply_group_lines;
using fem_apply::Slab;
using fem_apply::apply_group;
using fem_apply::apply_smem_bytes;

struct BatchProblem {
  int P, Q, ncomp;
  int64_t N, E, n;
  const int32_t *elem_nodes;
  const uint8_t *dir;
  const float *qdata32, *B32, *Dq32;
  const double *qdata64, *B64, *Dq64;
  const double *diag;
  // outer (FP64) and inner (FP32) vectors
  const double *b;
  double *x, *y64;
  float *r, *z, *p, *y, *d, *dinv;
};

struct BatchScalars {
  double pAp[2], rz[2], rr[2];
  double rr64, bb64, rz0, rr0;   // residual-kernel accumulators
  double thresh;                  // inner threshold on ||r||^2
  double rr64_last, bb64_last;    // outer residual of the latest check
  int done_at;                    // iteration at which the inner solve ended
  int iter;                       // inner iterations of this outer step
  int total_iter, outer, converged, status;
};

using BatchSync = FemGridSync;

struct fem_batch {
  int n = 0;
  std::vector<fem_op *> ops;
  cudaStream_t stream = nullptr;
  BatchProblem *d_prob = nullptr;
  BatchScalars *d_sc = nullptr;
  BatchSync *d_sync = nullptr;
  int64_t *d_gstart = nullptr;   // apply items prefix (inner shape)
  int64_t *d_gstart64 = nullptr; // apply items prefix (FP64 shape)
  int64_t *d_cstart = nullptr;   // vector chunk prefix
  // problem of every work item: one load instead of a binary search over the
  // prefixes at the head of each item's chain of dependent loads
  int *d_item_prob = nullptr;    // apply items (inner shape), reallocated by build_items
  int64_t item_prob_cap = 0;
  int *d_item64_prob = nullptr;  // FP64 apply items
  int *d_chunk_prob = nullptr;   // vector chunks
  int64_t n_items = 0, n_items64 = 0, n_chunks = 0;
  std::vector<BatchProblem> h_prob;
  std::vector<void *> allocs;
  int nt_choice = 1;             // inner kernel block size index: 128, 256, 512
  int bps = 0;                   // blocks per SM of the persistent kernel (0 = max)
  double timeout_ms = 2000.0;
  int64_t bytes = 0;
  // Split batch: problems of at least solo_dofs unknowns are solved one
  // after another by fem_solve_refined (order-specialized kernels); the rest
  // form the persistent batch `inner`.  A split batch holds no device data.
  bool split = false;
  std::vector<int> solo, rest;
  fem_batch *inner = nullptr;
  // the refinement loop as one CUDA graph (conditional WHILE node over the
  // outer steps), keyed by what its launches capture by value
  cudaStream_t cap = nullptr, cap2 = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int *d_steps = nullptr;
  int g_nt = -1, g_bps = -1, g_maxit = -1, g_max_outer = -1;
  double g_rtol = -1.0, g_inner = -1.0, g_timeout = -1.0;
  bool graph_refused = false;    // capture refused: host-driven outer loop
};

namespace {

constexpr int kChunk = 2048;     // vector entries per work item
constexpr int kNT64 = 256;       // block size of the FP64 batched apply

__device__ __forceinline__ double block_sum(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = fem_warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; w++) s += red[w];
  return s;  // valid in thread 0
}

// Two block sums with one pair of barriers (red holds 64 doubles).
__device__ __forceinline__ void block_sum2(double &v0, double &v1, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v0 = fem_warp_sum(v0);
  v1 = fem_warp_sum(v1);
  __syncthreads();
  if (lane == 0) { red[warp] = v0; red[32 + warp] = v1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < nw; w++) { s0 += red[w]; s1 += red[32 + w]; }
    v0 = s0; v1 = s1;   // valid in thread 0
  }
}

template <int NT, int Q>
struct BatchEpb {
  static constexpr int value = NT / (Q * Q) > 0 ? NT / (Q * Q) : 1;
};

// One element group of problem `pr` in precision T (FP32 inner / FP64 outer).
template <typename T, int NT, int P>
__device__ void batch_group(const BatchProblem &pr, int64_t g, const T *x, T *y,
                            unsigned char *smem, double &dot, bool reload) {
  constexpr int Q = P + 1;
  constexpr int EPB = BatchEpb<NT, Q>::value;
  ApplyParams<T> prm;
  prm.x = x; prm.y = y; prm.elem_nodes = pr.elem_nodes; prm.list = nullptr; prm.nsel = pr.E;
  prm.N = pr.N; prm.ncomp = pr.ncomp;
  if constexpr (sizeof(T) == 4) { prm.qdata = (const T *)pr.qdata32; prm.B = (const T *)pr.B32; prm.Dq = (const T *)pr.Dq32; }
  else { prm.qdata = (const T *)pr.qdata64; prm.B = (const T *)pr.B64; prm.Dq = (const T *)pr.Dq64; }
  prm.partials = nullptr; prm.counter = nullptr; prm.dot_out = nullptr;
  // x (the direction p) was written by other blocks before the last grid
  // barrier, whose fence.sc / bar.sync pair orders it before these loads
  // (the pattern of a cooperative grid sync): ordinary loads see it
  prm.x_l2_only = 0;
  Slab<T, P, Q, FEM_DIFFUSION, EPB> sl(smem);
  if (reload) {  // a new problem: its tables (the previous item may still read the old ones)
    __syncthreads();
    sl.load_tables(prm.B, prm.Dq);
    __syncthreads();
  }
  apply_group<T, P, Q, FEM_DIFFUSION, false, EPB>(prm, g, sl, dot);
}

template <typename T, int NT>
__device__ void batch_group_p(const BatchProblem &pr, int64_t g, const T *x, T *y,
                              unsigned char *smem, double &dot, bool reload) {
  switch (pr.P) {
    case 2: batch_group<T, NT, 2>(pr, g, x, y, smem, dot, reload); break;
    case 3: batch_group<T, NT, 3>(pr, g, x, y, smem, dot, reload); break;
    case 4: batch_group<T, NT, 4>(pr, g, x, y, smem, dot, reload); break;
    case 5: batch_group<T, NT, 5>(pr, g, x, y, smem, dot, reload); break;
    case 6: batch_group<T, NT, 6>(pr, g, x, y, smem, dot, reload); break;
    case 7: batch_group<T, NT, 7>(pr, g, x, y, smem, dot, reload); break;
    case 8: batch_group<T, NT, 8>(pr, g, x, y, smem, dot, reload); break;
    case 9: batch_group<T, NT, 9>(pr, g, x, y, smem, dot, reload); break;
  }
}

// FP32 inner apply with the line-based even-odd body.  The split tables of
// a BP3-type problem depend on its order alone (Gauss-Legendre, q = p+2), so
// one set per order lives in constant memory and is read like the kernel
// parameters of the single-operator kernel: operands of the FMAs, not values
// held in registers.  fem_batch_create writes the slots of the orders it
// holds (the same values for every batch, so concurrent batches agree).
struct BatchLineTables {
  LineTables<float, 2, 3> t2;
  LineTables<float, 3, 4> t3;
  LineTables<float, 4, 5> t4;
  LineTables<float, 5, 6> t5;
  LineTables<float, 6, 7> t6;
  LineTables<float, 7, 8> t7;
  LineTables<float, 8, 9> t8;
  LineTables<float, 9, 10> t9;
};
__constant__ BatchLineTables c_ltab;

template <int P>
__device__ __forceinline__ const LineTables<float, P, P + 1> &batch_ltab() {
  if constexpr (P == 2) return c_ltab.t2;
  else if constexpr (P == 3) return c_ltab.t3;
  else if constexpr (P == 4) return c_ltab.t4;
  else if constexpr (P == 5) return c_ltab.t5;
  else if constexpr (P == 6) return c_ltab.t6;
  else if constexpr (P == 7) return c_ltab.t7;
  else if constexpr (P == 8) return c_ltab.t8;
  else return c_ltab.t9;
}

template <int NT, int P>
__device__ void batch_group_lines(const BatchProblem &pr, int64_t g, unsigned char *smem,
                                  double &dot) {
  constexpr int Q = P + 1;
  constexpr int EPB = BatchEpb<NT, Q>::value;
  float *cubes = reinterpret_cast<float *>(smem);
  ApplyParams<float> prm;
  prm.x = pr.p; prm.y = pr.y; prm.elem_nodes = pr.elem_nodes; prm.list = nullptr; prm.nsel = pr.E;
  prm.N = pr.N; prm.ncomp = pr.ncomp;
  prm.qdata = pr.qdata32; prm.B = pr.B32; prm.Dq = pr.Dq32;
  prm.partials = nullptr; prm.counter = nullptr; prm.dot_out = nullptr;
  prm.x_l2_only = 0;  // written before the last grid barrier (see fem_grid_barrier)
  prm.want_dot = 1;   // p^T A p of the problem
  apply_group_lines<float, P, Q, false, EPB, false, false>(prm, batch_ltab<P>(), g, cubes, dot);
}

template <int NT>
__device__ void batch_group_lines_p(const BatchProblem &pr, int64_t g, unsigned char *smem,
                                    double &dot) {
  switch (pr.P) {
    case 2: batch_group_lines<NT, 2>(pr, g, smem, dot); break;
    case 3: batch_group_lines<NT, 3>(pr, g, smem, dot); break;
    case 4: batch_group_lines<NT, 4>(pr, g, smem, dot); break;
    case 5: batch_group_lines<NT, 5>(pr, g, smem, dot); break;
    case 6: batch_group_lines<NT, 6>(pr, g, smem, dot); break;
    case 7: batch_group_lines<NT, 7>(pr, g, smem, dot); break;
    case 8: batch_group_lines<NT, 8>(pr, g, smem, dot); break;
    case 9: batch_group_lines<NT, 9>(pr, g, smem, dot); break;
  }
}

template <int NT>
constexpr size_t batch_lines_smem() {
  size_t m = 0;
#define FEM_BL(P) { size_t s = fem_apply::lines_smem_bytes<float, P + 1, BatchEpb<NT, P + 1>::value, false>(); if (s > m) m = s; }
  FEM_BL(2) FEM_BL(3) FEM_BL(4) FEM_BL(5) FEM_BL(6) FEM_BL(7) FEM_BL(8) FEM_BL(9)
#undef FEM_BL
  return m;
}

template <typename T, int NT>
constexpr size_t batch_smem() {
  size_t m = 0;
#define FEM_BS(P) { size_t s = apply_smem_bytes<T, P + 1, P, FEM_DIFFUSION, BatchEpb<NT, P + 1>::value>(); if (s > m) m = s; }
  FEM_BS(2) FEM_BS(3) FEM_BS(4) FEM_BS(5) FEM_BS(6) FEM_BS(7) FEM_BS(8) FEM_BS(9)
#undef FEM_BS
  return m;
}

struct BatchArgs {
  BatchProblem *prob;
  BatchScalars *sc;
  BatchSync *sync;
  const int64_t *gstart;   // [n+1] apply items
  const int64_t *cstart;   // [n+1] vector chunks
  const int *item_prob;    // [n_items] problem of each apply item
  const int *item64_prob;  // [n_items64] problem of each FP64 apply item
  const int *chunk_prob;   // [n_chunks] problem of each vector chunk
  int n;
  int maxit;
  unsigned barrier_extra;
  unsigned long long timeout_ns;
};

// ---- the persistent inner FP32 PCG over all problems
template <int NT>
__global__ void __launch_bounds__(NT) batch_inner_kernel(const BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[64];
  // problem i is inactive in iteration k once its done_at < k; done_at only
  // changes in the direction phase (block 0), so the flags read at the top
  // of an iteration hold for all its phases
  __shared__ unsigned char s_inactive[1024];
  __shared__ int s_active;
  const int64_t n_items = a.gstart[a.n], n_chunks = a.cstart[a.n];
  for (int k = 0; k < a.maxit; k++) {
    const int cur = k & 1, prev = cur ^ 1;
    if (threadIdx.x == 0) s_active = 0;
    __syncthreads();
    {
      int mine = 0;
      for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        const bool off = __ldcg(&a.sc[i].done_at) < k;
        s_inactive[i] = off ? 1 : 0;
        mine += off ? 0 : 1;
      }
      if (mine) atomicAdd(&s_active, mine);
    }
    __syncthreads();
    if (s_active == 0) return;   // every problem done (uniform across blocks)
    // -------- apply phase
    if (blockIdx.x == 0) {
      // rz[cur], rr[cur] were last read in the direction phase of k-1
      for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        a.sc[i].rz[cur] = 0.0;
        a.sc[i].rr[cur] = 0.0;
      }
    }
    // a block's items of one problem are consecutive in its stride: p^T A p
    // is flushed once per problem, not per item
    int cur_prob = -1;
    double dot = 0.0;
    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
      const int i = a.item_prob[it];
      if (s_inactive[i]) continue;   // uniform per block
      if (i != cur_prob) {
        if (cur_prob >= 0) {
          const double s = block_sum(dot, red);
          if (threadIdx.x == 0) atomicAdd(&a.sc[cur_prob].pAp[cur], s);
        }
        dot = 0.0;
      }
      const BatchProblem &pr = a.prob[i];
      batch_group_lines_p<NT>(pr, it - a.gstart[i], smem, dot);
      cur_prob = i;
    }
    if (cur_prob >= 0) {
      const double s = block_sum(dot, red);
      if (threadIdx.x == 0) atomicAdd(&a.sc[cur_prob].pAp[cur], s);
    }
    if (!fem_grid_barrier(a.sync, a.barrier_extra, a.timeout_ns)) return;
    // -------- update phase
    for (int64_t it = blockIdx.x; it < n_chunks; it += gridDim.x) {
      const int i = a.chunk_prob[it];
      if (s_inactive[i]) continue;
      const BatchProblem &pr = a.prob[i];
      const double pAp = __ldcg(&a.sc[i].pAp[cur]);
      const double alpha = __ldcg(&a.sc[i].rz[prev]) / pAp;
      if (!(pAp > 0.0) || !isfinite(alpha)) continue;
      const float af = (float)alpha;
      const int64_t lo = (it - a.cstart[i]) * kChunk;
      const int64_t hi = lo + kChunk < pr.n ? lo + kChunk : pr.n;
      double v0 = 0.0, v1 = 0.0;
      for (int64_t j = lo + threadIdx.x; j < hi; j += NT) {
        const bool fixed = pr.dir && pr.dir[fem_node_of(j, pr.N)];
        float r = pr.r[j];
        pr.d[j] += af * pr.p[j];
        if (!fixed) r -= af * pr.y[j];  // atomics of other blocks, before the barrier
        pr.r[j] = r;
        const float z = pr.dinv[j] * r;
        pr.z[j] = z;
        v0 += (double)r * (double)z;
        v1 += (double)r * (double)r;
      }
      block_sum2(v0, v1, red);
      if (threadIdx.x == 0) {
        atomicAdd(&a.sc[i].rz[cur], v0);
        atomicAdd(&a.sc[i].rr[cur], v1);
      }
    }
    if (!fem_grid_barrier(a.sync, a.barrier_extra, a.timeout_ns)) return;
    // -------- direction phase
    if (blockIdx.x == 0) for (int ii = threadIdx.x; ii < a.n; ii += blockDim.x) {
      BatchScalars &s = a.sc[ii];
      if (!(s.done_at < k)) {
        // pAp[prev] was last read in the update phase of k-1
        s.pAp[prev] = 0.0;
        const double pAp = __ldcg(&s.pAp[cur]);
        const bool ok = (pAp > 0.0) && isfinite(__ldcg(&s.rz[prev]) / pAp);
        if (ok) { s.iter += 1; s.total_iter += 1; }
        const double rzc = __ldcg(&s.rz[cur]), rrc = __ldcg(&s.rr[cur]);
        if (!ok || !isfinite(rzc) || rrc <= s.thresh || s.iter >= a.maxit) s.done_at = k;
      }
    }
    for (int64_t it = blockIdx.x; it < n_chunks; it += gridDim.x) {
      const int i = a.chunk_prob[it];
      if (s_inactive[i]) continue;
      const BatchProblem &pr = a.prob[i];
      const float beta = (float)(__ldcg(&a.sc[i].rz[cur]) / __ldcg(&a.sc[i].rz[prev]));
      const int64_t lo = (it - a.cstart[i]) * kChunk;
      const int64_t hi = lo + kChunk < pr.n ? lo + kChunk : pr.n;
      for (int64_t j = lo + threadIdx.x; j < hi; j += NT) {
        pr.p[j] = pr.z[j] + beta * pr.p[j];
        pr.y[j] = 0.0f;
      }
    }
    if (!fem_grid_barrier(a.sync, a.barrier_extra, a.timeout_ns)) return;
  }
}

// ---- FP64 batched apply y64 = A_64 x for every problem not yet converged
__global__ void __launch_bounds__(kNT64) batch_apply64_kernel(const BatchArgs a, const int64_t *gstart64) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t n_items = gstart64[a.n];
  int cur_prob = -1;
  for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int i = a.item64_prob[it];
    if (a.sc[i].converged) continue;
    const BatchProblem &pr = a.prob[i];
    double dot = 0.0;
    batch_group_p<double, kNT64>(pr, it - gstart64[i], pr.x, pr.y64, smem, dot, i != cur_prob);
    cur_prob = i;
  }
}

// r64 = M (b - A x); inner start d = 0, r = r64, z = dinv r, p = z
__global__ void batch_residual_kernel(const BatchArgs a) {
  __shared__ double red[32];
  const int64_t n_chunks = a.cstart[a.n];
  for (int64_t it = blockIdx.x; it < n_chunks; it += gridDim.x) {
    const int i = a.chunk_prob[it];
    if (a.sc[i].converged) continue;
    const BatchProblem &pr = a.prob[i];
    const int64_t lo = (it - a.cstart[i]) * kChunk;
    const int64_t hi = lo + kChunk < pr.n ? lo + kChunk : pr.n;
    double v[4] = {0, 0, 0, 0};
    for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
      const bool fixed = pr.dir && pr.dir[fem_node_of(j, pr.N)];
      const double bj = fixed ? 0.0 : pr.b[j];
      const double r64 = fixed ? 0.0 : bj - pr.y64[j];
      const float r = (float)r64, z = pr.dinv[j] * r;
      pr.p[j] += z - pr.z[j];  // reliable update: swap the residual part of p
      pr.r[j] = r; pr.z[j] = z; pr.d[j] = 0.0f; pr.y[j] = 0.0f;
      pr.y64[j] = 0.0;
      v[0] += r64 * r64; v[1] += bj * bj; v[2] += (double)r * z; v[3] += (double)r * r;
    }
    for (int q = 0; q < 4; q++) {
      const double s = block_sum(v[q], red);
      if (threadIdx.x == 0) {
        double *dst = q == 0 ? &a.sc[i].rr64 : q == 1 ? &a.sc[i].bb64 : q == 2 ? &a.sc[i].rz0 : &a.sc[i].rr0;
        atomicAdd(dst, s);
      }
    }
  }
}

// Outer test and inner start state, one thread per problem.
__global__ void batch_finalize_kernel(const BatchArgs a, double rtol2, double inner_rtol2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  BatchScalars &s = a.sc[i];
  if (!s.converged) {
    s.rr64_last = s.rr64; s.bb64_last = s.bb64;
    if (!isfinite(s.rr64) || !isfinite(s.rz0)) { s.status = FEM_EBREAKDOWN; s.converged = 1; }
    else if (!(s.bb64 > 0.0) || s.rr64 <= rtol2 * s.bb64) s.converged = 1;
  }
  s.pAp[0] = s.pAp[1] = 0.0;
  s.rz[0] = 0.0; s.rz[1] = s.rz0;   // iteration 0 reads rz[1]
  s.rr[0] = s.rr[1] = 0.0;
  s.thresh = inner_rtol2 * s.rr0;
  s.iter = 0;
  s.done_at = s.converged ? -1 : INT_MAX;
}

// x += d for problems still refining; clear the residual accumulators.
__global__ void batch_correct_kernel(const BatchArgs a) {
  const int64_t n_chunks = a.cstart[a.n];
  for (int64_t it = blockIdx.x; it < n_chunks; it += gridDim.x) {
    const int i = a.chunk_prob[it];
    if (a.sc[i].converged) continue;
    const BatchProblem &pr = a.prob[i];
    const int64_t lo = (it - a.cstart[i]) * kChunk;
    const int64_t hi = lo + kChunk < pr.n ? lo + kChunk : pr.n;
    for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) pr.x[j] += (double)pr.d[j];
  }
}

__global__ void batch_step_end_kernel(const BatchArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  BatchScalars &s = a.sc[i];
  if (!s.converged) s.outer += 1;
  s.rr64 = s.bb64 = s.rz0 = s.rr0 = 0.0;
}

__global__ void batch_prepare_kernel(const BatchArgs a) {
  const int64_t n_chunks = a.cstart[a.n];
  for (int64_t it = blockIdx.x; it < n_chunks; it += gridDim.x) {
    const int i = a.chunk_prob[it];
    const BatchProblem &pr = a.prob[i];
    const int64_t lo = (it - a.cstart[i]) * kChunk;
    const int64_t hi = lo + kChunk < pr.n ? lo + kChunk : pr.n;
    for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
      const int64_t node = fem_node_of(j, pr.N);
      if (pr.dir && pr.dir[node]) pr.x[j] = 0.0;
      pr.y64[j] = 0.0;
      pr.p[j] = 0.0f;
      pr.z[j] = 0.0f;
      pr.dinv[j] = (pr.dir && pr.dir[node]) ? 0.0f : (float)(1.0 / pr.diag[node]);
    }
  }
}

const int kNtChoices[3] = {128, 256, 512};

template <int NT>
int launch_inner_nt(fem_batch *b, const BatchArgs &a, int bps) {
  auto kern = batch_inner_kernel<NT>;
  constexpr size_t smem = batch_lines_smem<NT>();
  FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
  if (per_sm < 1) { fem_set_error("batch: inner kernel does not fit on an SM"); return FEM_ECUDA; }
  const int use = (bps <= 0 || bps > per_sm) ? per_sm : bps;
  int nsm = b->ops[0]->nsm;
  dim3 grid((unsigned)(nsm * use)), block(NT);
  void *args[] = {(void *)&a};
  FEM_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)kern, grid, block, args, smem, b->stream));
  return FEM_OK;
}

int launch_inner(fem_batch *b, const BatchArgs &a, int nt_choice, int bps) {
  switch (nt_choice) {
    case 0: return launch_inner_nt<128>(b, a, bps);
    case 2: return launch_inner_nt<512>(b, a, bps);
    default: return launch_inner_nt<256>(b, a, bps);
  }
}

int64_t groups_for(const BatchProblem &p, int nt) {
  const int Q = p.Q;
  int epb = nt / (Q * Q);
  if (epb < 1) epb = 1;
  return (p.E + epb - 1) / epb;
}

// Problem of each of the n_items work items of a prefix table.
std::vector<int> item_problems(const std::vector<int64_t> &start, int n) {
  std::vector<int> m((size_t)start[n]);
  for (int i = 0; i < n; i++)
    for (int64_t it = start[i]; it < start[i + 1]; it++) m[(size_t)it] = i;
  return m;
}

int build_items(fem_batch *b, int nt) {
  std::vector<int64_t> gs(b->n + 1, 0);
  for (int i = 0; i < b->n; i++) gs[i + 1] = gs[i] + groups_for(b->h_prob[i], nt);
  b->n_items = gs[b->n];
  const std::vector<int> ip = item_problems(gs, b->n);
  if (b->item_prob_cap < b->n_items) {
    cudaFree(b->d_item_prob);
    b->d_item_prob = nullptr;
    b->item_prob_cap = 0;
    if (cudaMalloc(&b->d_item_prob, sizeof(int) * (size_t)b->n_items) != cudaSuccess) {
      cudaGetLastError();
      fem_set_error("batch: allocation of the work-item table failed");
      return FEM_ENOMEM;
    }
    b->item_prob_cap = b->n_items;
  }
  FEM_CUDA_TRY(cudaMemcpyAsync(b->d_gstart, gs.data(), sizeof(int64_t) * (b->n + 1),
                               cudaMemcpyHostToDevice, b->stream));
  FEM_CUDA_TRY(cudaMemcpyAsync(b->d_item_prob, ip.data(), sizeof(int) * ip.size(),
                               cudaMemcpyHostToDevice, b->stream));
  FEM_CUDA_TRY(cudaStreamSynchronize(b->stream));
  return FEM_OK;
}

BatchArgs args_of(fem_batch *b, int maxit, unsigned extra) {
  BatchArgs a;
  a.prob = b->d_prob; a.sc = b->d_sc; a.sync = b->d_sync; a.gstart = b->d_gstart;
  a.cstart = b->d_cstart; a.n = b->n; a.maxit = maxit; a.barrier_extra = extra;
  a.item_prob = b->d_item_prob; a.item64_prob = b->d_item64_prob; a.chunk_prob = b->d_chunk_prob;
  a.timeout_ns = (unsigned long long)(b->timeout_ms * 1e6);
  return a;
}

int read_error(fem_batch *b) {
  BatchSync s;
  FEM_CUDA_TRY(cudaMemcpyAsync(&s, b->d_sync, sizeof(s), cudaMemcpyDeviceToHost, b->stream));
  FEM_CUDA_TRY(cudaStreamSynchronize(b->stream));
  if (s.error) {
    BatchSync z = {0, 0, 0, 0};
    FEM_CUDA_TRY(cudaMemcpyAsync(b->d_sync, &z, sizeof(z), cudaMemcpyHostToDevice, b->stream));
    FEM_CUDA_TRY(cudaStreamSynchronize(b->stream));
    fem_set_error("batch: a grid barrier of the persistent kernel timed out");
    return FEM_ETIMEOUT;
  }
  return FEM_OK;
}

// Outer test of the graph-driven loop: stop once every problem converged,
// after max_outer + 1 steps (as the host loop), or when a barrier ran out.
__global__ void batch_decide_kernel(const BatchArgs a, int *steps, int max_outer,
                                    cudaGraphConditionalHandle h) {
  __shared__ int s_open;
  if (threadIdx.x == 0) s_open = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < a.n; i += blockDim.x)
    if (!a.sc[i].converged) atomicOr(&s_open, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int st = *steps + 1;
    *steps = st;
    const bool stop = !s_open || st > max_outer || ((volatile BatchSync *)a.sync)->error;
    cudaGraphSetConditional(h, stop ? 0u : 1u);
  }
}

__global__ void batch_zero_steps_kernel(int *steps) { *steps = 0; }

void destroy_solve_graph(fem_batch *b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
}

// One outer refinement step (all problems) on stream s.
int launch_outer_step(fem_batch *b, const BatchArgs &a, const fem_cg_opts *o, cudaStream_t s) {
  const int g = b->ops[0]->nsm * 8;
  batch_apply64_kernel<<<b->ops[0]->nsm * 4, kNT64, batch_smem<double, kNT64>(), s>>>(a, b->d_gstart64);
  FEM_CHECK_LAUNCH();
  batch_residual_kernel<<<g, 256, 0, s>>>(a);
  FEM_CHECK_LAUNCH();
  batch_finalize_kernel<<<(b->n + 127) / 128, 128, 0, s>>>(a, o->rtol * o->rtol,
                                                          o->inner_rtol * o->inner_rtol);
  FEM_CHECK_LAUNCH();
  cudaStream_t saved = b->stream;
  b->stream = s;   // the persistent kernel's launcher uses the batch stream
  int rc = launch_inner(b, a, b->nt_choice, b->bps);
  b->stream = saved;
  if (rc) return rc;
  batch_correct_kernel<<<g, 256, 0, s>>>(a);
  FEM_CHECK_LAUNCH();
  batch_step_end_kernel<<<(b->n + 127) / 128, 128, 0, s>>>(a);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

// Capture the refinement loop: steps = 0; WHILE (open) { outer step; decide }.
// Returns FEM_ECUDA (error cleared) if the runtime refuses the capture, e.g.
// of the cooperative launch inside the conditional body.
int build_solve_graph(fem_batch *b, const fem_cg_opts *o) {
  destroy_solve_graph(b);
  if (!b->cap) {
    FEM_CUDA_TRY(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    FEM_CUDA_TRY(cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking));
  }
  BatchArgs a = args_of(b, o->maxit, 0);
  cudaGraph_t graph = nullptr;
  int rc = FEM_OK;
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) { cudaGetLastError(); return FEM_ECUDA; }
  do {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaGraphConditionalHandle h = 0;
    e = cudaStreamGetCaptureInfo(b->cap, &st, nullptr, &graph, nullptr, nullptr, nullptr);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
    batch_zero_steps_kernel<<<1, 1, 0, b->cap>>>(b->d_steps);
    e = cudaStreamGetCaptureInfo(b->cap, &st, nullptr, &graph, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    if ((e = cudaGraphAddNode(&cnode, graph, deps, nullptr, ndeps, &cp)) != cudaSuccess) { rc = FEM_ECUDA; break; }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamUpdateCaptureDependencies(b->cap, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
    e = cudaStreamBeginCaptureToGraph(b->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
    rc = launch_outer_step(b, a, o, b->cap2);
    if (!rc) {
      batch_decide_kernel<<<1, 256, 0, b->cap2>>>(a, b->d_steps, o->max_outer, h);
      if (cudaPeekAtLastError() != cudaSuccess) rc = FEM_ECUDA;
    }
    cudaGraph_t tmp;
    cudaError_t e2 = cudaStreamEndCapture(b->cap2, &tmp);
    if (!rc && e2 != cudaSuccess) rc = FEM_ECUDA;
  } while (0);
  cudaGraph_t g2 = nullptr;
  cudaError_t e3 = cudaStreamEndCapture(b->cap, &g2);
  if (!rc && e3 != cudaSuccess) rc = FEM_ECUDA;
  if (!rc && cudaGraphInstantiate(&b->gexec, g2, 0) != cudaSuccess) { b->gexec = nullptr; rc = FEM_ECUDA; }
  if (g2) cudaGraphDestroy(g2);
  if (rc) { cudaGetLastError(); return rc; }
  b->g_nt = b->nt_choice; b->g_bps = b->bps; b->g_maxit = o->maxit; b->g_max_outer = o->max_outer;
  b->g_rtol = o->rtol; b->g_inner = o->inner_rtol; b->g_timeout = b->timeout_ms;
  return FEM_OK;
}

constexpr int kGraphRefused = -1;

// The refinement loop as one graph launch; the host synchronizes once.
int run_solve_graph(fem_batch *b, const fem_cg_opts *o, int *steps_out) {
  const bool stale = !b->gexec || b->g_nt != b->nt_choice || b->g_bps != b->bps ||
                     b->g_maxit != o->maxit || b->g_max_outer != o->max_outer ||
                     b->g_rtol != o->rtol || b->g_inner != o->inner_rtol ||
                     b->g_timeout != b->timeout_ms;
  if (stale) {
    FEM_CUDA_TRY(cudaStreamSynchronize(b->stream));   // the capture streams must see prior work
    if (build_solve_graph(b, o)) {
      b->graph_refused = true;   // the host-driven loop from now on
      return kGraphRefused;
    }
  }
  FEM_CUDA_TRY(cudaGraphLaunch(b->gexec, b->stream));
  int rc = read_error(b);   // synchronizes
  if (rc) return rc;
  int steps = 0;
  FEM_CUDA_TRY(cudaMemcpyAsync(&steps, b->d_steps, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  FEM_CUDA_TRY(cudaStreamSynchronize(b->stream));
  *steps_out = steps;
  return FEM_OK;
}

// Runs outer refinement steps until every problem converges (or max_outer
// + 1 steps), one host-launched step at a time.
int run_solve(fem_batch *b, const fem_cg_opts *o, int *steps_out) {
  BatchArgs a = args_of(b, o->maxit, 0);
  std::vector<BatchScalars> h(b->n);
  int steps = 0;
  for (;;) {
    int rc = launch_outer_step(b, a, o, b->stream);
    if (rc) return rc;
    rc = read_error(b);
    if (rc) return rc;
    FEM_CUDA_TRY(cudaMemcpyAsync(h.data(), b->d_sc, sizeof(BatchScalars) * b->n,
                                 cudaMemcpyDeviceToHost, b->stream));
    FEM_CUDA_TRY(cudaStreamSynchronize(b->stream));
    steps++;
    bool all = true;
    for (int i = 0; i < b->n; i++) all = all && h[i].converged;
    if (all || steps > o->max_outer) break;
  }
  *steps_out = steps;
  return FEM_OK;
}

}  // namespace

static int validate_ops(fem_op *const *ops, int n) {
  if (!ops || n < 1 || n > 1024) { fem_set_error("fem_batch_create: need 1..1024 operators"); return FEM_EINVAL; }
  for (int i = 0; i < n; i++) {
    const fem_op *op = ops[i];
    if (!op || op->kind != FEM_DIFFUSION || op->quad != FEM_GAUSS || op->Q != op->P + 1 ||
        !op->d_qdata32) {
      fem_set_error("fem_batch_create: operator %d must be a FEM_F32 diffusion operator with "
                    "Gauss q = p+2", i);
      return FEM_EINVAL;
    }
    if (op->stream() != ops[0]->stream()) {
      fem_set_error("fem_batch_create: all operators must share one stream");
      return FEM_EINVAL;
    }
  }
  return FEM_OK;
}

// The persistent batch over all of ops (validated).
static int create_persistent(fem_op *const *ops, int n, fem_batch **out) {
  fem_batch *b = new fem_batch();
  b->n = n;
  b->ops.assign(ops, ops + n);
  b->stream = ops[0]->stream();
  auto dalloc = [&](void **p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); return false; }
    b->allocs.push_back(*p);
    b->bytes += (int64_t)bytes;
    return true;
  };
  bool ok = dalloc((void **)&b->d_prob, sizeof(BatchProblem) * n) &&
            dalloc((void **)&b->d_sc, sizeof(BatchScalars) * n) &&
            dalloc((void **)&b->d_sync, sizeof(BatchSync)) &&
            dalloc((void **)&b->d_gstart, sizeof(int64_t) * (n + 1)) &&
            dalloc((void **)&b->d_gstart64, sizeof(int64_t) * (n + 1)) &&
            dalloc((void **)&b->d_cstart, sizeof(int64_t) * (n + 1)) &&
            dalloc((void **)&b->d_steps, sizeof(int));
  b->h_prob.resize(n);
  std::vector<int64_t> cs(n + 1, 0), g64(n + 1, 0);
  BatchLineTables htab;   // host image of the constant tables (uploaded per slot)
  bool have_tab[FEM_MAX_P + 1] = {};
  for (int i = 0; ok && i < n; i++) {
    // the batch's FP64 residual kernel reads the FP64 qdata
    if (fem_ensure_qdata64(ops[i]) != FEM_OK) { ok = false; break; }
    const fem_op *op = ops[i];
    BatchProblem &p = b->h_prob[i];
    p.P = op->P; p.Q = op->Q; p.ncomp = op->ncomp; p.N = op->N; p.E = op->E;
    p.n = op->N * op->ncomp;
    p.elem_nodes = op->mesh->d_elem_nodes; p.dir = op->mesh->d_dirichlet;
    p.qdata32 = op->d_qdata32; p.B32 = op->d_B32; p.Dq32 = op->d_Dq32;
    p.qdata64 = op->d_qdata; p.B64 = op->d_B; p.Dq64 = op->d_Dq;
    p.diag = op->d_diag;
    p.b = nullptr; p.x = nullptr;
    if (!have_tab[op->P]) {
      // split tables of the line-based body, built on the host from FP64
      have_tab[op->P] = true;
      double Bt[FEM_MAX_P * FEM_MAX_Q], Dt[FEM_MAX_Q * FEM_MAX_Q];
      const int P_ = op->P, Q_ = op->Q;
      for (int k = 0; k < Q_; k++)
        for (int a2 = 0; a2 < P_; a2++) Bt[a2 * Q_ + k] = op->tab.B[k * P_ + a2];
      for (int k = 0; k < Q_; k++)
        for (int m2 = 0; m2 < Q_; m2++) Dt[m2 * Q_ + k] = op->tab.Dq[k * Q_ + m2];
      auto fill = [&](auto &lt) {
        using LT = typename std::remove_reference<decltype(lt)>::type;
        constexpr int PP_ = LT::kP, QQ_ = LT::kQ;
        fem_apply::make_symtab<float, PP_, QQ_>(op->tab.B, lt.Bf);
        fem_apply::make_symtab<float, QQ_, PP_>(Bt, lt.Bt);
        fem_apply::make_symtab<float, QQ_, QQ_>(op->tab.Dq, lt.Df);
        fem_apply::make_symtab<float, QQ_, QQ_>(Dt, lt.Dt);
        const size_t off = (size_t)((const unsigned char *)&lt - (const unsigned char *)&htab);
        if (ok && cudaMemcpyToSymbolAsync(c_ltab, &lt, sizeof(LT), off, cudaMemcpyHostToDevice,
                                          b->stream) != cudaSuccess) {
          cudaGetLastError();
          ok = false;
        }
      };
      switch (P_) {
        case 2: fill(htab.t2); break;
        case 3: fill(htab.t3); break;
        case 4: fill(htab.t4); break;
        case 5: fill(htab.t5); break;
        case 6: fill(htab.t6); break;
        case 7: fill(htab.t7); break;
        case 8: fill(htab.t8); break;
        case 9: fill(htab.t9); break;
      }
    }
    const size_t nn = (size_t)p.n;
    ok = ok && dalloc((void **)&p.y64, 8 * nn) && dalloc((void **)&p.r, 4 * nn) &&
         dalloc((void **)&p.z, 4 * nn) && dalloc((void **)&p.p, 4 * nn) &&
         dalloc((void **)&p.y, 4 * nn) && dalloc((void **)&p.d, 4 * nn) &&
         dalloc((void **)&p.dinv, 4 * nn);
    cs[i + 1] = cs[i] + (p.n + kChunk - 1) / kChunk;
    g64[i + 1] = g64[i] + groups_for(p, kNT64);
  }
  if (!ok) {
    fem_set_error("fem_batch_create: device allocation failed");
    fem_batch_destroy(b);
    return FEM_ENOMEM;
  }
  b->n_chunks = cs[n];
  b->n_items64 = g64[n];
  const std::vector<int> chunk_prob = item_problems(cs, n), item64_prob = item_problems(g64, n);
  if (!dalloc((void **)&b->d_chunk_prob, sizeof(int) * chunk_prob.size()) ||
      !dalloc((void **)&b->d_item64_prob, sizeof(int) * item64_prob.size())) {
    fem_set_error("fem_batch_create: device allocation failed");
    fem_batch_destroy(b);
    return FEM_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(b->d_cstart, cs.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_gstart64, g64.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_chunk_prob, chunk_prob.data(), sizeof(int) * chunk_prob.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_item64_prob, item64_prob.data(), sizeof(int) * item64_prob.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_sync, 0, sizeof(BatchSync), b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    fem_set_error("fem_batch_create: upload failed: %s", cudaGetErrorString(e));
    fem_batch_destroy(b);
    return FEM_ECUDA;
  }
  auto kern64 = batch_apply64_kernel;
  if (cudaFuncSetAttribute(kern64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)batch_smem<double, kNT64>()) != cudaSuccess) {
    fem_set_error("fem_batch_create: kernel attribute failed");
    fem_batch_destroy(b);
    return FEM_ECUDA;
  }
  int rc = build_items(b, kNtChoices[b->nt_choice]);
  if (rc) { fem_batch_destroy(b); return rc; }
  *out = b;
  return FEM_OK;
}

extern "C" fem_status fem_batch_create_split(fem_op *const *ops, int n, int64_t solo_dofs,
                                             fem_batch **out) {
  if (!out) { fem_set_error("fem_batch_create: out is NULL"); return FEM_EINVAL; }
  *out = nullptr;
  int rc = validate_ops(ops, n);
  if (rc) return rc;
  std::vector<int> solo, rest;
  for (int i = 0; i < n; i++) {
    if (solo_dofs > 0 && ops[i]->N * ops[i]->ncomp >= solo_dofs) solo.push_back(i);
    else rest.push_back(i);
  }
  if (solo.empty()) return create_persistent(ops, n, out);
  fem_batch *b = new fem_batch();
  b->n = n;
  b->ops.assign(ops, ops + n);
  b->stream = ops[0]->stream();
  b->split = true;
  b->solo = solo;
  b->rest = rest;
  if (!rest.empty()) {
    std::vector<fem_op *> sub;
    for (int i : rest) sub.push_back(ops[i]);
    if ((rc = create_persistent(sub.data(), (int)sub.size(), &b->inner))) { delete b; return rc; }
  }
  *out = b;
  return FEM_OK;
}

extern "C" fem_status fem_batch_create(fem_op *const *ops, int n, fem_batch **out) {
  return fem_batch_create_split(ops, n, FEM_BATCH_SOLO_DOFS, out);
}

extern "C" fem_status fem_batch_destroy(fem_batch *b) {
  if (!b) return FEM_OK;
  if (b->inner) fem_batch_destroy(b->inner);
  destroy_solve_graph(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->cap2) cudaStreamDestroy(b->cap2);
  cudaFree(b->d_item_prob);
  for (void *p : b->allocs) cudaFree(p);
  delete b;
  return FEM_OK;
}

extern "C" fem_status fem_batch_set_shape(fem_batch *b, int nt_choice, int blocks_per_sm,
                                          double timeout_ms) {
  if (!b || nt_choice < 0 || nt_choice > 2 || blocks_per_sm < 0 || !(timeout_ms > 0)) {
    fem_set_error("fem_batch_set_shape: invalid arguments");
    return FEM_EINVAL;
  }
  if (b->split) return b->inner ? fem_batch_set_shape(b->inner, nt_choice, blocks_per_sm, timeout_ms) : FEM_OK;
  b->nt_choice = nt_choice;
  b->bps = blocks_per_sm;
  b->timeout_ms = timeout_ms;
  return build_items(b, kNtChoices[nt_choice]);
}

static int bind_vectors(fem_batch *b, const double *const *bv, double *const *xv) {
  for (int i = 0; i < b->n; i++) {
    if (!bv[i] || !xv[i] || bv[i] == xv[i]) {
      fem_set_error("fem_batch_solve: invalid vectors for problem %d", i);
      return FEM_EINVAL;
    }
    b->h_prob[i].b = bv[i];
    b->h_prob[i].x = xv[i];
  }
  FEM_CUDA_TRY(cudaMemcpyAsync(b->d_prob, b->h_prob.data(), sizeof(BatchProblem) * b->n,
                               cudaMemcpyHostToDevice, b->stream));
  return FEM_OK;
}

// Split batch: the large problems one after another with their own
// refined solves, then the persistent batch of the rest.
static int solve_split(fem_batch *b, const double *const *bv, double *const *xv,
                       const fem_cg_opts *o, fem_cg_stats *stats) {
  for (int i = 0; i < b->n; i++) {
    if (!bv[i] || !xv[i] || bv[i] == xv[i]) {
      fem_set_error("fem_batch_solve: invalid vectors for problem %d", i);
      return FEM_EINVAL;
    }
  }
  int status = FEM_OK;
  for (int i : b->solo) {
    fem_cg_stats st = {};
    const int rc = fem_solve_refined(b->ops[i], bv[i], xv[i], o, &st);
    if (rc != FEM_OK && rc != FEM_ENOCONV && rc != FEM_EBREAKDOWN) return rc;
    if (stats) stats[i] = st;
    if (st.status != FEM_OK && status == FEM_OK) status = st.status;
  }
  if (b->inner) {
    std::vector<const double *> sb;
    std::vector<double *> sx;
    std::vector<fem_cg_stats> ss(b->rest.size());
    for (int i : b->rest) { sb.push_back(bv[i]); sx.push_back(xv[i]); }
    const int rc = fem_batch_solve(b->inner, sb.data(), sx.data(), o, ss.data());
    if (rc != FEM_OK && rc != FEM_ENOCONV && rc != FEM_EBREAKDOWN) return rc;
    for (size_t k = 0; k < b->rest.size(); k++) {
      if (stats) stats[b->rest[k]] = ss[k];
      if (ss[k].status != FEM_OK && status == FEM_OK) status = ss[k].status;
    }
  }
  return status;
}

static int reset_scalars(fem_batch *b) {
  std::vector<BatchScalars> z(b->n);
  memset(z.data(), 0, sizeof(BatchScalars) * b->n);
  FEM_CUDA_TRY(cudaMemcpyAsync(b->d_sc, z.data(), sizeof(BatchScalars) * b->n,
                               cudaMemcpyHostToDevice, b->stream));
  FEM_CUDA_TRY(cudaStreamSynchronize(b->stream));
  return FEM_OK;
}

extern "C" fem_status fem_batch_solve(fem_batch *b, const double *const *bv, double *const *xv,
                                      const fem_cg_opts *o, fem_cg_stats *stats) {
  if (!b || !bv || !xv || !o) { fem_set_error("fem_batch_solve: invalid arguments"); return FEM_EINVAL; }
  if (!(o->rtol > 0.0) || !(o->inner_rtol > 0.0) || o->maxit < 1 || o->max_outer < 1 ||
      o->precond != FEM_PC_JACOBI) {
    fem_set_error("fem_batch_solve: need Jacobi, rtol > 0, inner_rtol > 0, maxit >= 1, max_outer >= 1");
    return FEM_EINVAL;
  }
  if (b->split) return solve_split(b, bv, xv, o, stats);
  int rc = bind_vectors(b, bv, xv);
  if (rc) return rc;
  if ((rc = reset_scalars(b))) return rc;
  BatchArgs a = args_of(b, o->maxit, 0);
  batch_prepare_kernel<<<b->ops[0]->nsm * 8, 256, 0, b->stream>>>(a);
  FEM_CHECK_LAUNCH();
  int steps = 0;
  rc = b->graph_refused ? kGraphRefused : run_solve_graph(b, o, &steps);
  if (rc == kGraphRefused) rc = run_solve(b, o, &steps);
  if (rc) return rc;
  std::vector<BatchScalars> h(b->n);
  FEM_CUDA_TRY(cudaMemcpyAsync(h.data(), b->d_sc, sizeof(BatchScalars) * b->n,
                               cudaMemcpyDeviceToHost, b->stream));
  FEM_CUDA_TRY(cudaStreamSynchronize(b->stream));
  int status = FEM_OK;
  for (int i = 0; i < b->n; i++) {
    int st = h[i].status;
    if (st == FEM_OK && !h[i].converged) st = FEM_ENOCONV;
    if (stats) {
      stats[i].iterations = h[i].total_iter;
      stats[i].outer = h[i].outer;
      stats[i].status = st;
      stats[i].rnorm = sqrt(h[i].rr64_last);
      stats[i].bnorm = sqrt(h[i].bb64_last);
      stats[i].true_rel = h[i].bb64_last > 0 ? sqrt(h[i].rr64_last / h[i].bb64_last) : 0.0;
      stats[i].fallback = 0;
    }
    if (st != FEM_OK && status == FEM_OK) status = st;
  }
  return status;
}

extern "C" fem_status fem_batch_graph_state(const fem_batch *b, int *state) {
  if (!b || !state) { fem_set_error("fem_batch_graph_state: invalid arguments"); return FEM_EINVAL; }
  if (b->split) {
    if (b->inner) return fem_batch_graph_state(b->inner, state);
    *state = 0;
    return FEM_OK;
  }
  *state = b->graph_refused ? -1 : (b->gexec ? 1 : 0);
  return FEM_OK;
}

// Test hook of the bounded grid barrier: launches the persistent kernel with
// one arrival that never comes, so the first barrier must run out after
// timeout_ms; returns what the host reads (FEM_ETIMEOUT).  The batch stays
// usable afterwards.
extern "C" fem_status fem_batch_barrier_selftest(fem_batch *b, double timeout_ms) {
  if (b && b->split) {
    if (b->inner) return fem_batch_barrier_selftest(b->inner, timeout_ms);
    fem_set_error("fem_batch_barrier_selftest: every problem of this batch is solved alone");
    return FEM_EINVAL;
  }
  if (!b || !(timeout_ms > 0) || b->h_prob[0].x == nullptr) {
    fem_set_error("fem_batch_barrier_selftest: invalid arguments (solve once first)");
    return FEM_EINVAL;
  }
  const double saved = b->timeout_ms;
  b->timeout_ms = timeout_ms;
  // every problem active (done_at = INT_MAX), so that the kernel reaches
  // its first grid barrier
  std::vector<BatchScalars> h(b->n);
  memset(h.data(), 0, sizeof(BatchScalars) * b->n);
  for (auto &s : h) s.done_at = INT_MAX;
  cudaError_t e = cudaMemcpyAsync(b->d_sc, h.data(), sizeof(BatchScalars) * b->n,
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    b->timeout_ms = saved;
    fem_set_error("fem_batch_barrier_selftest: %s", cudaGetErrorString(e));
    return FEM_ECUDA;
  }
  BatchArgs a = args_of(b, 1, 1u);
  int rc = launch_inner(b, a, b->nt_choice, b->bps);
  b->timeout_ms = saved;
  if (rc) return rc;
  return read_error(b);
}

// Batch autotuner: time the persistent inner kernel's shapes (block size 128 /
// 256 / 512, blocks per SM) on `iters` inner iterations of this batch from the
// same start state, keep the fastest.  Needs the batch's vectors (b, x).
extern "C" fem_status fem_batch_autotune(fem_batch *b, const double *const *bv,
                                         double *const *xv, int iters, fem_tune_result *res) {
  if (!b || !bv || !xv || iters < 1) { fem_set_error("fem_batch_autotune: invalid arguments"); return FEM_EINVAL; }
  if (b->split) {
    if (!b->inner) {
      if (res) { memset(res, 0, sizeof(*res)); res->epb_choice = b->nt_choice; }
      return FEM_OK;
    }
    std::vector<const double *> sb;
    std::vector<double *> sx;
    for (int i : b->rest) { sb.push_back(bv[i]); sx.push_back(xv[i]); }
    return fem_batch_autotune(b->inner, sb.data(), sx.data(), iters, res);
  }
  int rc = bind_vectors(b, bv, xv);
  if (rc) return rc;
  const int bps_cand[] = {1, 2, 0};
  cudaEvent_t e0, e1;
  FEM_CUDA_TRY(cudaEventCreate(&e0));
  FEM_CUDA_TRY(cudaEventCreate(&e1));
  double best = 1e300;
  int best_nt = 1, best_bps = 0, ncand = 0;
  for (int nt = 0; nt < 3 && rc == FEM_OK; nt++) {
    if ((rc = build_items(b, kNtChoices[nt]))) break;
    for (int bps : bps_cand) {
      if ((rc = reset_scalars(b))) break;
      BatchArgs a = args_of(b, iters, 0);
      batch_prepare_kernel<<<b->ops[0]->nsm * 8, 256, 0, b->stream>>>(a);
      batch_apply64_kernel<<<b->ops[0]->nsm * 4, kNT64, batch_smem<double, kNT64>(), b->stream>>>(a, b->d_gstart64);
      batch_residual_kernel<<<b->ops[0]->nsm * 8, 256, 0, b->stream>>>(a);
      batch_finalize_kernel<<<(b->n + 127) / 128, 128, 0, b->stream>>>(a, 0.0, 0.0);
      // keep every problem active for the timed iterations
      std::vector<BatchScalars> h(b->n);
      FEM_CUDA_TRY(cudaMemcpyAsync(h.data(), b->d_sc, sizeof(BatchScalars) * b->n, cudaMemcpyDeviceToHost, b->stream));
      FEM_CUDA_TRY(cudaStreamSynchronize(b->stream));
      for (auto &s : h) { s.converged = 0; s.done_at = INT_MAX; s.thresh = 0.0; }
      FEM_CUDA_TRY(cudaMemcpyAsync(b->d_sc, h.data(), sizeof(BatchScalars) * b->n, cudaMemcpyHostToDevice, b->stream));
      FEM_CUDA_TRY(cudaEventRecord(e0, b->stream));
      if ((rc = launch_inner(b, a, nt, bps))) break;
      FEM_CUDA_TRY(cudaEventRecord(e1, b->stream));
      if ((rc = read_error(b))) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ncand++;
      if (ms < best) { best = ms; best_nt = nt; best_bps = bps; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  b->nt_choice = best_nt;
  b->bps = best_bps;
  if ((rc = build_items(b, kNtChoices[best_nt]))) return rc;
  if (res) {
    res->epb_choice = best_nt; res->blocks_per_sm = best_bps; res->us = 1e3 * best / iters;
    res->from_cache = 0; res->candidates = ncand;
  }
  return FEM_OK;
}
