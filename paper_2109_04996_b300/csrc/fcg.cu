// Learned preconditioner and flexible CG (no counterpart in the paper; its
// preconditioning discussion is the section "Ecosystem").
//
// Preconditioner  z = B(r) = dinv * r + sum_e G_e^T ( w * ||r_e|| f(r_e/||r_e||, g_e) )
// with f the per-element MLP (mlp.cu), g_e element features (vertex offsets
// from the centroid scaled by the element size, log kappa at the vertices),
// w = 1 / node multiplicity; or z = B(r) = V(r), one FP32 V-cycle of a
// p-multigrid hierarchy (pmg.cu).  B is nonlinear (the network; the fixed-
// count coarse PCG of the V-cycle), so the Krylov method is
// flexible CG with one stored direction (Notay 2000):
//   p_k = z_k - (z_k^T A p_{k-1} / p_{k-1}^T A p_{k-1}) p_{k-1},
//   alpha_k = p_k^T r_k / p_k^T A p_k.
// It runs as the inner FP32 solve of FP64 iterative refinement, as in
// refine.cu: each outer step is one CUDA graph (FP64 residual, preconditioner
// of r_0, conditional WHILE over the FCG body, FP64 correction), and the
// direction carries over from one outer step to the next.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include <cuda_bf16.h>

#include "fem_internal.h"

int fem_mlp_forward_rows(fem_mlp *n, const void *X, int64_t rows, float *Y);
int fem_mlp_mode(const fem_mlp *n);
int fem_mlp_nin(const fem_mlp *n);
int fem_mlp_nout(const fem_mlp *n);
int fem_mlp_reserve(fem_mlp *n, int64_t rows);
void fem_mlp_set_stream(fem_mlp *n, cudaStream_t s, cudaStream_t *old);

constexpr int kNumFeat = 32;  // 24 vertex offsets + 8 log kappa

struct FcgScalars {
  double pAp, pr, zy, rr, rr0;
  double rr64, bb64, rtol2, inner_rtol2, thresh;
  double gamma;     // weight of the learned correction
  double rr_check;  // ||r||^2 at the last stagnation check
  int iter, maxit, done, converged, outer, total_iter, status;
  int fallback;     // 1: learned part switched off for the rest of the solve
};

// Stagnation test of the learned preconditioner: every kCheck inner
// iterations the residual must have dropped by kDrop, else the solve falls
// back to the Jacobi part alone (Jacobi-FCG = Jacobi-PCG).
constexpr int kCheck = 64;
constexpr double kDrop = 0.25;

struct fem_precond {
  fem_op *op = nullptr;
  fem_mlp *mlp = nullptr;      // null: Jacobi only
  fem_pmg *pmg = nullptr;      // set: z = V(r), one FP32 p-multigrid V-cycle
  int64_t E = 0, N = 0, n = 0;
  int P3 = 0, n_in = 0, n_out = 0, esz = 2;
  float *feat = nullptr;       // [E][32]
  float *w = nullptr;          // [N] inverse multiplicity
  void *X = nullptr;           // [E][n_in] compute type
  float *Y = nullptr;          // [E][n_out]
  float *scale = nullptr;      // [E] ||r_e||
  // FCG work
  double *y64 = nullptr;
  float *r = nullptr, *z = nullptr, *p = nullptr, *y = nullptr, *d = nullptr, *dinv = nullptr;
  FcgScalars *sc = nullptr;
  double *partials = nullptr;
  unsigned *counter = nullptr;
  cudaStream_t cap = nullptr, cap2 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const double *g_b = nullptr;
  double *g_x = nullptr;
  double gamma = 1.0;
  double gamma_built = -1.0;   // gamma baked into the scatter launch of the graph
  cudaStream_t cap3 = nullptr;
};

namespace {

constexpr int kT = 256;
int gridn(int64_t n) {
  int64_t g = (n + kT - 1) / kT;
  if (g > 148 * 8) g = 148 * 8;
  return g < 1 ? 1 : (int)g;
}

__global__ void multiplicity_kernel(const int32_t *en, int64_t total, float *w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&w[en[i]], 1.0f);
}
__global__ void invert_kernel(float *w, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] = w[i] > 0.0f ? 1.0f / w[i] : 0.0f;
}

// Element features: the 8 corner nodes' offsets from the centroid divided by
// the element size h (h = 2/sqrt(3) * rms corner distance: the side of a
// cube), then log kappa at the corners (0 without a coefficient).
__global__ void features_kernel(const int32_t *en, const double *xyz, int64_t N, int64_t E,
                                int P, const double *rff, int M, double sigma, float *feat) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int P3 = P * P * P;
    double c[8][3], cen[3] = {0, 0, 0};
    for (int v = 0; v < 8; v++) {
      const int a = (v & 1) ? P - 1 : 0, b = (v & 2) ? P - 1 : 0, k = (v & 4) ? P - 1 : 0;
      const int64_t g = en[e * P3 + a + P * b + P * P * k];
      for (int d = 0; d < 3; d++) { c[v][d] = xyz[d * N + g]; cen[d] += c[v][d] / 8.0; }
    }
    double ms = 0.0;
    for (int v = 0; v < 8; v++)
      for (int d = 0; d < 3; d++) ms += (c[v][d] - cen[d]) * (c[v][d] - cen[d]);
    const double h = 2.0 / sqrt(3.0) * sqrt(ms / 8.0);
    float *f = feat + e * kNumFeat;
    for (int v = 0; v < 8; v++)
      for (int d = 0; d < 3; d++) f[3 * v + d] = (float)((c[v][d] - cen[d]) / h);
    for (int v = 0; v < 8; v++) {
      double lk = 0.0;
      if (rff) {
        double s = 0.0;
        for (int m = 0; m < M; m++)
          s += cos(rff[4 * m] * c[v][0] + rff[4 * m + 1] * c[v][1] + rff[4 * m + 2] * c[v][2] + rff[4 * m + 3]);
        lk = sigma * sqrt(2.0 / M) * s;
      }
      f[24 + v] = (float)lk;
    }
  }
}

template <typename TO>
__device__ __forceinline__ TO to_t(float v) {
  if constexpr (sizeof(TO) == 2) return __float2bfloat16(v);
  else return v;
}

// One warp per element: gather r_e (any input precision), its norm, and the
// network input row; optionally the target row t = e_e / ||r_e||.
template <typename TR, typename TO>
__global__ void build_rows_kernel(const int32_t *en, int64_t E, int P3, int64_t N,
                                  const TR *r, const double *xs, const double *xk,
                                  const float *feat, int n_in,
                                  int n_out, TO *X, float *T, float *scale) {
  const int lane = threadIdx.x & 31;
  for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < E;
       e += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t *g = en + e * P3;
    double ss = 0.0;
    for (int a = lane; a < P3; a += 32) { const double v = (double)r[g[a]]; ss += v * v; }
    ss = fem_warp_sum(ss);
    ss = __shfl_sync(0xffffffffu, ss, 0);
    const double nr = sqrt(ss);
    const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
    TO *xr = X + e * (int64_t)n_in;
    for (int a = lane; a < n_in; a += 32) {
      float v = 0.0f;
      if (a < P3) v = (float)((double)r[g[a]] * inv);
      else if (a < P3 + kNumFeat) v = feat[e * kNumFeat + (a - P3)];
      xr[a] = to_t<TO>(v);
    }
    if (T) {
      float *tr = T + e * (int64_t)n_out;
      for (int a = lane; a < n_out; a += 32)
        tr[a] = a < P3 ? (float)((xs[g[a]] - xk[g[a]]) * inv) : 0.0f;
    }
    if (lane == 0 && scale) scale[e] = (float)nr;
  }
}

// z += sum_e G_e^T (w * scale_e * Y_e)
__global__ void scatter_correction_kernel(const int32_t *en, int64_t E, int P3, const float *Y,
                                          int n_out, const float *scale, const float *w,
                                          const uint8_t *dir, float gamma, float *z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E * P3;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / P3;
    const int a = (int)(i - e * P3);
    const int32_t g = en[i];
    if (dir && dir[g]) continue;
    atomicAdd(&z[g], gamma * w[g] * scale[e] * Y[e * n_out + a]);
  }
}

__global__ void mul_kernel(const float *a, const float *b, float *o, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    o[i] = a[i] * b[i];
}

struct FParams {
  const double *b;
  double *x, *y64;
  float *r, *z, *p, *y, *d;
  const float *dinv;
  const uint8_t *dir;
  int64_t N, n;
  FcgScalars *sc;
  double *partials;
  unsigned *counter;
  cudaGraphConditionalHandle handle;
  cudaGraphConditionalHandle learned;   // IF node around the learned correction
  int has_learned;                       // 1 if that node exists (a network is set)
};

__device__ __forceinline__ bool learned_active(const FcgScalars *s) {
  return !s->fallback && s->gamma != 0.0;
}

// start of a solve: Dirichlet entries of x, the FP64 scratch, and the inner
// direction state (p = z = y = 0, so the first outer step starts with p = z)
__global__ void f_prepare_kernel(double *x, double *y64, float *p, float *z, float *y,
                                 const uint8_t *dir, int64_t N, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (dir && dir[fem_node_of(i, N)]) x[i] = 0.0;
    y64[i] = 0.0;
    p[i] = 0.0f; z[i] = 0.0f; y[i] = 0.0f;
  }
}

__global__ void f_dinv_kernel(const double *diag, const uint8_t *dir, int64_t N, int64_t n, float *dinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dinv[i] = (dir && dir[fem_node_of(i, N)]) ? 0.0f : (float)(1.0 / diag[fem_node_of(i, N)]);
}

// outer residual; inner start r = r64, d = 0, y = 0, z = dinv r (the learned
// part is added by the preconditioner kernels that follow).  The direction is
// kept across outer steps with its preconditioned-residual part swapped
// (reliable update, as in refine.cu): here p -= z_old, and
// f_restart_kernel adds the new z once it is complete.
__global__ void f_residual_kernel(const FParams c) {
  double v[3] = {0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool fixed = c.dir && c.dir[fem_node_of(i, c.N)];
    const double bi = fixed ? 0.0 : c.b[i];
    const double r64 = fixed ? 0.0 : bi - c.y64[i];
    const float r = (float)r64;
    c.p[i] -= c.z[i];
    c.r[i] = r; c.z[i] = c.dinv[i] * r; c.d[i] = 0.0f; c.y[i] = 0.0f;
    c.y64[i] = 0.0;
    v[0] += r64 * r64; v[1] += bi * bi; v[2] += (double)r * r;
  }
  __shared__ double tot[3];
  if (fem_grid_sum<3>(v, c.partials, c.counter, tot) && threadIdx.x == 0) {
    FcgScalars *s = c.sc;
    s->rr64 = tot[0]; s->bb64 = tot[1]; s->rr0 = tot[2]; s->rr = tot[2];
    const bool conv = !(tot[1] > 0.0) || tot[0] <= s->rtol2 * tot[1];
    const bool bad = !isfinite(tot[0]);
    s->converged = conv ? 1 : 0;
    if (bad) { s->status = FEM_EBREAKDOWN; s->converged = 1; }
    s->thresh = s->inner_rtol2 * tot[2];
    s->iter = 0; s->pAp = 0.0; s->zy = 0.0; s->pr = 0.0;
    s->rr_check = tot[2];
    s->done = (s->converged || s->maxit <= 0) ? 1 : 0;
    cudaGraphSetConditional(c.handle, s->done ? 0u : 1u);
    if (c.has_learned) cudaGraphSetConditional(c.learned, (!s->done && learned_active(s)) ? 1u : 0u);
  }
}

// zy = z^T y (y = A p_{k-1}, 0 at the start), beta = -zy / pAp
__global__ void f_dots_kernel(const FParams c) {
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[0] += (double)c.z[i] * (double)c.y[i];
  __shared__ double tot[1];
  if (fem_grid_sum<1>(v, c.partials, c.counter, tot) && threadIdx.x == 0) c.sc->zy = tot[0];
}

// p = z + beta p with beta = -zy/pAp (0 at the start); y = 0; pr = p^T r
__global__ void f_direction_kernel(const FParams c) {
  const double pAp = c.sc->pAp;
  const float beta = pAp > 0.0 ? (float)(-c.sc->zy / pAp) : 0.0f;
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float pv = c.z[i] + beta * c.p[i];
    c.p[i] = pv;
    c.y[i] = 0.0f;
    v[0] += (double)pv * (double)c.r[i];
  }
  __shared__ double tot[1];
  if (fem_grid_sum<1>(v, c.partials, c.counter, tot) && threadIdx.x == 0) c.sc->pr = tot[0];
}

// first direction of an outer step: p += z (z complete, learned part
// included; p held p_old - z_old); y = 0; pr = p^T r
__global__ void f_restart_kernel(const FParams c) {
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float pv = c.p[i] + c.z[i];
    c.p[i] = pv;
    c.y[i] = 0.0f;
    v[0] += (double)pv * (double)c.r[i];
  }
  __shared__ double tot[1];
  if (fem_grid_sum<1>(v, c.partials, c.counter, tot) && threadIdx.x == 0) c.sc->pr = tot[0];
}

// alpha = pr / pAp; d += alpha p; r -= alpha y; z = dinv r; ||r||^2; decide
__global__ void f_update_kernel(const FParams c) {
  FcgScalars *s = c.sc;
  const double pAp = s->pAp;
  const double alpha = s->pr / pAp;
  const bool ok = (pAp > 0.0) && isfinite(alpha);
  const float af = (float)alpha;
  double v[1] = {0.0};
  if (ok) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n;
         i += (int64_t)gridDim.x * blockDim.x) {
      const bool fixed = c.dir && c.dir[fem_node_of(i, c.N)];
      float r = c.r[i];
      c.d[i] += af * c.p[i];
      if (!fixed) r -= af * c.y[i];
      c.r[i] = r;
      c.z[i] = c.dinv[i] * r;
      v[0] += (double)r * (double)r;
    }
  }
  __shared__ double tot[1];
  if (fem_grid_sum<1>(v, c.partials, c.counter, tot) && threadIdx.x == 0) {
    int done = 0;
    if (!ok) done = 1;
    else {
      s->rr = tot[0];
      s->iter += 1;
      s->total_iter += 1;
      if (!isfinite(tot[0]) || tot[0] <= s->thresh || s->iter >= s->maxit) done = 1;
      if (!done && learned_active(s) && s->iter % kCheck == 0) {
        if (tot[0] > kDrop * s->rr_check) { s->fallback = 1; done = 1; }
        s->rr_check = tot[0];
      }
    }
    s->done = done;
    cudaGraphSetConditional(c.handle, done ? 0u : 1u);
    if (c.has_learned) cudaGraphSetConditional(c.learned, (!done && learned_active(s)) ? 1u : 0u);
  }
}

__global__ void f_correct_kernel(const FParams c) {
  if (c.sc->converged) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n;
       i += (int64_t)gridDim.x * blockDim.x)
    c.x[i] += (double)c.d[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) c.sc->outer += 1;
}

// z (Jacobi part already in place) += learned correction of r; with a
// p-multigrid hierarchy instead z = V(r)
int launch_learned(fem_precond *pc, cudaStream_t s) {
  if (pc->pmg) return fem_pmg_enqueue_vcycle32(pc->pmg, pc->r, pc->z, s);
  if (!pc->mlp) return FEM_OK;
  fem_op *op = pc->op;
  const int64_t warps_grid = 148 * 16;
  if (pc->esz == 2)
    build_rows_kernel<float, __nv_bfloat16><<<warps_grid, 256, 0, s>>>(
        op->mesh->d_elem_nodes, pc->E, pc->P3, pc->N, pc->r, nullptr, nullptr, pc->feat,
        pc->n_in, pc->n_out, (__nv_bfloat16 *)pc->X, nullptr, pc->scale);
  else
    build_rows_kernel<float, float><<<warps_grid, 256, 0, s>>>(
        op->mesh->d_elem_nodes, pc->E, pc->P3, pc->N, pc->r, nullptr, nullptr, pc->feat,
        pc->n_in, pc->n_out, (float *)pc->X, nullptr, pc->scale);
  FEM_CHECK_LAUNCH();
  int rc = fem_mlp_forward_rows(pc->mlp, pc->X, pc->E, pc->Y);
  if (rc) return rc;
  scatter_correction_kernel<<<gridn(pc->E * pc->P3), kT, 0, s>>>(
      op->mesh->d_elem_nodes, pc->E, pc->P3, pc->Y, pc->n_out, pc->scale, pc->w,
      op->mesh->d_dirichlet, (float)pc->gamma, pc->z);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

FParams fparams(fem_precond *pc, const double *b, double *x, cudaGraphConditionalHandle h) {
  FParams c;
  c.b = b; c.x = x; c.y64 = pc->y64; c.r = pc->r; c.z = pc->z; c.p = pc->p; c.y = pc->y;
  c.d = pc->d; c.dinv = pc->dinv; c.dir = pc->op->mesh->d_dirichlet; c.N = pc->N; c.n = pc->n;
  c.sc = pc->sc; c.partials = pc->partials; c.counter = pc->counter; c.handle = h;
  c.learned = 0;
  c.has_learned = 0;
  return c;
}

// Append to the capture of `s` a conditional IF node (handle h) whose body,
// captured on `s2`, adds the learned correction to z.
int add_learned_if(fem_precond *pc, cudaStream_t s, cudaStream_t s2, cudaGraphConditionalHandle h,
                   cudaError_t *err) {
  cudaStreamCaptureStatus st;
  cudaGraph_t graph;
  const cudaGraphNode_t *deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &graph, &deps, nullptr, &ndeps);
  if (e != cudaSuccess) { *err = e; return FEM_ECUDA; }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &cp)) != cudaSuccess) { *err = e; return FEM_ECUDA; }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) != cudaSuccess) {
    *err = e;
    return FEM_ECUDA;
  }
  fem_mesh *mesh = const_cast<fem_mesh *>(pc->op->mesh);
  cudaStream_t saved = mesh->stream, saved_mlp = nullptr;
  mesh->stream = s2;
  if (pc->mlp) fem_mlp_set_stream(pc->mlp, s2, &saved_mlp);
  if ((e = cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) != cudaSuccess) {
    mesh->stream = saved;
    if (pc->mlp) fem_mlp_set_stream(pc->mlp, saved_mlp, nullptr);
    *err = e;
    return FEM_ECUDA;
  }
  int rc = launch_learned(pc, s2);
  cudaGraph_t tmp;
  cudaError_t e2 = cudaStreamEndCapture(s2, &tmp);
  mesh->stream = saved;
  if (pc->mlp) fem_mlp_set_stream(pc->mlp, saved_mlp, nullptr);
  if (!rc && e2 != cudaSuccess) { *err = e2; rc = FEM_ECUDA; }
  return rc;
}

void destroy_graph(fem_precond *pc) {
  if (pc->exec) cudaGraphExecDestroy(pc->exec);
  if (pc->graph) cudaGraphDestroy(pc->graph);
  pc->exec = nullptr; pc->graph = nullptr;
}

int build_graph(fem_precond *pc, const double *b, double *x) {
  destroy_graph(pc);
  fem_op *op = pc->op;
  fem_mesh *mesh = const_cast<fem_mesh *>(op->mesh);
  cudaStream_t user = mesh->stream;
  cudaStream_t saved_mlp = nullptr;
  if (!pc->cap) {
    FEM_CUDA_TRY(cudaStreamCreateWithFlags(&pc->cap, cudaStreamNonBlocking));
    FEM_CUDA_TRY(cudaStreamCreateWithFlags(&pc->cap2, cudaStreamNonBlocking));
    FEM_CUDA_TRY(cudaStreamCreateWithFlags(&pc->cap3, cudaStreamNonBlocking));
  }
  int rc = FEM_OK;
  cudaError_t e = cudaSuccess;
  cudaGraph_t graph = nullptr;
  mesh->stream = pc->cap;
  if (pc->mlp) fem_mlp_set_stream(pc->mlp, pc->cap, &saved_mlp);
  FEM_CUDA_TRY(cudaStreamBeginCapture(pc->cap, cudaStreamCaptureModeRelaxed));
  do {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaGraphConditionalHandle h = 0, hl0 = 0, hl = 0;
    e = cudaStreamGetCaptureInfo(pc->cap, &st, nullptr, &graph, nullptr, nullptr, nullptr);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    const bool extra = pc->mlp || pc->pmg;   // preconditioner part behind an IF node
    if (e == cudaSuccess && extra)
      e = cudaGraphConditionalHandleCreate(&hl0, graph, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
    FParams c = fparams(pc, b, x, h);
    c.learned = hl0;
    c.has_learned = extra ? 1 : 0;
    const int g = gridn(c.n);
    if ((rc = fem_launch_apply_f64(op, x, pc->y64, nullptr, op->E, nullptr))) break;
    f_residual_kernel<<<g, kT, 0, pc->cap>>>(c);
    // IF (learned part active) { z += learned correction of r_0 } (or z = V(r_0))
    if (extra) {
      if ((rc = add_learned_if(pc, pc->cap, pc->cap3, hl0, &e))) break;
    }
    f_restart_kernel<<<g, kT, 0, pc->cap>>>(c);  // p = p_old + (z - z_old), pr
    e = cudaStreamGetCaptureInfo(pc->cap, &st, nullptr, &graph, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    if ((e = cudaGraphAddNode(&cnode, graph, deps, nullptr, ndeps, &cp)) != cudaSuccess) { rc = FEM_ECUDA; break; }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamUpdateCaptureDependencies(pc->cap, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
    mesh->stream = pc->cap2;
    if (pc->mlp) fem_mlp_set_stream(pc->mlp, pc->cap2, nullptr);
    e = cudaStreamBeginCaptureToGraph(pc->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
    if (extra && (e = cudaGraphConditionalHandleCreate(&hl, body, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
      rc = FEM_ECUDA;
    FParams cb = c;
    cb.learned = hl;
    if (!rc) rc = fem_launch_apply_f32(op, c.p, c.y, nullptr, op->E, &c.sc->pAp);
    if (!rc) {
      f_update_kernel<<<g, kT, 0, pc->cap2>>>(cb);
      if (extra) rc = add_learned_if(pc, pc->cap2, pc->cap3, hl, &e);
    }
    if (!rc) {
      f_dots_kernel<<<g, kT, 0, pc->cap2>>>(cb);
      f_direction_kernel<<<g, kT, 0, pc->cap2>>>(cb);
    }
    cudaGraph_t tmp;
    cudaError_t e2 = cudaStreamEndCapture(pc->cap2, &tmp);
    if (!rc && e2 != cudaSuccess) { e = e2; rc = FEM_ECUDA; }
    mesh->stream = pc->cap;
    if (rc) break;
    f_correct_kernel<<<g, kT, 0, pc->cap>>>(c);
  } while (0);
  cudaGraph_t g2 = nullptr;
  cudaError_t e3 = cudaStreamEndCapture(pc->cap, &g2);
  mesh->stream = user;
  if (pc->mlp) fem_mlp_set_stream(pc->mlp, saved_mlp, nullptr);
  if (rc == FEM_OK && e3 != cudaSuccess) { rc = FEM_ECUDA; e = e3; }
  if (rc != FEM_OK) {
    if (g2) cudaGraphDestroy(g2);
    cudaGetLastError();
    if (rc == FEM_ECUDA) fem_set_error("fem_fcg_solve: building the CUDA graph failed: %s", cudaGetErrorString(e));
    return rc;
  }
  pc->graph = g2;
  FEM_CUDA_TRY(cudaGraphInstantiate(&pc->exec, pc->graph, 0));
  pc->g_b = b; pc->g_x = x;
  return FEM_OK;
}

}  // namespace

extern "C" fem_status fem_precond_create(fem_op *op, fem_mlp *mlp, fem_precond **out) {
  if (!op || !out || !op->d_qdata32) {
    fem_set_error("fem_precond_create: need an operator created with FEM_F32");
    return FEM_EINVAL;
  }
  if (op->ncomp != 1) { fem_set_error("fem_precond_create: scalar operators only"); return FEM_EINVAL; }
  const int P3 = op->P * op->P * op->P;
  if (mlp && (fem_mlp_nin(mlp) < P3 + kNumFeat || fem_mlp_nout(mlp) < P3)) {
    fem_set_error("fem_precond_create: network needs n_in >= %d and n_out >= %d", P3 + kNumFeat, P3);
    return FEM_EINVAL;
  }
  fem_precond *pc = new fem_precond();
  pc->op = op; pc->mlp = mlp; pc->E = op->E; pc->N = op->N; pc->n = op->N; pc->P3 = P3;
  pc->n_in = mlp ? fem_mlp_nin(mlp) : 0;
  pc->n_out = mlp ? fem_mlp_nout(mlp) : 0;
  pc->esz = (mlp && fem_mlp_mode(mlp) == 1) ? 4 : 2;
  const size_t n = (size_t)pc->n, E = (size_t)pc->E;
  bool ok = cudaMalloc(&pc->feat, sizeof(float) * E * kNumFeat) == cudaSuccess &&
            cudaMalloc(&pc->w, sizeof(float) * n) == cudaSuccess &&
            cudaMalloc(&pc->scale, sizeof(float) * (E + 1)) == cudaSuccess &&
            cudaMalloc(&pc->y64, 8 * n) == cudaSuccess && cudaMalloc(&pc->r, 4 * n) == cudaSuccess &&
            cudaMalloc(&pc->z, 4 * n) == cudaSuccess && cudaMalloc(&pc->p, 4 * n) == cudaSuccess &&
            cudaMalloc(&pc->y, 4 * n) == cudaSuccess && cudaMalloc(&pc->d, 4 * n) == cudaSuccess &&
            cudaMalloc(&pc->dinv, 4 * n) == cudaSuccess &&
            cudaMalloc(&pc->sc, sizeof(FcgScalars)) == cudaSuccess &&
            cudaMalloc(&pc->partials, sizeof(double) * 4 * FEM_MAX_BLOCKS) == cudaSuccess &&
            cudaMalloc(&pc->counter, sizeof(unsigned) * 4) == cudaSuccess;
  if (ok && mlp)
    ok = cudaMalloc(&pc->X, (size_t)pc->esz * E * pc->n_in) == cudaSuccess &&
         cudaMalloc(&pc->Y, sizeof(float) * E * pc->n_out) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    fem_precond_destroy(pc);
    fem_set_error("fem_precond_create: allocation failed");
    return FEM_ENOMEM;
  }
  cudaStream_t s = op->stream();
  if (mlp) {
    // the network's activation workspace must exist before any graph capture
    int rc = fem_mlp_reserve(mlp, (int64_t)E);
    if (rc) { fem_precond_destroy(pc); return rc; }
    fem_mlp_set_stream(mlp, s, nullptr);
  }
  FEM_CUDA_TRY(cudaMemsetAsync(pc->counter, 0, sizeof(unsigned) * 4, s));
  FEM_CUDA_TRY(cudaMemsetAsync(pc->w, 0, sizeof(float) * n, s));
  multiplicity_kernel<<<gridn(E * P3), kT, 0, s>>>(op->mesh->d_elem_nodes, (int64_t)(E * P3), pc->w);
  invert_kernel<<<gridn(n), kT, 0, s>>>(pc->w, (int64_t)n);
  features_kernel<<<gridn(E), kT, 0, s>>>(op->mesh->d_elem_nodes, op->mesh->d_xyz, op->N, op->E,
                                         op->P, op->d_rff, op->M, op->sigma, pc->feat);
  f_dinv_kernel<<<gridn(n), kT, 0, s>>>(op->d_diag, op->mesh->d_dirichlet, op->N, (int64_t)n, pc->dinv);
  FEM_CHECK_LAUNCH();
  FEM_CUDA_TRY(cudaStreamSynchronize(s));
  *out = pc;
  return FEM_OK;
}

extern "C" fem_status fem_precond_create_pmg(fem_pmg *pmg, fem_precond **out) {
  if (!pmg || !out) { fem_set_error("fem_precond_create_pmg: invalid arguments"); return FEM_EINVAL; }
  *out = nullptr;
  if (fem_pmg_precision(pmg) != FEM_F32) {
    fem_set_error("fem_precond_create_pmg: the hierarchy must run its V-cycle in FEM_F32");
    return FEM_EINVAL;
  }
  fem_precond *pc = nullptr;
  int rc = fem_precond_create(fem_pmg_finest(pmg), nullptr, &pc);
  if (rc) return rc;
  pc->pmg = pmg;
  *out = pc;
  return FEM_OK;
}

extern "C" fem_status fem_precond_destroy(fem_precond *pc) {
  if (!pc) return FEM_OK;
  destroy_graph(pc);
  if (pc->cap) cudaStreamDestroy(pc->cap);
  if (pc->cap2) cudaStreamDestroy(pc->cap2);
  if (pc->cap3) cudaStreamDestroy(pc->cap3);
  cudaFree(pc->feat); cudaFree(pc->w); cudaFree(pc->X); cudaFree(pc->Y); cudaFree(pc->scale);
  cudaFree(pc->y64); cudaFree(pc->r); cudaFree(pc->z); cudaFree(pc->p); cudaFree(pc->y);
  cudaFree(pc->d); cudaFree(pc->dinv); cudaFree(pc->sc); cudaFree(pc->partials); cudaFree(pc->counter);
  delete pc;
  return FEM_OK;
}

extern "C" fem_status fem_precond_features(fem_precond *pc, float *feat_host) {
  if (!pc || !feat_host) { fem_set_error("fem_precond_features: invalid arguments"); return FEM_EINVAL; }
  FEM_CUDA_TRY(cudaMemcpyAsync(feat_host, pc->feat, sizeof(float) * pc->E * kNumFeat,
                               cudaMemcpyDeviceToHost, pc->op->stream()));
  FEM_CUDA_TRY(cudaStreamSynchronize(pc->op->stream()));
  return FEM_OK;
}

// Training samples of the plain solver's iterate x_k (FP64 device [N]):
// r = M (b - A x_k) (in the FP64 scratch y64), e = x_star - x_k; per element
// X = [r_e / ||r_e||, g_e, 0...], T = [e_e / ||r_e||, 0...].
extern "C" fem_status fem_precond_samples(fem_precond *pc, const double *b, const double *x_star,
                                          const double *x_k, void *X, float *T) {
  if (!pc || !pc->mlp || !b || !x_star || !x_k || !X || !T) {
    fem_set_error("fem_precond_samples: invalid arguments (needs a network)");
    return FEM_EINVAL;
  }
  int rc = fem_op_residual(pc->op, b, x_k, pc->y64);
  if (rc) return rc;
  cudaStream_t s = pc->op->stream();
  if (pc->esz == 2)
    build_rows_kernel<double, __nv_bfloat16><<<148 * 16, 256, 0, s>>>(
        pc->op->mesh->d_elem_nodes, pc->E, pc->P3, pc->N, pc->y64, x_star, x_k, pc->feat,
        pc->n_in, pc->n_out, (__nv_bfloat16 *)X, T, nullptr);
  else
    build_rows_kernel<double, float><<<148 * 16, 256, 0, s>>>(
        pc->op->mesh->d_elem_nodes, pc->E, pc->P3, pc->N, pc->y64, x_star, x_k, pc->feat,
        pc->n_in, pc->n_out, (float *)X, T, nullptr);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

// z = B(r) for a given FP32 residual (for tests): r, z device [N] float.
extern "C" fem_status fem_precond_apply(fem_precond *pc, const float *r, float *z) {
  if (!pc || !r || !z) { fem_set_error("fem_precond_apply: invalid arguments"); return FEM_EINVAL; }
  cudaStream_t s = pc->op->stream();
  FEM_CUDA_TRY(cudaMemcpyAsync(pc->r, r, sizeof(float) * pc->n, cudaMemcpyDeviceToDevice, s));
  // z = dinv r
  f_dinv_kernel<<<gridn(pc->n), kT, 0, s>>>(pc->op->d_diag, pc->op->mesh->d_dirichlet, pc->N, pc->n, pc->dinv);
  mul_kernel<<<gridn(pc->n), kT, 0, s>>>(pc->dinv, pc->r, pc->z, pc->n);
  int rc = launch_learned(pc, s);
  if (rc) return rc;
  FEM_CUDA_TRY(cudaMemcpyAsync(z, pc->z, sizeof(float) * pc->n, cudaMemcpyDeviceToDevice, s));
  return FEM_OK;
}

extern "C" fem_status fem_fcg_solve(fem_precond *pc, const double *b, double *x,
                                    const fem_cg_opts *o, fem_cg_stats *st) {
  if (!pc || !b || !x || !o || b == x) { fem_set_error("fem_fcg_solve: invalid arguments"); return FEM_EINVAL; }
  if (!(o->rtol > 0.0) || !(o->inner_rtol > 0.0) || o->maxit < 1 || o->max_outer < 1) {
    fem_set_error("fem_fcg_solve: need rtol > 0, inner_rtol > 0, maxit >= 1, max_outer >= 1");
    return FEM_EINVAL;
  }
  fem_op *op = pc->op;
  cudaStream_t s = op->stream();
  FcgScalars init = {};
  init.maxit = o->maxit;
  init.rtol2 = o->rtol * o->rtol;
  init.inner_rtol2 = o->inner_rtol * o->inner_rtol;
  init.gamma = pc->pmg ? 1.0 : (pc->mlp ? pc->gamma : 0.0);
  FEM_CUDA_TRY(cudaMemcpyAsync(pc->sc, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  f_dinv_kernel<<<gridn(pc->n), kT, 0, s>>>(op->d_diag, op->mesh->d_dirichlet, pc->N, pc->n, pc->dinv);
  f_prepare_kernel<<<gridn(pc->n), kT, 0, s>>>(x, pc->y64, pc->p, pc->z, pc->y,
                                               op->mesh->d_dirichlet, pc->N, pc->n);
  FEM_CHECK_LAUNCH();
  if (!pc->exec || pc->g_b != b || pc->g_x != x || pc->gamma_built != pc->gamma) {
    FEM_CUDA_TRY(cudaStreamSynchronize(s));
    int rc = build_graph(pc, b, x);
    if (rc) return rc;
    pc->gamma_built = pc->gamma;
  }
  FcgScalars out = {};
  int steps = 0;
  for (;;) {
    FEM_CUDA_TRY(cudaGraphLaunch(pc->exec, s));
    FEM_CUDA_TRY(cudaMemcpyAsync(&out, pc->sc, sizeof(out), cudaMemcpyDeviceToHost, s));
    FEM_CUDA_TRY(cudaStreamSynchronize(s));
    steps++;
    if (out.converged || out.status != FEM_OK || steps > o->max_outer) break;
  }
  int status = out.status;
  if (status == FEM_OK && !out.converged) status = FEM_ENOCONV;
  if (st) {
    st->iterations = out.total_iter;
    st->outer = out.outer;
    st->status = status;
    st->rnorm = sqrt(out.rr64);
    st->bnorm = sqrt(out.bb64);
    st->true_rel = out.bb64 > 0 ? sqrt(out.rr64 / out.bb64) : 0.0;
    st->fallback = out.fallback;
  }
  return status;
}

extern "C" fem_status fem_precond_calibrate(fem_precond *pc, const double *b, double *x,
                                            const double *gammas, int n, int probe_iters,
                                            double *best_gamma) {
  if (!pc || !b || !x || !gammas || n < 1 || probe_iters < 1 || !best_gamma || b == x) {
    fem_set_error("fem_precond_calibrate: invalid arguments");
    return FEM_EINVAL;
  }
  for (int i = 0; i < n; i++)
    if (!(gammas[i] >= 0.0) || !isfinite(gammas[i])) {
      fem_set_error("fem_precond_calibrate: gamma %d must be finite and >= 0", i);
      return FEM_EINVAL;
    }
  const double keep = pc->gamma;
  fem_cg_opts o = {};
  o.precond = FEM_PC_LEARNED;
  o.maxit = probe_iters;
  o.rtol = 1e-14;
  o.inner_rtol = 1e-14;
  o.max_outer = 1;
  double best = 0.0, best_score = INFINITY;
  bool have = false;
  const size_t vb = sizeof(double) * (size_t)pc->n;
  for (int i = 0; i < n; i++) {
    pc->gamma = gammas[i];
    FEM_CUDA_TRY(cudaMemsetAsync(x, 0, vb, pc->op->stream()));
    fem_cg_stats st = {};
    const int rc = fem_fcg_solve(pc, b, x, &o, &st);
    if (rc != FEM_OK && rc != FEM_ENOCONV) { pc->gamma = keep; return rc; }
    const double score = st.fallback ? INFINITY : st.true_rel;
    if (!have || score < best_score) { best = gammas[i]; best_score = score; have = true; }
  }
  pc->gamma = best;
  *best_gamma = best;
  return FEM_OK;
}

extern "C" fem_status fem_precond_set_gamma(fem_precond *pc, double gamma) {
  if (!pc || !(gamma >= 0.0) || !isfinite(gamma)) {
    fem_set_error("fem_precond_set_gamma: gamma must be finite and >= 0");
    return FEM_EINVAL;
  }
  pc->gamma = gamma;
  return FEM_OK;
}
