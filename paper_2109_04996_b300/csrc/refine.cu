// Mixed-precision solve: FP64 iterative refinement around an FP32 inner
// Jacobi-PCG.  The paper fixes the operator and the CG solve (sections
// "Benchmarks" and "libCEED"); the refinement is classical iterative
// refinement (Wilkinson; Carson & Higham 2018) with "reliable updates"
// (Strzodka & Goeddeke 2006; Clark et al. 2010): the inner CG is not
// restarted at each outer step, only its residual is replaced.
//
//   repeat:  r = b - A_64 x          (FP64 fused apply, FP64 vectors)
//            stop if ||r|| <= rtol ||b||
//            r_32 = r, z = dinv r_32 and p += z - z_old: the direction
//            keeps its history (the last inner step formed p = z_old +
//            beta p_prev; its residual part is swapped for the true one;
//            p = z at the first step, where p = z_old = 0)
//            continue the FP32 CG on A_32 d = r (FP32 apply, FP32 vectors,
//            FP64 dot products and scalars) until ||r_32|| <= inner_rtol ||r||
//            x = x + d               (FP64)
//
// Each outer step is one CUDA graph launch: residual kernel, direction
// kernel, a conditional WHILE node over the inner CG body (apply, update,
// direction), correction kernel.  The host reads one status word per step.
#include <math.h>

#include "fem_internal.h"

struct RefineScalars {
  CgScalars in;      // inner CG scalars (rz, pAp, rr, tol2 = inner threshold, ...)
  double rr64, bb64; // outer residual and right-hand side, squared
  double rtol2;      // outer rtol^2
  double inner_rtol2;   // inner relative tolerance, squared
  double inner_thresh;  // absolute inner threshold on ||r_inner||^2 of this step
  int outer;         // corrections applied
  int total_iter;    // inner iterations over all outer steps
  int converged;     // outer test met
  int status;
};

struct RefineWork {
  int64_t n = 0;
  int dinv_pc = -1;
  double *y64 = nullptr;
  float *r = nullptr, *z = nullptr, *p = nullptr, *y = nullptr, *d = nullptr, *dinv = nullptr;
  RefineScalars *sc = nullptr;
  double *partials = nullptr;
  unsigned *counter = nullptr;
  cudaStream_t cap = nullptr, cap2 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const double *g_b = nullptr;
  double *g_x = nullptr;
};

namespace {

constexpr int kT = 256;

int grid_for(int64_t n) {
  int64_t g = (n + kT - 1) / kT;
  if (g > 148 * 8) g = 148 * 8;
  return g < 1 ? 1 : (int)g;
}

struct RParams {
  const double *b;
  double *x, *y64;
  float *r, *z, *p, *y, *d;
  const float *dinv;
  const uint8_t *dir;
  int64_t N, n;
  RefineScalars *sc;
  double *partials;
  unsigned *counter;
  cudaGraphConditionalHandle handle;
};

__global__ void rf_dinv_kernel(const double *diag, const uint8_t *dir, int64_t N, int64_t n,
                               int pc, float *dinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = fem_node_of(i, N);
    dinv[i] = (dir && dir[node]) ? 0.0f : (pc == FEM_PC_JACOBI ? (float)(1.0 / diag[node]) : 1.0f);
  }
}

// x <- M x, y64 <- 0, p <- 0, z <- 0 (before the first residual)
__global__ void rf_prepare_kernel(double *x, double *y64, float *p, float *z, const uint8_t *dir,
                                  int64_t N, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (dir && dir[fem_node_of(i, N)]) x[i] = 0.0;
    y64[i] = 0.0;
    p[i] = 0.0f;
    z[i] = 0.0f;
  }
}

// Outer residual r64 = M (b - A x) (FP64), rounded to FP32: the inner
// solve's residual is replaced, r = r64, z = dinv r, d = 0, and the
// direction's residual part is swapped, p += z - z_old (reliable update).
__global__ void rf_residual_kernel(const RParams c) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool fixed = c.dir && c.dir[fem_node_of(i, c.N)];
    const double bi = fixed ? 0.0 : c.b[i];
    const double r64 = fixed ? 0.0 : bi - c.y64[i];
    const float r = (float)r64;
    const float z = c.dinv[i] * r;
    c.p[i] += z - c.z[i];
    c.r[i] = r; c.z[i] = z; c.d[i] = 0.0f; c.y[i] = 0.0f;
    c.y64[i] = 0.0;
    v[0] += r64 * r64; v[1] += bi * bi; v[2] += (double)r * (double)z; v[3] += (double)r * r;
  }
  __shared__ double tot[4];
  if (fem_grid_sum<4>(v, c.partials, c.counter, tot) && threadIdx.x == 0) {
    RefineScalars *s = c.sc;
    s->rr64 = tot[0]; s->bb64 = tot[1];
    CgScalars &in = s->in;
    in.beta = 0.0;
    in.rz = tot[2]; in.rr = tot[3]; in.iter = 0; in.status = FEM_OK;
    in.pAp = 0.0; in.alpha = 0.0;
    const bool conv = !(tot[1] > 0.0) || tot[0] <= s->rtol2 * tot[1];
    const bool bad = !isfinite(tot[0]) || !isfinite(tot[2]);
    s->converged = conv ? 1 : 0;
    if (bad) s->status = FEM_EBREAKDOWN;
    s->inner_thresh = s->inner_rtol2 * tot[3];  // relative to this step's FP32 residual
    in.done = (conv || bad || in.maxit <= 0) ? 1 : 0;
    cudaGraphSetConditional(c.handle, in.done ? 0u : 1u);
  }
}

__global__ void rf_update_kernel(const RParams c) {
  CgScalars &s = c.sc->in;
  const double pAp = s.pAp;
  const double alpha = s.rz / pAp;
  const bool ok = (pAp > 0.0) && isfinite(alpha);
  const float af = (float)alpha;
  double v[2] = {0.0, 0.0};
  if (ok) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n;
         i += (int64_t)gridDim.x * blockDim.x) {
      const bool fixed = c.dir && c.dir[fem_node_of(i, c.N)];
      float r = c.r[i];
      c.d[i] += af * c.p[i];
      if (!fixed) r -= af * c.y[i];
      c.r[i] = r;
      const float z = c.dinv[i] * r;
      c.z[i] = z;
      v[0] += (double)r * (double)z; v[1] += (double)r * (double)r;
    }
  }
  __shared__ double tot[2];
  if (fem_grid_sum<2>(v, c.partials, c.counter, tot) && threadIdx.x == 0) {
    int done = 0;
    if (!ok) {
      // FP32 breakdown (e.g. the residual reached FP32 noise): stop the inner
      // solve and let the FP64 refinement decide.
      done = 1;
    } else {
      s.beta = tot[0] / s.rz;
      s.rz = tot[0]; s.rr = tot[1];
      s.iter += 1;
      c.sc->total_iter += 1;
      if (!isfinite(tot[0])) done = 1;
      else if (tot[1] <= c.sc->inner_thresh) done = 1;
      else if (s.iter >= s.maxit) done = 1;
    }
    s.done = done;
    cudaGraphSetConditional(c.handle, done ? 0u : 1u);
  }
}

__global__ void rf_direction_kernel(const RParams c) {
  const float beta = (float)c.sc->in.beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    c.p[i] = c.z[i] + beta * c.p[i];
    c.y[i] = 0.0f;
  }
}

// x += d (FP64), unless the outer test was already met.
__global__ void rf_correct_kernel(const RParams c) {
  if (c.sc->converged) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n;
       i += (int64_t)gridDim.x * blockDim.x)
    c.x[i] += (double)c.d[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) c.sc->outer += 1;
}

int ensure(fem_op *op) {
  if (op->ir) return FEM_OK;
  RefineWork *w = new RefineWork();
  op->ir = w;
  w->n = op->N * op->ncomp;
  const size_t n = (size_t)w->n;
  bool ok = cudaMalloc(&w->y64, 8 * n) == cudaSuccess && cudaMalloc(&w->r, 4 * n) == cudaSuccess &&
            cudaMalloc(&w->z, 4 * n) == cudaSuccess && cudaMalloc(&w->p, 4 * n) == cudaSuccess &&
            cudaMalloc(&w->y, 4 * n) == cudaSuccess && cudaMalloc(&w->d, 4 * n) == cudaSuccess &&
            cudaMalloc(&w->dinv, 4 * n) == cudaSuccess &&
            cudaMalloc(&w->sc, sizeof(RefineScalars)) == cudaSuccess &&
            cudaMalloc(&w->partials, sizeof(double) * 4 * FEM_MAX_BLOCKS) == cudaSuccess &&
            cudaMalloc(&w->counter, sizeof(unsigned) * 4) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    fem_set_error("fem_solve_refined: device allocation of the workspace failed");
    return FEM_ENOMEM;
  }
  cudaStream_t s = op->stream();
  FEM_CUDA_TRY(cudaMemsetAsync(w->counter, 0, sizeof(unsigned) * 4, s));
  op->bytes += 32 * (int64_t)n;
  return FEM_OK;
}

RParams params(fem_op *op, const double *b, double *x, cudaGraphConditionalHandle h) {
  RefineWork *w = op->ir;
  RParams c;
  c.b = b; c.x = x; c.y64 = w->y64; c.r = w->r; c.z = w->z; c.p = w->p; c.y = w->y; c.d = w->d;
  c.dinv = w->dinv; c.dir = op->mesh->d_dirichlet; c.N = op->N; c.n = w->n; c.sc = w->sc;
  c.partials = w->partials; c.counter = w->counter; c.handle = h;
  return c;
}

void destroy_graph(RefineWork *w) {
  if (w->exec) cudaGraphExecDestroy(w->exec);
  if (w->graph) cudaGraphDestroy(w->graph);
  w->exec = nullptr; w->graph = nullptr;
}

// One outer step as a graph: y64 = A_64 x; residual; WHILE(inner) {apply32,
// update, direction}; x += d.  (x has been masked and y64 zeroed before.)
int build_graph(fem_op *op, const double *b, double *x) {
  RefineWork *w = op->ir;
  destroy_graph(w);
  fem_mesh *mesh = const_cast<fem_mesh *>(op->mesh);
  cudaStream_t user = mesh->stream;
  if (!w->cap) {
    FEM_CUDA_TRY(cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking));
    FEM_CUDA_TRY(cudaStreamCreateWithFlags(&w->cap2, cudaStreamNonBlocking));
  }
  int rc = FEM_OK;
  cudaError_t e = cudaSuccess;
  cudaGraph_t graph = nullptr;
  mesh->stream = w->cap;
  FEM_CUDA_TRY(cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeRelaxed));
  do {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaGraphConditionalHandle h = 0;
    e = cudaStreamGetCaptureInfo(w->cap, &st, nullptr, &graph, nullptr, nullptr, nullptr);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
    RParams c = params(op, b, x, h);
    const int g = grid_for(c.n);
    rc = fem_launch_apply_f64(op, x, w->y64, nullptr, op->E, nullptr);
    if (rc) break;
    rf_residual_kernel<<<g, kT, 0, w->cap>>>(c);
    e = cudaGetLastError();
    if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
    e = cudaStreamGetCaptureInfo(w->cap, &st, nullptr, &graph, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    e = cudaGraphAddNode(&cnode, graph, deps, nullptr, ndeps, &cp);
    if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamUpdateCaptureDependencies(w->cap, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
    mesh->stream = w->cap2;
    e = cudaStreamBeginCaptureToGraph(w->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
    rc = fem_launch_apply_f32(op, c.p, c.y, nullptr, op->E, &c.sc->in.pAp);
    if (!rc) {
      rf_update_kernel<<<g, kT, 0, w->cap2>>>(c);
      rf_direction_kernel<<<g, kT, 0, w->cap2>>>(c);
    }
    cudaGraph_t tmp;
    cudaError_t e2 = cudaStreamEndCapture(w->cap2, &tmp);
    if (!rc && e2 != cudaSuccess) { e = e2; rc = FEM_ECUDA; }
    mesh->stream = w->cap;
    if (rc) break;
    rf_correct_kernel<<<g, kT, 0, w->cap>>>(c);
  } while (0);
  cudaGraph_t g2 = nullptr;
  cudaError_t e3 = cudaStreamEndCapture(w->cap, &g2);
  mesh->stream = user;
  if (rc == FEM_OK && e3 != cudaSuccess) { rc = FEM_ECUDA; e = e3; }
  if (rc != FEM_OK) {
    if (g2) cudaGraphDestroy(g2);
    cudaGetLastError();
    if (rc == FEM_ECUDA)
      fem_set_error("fem_solve_refined: building the CUDA graph failed: %s", cudaGetErrorString(e));
    return rc;
  }
  w->graph = g2;
  FEM_CUDA_TRY(cudaGraphInstantiate(&w->exec, w->graph, 0));
  w->g_b = b; w->g_x = x;
  return FEM_OK;
}

}  // namespace

extern "C" fem_status fem_solve_refined(fem_op *op, const double *b, double *x,
                                        const fem_cg_opts *o, fem_cg_stats *st) {
  if (!op || !b || !x || !o || b == x) { fem_set_error("fem_solve_refined: invalid arguments"); return FEM_EINVAL; }
  if (!op->d_qdata32) { fem_set_error("fem_solve_refined: operator not created with FEM_F32"); return FEM_EINVAL; }
  if (o->precond != FEM_PC_JACOBI && o->precond != FEM_PC_NONE) {
    fem_set_error("fem_solve_refined: preconditioner %d not available", o->precond);
    return FEM_EINVAL;
  }
  if (!(o->rtol > 0.0) || !(o->inner_rtol > 0.0) || o->maxit < 1 || o->max_outer < 1) {
    fem_set_error("fem_solve_refined: need rtol > 0, inner_rtol > 0, maxit >= 1, max_outer >= 1");
    return FEM_EINVAL;
  }
  int rc = ensure(op);
  if (rc) return rc;
  RefineWork *w = op->ir;
  cudaStream_t s = op->stream();
  if (w->dinv_pc != o->precond) {
    rf_dinv_kernel<<<grid_for(w->n), kT, 0, s>>>(op->d_diag, op->mesh->d_dirichlet, op->N, w->n,
                                                  o->precond, w->dinv);
    FEM_CHECK_LAUNCH();
    w->dinv_pc = o->precond;
  }
  RefineScalars init = {};
  init.in.maxit = o->maxit;
  init.inner_rtol2 = o->inner_rtol * o->inner_rtol;
  init.rtol2 = o->rtol * o->rtol;
  FEM_CUDA_TRY(cudaMemcpyAsync(w->sc, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  rf_prepare_kernel<<<grid_for(w->n), kT, 0, s>>>(x, w->y64, w->p, w->z, op->mesh->d_dirichlet,
                                                   op->N, w->n);
  FEM_CHECK_LAUNCH();
  if (!w->exec || w->g_b != b || w->g_x != x) {
    FEM_CUDA_TRY(cudaStreamSynchronize(s));
    rc = build_graph(op, b, x);
    if (rc) return rc;
  }
  RefineScalars out = {};
  int steps = 0;
  for (;;) {
    FEM_CUDA_TRY(cudaGraphLaunch(w->exec, s));
    FEM_CUDA_TRY(cudaMemcpyAsync(&out, w->sc, sizeof(out), cudaMemcpyDeviceToHost, s));
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
    st->fallback = 0;
  }
  return status;
}

void fem_refine_free(fem_op *op) {
  RefineWork *w = op->ir;
  if (!w) return;
  destroy_graph(w);
  if (w->cap) cudaStreamDestroy(w->cap);
  if (w->cap2) cudaStreamDestroy(w->cap2);
  cudaFree(w->y64); cudaFree(w->r); cudaFree(w->z); cudaFree(w->p); cudaFree(w->y);
  cudaFree(w->d); cudaFree(w->dinv); cudaFree(w->sc); cudaFree(w->partials); cudaFree(w->counter);
  delete w;
  op->ir = nullptr;
}
