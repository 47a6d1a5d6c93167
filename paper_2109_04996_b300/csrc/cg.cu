// Preconditioned conjugate gradients on the Dirichlet-constrained bake-off
// systems (section "Benchmarks": CG iterations with their global reductions;
// diagonal preconditioner as in Nekbone, section "Miniapps").
//
// Per iteration three kernels, all scalars resident on the device:
//   apply      y = A p, with p^T A p summed in the same kernel (the element
//              contributions p_e^T A_e p_e add up to p^T A p);
//   update     alpha = rz / pAp; x += alpha p; r -= alpha y (interior only);
//              z = r / diag (Jacobi) or z = r; r^T z and ||r||^2 by a
//              deterministic grid reduction whose last block forms beta,
//              counts the iteration and decides convergence;
//   direction  p = z + beta p; y = 0 (ready for the next atomic apply).
// With use_graph the loop is one CUDA graph: a conditional WHILE node whose
// flag the update kernel's last block clears, so the host never sees a
// scalar until the solve ends (the paper's Laghos note: one dot product per
// iteration brought back to the CPU; here none is).
#include <math.h>
#include <string.h>

#include "fem_internal.h"

struct CgWork {
  int64_t n = 0;
  double *r = nullptr, *z = nullptr, *p = nullptr, *y = nullptr, *dinv = nullptr;
  CgScalars *sc = nullptr;
  double *partials = nullptr;
  unsigned *counter = nullptr;
  int dinv_pc = -1;          // preconditioner dinv currently holds
  cudaStream_t cap = nullptr, cap2 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const double *g_b = nullptr;
  double *g_x = nullptr;
  int g_zero = 0;                 // the graph's prologue starts from x = 0
};

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 4;   // CG iterations per pass of the graph's WHILE body

int grid_for(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  if (g > 148 * 8) g = 148 * 8;
  if (g < 1) g = 1;
  return (int)g;
}

__global__ void cg_dinv_kernel(const double *diag, const uint8_t *dir, int64_t N, int64_t n,
                               int pc, double *dinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = fem_node_of(i, N);
    const bool fixed = dir && dir[node];
    dinv[i] = fixed ? 0.0 : (pc == FEM_PC_JACOBI ? 1.0 / diag[node] : 1.0);
  }
}

// x <- M x (Dirichlet entries to 0; every entry with zero = 1), y <- 0
__global__ void cg_prepare_kernel(double *x, double *y, const uint8_t *dir, int64_t N,
                                  int64_t n, int zero) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (zero || (dir && dir[fem_node_of(i, N)])) x[i] = 0.0;
    y[i] = 0.0;
  }
}

struct CgParams {
  const double *b;
  double *x, *r, *z, *p, *y;
  const double *dinv;
  const uint8_t *dir;
  int64_t N, n;
  CgScalars *sc;
  double *partials;
  unsigned *counter;
  cudaGraphConditionalHandle handle;
  int use_graph;
};

__device__ void cg_set_continue(const CgParams &c, int cont) {
  if (c.use_graph) cudaGraphSetConditional(c.handle, cont ? 1u : 0u);
}

// r = M (b - A x0); z = dinv r; p = z; y = 0; rz, rr, bb.
__global__ void cg_init_kernel(const CgParams c) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool fixed = c.dir && c.dir[fem_node_of(i, c.N)];
    const double bi = fixed ? 0.0 : c.b[i];
    const double ri = fixed ? 0.0 : bi - c.y[i];
    const double zi = c.dinv[i] * ri;
    c.r[i] = ri; c.z[i] = zi; c.p[i] = zi; c.y[i] = 0.0;
    v[0] += ri * zi; v[1] += ri * ri; v[2] += bi * bi;
  }
  __shared__ double tot[3];
  if (fem_grid_sum<3>(v, c.partials, c.counter, tot) && threadIdx.x == 0) {
    CgScalars *s = c.sc;
    s->rz = tot[0]; s->rr = tot[1]; s->bb = tot[2];
    s->tol2 = s->tol2 * tot[2];  // host stored rtol^2
    s->iter = 0; s->pAp = 0.0; s->alpha = 0.0; s->beta = 0.0;
    s->status = FEM_OK;
    int done = 0;
    if (!(tot[2] > 0.0)) done = 1;                       // b = 0: x = x0 (= 0 interior)
    else if (s->tol2 > 0.0 && tot[1] <= s->tol2) done = 1;
    else if (s->maxit <= 0) { done = 1; if (s->tol2 > 0.0) s->status = FEM_ENOCONV; }
    if (!isfinite(tot[0]) || !isfinite(tot[1])) { done = 1; s->status = FEM_EBREAKDOWN; }
    s->done = done;
    cg_set_continue(c, !done);
  }
}

__global__ void cg_update_kernel(const CgParams c) {
  CgScalars *s = c.sc;
  if (s->done) return;  // host-driven loop ran past convergence
  const double pAp = s->pAp;
  const double alpha = s->rz / pAp;
  const bool ok = (pAp > 0.0) && isfinite(alpha);
  double v[2] = {0.0, 0.0};
  if (ok) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n;
         i += (int64_t)gridDim.x * blockDim.x) {
      const double di = c.dinv[i];
      const bool fixed = c.dir && c.dir[fem_node_of(i, c.N)];
      double ri = c.r[i];
      c.x[i] += alpha * c.p[i];
      if (!fixed) ri -= alpha * c.y[i];
      c.r[i] = ri;
      const double zi = di * ri;
      c.z[i] = zi;
      v[0] += ri * zi; v[1] += ri * ri;
    }
  }
  __shared__ double tot[2];
  if (fem_grid_sum<2>(v, c.partials, c.counter, tot) && threadIdx.x == 0) {
    int done = 0;
    if (!ok) {
      s->status = FEM_EBREAKDOWN; done = 1;
    } else {
      s->alpha = alpha;
      s->beta = tot[0] / s->rz;
      s->rz = tot[0]; s->rr = tot[1];
      s->iter += 1;
      if (!isfinite(tot[0]) || !isfinite(tot[1])) { s->status = FEM_EBREAKDOWN; done = 1; }
      else if (s->tol2 > 0.0 && tot[1] <= s->tol2) done = 1;
      else if (s->iter >= s->maxit) { done = 1; if (s->tol2 > 0.0) s->status = FEM_ENOCONV; }
    }
    s->done = done;
    cg_set_continue(c, !done);
  }
}

__global__ void cg_direction_kernel(const CgParams c) {
  const double beta = c.sc->beta;
  if (c.sc->done) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    c.p[i] = c.z[i] + beta * c.p[i];
    c.y[i] = 0.0;
  }
}

int ensure_work(fem_op *op) {
  if (op->cg) return FEM_OK;
  CgWork *w = new CgWork();
  op->cg = w;
  w->n = op->N * op->ncomp;
  const size_t vb = sizeof(double) * (size_t)w->n;
  if (cudaMalloc(&w->r, vb) != cudaSuccess || cudaMalloc(&w->z, vb) != cudaSuccess ||
      cudaMalloc(&w->p, vb) != cudaSuccess || cudaMalloc(&w->y, vb) != cudaSuccess ||
      cudaMalloc(&w->dinv, vb) != cudaSuccess || cudaMalloc(&w->sc, sizeof(CgScalars)) != cudaSuccess ||
      cudaMalloc(&w->partials, sizeof(double) * 4 * FEM_MAX_BLOCKS) != cudaSuccess ||
      cudaMalloc(&w->counter, sizeof(unsigned) * 4) != cudaSuccess) {
    cudaGetLastError();
    fem_set_error("fem_cg_solve: device allocation of the CG workspace failed");
    return FEM_ENOMEM;
  }
  FEM_CUDA_TRY(cudaMemsetAsync(w->counter, 0, sizeof(unsigned) * 4, op->stream()));
  op->bytes += 5 * vb;
  return FEM_OK;
}

CgParams make_params(fem_op *op, const double *b, double *x, cudaGraphConditionalHandle h,
                     int use_graph) {
  CgWork *w = op->cg;
  CgParams c;
  c.b = b; c.x = x; c.r = w->r; c.z = w->z; c.p = w->p; c.y = w->y; c.dinv = w->dinv;
  c.dir = op->mesh->d_dirichlet; c.N = op->N; c.n = w->n; c.sc = w->sc;
  c.partials = w->partials; c.counter = w->counter; c.handle = h; c.use_graph = use_graph;
  return c;
}

// The launches of one solve before the loop.  zero_guess: x = 0, so A x = 0
// (y stays zero) and no apply is needed for the initial residual.
int launch_prologue(fem_op *op, const CgParams &c, cudaStream_t s, int zero_guess = 0) {
  const int g = grid_for(c.n);
  cg_prepare_kernel<<<g, kThreads, 0, s>>>(c.x, c.y, c.dir, c.N, c.n, zero_guess);
  FEM_CHECK_LAUNCH();
  if (!zero_guess) {
    // the apply launcher uses the operator's stream; route it to s
    int rc = fem_launch_apply_f64(op, c.x, c.y, nullptr, op->E, nullptr);
    if (rc) return rc;
  }
  cg_init_kernel<<<g, kThreads, 0, s>>>(c);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

int launch_body(fem_op *op, const CgParams &c, cudaStream_t s) {
  const int g = grid_for(c.n);
  // the apply does nothing once the solve is done (unrolled graph bodies)
  int rc = fem_launch_apply_f64(op, c.p, c.y, nullptr, op->E, &c.sc->pAp, &c.sc->done);
  if (rc) return rc;
  cg_update_kernel<<<g, kThreads, 0, s>>>(c);
  FEM_CHECK_LAUNCH();
  cg_direction_kernel<<<g, kThreads, 0, s>>>(c);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

void destroy_graph(CgWork *w) {
  if (w->exec) cudaGraphExecDestroy(w->exec);
  if (w->graph) cudaGraphDestroy(w->graph);
  w->exec = nullptr; w->graph = nullptr;
}

}  // namespace

// Streams used while capturing: the apply launcher enqueues on
// op->stream(), so capture happens on the operator's own stream (mesh stream
// swapped for the duration of the capture).
static int build_graph(fem_op *op, const double *b, double *x, int zero_guess) {
  CgWork *w = op->cg;
  destroy_graph(w);
  fem_mesh *mesh = const_cast<fem_mesh *>(op->mesh);
  cudaStream_t user = mesh->stream;
  if (!w->cap) {
    FEM_CUDA_TRY(cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking));
    FEM_CUDA_TRY(cudaStreamCreateWithFlags(&w->cap2, cudaStreamNonBlocking));
  }
  int rc = FEM_OK;
  cudaGraph_t graph = nullptr;
  mesh->stream = w->cap;
  FEM_CUDA_TRY(cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeRelaxed));
  {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaGraphConditionalHandle h = 0;
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t cnode;
    cudaGraph_t body;
    CgParams c;
    cudaError_t e = cudaStreamGetCaptureInfo(w->cap, &st, nullptr, &graph, nullptr, nullptr, nullptr);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { rc = FEM_ECUDA; goto end_capture; }
    c = make_params(op, b, x, h, 1);
    rc = launch_prologue(op, c, w->cap, zero_guess);
    if (rc) goto end_capture;
    e = cudaStreamGetCaptureInfo(w->cap, &st, nullptr, &graph, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) { rc = FEM_ECUDA; goto end_capture; }
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&cnode, graph, deps, nullptr, ndeps, &cp);
    if (e != cudaSuccess) { rc = FEM_ECUDA; goto end_capture; }
    body = cp.conditional.phGraph_out[0];
    e = cudaStreamUpdateCaptureDependencies(w->cap, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) { rc = FEM_ECUDA; goto end_capture; }
    mesh->stream = w->cap2;
    e = cudaStreamBeginCaptureToGraph(w->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { rc = FEM_ECUDA; goto end_capture; }
    // kUnroll iterations per pass of the WHILE body: the conditional node's
    // per-pass cost is paid once per kUnroll iterations; iterations after
    // convergence within a pass do nothing (their kernels test `done`)
    for (int u = 0; u < kUnroll && !rc; u++) rc = launch_body(op, c, w->cap2);
    {
      cudaGraph_t tmp;
      cudaError_t e2 = cudaStreamEndCapture(w->cap2, &tmp);
      if (!rc && e2 != cudaSuccess) rc = FEM_ECUDA;
    }
    mesh->stream = w->cap;
  }
end_capture : {
  cudaGraph_t g2 = nullptr;
  cudaError_t e = cudaStreamEndCapture(w->cap, &g2);
  mesh->stream = user;
  if (rc == FEM_OK && e != cudaSuccess) rc = FEM_ECUDA;
  if (rc != FEM_OK) {
    if (g2) cudaGraphDestroy(g2);
    cudaGetLastError();
    if (rc == FEM_ECUDA) fem_set_error("fem_cg_solve: building the CUDA graph failed: %s", cudaGetErrorString(e));
    return rc;
  }
  w->graph = g2;
}
  FEM_CUDA_TRY(cudaGraphInstantiate(&w->exec, w->graph, 0));
  w->g_b = b; w->g_x = x; w->g_zero = zero_guess;
  return FEM_OK;
}

int fem_cg_run(fem_op *op, const double *b, double *x, const fem_cg_opts *o,
               fem_cg_stats *st) {
  int rc = ensure_work(op);
  if (rc) return rc;
  CgWork *w = op->cg;
  cudaStream_t s = op->stream();
  if (w->dinv_pc != o->precond) {
    cg_dinv_kernel<<<grid_for(w->n), kThreads, 0, s>>>(op->d_diag, op->mesh->d_dirichlet, op->N,
                                                       w->n, o->precond, w->dinv);
    FEM_CHECK_LAUNCH();
    w->dinv_pc = o->precond;
  }
  CgScalars init = {};
  init.maxit = o->maxit;
  init.tol2 = o->rtol * o->rtol;
  FEM_CUDA_TRY(cudaMemcpyAsync(w->sc, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  if (o->use_graph) {
    const int zero = o->zero_guess ? 1 : 0;
    if (!w->exec || w->g_b != b || w->g_x != x || w->g_zero != zero) {
      // the capture streams must see the work queued so far on s
      FEM_CUDA_TRY(cudaStreamSynchronize(s));
      rc = build_graph(op, b, x, zero);
      if (rc) return rc;
    }
    FEM_CUDA_TRY(cudaGraphLaunch(w->exec, s));
  } else {
    CgParams c = make_params(op, b, x, 0, 0);
    rc = launch_prologue(op, c, s, o->zero_guess ? 1 : 0);
    if (rc) return rc;
    for (int it = 0; it < o->maxit; it++) {
      rc = launch_body(op, c, s);
      if (rc) return rc;
      if ((it & 7) == 7 || it == o->maxit - 1) {
        int done = 0;
        FEM_CUDA_TRY(cudaMemcpyAsync(&done, &w->sc->done, sizeof(int), cudaMemcpyDeviceToHost, s));
        FEM_CUDA_TRY(cudaStreamSynchronize(s));
        if (done) break;
      }
    }
  }
  CgScalars out;
  FEM_CUDA_TRY(cudaMemcpyAsync(&out, w->sc, sizeof(out), cudaMemcpyDeviceToHost, s));
  FEM_CUDA_TRY(cudaStreamSynchronize(s));
  if (st) {
    st->iterations = out.iter;
    st->outer = 0;
    st->status = out.status;
    st->rnorm = sqrt(out.rr);
    st->bnorm = sqrt(out.bb);
    st->true_rel = -1.0;
    st->fallback = 0;
  }
  return out.status;
}

// ---------------------------------------------------------------------------
// Checkpoint / restore / resume of an interrupted CG solve.  A solve that
// stopped at its iteration cap leaves, in the operator's workspace, the
// iterate's residual r_k, z_k = M^-1 r_k, the previous direction p_{k-1} and
// the scalars (r^T z, beta_k, ||b||^2, the iteration count): everything CG
// needs besides x_k, which is the caller's.  Resuming forms p_k = z_k +
// beta_k p_{k-1} and continues with the same kernels, so the resumed solve
// is the uninterrupted one up to the order of the apply's atomic additions.

namespace {
struct CgCheckpointHeader {
  char tag[8];      // "FEMCGCK1"
  int64_t n;        // ncomp * N
  int32_t pc;       // preconditioner of the interrupted solve
  int32_t pad;
};
const char kCgTag[8] = {'F', 'E', 'M', 'C', 'G', 'C', 'K', '1'};

__global__ void cg_resume_direction_kernel(const CgParams c) {
  const double beta = c.sc->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    c.p[i] = c.z[i] + beta * c.p[i];
    c.y[i] = 0.0;
  }
}
}  // namespace

int64_t fem_cg_checkpoint_bytes(const fem_op *op) {
  return (int64_t)sizeof(CgCheckpointHeader) + (int64_t)sizeof(CgScalars) +
         3 * (int64_t)sizeof(double) * op->N * op->ncomp;
}

int fem_cg_checkpoint_save(fem_op *op, void *host) {
  CgWork *w = op->cg;
  if (!w || w->dinv_pc < 0) {
    fem_set_error("fem_cg_checkpoint: the operator has run no CG solve");
    return FEM_EINVAL;
  }
  cudaStream_t s = op->stream();
  CgCheckpointHeader h;
  memcpy(h.tag, kCgTag, 8);
  h.n = w->n; h.pc = w->dinv_pc; h.pad = 0;
  char *out = (char *)host;
  memcpy(out, &h, sizeof(h));
  char *q = out + sizeof(h);
  FEM_CUDA_TRY(cudaMemcpyAsync(q, w->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
  q += sizeof(CgScalars);
  const size_t vb = sizeof(double) * (size_t)w->n;
  FEM_CUDA_TRY(cudaMemcpyAsync(q, w->r, vb, cudaMemcpyDeviceToHost, s));
  FEM_CUDA_TRY(cudaMemcpyAsync(q + vb, w->z, vb, cudaMemcpyDeviceToHost, s));
  FEM_CUDA_TRY(cudaMemcpyAsync(q + 2 * vb, w->p, vb, cudaMemcpyDeviceToHost, s));
  FEM_CUDA_TRY(cudaStreamSynchronize(s));
  return FEM_OK;
}

int fem_cg_checkpoint_restore(fem_op *op, const void *host) {
  CgCheckpointHeader h;
  memcpy(&h, host, sizeof(h));
  if (memcmp(h.tag, kCgTag, 8) != 0 || h.n != op->N * op->ncomp ||
      (h.pc != FEM_PC_NONE && h.pc != FEM_PC_JACOBI)) {
    fem_set_error("fem_cg_restore: not a checkpoint of a CG solve on an operator of this size");
    return FEM_EINVAL;
  }
  int rc = ensure_work(op);
  if (rc) return rc;
  CgWork *w = op->cg;
  cudaStream_t s = op->stream();
  const char *q = (const char *)host + sizeof(h);
  FEM_CUDA_TRY(cudaMemcpyAsync(w->sc, q, sizeof(CgScalars), cudaMemcpyHostToDevice, s));
  q += sizeof(CgScalars);
  const size_t vb = sizeof(double) * (size_t)w->n;
  FEM_CUDA_TRY(cudaMemcpyAsync(w->r, q, vb, cudaMemcpyHostToDevice, s));
  FEM_CUDA_TRY(cudaMemcpyAsync(w->z, q + vb, vb, cudaMemcpyHostToDevice, s));
  FEM_CUDA_TRY(cudaMemcpyAsync(w->p, q + 2 * vb, vb, cudaMemcpyHostToDevice, s));
  cg_dinv_kernel<<<grid_for(w->n), kThreads, 0, s>>>(op->d_diag, op->mesh->d_dirichlet, op->N,
                                                     w->n, h.pc, w->dinv);
  FEM_CHECK_LAUNCH();
  w->dinv_pc = h.pc;
  FEM_CUDA_TRY(cudaStreamSynchronize(s));
  return FEM_OK;
}

int fem_cg_resume_run(fem_op *op, const double *b, double *x, const fem_cg_opts *o,
                      fem_cg_stats *st) {
  CgWork *w = op->cg;
  if (!w || w->dinv_pc < 0) {
    fem_set_error("fem_cg_resume: no interrupted CG solve on this operator (run or restore one)");
    return FEM_EINVAL;
  }
  if (o->precond != w->dinv_pc) {
    fem_set_error("fem_cg_resume: preconditioner %d differs from the interrupted solve's %d",
                  o->precond, w->dinv_pc);
    return FEM_EINVAL;
  }
  cudaStream_t s = op->stream();
  CgScalars sc;
  FEM_CUDA_TRY(cudaMemcpyAsync(&sc, w->sc, sizeof(sc), cudaMemcpyDeviceToHost, s));
  FEM_CUDA_TRY(cudaStreamSynchronize(s));
  const bool capped = sc.done && sc.iter >= sc.maxit &&
                      (sc.status == FEM_ENOCONV || (sc.status == FEM_OK && !(sc.tol2 > 0.0)));
  if (!capped) {
    fem_set_error("fem_cg_resume: the last solve did not stop at its iteration cap "
                  "(status %d, %d of %d iterations)", sc.status, sc.iter, sc.maxit);
    return FEM_EINVAL;
  }
  sc.maxit = sc.iter + o->maxit;
  sc.tol2 = o->rtol * o->rtol * sc.bb;
  sc.status = FEM_OK;
  sc.done = 0;
  if (sc.tol2 > 0.0 && sc.rr <= sc.tol2) sc.done = 1;   // already converged to the new rtol
  if (o->maxit == 0) sc.done = 1;
  FEM_CUDA_TRY(cudaMemcpyAsync(w->sc, &sc, sizeof(sc), cudaMemcpyHostToDevice, s));
  CgParams c = make_params(op, b, x, 0, 0);
  if (!sc.done) {
    cg_resume_direction_kernel<<<grid_for(c.n), kThreads, 0, s>>>(c);
    FEM_CHECK_LAUNCH();
    for (int it = 0; it < o->maxit; it++) {
      int rc = launch_body(op, c, s);
      if (rc) return rc;
      if ((it & 7) == 7 || it == o->maxit - 1) {
        int done = 0;
        FEM_CUDA_TRY(cudaMemcpyAsync(&done, &w->sc->done, sizeof(int), cudaMemcpyDeviceToHost, s));
        FEM_CUDA_TRY(cudaStreamSynchronize(s));
        if (done) break;
      }
    }
  }
  CgScalars out;
  FEM_CUDA_TRY(cudaMemcpyAsync(&out, w->sc, sizeof(out), cudaMemcpyDeviceToHost, s));
  FEM_CUDA_TRY(cudaStreamSynchronize(s));
  if (!sc.done && out.status == FEM_OK && out.iter >= out.maxit && out.tol2 > 0.0 && out.rr > out.tol2)
    out.status = FEM_ENOCONV;
  if (st) {
    st->iterations = out.iter;
    st->outer = 0;
    st->status = out.status;
    st->rnorm = sqrt(out.rr);
    st->bnorm = sqrt(out.bb);
    st->true_rel = -1.0;
    st->fallback = 0;
  }
  return out.status;
}

void fem_cg_free(fem_op *op) {
  CgWork *w = op->cg;
  if (!w) return;
  destroy_graph(w);
  if (w->cap) cudaStreamDestroy(w->cap);
  if (w->cap2) cudaStreamDestroy(w->cap2);
  cudaFree(w->r); cudaFree(w->z); cudaFree(w->p); cudaFree(w->y); cudaFree(w->dinv);
  cudaFree(w->sc); cudaFree(w->partials); cudaFree(w->counter);
  delete w;
  op->cg = nullptr;
}

// ---------------------------------------------------------------------------
// fem_cg_solve_noalloc: the same Jacobi/plain CG as fem_cg_solve, for callers
// that must not allocate device memory while solving (a fixed memory budget
// handed out once at start-up, a real-time loop where cudaMalloc's implicit
// device-wide synchronization is not acceptable).  Its workspace is one
// file-scope device array of fixed size instead of cudaMalloc'd buffers.
//
// Layout of the array: 5 vectors r, z, p, y, dinv of FEM_NOALLOC_MAX_N
// doubles each, the grid-reduction partials, the CG scalars and the ticket
// counters.  Every GPU that loads the library holds it until the process
// exits.  All calls share it and it keeps the last call's contents; each call
// rewrites every part it reads before reading it.  Calls that overlap on the
// GPU (two streams, two host threads) race on it.
namespace {

constexpr size_t kNaVec = (size_t)FEM_NOALLOC_MAX_N * sizeof(double);
constexpr size_t kNaPart = (size_t)4 * FEM_MAX_BLOCKS * sizeof(double);
constexpr size_t kNaScal = ((sizeof(CgScalars) + 255) / 256) * 256;
constexpr size_t kNaBytes = 5 * kNaVec + kNaPart + kNaScal + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kMaxDevices = 64;
unsigned char *g_noalloc_base[kMaxDevices] = {nullptr};

// Device address of the array on the current device, looked up once per
// device (host code cannot use the symbol's name as a device address).
int noalloc_base(unsigned char **out) {
  int dev = 0;
  FEM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    fem_set_error("fem_cg_solve_noalloc: device %d beyond the %d supported", dev, kMaxDevices);
    return FEM_EINVAL;
  }
  if (!g_noalloc_base[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      fem_set_error("fem_cg_solve_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return FEM_ECUDA;
    }
    g_noalloc_base[dev] = (unsigned char *)p;
  }
  *out = g_noalloc_base[dev];
  return FEM_OK;
}

__global__ void cg_noalloc_reset_kernel(CgScalars *sc, unsigned *counter, int maxit, double tol2) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    CgScalars s = {};
    s.maxit = maxit;
    s.tol2 = tol2;
    *sc = s;
    for (int i = 0; i < 4; i++) counter[i] = 0u;
  }
}

}  // namespace

extern "C" fem_status fem_cg_solve_noalloc(fem_op *op, const double *b, double *x,
                                           const fem_cg_opts *o, fem_cg_stats *st) {
  if (!op || !b || !x || !o || b == x) {
    fem_set_error("fem_cg_solve_noalloc: invalid arguments");
    return FEM_EINVAL;
  }
  if (o->precond != FEM_PC_NONE && o->precond != FEM_PC_JACOBI) {
    fem_set_error("fem_cg_solve_noalloc: preconditioner %d not available", o->precond);
    return FEM_EINVAL;
  }
  if (o->maxit < 0 || !(o->rtol >= 0.0)) {
    fem_set_error("fem_cg_solve_noalloc: bad maxit/rtol");
    return FEM_EINVAL;
  }
  const int64_t n = op->N * op->ncomp;
  if (n > FEM_NOALLOC_MAX_N) {
    fem_set_error("fem_cg_solve_noalloc: ncomp*N = %lld exceeds the fixed workspace of %d entries",
                  (long long)n, FEM_NOALLOC_MAX_N);
    return FEM_EINVAL;
  }
  unsigned char *base = nullptr;
  int rc = noalloc_base(&base);
  if (rc) return rc;
  double *vec = (double *)base;
  double *partials = (double *)(base + 5 * kNaVec);
  CgScalars *sc = (CgScalars *)(base + 5 * kNaVec + kNaPart);
  unsigned *counter = (unsigned *)(base + 5 * kNaVec + kNaPart + kNaScal);
  cudaStream_t s = op->stream();
  cg_noalloc_reset_kernel<<<1, 32, 0, s>>>(sc, counter, o->maxit, o->rtol * o->rtol);
  FEM_CHECK_LAUNCH();
  CgParams c;
  c.b = b; c.x = x;
  c.r = vec; c.z = vec + FEM_NOALLOC_MAX_N; c.p = vec + 2 * (size_t)FEM_NOALLOC_MAX_N;
  c.y = vec + 3 * (size_t)FEM_NOALLOC_MAX_N;
  double *dinv = vec + 4 * (size_t)FEM_NOALLOC_MAX_N;
  c.dinv = dinv;
  c.dir = op->mesh->d_dirichlet; c.N = op->N; c.n = n; c.sc = sc;
  c.partials = partials; c.counter = counter; c.handle = 0; c.use_graph = 0;
  cg_dinv_kernel<<<grid_for(n), kThreads, 0, s>>>(op->d_diag, op->mesh->d_dirichlet, op->N, n,
                                                  o->precond, dinv);
  FEM_CHECK_LAUNCH();
  rc = launch_prologue(op, c, s, o->zero_guess ? 1 : 0);
  if (rc) return rc;
  for (int it = 0; it < o->maxit; it++) {
    rc = launch_body(op, c, s);
    if (rc) return rc;
    if ((it & 7) == 7 || it == o->maxit - 1) {
      int done = 0;
      FEM_CUDA_TRY(cudaMemcpyAsync(&done, &sc->done, sizeof(int), cudaMemcpyDeviceToHost, s));
      FEM_CUDA_TRY(cudaStreamSynchronize(s));
      if (done) break;
    }
  }
  CgScalars out;
  FEM_CUDA_TRY(cudaMemcpyAsync(&out, sc, sizeof(out), cudaMemcpyDeviceToHost, s));
  FEM_CUDA_TRY(cudaStreamSynchronize(s));
  if (st) {
    st->iterations = out.iter;
    st->outer = 0;
    st->status = out.status;
    st->rnorm = sqrt(out.rr);
    st->bnorm = sqrt(out.bb);
    st->true_rel = -1.0;
    st->fallback = 0;
  }
  return out.status;
}
