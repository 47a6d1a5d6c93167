// Jacobi-PCG on an element-partitioned system (the paper's parallel form,
// sections "libCEED" and "Nek and MFEM": A = P^T G^T B^T D B G P with P the
// subdomain restriction; P^T is the interface sum over the ranks that share
// a node -- gslib's gather-scatter -- and CG's dot products are global sums).
//
// Each rank calls fem_pcg_dist with its own operator on its local mesh; the
// library runs the applies and every vector operation in its kernels, and
// hands two steps to the caller through host callbacks: the interface sum of
// a local vector and the sum over ranks of a few host scalars.  Per
// iteration: one apply, one interface sum, two all-reduces (p^T A p, then
// r^T z and ||r||^2 together).  The callbacks run on the calling thread
// between kernel launches (the stream is synchronized before each), so no
// kernel ever waits on another rank.
#include <math.h>

#include "fem_internal.h"

namespace {

constexpr int kT = 256;

int grid_n(int64_t n) {
  int64_t g = (n + kT - 1) / kT;
  if (g > 148 * 8) g = 148 * 8;
  if (g < 1) g = 1;
  return (int)g;
}

struct DistVecs {
  const double *b;
  double *x, *r, *z, *p, *y, *dinv;
  const uint8_t *dir, *owned;
  int64_t N, n;
  double *partials;
  unsigned *counter;
  double *out;      // device scalars of the last reduction
};

// dinv = 1 / diag on interior entries (diag assembled by the caller's
// interface sum; diag = NULL: 1, plain CG), 0 on Dirichlet entries
__global__ void dist_dinv_kernel(const double *diag, const uint8_t *dir, int64_t N, int64_t n,
                                 double *dinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = fem_node_of(i, N);
    dinv[i] = (dir && dir[node]) ? 0.0 : (diag ? 1.0 / diag[node] : 1.0);
  }
}

// x <- M x (zero_guess: x <- 0), y <- 0
__global__ void dist_prepare_kernel(double *x, double *y, const uint8_t *dir, int64_t N,
                                    int64_t n, int zero) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (zero || (dir && dir[fem_node_of(i, N)])) x[i] = 0.0;
    y[i] = 0.0;
  }
}

// r = M (b - y), z = dinv r, p = z, y = 0; owned sums r.z, r.r, b.b
__global__ void dist_init_kernel(const DistVecs v) {
  double s[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < v.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = fem_node_of(i, v.N);
    const bool fixed = v.dir && v.dir[node];
    const double bi = fixed ? 0.0 : v.b[i];
    const double ri = fixed ? 0.0 : bi - v.y[i];
    const double zi = v.dinv[i] * ri;
    v.r[i] = ri; v.z[i] = zi; v.p[i] = zi; v.y[i] = 0.0;
    if (v.owned[node]) { s[0] += ri * zi; s[1] += ri * ri; s[2] += bi * bi; }
  }
  __shared__ double tot[3];
  if (fem_grid_sum<3>(s, v.partials, v.counter, tot) && threadIdx.x == 0)
    for (int k = 0; k < 3; k++) v.out[k] = tot[k];
}

// owned sum of p.y (y = the assembled A p)
__global__ void dist_pap_kernel(const DistVecs v) {
  double s[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < v.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = fem_node_of(i, v.N);
    const bool fixed = v.dir && v.dir[node];
    if (v.owned[node] && !fixed) s[0] += v.p[i] * v.y[i];
  }
  __shared__ double tot[1];
  if (fem_grid_sum<1>(s, v.partials, v.counter, tot) && threadIdx.x == 0) v.out[0] = tot[0];
}

// x += alpha p; r -= alpha y (interior); z = dinv r; owned sums r.z, r.r
__global__ void dist_update_kernel(const DistVecs v, double alpha) {
  double s[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < v.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = fem_node_of(i, v.N);
    const bool fixed = v.dir && v.dir[node];
    double ri = v.r[i];
    v.x[i] += alpha * v.p[i];
    if (!fixed) ri -= alpha * v.y[i];
    v.r[i] = ri;
    const double zi = v.dinv[i] * ri;
    v.z[i] = zi;
    if (v.owned[node]) { s[0] += ri * zi; s[1] += ri * ri; }
  }
  __shared__ double tot[2];
  if (fem_grid_sum<2>(s, v.partials, v.counter, tot) && threadIdx.x == 0) {
    v.out[0] = tot[0];
    v.out[1] = tot[1];
  }
}

// p = z + beta p; y = 0
__global__ void dist_direction_kernel(const DistVecs v, double beta) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < v.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    v.p[i] = v.z[i] + beta * v.p[i];
    v.y[i] = 0.0;
  }
}

}  // namespace

// Device scalars of the last reduction to host, summed over the ranks.
static int reduce_scalars(cudaStream_t s, const DistVecs &v, int count, const fem_comm *comm,
                          double *out) {
  FEM_CUDA_TRY(cudaMemcpyAsync(out, v.out, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
  FEM_CUDA_TRY(cudaStreamSynchronize(s));
  if (comm->allreduce(comm->ctx, out, count) != 0) {
    fem_set_error("fem_pcg_dist: the all-reduce callback failed");
    return FEM_EINVAL;
  }
  return FEM_OK;
}

// y = A p: local element operator, then the caller's interface sum.
static int apply_assembled(fem_op *op, const double *p, double *y, const fem_comm *comm) {
  cudaStream_t s = op->stream();
  int rc = fem_launch_apply_f64(op, p, y, nullptr, op->E, nullptr);
  if (rc) return rc;
  FEM_CUDA_TRY(cudaStreamSynchronize(s));
  if (comm->sum_interfaces(comm->ctx, y) != 0) {
    fem_set_error("fem_pcg_dist: the interface-sum callback failed");
    return FEM_EINVAL;
  }
  return FEM_OK;
}

extern "C" fem_status fem_pcg_dist(fem_op *op, const uint8_t *owned, const double *b, double *x,
                                   double *y, const fem_cg_opts *o, const fem_comm *comm,
                                   fem_cg_stats *st) {
  if (!op || !owned || !b || !x || !y || !o || !comm || !comm->sum_interfaces ||
      !comm->allreduce || b == x || y == x || y == b) {
    fem_set_error("fem_pcg_dist: invalid arguments");
    return FEM_EINVAL;
  }
  if (o->precond != FEM_PC_JACOBI && o->precond != FEM_PC_NONE) {
    fem_set_error("fem_pcg_dist: preconditioner %d not available", o->precond);
    return FEM_EINVAL;
  }
  if (o->maxit < 0 || !(o->rtol >= 0.0)) { fem_set_error("fem_pcg_dist: bad maxit/rtol"); return FEM_EINVAL; }
  const int64_t N = op->N, n = N * op->ncomp;
  cudaStream_t s = op->stream();
  // work vectors r, z, p, dinv, the reduction scratch and scalars
  double *buf = nullptr;
  double *partials = nullptr;
  unsigned *counter = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * (4 * (size_t)n + 4)) != cudaSuccess ||
      cudaMalloc(&partials, sizeof(double) * 4 * FEM_MAX_BLOCKS) != cudaSuccess ||
      cudaMalloc(&counter, sizeof(unsigned) * 4) != cudaSuccess) {
    cudaFree(buf); cudaFree(partials);
    cudaGetLastError();
    fem_set_error("fem_pcg_dist: allocation of the work vectors failed");
    return FEM_ENOMEM;
  }
  DistVecs v;
  v.b = b; v.x = x; v.y = y;
  v.r = buf; v.z = buf + n; v.p = buf + 2 * n; v.dinv = buf + 3 * n; v.out = buf + 4 * n;
  v.dir = op->mesh->d_dirichlet; v.owned = owned; v.N = N; v.n = n;
  v.partials = partials; v.counter = counter;
  int rc = FEM_OK;
  int iters = 0, status = FEM_OK;
  double h[3] = {0, 0, 0}, rz = 0, rr = 0, bb = 0;
  const int g = grid_n(n);
  auto fail = [&](int code) { rc = code; };
  do {
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned) * 4, s) != cudaSuccess) {
      fem_set_error("fem_pcg_dist: memset failed"); fail(FEM_ECUDA); break;
    }
    if (o->precond == FEM_PC_JACOBI) {
      // assembled diagonal: the local one summed over the interfaces (in y)
      if (cudaMemsetAsync(y, 0, sizeof(double) * n, s) != cudaSuccess ||
          cudaMemcpyAsync(y, op->d_diag, sizeof(double) * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        fem_set_error("fem_pcg_dist: copy of the diagonal failed"); fail(FEM_ECUDA); break;
      }
      if (comm->sum_interfaces(comm->ctx, y) != 0) {
        fem_set_error("fem_pcg_dist: the interface-sum callback failed"); fail(FEM_EINVAL); break;
      }
      dist_dinv_kernel<<<g, kT, 0, s>>>(y, v.dir, N, n, v.dinv);
    } else {
      dist_dinv_kernel<<<g, kT, 0, s>>>(nullptr, v.dir, N, n, v.dinv);
    }
    dist_prepare_kernel<<<g, kT, 0, s>>>(x, y, v.dir, N, n, o->zero_guess ? 1 : 0);
    if (cudaGetLastError() != cudaSuccess) { fem_set_error("fem_pcg_dist: launch failed"); fail(FEM_ECUDA); break; }
    if (!o->zero_guess && (rc = apply_assembled(op, x, y, comm))) break;
    dist_init_kernel<<<g, kT, 0, s>>>(v);
    if ((rc = reduce_scalars(s, v, 3, comm, h))) break;
    rz = h[0]; rr = h[1]; bb = h[2];
    const double tol2 = o->rtol * o->rtol * bb;
    if (!(bb > 0.0)) break;
    while (true) {
      if (tol2 > 0.0 && rr <= tol2) break;
      if (iters >= o->maxit) { if (tol2 > 0.0) status = FEM_ENOCONV; break; }
      if ((rc = apply_assembled(op, v.p, y, comm))) break;
      dist_pap_kernel<<<g, kT, 0, s>>>(v);
      double pap = 0.0;
      if ((rc = reduce_scalars(s, v, 1, comm, &pap))) break;
      const double alpha = rz / pap;
      if (!(pap > 0.0) || !isfinite(alpha)) { status = FEM_EBREAKDOWN; break; }
      dist_update_kernel<<<g, kT, 0, s>>>(v, alpha);
      if ((rc = reduce_scalars(s, v, 2, comm, h))) break;
      const double beta = h[0] / rz;
      rz = h[0]; rr = h[1];
      iters++;
      if (!isfinite(rz) || !isfinite(rr)) { status = FEM_EBREAKDOWN; break; }
      dist_direction_kernel<<<g, kT, 0, s>>>(v, beta);
    }
  } while (0);
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(buf); cudaFree(partials); cudaFree(counter);
  if (rc) return rc;
  if (e != cudaSuccess) { fem_set_error("fem_pcg_dist: %s", cudaGetErrorString(e)); return FEM_ECUDA; }
  if (st) {
    st->iterations = iters;
    st->outer = 0;
    st->status = status;
    st->rnorm = sqrt(rr);
    st->bnorm = sqrt(bb);
    st->true_rel = -1.0;
    st->fallback = 0;
  }
  return status;
}
