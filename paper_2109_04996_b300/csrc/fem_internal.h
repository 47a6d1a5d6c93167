// Internal declarations of the FEM library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/fem.h"
#include "dw.cuh"

#define FEM_MAX_P 9    // P = p + 1 <= 9
#define FEM_MAX_Q 10   // q <= p + 2 <= 10

// Thread-local error message, set by every failing entry point.
void fem_set_error(const char *fmt, ...);

#define FEM_CUDA_TRY(call)                                                   \
  do {                                                                       \
    cudaError_t err_ = (call);                                               \
    if (err_ != cudaSuccess) {                                               \
      fem_set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(err_), \
                    __FILE__, __LINE__);                                     \
      return FEM_ECUDA;                                                      \
    }                                                                        \
  } while (0)

#define FEM_CHECK_LAUNCH()                                                   \
  do {                                                                       \
    cudaError_t err_ = cudaGetLastError();                                   \
    if (err_ != cudaSuccess) {                                               \
      fem_set_error("kernel launch failed: %s (%s:%d)",                      \
                    cudaGetErrorString(err_), __FILE__, __LINE__);           \
      return FEM_ECUDA;                                                      \
    }                                                                        \
  } while (0)

// 1D tables of one operator, host FP64 (basis.cu).
struct BasisTables {
  int p, P, q, quad;
  double z[FEM_MAX_P];                    // Gauss-Lobatto nodes of the basis
  double r[FEM_MAX_Q], w[FEM_MAX_Q];      // quadrature points / weights
  double B[FEM_MAX_Q * FEM_MAX_P];        // l_a(r_k)          [k][a]
  double G[FEM_MAX_Q * FEM_MAX_P];        // l_a'(r_k)         [k][a]
  double Dq[FEM_MAX_Q * FEM_MAX_Q];       // derivative of the Lagrange basis
                                          // on the quadrature points, at them
};
int fem_build_tables(int p, int q, int quad, BasisTables *t);
// I[k][a] = l_a(x_k), Lagrange basis of order p on its Gauss-Lobatto nodes
int fem_basis_interp(int p, const double *x, int npts, double *I);

// Scalars of one CG run, resident on the device.
struct CgScalars {
  double rz;       // r^T z of the current iterate
  double rz_new;
  double pAp;      // fused into the apply
  double rr;       // ||r||^2
  double bb;       // ||b||^2 (constrained)
  double alpha, beta;
  double tol2;     // rtol^2 * bb
  int iter, maxit;
  int status;      // FEM_OK / FEM_ENOCONV / FEM_EBREAKDOWN
  int done;
};

struct fem_mesh {
  int p, P;
  int64_t N, E;
  int32_t *d_elem_nodes = nullptr;  // [E][P^3]
  double *d_xyz = nullptr;          // [3][N] (SoA)
  uint8_t *d_dirichlet = nullptr;   // [N], 1 = constrained
  cudaStream_t stream = nullptr;
  int64_t bytes = 0;
};

struct CgWork;
struct RefineWork;

struct fem_op {
  const fem_mesh *mesh = nullptr;
  int kind, quad, q, ncomp, prec;
  int P, Q;
  bool colloc;                    // Gauss-Lobatto with q = p+1: B = identity
  int64_t N, E;
  BasisTables tab;
  double *d_B = nullptr, *d_Dq = nullptr;   // device copies of B [Q][P], Dq [Q][Q]
  float *d_B32 = nullptr, *d_Dq32 = nullptr;
  double *d_qdata = nullptr;      // [E][nd][Q^3]
  float *d_qdata32 = nullptr;     // FP32 copy (prec == FEM_F32)
  dw *d_qdw = nullptr;            // double-word split (line-body choices 8..23), made
                                  // when one of them is first selected
  // trilinear Gauss diffusion only (P = 2), made when the trilinear body is
  // first selected (fem_ensure_qsum): line sums of the diagonal qdata
  // components, [E][3][Q^2]: sum over i of D00 at (j, k) (index j + Q k),
  // over j of D11 at (i, k) (i + Q k), over k of D22 at (i, j) (i + Q j)
  double *d_qsum = nullptr;
  float *d_qsum32 = nullptr;
  // Gauss diffusion at P = 2 and 3 only: the element matrices
  // K_e = sum_q grad phi_a^T D grad phi_b, upper triangle packed by rows
  // (a <= b), entry-major [P^3 (P^3 + 1) / 2][E]
  double *d_kel = nullptr;
  float *d_kel32 = nullptr;
  dw *d_keldw = nullptr;          // double-word split of d_kel (choice 11)
  // p = 1 Gauss diffusion on a lattice mesh (stencil.cu, choice 24): the
  // assembled 27-point stencil [27][N] in double words, the split input
  // [N], and the lattice size n (-1: not checked yet, 0: not a lattice)
  dw *d_stencil = nullptr;
  dw *d_xdw = nullptr;
  float *d_stencil32 = nullptr;   // the same in FP32 (FP32 operators)
  int64_t lattice_n = -1;
  double *d_diag = nullptr;       // [N] scalar diagonal
  double *d_rff = nullptr;        // [M][4]
  int M = 0;
  double sigma = 1.0;
  // reduction scratch for the fused dot products
  double *d_partials = nullptr;   // [FEM_MAX_BLOCKS * 4]
  unsigned *d_counter = nullptr;  // [4]
  int64_t bytes = 0;
  int nsm = 148;                  // SMs of the device the operator lives on
  int tune_epb[2] = {0, 0};       // launch shape of the apply per precision:
  int tune_bps[2] = {0, 0};       //   EPB choice index, blocks per SM (0 = max)
  CgWork *cg = nullptr;
  RefineWork *ir = nullptr;
  cudaStream_t stream() const { return mesh->stream; }
};

#define FEM_MAX_BLOCKS 8192

// Per-device facts of one kernel that are set up at its first launch on a
// device (the dynamic shared-memory attribute, the resident blocks per SM):
// both belong to the current device, not to the process.
constexpr int FEM_MAX_DEVICES = 64;
struct FemKernelCache {
  int v[FEM_MAX_DEVICES];
  FemKernelCache() { for (int &x : v) x = -1; }
  int &here() {
    int d = 0;
    cudaGetDevice(&d);
    return v[(d >= 0 && d < FEM_MAX_DEVICES) ? d : 0];
  }
};

// Device table block of an operator: B [Q][P] | Dq [Q][Q] | G [Q][P] | w [Q]
// at fixed offsets (FP64 and FP32 copies).
#define TAB_B 0
#define TAB_DQ (FEM_MAX_Q * FEM_MAX_P)
#define TAB_G (TAB_DQ + FEM_MAX_Q * FEM_MAX_Q)
#define TAB_W (TAB_G + FEM_MAX_Q * FEM_MAX_P)
#define TAB_SIZE (TAB_W + FEM_MAX_Q)

// Node of entry i of a component-major vector of N-node components: i mod N
// without the 64-bit division of `%` (tens of instructions per entry in the
// bandwidth-bound vector kernels).  Operators have at most 3 components.
__host__ __device__ __forceinline__ int64_t fem_node_of(int64_t i, int64_t N) {
  return i < N ? i : (i < 2 * N ? i - N : (i < 3 * N ? i - 2 * N : i % N));
}

// ---- launchers (apply.cu)
// skip: optional device flag; nonzero when the launch runs makes it a no-op
// (the loop body of a solve that has converged)
int fem_launch_apply_f64(fem_op *op, const double *x, double *y,
                         const int32_t *list, int64_t nsel, double *dot_out,
                         const int *skip = nullptr);
int fem_launch_apply_f32(fem_op *op, const float *x, float *y,
                         const int32_t *list, int64_t nsel, double *dot_out,
                         const int *skip = nullptr);
// explicit launch shape (autotuner): body / elements-per-block choice
// (fem_apply_choices), blocks per SM (0 = max)
int fem_launch_apply_f64_shape(fem_op *op, const double *x, double *y, const int32_t *list,
                               int64_t nsel, double *dot_out, int choice, int bps,
                               const int *skip = nullptr);
int fem_launch_apply_f32_shape(fem_op *op, const float *x, float *y, const int32_t *list,
                               int64_t nsel, double *dot_out, int choice, int bps,
                               const int *skip = nullptr);
// the double-word bodies (choices 8..23) of the FP64 apply (apply_dw.cu)
int fem_launch_apply_dw_shape(fem_op *op, const double *x, double *y, const int32_t *list,
                              int64_t nsel, double *dot_out, int choice, int bps,
                              const int *skip = nullptr);
// Launch shape choices of an operator's apply: 0..2 the line-based body
// (elements per block default, half, double), 3..5 the slab body, 6 the
// trilinear body (Gauss diffusion at p = 1; at p = 2 the slab body's
// default again), 7 the element-matrix body (Gauss diffusion at p = 1, 2);
// the collocated mass operator (pointwise) has one.  The FP64 apply also
// has the double-word bodies (FP64-accurate arithmetic on the FP32 pipe):
// 8..10 the line-based body with the three elements-per-block sizes, 11 the
// element-matrix body, 12..14 the line-based body with the next element
// group's x gather carried one group ahead (scalar operators over whole
// meshes; element lists and vector operators take 8..10's body), 15..17 the
// line-based body with its even and odd contractions carried as packed
// f32x2 pairs, 18..23 those with an L2 prefetch of the next group's qdata;
// 24 (FP64 and FP32) the assembled stencil of p = 1 Gauss diffusion on a
// lattice mesh (stencil.cu).
inline bool fem_has_elmat(int kind, bool colloc, int P) {
  return kind == FEM_DIFFUSION && !colloc && (P == 2 || P == 3);
}
// Element matrices at P = 3 in the double-word layered body's entry order
// (apply_elmat.cuh): the upper triangles of the three diagonal layer blocks
// (45 entries each, row-major, i <= j), then the off-diagonal blocks K of
// layer t against layer t+1 mod 3 (81 entries each, row-major).  Returns
// the index of layered entry n in the row-packed upper triangle (a <= b).
#ifdef __CUDACC__
__host__ __device__
#endif
inline int fem_elmat_layer_src(int n) {
  constexpr int P3 = 27, L = 9, NL = 3, TRI = L * (L + 1) / 2;
  int a, b;
  if (n < NL * TRI) {
    const int t = n / TRI;
    int r = n - t * TRI, i = 0;
    while (r >= L - i) { r -= L - i; i++; }
    a = L * t + i;
    b = L * t + i + r;
  } else {
    const int m = n - NL * TRI, t = m / (L * L), ij = m - t * L * L;
    a = L * t + ij / L;
    b = L * ((t + 1) % NL) + ij % L;
  }
  if (a > b) { const int u = a; a = b; b = u; }
  return a * P3 - a * (a - 1) / 2 + (b - a);
}
inline int fem_apply_choices(const fem_op *op) {
  if (fem_has_elmat(op->kind, op->colloc, op->P)) return 8;
  return (op->kind == FEM_DIFFUSION || !op->colloc) ? 6 : 1;
}
constexpr int FEM_CHOICE_DW_LINES = 8;   // 8, 9, 10
constexpr int FEM_CHOICE_DW_ELMAT = 11;
constexpr int FEM_CHOICE_DW_PIPE = 12;   // 12, 13, 14
constexpr int FEM_CHOICE_DW_PACKED = 15; // 15, 16, 17
constexpr int FEM_CHOICE_DW_PF = 18;     // 18, 19, 20 (21, 22, 23: with the pipelined gather)
constexpr int FEM_CHOICE_DW_STENCIL = 24;
constexpr int FEM_APPLY_CHOICES_MAX = 25;
inline bool fem_choice_is_dw(int c) { return c >= FEM_CHOICE_DW_LINES && c < FEM_APPLY_CHOICES_MAX; }
// Allocate and compute the trilinear body's line sums if op has none yet
// (capi.cu); called where choice 6 is selected, outside stream capture.
int fem_ensure_qsum(fem_op *op);

// Choice c is a valid launch shape of op's apply in precision prec (6
// exists at P = 2 only; 8..24 in FP64 only).
bool fem_op_is_lattice(fem_op *op);
inline bool fem_apply_choice_valid(const fem_op *op, int prec, int c) {
  if (c == FEM_CHOICE_DW_STENCIL)   // FP64 (double words) and FP32
    return (prec == FEM_F64 || op->prec == FEM_F32) && fem_has_elmat(op->kind, op->colloc, op->P) &&
           op->P == 2 && op->ncomp == 1 && op->lattice_n > 0;
  if ((c >= FEM_CHOICE_DW_LINES && c < FEM_CHOICE_DW_ELMAT) ||
      (c >= FEM_CHOICE_DW_PIPE && c < FEM_CHOICE_DW_STENCIL))   // 8..10, 12..23
    return prec == FEM_F64 && (op->kind == FEM_DIFFUSION || !op->colloc);
  if (c == FEM_CHOICE_DW_ELMAT) return prec == FEM_F64 && fem_has_elmat(op->kind, op->colloc, op->P);
  return c >= 0 && c < fem_apply_choices(op) && !(c == 6 && op->P != 2);
}
// Make the data a launch choice of precision prec reads (FP64 qdata or
// element matrices, the trilinear line sums, the double-word copies) if op
// has none yet (capi.cu); called where the choice is selected, outside
// stream capture.  Operators whose FP64 default is a double-word body
// release their FP64 qdata and element matrices after set-up; these calls
// rebuild them.
int fem_ensure_choice_data(fem_op *op, int prec, int choice);
// The assembled stencil of a lattice p = 1 diffusion operator (stencil.cu).
int fem_ensure_stencil(fem_op *op, int prec);
int fem_launch_apply_stencil(fem_op *op, const double *x, double *y, double *dot_out, const int *skip);
int fem_launch_apply_stencil_f32(fem_op *op, const float *x, float *y, double *dot_out, const int *skip);
// The FP64 qdata (recomputed from the mesh if released).
int fem_ensure_qdata64(fem_op *op);
// ---- p-multigrid internals used by the refined flexible CG (pmg.cu)
struct fem_pmg;
int fem_pmg_enqueue_vcycle32(fem_pmg *m, const float *r, float *z, cudaStream_t s);
fem_op *fem_pmg_finest(const fem_pmg *m);
int fem_pmg_precision(const fem_pmg *m);
// ---- setup (setup.cu)
int fem_setup_qdata(fem_op *op);
int fem_setup_diagonal(fem_op *op);
int fem_launch_rhs(fem_op *op, int which, double *b);
// ---- CG (cg.cu)
int fem_cg_run(fem_op *op, const double *b, double *x, const fem_cg_opts *o,
               fem_cg_stats *st);
void fem_cg_free(fem_op *op);
int64_t fem_cg_checkpoint_bytes(const fem_op *op);
int fem_cg_checkpoint_save(fem_op *op, void *host);
int fem_cg_checkpoint_restore(fem_op *op, const void *host);
int fem_cg_resume_run(fem_op *op, const double *b, double *x, const fem_cg_opts *o,
                      fem_cg_stats *st);
// ---- mixed precision (refine.cu)
void fem_refine_free(fem_op *op);

// ---------------------------------------------------------------- device helpers
#ifdef __CUDACC__
__device__ __forceinline__ double fem_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic grid-wide sum of NV doubles per thread.  Every block writes
// its partial sums; the last block to arrive (ticket counter) adds the
// partials in block order and leaves the totals in `tot` (shared, valid in
// the last block only) and resets the counter.  Returns true in the last
// block.  blockDim.x must be a multiple of 32.  No block waits on another.
template <int NV>
__device__ bool fem_grid_sum(const double (&v)[NV], double *partials,
                             unsigned *counter, double (&tot)[NV]) {
  __shared__ double red[NV][32];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; k++) {
    double s = fem_warp_sum(v[k]);
    if (lane == 0) red[k][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; k++) {
      double s = lane < nwarps ? red[k][lane] : 0.0;
      s = fem_warp_sum(s);
      if (lane == 0) partials[(size_t)k * FEM_MAX_BLOCKS + blockIdx.x] = s;
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned ticket = atomicAdd(counter, 1u);
    s_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < NV; k++) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      s += ((volatile double *)partials)[(size_t)k * FEM_MAX_BLOCKS + b];
    s = fem_warp_sum(s);
    if (lane == 0) red[k][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; k++) {
      double s = 0.0;
      for (int w = 0; w < nwarps; w++) s += red[k][w];
      tot[k] = s;
    }
    *counter = 0u;
  }
  __syncthreads();
  return true;
}
#endif
