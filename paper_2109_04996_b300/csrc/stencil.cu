// Globally assembled operator for p = 1 Gauss diffusion on a lattice mesh
// (launch choice 24 of an FP64 operator), in double-word arithmetic.
//
// The paper keeps full assembly for first and second order and partial
// assembly for high order (section "Miniapps": Laghos' full and partial
// assembly options).  At p = 1 the element matrices (36 packed entries per
// element, about one element per node) cost 288 bytes per node per apply
// plus the node ids and the atomic scatter; the assembled operator of a
// lattice mesh -- the n x n x n brick with lexicographic nodes and elements,
// as the bake-off meshes are -- is a 27-point stencil whose columns need no
// ids: node i's neighbours are i + dx + M dy + M^2 dz (M = n + 1, d in
// {-1, 0, 1}^3).  Its rows sum to zero (the basis is a partition of unity,
// so K_e annihilates constants), so a row is stored as its 26 off-diagonal
// coefficients (208 bytes) and applied in difference form,
//   (A x)_i = sum_{j != i} A_ij (x_j - x_i),
// which is exact for constants and, on smooth fields, multiplies small
// differences instead of cancelling large products (5e7 DOFs, smoothest
// sine: 1.9e-12 from the oracle against 5.5e-12 for the plain 27-term sum,
// for 2.27 against 2.17 ms per apply).  The launch bound of three blocks of
// 256 threads per SM lets the compiler keep the coefficient loads in flight
// together (80 registers; without a bound it took 48 and issued them a few
// at a time: 3.5 ms).
//
//   set-up:  A[s][i] = sum over the (up to 8) elements holding node i of
//            K_e[a(i)][b], for the local node b at offset s != 0 from i;
//            each row gathers its own terms in a fixed order (deterministic),
//            in FP64, then split into double words, stored slot-major
//            [26][N];
//   apply:   x split once into double words (one pass), then one thread per
//            row: y_i += sum_s A[s][i] (x[i + off_s] - x_i) in double words,
//            with x^T y fused (the element bodies' x_e^T A_e x_e summed the
//            other way round), y written once without atomics.
//
// Only whole-mesh scalar applies take this path; element lists fall back to
// the element-matrix body (choice 11), which the selection also prepares.
#include <math.h>

#include <type_traits>

#include "apply_kernel.cuh"

namespace {

constexpr int kThreads = 256;

// The lattice test: E = n^3, N = (n+1)^3 and element e = ex + n ey + n^2 ez
// holds node (ex + ax) + M (ey + ay) + M^2 (ez + az) as local node
// ax + 2 ay + 4 az.
__global__ void lattice_check_kernel(const int32_t *en, int64_t E, int64_t n, unsigned *bad) {
  const int64_t M = n + 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ex = e % n, ey = (e / n) % n, ez = e / (n * n);
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 8; a++) {
      const int64_t want = (ex + (a & 1)) + M * (ey + ((a >> 1) & 1)) + M * M * (ez + (a >> 2));
      ok = ok && (int64_t)en[e * 8 + a] == want;
    }
    if (!ok) atomicOr(bad, 1u);
  }
}

// Row i of the stencil from the FP64 element matrices (row-packed upper
// triangle, entry-major [36][E]): the 26 off-diagonal slots, slot s of
// offset d at s' = s - (s > 13) with s = (dx+1) + 3 (dy+1) + 9 (dz+1).
template <typename T>
__global__ void stencil_assemble_kernel(const double *kel, int64_t E, int64_t n, T *A) {
  const int64_t M = n + 1, N = M * M * M;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ix = i % M, iy = (i / M) % M, iz = i / (M * M);
    double acc[27];
#pragma unroll
    for (int s = 0; s < 27; s++) acc[s] = 0.0;
#pragma unroll
    for (int a = 0; a < 8; a++) {
      const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
      const int64_t ex = ix - ax, ey = iy - ay, ez = iz - az;
      if (ex < 0 || ey < 0 || ez < 0 || ex >= n || ey >= n || ez >= n) continue;
      const int64_t e = ex + n * (ey + n * ez);
#pragma unroll
      for (int b = 0; b < 8; b++) {
        const int lo = a < b ? a : b, hi = a < b ? b : a;
        const int idx = lo * 8 - lo * (lo - 1) / 2 + (hi - lo);
        const int s = ((b & 1) - ax + 1) + 3 * (((b >> 1) & 1) - ay + 1) + 9 * ((b >> 2) - az + 1);
        acc[s] += kel[(int64_t)idx * E + e];
      }
    }
#pragma unroll
    for (int s = 0; s < 27; s++) {
      if (s == 13) continue;
      if constexpr (std::is_same<T, dw>::value) A[(int64_t)(s - (s > 13)) * N + i] = dw_from_double(acc[s]);
      else A[(int64_t)(s - (s > 13)) * N + i] = (T)acc[s];
    }
  }
}

__global__ void fem_apply_split_kernel(const double *x, dw *xd, int64_t N, const int *skip) {
  if (skip && *(volatile const int *)skip) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    xd[i] = dw_from_double_int(x[i]);
}

struct StencilParams {
  const dw *A;         // [26][N], the off-diagonal coefficients
  const dw *x;         // [N], the double-word split of the input
  double *y;           // [N], accumulated
  int64_t N;
  int M;               // lattice nodes per direction
  double *partials;
  unsigned *counter;
  double *dot_out;     // x^T (A x), or nullptr
  const int *skip;
};

__device__ __forceinline__ dw ld_stream(const dw *p) {
  const float2 v = __ldcs(reinterpret_cast<const float2 *>(p));
  return dw(v.x, v.y);
}

__global__ void __launch_bounds__(kThreads, 3) fem_apply_stencil27_kernel(const StencilParams sp) {
  if (sp.skip && *(volatile const int *)sp.skip) return;
  const int M = sp.M;
  const int64_t M2 = (int64_t)M * M;
  dw dot(0.0f, 0.0f);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sp.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    // N < 2^31 (int32 node ids), so 32-bit coordinates
    const unsigned u = (unsigned)i, um = (unsigned)M;
    const unsigned ix = u % um, t = u / um, iy = t % um, iz = t / um;
    // every load unconditional, so that all of them can be in flight at
    // once: a neighbour outside the lattice has a zero coefficient and
    // reads x_i instead
    dw a[26];
#pragma unroll
    for (int s = 0; s < 26; s++) a[s] = ld_stream(sp.A + (int64_t)s * sp.N + i);
    // (keeps the compiler from sinking those loads towards their uses: the
    // 26 coefficient streams are then in flight together)
    asm volatile("" ::: "memory");
    const float2 xi2 = *reinterpret_cast<const float2 *>(sp.x + i);
    const dw xi(xi2.x, xi2.y);
    dw acc(0.0f, 0.0f);
#pragma unroll
    for (int dz = -1; dz <= 1; dz++) {
#pragma unroll
      for (int dy = -1; dy <= 1; dy++) {
#pragma unroll
        for (int dx = -1; dx <= 1; dx++) {
          const int s = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
          if (s == 13) continue;
          const bool in = (dx >= 0 || ix > 0) && (dx <= 0 || ix + 1 < um) && (dy >= 0 || iy > 0) &&
                          (dy <= 0 || iy + 1 < um) && (dz >= 0 || iz > 0) && (dz <= 0 || iz + 1 < um);
          const int64_t j = in ? i + dx + (int64_t)M * dy + M2 * dz : i;
          const float2 xv = *reinterpret_cast<const float2 *>(sp.x + j);
          acc += a[s - (s > 13)] * (dw(xv.x, xv.y) - xi);
        }
      }
    }
    dot += acc * xi;
    sp.y[i] += dw_to_double_int(acc);
  }
  if (sp.dot_out) {
    double v[1] = {dw_to_double(dot)};
    __shared__ double tot[1];
    if (fem_grid_sum<1>(v, sp.partials, sp.counter, tot) && threadIdx.x == 0) *sp.dot_out = tot[0];
  }
}

// The same stencil in FP32 (FP32 operators, e.g. the coarse levels of an
// FP32 p-multigrid V-cycle): FP32 coefficients (104 bytes a row) and x, no
// split pass, x^T y by the FP32 bodies' compensated accumulation.
struct StencilParams32 {
  const float *A;      // [26][N]
  const float *x;
  float *y;            // accumulated
  int64_t N;
  int M;
  double *partials;
  unsigned *counter;
  double *dot_out;
  const int *skip;
};

__global__ void __launch_bounds__(kThreads, 3) fem_apply_stencil27_f32_kernel(const StencilParams32 sp) {
  if (sp.skip && *(volatile const int *)sp.skip) return;
  const int M = sp.M;
  const int64_t M2 = (int64_t)M * M;
  fem_apply::DotAcc<float> dl;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sp.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned u = (unsigned)i, um = (unsigned)M;
    const unsigned ix = u % um, t = u / um, iy = t % um, iz = t / um;
    float a[26];
#pragma unroll
    for (int s = 0; s < 26; s++) a[s] = __ldcs(sp.A + (int64_t)s * sp.N + i);
    asm volatile("" ::: "memory");
    const float xi = sp.x[i];
    float acc = 0.0f;
#pragma unroll
    for (int dz = -1; dz <= 1; dz++) {
#pragma unroll
      for (int dy = -1; dy <= 1; dy++) {
#pragma unroll
        for (int dx = -1; dx <= 1; dx++) {
          const int s = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
          if (s == 13) continue;
          const bool in = (dx >= 0 || ix > 0) && (dx <= 0 || ix + 1 < um) && (dy >= 0 || iy > 0) &&
                          (dy <= 0 || iy + 1 < um) && (dz >= 0 || iz > 0) && (dz <= 0 || iz + 1 < um);
          const int64_t j = in ? i + dx + (int64_t)M * dy + M2 * dz : i;
          acc = fmaf(a[s - (s > 13)], sp.x[j] - xi, acc);
        }
      }
    }
    dl.add(acc, xi);
    sp.y[i] += acc;
  }
  if (sp.dot_out) {
    double v[1] = {dl.get()};
    __shared__ double tot[1];
    if (fem_grid_sum<1>(v, sp.partials, sp.counter, tot) && threadIdx.x == 0) *sp.dot_out = tot[0];
  }
}

}  // namespace

// Is op's mesh a lattice (see lattice_check_kernel)?  Checked once per
// operator, outside stream capture (a host synchronization).
bool fem_op_is_lattice(fem_op *op) {
  if (op->lattice_n >= 0) return op->lattice_n > 0;
  op->lattice_n = 0;
  if (op->P != 2 || op->E < 1) return false;
  int64_t n = (int64_t)llround(cbrt((double)op->E));
  while (n * n * n > op->E) n--;
  while ((n + 1) * (n + 1) * (n + 1) <= op->E) n++;
  if (n * n * n != op->E || (n + 1) * (n + 1) * (n + 1) != op->N) return false;
  unsigned *bad = nullptr;
  if (cudaMalloc(&bad, sizeof(unsigned)) != cudaSuccess) { cudaGetLastError(); return false; }
  unsigned h = 1;
  bool ok = cudaMemsetAsync(bad, 0, sizeof(unsigned), op->stream()) == cudaSuccess;
  if (ok) {
    lattice_check_kernel<<<op->nsm * 8, kThreads, 0, op->stream()>>>(op->mesh->d_elem_nodes, op->E, n, bad);
    ok = cudaGetLastError() == cudaSuccess &&
         cudaMemcpyAsync(&h, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, op->stream()) == cudaSuccess &&
         cudaStreamSynchronize(op->stream()) == cudaSuccess;
  }
  cudaFree(bad);
  if (ok && h == 0) op->lattice_n = n;
  return op->lattice_n > 0;
}

// The stencil coefficients and, in FP64, the split-input buffer (needs the
// FP64 element matrices, which the caller makes first).
int fem_ensure_stencil(fem_op *op, int prec) {
  if (prec == FEM_F32) {
    if (op->d_stencil32) return FEM_OK;
    if (!fem_op_is_lattice(op) || !op->d_kel) {
      fem_set_error("apply: the assembled stencil (choice 24) needs p = 1 Gauss diffusion on a lattice mesh");
      return FEM_EINVAL;
    }
    if (cudaMalloc(&op->d_stencil32, sizeof(float) * 26 * (size_t)op->N) != cudaSuccess) {
      cudaGetLastError();
      op->d_stencil32 = nullptr;
      fem_set_error("apply: device allocation of the stencil failed");
      return FEM_ENOMEM;
    }
    op->bytes += (int64_t)(sizeof(float) * 26 * (size_t)op->N);
    stencil_assemble_kernel<float><<<op->nsm * 8, kThreads, 0, op->stream()>>>(op->d_kel, op->E, op->lattice_n,
                                                                                op->d_stencil32);
    FEM_CHECK_LAUNCH();
    return FEM_OK;
  }
  if (op->d_stencil && op->d_xdw) return FEM_OK;
  if (!fem_op_is_lattice(op) || !op->d_kel) {
    fem_set_error("apply: the assembled stencil (choice 24) needs p = 1 Gauss diffusion on a lattice mesh");
    return FEM_EINVAL;
  }
  const int64_t N = op->N;
  if (!op->d_stencil) {
    if (cudaMalloc(&op->d_stencil, sizeof(dw) * 26 * (size_t)N) != cudaSuccess) {
      cudaGetLastError();
      op->d_stencil = nullptr;
      fem_set_error("apply: device allocation of the stencil failed");
      return FEM_ENOMEM;
    }
    op->bytes += (int64_t)(sizeof(dw) * 26 * (size_t)N);
    stencil_assemble_kernel<dw><<<op->nsm * 8, kThreads, 0, op->stream()>>>(op->d_kel, op->E, op->lattice_n,
                                                                             op->d_stencil);
    FEM_CHECK_LAUNCH();
  }
  if (!op->d_xdw) {
    if (cudaMalloc(&op->d_xdw, sizeof(dw) * (size_t)N) != cudaSuccess) {
      cudaGetLastError();
      op->d_xdw = nullptr;
      fem_set_error("apply: device allocation of the stencil input failed");
      return FEM_ENOMEM;
    }
    op->bytes += (int64_t)(sizeof(dw) * (size_t)N);
  }
  return FEM_OK;
}

int fem_launch_apply_stencil(fem_op *op, const double *x, double *y, double *dot_out, const int *skip) {
  if (!op->d_stencil || !op->d_xdw) {
    fem_set_error("apply: the assembled stencil is not set up");
    return FEM_EINVAL;
  }
  static FemKernelCache cache;
  int &per_sm = cache.here();
  if (per_sm < 0) {
    int b = 0;
    FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fem_apply_stencil27_kernel, kThreads, 0));
    per_sm = b < 1 ? 1 : b;
  }
  const int64_t N = op->N;
  int64_t grid = (int64_t)op->nsm * per_sm, need = (N + kThreads - 1) / kThreads;
  if (grid > need) grid = need;
  if (grid > FEM_MAX_BLOCKS) grid = FEM_MAX_BLOCKS;
  if (grid < 1) grid = 1;
  // (a plain stream: its own, larger grid -- at the stencil's two blocks
  // per SM it ran at a third of the copy rate)
  int64_t gsplit = (int64_t)op->nsm * 16;
  if (gsplit > need) gsplit = need;
  if (gsplit < 1) gsplit = 1;
  fem_apply_split_kernel<<<(unsigned)gsplit, kThreads, 0, op->stream()>>>(x, op->d_xdw, N, skip);
  FEM_CHECK_LAUNCH();
  StencilParams sp;
  sp.A = op->d_stencil; sp.x = op->d_xdw; sp.y = y; sp.N = N; sp.M = (int)(op->lattice_n + 1);
  sp.partials = op->d_partials; sp.counter = op->d_counter; sp.dot_out = dot_out; sp.skip = skip;
  fem_apply_stencil27_kernel<<<(unsigned)grid, kThreads, 0, op->stream()>>>(sp);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

int fem_launch_apply_stencil_f32(fem_op *op, const float *x, float *y, double *dot_out, const int *skip) {
  if (!op->d_stencil32) {
    fem_set_error("apply_f32: the assembled stencil is not set up");
    return FEM_EINVAL;
  }
  static FemKernelCache cache;
  int &per_sm = cache.here();
  if (per_sm < 0) {
    int b = 0;
    FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fem_apply_stencil27_f32_kernel, kThreads, 0));
    per_sm = b < 1 ? 1 : b;
  }
  const int64_t N = op->N;
  int64_t grid = (int64_t)op->nsm * per_sm, need = (N + kThreads - 1) / kThreads;
  if (grid > need) grid = need;
  if (grid > FEM_MAX_BLOCKS) grid = FEM_MAX_BLOCKS;
  if (grid < 1) grid = 1;
  StencilParams32 sp;
  sp.A = op->d_stencil32; sp.x = x; sp.y = y; sp.N = N; sp.M = (int)(op->lattice_n + 1);
  sp.partials = op->d_partials; sp.counter = op->d_counter; sp.dot_out = dot_out; sp.skip = skip;
  fem_apply_stencil27_f32_kernel<<<(unsigned)grid, kThreads, 0, op->stream()>>>(sp);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}
