// p-multigrid preconditioner and the flexible CG around it.  The paper
// (section "Ecosystem", matrix-free preconditioning) names p-multigrid -- a
// hierarchy of polynomial degrees on one mesh with matrix-free smoothers --
// as the route to scalable matrix-free solvers; its parts here:
//
//   levels      operators of decreasing order on the same elements (the
//               caller's meshes, Gauss-Lobatto nodes), each its own
//               discretization;
//   transfers   prolongation P: coarse element values interpolated at the
//               fine element's nodes by the 1D coarse Lagrange basis in each
//               direction, scatter-added with weight 1/multiplicity (the
//               average over the elements sharing a node); restriction
//               R = P^T, the same steps transposed;
//   smoother    m steps of the Chebyshev iteration (Saad 2003, Alg. 12.1) on
//               D^-1 A over [lo, hi] * lmax, lmax from power iterations with
//               the Rayleigh quotient v^T A v / v^T D v, started from the
//               SplitMix64 vector (Steele, Lea & Flood 2014);
//   coarsest    k_c Jacobi-PCG iterations from zero;
//   V-cycle     z = S(r); z += P V(R (r - A z)); z += S(r - A z).
// Every vector of a level vanishes on its Dirichlet nodes (A stands for
// M A M + (I - M)).  The V-cycle has a fixed launch sequence (no data-
// dependent control), so it is captured once into a CUDA graph; the outer
// flexible CG (Notay 2000, one stored direction, FP64) is one graph with a
// conditional WHILE node, as in cg.cu.  With prec = FEM_F32 the V-cycle runs
// on the levels' FP32 operators and vectors, with FP64 dot products.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "fem_internal.h"

namespace {

constexpr int kT = 256;

int gridn(int64_t n) {
  int64_t g = (n + kT - 1) / kT;
  if (g > 148 * 8) g = 148 * 8;
  return g < 1 ? 1 : (int)g;
}

template <typename T>
struct LevelVecs {
  T *r = nullptr, *z = nullptr, *t = nullptr, *d = nullptr, *y = nullptr;
  T *dinv = nullptr;   // 1/diag on interior nodes, 0 on Dirichlet nodes  [n]
  T *wm = nullptr;     // 1/multiplicity on interior nodes, 0 else        [N]
  T *msk = nullptr;    // 1 on interior nodes, 0 else                      [N]
  T *I = nullptr;      // interpolation from the next coarser level [P][Pc]
};

struct Level {
  fem_op *op = nullptr;
  int P = 0, Pc = 0;   // this level's P = p+1; the next coarser level's
  int64_t N = 0, E = 0, n = 0;
  double lmax = 0.0;
  LevelVecs<double> v64;
  LevelVecs<float> v32;
};

}  // namespace

struct fem_pmg {
  std::vector<Level> lv;
  fem_pmg_opts o;
  cudaStream_t stream = nullptr;
  std::vector<void *> allocs;
  double *sc = nullptr;          // device scalars (see kS*)
  double *partials = nullptr;    // [4 * FEM_MAX_BLOCKS]
  unsigned *counter = nullptr;
  // outer FCG (FP64, finest level)
  double *x_r = nullptr, *x_z = nullptr, *x_p = nullptr, *x_y = nullptr;
  cudaStream_t cap = nullptr, cap2 = nullptr;
  cudaGraphExec_t vexec = nullptr;     // V-cycle (level-0 buffers of o.prec)
  cudaGraphExec_t sexec = nullptr;     // solve
  const double *g_b = nullptr;
  double *g_x = nullptr;
};

namespace {

// device scalar slots
enum {
  kSRs0 = 0, kSRs1 = 1,   // coarse PCG r^T D^-1 r, ping-pong by iteration parity
  kSPAp = 2,              // coarse PCG p^T A p
  kSNorm = 3,             // power iteration ||v||^2 / v^T A v
  kSDen = 4,              // power iteration v^T D v
  kFZy = 8, kFPr = 9, kFPAp = 10, kFPApOld = 11, kFRr = 12, kFBb = 13,
  kFIter = 14, kFStatus = 15, kFRtol2 = 16, kFMaxit = 17,
  kNumScalars = 24
};

// ---------------------------------------------------------------- helpers
template <typename T>
__global__ void fill_kernel(T *a, T v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

__global__ void count_kernel(const int32_t *en, int64_t total, float *cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[en[i]], 1.0f);
}

// wm = inner / multiplicity, msk = inner, dinv = inner / diag (per component)
template <typename T>
__global__ void level_setup_kernel(const float *cnt, const uint8_t *dir, const double *diag,
                                   int64_t N, int ncomp, T *wm, T *msk, T *dinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool in = !(dir && dir[i]);
    wm[i] = in && cnt[i] > 0.0f ? (T)(1.0 / (double)cnt[i]) : (T)0;
    msk[i] = in ? (T)1 : (T)0;
    for (int c = 0; c < ncomp; c++) dinv[c * N + i] = in ? (T)(1.0 / diag[i]) : (T)0;
  }
}

// ---------------------------------------------------------------- transfers
// One block takes `epb` elements; shared memory per element: the coarse cube
// Pc^3, the two partial contractions Pc^2 Pf and Pc Pf^2, the fine cube Pf^3.
// Element-local node order a + P b + P^2 c.
template <typename T>
__global__ void prolong_kernel(const int32_t *enc, const int32_t *enf, int64_t E, int Pc, int Pf,
                               int epb, const T *I, const T *xc, const T *mskc, const T *wmf,
                               int64_t Nc, int64_t Nf, int ncomp, T *xf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sI = reinterpret_cast<T *>(smem_raw);
  const int Pc3 = Pc * Pc * Pc, Pf3 = Pf * Pf * Pf, Pc2f = Pc * Pc * Pf, Pcf2 = Pc * Pf * Pf;
  const int per = Pc3 + Pc2f + Pcf2 + Pf3;
  T *buf = sI + Pf * Pc;
  for (int i = threadIdx.x; i < Pf * Pc; i += blockDim.x) sI[i] = I[i];
  const int64_t ngroups = (E + epb - 1) / epb;
  for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const int64_t e0 = g * epb;
    const int ne = (int)(E - e0 < epb ? E - e0 : epb);
    for (int c = 0; c < ncomp; c++) {
      __syncthreads();
      for (int i = threadIdx.x; i < ne * Pc3; i += blockDim.x) {
        const int s = i / Pc3, l = i - s * Pc3;
        const int64_t node = enc[(e0 + s) * Pc3 + l];
        buf[s * per + l] = xc[c * Nc + node] * mskc[node];
      }
      __syncthreads();
      // u1[c][b][i] = sum_a I[i][a] u0[c][b][a]
      for (int o = threadIdx.x; o < ne * Pc2f; o += blockDim.x) {
        const int s = o / Pc2f, l = o - s * Pc2f;
        const int i = l % Pf, cb = l / Pf;
        const T *u0 = buf + s * per + cb * Pc;
        T acc = 0;
        for (int a = 0; a < Pc; a++) acc += sI[i * Pc + a] * u0[a];
        buf[s * per + Pc3 + l] = acc;
      }
      __syncthreads();
      // u2[c][j][i] = sum_b I[j][b] u1[c][b][i]
      for (int o = threadIdx.x; o < ne * Pcf2; o += blockDim.x) {
        const int s = o / Pcf2, l = o - s * Pcf2;
        const int i = l % Pf, j = (l / Pf) % Pf, cc = l / (Pf * Pf);
        const T *u1 = buf + s * per + Pc3 + cc * Pc * Pf + i;
        T acc = 0;
        for (int b = 0; b < Pc; b++) acc += sI[j * Pc + b] * u1[b * Pf];
        buf[s * per + Pc3 + Pc2f + l] = acc;
      }
      __syncthreads();
      // u3[k][j][i] = sum_c I[k][c] u2[c][j][i]; scatter with the fine weights
      for (int o = threadIdx.x; o < ne * Pf3; o += blockDim.x) {
        const int s = o / Pf3, l = o - s * Pf3;
        const int ji = l % (Pf * Pf), k = l / (Pf * Pf);
        const T *u2 = buf + s * per + Pc3 + Pc2f + ji;
        T acc = 0;
        for (int cc = 0; cc < Pc; cc++) acc += sI[k * Pc + cc] * u2[cc * Pf * Pf];
        const int64_t node = enf[(e0 + s) * Pf3 + l];
        const T w = wmf[node];
        if (w != (T)0) atomicAdd(&xf[c * Nf + node], w * acc);
      }
    }
  }
}

template <typename T>
__global__ void restrict_kernel(const int32_t *enc, const int32_t *enf, int64_t E, int Pc, int Pf,
                                int epb, const T *I, const T *rf, const T *wmf, const T *mskc,
                                int64_t Nc, int64_t Nf, int ncomp, T *rc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sI = reinterpret_cast<T *>(smem_raw);
  const int Pc3 = Pc * Pc * Pc, Pf3 = Pf * Pf * Pf, Pc2f = Pc * Pc * Pf, Pcf2 = Pc * Pf * Pf;
  const int per = Pc3 + Pc2f + Pcf2 + Pf3;
  T *buf = sI + Pf * Pc;
  for (int i = threadIdx.x; i < Pf * Pc; i += blockDim.x) sI[i] = I[i];
  const int64_t ngroups = (E + epb - 1) / epb;
  for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const int64_t e0 = g * epb;
    const int ne = (int)(E - e0 < epb ? E - e0 : epb);
    for (int c = 0; c < ncomp; c++) {
      __syncthreads();
      // fine cube, weighted: u[k][j][i]
      for (int i = threadIdx.x; i < ne * Pf3; i += blockDim.x) {
        const int s = i / Pf3, l = i - s * Pf3;
        const int64_t node = enf[(e0 + s) * Pf3 + l];
        buf[s * per + Pc3 + Pc2f + Pcf2 + l] = rf[c * Nf + node] * wmf[node];
      }
      __syncthreads();
      // v1[c][j][i] = sum_k I[k][c] u[k][j][i]
      for (int o = threadIdx.x; o < ne * Pcf2; o += blockDim.x) {
        const int s = o / Pcf2, l = o - s * Pcf2;
        const int ji = l % (Pf * Pf), cc = l / (Pf * Pf);
        const T *u = buf + s * per + Pc3 + Pc2f + Pcf2 + ji;
        T acc = 0;
        for (int k = 0; k < Pf; k++) acc += sI[k * Pc + cc] * u[k * Pf * Pf];
        buf[s * per + Pc3 + Pc2f + l] = acc;
      }
      __syncthreads();
      // v2[c][b][i] = sum_j I[j][b] v1[c][j][i]
      for (int o = threadIdx.x; o < ne * Pc2f; o += blockDim.x) {
        const int s = o / Pc2f, l = o - s * Pc2f;
        const int i = l % Pf, b = (l / Pf) % Pc, cc = l / (Pf * Pc);
        const T *v1 = buf + s * per + Pc3 + Pc2f + cc * Pf * Pf + i;
        T acc = 0;
        for (int j = 0; j < Pf; j++) acc += sI[j * Pc + b] * v1[j * Pf];
        buf[s * per + Pc3 + l] = acc;
      }
      __syncthreads();
      // v3[c][b][a] = sum_i I[i][a] v2[c][b][i]; scatter to the coarse nodes
      for (int o = threadIdx.x; o < ne * Pc3; o += blockDim.x) {
        const int s = o / Pc3, l = o - s * Pc3;
        const int a = l % Pc, cb = l / Pc;
        const T *v2 = buf + s * per + Pc3 + cb * Pf;
        T acc = 0;
        for (int i = 0; i < Pf; i++) acc += sI[i * Pc + a] * v2[i];
        const int64_t node = enc[(e0 + s) * Pc3 + l];
        if (mskc[node] != (T)0) atomicAdd(&rc[c * Nc + node], acc);
      }
    }
  }
}

int transfer_epb(int Pf) {
  const int Pf3 = Pf * Pf * Pf;
  return Pf3 >= 256 ? 1 : 256 / Pf3;
}

template <typename T>
size_t transfer_smem(int Pc, int Pf) {
  const int per = Pc * Pc * Pc + Pc * Pc * Pf + Pc * Pf * Pf + Pf * Pf * Pf;
  return sizeof(T) * ((size_t)Pf * Pc + (size_t)transfer_epb(Pf) * per);
}

// xf += P xc (xf accumulates), level l <- l+1
template <typename T>
int launch_prolong(fem_pmg *m, int l, const T *xc, T *xf, cudaStream_t s) {
  Level &f = m->lv[l], &c = m->lv[l + 1];
  const LevelVecs<T> &vf = *reinterpret_cast<const LevelVecs<T> *>(sizeof(T) == 8 ? (void *)&f.v64 : (void *)&f.v32);
  const LevelVecs<T> &vc = *reinterpret_cast<const LevelVecs<T> *>(sizeof(T) == 8 ? (void *)&c.v64 : (void *)&c.v32);
  const int epb = transfer_epb(f.P);
  const int64_t ng = (f.E + epb - 1) / epb;
  const int grid = (int)(ng < 148 * 8 ? ng : 148 * 8);
  prolong_kernel<T><<<grid, kT, transfer_smem<T>(c.P, f.P), s>>>(
      c.op->mesh->d_elem_nodes, f.op->mesh->d_elem_nodes, f.E, c.P, f.P, epb, vf.I, xc, vc.msk,
      vf.wm, c.N, f.N, f.op->ncomp, xf);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

// rc += R rf (rc accumulates), level l -> l+1
template <typename T>
int launch_restrict(fem_pmg *m, int l, const T *rf, T *rc, cudaStream_t s) {
  Level &f = m->lv[l], &c = m->lv[l + 1];
  const LevelVecs<T> &vf = *reinterpret_cast<const LevelVecs<T> *>(sizeof(T) == 8 ? (void *)&f.v64 : (void *)&f.v32);
  const LevelVecs<T> &vc = *reinterpret_cast<const LevelVecs<T> *>(sizeof(T) == 8 ? (void *)&c.v64 : (void *)&c.v32);
  const int epb = transfer_epb(f.P);
  const int64_t ng = (f.E + epb - 1) / epb;
  const int grid = (int)(ng < 148 * 8 ? ng : 148 * 8);
  restrict_kernel<T><<<grid, kT, transfer_smem<T>(c.P, f.P), s>>>(
      c.op->mesh->d_elem_nodes, f.op->mesh->d_elem_nodes, f.E, c.P, f.P, epb, vf.I, rf, vf.wm,
      vc.msk, c.N, f.N, f.op->ncomp, rc);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

// ---------------------------------------------------------------- smoother
// first Chebyshev step on residual src (may alias t): d = dinv src / theta;
// z = d (acc = 0) or z += d (acc = 1); t = src; y = 0
template <typename T>
__global__ void cheb_first_kernel(const T *src, const T *dinv, double inv_theta, int acc, T *d,
                                  T *z, T *t, T *y, int64_t n) {
  const T it = (T)inv_theta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T r = src[i];
    const T di = it * dinv[i] * r;
    d[i] = di;
    z[i] = acc ? z[i] + di : di;
    t[i] = r;
    y[i] = (T)0;
  }
}

// later steps, after y = A d: t = M (t - y); d = c1 d + c2 dinv t; z += d; y = 0
template <typename T>
__global__ void cheb_step_kernel(T *t, T *y, T *d, T *z, const T *dinv, const T *msk, int64_t N,
                                 double c1, double c2, int64_t n) {
  const T a = (T)c1, b = (T)c2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T tk = msk[fem_node_of(i, N)] * (t[i] - y[i]);
    const T di = a * d[i] + b * dinv[i] * tk;
    t[i] = tk;
    d[i] = di;
    z[i] += di;
    y[i] = (T)0;
  }
}

// t = M (r - y); y = 0
template <typename T>
__global__ void residual_kernel(const T *r, T *y, const T *msk, int64_t N, T *t, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    t[i] = msk[fem_node_of(i, N)] * (r[i] - y[i]);
    y[i] = (T)0;
  }
}

// ---------------------------------------------------------------- coarse PCG
// z = 0; t = r; d = dinv t; y = 0; rs[0] = t^T dinv t
template <typename T>
__global__ void cpcg_init_kernel(const T *r, const T *dinv, T *z, T *t, T *d, T *y, int64_t n,
                                 double *sc, double *partials, unsigned *counter) {
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T ri = r[i], si = dinv[i] * ri;
    z[i] = (T)0; t[i] = ri; d[i] = si; y[i] = (T)0;
    v[0] += (double)ri * (double)si;
  }
  __shared__ double tot[1];
  if (fem_grid_sum<1>(v, partials, counter, tot) && threadIdx.x == 0) sc[kSRs0] = tot[0];
}

// after y = A d (p^T A p in sc[kSPAp]): alpha = rs/pAp; z += alpha d;
// t = M (t - alpha y); rs_new = t^T dinv t into the other parity slot
template <typename T>
__global__ void cpcg_update_kernel(T *z, T *t, const T *d, const T *y, const T *dinv, const T *msk,
                                   int64_t N, int64_t n, int par, double *sc, double *partials,
                                   unsigned *counter) {
  const double rs = sc[kSRs0 + par], pAp = sc[kSPAp];
  const double alpha = (pAp > 0.0 && rs > 0.0) ? rs / pAp : 0.0;
  const T a = (T)alpha;
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    z[i] += a * d[i];
    const T ti = msk[fem_node_of(i, N)] * (t[i] - a * y[i]);
    t[i] = ti;
    v[0] += (double)ti * (double)(dinv[i] * ti);
  }
  __shared__ double tot[1];
  if (fem_grid_sum<1>(v, partials, counter, tot) && threadIdx.x == 0) sc[kSRs0 + (par ^ 1)] = tot[0];
}

// d = dinv t + beta d, beta = rs_new / rs; y = 0
template <typename T>
__global__ void cpcg_dir_kernel(const T *t, const T *dinv, T *d, T *y, int64_t n, int par,
                                const double *sc) {
  const double rs = sc[kSRs0 + par], rsn = sc[kSRs0 + (par ^ 1)];
  const T beta = (T)(rs > 0.0 ? rsn / rs : 0.0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    d[i] = dinv[i] * t[i] + beta * d[i];
    y[i] = (T)0;
  }
}

// ---------------------------------------------------------------- power iteration
// SplitMix64 output i of a generator whose state starts at `seed`
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                            unsigned long long i) {
  unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void power_start_kernel(const double *msk, int64_t N, int64_t n, double *v, double *y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double u = (double)(splitmix64_at(0ull, (unsigned long long)i) >> 11) * 0x1.0p-53 - 0.5;
    v[i] = msk[fem_node_of(i, N)] * u;
    y[i] = 0.0;
  }
}

// v = dinv y (masked by dinv), y = 0, ||v||^2 into sc[kSNorm]
__global__ void power_step_kernel(const double *dinv, double *v, double *y, int64_t n, double *sc,
                                  double *partials, unsigned *counter) {
  double s[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double vi = dinv[i] * y[i];
    v[i] = vi;
    y[i] = 0.0;
    s[0] += vi * vi;
  }
  __shared__ double tot[1];
  if (fem_grid_sum<1>(s, partials, counter, tot) && threadIdx.x == 0) sc[kSNorm] = tot[0];
}

__global__ void power_scale_kernel(double *v, int64_t n, const double *sc) {
  const double nv = sc[kSNorm];
  const double f = nv > 0.0 ? 1.0 / sqrt(nv) : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] *= f;
}

// v^T D v (D = 1/dinv on interior nodes) into sc[kSDen]
__global__ void power_den_kernel(const double *v, const double *dinv, int64_t n, double *sc,
                                 double *partials, unsigned *counter) {
  double s[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (dinv[i] != 0.0) s[0] += v[i] * v[i] / dinv[i];
  __shared__ double tot[1];
  if (fem_grid_sum<1>(s, partials, counter, tot) && threadIdx.x == 0) sc[kSDen] = tot[0];
}

// ---------------------------------------------------------------- conversions
__global__ void to_f32_kernel(const double *a, float *b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void copy_f32_kernel(const float *a, float *b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}
__global__ void to_f64_kernel(const float *a, double *b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

// ---------------------------------------------------------------- apply wrappers
int apply(Level &L, const double *x, double *y, double *dot) {
  return fem_launch_apply_f64(L.op, x, y, nullptr, L.E, dot);
}
int apply(Level &L, const float *x, float *y, double *dot) {
  return fem_launch_apply_f32(L.op, x, y, nullptr, L.E, dot);
}
template <typename T>
LevelVecs<T> &vecs(Level &L);
template <>
LevelVecs<double> &vecs<double>(Level &L) { return L.v64; }
template <>
LevelVecs<float> &vecs<float>(Level &L) { return L.v32; }

// ---------------------------------------------------------------- V-cycle
// m Chebyshev steps on the residual `src` of level l (src may be V.t),
// z = result (acc = 0) or z += result (acc = 1)
template <typename T>
int smooth(fem_pmg *m, int l, const T *src, int acc, cudaStream_t s) {
  Level &L = m->lv[l];
  LevelVecs<T> &V = vecs<T>(L);
  const double lo = m->o.cheb_lo * L.lmax, hi = m->o.cheb_hi * L.lmax;
  const double theta = 0.5 * (lo + hi), delta = 0.5 * (hi - lo);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  const int g = gridn(L.n);
  cheb_first_kernel<T><<<g, kT, 0, s>>>(src, V.dinv, 1.0 / theta, acc, V.d, V.z, V.t, V.y, L.n);
  FEM_CHECK_LAUNCH();
  for (int k = 1; k < m->o.cheb_degree; k++) {
    int rc = apply(L, V.d, V.y, nullptr);
    if (rc) return rc;
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    cheb_step_kernel<T><<<g, kT, 0, s>>>(V.t, V.y, V.d, V.z, V.dinv, V.msk, L.N, rho_new * rho,
                                         2.0 * rho_new / delta, L.n);
    FEM_CHECK_LAUNCH();
    rho = rho_new;
  }
  return FEM_OK;
}

template <typename T>
int coarse_solve(fem_pmg *m, int l, cudaStream_t s) {
  Level &L = m->lv[l];
  LevelVecs<T> &V = vecs<T>(L);
  const int g = gridn(L.n);
  cpcg_init_kernel<T><<<g, kT, 0, s>>>(V.r, V.dinv, V.z, V.t, V.d, V.y, L.n, m->sc, m->partials,
                                       m->counter);
  FEM_CHECK_LAUNCH();
  for (int k = 0; k < m->o.coarse_its; k++) {
    const int par = k & 1;
    int rc = apply(L, V.d, V.y, m->sc + kSPAp);
    if (rc) return rc;
    cpcg_update_kernel<T><<<g, kT, 0, s>>>(V.z, V.t, V.d, V.y, V.dinv, V.msk, L.N, L.n, par, m->sc,
                                           m->partials, m->counter);
    FEM_CHECK_LAUNCH();
    if (k + 1 < m->o.coarse_its) {
      cpcg_dir_kernel<T><<<g, kT, 0, s>>>(V.t, V.dinv, V.d, V.y, L.n, par, m->sc);
      FEM_CHECK_LAUNCH();
    }
  }
  return FEM_OK;
}

// z_l = V(r_l), both in level l's buffers of precision T
template <typename T>
int vcycle(fem_pmg *m, int l, cudaStream_t s) {
  Level &L = m->lv[l];
  LevelVecs<T> &V = vecs<T>(L);
  if (l == (int)m->lv.size() - 1) return coarse_solve<T>(m, l, s);
  Level &C = m->lv[l + 1];
  LevelVecs<T> &VC = vecs<T>(C);
  const int g = gridn(L.n);
  int rc = smooth<T>(m, l, V.r, 0, s);                      // z = S(r), y = 0
  if (rc) return rc;
  if ((rc = apply(L, V.z, V.y, nullptr))) return rc;       // y = A z
  residual_kernel<T><<<g, kT, 0, s>>>(V.r, V.y, V.msk, L.N, V.t, L.n);   // t = M(r - y), y = 0
  FEM_CHECK_LAUNCH();
  fill_kernel<T><<<gridn(C.n), kT, 0, s>>>(VC.r, (T)0, C.n);
  FEM_CHECK_LAUNCH();
  if ((rc = launch_restrict<T>(m, l, V.t, VC.r, s))) return rc;   // r_c = R t
  if ((rc = vcycle<T>(m, l + 1, s))) return rc;                    // z_c = V(r_c)
  if ((rc = launch_prolong<T>(m, l, VC.z, V.z, s))) return rc;     // z += P z_c
  if ((rc = apply(L, V.z, V.y, nullptr))) return rc;               // y = A z
  residual_kernel<T><<<g, kT, 0, s>>>(V.r, V.y, V.msk, L.N, V.t, L.n);
  FEM_CHECK_LAUNCH();
  return smooth<T>(m, l, V.t, 1, s);                               // z += S(t)
}

// Capture the whole V-cycle (level-0 r -> z in precision o.prec) on the
// capture stream, with every level's mesh stream pointed at it.
int capture_vcycle(fem_pmg *m, cudaStream_t s, bool f32) {
  return f32 ? vcycle<float>(m, 0, s) : vcycle<double>(m, 0, s);
}

struct StreamSwap {
  fem_pmg *m;
  std::vector<cudaStream_t> saved;
  StreamSwap(fem_pmg *mm, cudaStream_t s) : m(mm) {
    for (Level &L : m->lv) {
      fem_mesh *mesh = const_cast<fem_mesh *>(L.op->mesh);
      saved.push_back(mesh->stream);
      mesh->stream = s;
    }
  }
  ~StreamSwap() {
    for (size_t i = 0; i < m->lv.size(); i++)
      const_cast<fem_mesh *>(m->lv[i].op->mesh)->stream = saved[i];
  }
};

}  // namespace

// One FP32 V-cycle z = V(r) between the caller's level-0 FP32 vectors,
// enqueued on s (which may be capturing) with every level's mesh stream
// pointed at s meanwhile.  Used by the refined flexible CG (fcg.cu); the
// hierarchy must have prec = FEM_F32.
int fem_pmg_enqueue_vcycle32(fem_pmg *m, const float *r, float *z, cudaStream_t s) {
  Level &L = m->lv[0];
  StreamSwap sw(m, s);
  copy_f32_kernel<<<gridn(L.n), kT, 0, s>>>(r, L.v32.r, L.n);
  FEM_CHECK_LAUNCH();
  int rc = vcycle<float>(m, 0, s);
  if (rc) return rc;
  copy_f32_kernel<<<gridn(L.n), kT, 0, s>>>(L.v32.z, z, L.n);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}
fem_op *fem_pmg_finest(const fem_pmg *m) { return m->lv[0].op; }
int fem_pmg_precision(const fem_pmg *m) { return m->o.prec; }

namespace {

int build_vcycle_graph(fem_pmg *m) {
  if (m->vexec) return FEM_OK;
  if (!m->cap) {
    FEM_CUDA_TRY(cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking));
    FEM_CUDA_TRY(cudaStreamCreateWithFlags(&m->cap2, cudaStreamNonBlocking));
  }
  cudaGraph_t graph = nullptr;
  int rc;
  {
    StreamSwap sw(m, m->cap);
    FEM_CUDA_TRY(cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeRelaxed));
    rc = capture_vcycle(m, m->cap, m->o.prec == FEM_F32);
    cudaError_t e = cudaStreamEndCapture(m->cap, &graph);
    if (!rc && e != cudaSuccess) {
      fem_set_error("fem_pmg: V-cycle capture failed: %s", cudaGetErrorString(e));
      rc = FEM_ECUDA;
    }
  }
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc;
  }
  cudaError_t e = cudaGraphInstantiate(&m->vexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    m->vexec = nullptr;
    fem_set_error("fem_pmg: V-cycle graph instantiation failed: %s", cudaGetErrorString(e));
    return FEM_ECUDA;
  }
  return FEM_OK;
}

// ---------------------------------------------------------------- outer FCG (FP64)
struct FcgArgs {
  const double *b;
  double *x, *r, *z, *p, *y;
  const double *msk;
  int64_t N, n;
  double *sc, *partials;
  unsigned *counter;
  cudaGraphConditionalHandle handle;
};

// r = M (b - y) (y = A x); ||r||^2, ||M b||^2; p = 0, y = 0; decide start
__global__ void fcg_init_kernel(const FcgArgs a) {
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double m = a.msk[fem_node_of(i, a.N)];
    const double bi = m * a.b[i];
    const double ri = bi - m * a.y[i];
    a.r[i] = ri; a.p[i] = 0.0; a.y[i] = 0.0;
    v[0] += ri * ri; v[1] += bi * bi;
  }
  __shared__ double tot[2];
  if (fem_grid_sum<2>(v, a.partials, a.counter, tot) && threadIdx.x == 0) {
    double *s = a.sc;
    s[kFRr] = tot[0]; s[kFBb] = tot[1];
    s[kFPApOld] = 0.0; s[kFZy] = 0.0; s[kFIter] = 0.0; s[kFStatus] = 0.0;
    const bool done = !(tot[1] > 0.0) || tot[0] <= s[kFRtol2] * tot[1] || s[kFMaxit] < 1.0;
    cudaGraphSetConditional(a.handle, done ? 0u : 1u);
  }
}

// zy = z^T y (y = A p_old, zero at the start)
__global__ void fcg_dots_kernel(const FcgArgs a) {
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[0] += a.z[i] * a.y[i];
  __shared__ double tot[1];
  if (fem_grid_sum<1>(v, a.partials, a.counter, tot) && threadIdx.x == 0) a.sc[kFZy] = tot[0];
}

// p = z - (zy / pAp_old) p; y = 0; pr = p^T r
__global__ void fcg_dir_kernel(const FcgArgs a) {
  const double pAp = a.sc[kFPApOld];
  const double beta = pAp > 0.0 ? a.sc[kFZy] / pAp : 0.0;
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double pi = a.z[i] - beta * a.p[i];
    a.p[i] = pi;
    a.y[i] = 0.0;
    v[0] += pi * a.r[i];
  }
  __shared__ double tot[1];
  if (fem_grid_sum<1>(v, a.partials, a.counter, tot) && threadIdx.x == 0) a.sc[kFPr] = tot[0];
}

// after y = A p (pAp in sc[kFPAp]): alpha = pr / pAp; x += alpha p;
// r = M (r - alpha y); ||r||^2; decide
__global__ void fcg_update_kernel(const FcgArgs a) {
  const double pAp = a.sc[kFPAp];
  const double alpha = a.sc[kFPr] / pAp;
  const bool ok = pAp > 0.0 && isfinite(alpha);
  double v[1] = {0.0};
  if (ok) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
         i += (int64_t)gridDim.x * blockDim.x) {
      a.x[i] += alpha * a.p[i];
      const double ri = a.msk[fem_node_of(i, a.N)] * (a.r[i] - alpha * a.y[i]);
      a.r[i] = ri;
      v[0] += ri * ri;
    }
  }
  __shared__ double tot[1];
  if (fem_grid_sum<1>(v, a.partials, a.counter, tot) && threadIdx.x == 0) {
    double *s = a.sc;
    bool done = false;
    if (!ok) {
      s[kFStatus] = (double)FEM_EBREAKDOWN;
      done = true;
    } else {
      s[kFRr] = tot[0];
      s[kFPApOld] = pAp;
      s[kFIter] += 1.0;
      if (!isfinite(tot[0])) { s[kFStatus] = (double)FEM_EBREAKDOWN; done = true; }
      else if (tot[0] <= s[kFRtol2] * s[kFBb]) done = true;
      else if (s[kFIter] >= s[kFMaxit]) { s[kFStatus] = (double)FEM_ENOCONV; done = true; }
    }
    cudaGraphSetConditional(a.handle, done ? 0u : 1u);
  }
}

// preconditioner input / output between the FCG vectors and level 0
int precond_into_graph(fem_pmg *m, const FcgArgs &a, cudaStream_t s) {
  Level &L = m->lv[0];
  const int g = gridn(L.n);
  if (m->o.prec == FEM_F32) {
    to_f32_kernel<<<g, kT, 0, s>>>(a.r, L.v32.r, L.n);
    FEM_CHECK_LAUNCH();
    int rc = vcycle<float>(m, 0, s);
    if (rc) return rc;
    to_f64_kernel<<<g, kT, 0, s>>>(L.v32.z, a.z, L.n);
    FEM_CHECK_LAUNCH();
  } else {
    // level-0 r is the FCG residual itself; z written by the V-cycle
    int rc = vcycle<double>(m, 0, s);
    if (rc) return rc;
  }
  return FEM_OK;
}

void destroy_solve_graph(fem_pmg *m) {
  if (m->sexec) cudaGraphExecDestroy(m->sexec);
  m->sexec = nullptr;
}

int build_solve_graph(fem_pmg *m, const double *b, double *x) {
  destroy_solve_graph(m);
  if (!m->cap) {
    FEM_CUDA_TRY(cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking));
    FEM_CUDA_TRY(cudaStreamCreateWithFlags(&m->cap2, cudaStreamNonBlocking));
  }
  Level &L = m->lv[0];
  int rc = FEM_OK;
  cudaError_t e = cudaSuccess;
  cudaGraph_t graph = nullptr;
  {
    StreamSwap sw(m, m->cap);
    FEM_CUDA_TRY(cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeRelaxed));
    do {
      cudaStreamCaptureStatus st;
      const cudaGraphNode_t *deps = nullptr;
      size_t ndeps = 0;
      cudaGraphConditionalHandle h = 0;
      e = cudaStreamGetCaptureInfo(m->cap, &st, nullptr, &graph, nullptr, nullptr, nullptr);
      if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
      if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
      FcgArgs a;
      a.b = b; a.x = x; a.r = m->x_r; a.z = m->x_z; a.p = m->x_p; a.y = m->x_y;
      a.msk = L.v64.msk; a.N = L.N; a.n = L.n; a.sc = m->sc; a.partials = m->partials;
      a.counter = m->counter; a.handle = h;
      const int g = gridn(L.n);
      fill_kernel<double><<<g, kT, 0, m->cap>>>(m->x_y, 0.0, L.n);
      if ((rc = apply(L, x, m->x_y, nullptr))) break;
      fcg_init_kernel<<<g, kT, 0, m->cap>>>(a);
      e = cudaStreamGetCaptureInfo(m->cap, &st, nullptr, &graph, &deps, nullptr, &ndeps);
      if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t cnode;
      if ((e = cudaGraphAddNode(&cnode, graph, deps, nullptr, ndeps, &cp)) != cudaSuccess) { rc = FEM_ECUDA; break; }
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      e = cudaStreamUpdateCaptureDependencies(m->cap, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
      if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
      // loop body on the second capture stream
      {
        StreamSwap sw2(m, m->cap2);
        e = cudaStreamBeginCaptureToGraph(m->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) { rc = FEM_ECUDA; break; }
        rc = precond_into_graph(m, a, m->cap2);                // z = B(r)
        if (!rc) {
          fcg_dots_kernel<<<g, kT, 0, m->cap2>>>(a);            // zy = z^T A p_old
          fcg_dir_kernel<<<g, kT, 0, m->cap2>>>(a);             // p, pr, y = 0
          rc = apply(L, m->x_p, m->x_y, m->sc + kFPAp);         // y = A p, pAp
        }
        if (!rc) fcg_update_kernel<<<g, kT, 0, m->cap2>>>(a);   // x, r, decide
        cudaGraph_t tmp;
        cudaError_t e2 = cudaStreamEndCapture(m->cap2, &tmp);
        if (!rc && e2 != cudaSuccess) { e = e2; rc = FEM_ECUDA; }
      }
    } while (0);
    cudaGraph_t g2 = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(m->cap, &g2);
    if (rc == FEM_OK && e3 != cudaSuccess) { rc = FEM_ECUDA; e = e3; }
    graph = g2;
  }
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (rc == FEM_ECUDA) fem_set_error("fem_pmg_solve: building the CUDA graph failed: %s", cudaGetErrorString(e));
    return rc;
  }
  e = cudaGraphInstantiate(&m->sexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    m->sexec = nullptr;
    fem_set_error("fem_pmg_solve: graph instantiation failed: %s", cudaGetErrorString(e));
    return FEM_ECUDA;
  }
  m->g_b = b; m->g_x = x;
  return FEM_OK;
}

// lmax of D^-1 A on level l by power iteration (FP64, setup; synchronizes)
int estimate_lmax(fem_pmg *m, int l, double *out) {
  Level &L = m->lv[l];
  cudaStream_t s = m->stream;
  LevelVecs<double> &V = L.v64;
  const int g = gridn(L.n);
  power_start_kernel<<<g, kT, 0, s>>>(V.msk, L.N, L.n, V.d, V.y);
  FEM_CHECK_LAUNCH();
  for (int k = 0; k < m->o.power_its; k++) {
    int rc = apply(L, V.d, V.y, nullptr);
    if (rc) return rc;
    power_step_kernel<<<g, kT, 0, s>>>(V.dinv, V.d, V.y, L.n, m->sc, m->partials, m->counter);
    power_scale_kernel<<<g, kT, 0, s>>>(V.d, L.n, m->sc);
    FEM_CHECK_LAUNCH();
  }
  int rc = apply(L, V.d, V.y, m->sc + kSNorm);   // v^T A v
  if (rc) return rc;
  power_den_kernel<<<g, kT, 0, s>>>(V.d, V.dinv, L.n, m->sc, m->partials, m->counter);
  FEM_CHECK_LAUNCH();
  double h[kNumScalars];
  FEM_CUDA_TRY(cudaMemcpyAsync(h, m->sc, sizeof(h), cudaMemcpyDeviceToHost, s));
  FEM_CUDA_TRY(cudaStreamSynchronize(s));
  if (!(h[kSDen] > 0.0) || !isfinite(h[kSNorm])) {
    fem_set_error("fem_pmg_create: power iteration on level %d failed", l);
    return FEM_EBREAKDOWN;
  }
  *out = h[kSNorm] / h[kSDen];
  return FEM_OK;
}

// I[i][a]: the order-pc Gauss-Lobatto Lagrange basis at the order-pf nodes
int interpolation_1d(int pc, int pf, double *I) {
  BasisTables tf;
  if (fem_build_tables(pf, pf + 1, FEM_LOBATTO, &tf) != FEM_OK) return FEM_EINVAL;
  return fem_basis_interp(pc, tf.z, pf + 1, I);
}

}  // namespace

extern "C" fem_status fem_pmg_create(fem_op *const *levels, int nlevels, const fem_pmg_opts *opts,
                                     fem_pmg **out) {
  if (!out || !levels || nlevels < 1 || nlevels > 8) {
    fem_set_error("fem_pmg_create: need 1..8 levels");
    return FEM_EINVAL;
  }
  *out = nullptr;
  fem_pmg_opts o = {4, 0.1, 1.1, 20, 30, FEM_F64};
  if (opts) o = *opts;
  if (o.cheb_degree < 1 || !(o.cheb_lo > 0.0) || !(o.cheb_hi > o.cheb_lo) || o.power_its < 1 ||
      o.coarse_its < 1 || (o.prec != FEM_F64 && o.prec != FEM_F32)) {
    fem_set_error("fem_pmg_create: invalid options");
    return FEM_EINVAL;
  }
  for (int l = 0; l < nlevels; l++) {
    const fem_op *op = levels[l];
    if (!op || op->kind != levels[0]->kind || op->ncomp != levels[0]->ncomp || op->E != levels[0]->E ||
        op->stream() != levels[0]->stream() || (o.prec == FEM_F32 && !op->d_qdata32) ||
        (l > 0 && op->P >= levels[l - 1]->P)) {
      fem_set_error("fem_pmg_create: level %d must have the kind, ncomp, element count and stream "
                    "of level 0, an order below level %d's%s", l, l - 1,
                    o.prec == FEM_F32 ? ", and FEM_F32 data" : "");
      return FEM_EINVAL;
    }
  }
  fem_pmg *m = new fem_pmg();
  m->o = o;
  m->stream = levels[0]->stream();
  m->lv.resize(nlevels);
  auto dalloc = [&](void **p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); return false; }
    m->allocs.push_back(*p);
    return true;
  };
  bool ok = dalloc((void **)&m->sc, sizeof(double) * kNumScalars) &&
            dalloc((void **)&m->partials, sizeof(double) * 4 * FEM_MAX_BLOCKS) &&
            dalloc((void **)&m->counter, sizeof(unsigned) * 4);
  float *cnt = nullptr;
  for (int l = 0; ok && l < nlevels; l++) {
    Level &L = m->lv[l];
    L.op = levels[l];
    L.P = L.op->P; L.N = L.op->N; L.E = L.op->E; L.n = L.op->N * L.op->ncomp;
    L.Pc = l + 1 < nlevels ? levels[l + 1]->P : 0;
    const size_t n = (size_t)L.n, N = (size_t)L.N;
    LevelVecs<double> &V = L.v64;
    ok = dalloc((void **)&V.r, 8 * n) && dalloc((void **)&V.z, 8 * n) && dalloc((void **)&V.t, 8 * n) &&
         dalloc((void **)&V.d, 8 * n) && dalloc((void **)&V.y, 8 * n) && dalloc((void **)&V.dinv, 8 * n) &&
         dalloc((void **)&V.wm, 8 * N) && dalloc((void **)&V.msk, 8 * N);
    if (ok && o.prec == FEM_F32) {
      LevelVecs<float> &W = L.v32;
      ok = dalloc((void **)&W.r, 4 * n) && dalloc((void **)&W.z, 4 * n) && dalloc((void **)&W.t, 4 * n) &&
           dalloc((void **)&W.d, 4 * n) && dalloc((void **)&W.y, 4 * n) && dalloc((void **)&W.dinv, 4 * n) &&
           dalloc((void **)&W.wm, 4 * N) && dalloc((void **)&W.msk, 4 * N);
    }
    if (ok && L.Pc) {
      ok = dalloc((void **)&V.I, 8 * L.P * L.Pc) && (o.prec != FEM_F32 || dalloc((void **)&L.v32.I, 4 * L.P * L.Pc));
    }
  }
  if (ok) ok = cudaMalloc(&cnt, sizeof(float) * (size_t)m->lv[0].N) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    if (cnt) cudaFree(cnt);
    fem_pmg_destroy(m);
    fem_set_error("fem_pmg_create: device allocation failed");
    return FEM_ENOMEM;
  }
  cudaStream_t s = m->stream;
  int rc = FEM_OK;
  for (int l = 0; l < nlevels && rc == FEM_OK; l++) {
    Level &L = m->lv[l];
    const fem_mesh *mesh = L.op->mesh;
    if (cudaMemsetAsync(cnt, 0, sizeof(float) * (size_t)L.N, s) != cudaSuccess) { rc = FEM_ECUDA; break; }
    count_kernel<<<gridn(L.E * L.P * L.P * L.P), kT, 0, s>>>(mesh->d_elem_nodes, L.E * L.P * L.P * L.P, cnt);
    level_setup_kernel<double><<<gridn(L.N), kT, 0, s>>>(cnt, mesh->d_dirichlet, L.op->d_diag, L.N,
                                                         L.op->ncomp, L.v64.wm, L.v64.msk, L.v64.dinv);
    if (o.prec == FEM_F32)
      level_setup_kernel<float><<<gridn(L.N), kT, 0, s>>>(cnt, mesh->d_dirichlet, L.op->d_diag, L.N,
                                                          L.op->ncomp, L.v32.wm, L.v32.msk, L.v32.dinv);
    if (cudaGetLastError() != cudaSuccess) { rc = FEM_ECUDA; break; }
    if (L.Pc) {
      double I[FEM_MAX_P * FEM_MAX_P];
      if (interpolation_1d(L.Pc - 1, L.P - 1, I) != FEM_OK) { rc = FEM_EINVAL; break; }
      float I32[FEM_MAX_P * FEM_MAX_P];
      for (int i = 0; i < L.P * L.Pc; i++) I32[i] = (float)I[i];
      if (cudaMemcpyAsync(L.v64.I, I, sizeof(double) * L.P * L.Pc, cudaMemcpyHostToDevice, s) != cudaSuccess ||
          (o.prec == FEM_F32 &&
           cudaMemcpyAsync(L.v32.I, I32, sizeof(float) * L.P * L.Pc, cudaMemcpyHostToDevice, s) != cudaSuccess) ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        rc = FEM_ECUDA;
        break;
      }
    }
  }
  if (rc == FEM_OK && (cudaMemsetAsync(m->counter, 0, sizeof(unsigned) * 4, s) != cudaSuccess ||
                       cudaMemsetAsync(m->sc, 0, sizeof(double) * kNumScalars, s) != cudaSuccess))
    rc = FEM_ECUDA;
  if (rc == FEM_ECUDA) fem_set_error("fem_pmg_create: setup failed: %s", cudaGetErrorString(cudaGetLastError()));
  for (int l = 0; rc == FEM_OK && l + 1 < nlevels; l++) rc = estimate_lmax(m, l, &m->lv[l].lmax);
  cudaStreamSynchronize(s);
  cudaFree(cnt);
  if (rc) {
    fem_pmg_destroy(m);
    return rc;
  }
  *out = m;
  return FEM_OK;
}

extern "C" fem_status fem_pmg_destroy(fem_pmg *m) {
  if (!m) return FEM_OK;
  if (m->vexec) cudaGraphExecDestroy(m->vexec);
  destroy_solve_graph(m);
  if (m->cap) cudaStreamDestroy(m->cap);
  if (m->cap2) cudaStreamDestroy(m->cap2);
  for (void *p : m->allocs) cudaFree(p);
  delete m;
  return FEM_OK;
}

extern "C" fem_status fem_pmg_get_lmax(const fem_pmg *m, int level, double *lmax) {
  if (!m || !lmax || level < 0 || level >= (int)m->lv.size()) {
    fem_set_error("fem_pmg_get_lmax: invalid arguments");
    return FEM_EINVAL;
  }
  *lmax = m->lv[level].lmax;
  return FEM_OK;
}

extern "C" fem_status fem_pmg_set_lmax(fem_pmg *m, int level, double lmax) {
  if (!m || level < 0 || level + 1 >= (int)m->lv.size() || !(lmax > 0.0) || !isfinite(lmax)) {
    fem_set_error("fem_pmg_set_lmax: need a smoothed level (not the coarsest) and lmax > 0");
    return FEM_EINVAL;
  }
  m->lv[level].lmax = lmax;
  if (m->vexec) { cudaGraphExecDestroy(m->vexec); m->vexec = nullptr; }
  destroy_solve_graph(m);
  return FEM_OK;
}

extern "C" fem_status fem_pmg_prolong(fem_pmg *m, int level, const double *xc, double *xf) {
  if (!m || !xc || !xf || level < 0 || level + 1 >= (int)m->lv.size()) {
    fem_set_error("fem_pmg_prolong: invalid arguments");
    return FEM_EINVAL;
  }
  Level &F = m->lv[level];
  FEM_CUDA_TRY(cudaMemsetAsync(xf, 0, sizeof(double) * (size_t)F.n, m->stream));
  return launch_prolong<double>(m, level, xc, xf, m->stream);
}

extern "C" fem_status fem_pmg_restrict(fem_pmg *m, int level, const double *rf, double *rc) {
  if (!m || !rf || !rc || level < 0 || level + 1 >= (int)m->lv.size()) {
    fem_set_error("fem_pmg_restrict: invalid arguments");
    return FEM_EINVAL;
  }
  Level &C = m->lv[level + 1];
  FEM_CUDA_TRY(cudaMemsetAsync(rc, 0, sizeof(double) * (size_t)C.n, m->stream));
  return launch_restrict<double>(m, level, rf, rc, m->stream);
}

extern "C" fem_status fem_pmg_vcycle(fem_pmg *m, const double *r, double *z) {
  if (!m || !r || !z) {
    fem_set_error("fem_pmg_vcycle: invalid arguments");
    return FEM_EINVAL;
  }
  Level &L = m->lv[0];
  cudaStream_t s = m->stream;
  int rc = build_vcycle_graph(m);
  if (rc) return rc;
  if (m->o.prec == FEM_F32) {
    to_f32_kernel<<<gridn(L.n), kT, 0, s>>>(r, L.v32.r, L.n);
    FEM_CHECK_LAUNCH();
  } else {
    FEM_CUDA_TRY(cudaMemcpyAsync(L.v64.r, r, sizeof(double) * (size_t)L.n, cudaMemcpyDeviceToDevice, s));
  }
  FEM_CUDA_TRY(cudaGraphLaunch(m->vexec, s));
  if (m->o.prec == FEM_F32) {
    to_f64_kernel<<<gridn(L.n), kT, 0, s>>>(L.v32.z, z, L.n);
    FEM_CHECK_LAUNCH();
  } else {
    FEM_CUDA_TRY(cudaMemcpyAsync(z, L.v64.z, sizeof(double) * (size_t)L.n, cudaMemcpyDeviceToDevice, s));
  }
  return FEM_OK;
}

extern "C" fem_status fem_pmg_solve(fem_pmg *m, const double *b, double *x, const fem_cg_opts *o,
                                    fem_cg_stats *st) {
  if (!m || !b || !x || !o || b == x || !(o->rtol > 0.0) || o->maxit < 1) {
    fem_set_error("fem_pmg_solve: invalid arguments (need rtol > 0, maxit >= 1)");
    return FEM_EINVAL;
  }
  Level &L = m->lv[0];
  cudaStream_t s = m->stream;
  if (!m->x_p) {
    const size_t bytes = sizeof(double) * (size_t)L.n;
    auto dalloc = [&](double **p) -> bool {
      if (cudaMalloc((void **)p, bytes) != cudaSuccess) { cudaGetLastError(); *p = nullptr; return false; }
      m->allocs.push_back(*p);
      return true;
    };
    bool ok = true;
    if (m->o.prec == FEM_F64) {
      // the FP64 V-cycle reads level 0's r and writes its z: the FCG uses them
      m->x_r = L.v64.r;
      m->x_z = L.v64.z;
    } else {
      ok = dalloc(&m->x_r) && dalloc(&m->x_z);
    }
    ok = ok && dalloc(&m->x_y) && dalloc(&m->x_p);
    if (!ok) {
      fem_set_error("fem_pmg_solve: allocation failed");
      return FEM_ENOMEM;
    }
  }
  double h[kNumScalars] = {0};
  h[kFRtol2] = o->rtol * o->rtol;
  h[kFMaxit] = (double)o->maxit;
  FEM_CUDA_TRY(cudaMemcpyAsync(m->sc + kFRtol2, h + kFRtol2, sizeof(double) * 2, cudaMemcpyHostToDevice, s));
  if (!m->sexec || m->g_b != b || m->g_x != x) {
    FEM_CUDA_TRY(cudaStreamSynchronize(s));
    int rc = build_solve_graph(m, b, x);
    if (rc) return rc;
  }
  FEM_CUDA_TRY(cudaGraphLaunch(m->sexec, s));
  FEM_CUDA_TRY(cudaMemcpyAsync(h, m->sc, sizeof(h), cudaMemcpyDeviceToHost, s));
  FEM_CUDA_TRY(cudaStreamSynchronize(s));
  int status = (int)h[kFStatus];
  if (st) {
    st->iterations = (int)h[kFIter];
    st->outer = 0;
    st->status = status;
    st->rnorm = sqrt(h[kFRr]);
    st->bnorm = sqrt(h[kFBb]);
    st->true_rel = h[kFBb] > 0.0 ? sqrt(h[kFRr] / h[kFBb]) : 0.0;
    st->fallback = 0;
  }
  return status;
}
