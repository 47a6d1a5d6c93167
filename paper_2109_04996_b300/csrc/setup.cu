// Operator setup on the GPU, FP64 throughout:
//  * qdata (the D of the decomposition, section "libCEED"): at every
//    quadrature point the Jacobian J = dx/dr of the isoparametric map is the
//    sum-factorized gradient of the node coordinates; D stores w det J kappa
//    (mass) or the symmetric w det J kappa J^{-1} J^{-T} (diffusion), with
//    J^{-1} = adj(J) / det J.  kappa(x) is evaluated at the physical point.
//  * the diagonal of the assembled operator: diag_i = sum over the 3x3 entries
//    of D of 3-stage contractions of products of 1D tables, then a scatter-add.
//  * the manufactured load b_i = int phi_i f dV.
#include <math.h>

#include "fem_internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

struct GeomParams {
  const int32_t *elem_nodes;
  const double *xyz;   // [3][N]
  int64_t N, E;
  const double *B, *Dq, *w;  // [Q][P], [Q][Q], [Q]
  const double *rff;   // [M][4] or null
  int M;
  double sigma;
  int kind;            // FEM_MASS / FEM_DIFFUSION
  int mode;            // 0 = qdata, 1 = load b (f = sin sin sin * scale)
  double scale;
  double *qdata;       // [E][nd][Q^3]
  double *b;           // [N]
};

// One element per block, q x q threads (rounded up to whole warps).
template <int P, int Q>
__global__ void fem_geometry_kernel(const GeomParams prm) {
  constexpr int Q2 = Q * Q, Q3 = Q2 * Q, P2 = P * P, P3 = P2 * P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *sB = reinterpret_cast<double *>(smem_raw);
  double *sD = sB + Q * P;
  double *sw = sD + Q * Q;
  double *su = sw + Q;      // [Q3]
  double *sv = su + Q3;     // [Q3]
  double *sJ = sv + Q3;     // [9][Q3], J[d][c] = dx_d / dr_c
  double *sX = sJ + 9 * Q3; // [3][Q3]
  for (int i = threadIdx.x; i < Q * P; i += blockDim.x) sB[i] = prm.B[i];
  for (int i = threadIdx.x; i < Q * Q; i += blockDim.x) sD[i] = prm.Dq[i];
  for (int i = threadIdx.x; i < Q; i += blockDim.x) sw[i] = prm.w[i];
  __syncthreads();
  const bool live = threadIdx.x < Q2;
  const int tx = live ? threadIdx.x % Q : 0, ty = live ? threadIdx.x / Q : 0;
  const bool own = live && tx < P && ty < P;

  for (int64_t e = blockIdx.x; e < prm.E; e += gridDim.x) {
    const int32_t *en = prm.elem_nodes + e * P3;
    for (int d = 0; d < 3; d++) {
      double r[P], tq[Q];
#pragma unroll
      for (int k = 0; k < P; k++) r[k] = own ? prm.xyz[d * prm.N + en[tx + P * ty + P2 * k]] : 0.0;
#pragma unroll
      for (int kq = 0; kq < Q; kq++) {
        double s = 0;
#pragma unroll
        for (int k = 0; k < P; k++) s += sB[kq * P + k] * r[k];
        tq[kq] = s;
      }
      if (own)
        for (int kq = 0; kq < Q; kq++) su[(kq * Q + ty) * Q + tx] = tq[kq];
      __syncthreads();
      if (live && tx < P)
        for (int kq = 0; kq < Q; kq++) {
          double s = 0;
          for (int j = 0; j < P; j++) s += sB[ty * P + j] * su[(kq * Q + j) * Q + tx];
          sv[(kq * Q + ty) * Q + tx] = s;
        }
      __syncthreads();
      if (live)
        for (int kq = 0; kq < Q; kq++) {
          double s = 0;
          for (int i = 0; i < P; i++) s += sB[tx * P + i] * sv[(kq * Q + ty) * Q + i];
          tq[kq] = s;
          su[(kq * Q + ty) * Q + tx] = s;
          sX[d * Q3 + (kq * Q + ty) * Q + tx] = s;
        }
      __syncthreads();
      if (live)
        for (int kq = 0; kq < Q; kq++) {
          double gx = 0, gy = 0, gz = 0;
          for (int m = 0; m < Q; m++) {
            gx += sD[tx * Q + m] * su[(kq * Q + ty) * Q + m];
            gy += sD[ty * Q + m] * su[(kq * Q + m) * Q + tx];
            gz += sD[kq * Q + m] * tq[m];
          }
          const int pt = (kq * Q + ty) * Q + tx;
          sJ[(3 * d + 0) * Q3 + pt] = gx;
          sJ[(3 * d + 1) * Q3 + pt] = gy;
          sJ[(3 * d + 2) * Q3 + pt] = gz;
        }
      __syncthreads();
    }
    // pointwise data at this thread's column of quadrature points
    double tq[Q];
    if (live) {
      for (int kq = 0; kq < Q; kq++) {
        const int pt = (kq * Q + ty) * Q + tx;
        double J[3][3];
        for (int a = 0; a < 3; a++)
          for (int c = 0; c < 3; c++) J[a][c] = sJ[(3 * a + c) * Q3 + pt];
        // cofactors: C[a][c] = (-1)^{a+c} minor(a,c);  adj = C^T
        double C00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        double C01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        double C02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        double C10 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        double C11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        double C12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        double C20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        double C21 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        double C22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        double det = J[0][0] * C00 + J[0][1] * C01 + J[0][2] * C02;
        double x0 = sX[pt], x1 = sX[Q3 + pt], x2 = sX[2 * Q3 + pt];
        double kap = 1.0;
        if (prm.rff) {
          double s = 0.0;
          for (int m = 0; m < prm.M; m++) {
            const double *f = prm.rff + 4 * m;
            s += cos(f[0] * x0 + f[1] * x1 + f[2] * x2 + f[3]);
          }
          kap = exp(prm.sigma * sqrt(2.0 / prm.M) * s);
        }
        const double wdet = sw[tx] * sw[ty] * sw[kq] * det;
        if (prm.mode == 0) {
          double *out = prm.qdata + e * (int64_t)((prm.kind == FEM_DIFFUSION ? 6 : 1) * Q3) + pt;
          if (prm.kind == FEM_MASS) {
            out[0] = wdet * kap;
          } else {
            // J^{-1} J^{-T} = adj adj^T / det^2; adj[i][m] = C[m][i]
            const double c = sw[tx] * sw[ty] * sw[kq] * kap / det;
            // (adj adj^T)[i][k] = sum_m C[m][i] C[m][k]
            out[0 * Q3] = c * (C00 * C00 + C10 * C10 + C20 * C20);
            out[1 * Q3] = c * (C01 * C01 + C11 * C11 + C21 * C21);
            out[2 * Q3] = c * (C02 * C02 + C12 * C12 + C22 * C22);
            out[3 * Q3] = c * (C01 * C02 + C11 * C12 + C21 * C22);
            out[4 * Q3] = c * (C00 * C02 + C10 * C12 + C20 * C22);
            out[5 * Q3] = c * (C00 * C01 + C10 * C11 + C20 * C21);
          }
        } else {
          const double f = prm.scale * sin(kPi * x0) * sin(kPi * x1) * sin(kPi * x2);
          tq[kq] = wdet * f;
        }
      }
    }
    if (prm.mode == 1) {
      // b_e = B^T (w det J f): transposed interpolation, then scatter-add
      if (live)
        for (int kq = 0; kq < Q; kq++) su[(kq * Q + ty) * Q + tx] = tq[kq];
      __syncthreads();
      if (live && tx < P)
        for (int kq = 0; kq < Q; kq++) {
          double s = 0;
          for (int m = 0; m < Q; m++) s += sB[m * P + tx] * su[(kq * Q + ty) * Q + m];
          sv[(kq * Q + ty) * Q + tx] = s;
        }
      __syncthreads();
      if (own) {
        for (int kq = 0; kq < Q; kq++) {
          double s = 0;
          for (int m = 0; m < Q; m++) s += sB[m * P + ty] * sv[(kq * Q + m) * Q + tx];
          tq[kq] = s;
        }
        for (int k = 0; k < P; k++) {
          double s = 0;
          for (int kq = 0; kq < Q; kq++) s += sB[kq * P + k] * tq[kq];
          atomicAdd(&prm.b[en[tx + P * ty + P2 * k]], s);
        }
      }
    }
    __syncthreads();
  }
}

// Diagonal: for each stored entry D_ab (a, b in {x, y, z}) the element
// contribution at node (i, j, k) is sum_q D_ab(q) F_a,b^x[q1][i] F^y[q2][j]
// F^z[q3][k] with F^d[q][i] = T_a^d[q][i] T_b^d[q][i], T_a^d = G (the 1D
// derivative table) when a == d, else B.  Three contraction stages, one
// element per block.
struct DiagParams {
  const int32_t *elem_nodes;
  int64_t E;
  const double *B, *G;   // [Q][P] each
  const double *qdata;
  int kind;
  double *diag;          // [N]
};

template <int P, int Q>
__global__ void fem_diagonal_kernel(const DiagParams prm) {
  constexpr int Q2 = Q * Q, Q3 = Q2 * Q, P2 = P * P, P3 = P2 * P;
  __shared__ double sB[Q * P], sG[Q * P];
  __shared__ double s1[Q * Q * P];  // [c][jq][iq]  after the z stage
  __shared__ double s2[P * P * Q];  // [c][b][iq]   after the y stage
  for (int i = threadIdx.x; i < Q * P; i += blockDim.x) { sB[i] = prm.B[i]; sG[i] = prm.G[i]; }
  __syncthreads();
  const int nterm = prm.kind == FEM_DIFFUSION ? 6 : 1;
  // (a, b) of the stored components (11, 22, 33, 23, 13, 12), weight 2 off-diagonal
  const int ta[6] = {0, 1, 2, 1, 0, 0}, tb[6] = {0, 1, 2, 2, 2, 1};
  const double tw[6] = {1, 1, 1, 2, 2, 2};
  for (int64_t e = blockIdx.x; e < prm.E; e += gridDim.x) {
    const double *qd = prm.qdata + e * (int64_t)(nterm * Q3);
    double acc = 0.0;  // thread -> node (i, j, k) = threadIdx.x < P3
    for (int tm = 0; tm < nterm; tm++) {
      const int a = ta[tm], b = tb[tm];
      auto F = [&](int d, int q, int i) -> double {
        if (prm.kind == FEM_MASS) return sB[q * P + i] * sB[q * P + i];
        const double u = (a == d) ? sG[q * P + i] : sB[q * P + i];
        const double v = (b == d) ? sG[q * P + i] : sB[q * P + i];
        return u * v;
      };
      // z stage: s1[c][jq][iq] = sum_kq D(iq,jq,kq) F^z[kq][c]
      for (int t = threadIdx.x; t < P * Q2; t += blockDim.x) {
        const int c = t / Q2, jq = (t / Q) % Q, iq = t % Q;
        double s = 0;
        for (int kq = 0; kq < Q; kq++) s += qd[tm * Q3 + (kq * Q + jq) * Q + iq] * F(2, kq, c);
        s1[t] = s;
      }
      __syncthreads();
      // y stage: s2[c][b][iq] = sum_jq F^y[jq][b] s1[c][jq][iq]
      for (int t = threadIdx.x; t < P2 * Q; t += blockDim.x) {
        const int c = t / (P * Q), bb = (t / Q) % P, iq = t % Q;
        double s = 0;
        for (int jq = 0; jq < Q; jq++) s += F(1, jq, bb) * s1[(c * Q + jq) * Q + iq];
        s2[t] = s;
      }
      __syncthreads();
      // x stage
      if (threadIdx.x < P3) {
        const int c = threadIdx.x / P2, bb = (threadIdx.x / P) % P, aa = threadIdx.x % P;
        double s = 0;
        for (int iq = 0; iq < Q; iq++) s += F(0, iq, aa) * s2[(c * P + bb) * Q + iq];
        acc += tw[tm] * s;
      }
      __syncthreads();
    }
    if (threadIdx.x < P3) atomicAdd(&prm.diag[prm.elem_nodes[e * P3 + threadIdx.x]], acc);
  }
}

template <int P, int Q>
int launch_geometry(fem_op *op, int mode, double scale, double *b) {
  const fem_mesh *m = op->mesh;
  GeomParams prm;
  prm.elem_nodes = m->d_elem_nodes; prm.xyz = m->d_xyz; prm.N = m->N; prm.E = m->E;
  prm.B = op->d_B; prm.Dq = op->d_Dq;
  prm.w = op->d_B - TAB_B + TAB_W;
  prm.rff = op->d_rff; prm.M = op->M; prm.sigma = op->sigma;
  prm.kind = op->kind; prm.mode = mode; prm.scale = scale;
  prm.qdata = op->d_qdata; prm.b = b;
  constexpr int Q3 = Q * Q * Q;
  const size_t smem = sizeof(double) * (Q * P + Q * Q + Q + 2 * Q3 + 12 * Q3);
  auto kern = fem_geometry_kernel<P, Q>;
  FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int nt = ((Q * Q + 31) / 32) * 32;
  int64_t grid = m->E < 148 * 16 ? m->E : 148 * 16;
  if (grid < 1) return FEM_OK;
  kern<<<(unsigned)grid, nt, smem, op->stream()>>>(prm);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

template <int P, int Q>
int launch_diagonal(fem_op *op) {
  DiagParams prm;
  prm.elem_nodes = op->mesh->d_elem_nodes; prm.E = op->E;
  prm.B = op->d_B; prm.G = op->d_B - TAB_B + TAB_G;
  prm.qdata = op->d_qdata; prm.kind = op->kind; prm.diag = op->d_diag;
  int nt = P * P * P;
  nt = ((nt + 31) / 32) * 32;
  if (nt < 128) nt = 128;
  int64_t grid = op->E < 148 * 16 ? op->E : 148 * 16;
  if (grid < 1) return FEM_OK;
  fem_diagonal_kernel<P, Q><<<(unsigned)grid, nt, 0, op->stream()>>>(prm);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

template <int P>
int geom_q(fem_op *op, int mode, double scale, double *b) {
  if (op->Q == P) return launch_geometry<P, P>(op, mode, scale, b);
  if constexpr (P + 1 <= FEM_MAX_Q) {
    if (op->Q == P + 1) return launch_geometry<P, P + 1>(op, mode, scale, b);
  }
  fem_set_error("setup: unsupported q");
  return FEM_EINVAL;
}

template <int P>
int diag_q(fem_op *op) {
  if (op->Q == P) return launch_diagonal<P, P>(op);
  if constexpr (P + 1 <= FEM_MAX_Q) {
    if (op->Q == P + 1) return launch_diagonal<P, P + 1>(op);
  }
  fem_set_error("diagonal: unsupported q");
  return FEM_EINVAL;
}

int geom_dispatch(fem_op *op, int mode, double scale, double *b) {
  switch (op->P) {
    case 2: return geom_q<2>(op, mode, scale, b);
    case 3: return geom_q<3>(op, mode, scale, b);
    case 4: return geom_q<4>(op, mode, scale, b);
    case 5: return geom_q<5>(op, mode, scale, b);
    case 6: return geom_q<6>(op, mode, scale, b);
    case 7: return geom_q<7>(op, mode, scale, b);
    case 8: return geom_q<8>(op, mode, scale, b);
    case 9: return geom_q<9>(op, mode, scale, b);
  }
  fem_set_error("setup: unsupported P");
  return FEM_EINVAL;
}

}  // namespace

int fem_setup_qdata(fem_op *op) { return geom_dispatch(op, 0, 1.0, nullptr); }

int fem_launch_rhs(fem_op *op, int which, double *b) {
  FEM_CUDA_TRY(cudaMemsetAsync(b, 0, sizeof(double) * op->N, op->stream()));
  return geom_dispatch(op, 1, which == 1 ? 3.0 * kPi * kPi : 1.0, b);
}

int fem_setup_diagonal(fem_op *op) {
  FEM_CUDA_TRY(cudaMemsetAsync(op->d_diag, 0, sizeof(double) * op->N, op->stream()));
  switch (op->P) {
    case 2: return diag_q<2>(op);
    case 3: return diag_q<3>(op);
    case 4: return diag_q<4>(op);
    case 5: return diag_q<5>(op);
    case 6: return diag_q<6>(op);
    case 7: return diag_q<7>(op);
    case 8: return diag_q<8>(op);
    case 9: return diag_q<9>(op);
  }
  fem_set_error("diagonal: unsupported P");
  return FEM_EINVAL;
}
