// Element body of the fused diffusion apply for trilinear elements (p = 1,
// any Gauss rule with q points per direction), one thread per element.
//
// The operator is the same y = G^T B^T D B G x as in the other bodies
// (section "libCEED": operator decomposition).  What changes is the order of
// the 1D contractions: for p = 1 the reference derivative of the 1D basis is
// the constant -1/2 (vertex 0) and +1/2 (vertex 1), so the x-derivative of
// the trilinear interpolant does not depend on x.  Per direction the
// gradient is therefore the difference of the two vertex faces followed by
// two 2 x q interpolations, and its transpose is a sum over the q points of
// the line followed by the two transposed interpolations:
//
//   gx[j][k] = sum_b B[j][b] sum_c H[k][c] (u[1][b][c] - u[0][b][c])
//   gy[i][k] = sum_a B[i][a] sum_c H[k][c] (u[a][1][c] - u[a][0][c])
//   gz[i][j] = sum_a B[i][a] sum_b H[j][b] (u[a][b][1] - u[a][b][0])
//
// (u[a][b][c] = x at vertex a + 2b + 4c, B the q x 2 interpolation table,
// H = B / 2), then v = D grad u at every quadrature point (i, j, k), summed
// along the direction the gradient component does not depend on:
//
//   Sx[j][k] = sum_i vx(i, j, k),  Sy[i][k] = sum_j vy,  Sz[i][j] = sum_k vz,
//
// and y[a][b][c] += (2a-1) rx[b][c] + (2b-1) ry[a][c] + (2c-1) rz[a][b] with
// rx[b][c] = sum_j B[j][b] sum_k H[k][c] Sx[j][k] (likewise ry, rz).  In Sx
// the term D00 gx has gx constant along i, so it is gx[j][k] times the line
// sum of D00 over i, computed once at set-up (fem_op::d_qsum; likewise D11
// in Sy, D22 in Sz): per point only the three off-diagonal entries are read
// and applied.
//
// At q = 3 this takes about 400 FP64 operations per element (737 flops)
// against about 1050 lane-slots of the slab body: the B300's FP64 pipe
// (2 FMA per SM per clock) is the bound of the FP64 apply, so the
// instruction count is what matters.  Everything stays in registers; qdata is
// read in quadrature-point order, so a thread's consecutive loads of one
// component share sectors.
#pragma once
#include "apply_kernel.cuh"

namespace fem_apply {

template <typename T, int Q>
struct TrilinearTables {
  T B[Q][2];   // B[k][a]: 1D vertex basis a at Gauss point k
  T H[Q][2];   // B / 2 (exact: a power of two)
};

template <typename T, int Q>
struct TrilinearParams {
  ApplyParams<T> a;
  TrilinearTables<T, Q> t;
  const T *qsum;   // [E][3][Q^2] line sums of D00, D11, D22 (fem_op::d_qsum)
};

constexpr int kTrilinearThreads = 128;

// Element e: y += A_e x_e (all components) and this thread's share of x.y.
template <typename T, int Q>
__device__ __forceinline__ void trilinear_element(const ApplyParams<T> &prm,
                                                  const TrilinearTables<T, Q> &t,
                                                  const T *qsum, int64_t e, DotAcc<T> &dl) {
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q;
  int id[8];
  {
    const int4 *ip = reinterpret_cast<const int4 *>(prm.elem_nodes + e * 8);
    const int4 i0 = ip[0], i1 = ip[1];
    id[0] = i0.x; id[1] = i0.y; id[2] = i0.z; id[3] = i0.w;
    id[4] = i1.x; id[5] = i1.y; id[6] = i1.z; id[7] = i1.w;
  }
  const T *qd = prm.qdata + e * (int64_t)(6 * Q3);
  for (int c = 0; c < prm.ncomp; c++) {
    const T *xc = prm.x + c * prm.N;
    T *yc = prm.y + c * prm.N;
    T u[8];
#pragma unroll
    for (int n = 0; n < 8; n++) u[n] = gather_load(&xc[id[n]], prm.x_l2_only);
    // vertex differences: dx[b][c] = u[1bc] - u[0bc], dy[a][c], dz[a][b]
    T dx[2][2], dy[2][2], dz[2][2];
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
      for (int r = 0; r < 2; r++) {
        dx[s][r] = u[1 + 2 * s + 4 * r] - u[2 * s + 4 * r];
        dy[s][r] = u[s + 2 + 4 * r] - u[s + 4 * r];
        dz[s][r] = u[s + 2 * r + 4] - u[s + 2 * r];
      }
    // gradients, each constant along its own direction
    T gx[Q][Q], gy[Q][Q], gz[Q][Q];   // gx[j][k], gy[i][k], gz[i][j]
    {
      T hx[2][Q], hy[2][Q], hz[2][Q];
#pragma unroll
      for (int s = 0; s < 2; s++)
#pragma unroll
        for (int m = 0; m < Q; m++) {
          hx[s][m] = t.H[m][0] * dx[s][0] + t.H[m][1] * dx[s][1];
          hy[s][m] = t.H[m][0] * dy[s][0] + t.H[m][1] * dy[s][1];
          hz[s][m] = t.H[m][0] * dz[s][0] + t.H[m][1] * dz[s][1];
        }
#pragma unroll
      for (int l = 0; l < Q; l++)
#pragma unroll
        for (int m = 0; m < Q; m++) {
          gx[l][m] = t.B[l][0] * hx[0][m] + t.B[l][1] * hx[1][m];
          gy[l][m] = t.B[l][0] * hy[0][m] + t.B[l][1] * hy[1][m];
          gz[l][m] = t.B[l][0] * hz[0][m] + t.B[l][1] * hz[1][m];
        }
    }
    // D at every quadrature point, summed along the constant direction
    T Sx[Q][Q], Sy[Q][Q], Sz[Q][Q];
#pragma unroll
    for (int l = 0; l < Q; l++)
#pragma unroll
      for (int m = 0; m < Q; m++) { Sx[l][m] = 0; Sy[l][m] = 0; Sz[l][m] = 0; }
#pragma unroll
    for (int k = 0; k < Q; k++)
#pragma unroll
      for (int j = 0; j < Q; j++)
#pragma unroll
        for (int i = 0; i < Q; i++) {
          const T *qk = qd + i + Q * j + Q2 * k;
          const T G12 = qk[3 * Q3], G02 = qk[4 * Q3], G01 = qk[5 * Q3];
          const T ax = gx[j][k], ay = gy[i][k], az = gz[i][j];
          // the off-diagonal terms, one multiply-add each (6 per point); a
          // diagonal term's gradient is constant along the line it is summed
          // over, so it enters below through the line sum of its D entry
          Sx[j][k] += G01 * ay; Sx[j][k] += G02 * az;
          Sy[i][k] += G01 * ax; Sy[i][k] += G12 * az;
          Sz[i][j] += G02 * ax; Sz[i][j] += G12 * ay;
        }
    {
      const T *qs = qsum + e * (int64_t)(3 * Q2);
#pragma unroll
      for (int l = 0; l < Q; l++)
#pragma unroll
        for (int m = 0; m < Q; m++) {
          Sx[l][m] += qs[l + Q * m] * gx[l][m];            // sum_i D00(i, l, m)
          Sy[l][m] += qs[Q2 + l + Q * m] * gy[l][m];       // sum_j D11(l, j, m)
          Sz[l][m] += qs[2 * Q2 + l + Q * m] * gz[l][m];   // sum_k D22(l, m, k)
        }
    }
    // transposed interpolations: r[s][r] per direction
    T rx[2][2], ry[2][2], rz[2][2];
    {
      T wx[Q][2], wy[Q][2], wz[Q][2];
#pragma unroll
      for (int l = 0; l < Q; l++)
#pragma unroll
        for (int r = 0; r < 2; r++) {
          T sx = 0, sy = 0, sz = 0;
#pragma unroll
          for (int m = 0; m < Q; m++) {
            sx += t.H[m][r] * Sx[l][m];
            sy += t.H[m][r] * Sy[l][m];
            sz += t.H[m][r] * Sz[l][m];
          }
          wx[l][r] = sx; wy[l][r] = sy; wz[l][r] = sz;
        }
#pragma unroll
      for (int s = 0; s < 2; s++)
#pragma unroll
        for (int r = 0; r < 2; r++) {
          T sx = 0, sy = 0, sz = 0;
#pragma unroll
          for (int l = 0; l < Q; l++) {
            sx += t.B[l][s] * wx[l][r];
            sy += t.B[l][s] * wy[l][r];
            sz += t.B[l][s] * wz[l][r];
          }
          rx[s][r] = sx; ry[s][r] = sy; rz[s][r] = sz;
        }
    }
    // vertex (a, b, c): derivative weights -1/2 (0) and +1/2 (1), the 1/2
    // already in H
#pragma unroll
    for (int n = 0; n < 8; n++) {
      const int a = n & 1, b = (n >> 1) & 1, cc = n >> 2;
      const T vx = a ? rx[b][cc] : -rx[b][cc];
      const T vy = b ? ry[a][cc] : -ry[a][cc];
      const T vz = cc ? rz[a][b] : -rz[a][b];
      const T v = vx + vy + vz;
      atomic_add(&yc[id[n]], v);
      dl.add(v, u[n]);
    }
  }
}

template <typename T, int Q>
__global__ void __launch_bounds__(kTrilinearThreads)
    fem_apply_trilinear_kernel(const TrilinearParams<T, Q> tp) {
  const ApplyParams<T> &prm = tp.a;
  if (apply_skipped(prm)) return;
  DotAcc<T> dl;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k_el = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k_el < prm.nsel; k_el += stride)
    trilinear_element<T, Q>(prm, tp.t, tp.qsum, prm.list ? (int64_t)prm.list[k_el] : k_el, dl);
  if (prm.dot_out) {
    double v[1] = {dl.get()};
    __shared__ double tot[1];
    if (fem_grid_sum<1>(v, prm.partials, prm.counter, tot) && threadIdx.x == 0)
      *prm.dot_out = tot[0];
  }
}

}  // namespace fem_apply
