/*
 * oracle.c -- plain FP64 CPU oracle for the matrix-free high-order finite
 * element operators of the CEED bake-off problems (Kolev et al., "Efficient
 * Exascale Discretizations: High-Order Finite Element Methods", section
 * "Benchmarks" and section "libCEED").
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library; it is deliberately slow and
 * written so that every step can be compared with the paper by eye:
 *
 *   - the 1D rules (Gauss-Legendre with q points for BP1-BP4, Gauss-Lobatto-
 *     Legendre with q = p+1 points for BP5/BP6; section "Benchmarks") come
 *     from Newton's method on the Legendre three-term recurrence;
 *   - the C0 Lagrange basis phi_i on the Gauss-Lobatto nodes is evaluated by
 *     the product formula, its derivative by the sum-of-products rule;
 *   - 3D reference values and gradients are formed point by point as plain
 *     products (NO sum factorization): dense tables of size q^3 x (p+1)^3;
 *   - each element is the isoparametric map x^e(r) = sum_a x_a phi_a(r) of
 *     its nodes, J = dx/dr is summed over all nodes at every quadrature
 *     point, det J and J^{-1} come from the explicit cofactor formula;
 *   - the element operator is the definition of the bilinear forms
 *        A_ij = int grad phi_i . grad phi_j dV,  B_ij = int phi_i phi_j dV
 *     (section "Benchmarks") evaluated by the tensor quadrature, optionally
 *     weighted by a coefficient kappa(x) at the physical quadrature point;
 *   - y = sum_e G_e^T K_e G_e x with G_e the element gather of the element
 *     restriction (section "libCEED", operator decomposition).
 *
 * Vector problems (ncomp = 3, BP2/BP4/BP6) apply the same scalar operator to
 * each component; vectors are component-major [ncomp][N].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MASS 0
#define OR_DIFFUSION 1
#define OR_GAUSS 0
#define OR_LOBATTO 1
#define OR_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------ */
/* 1D rules                                                            */
/* ------------------------------------------------------------------ */

/* Legendre P_n(x) and P_n'(x) by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, and the derivative identity
 * (1-x^2) P_n' = n (P_{n-1} - x P_n) away from x = +-1. */
static void legendre(int n, double x, double *Pn, double *dPn, double *Pnm1) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    *Pn = 1.0; *dPn = 0.0; if (Pnm1) *Pnm1 = 0.0;
    return;
  }
  for (int k = 1; k < n; k++) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1; p1 = p2;
  }
  *Pn = p1;
  if (Pnm1) *Pnm1 = p0;
  if (fabs(fabs(x) - 1.0) < 1e-300) {
    /* P_n'(1) = n(n+1)/2,  P_n'(-1) = (-1)^{n-1} n(n+1)/2 */
    double s = (x > 0 || n % 2 == 1) ? 1.0 : -1.0;
    *dPn = s * 0.5 * n * (n + 1.0);
  } else {
    *dPn = n * (p0 - x * p1) / (1.0 - x * x);
  }
}

/* Gauss-Legendre rule with q points: the roots of P_q, weights
 * w = 2 / ((1 - x^2) P_q'(x)^2).  Nodes ascending. */
int oracle_gauss_legendre(int q, double *x, double *w) {
  if (q < 1 || q > 64) return 1;
  for (int i = 0; i < q; i++) {
    /* initial guess: Chebyshev-like estimate of the (q-i)-th root */
    double r = -cos(OR_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; it++) {
      double P, dP;
      legendre(q, r, &P, &dP, NULL);
      double dr = P / dP;
      r -= dr;
      if (fabs(dr) < 1e-16) break;
    }
    double P, dP;
    legendre(q, r, &P, &dP, NULL);
    x[i] = r;
    w[i] = 2.0 / ((1.0 - r * r) * dP * dP);
  }
  return 0;
}

/* Gauss-Lobatto-Legendre rule with P = p+1 points: x = +-1 and the roots of
 * P_p'; weights w = 2 / (p (p+1) P_p(x)^2).  Nodes ascending. */
int oracle_gauss_lobatto(int P, double *x, double *w) {
  if (P < 2 || P > 64) return 1;
  int p = P - 1;
  x[0] = -1.0; x[p] = 1.0;
  for (int i = 1; i < p; i++) {
    /* Chebyshev-Gauss-Lobatto initial guess */
    double r = -cos(OR_PI * i / p);
    for (int it = 0; it < 100; it++) {
      double Pn, dPn;
      legendre(p, r, &Pn, &dPn, NULL);
      /* Legendre ODE: (1-x^2) P'' = 2x P' - p(p+1) P */
      double d2 = (2.0 * r * dPn - p * (p + 1.0) * Pn) / (1.0 - r * r);
      double dr = dPn / d2;
      r -= dr;
      if (fabs(dr) < 1e-16) break;
    }
    x[i] = r;
  }
  for (int i = 0; i <= p; i++) {
    double Pn, dPn;
    legendre(p, x[i], &Pn, &dPn, NULL);
    w[i] = 2.0 / (p * (p + 1.0) * Pn * Pn);
  }
  return 0;
}

/* Lagrange polynomial l_a on the nodes z[0..P-1] at r (product formula). */
static double lag(const double *z, int P, int a, double r) {
  double v = 1.0;
  for (int b = 0; b < P; b++)
    if (b != a) v *= (r - z[b]) / (z[a] - z[b]);
  return v;
}

/* l_a'(r) = sum_{c != a} 1/(z_a - z_c) prod_{b != a,c} (r - z_b)/(z_a - z_b) */
static double dlag(const double *z, int P, int a, double r) {
  double s = 0.0;
  for (int c = 0; c < P; c++) {
    if (c == a) continue;
    double t = 1.0 / (z[a] - z[c]);
    for (int b = 0; b < P; b++)
      if (b != a && b != c) t *= (r - z[b]) / (z[a] - z[b]);
    s += t;
  }
  return s;
}

/* Evaluate the 1D basis on the Gauss-Lobatto nodes of order p at the points r:
 * val[k*P + a] = l_a(r_k), der[k*P + a] = l_a'(r_k). */
int oracle_lagrange_1d(int p, int n, const double *r, double *val, double *der) {
  int P = p + 1;
  double z[65], wz[65];
  if (oracle_gauss_lobatto(P, z, wz)) return 1;
  for (int k = 0; k < n; k++)
    for (int a = 0; a < P; a++) {
      if (val) val[k * P + a] = lag(z, P, a, r[k]);
      if (der) der[k * P + a] = dlag(z, P, a, r[k]);
    }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Mesh: high-order node coordinates of trilinear bricks               */
/* ------------------------------------------------------------------ */

/* Each hexahedron is the trilinear map of its 8 vertices (vertex v = vi + 2 vj
 * + 4 vk, lexicographic); its Q_p nodes are the images of the tensor
 * Gauss-Lobatto nodes.  Node (a,b,c) of element e is elem_nodes[e*P^3 +
 * a + P b + P^2 c]; shared nodes are written more than once with the same
 * value (up to rounding). */
int oracle_nodes_from_vertices(int p, int64_t E, const double *vxyz,
                               const int32_t *elem_verts,
                               const int32_t *elem_nodes, double *node_xyz) {
  int P = p + 1, P3 = P * P * P;
  double z[65], wz[65];
  if (oracle_gauss_lobatto(P, z, wz)) return 1;
  for (int64_t e = 0; e < E; e++) {
    for (int c = 0; c < P; c++)
      for (int b = 0; b < P; b++)
        for (int a = 0; a < P; a++) {
          double xi[3] = {z[a], z[b], z[c]};
          double X[3] = {0, 0, 0};
          for (int v = 0; v < 8; v++) {
            int bits[3] = {v & 1, (v >> 1) & 1, (v >> 2) & 1};
            double Nv = 1.0;
            for (int d = 0; d < 3; d++)
              Nv *= bits[d] ? 0.5 * (1.0 + xi[d]) : 0.5 * (1.0 - xi[d]);
            const double *xv = vxyz + 3 * (int64_t)elem_verts[e * 8 + v];
            for (int d = 0; d < 3; d++) X[d] += Nv * xv[d];
          }
          int64_t g = elem_nodes[e * P3 + a + P * b + P * P * c];
          for (int d = 0; d < 3; d++) node_xyz[3 * g + d] = X[d];
        }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Operator                                                            */
/* ------------------------------------------------------------------ */

typedef struct {
  int p, P, P3, q, Q3, quad, kind, ncomp;
  int64_t N, E;
  const int32_t *elem_nodes; /* [E][P^3], caller-owned */
  const double *node_xyz;    /* [N][3], caller-owned */
  /* coefficient kappa(x) = exp(sigma sqrt(2/M) sum_m cos(w_m . x + b_m)) */
  int M;
  double sigma;
  double *rff; /* [M][4] = (w_x, w_y, w_z, b) */
  /* dense reference tables at the tensor quadrature points */
  double *W;   /* [Q3] tensor weights */
  double *rq;  /* [Q3][3] reference coordinates */
  double *phi; /* [Q3][P3] */
  double *dphi;/* [3][Q3][P3] */
} oracle_op;

oracle_op *oracle_op_new(int p, int q, int quad, int kind, int ncomp, int64_t N,
                         int64_t E, const int32_t *elem_nodes,
                         const double *node_xyz, int M, double sigma,
                         const double *rff) {
  if (p < 1 || p > 16 || q < 1 || q > 32 || (ncomp != 1 && ncomp != 3)) return NULL;
  if (quad == OR_LOBATTO && q < 2) return NULL;
  oracle_op *op = (oracle_op *)calloc(1, sizeof(oracle_op));
  op->p = p; op->P = p + 1; op->P3 = op->P * op->P * op->P;
  op->q = q; op->Q3 = q * q * q; op->quad = quad; op->kind = kind;
  op->ncomp = ncomp; op->N = N; op->E = E;
  op->elem_nodes = elem_nodes; op->node_xyz = node_xyz;
  op->M = M; op->sigma = sigma;
  if (M > 0) {
    op->rff = (double *)malloc(sizeof(double) * 4 * M);
    memcpy(op->rff, rff, sizeof(double) * 4 * M);
  }
  double r1[64], w1[64];
  if (quad == OR_GAUSS) oracle_gauss_legendre(q, r1, w1);
  else oracle_gauss_lobatto(q, r1, w1);
  double z[65], wz[65];
  oracle_gauss_lobatto(op->P, z, wz);
  int P = op->P, P3 = op->P3, Q3 = op->Q3;
  op->W = (double *)malloc(sizeof(double) * Q3);
  op->rq = (double *)malloc(sizeof(double) * 3 * Q3);
  op->phi = (double *)malloc(sizeof(double) * (size_t)Q3 * P3);
  op->dphi = (double *)malloc(sizeof(double) * 3 * (size_t)Q3 * P3);
  for (int k = 0; k < q; k++)
    for (int j = 0; j < q; j++)
      for (int i = 0; i < q; i++) {
        int Qi = i + q * j + q * q * k;
        double r[3] = {r1[i], r1[j], r1[k]};
        op->W[Qi] = w1[i] * w1[j] * w1[k];
        for (int d = 0; d < 3; d++) op->rq[3 * Qi + d] = r[d];
        for (int c = 0; c < P; c++)
          for (int b = 0; b < P; b++)
            for (int a = 0; a < P; a++) {
              int A = a + P * b + P * P * c;
              double la = lag(z, P, a, r[0]), lb = lag(z, P, b, r[1]), lc = lag(z, P, c, r[2]);
              double da = dlag(z, P, a, r[0]), db = dlag(z, P, b, r[1]), dc = dlag(z, P, c, r[2]);
              op->phi[(size_t)Qi * P3 + A] = la * lb * lc;
              op->dphi[(0 * (size_t)Q3 + Qi) * P3 + A] = da * lb * lc;
              op->dphi[(1 * (size_t)Q3 + Qi) * P3 + A] = la * db * lc;
              op->dphi[(2 * (size_t)Q3 + Qi) * P3 + A] = la * lb * dc;
            }
      }
  return op;
}

void oracle_op_free(oracle_op *op) {
  if (!op) return;
  free(op->rff); free(op->W); free(op->rq); free(op->phi); free(op->dphi);
  free(op);
}

/* kappa(x) by random Fourier features of a squared-exponential field. */
double oracle_kappa(const oracle_op *op, const double *x) {
  if (op->M <= 0) return 1.0;
  double s = 0.0;
  for (int m = 0; m < op->M; m++) {
    const double *f = op->rff + 4 * m;
    s += cos(f[0] * x[0] + f[1] * x[1] + f[2] * x[2] + f[3]);
  }
  return exp(op->sigma * sqrt(2.0 / op->M) * s);
}

/* Geometry of element e at quadrature point Qi: physical point x, Jacobian
 * J[d][c] = dx_d/dr_c, det J and J^{-1} by cofactors. */
static void element_geometry(const oracle_op *op, const double *Xe, int Qi,
                             double x[3], double J[3][3], double *detJ,
                             double Ji[3][3]) {
  int P3 = op->P3;
  const double *ph = op->phi + (size_t)Qi * P3;
  for (int d = 0; d < 3; d++) {
    x[d] = 0.0;
    for (int c = 0; c < 3; c++) J[d][c] = 0.0;
  }
  for (int A = 0; A < P3; A++) {
    for (int d = 0; d < 3; d++) {
      x[d] += Xe[3 * A + d] * ph[A];
      for (int c = 0; c < 3; c++)
        J[d][c] += Xe[3 * A + d] * op->dphi[((size_t)c * op->Q3 + Qi) * P3 + A];
    }
  }
  double C[3][3]; /* cofactor matrix */
  C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  C[0][1] = -(J[1][0] * J[2][2] - J[1][2] * J[2][0]);
  C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  C[1][0] = -(J[0][1] * J[2][2] - J[0][2] * J[2][1]);
  C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  C[1][2] = -(J[0][0] * J[2][1] - J[0][1] * J[2][0]);
  C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  C[2][1] = -(J[0][0] * J[1][2] - J[0][2] * J[1][0]);
  C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
  *detJ = det;
  /* J^{-1} = adj(J)/det = C^T / det */
  for (int i = 0; i < 3; i++)
    for (int k = 0; k < 3; k++) Ji[i][k] = C[k][i] / det;
}

static void element_coords(const oracle_op *op, int64_t e, double *Xe) {
  for (int A = 0; A < op->P3; A++) {
    int64_t g = op->elem_nodes[e * op->P3 + A];
    for (int d = 0; d < 3; d++) Xe[3 * A + d] = op->node_xyz[3 * g + d];
  }
}

/* Pointwise data at every quadrature point of element e (the D of the
 * decomposition): mass -> w detJ kappa; diffusion -> the symmetric 3x3
 * w detJ kappa J^{-1} J^{-T} stored as (11, 22, 33, 23, 13, 12).
 * out has Q3 (mass) or 6*Q3 (diffusion, component-major) entries. */
int oracle_qdata(const oracle_op *op, int64_t e, double *out) {
  if (e < 0 || e >= op->E) return 1;
  double *Xe = (double *)malloc(sizeof(double) * 3 * op->P3);
  element_coords(op, e, Xe);
  for (int Qi = 0; Qi < op->Q3; Qi++) {
    double x[3], J[3][3], Ji[3][3], det;
    element_geometry(op, Xe, Qi, x, J, &det, Ji);
    double c = op->W[Qi] * det * oracle_kappa(op, x);
    if (op->kind == OR_MASS) {
      out[Qi] = c;
    } else {
      double G[3][3];
      for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++) {
          G[i][k] = 0.0;
          for (int m = 0; m < 3; m++) G[i][k] += Ji[i][m] * Ji[k][m];
          G[i][k] *= c;
        }
      out[0 * op->Q3 + Qi] = G[0][0];
      out[1 * op->Q3 + Qi] = G[1][1];
      out[2 * op->Q3 + Qi] = G[2][2];
      out[3 * op->Q3 + Qi] = G[1][2];
      out[4 * op->Q3 + Qi] = G[0][2];
      out[5 * op->Q3 + Qi] = G[0][1];
    }
  }
  free(Xe);
  return 0;
}

/* Element matrix K_e (P3 x P3, row-major) of the scalar operator:
 *   mass:      K[i][j] = sum_Q w detJ kappa phi_i phi_j
 *   diffusion: K[i][j] = sum_Q w detJ kappa (J^{-T} grad phi_i).(J^{-T} grad phi_j) */
int oracle_element_matrix(const oracle_op *op, int64_t e, double *K) {
  if (e < 0 || e >= op->E) return 1;
  int P3 = op->P3, Q3 = op->Q3;
  double *Xe = (double *)malloc(sizeof(double) * 3 * P3);
  double *gphys = (double *)malloc(sizeof(double) * 3 * P3);
  element_coords(op, e, Xe);
  memset(K, 0, sizeof(double) * (size_t)P3 * P3);
  for (int Qi = 0; Qi < Q3; Qi++) {
    double x[3], J[3][3], Ji[3][3], det;
    element_geometry(op, Xe, Qi, x, J, &det, Ji);
    double c = op->W[Qi] * det * oracle_kappa(op, x);
    if (op->kind == OR_MASS) {
      const double *ph = op->phi + (size_t)Qi * P3;
      for (int i = 0; i < P3; i++)
        for (int j = 0; j < P3; j++) K[(size_t)i * P3 + j] += c * ph[i] * ph[j];
    } else {
      for (int i = 0; i < P3; i++)
        for (int d = 0; d < 3; d++) {
          /* (J^{-T} g)_d = sum_m Ji[m][d] g_m */
          double s = 0.0;
          for (int m = 0; m < 3; m++)
            s += Ji[m][d] * op->dphi[((size_t)m * Q3 + Qi) * P3 + i];
          gphys[3 * i + d] = s;
        }
      for (int i = 0; i < P3; i++)
        for (int j = 0; j < P3; j++)
          K[(size_t)i * P3 + j] += c * (gphys[3 * i] * gphys[3 * j] +
                                        gphys[3 * i + 1] * gphys[3 * j + 1] +
                                        gphys[3 * i + 2] * gphys[3 * j + 2]);
    }
  }
  free(Xe); free(gphys);
  return 0;
}

/* y_e = K_e x_e for one element without forming K_e: evaluate u (mass) or the
 * reference gradient of u (diffusion) at every quadrature point with the
 * dense tables, apply the pointwise data, and test against every basis
 * function.  xe, ye have P3 entries. */
static void element_apply(const oracle_op *op, const double *Xe,
                          const double *xe, double *ye) {
  int P3 = op->P3, Q3 = op->Q3;
  for (int A = 0; A < P3; A++) ye[A] = 0.0;
  for (int Qi = 0; Qi < Q3; Qi++) {
    double x[3], J[3][3], Ji[3][3], det;
    element_geometry(op, Xe, Qi, x, J, &det, Ji);
    double c = op->W[Qi] * det * oracle_kappa(op, x);
    if (op->kind == OR_MASS) {
      const double *ph = op->phi + (size_t)Qi * P3;
      double u = 0.0;
      for (int A = 0; A < P3; A++) u += ph[A] * xe[A];
      u *= c;
      for (int A = 0; A < P3; A++) ye[A] += ph[A] * u;
    } else {
      const double *d0 = op->dphi + ((size_t)0 * Q3 + Qi) * P3;
      const double *d1 = op->dphi + ((size_t)1 * Q3 + Qi) * P3;
      const double *d2 = op->dphi + ((size_t)2 * Q3 + Qi) * P3;
      double g[3] = {0, 0, 0};
      for (int A = 0; A < P3; A++) {
        g[0] += d0[A] * xe[A];
        g[1] += d1[A] * xe[A];
        g[2] += d2[A] * xe[A];
      }
      /* physical gradient J^{-T} g, flux c * J^{-1} J^{-T} g */
      double gp[3], f[3];
      for (int d = 0; d < 3; d++) gp[d] = Ji[0][d] * g[0] + Ji[1][d] * g[1] + Ji[2][d] * g[2];
      for (int m = 0; m < 3; m++) f[m] = c * (Ji[m][0] * gp[0] + Ji[m][1] * gp[1] + Ji[m][2] * gp[2]);
      for (int A = 0; A < P3; A++) ye[A] += d0[A] * f[0] + d1[A] * f[1] + d2[A] * f[2];
    }
  }
}

/* y = sum_{e in list} G_e^T K_e G_e x  (list = NULL: all elements).
 * x, y are [ncomp][N]; y is overwritten.  nthreads <= 0: OpenMP default. */
int oracle_apply(const oracle_op *op, const double *x, double *y,
                 const int32_t *elems, int64_t nel, int nthreads) {
  int64_t N = op->N;
  int P3 = op->P3, nc = op->ncomp;
  memset(y, 0, sizeof(double) * (size_t)nc * N);
  int64_t n = elems ? nel : op->E;
  for (int64_t k = 0; k < n; k++) {
    int64_t e = elems ? elems[k] : k;
    if (e < 0 || e >= op->E) return 1;
  }
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
  {
    double *Xe = (double *)malloc(sizeof(double) * 3 * P3);
    double *xe = (double *)malloc(sizeof(double) * P3);
    double *ye = (double *)malloc(sizeof(double) * P3);
#pragma omp for schedule(dynamic, 4)
    for (int64_t k = 0; k < n; k++) {
      int64_t e = elems ? elems[k] : k;
      element_coords(op, e, Xe);
      const int32_t *gi = op->elem_nodes + e * P3;
      for (int c = 0; c < nc; c++) {
        for (int A = 0; A < P3; A++) xe[A] = x[(int64_t)c * N + gi[A]];
        element_apply(op, Xe, xe, ye);
        for (int A = 0; A < P3; A++) {
#pragma omp atomic
          y[(int64_t)c * N + gi[A]] += ye[A];
        }
      }
    }
    free(Xe); free(xe); free(ye);
  }
  return 0;
}

/* y_i for a list of global rows i: sum over the elements listed for each row
 * (CSR: row_elems[row_ptr[k] .. row_ptr[k+1]) are the elements that contain
 * node rows[k]) of the row of K_e x_e belonging to that node.  Used to check
 * sampled entries of a full-size product.  Scalar operators only. */
int oracle_apply_rows(const oracle_op *op, const double *x, int64_t nrows,
                      const int64_t *rows, const int64_t *row_ptr,
                      const int64_t *row_elems, double *yrows, int nthreads) {
  int P3 = op->P3;
  if (op->ncomp != 1) return 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  int bad = 0;
#pragma omp parallel
  {
    double *Xe = (double *)malloc(sizeof(double) * 3 * P3);
    double *xe = (double *)malloc(sizeof(double) * P3);
    double *ye = (double *)malloc(sizeof(double) * P3);
#pragma omp for schedule(dynamic, 1)
    for (int64_t k = 0; k < nrows; k++) {
      double s = 0.0;
      for (int64_t t = row_ptr[k]; t < row_ptr[k + 1]; t++) {
        int64_t e = row_elems[t];
        if (e < 0 || e >= op->E) { bad = 1; continue; }
        const int32_t *gi = op->elem_nodes + e * P3;
        element_coords(op, e, Xe);
        for (int A = 0; A < P3; A++) xe[A] = x[gi[A]];
        element_apply(op, Xe, xe, ye);
        for (int A = 0; A < P3; A++)
          if (gi[A] == rows[k]) s += ye[A];
      }
      yrows[k] = s;
    }
    free(Xe); free(xe); free(ye);
  }
  return bad;
}

/* diag(A)_i = sum_e K_e[A][A] over the local nodes A of e mapping to i
 * (scalar operator; vector operators repeat it per component). */
int oracle_diagonal(const oracle_op *op, double *d) {
  int P3 = op->P3, Q3 = op->Q3;
  memset(d, 0, sizeof(double) * (size_t)op->N);
#pragma omp parallel
  {
    double *Xe = (double *)malloc(sizeof(double) * 3 * P3);
    double *de = (double *)malloc(sizeof(double) * P3);
#pragma omp for schedule(dynamic, 4)
    for (int64_t e = 0; e < op->E; e++) {
      element_coords(op, e, Xe);
      for (int A = 0; A < P3; A++) de[A] = 0.0;
      for (int Qi = 0; Qi < Q3; Qi++) {
        double x[3], J[3][3], Ji[3][3], det;
        element_geometry(op, Xe, Qi, x, J, &det, Ji);
        double c = op->W[Qi] * det * oracle_kappa(op, x);
        for (int A = 0; A < P3; A++) {
          if (op->kind == OR_MASS) {
            double ph = op->phi[(size_t)Qi * P3 + A];
            de[A] += c * ph * ph;
          } else {
            double g[3], gp[3];
            for (int m = 0; m < 3; m++) g[m] = op->dphi[((size_t)m * Q3 + Qi) * P3 + A];
            for (int k = 0; k < 3; k++) gp[k] = Ji[0][k] * g[0] + Ji[1][k] * g[1] + Ji[2][k] * g[2];
            de[A] += c * (gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2]);
          }
        }
      }
      const int32_t *gi = op->elem_nodes + e * P3;
      for (int A = 0; A < P3; A++) {
#pragma omp atomic
        d[gi[A]] += de[A];
      }
    }
    free(Xe); free(de);
  }
  return 0;
}

/* Manufactured right-hand sides b_i = int phi_i f dV (same quadrature as the
 * operator, f at the physical quadrature point):
 *   which = 0: f = sin(pi x) sin(pi y) sin(pi z)              (BP1 / BP2)
 *   which = 1: f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z), the Poisson load of
 *              u = sin sin sin with kappa = 1                   (BP3 - BP6)
 * b is [N] (scalar). */
int oracle_rhs(const oracle_op *op, int which, double *b) {
  int P3 = op->P3, Q3 = op->Q3;
  memset(b, 0, sizeof(double) * (size_t)op->N);
#pragma omp parallel
  {
    double *Xe = (double *)malloc(sizeof(double) * 3 * P3);
    double *be = (double *)malloc(sizeof(double) * P3);
#pragma omp for schedule(dynamic, 4)
    for (int64_t e = 0; e < op->E; e++) {
      element_coords(op, e, Xe);
      for (int A = 0; A < P3; A++) be[A] = 0.0;
      for (int Qi = 0; Qi < Q3; Qi++) {
        double x[3], J[3][3], Ji[3][3], det;
        element_geometry(op, Xe, Qi, x, J, &det, Ji);
        double f = sin(OR_PI * x[0]) * sin(OR_PI * x[1]) * sin(OR_PI * x[2]);
        if (which == 1) f *= 3.0 * OR_PI * OR_PI;
        double c = op->W[Qi] * det * f;
        for (int A = 0; A < P3; A++) be[A] += c * op->phi[(size_t)Qi * P3 + A];
      }
      const int32_t *gi = op->elem_nodes + e * P3;
      for (int A = 0; A < P3; A++) {
#pragma omp atomic
        b[gi[A]] += be[A];
      }
    }
    free(Xe); free(be);
  }
  return 0;
}

/* Errors of the discrete field u (nodal values [N]) against the exact
 * u* = sin(pi x) sin(pi y) sin(pi z), integrated with this operator's
 * quadrature:  out[0] = ||u - u*||_L2,  out[1] = |u - u*|_H1. */
int oracle_error_norms(const oracle_op *op, const double *u, double *out) {
  int P3 = op->P3, Q3 = op->Q3;
  double l2 = 0.0, h1 = 0.0;
#pragma omp parallel reduction(+ : l2, h1)
  {
    double *Xe = (double *)malloc(sizeof(double) * 3 * P3);
#pragma omp for schedule(dynamic, 4)
    for (int64_t e = 0; e < op->E; e++) {
      element_coords(op, e, Xe);
      const int32_t *gi = op->elem_nodes + e * P3;
      for (int Qi = 0; Qi < Q3; Qi++) {
        double x[3], J[3][3], Ji[3][3], det;
        element_geometry(op, Xe, Qi, x, J, &det, Ji);
        double uh = 0.0, g[3] = {0, 0, 0};
        for (int A = 0; A < P3; A++) {
          double ua = u[gi[A]];
          uh += op->phi[(size_t)Qi * P3 + A] * ua;
          for (int m = 0; m < 3; m++) g[m] += op->dphi[((size_t)m * Q3 + Qi) * P3 + A] * ua;
        }
        double gp[3];
        for (int k = 0; k < 3; k++) gp[k] = Ji[0][k] * g[0] + Ji[1][k] * g[1] + Ji[2][k] * g[2];
        double sx = sin(OR_PI * x[0]), sy = sin(OR_PI * x[1]), sz = sin(OR_PI * x[2]);
        double cx = cos(OR_PI * x[0]), cy = cos(OR_PI * x[1]), cz = cos(OR_PI * x[2]);
        double ue = sx * sy * sz;
        double ge[3] = {OR_PI * cx * sy * sz, OR_PI * sx * cy * sz, OR_PI * sx * sy * cz};
        double wd = op->W[Qi] * det;
        l2 += wd * (uh - ue) * (uh - ue);
        for (int k = 0; k < 3; k++) h1 += wd * (gp[k] - ge[k]) * (gp[k] - ge[k]);
      }
    }
    free(Xe);
  }
  out[0] = sqrt(l2);
  out[1] = sqrt(h1);
  return 0;
}

/* Physical coordinates of every quadrature point of element e: out [Q3][3]. */
int oracle_quadrature_points(const oracle_op *op, int64_t e, double *out) {
  if (e < 0 || e >= op->E) return 1;
  double *Xe = (double *)malloc(sizeof(double) * 3 * op->P3);
  element_coords(op, e, Xe);
  for (int Qi = 0; Qi < op->Q3; Qi++) {
    double x[3], J[3][3], Ji[3][3], det;
    element_geometry(op, Xe, Qi, x, J, &det, Ji);
    for (int d = 0; d < 3; d++) out[3 * Qi + d] = x[d];
  }
  free(Xe);
  return 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
