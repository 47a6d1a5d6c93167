// 1D tables of the tensor-product basis (host, FP64), the error channel and
// the basis/mesh entry points.
//
// Quadrature (section "Benchmarks"): Gauss-Legendre with q points (q = p+2 for
// BP1-BP4) or Gauss-Lobatto-Legendre with q = p+1 points (BP5/BP6, where the
// quadrature points are the nodes and interpolation is the identity).
// Basis: C0 Lagrange polynomials on the p+1 Gauss-Lobatto nodes, evaluated
// with the barycentric formula.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "fem_internal.h"

static thread_local char g_err[512] = "";

void fem_set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

extern "C" const char *fem_last_error(void) { return g_err; }
extern "C" int fem_version(void) { return 100; }

// P_n and P_n' at x by the Bonnet recurrence; derivative from
// P_n' = n (x P_n - P_{n-1}) / (x^2 - 1) (interior points only).
static void legendre_pair(int n, double x, double *pn, double *pnm1) {
  double a = 1.0, b = x;  // P_0, P_1
  if (n == 0) { *pn = 1.0; *pnm1 = 0.0; return; }
  for (int k = 2; k <= n; k++) {
    double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
    a = b; b = c;
  }
  *pn = b; *pnm1 = a;
}

// Gauss-Legendre: Newton on P_q from Tricomi's estimate cos(pi (4i+3)/(4q+2)),
// nodes returned in ascending order.
static void gauss_legendre(int q, double *r, double *w) {
  for (int i = 0; i < q; i++) {
    double x = cos(M_PI * (4.0 * i + 3.0) / (4.0 * q + 2.0));
    for (int it = 0; it < 60; it++) {
      double pn, pm;
      legendre_pair(q, x, &pn, &pm);
      double dp = q * (x * pn - pm) / (x * x - 1.0);
      double dx = pn / dp;
      x -= dx;
      if (fabs(dx) <= 1e-17) break;
    }
    double pn, pm;
    legendre_pair(q, x, &pn, &pm);
    double dp = q * (x * pn - pm) / (x * x - 1.0);
    r[q - 1 - i] = x;
    w[q - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

// Gauss-Lobatto-Legendre with n = p+1 points: the zeros of
// f(x) = P_{p+1}(x) - P_{p-1}(x) = (2p+1)/(p(p+1)) ... (1 - x^2) P_p'(x) up to a
// constant, which include +-1.  Newton on f with f' = (2p+1) P_p; weights
// 2 / (p (p+1) P_p(x)^2).  Ascending order.
static void gauss_lobatto(int n, double *r, double *w) {
  int p = n - 1;
  for (int i = 0; i < n; i++) {
    double x = -cos(M_PI * i / p);
    if (i > 0 && i < p) {
      for (int it = 0; it < 60; it++) {
        double pp1, pp, pm1, dummy;
        legendre_pair(p + 1, x, &pp1, &pp);
        legendre_pair(p - 1 < 0 ? 0 : p - 1, x, &pm1, &dummy);
        double f = pp1 - pm1;
        double df = (2.0 * p + 1.0) * pp;
        double dx = f / df;
        x -= dx;
        if (fabs(dx) <= 1e-17) break;
      }
    }
    r[i] = x;
    double pp, pm;
    legendre_pair(p, x, &pp, &pm);
    w[i] = 2.0 / (p * (p + 1.0) * pp * pp);
  }
}

// Barycentric Lagrange values l_a(x) on the nodes z[0..n-1].
static void bary_values(int n, const double *z, const double *bw, double x, double *l) {
  for (int a = 0; a < n; a++) {
    if (x == z[a]) {
      for (int b = 0; b < n; b++) l[b] = (a == b) ? 1.0 : 0.0;
      return;
    }
  }
  double s = 0.0;
  for (int a = 0; a < n; a++) { l[a] = bw[a] / (x - z[a]); s += l[a]; }
  for (int a = 0; a < n; a++) l[a] /= s;
}

static void bary_weights(int n, const double *z, double *bw) {
  for (int a = 0; a < n; a++) {
    double prod = 1.0;
    for (int b = 0; b < n; b++) if (b != a) prod *= (z[a] - z[b]);
    bw[a] = 1.0 / prod;
  }
}

// Differentiation matrix on the nodes: Dn[b][a] = l_a'(z_b).
static void bary_diff(int n, const double *z, const double *bw, double *Dn) {
  for (int b = 0; b < n; b++) {
    double diag = 0.0;
    for (int a = 0; a < n; a++) {
      if (a == b) continue;
      double v = (bw[a] / bw[b]) / (z[b] - z[a]);
      Dn[b * n + a] = v;
      diag -= v;
    }
    Dn[b * n + b] = diag;
  }
}

int fem_build_tables(int p, int q, int quad, BasisTables *t) {
  if (p < 1 || p + 1 > FEM_MAX_P) return FEM_EINVAL;
  if (quad == FEM_GAUSS) {
    if (q != p + 1 && q != p + 2) return FEM_EINVAL;
  } else if (quad == FEM_LOBATTO) {
    if (q != p + 1) return FEM_EINVAL;
  } else {
    return FEM_EINVAL;
  }
  memset(t, 0, sizeof(*t));
  t->p = p; t->P = p + 1; t->q = q; t->quad = quad;
  const int P = p + 1;
  double zw[FEM_MAX_P];
  gauss_lobatto(P, t->z, zw);
  if (quad == FEM_GAUSS) gauss_legendre(q, t->r, t->w);
  else gauss_lobatto(q, t->r, t->w);
  double bw[FEM_MAX_P], Dn[FEM_MAX_P * FEM_MAX_P];
  bary_weights(P, t->z, bw);
  bary_diff(P, t->z, bw, Dn);
  for (int k = 0; k < q; k++) {
    double l[FEM_MAX_P];
    bary_values(P, t->z, bw, t->r[k], l);
    for (int a = 0; a < P; a++) {
      t->B[k * P + a] = l[a];
      // l_a' has degree p-1 and lies in the span of the l_b: l_a' = sum_b l_a'(z_b) l_b
      double d = 0.0;
      for (int b = 0; b < P; b++) d += Dn[b * P + a] * l[b];
      t->G[k * P + a] = d;
    }
  }
  // derivative on the quadrature points (collocated gradient)
  double qbw[FEM_MAX_Q], Dqq[FEM_MAX_Q * FEM_MAX_Q];
  bary_weights(q, t->r, qbw);
  bary_diff(q, t->r, qbw, Dqq);
  for (int i = 0; i < q * q; i++) t->Dq[i] = Dqq[i];
  return FEM_OK;
}

// I[k][a] = l_a(x_k): the Lagrange basis of order p on its Gauss-Lobatto
// nodes at npts points x (p-multigrid transfers).
int fem_basis_interp(int p, const double *x, int npts, double *I) {
  if (p < 1 || p + 1 > FEM_MAX_P) return FEM_EINVAL;
  const int P = p + 1;
  double z[FEM_MAX_P], zw[FEM_MAX_P], bw[FEM_MAX_P];
  gauss_lobatto(P, z, zw);
  bary_weights(P, z, bw);
  for (int k = 0; k < npts; k++) bary_values(P, z, bw, x[k], I + k * P);
  return FEM_OK;
}

extern "C" fem_status fem_basis_tables(int p, int q, int quad, double *nodes,
                                       double *qpts, double *qwts,
                                       double *interp, double *grad) {
  BasisTables t;
  if (fem_build_tables(p, q, quad, &t) != FEM_OK) {
    fem_set_error("fem_basis_tables: unsupported p=%d q=%d quad=%d", p, q, quad);
    return FEM_EINVAL;
  }
  const int P = p + 1;
  if (nodes) memcpy(nodes, t.z, sizeof(double) * P);
  if (qpts) memcpy(qpts, t.r, sizeof(double) * q);
  if (qwts) memcpy(qwts, t.w, sizeof(double) * q);
  if (interp) memcpy(interp, t.B, sizeof(double) * q * P);
  if (grad) memcpy(grad, t.G, sizeof(double) * q * P);
  return FEM_OK;
}

extern "C" fem_status fem_mesh_nodes_from_vertices(
    int p, int64_t E, int64_t nvert, const double *vxyz, const int32_t *ev,
    const int32_t *en, int64_t N, double *node_xyz) {
  if (p < 1 || p + 1 > FEM_MAX_P || E < 0 || !vxyz || !ev || !en || !node_xyz) {
    fem_set_error("fem_mesh_nodes_from_vertices: invalid argument");
    return FEM_EINVAL;
  }
  const int P = p + 1, P3 = P * P * P;
  double z[FEM_MAX_P], zw[FEM_MAX_P];
  gauss_lobatto(P, z, zw);
  // 1D hat weights (1 - s)/2, (1 + s)/2 at each node
  double h0[FEM_MAX_P], h1[FEM_MAX_P];
  for (int a = 0; a < P; a++) { h0[a] = 0.5 * (1.0 - z[a]); h1[a] = 0.5 * (1.0 + z[a]); }
  for (int64_t e = 0; e < E; e++) {
    const int32_t *v = ev + 8 * e;
    for (int t = 0; t < 8; t++)
      if (v[t] < 0 || v[t] >= nvert) {
        fem_set_error("fem_mesh_nodes_from_vertices: vertex index out of range");
        return FEM_EINVAL;
      }
    for (int c = 0; c < P; c++)
      for (int b = 0; b < P; b++)
        for (int a = 0; a < P; a++) {
          int64_t g = en[e * P3 + a + P * b + P * P * c];
          if (g < 0 || g >= N) {
            fem_set_error("fem_mesh_nodes_from_vertices: node index out of range");
            return FEM_EINVAL;
          }
          double s[3] = {0, 0, 0};
          for (int t = 0; t < 8; t++) {
            double f = ((t & 1) ? h1[a] : h0[a]) * ((t & 2) ? h1[b] : h0[b]) *
                       ((t & 4) ? h1[c] : h0[c]);
            for (int d = 0; d < 3; d++) s[d] += f * vxyz[3 * (int64_t)v[t] + d];
          }
          for (int d = 0; d < 3; d++) node_xyz[3 * g + d] = s[d];
        }
  }
  return FEM_OK;
}
