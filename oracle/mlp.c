/*
 * mlp.c -- FP64 CPU oracle of the per-element multilayer perceptron used as
 * a learned preconditioner (TEST INFRASTRUCTURE; the paper has no such
 * network: its preconditioning discussion is the section "Ecosystem",
 * "matrix-free preconditioning").
 *
 * Network (row-vector convention, one sample per row):
 *     h1 = relu(x  W1^T + b1)     x  in R^{n_in},  W1 in R^{n_h  x n_in}
 *     h2 = relu(h1 W2^T + b2)                      W2 in R^{n_h  x n_h}
 *     y  =      h2 W3^T + b3                       W3 in R^{n_out x n_h}
 * loss over a batch of S samples with targets t:  L = (1/S) sum ||y - t||^2.
 * Parameters are one flat array in the order W1, b1, W2, b2, W3, b3.
 * Backward is the chain rule written out layer by layer; Adam (Kingma & Ba
 * 2015) with bias correction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int n_in, n_h, n_out;
} mlp_dims;

static int64_t n_params(mlp_dims d) {
  return (int64_t)d.n_h * d.n_in + d.n_h + (int64_t)d.n_h * d.n_h + d.n_h +
         (int64_t)d.n_out * d.n_h + d.n_out;
}

int64_t oracle_mlp_nparams(int n_in, int n_h, int n_out) {
  mlp_dims d = {n_in, n_h, n_out};
  return n_params(d);
}

/* y = x W^T + b for S rows */
static void dense(int S, int nin, int nout, const double *x, const double *W, const double *b,
                  double *y) {
  for (int s = 0; s < S; s++)
    for (int o = 0; o < nout; o++) {
      double acc = b[o];
      for (int i = 0; i < nin; i++) acc += x[(int64_t)s * nin + i] * W[(int64_t)o * nin + i];
      y[(int64_t)s * nout + o] = acc;
    }
}

/* Forward: y [S][n_out]; h1, h2 (post-activation) returned if non-NULL. */
int oracle_mlp_forward(int n_in, int n_h, int n_out, const double *params, int S,
                       const double *x, double *y, double *h1_out, double *h2_out) {
  const double *W1 = params, *b1 = W1 + (int64_t)n_h * n_in;
  const double *W2 = b1 + n_h, *b2 = W2 + (int64_t)n_h * n_h;
  const double *W3 = b2 + n_h, *b3 = W3 + (int64_t)n_out * n_h;
  double *h1 = (double *)malloc(sizeof(double) * (size_t)S * n_h);
  double *h2 = (double *)malloc(sizeof(double) * (size_t)S * n_h);
  dense(S, n_in, n_h, x, W1, b1, h1);
  for (int64_t i = 0; i < (int64_t)S * n_h; i++) h1[i] = h1[i] > 0 ? h1[i] : 0.0;
  dense(S, n_h, n_h, h1, W2, b2, h2);
  for (int64_t i = 0; i < (int64_t)S * n_h; i++) h2[i] = h2[i] > 0 ? h2[i] : 0.0;
  dense(S, n_h, n_out, h2, W3, b3, y);
  if (h1_out) memcpy(h1_out, h1, sizeof(double) * (size_t)S * n_h);
  if (h2_out) memcpy(h2_out, h2, sizeof(double) * (size_t)S * n_h);
  free(h1); free(h2);
  return 0;
}

/* Loss L = (1/S) sum ||y - t||^2 and its gradient with respect to every
 * parameter (grad has n_params entries, same order as params). */
double oracle_mlp_loss_grad(int n_in, int n_h, int n_out, const double *params, int S,
                            const double *x, const double *t, double *grad) {
  const double *W2 = params + (int64_t)n_h * n_in + n_h;
  const double *W3 = W2 + (int64_t)n_h * n_h + n_h;
  double *h1 = (double *)malloc(sizeof(double) * (size_t)S * n_h);
  double *h2 = (double *)malloc(sizeof(double) * (size_t)S * n_h);
  double *y = (double *)malloc(sizeof(double) * (size_t)S * n_out);
  oracle_mlp_forward(n_in, n_h, n_out, params, S, x, y, h1, h2);
  double L = 0.0;
  double *dy = (double *)malloc(sizeof(double) * (size_t)S * n_out);
  for (int64_t i = 0; i < (int64_t)S * n_out; i++) {
    double r = y[i] - t[i];
    L += r * r;
    dy[i] = 2.0 * r / S;
  }
  L /= S;
  if (grad) {
    double *gW1 = grad, *gb1 = gW1 + (int64_t)n_h * n_in;
    double *gW2 = gb1 + n_h, *gb2 = gW2 + (int64_t)n_h * n_h;
    double *gW3 = gb2 + n_h, *gb3 = gW3 + (int64_t)n_out * n_h;
    mlp_dims d = {n_in, n_h, n_out};
    memset(grad, 0, sizeof(double) * (size_t)n_params(d));
    double *dh2 = (double *)calloc((size_t)S * n_h, sizeof(double));
    double *dh1 = (double *)calloc((size_t)S * n_h, sizeof(double));
    /* layer 3: y = h2 W3^T + b3 */
    for (int s = 0; s < S; s++)
      for (int o = 0; o < n_out; o++) {
        double g = dy[(int64_t)s * n_out + o];
        gb3[o] += g;
        for (int i = 0; i < n_h; i++) {
          gW3[(int64_t)o * n_h + i] += g * h2[(int64_t)s * n_h + i];
          dh2[(int64_t)s * n_h + i] += g * W3[(int64_t)o * n_h + i];
        }
      }
    /* relu of layer 2 */
    for (int64_t i = 0; i < (int64_t)S * n_h; i++) if (!(h2[i] > 0)) dh2[i] = 0.0;
    for (int s = 0; s < S; s++)
      for (int o = 0; o < n_h; o++) {
        double g = dh2[(int64_t)s * n_h + o];
        gb2[o] += g;
        for (int i = 0; i < n_h; i++) {
          gW2[(int64_t)o * n_h + i] += g * h1[(int64_t)s * n_h + i];
          dh1[(int64_t)s * n_h + i] += g * W2[(int64_t)o * n_h + i];
        }
      }
    for (int64_t i = 0; i < (int64_t)S * n_h; i++) if (!(h1[i] > 0)) dh1[i] = 0.0;
    for (int s = 0; s < S; s++)
      for (int o = 0; o < n_h; o++) {
        double g = dh1[(int64_t)s * n_h + o];
        gb1[o] += g;
        for (int i = 0; i < n_in; i++) gW1[(int64_t)o * n_in + i] += g * x[(int64_t)s * n_in + i];
      }
    free(dh1); free(dh2);
  }
  free(h1); free(h2); free(y); free(dy);
  return L;
}

/* One Adam step (step number k >= 1) on params with gradient g:
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   p -= lr * (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps) */
void oracle_adam_step(int64_t n, double *p, const double *g, double *m, double *v, int k,
                      double lr, double b1, double b2, double eps) {
  double c1 = 1.0 - pow(b1, k), c2 = 1.0 - pow(b2, k);
  for (int64_t i = 0; i < n; i++) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}
