// C ABI entry points: mesh and operator lifecycle, apply, diagonal, solve.
#include <math.h>
#include <string.h>

#include <vector>

#include "fem_internal.h"

namespace {

template <typename T>
int dev_alloc(T **p, size_t count, int64_t *bytes) {
  if (count == 0) count = 1;
  if (cudaMalloc((void **)p, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    fem_set_error("device allocation of %zu bytes failed", sizeof(T) * count);
    return FEM_ENOMEM;
  }
  *bytes += (int64_t)(sizeof(T) * count);
  return FEM_OK;
}

// Line sums of the diagonal qdata components of trilinear elements (see
// fem_op::d_qsum): one thread per (element, component, line), summed in FP64.
__global__ void qdata_line_sums_kernel(const double *qd, int64_t E, int Q, double *qsum) {
  const int Q2 = Q * Q, Q3 = Q2 * Q;
  const int64_t total = E * 3 * Q2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / (3 * Q2);
    const int r = (int)(t - e * 3 * Q2), c = r / Q2, l = r - c * Q2;
    const int u = l % Q, v = l / Q;   // the two coordinates the line does not run along
    const double *q = qd + e * 6 * Q3 + (int64_t)c * Q3;
    double s = 0.0;
    for (int m = 0; m < Q; m++) {
      const int pt = c == 0 ? m + Q * u + Q2 * v : (c == 1 ? u + Q * m + Q2 * v : u + Q * v + Q2 * m);
      s += q[pt];
    }
    qsum[t] = s;
  }
}

// Element matrices of Gauss diffusion at P = 2, 3 (fem_op::d_kel):
//   K_e[a][b] = sum_q grad phi_a(q)^T D(q) grad phi_b(q),
// grad phi_a(q) = (G_i B_j B_k, B_i G_j B_k, B_i B_j G_k) at node a =
// (ax, ay, az), point q = (i, j, k), with the 1D tables taken at those
// indices.  One thread per (element, row a); per point, w = D grad phi_a and
// then w . grad phi_b for every b, factored direction by direction.
struct ElmatTabs {
  double B[FEM_MAX_Q * 3], G[FEM_MAX_Q * 3];   // [k][a], P <= 3
};

template <int P>
__global__ void elmat_setup_kernel(const double *qd, int64_t E, int Q, const ElmatTabs t, double *K) {
  constexpr int P3 = P * P * P;
  const int Q2 = Q * Q, Q3 = Q2 * Q;
  const int64_t total = E * P3;
  for (int64_t th = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; th < total;
       th += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = th / P3;
    const int a = (int)(th - e * P3);
    const int ax = a % P, ay = (a / P) % P, az = a / (P * P);
    double row[P3];
#pragma unroll
    for (int b = 0; b < P3; b++) row[b] = 0.0;
    const double *q = qd + e * 6 * (int64_t)Q3;
    for (int k = 0; k < Q; k++)
      for (int j = 0; j < Q; j++)
        for (int i = 0; i < Q; i++) {
          const int pt = i + Q * j + Q2 * k;
          const double ga0 = t.G[i * P + ax] * t.B[j * P + ay] * t.B[k * P + az];
          const double ga1 = t.B[i * P + ax] * t.G[j * P + ay] * t.B[k * P + az];
          const double ga2 = t.B[i * P + ax] * t.B[j * P + ay] * t.G[k * P + az];
          const double d00 = q[pt], d11 = q[Q3 + pt], d22 = q[2 * Q3 + pt];
          const double d12 = q[3 * Q3 + pt], d02 = q[4 * Q3 + pt], d01 = q[5 * Q3 + pt];
          const double w0 = d00 * ga0 + d01 * ga1 + d02 * ga2;
          const double w1 = d01 * ga0 + d11 * ga1 + d12 * ga2;
          const double w2 = d02 * ga0 + d12 * ga1 + d22 * ga2;
          // w . grad phi_b = (w0 G_i[bx] B_j[by] + w1 B_i[bx] G_j[by]) B_k[bz]
          //                + w2 B_i[bx] B_j[by] G_k[bz]
#pragma unroll
          for (int bx = 0; bx < P; bx++) {
            const double u0 = w0 * t.G[i * P + bx], u1 = w1 * t.B[i * P + bx], u2 = w2 * t.B[i * P + bx];
#pragma unroll
            for (int by = 0; by < P; by++) {
              const double s01 = u0 * t.B[j * P + by] + u1 * t.G[j * P + by];
              const double s2 = u2 * t.B[j * P + by];
#pragma unroll
              for (int bz = 0; bz < P; bz++)
                row[bx + P * by + P * P * bz] += s01 * t.B[k * P + bz] + s2 * t.G[k * P + bz];
            }
          }
        }
    // upper triangle of row a: packed entries a*P3 - a(a-1)/2 + (b - a)
    const int64_t start = (int64_t)a * P3 - (int64_t)a * (a - 1) / 2 - a;
#pragma unroll
    for (int b = 0; b < P3; b++)
      if (b >= a) K[(start + b) * E + e] = row[b];
  }
}

__global__ void f64_to_f32_kernel(const double *a, float *b, int64_t n);

// The trilinear body's line sums (fem_op::d_qsum), made when that body is
// first selected: the trilinear body applies the diagonal of D once per line.
int ensure_qdata64(fem_op *op);
int ensure_qsum(fem_op *op) {
  if (op->d_qsum || !(op->kind == FEM_DIFFUSION && !op->colloc && op->P == 2)) return FEM_OK;
  {
    const int rc0 = ensure_qdata64(op);
    if (rc0) return rc0;
  }
  const int Q = op->Q;
  const size_t ns = (size_t)op->E * 3 * Q * Q;
  cudaStream_t s = op->stream();
  int rc;
  if ((rc = dev_alloc(&op->d_qsum, ns, &op->bytes))) return rc;
  if (ns > 0) qdata_line_sums_kernel<<<148 * 8, 256, 0, s>>>(op->d_qdata, op->E, Q, op->d_qsum);
  if (op->d_qdata32) {
    if ((rc = dev_alloc(&op->d_qsum32, ns, &op->bytes))) return rc;
    if (ns > 0) f64_to_f32_kernel<<<148 * 8, 256, 0, s>>>(op->d_qsum, op->d_qsum32, (int64_t)ns);
  }
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

template <typename T>
void dev_release(T **p, size_t count, int64_t *bytes) {
  if (!*p) return;
  cudaFree(*p);
  *p = nullptr;
  *bytes -= (int64_t)(sizeof(T) * (count == 0 ? 1 : count));
}

size_t nq64(const fem_op *op) {
  return (size_t)op->E * (op->kind == FEM_DIFFUSION ? 6 : 1) * op->Q * op->Q * op->Q;
}
size_t nkel(const fem_op *op) {
  const size_t P3 = (size_t)op->P * op->P * op->P;
  return (size_t)op->E * (P3 * (P3 + 1) / 2);
}

__global__ void f64_to_f32_kernel(const double *a, float *b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

__global__ void f64_to_dw_kernel(const double *a, dw *b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = dw_from_double(a[i]);
}

// P = 3: the double-word element matrices in the layered body's entry order
// (fem_elmat_layer_src maps it to the row-packed FP64 order).
__global__ void kel_layers_dw_kernel(const double *a, dw *b, int64_t E) {
  const int64_t n = 378 * E;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / E, e = i - k * E;
    b[i] = dw_from_double(a[(int64_t)fem_elmat_layer_src((int)k) * E + e]);
  }
}

// The FP64 qdata, recomputed from the mesh when it was released.
int ensure_qdata64(fem_op *op) {
  if (op->d_qdata) return FEM_OK;
  int rc;
  if ((rc = dev_alloc(&op->d_qdata, nq64(op), &op->bytes))) return rc;
  return fem_setup_qdata(op);
}

// The FP64 element matrices (Gauss diffusion at P = 2, 3), built from the
// qdata: K_e = sum_q grad phi_a^T D grad phi_b.
int ensure_kel64(fem_op *op) {
  if (op->d_kel || !fem_has_elmat(op->kind, op->colloc, op->P)) return FEM_OK;
  int rc;
  if ((rc = ensure_qdata64(op))) return rc;
  const size_t nk = nkel(op);
  if ((rc = dev_alloc(&op->d_kel, nk, &op->bytes))) return rc;
  ElmatTabs et;
  memset(&et, 0, sizeof(et));
  memcpy(et.B, op->tab.B, sizeof(double) * op->Q * op->P);
  memcpy(et.G, op->tab.G, sizeof(double) * op->Q * op->P);
  if (nk > 0) {
    if (op->P == 2) elmat_setup_kernel<2><<<148 * 8, 128, 0, op->stream()>>>(op->d_qdata, op->E, op->Q, et, op->d_kel);
    else elmat_setup_kernel<3><<<148 * 8, 128, 0, op->stream()>>>(op->d_qdata, op->E, op->Q, et, op->d_kel);
    FEM_CHECK_LAUNCH();
  }
  return FEM_OK;
}

// The double-word split of the element matrices (choice 11), made when that
// body is first selected.
int ensure_keldw(fem_op *op) {
  if (op->d_keldw || !fem_has_elmat(op->kind, op->colloc, op->P)) return FEM_OK;
  int rc;
  if ((rc = ensure_kel64(op))) return rc;
  const int P3 = op->P * op->P * op->P;
  const size_t nk = (size_t)op->E * (size_t)(P3 * (P3 + 1) / 2);
  if ((rc = dev_alloc(&op->d_keldw, nk, &op->bytes))) return rc;
  if (nk > 0) {
    if (op->P == 3) kel_layers_dw_kernel<<<148 * 8, 256, 0, op->stream()>>>(op->d_kel, op->d_keldw, op->E);
    else f64_to_dw_kernel<<<148 * 8, 256, 0, op->stream()>>>(op->d_kel, op->d_keldw, (int64_t)nk);
  }
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

}  // namespace

int fem_ensure_qsum(fem_op *op) { return ensure_qsum(op); }

// The double-word split of the qdata (line-body choices), made when one of
// those bodies is first selected.
static int ensure_qdw(fem_op *op) {
  if (op->d_qdw) return FEM_OK;
  const size_t nq = nq64(op);
  int rc;
  if ((rc = ensure_qdata64(op))) return rc;
  if ((rc = dev_alloc(&op->d_qdw, nq, &op->bytes))) return rc;
  if (nq > 0) f64_to_dw_kernel<<<148 * 8, 256, 0, op->stream()>>>(op->d_qdata, op->d_qdw, (int64_t)nq);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

int fem_ensure_choice_data(fem_op *op, int prec, int choice) {
  if (choice == 6) return ensure_qsum(op);
  if (choice == FEM_CHOICE_DW_ELMAT) return ensure_keldw(op);
  if (choice == FEM_CHOICE_DW_STENCIL) {
    // the stencil, and the element matrices for element-list applies
    int rc = prec == FEM_F64 ? ensure_keldw(op) : ensure_kel64(op);
    return rc ? rc : fem_ensure_stencil(op, prec);
  }
  if (fem_choice_is_dw(choice)) return ensure_qdw(op);
  if (prec == FEM_F64) return choice == 7 ? ensure_kel64(op) : ensure_qdata64(op);
  return FEM_OK;   // the FP32 bodies read the FP32 copies made at set-up
}

int fem_ensure_qdata64(fem_op *op) { return ensure_qdata64(op); }

extern "C" fem_status fem_mesh_create(int p, int64_t N, int64_t E, const int32_t *en,
                                      const double *xyz, const uint8_t *dir, void *stream,
                                      fem_mesh **out) {
  if (!out) { fem_set_error("fem_mesh_create: out is NULL"); return FEM_EINVAL; }
  *out = nullptr;
  if (p < 1 || p + 1 > FEM_MAX_P) { fem_set_error("fem_mesh_create: p=%d not in [1, 8]", p); return FEM_EINVAL; }
  if (N < 1 || E < 0 || (E > 0 && !en) || !xyz) { fem_set_error("fem_mesh_create: invalid sizes or NULL arrays"); return FEM_EINVAL; }
  if (N > INT32_MAX) { fem_set_error("fem_mesh_create: N exceeds int32 node ids"); return FEM_EINVAL; }
  const int P = p + 1, P3 = P * P * P;
  for (int64_t i = 0; i < E * P3; i++)
    if (en[i] < 0 || en[i] >= N) {
      fem_set_error("fem_mesh_create: elem_nodes[%lld] = %d out of [0, %lld)", (long long)i, en[i], (long long)N);
      return FEM_EINVAL;
    }
  fem_mesh *m = new fem_mesh();
  m->p = p; m->P = P; m->N = N; m->E = E;
  m->stream = (cudaStream_t)stream;
  int rc;
  if ((rc = dev_alloc(&m->d_elem_nodes, (size_t)E * P3, &m->bytes)) ||
      (rc = dev_alloc(&m->d_xyz, (size_t)3 * N, &m->bytes)) ||
      (rc = dev_alloc(&m->d_dirichlet, (size_t)N, &m->bytes))) {
    fem_mesh_destroy(m);
    return rc;
  }
  std::vector<double> soa((size_t)3 * N);
  for (int64_t i = 0; i < N; i++)
    for (int d = 0; d < 3; d++) soa[(size_t)d * N + i] = xyz[3 * i + d];
  cudaError_t e = cudaMemcpyAsync(m->d_elem_nodes, en, sizeof(int32_t) * E * P3, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->d_xyz, soa.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) {
    if (dir) e = cudaMemcpyAsync(m->d_dirichlet, dir, N, cudaMemcpyHostToDevice, m->stream);
    else e = cudaMemsetAsync(m->d_dirichlet, 0, N, m->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    fem_set_error("fem_mesh_create: upload failed: %s", cudaGetErrorString(e));
    fem_mesh_destroy(m);
    return FEM_ECUDA;
  }
  *out = m;
  return FEM_OK;
}

namespace {
// Q_p node coordinates of trilinear bricks on the GPU (same map as
// fem_mesh_nodes_from_vertices): one thread per (element, local node).
__global__ void nodes_from_vertices_kernel(int P, int64_t E, const double *z, const double *vxyz,
                                           const int32_t *ev, const int32_t *en, int64_t N,
                                           double *xyz) {
  const int P3 = P * P * P;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E * P3;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / P3;
    const int l = (int)(i - e * P3);
    const int a = l % P, b = (l / P) % P, c = l / (P * P);
    const double h0[3] = {0.5 * (1.0 - z[a]), 0.5 * (1.0 - z[b]), 0.5 * (1.0 - z[c])};
    const double h1[3] = {0.5 * (1.0 + z[a]), 0.5 * (1.0 + z[b]), 0.5 * (1.0 + z[c])};
    double s[3] = {0, 0, 0};
    for (int t = 0; t < 8; t++) {
      const double f = ((t & 1) ? h1[0] : h0[0]) * ((t & 2) ? h1[1] : h0[1]) * ((t & 4) ? h1[2] : h0[2]);
      const int64_t v = ev[8 * e + t];
      for (int d = 0; d < 3; d++) s[d] += f * vxyz[3 * v + d];
    }
    const int64_t g = en[i];
    for (int d = 0; d < 3; d++) xyz[d * N + g] = s[d];
  }
}
}  // namespace

extern "C" fem_status fem_mesh_create_vertices(int p, int64_t N, int64_t E, const int32_t *en,
                                               int64_t nvert, const double *vxyz,
                                               const int32_t *ev, const uint8_t *dir,
                                               void *stream, fem_mesh **out) {
  if (!out) { fem_set_error("fem_mesh_create_vertices: out is NULL"); return FEM_EINVAL; }
  *out = nullptr;
  if (p < 1 || p + 1 > FEM_MAX_P || N < 1 || E < 0 || nvert < 1 || (E > 0 && (!en || !ev)) || !vxyz) {
    fem_set_error("fem_mesh_create_vertices: invalid arguments");
    return FEM_EINVAL;
  }
  if (N > INT32_MAX || nvert > INT32_MAX) { fem_set_error("fem_mesh_create_vertices: sizes exceed int32 ids"); return FEM_EINVAL; }
  const int P = p + 1, P3 = P * P * P;
  for (int64_t i = 0; i < E * P3; i++)
    if (en[i] < 0 || en[i] >= N) {
      fem_set_error("fem_mesh_create_vertices: elem_nodes[%lld] = %d out of [0, %lld)", (long long)i, en[i], (long long)N);
      return FEM_EINVAL;
    }
  for (int64_t i = 0; i < E * 8; i++)
    if (ev[i] < 0 || ev[i] >= nvert) {
      fem_set_error("fem_mesh_create_vertices: elem_verts[%lld] out of range", (long long)i);
      return FEM_EINVAL;
    }
  BasisTables t;
  fem_build_tables(p, p + 1, FEM_LOBATTO, &t);  // t.z: the Gauss-Lobatto nodes
  fem_mesh *m = new fem_mesh();
  m->p = p; m->P = P; m->N = N; m->E = E;
  m->stream = (cudaStream_t)stream;
  double *d_v = nullptr, *d_z = nullptr;
  int32_t *d_ev = nullptr;
  int rc;
  if ((rc = dev_alloc(&m->d_elem_nodes, (size_t)E * P3, &m->bytes)) ||
      (rc = dev_alloc(&m->d_xyz, (size_t)3 * N, &m->bytes)) ||
      (rc = dev_alloc(&m->d_dirichlet, (size_t)N, &m->bytes))) {
    fem_mesh_destroy(m);
    return rc;
  }
  int64_t tmp = 0;
  if ((rc = dev_alloc(&d_v, (size_t)3 * nvert, &tmp)) || (rc = dev_alloc(&d_ev, (size_t)8 * E, &tmp)) ||
      (rc = dev_alloc(&d_z, (size_t)FEM_MAX_P, &tmp))) {
    cudaFree(d_v); cudaFree(d_ev); cudaFree(d_z);
    fem_mesh_destroy(m);
    return rc;
  }
  cudaStream_t s = m->stream;
  cudaError_t e = cudaMemcpyAsync(m->d_elem_nodes, en, sizeof(int32_t) * E * P3, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_v, vxyz, sizeof(double) * 3 * nvert, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && E > 0) e = cudaMemcpyAsync(d_ev, ev, sizeof(int32_t) * 8 * E, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_z, t.z, sizeof(double) * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    if (dir) e = cudaMemcpyAsync(m->d_dirichlet, dir, N, cudaMemcpyHostToDevice, s);
    else e = cudaMemsetAsync(m->d_dirichlet, 0, N, s);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(m->d_xyz, 0, sizeof(double) * 3 * N, s);
  if (e == cudaSuccess && E > 0) {
    nodes_from_vertices_kernel<<<148 * 16, 256, 0, s>>>(P, E, d_z, d_v, d_ev, m->d_elem_nodes, N, m->d_xyz);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_v); cudaFree(d_ev); cudaFree(d_z);
  if (e != cudaSuccess) {
    fem_set_error("fem_mesh_create_vertices: %s", cudaGetErrorString(e));
    fem_mesh_destroy(m);
    return FEM_ECUDA;
  }
  *out = m;
  return FEM_OK;
}

// SplitMix64 output i of a generator whose state starts at `seed` (Steele,
// Lea & Flood 2014): a counter-based stream.
static uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

extern "C" fem_status fem_mesh_box(int p, int nx, int ny, int nz, double perturb, uint64_t seed,
                                   void *stream, fem_mesh **out) {
  if (!out) { fem_set_error("fem_mesh_box: out is NULL"); return FEM_EINVAL; }
  *out = nullptr;
  if (p < 1 || p + 1 > FEM_MAX_P || nx < 1 || ny < 1 || nz < 1 || !(perturb >= 0.0 && perturb < 0.5)) {
    fem_set_error("fem_mesh_box: need p in [1, 8], n >= 1 per direction, 0 <= perturb < 0.5");
    return FEM_EINVAL;
  }
  const int P = p + 1, P3 = P * P * P;
  const int64_t vx = nx + 1, vy = ny + 1, vz = nz + 1, nvert = vx * vy * vz;
  const int64_t Mx = (int64_t)p * nx + 1, My = (int64_t)p * ny + 1, Mz = (int64_t)p * nz + 1;
  const int64_t N = Mx * My * Mz, E = (int64_t)nx * ny * nz;
  if (N > INT32_MAX || nvert > INT32_MAX) {
    fem_set_error("fem_mesh_box: %lld nodes exceed int32 ids", (long long)N);
    return FEM_EINVAL;
  }
  std::vector<double> vxyz((size_t)3 * nvert);
  const int64_t nd[3] = {nx, ny, nz};
  for (int64_t k = 0; k < vz; k++)
    for (int64_t j = 0; j < vy; j++)
      for (int64_t i = 0; i < vx; i++) {
        const int64_t v = i + vx * (j + vy * k);
        const int64_t idx[3] = {i, j, k};
        for (int d = 0; d < 3; d++) {
          const double h = 1.0 / (double)nd[d];
          double c = (double)idx[d] * h;
          if (idx[d] > 0 && idx[d] < nd[d] && perturb > 0.0) {
            const double u = (double)(splitmix64_at(seed, (uint64_t)(3 * v + d)) >> 11) * 0x1.0p-53;
            c += perturb * h * (2.0 * u - 1.0);
          }
          vxyz[3 * v + d] = c;
        }
      }
  std::vector<int32_t> ev((size_t)8 * E), en((size_t)E * P3);
  for (int64_t ez = 0; ez < nz; ez++)
    for (int64_t ey = 0; ey < ny; ey++)
      for (int64_t ex = 0; ex < nx; ex++) {
        const int64_t e = ex + nx * (ey + ny * ez);
        for (int t = 0; t < 8; t++)
          ev[8 * e + t] = (int32_t)((ex + (t & 1)) + vx * ((ey + ((t >> 1) & 1)) + vy * (ez + ((t >> 2) & 1))));
        for (int c = 0; c < P; c++)
          for (int b = 0; b < P; b++)
            for (int a = 0; a < P; a++)
              en[(size_t)e * P3 + a + P * b + P * P * c] =
                  (int32_t)((p * ex + a) + Mx * ((p * ey + b) + My * (p * ez + c)));
      }
  std::vector<uint8_t> dir((size_t)N);
  for (int64_t K = 0; K < Mz; K++)
    for (int64_t J = 0; J < My; J++)
      for (int64_t I = 0; I < Mx; I++)
        dir[I + Mx * (J + My * K)] =
            (I == 0 || I == Mx - 1 || J == 0 || J == My - 1 || K == 0 || K == Mz - 1) ? 1 : 0;
  return fem_mesh_create_vertices(p, N, E, en.data(), nvert, vxyz.data(), ev.data(), dir.data(),
                                  stream, out);
}

extern "C" fem_status fem_mesh_node_coords(const fem_mesh *m, double *xyz_host) {
  if (!m || !xyz_host) { fem_set_error("fem_mesh_node_coords: invalid arguments"); return FEM_EINVAL; }
  std::vector<double> soa((size_t)3 * m->N);
  FEM_CUDA_TRY(cudaMemcpyAsync(soa.data(), m->d_xyz, sizeof(double) * 3 * m->N, cudaMemcpyDeviceToHost, m->stream));
  FEM_CUDA_TRY(cudaStreamSynchronize(m->stream));
  for (int64_t i = 0; i < m->N; i++)
    for (int d = 0; d < 3; d++) xyz_host[3 * i + d] = soa[(size_t)d * m->N + i];
  return FEM_OK;
}

extern "C" fem_status fem_mesh_destroy(fem_mesh *m) {
  if (!m) return FEM_OK;
  cudaFree(m->d_elem_nodes); cudaFree(m->d_xyz); cudaFree(m->d_dirichlet);
  delete m;
  return FEM_OK;
}


extern "C" fem_status fem_op_create(const fem_mesh *m, int kind, int quad, int q, int ncomp,
                                    int prec, const double *rff, int M, double sigma,
                                    fem_op **out) {
  if (!out || !m) { fem_set_error("fem_op_create: NULL argument"); return FEM_EINVAL; }
  *out = nullptr;
  if (kind != FEM_MASS && kind != FEM_DIFFUSION) { fem_set_error("fem_op_create: bad kind %d", kind); return FEM_EINVAL; }
  if (ncomp != 1 && ncomp != 3) { fem_set_error("fem_op_create: ncomp must be 1 or 3"); return FEM_EINVAL; }
  if (prec != FEM_F64 && prec != FEM_F32) { fem_set_error("fem_op_create: bad precision %d", prec); return FEM_EINVAL; }
  if (M < 0 || (M > 0 && !rff)) { fem_set_error("fem_op_create: bad coefficient arguments"); return FEM_EINVAL; }
  fem_op *op = new fem_op();
  if (fem_build_tables(m->p, q, quad, &op->tab) != FEM_OK) {
    fem_set_error("fem_op_create: unsupported quadrature (p=%d, q=%d, quad=%d)", m->p, q, quad);
    delete op;
    return FEM_EINVAL;
  }
  op->mesh = m; op->kind = kind; op->quad = quad; op->q = q; op->ncomp = ncomp; op->prec = prec;
  op->P = m->P; op->Q = q; op->N = m->N; op->E = m->E;
  op->colloc = (quad == FEM_LOBATTO && q == m->P);
  op->M = M; op->sigma = sigma;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&op->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (op->nsm < 1) op->nsm = 148;
  }
  const int P = op->P, Q = op->Q;
  const int64_t Q3 = (int64_t)Q * Q * Q;
  const int nd = kind == FEM_DIFFUSION ? 6 : 1;
  // Default launch shapes: the fastest choice (fem_apply_choices) of a
  // sweep of every choice at 8e6 DOFs on a B300 (the FP64 double-word
  // choices of BP3 at 5e7 DOFs, BP5 p = 7 at 3e7: median of four interleaved
  // rounds; at q = 10 after the launch bound of LinesMinBlocks), per
  // P = p + 1 (index P - 2): BP3 (Gauss q = p + 2), BP5
  // (collocated) and BP1 (Gauss mass).  FP32: the element-matrix body (7)
  // for Gauss diffusion at p = 1 (3.2x the trilinear body), the line body
  // elsewhere, often with half the default elements per block (1).  FP64:
  // the double-word bodies everywhere (8..10 line body, 12..14 with the
  // pipelined gather, 15..17 with packed f32x2 contractions, 18..23 packed
  // with the next group's qdata prefetched into L2 -- 21..23 also with the
  // pipelined gather --, 11 element matrices at p = 1, 2): double-word arithmetic
  // on the FP32 pipe, 4.4-5.2x the fastest FP64-arithmetic body for BP3
  // p = 3..7, 3.2x at p = 8, 1.4x (p = 1) and 1.08x (p = 2) over the FP64
  // element matrices, 3-4x for BP5 and BP1.
  static const int kDiffF32[8] = {7, 1, 1, 0, 1, 0, 0, 1};
  static const int kDiffF64[8] = {11, 11, 16, 15, 21, 21, 12, 15};
  static const int kCollF32[8] = {4, 1, 1, 1, 1, 0, 1, 1};
  static const int kCollF64[8] = {13, 9, 19, 16, 15, 21, 21, 12};
  static const int kMassF32[8] = {1, 1, 1, 1, 0, 1, 1, 1};
  static const int kMassF64[8] = {16, 16, 16, 12, 9, 9, 8, 12};
  // Vector diffusion (BP4, BP6): the pipelined gather serves scalar
  // operators only, so their FP64 defaults come from their own sweep (BP4 and
  // BP6 at about 4e6 nodes per component, BP6 p = 7 at 2.95e7).
  static const int kDiffVecF64[8] = {11, 11, 19, 15, 8, 18, 18, 15};
  static const int kCollVecF64[8] = {9, 9, 19, 16, 15, 16, 19, 15};
  const int ip = P - 2;   // P in 2..9
  const bool vec = ncomp > 1;
  if (kind == FEM_DIFFUSION && !op->colloc) {
    op->tune_epb[FEM_F32] = kDiffF32[ip];
    op->tune_epb[FEM_F64] = vec ? kDiffVecF64[ip] : kDiffF64[ip];
  } else if (kind == FEM_DIFFUSION) {
    op->tune_epb[FEM_F32] = kCollF32[ip];
    op->tune_epb[FEM_F64] = vec ? kCollVecF64[ip] : kCollF64[ip];
  } else if (!op->colloc) {
    op->tune_epb[FEM_F32] = kMassF32[ip];
    op->tune_epb[FEM_F64] = kMassF64[ip];
  }
  int rc;
  double *tab = nullptr;
  float *tab32 = nullptr;
  if ((rc = dev_alloc(&tab, TAB_SIZE, &op->bytes)) || (rc = dev_alloc(&tab32, TAB_SIZE, &op->bytes)) ||
      (rc = dev_alloc(&op->d_qdata, (size_t)op->E * nd * Q3, &op->bytes)) ||
      (rc = dev_alloc(&op->d_diag, (size_t)op->N, &op->bytes)) ||
      (rc = dev_alloc(&op->d_partials, (size_t)4 * FEM_MAX_BLOCKS, &op->bytes)) ||
      (rc = dev_alloc(&op->d_counter, 4, &op->bytes))) {
    op->d_B = tab; op->d_B32 = tab32;
    fem_op_destroy(op);
    return rc;
  }
  op->d_B = tab + TAB_B; op->d_Dq = tab + TAB_DQ;
  op->d_B32 = tab32 + TAB_B; op->d_Dq32 = tab32 + TAB_DQ;
  std::vector<double> h(TAB_SIZE, 0.0);
  std::vector<float> h32(TAB_SIZE, 0.0f);
  memcpy(&h[TAB_B], op->tab.B, sizeof(double) * Q * P);
  memcpy(&h[TAB_DQ], op->tab.Dq, sizeof(double) * Q * Q);
  memcpy(&h[TAB_G], op->tab.G, sizeof(double) * Q * P);
  memcpy(&h[TAB_W], op->tab.w, sizeof(double) * Q);
  for (int i = 0; i < TAB_SIZE; i++) h32[i] = (float)h[i];
  cudaStream_t s = m->stream;
  cudaError_t e = cudaMemcpyAsync(tab, h.data(), sizeof(double) * TAB_SIZE, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tab32, h32.data(), sizeof(float) * TAB_SIZE, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(op->d_counter, 0, sizeof(unsigned) * 4, s);
  if (e == cudaSuccess && M > 0) {
    if ((rc = dev_alloc(&op->d_rff, (size_t)4 * M, &op->bytes))) { fem_op_destroy(op); return rc; }
    e = cudaMemcpyAsync(op->d_rff, rff, sizeof(double) * 4 * M, cudaMemcpyHostToDevice, s);
  }
  if (e != cudaSuccess) {
    fem_set_error("fem_op_create: upload failed: %s", cudaGetErrorString(e));
    fem_op_destroy(op);
    return FEM_ECUDA;
  }
  if ((rc = fem_setup_qdata(op)) || (rc = fem_setup_diagonal(op))) {
    fem_op_destroy(op);
    return rc;
  }
  if (prec == FEM_F32) {
    const size_t nq = (size_t)op->E * nd * Q3;
    if ((rc = dev_alloc(&op->d_qdata32, nq, &op->bytes))) { fem_op_destroy(op); return rc; }
    if (nq > 0) f64_to_f32_kernel<<<148 * 8, 256, 0, s>>>(op->d_qdata, op->d_qdata32, (int64_t)nq);
  }
  if (fem_has_elmat(kind, op->colloc, P)) {
    // element matrices for the element-matrix bodies (launch choices 7, 11)
    if ((rc = ensure_kel64(op))) { fem_op_destroy(op); return rc; }
    if (prec == FEM_F32) {
      const int P3 = P * P * P;
      const size_t nk = (size_t)op->E * (size_t)(P3 * (P3 + 1) / 2);
      if ((rc = dev_alloc(&op->d_kel32, nk, &op->bytes))) { fem_op_destroy(op); return rc; }
      if (nk > 0) f64_to_f32_kernel<<<148 * 8, 256, 0, s>>>(op->d_kel, op->d_kel32, (int64_t)nk);
    }
  }
  // p = 1 Gauss diffusion on a lattice mesh: the assembled stencil (24)
  // replaces the element matrices as the FP64 default
  if (fem_has_elmat(kind, op->colloc, P) && P == 2 && op->ncomp == 1 && fem_op_is_lattice(op)) {
    if (op->tune_epb[FEM_F64] == FEM_CHOICE_DW_ELMAT) op->tune_epb[FEM_F64] = FEM_CHOICE_DW_STENCIL;
    if (prec == FEM_F32 && op->tune_epb[FEM_F32] == 7) op->tune_epb[FEM_F32] = FEM_CHOICE_DW_STENCIL;
  }
  // the data of the default launch choices (trilinear line sums, split
  // qdata or element matrices)
  if ((rc = fem_ensure_choice_data(op, FEM_F64, op->tune_epb[FEM_F64])) ||
      (rc = fem_ensure_choice_data(op, FEM_F32, op->tune_epb[FEM_F32]))) {
    fem_op_destroy(op);
    return rc;
  }
  // With a double-word body as the FP64 default, the FP64 qdata and element
  // matrices are read by nothing after set-up: release them (they are
  // rebuilt from the mesh when another body, a batch or fem_op_qdata needs
  // them).  At 5e7 DOFs this is 65 GB at p = 1.
  if (fem_choice_is_dw(op->tune_epb[FEM_F64])) {
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
      fem_set_error("fem_op_create: setup kernels failed: %s", cudaGetErrorString(e));
      fem_op_destroy(op);
      return FEM_ECUDA;
    }
    dev_release(&op->d_qdata, nq64(op), &op->bytes);
    if (op->d_kel) dev_release(&op->d_kel, nkel(op), &op->bytes);
  }
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    fem_set_error("fem_op_create: setup kernels failed: %s", cudaGetErrorString(e));
    fem_op_destroy(op);
    return FEM_ECUDA;
  }
  *out = op;
  return FEM_OK;
}

extern "C" fem_status fem_op_destroy(fem_op *op) {
  if (!op) return FEM_OK;
  fem_cg_free(op);
  fem_refine_free(op);
  if (op->d_B) cudaFree(op->d_B - TAB_B);
  if (op->d_B32) cudaFree(op->d_B32 - TAB_B);
  cudaFree(op->d_qdata); cudaFree(op->d_qdata32); cudaFree(op->d_diag); cudaFree(op->d_rff);
  cudaFree(op->d_qsum); cudaFree(op->d_qsum32);
  cudaFree(op->d_kel); cudaFree(op->d_kel32); cudaFree(op->d_keldw); cudaFree(op->d_qdw);
  cudaFree(op->d_stencil); cudaFree(op->d_xdw); cudaFree(op->d_stencil32);
  cudaFree(op->d_partials); cudaFree(op->d_counter);
  delete op;
  return FEM_OK;
}

extern "C" fem_status fem_op_sizes(const fem_op *op, int64_t *N, int64_t *E, int *ncomp, int *P,
                                   int *q, int64_t *bytes) {
  if (!op) { fem_set_error("fem_op_sizes: NULL operator"); return FEM_EINVAL; }
  if (N) *N = op->N;
  if (E) *E = op->E;
  if (ncomp) *ncomp = op->ncomp;
  if (P) *P = op->P;
  if (q) *q = op->Q;
  if (bytes) *bytes = op->bytes + op->mesh->bytes;
  return FEM_OK;
}

extern "C" fem_status fem_op_apply(fem_op *op, const double *x, double *y) {
  if (!op || !x || !y || x == y) { fem_set_error("fem_op_apply: invalid arguments"); return FEM_EINVAL; }
  FEM_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(double) * op->N * op->ncomp, op->stream()));
  return fem_launch_apply_f64(op, x, y, nullptr, op->E, nullptr);
}

extern "C" fem_status fem_op_apply_f32(fem_op *op, const float *x, float *y) {
  if (!op || !x || !y || x == y) { fem_set_error("fem_op_apply_f32: invalid arguments"); return FEM_EINVAL; }
  FEM_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(float) * op->N * op->ncomp, op->stream()));
  return fem_launch_apply_f32(op, x, y, nullptr, op->E, nullptr);
}

extern "C" fem_status fem_op_apply_elements(fem_op *op, const int32_t *elems, int64_t n,
                                            const double *x, double *y) {
  if (!op || !x || !y || x == y || n < 0 || (n > 0 && !elems)) {
    fem_set_error("fem_op_apply_elements: invalid arguments");
    return FEM_EINVAL;
  }
  FEM_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(double) * op->N * op->ncomp, op->stream()));
  return fem_launch_apply_f64(op, x, y, elems, n, nullptr);
}

extern "C" fem_status fem_op_diagonal(fem_op *op, double *d) {
  if (!op || !d) { fem_set_error("fem_op_diagonal: invalid arguments"); return FEM_EINVAL; }
  for (int c = 0; c < op->ncomp; c++)
    FEM_CUDA_TRY(cudaMemcpyAsync(d + c * op->N, op->d_diag, sizeof(double) * op->N,
                                 cudaMemcpyDeviceToDevice, op->stream()));
  return FEM_OK;
}

extern "C" fem_status fem_op_qdata_host(fem_op *op, int64_t e, double *out) {
  if (!op || !out || e < 0 || e >= op->E) { fem_set_error("fem_op_qdata_host: invalid arguments"); return FEM_EINVAL; }
  const int nd = op->kind == FEM_DIFFUSION ? 6 : 1;
  const int64_t Q3 = (int64_t)op->Q * op->Q * op->Q;
  {
    const int rc = ensure_qdata64(op);
    if (rc) return rc;
  }
  FEM_CUDA_TRY(cudaMemcpyAsync(out, op->d_qdata + e * nd * Q3, sizeof(double) * nd * Q3,
                               cudaMemcpyDeviceToHost, op->stream()));
  FEM_CUDA_TRY(cudaStreamSynchronize(op->stream()));
  return FEM_OK;
}

extern "C" fem_status fem_op_rhs(fem_op *op, int which, double *b) {
  if (!op || !b || (which != 0 && which != 1)) { fem_set_error("fem_op_rhs: invalid arguments"); return FEM_EINVAL; }
  return fem_launch_rhs(op, which, b);
}

extern "C" fem_status fem_cg_checkpoint_size(const fem_op *op, int64_t *bytes) {
  if (!op || !bytes) { fem_set_error("fem_cg_checkpoint_size: invalid arguments"); return FEM_EINVAL; }
  *bytes = fem_cg_checkpoint_bytes(op);
  return FEM_OK;
}

extern "C" fem_status fem_cg_checkpoint(fem_op *op, void *state_host) {
  if (!op || !state_host) { fem_set_error("fem_cg_checkpoint: invalid arguments"); return FEM_EINVAL; }
  return fem_cg_checkpoint_save(op, state_host);
}

extern "C" fem_status fem_cg_restore(fem_op *op, const void *state_host) {
  if (!op || !state_host) { fem_set_error("fem_cg_restore: invalid arguments"); return FEM_EINVAL; }
  return fem_cg_checkpoint_restore(op, state_host);
}

extern "C" fem_status fem_cg_resume(fem_op *op, const double *b, double *x, const fem_cg_opts *o,
                                    fem_cg_stats *st) {
  if (!op || !b || !x || !o || b == x || o->maxit < 0 || !(o->rtol >= 0.0)) {
    fem_set_error("fem_cg_resume: invalid arguments");
    return FEM_EINVAL;
  }
  return fem_cg_resume_run(op, b, x, o, st);
}

extern "C" fem_status fem_cg_solve(fem_op *op, const double *b, double *x, const fem_cg_opts *o,
                                   fem_cg_stats *st) {
  if (!op || !b || !x || !o || b == x) { fem_set_error("fem_cg_solve: invalid arguments"); return FEM_EINVAL; }
  if (o->precond != FEM_PC_NONE && o->precond != FEM_PC_JACOBI) {
    fem_set_error("fem_cg_solve: preconditioner %d not available in plain CG", o->precond);
    return FEM_EINVAL;
  }
  if (o->maxit < 0 || !(o->rtol >= 0.0)) { fem_set_error("fem_cg_solve: bad maxit/rtol"); return FEM_EINVAL; }
  return fem_cg_run(op, b, x, o, st);
}


namespace {
__global__ void residual_kernel(const double *b, double *r, const uint8_t *dir, int64_t N, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    r[i] = (dir && dir[fem_node_of(i, N)]) ? 0.0 : b[i] - r[i];
}
}  // namespace

extern "C" fem_status fem_op_residual(fem_op *op, const double *b, const double *x, double *r) {
  if (!op || !b || !x || !r || r == x || r == b) {
    fem_set_error("fem_op_residual: invalid arguments");
    return FEM_EINVAL;
  }
  int rc = fem_op_apply(op, x, r);
  if (rc) return rc;
  const int64_t n = op->N * op->ncomp;
  residual_kernel<<<148 * 8, 256, 0, op->stream()>>>(b, r, op->mesh->d_dirichlet, op->N, n);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}
