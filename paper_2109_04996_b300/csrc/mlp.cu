// Per-element multilayer perceptron used as a learned preconditioner, with
// its training (no counterpart in the paper, whose preconditioning material
// is the section "Ecosystem", matrix-free preconditioning):
//
//   input  x_e = [ r_e / ||r_e|| (the element's (p+1)^3 residual values),
//                  g_e (element features), zero padding ]        n_in
//   h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2), y = h2 W3^T + b3
//   correction  c_e = ||r_e|| * y[0 : (p+1)^3]
//   z = dinv * r + sum_e G_e^T (w_e * c_e),  w_e = 1 / node multiplicity.
//
// Weights are FP32 masters; the GEMMs run in bf16 with FP32 accumulation
// (tcgen05 tensor cores, mlp_tc.cuh), or in FP32 in the debug mode.  Training: mean squared error
// against e_e / ||r_e|| for residual/error pairs of the plain solver, Adam.
#include <cstdio>
#include <math.h>
#include <string.h>

#include <stdint.h>
#include <vector>

#include "mlp_gemm.cuh"
#include "mlp_tc.cuh"

using fem_mlp_k::GemmArgs;

struct fem_mlp {
  int n_in, n_h, n_out, mode;     // mode 0: bf16 GEMMs, 1: fp32 GEMMs
  int64_t np;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // masters, grad, Adam
  void *wq = nullptr;             // weights W1, W2, W3 in the compute type
  int step = 0;
  // activation workspace for `cap` rows
  int64_t cap = 0;
  void *h1 = nullptr, *h2 = nullptr, *dy = nullptr, *dh = nullptr;
  // minibatch buffers of fem_mlp_train
  int64_t bcap = 0;
  void *xb = nullptr;
  float *tb = nullptr;
  int32_t *perm = nullptr;
  int64_t perm_cap = 0;
  float *y = nullptr;
  double *loss = nullptr;
  int *tc_error = nullptr;        // set by a tensor-core GEMM whose wait ran out
  void *tA = nullptr, *tB = nullptr;   // K-major copies of transposed GEMM operands
  int64_t tcapA = 0, tcapB = 0;
  cudaStream_t stream = nullptr;
};

namespace {

size_t esz(const fem_mlp *n) { return n->mode == 0 ? 2 : 4; }
int64_t off_W1(const fem_mlp *) { return 0; }
int64_t off_b1(const fem_mlp *n) { return (int64_t)n->n_h * n->n_in; }
int64_t off_W2(const fem_mlp *n) { return off_b1(n) + n->n_h; }
int64_t off_b2(const fem_mlp *n) { return off_W2(n) + (int64_t)n->n_h * n->n_h; }
int64_t off_W3(const fem_mlp *n) { return off_b2(n) + n->n_h; }
int64_t off_b3(const fem_mlp *n) { return off_W3(n) + (int64_t)n->n_out * n->n_h; }

// weights in compute type, packed W1 | W2 | W3
void *wq_W1(const fem_mlp *n) { return n->wq; }
void *wq_W2(const fem_mlp *n) { return (char *)n->wq + esz(n) * (size_t)n->n_h * n->n_in; }
void *wq_W3(const fem_mlp *n) {
  return (char *)n->wq + esz(n) * ((size_t)n->n_h * n->n_in + (size_t)n->n_h * n->n_h);
}

__global__ void cast_weights_kernel(const float *p, int64_t b1off, int64_t W2off, int64_t b2off,
                                    int64_t W3off, int64_t b3off, void *out, int bf16) {
  // copy W1, W2, W3 (skip biases) into the packed compute-type array
  const int64_t n1 = b1off, n2 = b2off - W2off, n3 = b3off - W3off;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n1 + n2 + n3;
       i += (int64_t)gridDim.x * blockDim.x) {
    float v;
    if (i < n1) v = p[i];
    else if (i < n1 + n2) v = p[W2off + (i - n1)];
    else v = p[W3off + (i - n1 - n2)];
    if (bf16) ((__nv_bfloat16 *)out)[i] = __float2bfloat16(v);
    else ((float *)out)[i] = v;
  }
}

// dY = 2 (Y - T) / S over the first `valid` outputs (padding columns get 0),
// loss += sum (Y - T)^2 / S
template <typename TO>
__global__ void loss_grad_kernel(const float *Y, const float *T, int64_t S, int n_out, int valid,
                                 TO *dY, double *loss) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S * n_out;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % n_out);
    const float r = c < valid ? Y[i] - T[i] : 0.0f;
    acc += (double)r * r;
    const float gv = 2.0f * r / (float)S;
    if constexpr (sizeof(TO) == 2) dY[i] = __float2bfloat16(gv);
    else dY[i] = gv;
  }
  acc = fem_warp_sum(acc);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc / (double)S);
}

// bias gradient: column sums of D [S][n] into g[n] (atomic, g pre-zeroed)
template <typename T>
__global__ void colsum_kernel(const T *D, int64_t S, int n, float *g) {
  const int c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= n) return;
  float acc = 0.0f;
  for (int64_t r = blockIdx.x; r < S; r += gridDim.x) {
    if constexpr (sizeof(T) == 2) acc += __bfloat162float(D[r * n + c]);
    else acc += D[r * n + c];
  }
  atomicAdd(&g[c], acc);
}

__global__ void adam_kernel(int64_t n, float *p, const float *g, float *m, float *v, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi; v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

int gemm(const fem_mlp *n, const GemmArgs &a, bool AT, bool BT) {
  cudaStream_t s = n->stream;
  if (a.K % (32 * a.ksplit) != 0 || a.lda % 8 || a.ldb % 8) {
    fem_set_error("mlp gemm: K=%d (split %d) / leading dimensions not multiples of 32 / 8", a.K, a.ksplit);
    return FEM_EINVAL;
  }
  if (n->mode == 0) {
    // tcgen05 tensor cores.  The kernel takes both operands K-major; an
    // operand stored the other way ([K][M] or [K][N]: the backward products)
    // is first transposed into a scratch copy.
    fem_mlp_tc::TcArgs t;
    const __nv_bfloat16 *A = (const __nv_bfloat16 *)a.A, *B = (const __nv_bfloat16 *)a.B;
    int64_t lda = a.lda, ldb = a.ldb;
    auto scratch = [&](void **buf, int64_t *cap, int64_t elems) -> bool {
      if (*cap >= elems) return true;
      cudaFree(*buf);
      *buf = nullptr; *cap = 0;
      if (cudaMalloc(buf, sizeof(__nv_bfloat16) * (size_t)elems) != cudaSuccess) { cudaGetLastError(); return false; }
      *cap = elems;
      return true;
    };
    fem_mlp *nm = const_cast<fem_mlp *>(n);
    const dim3 tb(32, 8);
    if (AT) {   // A stored [K][M]
      if (!scratch(&nm->tA, &nm->tcapA, a.M * (int64_t)a.K)) { fem_set_error("mlp gemm: scratch allocation failed"); return FEM_ENOMEM; }
      fem_mlp_tc::transpose_bf16_kernel<<<dim3((unsigned)((a.K + 31) / 32), (unsigned)((a.M + 31) / 32)), tb, 0, s>>>(
          A, a.K, (int)a.M, lda, (__nv_bfloat16 *)nm->tA, a.K);
      A = (const __nv_bfloat16 *)nm->tA; lda = a.K;
    }
    if (BT) {   // B stored [K][N]
      if (!scratch(&nm->tB, &nm->tcapB, (int64_t)a.N * a.K)) { fem_set_error("mlp gemm: scratch allocation failed"); return FEM_ENOMEM; }
      fem_mlp_tc::transpose_bf16_kernel<<<dim3((unsigned)((a.K + 31) / 32), (unsigned)((a.N + 31) / 32)), tb, 0, s>>>(
          B, a.K, a.N, ldb, (__nv_bfloat16 *)nm->tB, a.K);
      B = (const __nv_bfloat16 *)nm->tB; ldb = a.K;
    }
    t.A = A; t.B = B; t.lda = lda; t.ldb = ldb; t.M = a.M; t.N = a.N; t.K = a.K;
    t.C = a.C; t.ldc = a.ldc; t.out_bf16 = a.out_bf16; t.accumulate = a.accumulate;
    t.bias = a.bias; t.relu = a.relu;
    t.mask = (const __nv_bfloat16 *)a.mask; t.ldm = a.ldm;
    t.error = n->tc_error;
    const int64_t tiles = ((a.M + fem_mlp_tc::TM - 1) / fem_mlp_tc::TM) * ((a.N + fem_mlp_tc::TN - 1) / fem_mlp_tc::TN);
    int ks = 1;
    if (a.accumulate) {
      // few output tiles and a long K (the weight gradients): split K so that
      // about three CTAs per SM run, each K chunk a multiple of the stage
      const int64_t want = (int64_t)3 * 148 / (tiles > 0 ? tiles : 1);
      const int64_t maxks = (a.K + fem_mlp_tc::TK - 1) / fem_mlp_tc::TK;
      ks = (int)(want < 1 ? 1 : (want > maxks ? maxks : want));
    }
    int kchunk = (a.K + ks - 1) / ks;
    kchunk = (kchunk + fem_mlp_tc::TK - 1) / fem_mlp_tc::TK * fem_mlp_tc::TK;
    ks = (a.K + kchunk - 1) / kchunk;
    t.kchunk = kchunk;
    static FemKernelCache attr;   // the attribute belongs to the current device
    int &set = attr.here();
    if (set < 0) {
      FEM_CUDA_TRY(cudaFuncSetAttribute(fem_mlp_tc::gemm_tc_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, fem_mlp_tc::kSmemBytes));
      set = 1;
    }
    if (tiles > 0x7fffffff) { fem_set_error("mlp gemm: %lld output tiles", (long long)tiles); return FEM_EINVAL; }
    dim3 grid((unsigned)tiles, 1, (unsigned)ks);
    fem_mlp_tc::gemm_tc_kernel<<<grid, fem_mlp_tc::NT, fem_mlp_tc::kSmemBytes, s>>>(t);
    FEM_CHECK_LAUNCH();
    return FEM_OK;
  }
  // mode 1: the FP32 debug network
  dim3 grid((unsigned)((a.M + 63) / 64), (unsigned)((a.N + 63) / 64), (unsigned)a.ksplit);
  if (!AT && !BT) fem_mlp_k::gemm_f32_kernel<false, false><<<grid, 256, 0, s>>>(a);
  else if (!AT && BT) fem_mlp_k::gemm_f32_kernel<false, true><<<grid, 256, 0, s>>>(a);
  else if (AT && BT) fem_mlp_k::gemm_f32_kernel<true, true><<<grid, 256, 0, s>>>(a);
  else fem_mlp_k::gemm_f32_kernel<true, false><<<grid, 256, 0, s>>>(a);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

GemmArgs ga(const void *A, int64_t lda, const void *B, int64_t ldb, int64_t M, int N, int K,
            void *C, int64_t ldc, int out_bf16) {
  GemmArgs a;
  memset(&a, 0, sizeof(a));
  a.A = A; a.B = B; a.lda = lda; a.ldb = ldb; a.M = M; a.N = N; a.K = K; a.ksplit = 1;
  a.C = C; a.ldc = ldc; a.out_bf16 = out_bf16;
  return a;
}

int ensure_cap(fem_mlp *n, int64_t rows) {
  if (rows <= n->cap) return FEM_OK;
  cudaFree(n->h1); cudaFree(n->h2); cudaFree(n->dy); cudaFree(n->dh); cudaFree(n->y);
  n->h1 = n->h2 = n->dy = n->dh = nullptr; n->y = nullptr;
  const size_t e = esz(n);
  if (cudaMalloc(&n->h1, e * rows * n->n_h) != cudaSuccess ||
      cudaMalloc(&n->h2, e * rows * n->n_h) != cudaSuccess ||
      cudaMalloc(&n->dh, e * rows * n->n_h) != cudaSuccess ||
      cudaMalloc(&n->dy, e * rows * n->n_out) != cudaSuccess ||
      cudaMalloc(&n->y, sizeof(float) * rows * n->n_out) != cudaSuccess) {
    cudaGetLastError();
    n->cap = 0;
    fem_set_error("mlp: workspace allocation for %lld rows failed", (long long)rows);
    return FEM_ENOMEM;
  }
  n->cap = rows;
  return FEM_OK;
}

}  // namespace

// Reads (and clears) the tensor-core GEMMs' timeout flag; synchronizes.
int fem_mlp_check_tc(fem_mlp *n) {
  int h = 0;
  FEM_CUDA_TRY(cudaMemcpyAsync(&h, n->tc_error, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
  FEM_CUDA_TRY(cudaStreamSynchronize(n->stream));
  if (h) {
    FEM_CUDA_TRY(cudaMemsetAsync(n->tc_error, 0, sizeof(int), n->stream));
    fem_set_error("mlp: a tensor-core GEMM's wait for its MMAs ran out");
    return FEM_ETIMEOUT;
  }
  return FEM_OK;
}

// ---- internal entry points used by the preconditioner (fcg.cu)
int fem_mlp_forward_rows(fem_mlp *n, const void *X, int64_t rows, float *Y) {
  const int b16 = n->mode == 0;
  int rc = ensure_cap(n, rows);
  if (rc) return rc;
  GemmArgs a = ga(X, n->n_in, wq_W1(n), n->n_in, rows, n->n_h, n->n_in, n->h1, n->n_h, b16);
  a.bias = n->p + off_b1(n); a.relu = 1;
  if ((rc = gemm(n, a, false, false))) return rc;
  a = ga(n->h1, n->n_h, wq_W2(n), n->n_h, rows, n->n_h, n->n_h, n->h2, n->n_h, b16);
  a.bias = n->p + off_b2(n); a.relu = 1;
  if ((rc = gemm(n, a, false, false))) return rc;
  a = ga(n->h2, n->n_h, wq_W3(n), n->n_h, rows, n->n_out, n->n_h, Y, n->n_out, 0);
  a.bias = n->p + off_b3(n);
  return gemm(n, a, false, false);
}

int fem_mlp_mode(const fem_mlp *n) { return n->mode; }
int fem_mlp_reserve(fem_mlp *n, int64_t rows) { return ensure_cap(n, rows); }
void fem_mlp_set_stream(fem_mlp *n, cudaStream_t s, cudaStream_t *old) {
  if (old) *old = n->stream;
  n->stream = s;
}
int fem_mlp_nin(const fem_mlp *n) { return n->n_in; }
int fem_mlp_nout(const fem_mlp *n) { return n->n_out; }

extern "C" fem_status fem_mlp_create(int n_in, int n_h, int n_out, int mode,
                                     const float *params_host, void *stream, fem_mlp **out) {
  if (!out || !params_host || n_in < 8 || n_h < 8 || n_out < 8 || n_in % 32 || n_h % 32 ||
      n_out % 32 || (mode != 0 && mode != 1)) {
    fem_set_error("fem_mlp_create: sizes must be multiples of 32, mode 0 (bf16) or 1 (fp32)");
    return FEM_EINVAL;
  }
  fem_mlp *n = new fem_mlp();
  n->n_in = n_in; n->n_h = n_h; n->n_out = n_out; n->mode = mode;
  n->stream = (cudaStream_t)stream;
  n->np = (int64_t)n_h * n_in + n_h + (int64_t)n_h * n_h + n_h + (int64_t)n_out * n_h + n_out;
  const size_t pb = sizeof(float) * n->np;
  if (cudaMalloc(&n->p, pb) != cudaSuccess || cudaMalloc(&n->g, pb) != cudaSuccess ||
      cudaMalloc(&n->m, pb) != cudaSuccess || cudaMalloc(&n->v, pb) != cudaSuccess ||
      cudaMalloc(&n->wq, esz(n) * n->np) != cudaSuccess ||
      cudaMalloc(&n->loss, sizeof(double)) != cudaSuccess ||
      cudaMalloc(&n->tc_error, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    fem_mlp_destroy(n);
    fem_set_error("fem_mlp_create: allocation failed");
    return FEM_ENOMEM;
  }
  cudaStream_t s = n->stream;
  cudaError_t e = cudaMemcpyAsync(n->p, params_host, pb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, pb, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, pb, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->tc_error, 0, sizeof(int), s);
  if (e != cudaSuccess) { fem_mlp_destroy(n); fem_set_error("fem_mlp_create: upload failed"); return FEM_ECUDA; }
  cast_weights_kernel<<<296, 256, 0, s>>>(n->p, off_b1(n), off_W2(n), off_b2(n), off_W3(n),
                                          off_b3(n), n->wq, mode == 0);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    fem_mlp_destroy(n);
    fem_set_error("fem_mlp_create: weight cast failed");
    return FEM_ECUDA;
  }
  *out = n;
  return FEM_OK;
}

extern "C" fem_status fem_mlp_destroy(fem_mlp *n) {
  if (!n) return FEM_OK;
  cudaFree(n->p); cudaFree(n->g); cudaFree(n->m); cudaFree(n->v); cudaFree(n->wq);
  cudaFree(n->h1); cudaFree(n->h2); cudaFree(n->dy); cudaFree(n->dh); cudaFree(n->y);
  cudaFree(n->loss); cudaFree(n->xb); cudaFree(n->tb); cudaFree(n->perm); cudaFree(n->tc_error);
  cudaFree(n->tA); cudaFree(n->tB);
  delete n;
  return FEM_OK;
}

extern "C" fem_status fem_mlp_params(fem_mlp *n, float *params_host, int64_t *np) {
  if (!n) { fem_set_error("fem_mlp_params: NULL"); return FEM_EINVAL; }
  if (np) *np = n->np;
  if (params_host) {
    FEM_CUDA_TRY(cudaMemcpyAsync(params_host, n->p, sizeof(float) * n->np, cudaMemcpyDeviceToHost, n->stream));
    FEM_CUDA_TRY(cudaStreamSynchronize(n->stream));
  }
  return FEM_OK;
}

// File layout of fem_mlp_save / fem_mlp_load: 8-byte tag "FEMMLP01", then
// int32 n_in, n_h, n_out, mode, step, 0, int64 np, then np FP32 values each of
// the parameters, Adam's first moments and Adam's second moments.
static const char kMlpTag[8] = {'F', 'E', 'M', 'M', 'L', 'P', '0', '1'};

extern "C" fem_status fem_mlp_save(fem_mlp *n, const char *path) {
  if (!n || !path) { fem_set_error("fem_mlp_save: invalid arguments"); return FEM_EINVAL; }
  std::vector<float> buf((size_t)3 * n->np);
  const size_t pb = sizeof(float) * n->np;
  FEM_CUDA_TRY(cudaMemcpyAsync(buf.data(), n->p, pb, cudaMemcpyDeviceToHost, n->stream));
  FEM_CUDA_TRY(cudaMemcpyAsync(buf.data() + n->np, n->m, pb, cudaMemcpyDeviceToHost, n->stream));
  FEM_CUDA_TRY(cudaMemcpyAsync(buf.data() + 2 * n->np, n->v, pb, cudaMemcpyDeviceToHost, n->stream));
  FEM_CUDA_TRY(cudaStreamSynchronize(n->stream));
  FILE *f = fopen(path, "wb");
  if (!f) { fem_set_error("fem_mlp_save: cannot open %s", path); return FEM_EINVAL; }
  const int32_t hdr[6] = {n->n_in, n->n_h, n->n_out, n->mode, n->step, 0};
  const int64_t np = n->np;
  bool ok = fwrite(kMlpTag, 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
            fwrite(&np, sizeof(np), 1, f) == 1 && fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  ok = (fclose(f) == 0) && ok;
  if (!ok) { fem_set_error("fem_mlp_save: writing %s failed", path); return FEM_EINVAL; }
  return FEM_OK;
}

extern "C" fem_status fem_mlp_load(const char *path, void *stream, fem_mlp **out) {
  if (!path || !out) { fem_set_error("fem_mlp_load: invalid arguments"); return FEM_EINVAL; }
  *out = nullptr;
  FILE *f = fopen(path, "rb");
  if (!f) { fem_set_error("fem_mlp_load: cannot open %s", path); return FEM_EINVAL; }
  char tag[8];
  int32_t hdr[6];
  int64_t np = 0;
  bool ok = fread(tag, 1, 8, f) == 8 && memcmp(tag, kMlpTag, 8) == 0 &&
            fread(hdr, sizeof(hdr), 1, f) == 1 && fread(&np, sizeof(np), 1, f) == 1;
  const int64_t want = ok ? (int64_t)hdr[1] * hdr[0] + hdr[1] + (int64_t)hdr[1] * hdr[1] + hdr[1] +
                                (int64_t)hdr[2] * hdr[1] + hdr[2]
                          : -1;
  ok = ok && np == want && np > 0 && hdr[4] >= 0;
  std::vector<float> buf;
  if (ok) {
    buf.resize((size_t)3 * np);
    ok = fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  }
  fclose(f);
  if (!ok) { fem_set_error("fem_mlp_load: %s is not a saved network (tag, sizes or length)", path); return FEM_EINVAL; }
  fem_mlp *n = nullptr;
  int rc = fem_mlp_create(hdr[0], hdr[1], hdr[2], hdr[3], buf.data(), stream, &n);
  if (rc) return rc;
  const size_t pb = sizeof(float) * np;
  cudaError_t e = cudaMemcpyAsync(n->m, buf.data() + np, pb, cudaMemcpyHostToDevice, n->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(n->v, buf.data() + 2 * np, pb, cudaMemcpyHostToDevice, n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) {
    fem_mlp_destroy(n);
    fem_set_error("fem_mlp_load: upload failed: %s", cudaGetErrorString(e));
    return FEM_ECUDA;
  }
  n->step = hdr[4];
  *out = n;
  return FEM_OK;
}

extern "C" fem_status fem_mlp_forward(fem_mlp *n, const void *X, int64_t rows, float *Y) {
  if (!n || !X || !Y || rows < 0) { fem_set_error("fem_mlp_forward: invalid arguments"); return FEM_EINVAL; }
  if (rows == 0) return FEM_OK;
  int rc = fem_mlp_forward_rows(n, X, rows, Y);
  if (rc) return rc;
  return fem_mlp_check_tc(n);
}

// One training step on S rows: forward, loss, backward, Adam.  X [S][n_in]
// (compute type), T [S][n_out] fp32 targets, `valid` leading outputs enter
// the loss.  If grad_host != NULL the gradient (fp32, parameter order) is
// copied out and NO update is made (gradient check).  loss_host: the loss.
extern "C" fem_status fem_mlp_train_step(fem_mlp *n, const void *X, const float *T, int64_t S,
                                         int valid, float lr, float *grad_host, double *loss_host) {
  if (!n || !X || !T || S < 32 || S % 32 || valid < 1 || valid > n->n_out) {
    fem_set_error("fem_mlp_train_step: invalid arguments (S must be a positive multiple of 32)");
    return FEM_EINVAL;
  }
  int rc = ensure_cap(n, S);
  if (rc) return rc;
  cudaStream_t s = n->stream;
  const int b16 = n->mode == 0;
  rc = fem_mlp_forward_rows(n, X, S, n->y);
  if (rc) return rc;
  FEM_CUDA_TRY(cudaMemsetAsync(n->loss, 0, sizeof(double), s));
  FEM_CUDA_TRY(cudaMemsetAsync(n->g, 0, sizeof(float) * n->np, s));
  if (b16)
    loss_grad_kernel<__nv_bfloat16><<<296, 256, 0, s>>>(n->y, T, S, n->n_out, valid, (__nv_bfloat16 *)n->dy, n->loss);
  else
    loss_grad_kernel<float><<<296, 256, 0, s>>>(n->y, T, S, n->n_out, valid, (float *)n->dy, n->loss);
  FEM_CHECK_LAUNCH();
  // split K = S over up to 32 z-slices for the weight gradients
  int ks = 1;
  while (ks < 32 && S % (64 * ks) == 0 && S / (2 * ks) >= 512) ks *= 2;
  auto colsum = [&](const void *D, int ncol, float *gout) {
    dim3 grid(256, (ncol + 255) / 256);
    if (b16) colsum_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>((const __nv_bfloat16 *)D, S, ncol, gout);
    else colsum_kernel<float><<<grid, 256, 0, s>>>((const float *)D, S, ncol, gout);
  };
  // layer 3
  GemmArgs a = ga(n->dy, n->n_out, n->h2, n->n_h, n->n_out, n->n_h, (int)S, n->g + off_W3(n), n->n_h, 0);
  a.accumulate = 1; a.ksplit = ks;
  if ((rc = gemm(n, a, true, true))) return rc;
  colsum(n->dy, n->n_out, n->g + off_b3(n));
  a = ga(n->dy, n->n_out, wq_W3(n), n->n_h, S, n->n_h, n->n_out, n->dh, n->n_h, b16);
  a.mask = n->h2; a.ldm = n->n_h;
  if ((rc = gemm(n, a, false, true))) return rc;
  // layer 2: dh holds dH2
  a = ga(n->dh, n->n_h, n->h1, n->n_h, n->n_h, n->n_h, (int)S, n->g + off_W2(n), n->n_h, 0);
  a.accumulate = 1; a.ksplit = ks;
  if ((rc = gemm(n, a, true, true))) return rc;
  colsum(n->dh, n->n_h, n->g + off_b2(n));
  // dH1 into h2's buffer (h2 is no longer needed)
  a = ga(n->dh, n->n_h, wq_W2(n), n->n_h, S, n->n_h, n->n_h, n->h2, n->n_h, b16);
  a.mask = n->h1; a.ldm = n->n_h;
  if ((rc = gemm(n, a, false, true))) return rc;
  // layer 1
  a = ga(n->h2, n->n_h, X, n->n_in, n->n_h, n->n_in, (int)S, n->g + off_W1(n), n->n_in, 0);
  a.accumulate = 1; a.ksplit = ks;
  if ((rc = gemm(n, a, true, true))) return rc;
  colsum(n->h2, n->n_h, n->g + off_b1(n));
  FEM_CHECK_LAUNCH();
  if (grad_host) {
    FEM_CUDA_TRY(cudaMemcpyAsync(grad_host, n->g, sizeof(float) * n->np, cudaMemcpyDeviceToHost, s));
  } else {
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)n->step), c2 = 1.0f - powf(b2, (float)n->step);
    adam_kernel<<<296, 256, 0, s>>>(n->np, n->p, n->g, n->m, n->v, lr, b1, b2, 1e-8f, c1, c2);
    cast_weights_kernel<<<296, 256, 0, s>>>(n->p, off_b1(n), off_W2(n), off_b2(n), off_W3(n),
                                            off_b3(n), n->wq, b16);
    FEM_CHECK_LAUNCH();
  }
  if (loss_host) FEM_CUDA_TRY(cudaMemcpyAsync(loss_host, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  FEM_CUDA_TRY(cudaStreamSynchronize(s));
  return FEM_OK;
}

namespace {
template <typename TX>
__global__ void gather_rows_kernel(const TX *X, const float *T, const int32_t *idx, int64_t rows,
                                   int n_in, int n_out, TX *xb, float *tb) {
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const int64_t s = idx[r];
    for (int c = threadIdx.x; c < n_in; c += blockDim.x) xb[r * n_in + c] = X[s * n_in + c];
    for (int c = threadIdx.x; c < n_out; c += blockDim.x) tb[r * n_out + c] = T[s * n_out + c];
  }
}
uint64_t splitmix64(uint64_t &s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
}  // namespace

// Minibatch Adam training over S samples (X [S][n_in] compute type, T [S][n_out]
// fp32): `epochs` passes, each over a fresh permutation (splitmix64-seeded
// Fisher-Yates on the host), floor(S / batch) steps of `batch` rows.
// loss_host[epochs]: mean training loss of each epoch.
extern "C" fem_status fem_mlp_train(fem_mlp *n, const void *X, const float *T, int64_t S,
                                    int valid, int epochs, int batch, float lr, uint64_t seed,
                                    double *loss_host) {
  if (!n || !X || !T || S < batch || batch < 32 || batch % 32 || epochs < 1) {
    fem_set_error("fem_mlp_train: invalid arguments (batch a multiple of 32, S >= batch)");
    return FEM_EINVAL;
  }
  cudaStream_t s = n->stream;
  const size_t e = esz(n);
  if (n->bcap < batch) {
    cudaFree(n->xb); cudaFree(n->tb);
    if (cudaMalloc(&n->xb, e * batch * n->n_in) != cudaSuccess ||
        cudaMalloc(&n->tb, sizeof(float) * batch * n->n_out) != cudaSuccess) {
      cudaGetLastError();
      n->bcap = 0;
      fem_set_error("fem_mlp_train: allocation failed");
      return FEM_ENOMEM;
    }
    n->bcap = batch;
  }
  if (n->perm_cap < S) {
    cudaFree(n->perm);
    if (cudaMalloc(&n->perm, sizeof(int32_t) * S) != cudaSuccess) {
      cudaGetLastError();
      n->perm_cap = 0;
      fem_set_error("fem_mlp_train: allocation failed");
      return FEM_ENOMEM;
    }
    n->perm_cap = S;
  }
  std::vector<int32_t> perm(S);
  uint64_t st = seed;
  const int64_t steps = S / batch;
  for (int ep = 0; ep < epochs; ep++) {
    for (int64_t i = 0; i < S; i++) perm[i] = (int32_t)i;
    for (int64_t i = S - 1; i > 0; i--) {
      const int64_t j = (int64_t)(splitmix64(st) % (uint64_t)(i + 1));
      int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    FEM_CUDA_TRY(cudaMemcpyAsync(n->perm, perm.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, s));
    double acc = 0.0;
    for (int64_t k = 0; k < steps; k++) {
      if (n->mode == 0)
        gather_rows_kernel<__nv_bfloat16><<<512, 128, 0, s>>>(
            (const __nv_bfloat16 *)X, T, n->perm + k * batch, batch, n->n_in, n->n_out,
            (__nv_bfloat16 *)n->xb, n->tb);
      else
        gather_rows_kernel<float><<<512, 128, 0, s>>>((const float *)X, T, n->perm + k * batch,
                                                      batch, n->n_in, n->n_out, (float *)n->xb, n->tb);
      FEM_CHECK_LAUNCH();
      double L = 0.0;
      int rc = fem_mlp_train_step(n, n->xb, n->tb, batch, valid, lr, nullptr, &L);
      if (rc) return rc;
      acc += L;
    }
    if (loss_host) loss_host[ep] = acc / steps;
  }
  return fem_mlp_check_tc(n);
}

// Minibatch training until the loss stops falling: chunks of `chunk` epochs
// (each a fem_mlp_train call with its own permutation seed), stopped when a
// chunk's mean loss is not below (1 - rel_tol) times the previous chunk's, or
// after max_epochs.  loss_host[max_epochs]: the mean loss per epoch run;
// *epochs_run: how many ran.
extern "C" fem_status fem_mlp_train_plateau(fem_mlp *n, const void *X, const float *T, int64_t S,
                                            int valid, int max_epochs, int chunk, double rel_tol,
                                            int batch, float lr, uint64_t seed, double *loss_host,
                                            int *epochs_run) {
  if (!n || !loss_host || !epochs_run || max_epochs < 1 || chunk < 1 || !(rel_tol >= 0.0)) {
    fem_set_error("fem_mlp_train_plateau: invalid arguments");
    return FEM_EINVAL;
  }
  int done = 0;
  double prev = INFINITY;
  while (done < max_epochs) {
    const int k = chunk < max_epochs - done ? chunk : max_epochs - done;
    const int rc = fem_mlp_train(n, X, T, S, valid, k, batch, lr,
                                 seed + 0x9E3779B97F4A7C15ull * (uint64_t)(done + 1), loss_host + done);
    if (rc) return rc;
    double mean = 0.0;
    for (int i = 0; i < k; i++) mean += loss_host[done + i] / k;
    done += k;
    if (!(mean < (1.0 - rel_tol) * prev)) break;
    prev = mean;
  }
  *epochs_run = done;
  return FEM_OK;
}
