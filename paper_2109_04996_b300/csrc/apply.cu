// Fused operator apply  y = G^T B^T D B G x  (section "libCEED": the
// operator decomposition; the fused single-kernel form of section "Nek and
// MFEM" / "libCEED" CPU and GPU performance).  One kernel per call:
//
//   G    gather of the element's (p+1)^3 values through elem_nodes,
//   B    sum-factorized interpolation to the q^3 quadrature points, one
//        direction at a time (section "Benchmarks", tensor-product sum
//        factorization), then the gradient on the quadrature points with the
//        collocated 1D derivative Dq (exact: the interpolant has degree p < q),
//   D    the pointwise 3x3 symmetric data (diffusion) or w det J (mass),
//   B^T  the transposed contractions in reverse order,
//   G^T  atomic scatter-add into y.
//
// Thread layout: q x q threads per element ("slab"); thread (i, j) owns the
// column of quadrature points (i, j, 0..q-1) in registers, contractions along
// the third direction stay in registers, the other two go through a q^3 cube
// in shared memory.  Several elements share a block; blocks loop over element
// groups (grid-stride) so that the grid is a small multiple of the SM count.
// Gauss-Lobatto with q = p+1 (BP5/BP6) skips the interpolation (identity).
#include "fem_internal.h"

namespace {

template <typename T>
struct ApplyParams {
  const T *x;
  T *y;
  const int32_t *elem_nodes;  // [E][P^3]
  const int32_t *list;        // optional element list
  int64_t nsel;               // number of elements to process
  int64_t N;
  int ncomp;
  const T *qdata;             // [E][nd][Q^3]
  const T *B;                 // [Q][P]
  const T *Dq;                // [Q][Q]
  double *partials;           // fused x.y (optional)
  unsigned *counter;
  double *dot_out;
};

template <int Q>
struct ApplyShape {
  static constexpr int Q2 = Q * Q;
  // elements per block: about 256 threads
  static constexpr int EPB = (256 / Q2) > 0 ? (256 / Q2) : 1;
  // block size rounded up to whole warps; the extra threads ("padding") share
  // the last slot's shared memory for reads but never write it
  static constexpr int NT = ((Q2 * EPB + 31) / 32) * 32;
};

template <typename T>
__device__ __forceinline__ void atomic_add(T *a, T v) { atomicAdd(a, v); }

template <typename T, int P, int Q, int KIND, bool COLLOC>
__global__ void __launch_bounds__(ApplyShape<Q>::NT)
    fem_apply_kernel(const ApplyParams<T> prm) {
  using S = ApplyShape<Q>;
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q, P2 = P * P, P3 = P * P * P;
  constexpr int ND = (KIND == FEM_DIFFUSION) ? 6 : 1;
  constexpr int NCUBE = (KIND == FEM_DIFFUSION) ? 3 : 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sB = reinterpret_cast<T *>(smem_raw);  // [Q][P]
  T *sD = sB + Q * P;                       // [Q][Q]
  T *cube = sD + Q * Q;
  const int slot_raw = threadIdx.x / Q2;
  const bool live = slot_raw < S::EPB;  // false for padding threads
  const int slot = live ? slot_raw : S::EPB - 1;
  const int t = threadIdx.x - slot_raw * Q2;
  const int tx = t % Q, ty = t / Q;
  T *su = cube + slot * NCUBE * Q3;
  T *sv = su + Q3;
  T *sw = (NCUBE == 3) ? sv + Q3 : sv;
  for (int i = threadIdx.x; i < Q * P; i += blockDim.x) sB[i] = prm.B[i];
  for (int i = threadIdx.x; i < Q * Q; i += blockDim.x) sD[i] = prm.Dq[i];
  __syncthreads();

  double dot = 0.0;
  const int64_t N = prm.N;
  const int64_t ngroups = (prm.nsel + S::EPB - 1) / S::EPB;
  for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const int64_t k_el = g * S::EPB + slot_raw;
    const bool valid = live && (k_el < prm.nsel);
    int64_t e = 0;
    if (valid) e = prm.list ? (int64_t)prm.list[k_el] : k_el;
    const int32_t *en = prm.elem_nodes + e * P3;
    const T *qd = prm.qdata + e * (int64_t)(ND * Q3) + (ty * Q + tx);
    for (int c = 0; c < prm.ncomp; c++) {
      const T *xc = prm.x + c * N;
      T *yc = prm.y + c * N;
      if constexpr (COLLOC && KIND == FEM_MASS) {
        // B = I and D diagonal: y_e = (w det J) x_e
        if (valid) {
#pragma unroll
          for (int k = 0; k < Q; k++) {
            const int64_t gi = en[tx + P * ty + P2 * k];
            const T xv = xc[gi];
            const T v = qd[k * Q2] * xv;
            atomic_add(&yc[gi], v);
            dot += (double)v * (double)xv;
          }
        }
      } else if constexpr (COLLOC) {
        // ---- BP5/BP6: gradients directly on the Gauss-Lobatto nodes
        T u[Q];
#pragma unroll
        for (int k = 0; k < Q; k++) u[k] = valid ? xc[en[tx + P * ty + P2 * k]] : T(0);
        if (live) {
#pragma unroll
          for (int k = 0; k < Q; k++) su[(k * Q + ty) * Q + tx] = u[k];
        }
        __syncthreads();
        T gx[Q], gy[Q], gz[Q];
#pragma unroll
        for (int k = 0; k < Q; k++) {
          T sx = 0, sy = 0, sz = 0;
#pragma unroll
          for (int m = 0; m < Q; m++) {
            sx += sD[tx * Q + m] * su[(k * Q + ty) * Q + m];
            sy += sD[ty * Q + m] * su[(k * Q + m) * Q + tx];
            sz += sD[k * Q + m] * u[m];
          }
          gx[k] = sx; gy[k] = sy; gz[k] = sz;
        }
#pragma unroll
        for (int k = 0; k < Q; k++) {
          T G00 = 0, G11 = 0, G22 = 0, G12 = 0, G02 = 0, G01 = 0;
          if (valid) {
            const T *qk = qd + k * Q2;
            G00 = qk[0]; G11 = qk[Q3]; G22 = qk[2 * Q3];
            G12 = qk[3 * Q3]; G02 = qk[4 * Q3]; G01 = qk[5 * Q3];
          }
          const T vx = G00 * gx[k] + G01 * gy[k] + G02 * gz[k];
          const T vy = G01 * gx[k] + G11 * gy[k] + G12 * gz[k];
          const T vz = G02 * gx[k] + G12 * gy[k] + G22 * gz[k];
          if (live) {
            sv[(k * Q + ty) * Q + tx] = vx;
            sw[(k * Q + ty) * Q + tx] = vy;
          }
          gz[k] = vz;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < Q; k++) {
          T s = 0;
#pragma unroll
          for (int m = 0; m < Q; m++) {
            s += sD[m * Q + tx] * sv[(k * Q + ty) * Q + m];
            s += sD[m * Q + ty] * sw[(k * Q + m) * Q + tx];
            s += sD[m * Q + k] * gz[m];
          }
          if (valid) {
            const int64_t gi = en[tx + P * ty + P2 * k];
            atomic_add(&yc[gi], s);
            dot += (double)s * (double)u[k];
          }
        }
      } else {
        // ---- Gauss-Legendre: interpolate, (gradient), D, transposes
        const bool own = (tx < P) && (ty < P);
        T r[P];
#pragma unroll
        for (int k = 0; k < P; k++) r[k] = (valid && own) ? xc[en[tx + P * ty + P2 * k]] : T(0);
        T tq[Q];
        // B along z (registers)
#pragma unroll
        for (int kq = 0; kq < Q; kq++) {
          T s = 0;
#pragma unroll
          for (int k = 0; k < P; k++) s += sB[kq * P + k] * r[k];
          tq[kq] = s;
        }
        if (own && live) {
#pragma unroll
          for (int kq = 0; kq < Q; kq++) su[(kq * Q + ty) * Q + tx] = tq[kq];
        }
        __syncthreads();
        // B along y: thread (i < P, jq)
        if (tx < P && live) {
#pragma unroll
          for (int kq = 0; kq < Q; kq++) {
            T s = 0;
#pragma unroll
            for (int j = 0; j < P; j++) s += sB[ty * P + j] * su[(kq * Q + j) * Q + tx];
            sv[(kq * Q + ty) * Q + tx] = s;
          }
        }
        __syncthreads();
        // B along x: thread (iq, jq) -> values at its column of quadrature points
#pragma unroll
        for (int kq = 0; kq < Q; kq++) {
          T s = 0;
#pragma unroll
          for (int i = 0; i < P; i++) s += sB[tx * P + i] * sv[(kq * Q + ty) * Q + i];
          tq[kq] = s;
        }
        if constexpr (KIND == FEM_MASS) {
#pragma unroll
          for (int kq = 0; kq < Q; kq++) {
            const T w = valid ? qd[kq * Q2] : T(0);
            if (live) su[(kq * Q + ty) * Q + tx] = w * tq[kq];
          }
          __syncthreads();
        } else {
          if (live) {
#pragma unroll
            for (int kq = 0; kq < Q; kq++) su[(kq * Q + ty) * Q + tx] = tq[kq];
          }
          __syncthreads();
          T gx[Q], gy[Q], gz[Q];
#pragma unroll
          for (int kq = 0; kq < Q; kq++) {
            T sx = 0, sy = 0, sz = 0;
#pragma unroll
            for (int m = 0; m < Q; m++) {
              sx += sD[tx * Q + m] * su[(kq * Q + ty) * Q + m];
              sy += sD[ty * Q + m] * su[(kq * Q + m) * Q + tx];
              sz += sD[kq * Q + m] * tq[m];
            }
            gx[kq] = sx; gy[kq] = sy; gz[kq] = sz;
          }
#pragma unroll
          for (int kq = 0; kq < Q; kq++) {
            T G00 = 0, G11 = 0, G22 = 0, G12 = 0, G02 = 0, G01 = 0;
            if (valid) {
              const T *qk = qd + kq * Q2;
              G00 = qk[0]; G11 = qk[Q3]; G22 = qk[2 * Q3];
              G12 = qk[3 * Q3]; G02 = qk[4 * Q3]; G01 = qk[5 * Q3];
            }
            const T vx = G00 * gx[kq] + G01 * gy[kq] + G02 * gz[kq];
            const T vy = G01 * gx[kq] + G11 * gy[kq] + G12 * gz[kq];
            const T vz = G02 * gx[kq] + G12 * gy[kq] + G22 * gz[kq];
            if (live) {
              sv[(kq * Q + ty) * Q + tx] = vx;
              sw[(kq * Q + ty) * Q + tx] = vy;
            }
            gz[kq] = vz;
          }
          __syncthreads();
          // transposed gradient, back on the quadrature points
#pragma unroll
          for (int kq = 0; kq < Q; kq++) {
            T s = 0;
#pragma unroll
            for (int m = 0; m < Q; m++) {
              s += sD[m * Q + tx] * sv[(kq * Q + ty) * Q + m];
              s += sD[m * Q + ty] * sw[(kq * Q + m) * Q + tx];
              s += sD[m * Q + kq] * gz[m];
            }
            tq[kq] = s;
          }
          if (live) {
#pragma unroll
            for (int kq = 0; kq < Q; kq++) su[(kq * Q + ty) * Q + tx] = tq[kq];
          }
          __syncthreads();
        }
        // B^T along x: thread (i < P, jq)
        if (tx < P && live) {
#pragma unroll
          for (int kq = 0; kq < Q; kq++) {
            T s = 0;
#pragma unroll
            for (int m = 0; m < Q; m++) s += sB[m * P + tx] * su[(kq * Q + ty) * Q + m];
            sv[(kq * Q + ty) * Q + tx] = s;
          }
        }
        __syncthreads();
        if (own) {
          // B^T along y: thread (i, j)
#pragma unroll
          for (int kq = 0; kq < Q; kq++) {
            T s = 0;
#pragma unroll
            for (int m = 0; m < Q; m++) s += sB[m * P + ty] * sv[(kq * Q + m) * Q + tx];
            tq[kq] = s;
          }
          // B^T along z (registers) and scatter-add
#pragma unroll
          for (int k = 0; k < P; k++) {
            T s = 0;
#pragma unroll
            for (int kq = 0; kq < Q; kq++) s += sB[kq * P + k] * tq[kq];
            if (valid) {
              const int64_t gi = en[tx + P * ty + P2 * k];
              atomic_add(&yc[gi], s);
              dot += (double)s * (double)r[k];
            }
          }
        }
      }
    }
  }
  if (prm.dot_out) {
    double v[1] = {dot};
    __shared__ double tot[1];
    if (fem_grid_sum<1>(v, prm.partials, prm.counter, tot) && threadIdx.x == 0)
      *prm.dot_out = tot[0];
  }
}

template <typename T, int P, int Q, int KIND, bool COLLOC>
int launch_one(fem_op *op, const ApplyParams<T> &prm) {
  using S = ApplyShape<Q>;
  constexpr int NCUBE = (KIND == FEM_DIFFUSION) ? 3 : 2;
  const size_t smem = sizeof(T) * (Q * P + Q * Q + (size_t)S::EPB * NCUBE * Q * Q * Q);
  auto kern = fem_apply_kernel<T, P, Q, KIND, COLLOC>;
  static bool attr_set = false;
  if (!attr_set) {
    FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
  }
  int dev = 0, nsm = 0, per_sm = 0;
  FEM_CUDA_TRY(cudaGetDevice(&dev));
  FEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, S::NT, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t ngroups = (prm.nsel + S::EPB - 1) / S::EPB;
  int64_t grid = (int64_t)nsm * per_sm;
  if (grid > ngroups) grid = ngroups;
  if (grid > FEM_MAX_BLOCKS) grid = FEM_MAX_BLOCKS;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, S::NT, smem, op->stream()>>>(prm);
  FEM_CHECK_LAUNCH();
  return FEM_OK;
}

template <typename T, int P>
int dispatch_q(fem_op *op, const ApplyParams<T> &prm) {
  constexpr int QG = (P + 1 <= FEM_MAX_Q) ? P + 1 : P;
  const bool diff = op->kind == FEM_DIFFUSION;
  if (op->Q == P) {
    if (op->colloc)
      return diff ? launch_one<T, P, P, FEM_DIFFUSION, true>(op, prm)
                  : launch_one<T, P, P, FEM_MASS, true>(op, prm);
    return diff ? launch_one<T, P, P, FEM_DIFFUSION, false>(op, prm)
                : launch_one<T, P, P, FEM_MASS, false>(op, prm);
  }
  if (op->Q == P + 1 && QG == P + 1)
    return diff ? launch_one<T, P, QG, FEM_DIFFUSION, false>(op, prm)
                : launch_one<T, P, QG, FEM_MASS, false>(op, prm);
  fem_set_error("apply: unsupported (P, q) = (%d, %d)", P, op->Q);
  return FEM_EINVAL;
}

template <typename T>
int dispatch(fem_op *op, const ApplyParams<T> &prm) {
  switch (op->P) {
    case 2: return dispatch_q<T, 2>(op, prm);
    case 3: return dispatch_q<T, 3>(op, prm);
    case 4: return dispatch_q<T, 4>(op, prm);
    case 5: return dispatch_q<T, 5>(op, prm);
    case 6: return dispatch_q<T, 6>(op, prm);
    case 7: return dispatch_q<T, 7>(op, prm);
    case 8: return dispatch_q<T, 8>(op, prm);
    case 9: return dispatch_q<T, 9>(op, prm);
  }
  fem_set_error("apply: unsupported P = %d", op->P);
  return FEM_EINVAL;
}

}  // namespace

int fem_launch_apply_f64(fem_op *op, const double *x, double *y,
                         const int32_t *list, int64_t nsel, double *dot_out) {
  ApplyParams<double> prm;
  prm.x = x; prm.y = y;
  prm.elem_nodes = op->mesh->d_elem_nodes;
  prm.list = list; prm.nsel = nsel;
  prm.N = op->N; prm.ncomp = op->ncomp;
  prm.qdata = op->d_qdata; prm.B = op->d_B; prm.Dq = op->d_Dq;
  prm.partials = op->d_partials; prm.counter = op->d_counter; prm.dot_out = dot_out;
  if (nsel == 0) return FEM_OK;
  return dispatch<double>(op, prm);
}

int fem_launch_apply_f32(fem_op *op, const float *x, float *y,
                         const int32_t *list, int64_t nsel, double *dot_out) {
  if (!op->d_qdata32) {
    fem_set_error("apply_f32: operator was not created with FEM_F32");
    return FEM_EINVAL;
  }
  ApplyParams<float> prm;
  prm.x = x; prm.y = y;
  prm.elem_nodes = op->mesh->d_elem_nodes;
  prm.list = list; prm.nsel = nsel;
  prm.N = op->N; prm.ncomp = op->ncomp;
  prm.qdata = op->d_qdata32; prm.B = op->d_B32; prm.Dq = op->d_Dq32;
  prm.partials = op->d_partials; prm.counter = op->d_counter; prm.dot_out = dot_out;
  if (nsel == 0) return FEM_OK;
  return dispatch<float>(op, prm);
}
