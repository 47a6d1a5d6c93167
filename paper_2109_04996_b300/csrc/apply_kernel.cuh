// Templates of the fused operator apply  y = G^T B^T D B G x  (section
// "libCEED": operator decomposition; fused single-kernel operator).  Shared by
// the single-operator kernels (apply_f64.cu, apply_f32.cu) and the batched
// persistent solver (batch.cu).
//
// Per element:
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
// in shared memory.  EPB elements share a block (the autotuned shape); blocks
// loop over element groups.  Gauss-Lobatto with q = p+1 (BP5/BP6) skips the
// interpolation (identity).
#pragma once
#include <type_traits>

#include "dw.cuh"
#include "fem_internal.h"

namespace fem_apply {

// Storage of the vectors and of the pointwise data for arithmetic type T:
// T itself for FP64 and FP32; the double-word bodies (T = dw) read and
// write the FP64 vectors, splitting each gathered x value into a double word
// by integer operations and rounding each element result back to FP64, and
// read the operator's double-word copy of the qdata (split once at set-up:
// FP64 <-> FP32 conversions run at the FP64 rate).
template <typename T>
struct Store {
  using V = T;   // x, y
  using Q = T;   // qdata, tables
};
template <>
struct Store<dw> {
  using V = double;
  using Q = dw;
};

// Value of a stored entry in arithmetic type T.
template <typename T, typename S>
__device__ __forceinline__ T to_arith(S v) {
  if constexpr (std::is_same<T, dw>::value && std::is_same<S, double>::value)
    return dw_from_double_int(v);
  else return v;
}

template <typename T>
struct ApplyParams {
  using V = typename Store<T>::V;
  using QS = typename Store<T>::Q;
  const V *x;
  V *y;
  const int32_t *elem_nodes;  // [E][P^3]
  const int32_t *list;        // optional element list
  int64_t nsel;               // number of elements to process
  int64_t N;
  int ncomp;
  const QS *qdata;            // [E][nd][Q^3]
  const QS *B;                // [Q][P]
  const QS *Dq;               // [Q][Q]
  double *partials;           // fused x.y (optional)
  unsigned *counter;
  double *dot_out;
  int x_l2_only = 0;          // 1: gather x with L2-only loads (x written by
                              // other blocks of a persistent kernel)
  int want_dot = 0;           // 1: accumulate x.y into the caller's `dot` even
                              // without dot_out (persistent batch kernel)
  const int *skip = nullptr;  // *skip != 0: the launch does nothing (a solve
                              // whose loop body outlived its convergence)
};

// Uniform early exit of a launch whose solve has finished (read once, before
// any barrier, by every thread).
template <typename T>
__device__ __forceinline__ bool apply_skipped(const ApplyParams<T> &prm) {
  return prm.skip && *(volatile const int *)prm.skip;
}

// Accumulator of a thread's share of x.y over one element.  FP64: plain.
// FP32: compensated (double-float) on the FP32 pipe -- each product is split
// exactly, a*b = p + e (FMA), p is added to hi by TwoSum and the rounding
// errors are collected in lo (Dekker 1971; Ogita, Rump & Oishi 2005) -- so
// that the FP32 kernel neither loses p^T A p to cancellation between a node's
// terms nor uses the 1/73-rate FP64 pipe per term.
template <typename T>
struct DotAcc {
  T v = 0;
  __device__ __forceinline__ void add(T a, T b) { v += a * b; }
  __device__ __forceinline__ double get() const { return (double)v; }
};
template <>
struct DotAcc<float> {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float s = hi + p;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += err + e;
  }
  __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};

// Double word: TwoSum accumulation of the exact double-word products.
template <>
struct DotAcc<dw> {
  dw v = dw(0.0f, 0.0f);
  __device__ __forceinline__ void add(dw a, dw b) { v += a * b; }
  __device__ __forceinline__ double get() const { return dw_to_double(v); }
};

template <typename T>
__device__ __forceinline__ T gather_load(const T *p, int l2_only) {
  return l2_only ? __ldcg(p) : *p;
}

// x entry in arithmetic type T (the double-word bodies split the FP64 value).
template <typename T, typename S>
__device__ __forceinline__ T gather_arith(const S *p, int l2_only) {
  return to_arith<T>(gather_load(p, l2_only));
}

// A pointwise-data entry in arithmetic type T.  The double-word bodies load
// their (h, l) pairs through the read-only path (ld.global.nc): the loads
// then cannot alias the shared-memory stores of the stage around them, so
// the compiler may issue the next point's loads ahead of those stores.
template <typename T, typename S>
__device__ __forceinline__ T ld_qdata(const S *p) {
  if constexpr (std::is_same<T, dw>::value && std::is_same<S, dw>::value) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return dw(v.x, v.y);
  } else {
    return to_arith<T>(*p);
  }
}

// The double-word diffusion bodies apply A_e to x_e - c 1 (c = x at the
// element's local node 0) instead of x_e: A_e annihilates constants, so the
// result and the element's x_e^T A_e x_e are unchanged, but the values that
// enter the double-word contractions are differences of nearby nodal values
// (the FP64 subtraction is exact for close values, Sterbenz 1974) rather
// than the values themselves.  The ~2^-47 relative noise of double-word
// arithmetic then scales with h |grad x| instead of |x|, which keeps smooth
// inputs -- whose gradients are interpolated from nearly equal values --
// within FP64-level accuracy.
template <typename T, int KIND>
struct ShiftX {
  static constexpr bool value = std::is_same<T, dw>::value && KIND == FEM_DIFFUSION;
};

template <typename T, bool SH, typename S>
__device__ __forceinline__ T gather_shifted(const S *p, int l2_only, double c) {
  if constexpr (SH) return to_arith<T>((double)gather_load(p, l2_only) - c);
  else return gather_arith<T>(p, l2_only);
}

// Elements per block of the default shape: about 256 threads.
template <int Q>
struct DefaultEpb {
  static constexpr int value = (256 / (Q * Q)) > 0 ? (256 / (Q * Q)) : 1;
};

template <int Q, int EPB>
struct ApplyShape {
  static constexpr int Q2 = Q * Q;
  // block size rounded up to whole warps; the extra threads ("padding") share
  // the last slot's shared memory for reads but never write it
  static constexpr int NT = ((Q2 * EPB + 31) / 32) * 32;
};

// The collocated FP32 diffusion kernel (BP5/BP6) stages each element group's
// pointwise data (6 q^3 values per element) in shared memory with cp.async,
// issued when the group starts so that its HBM latency hides behind the
// gather and the gradients.  (Measured: faster for the collocated kernel,
// slower for the Gauss-Legendre one, whose shared-memory traffic is higher;
// the FP64 kernels are bound by the FP64 pipe and read qdata directly.)
template <typename T, int KIND, bool COLLOC = true>
struct StageQ {
  static constexpr bool value = sizeof(T) == 4 && KIND == FEM_DIFFUSION && COLLOC;
};

// shared-memory offset (in T) of the staged qdata: after the tables and the
// cubes, rounded up to 16 bytes
template <typename T, int Q, int P, int KIND, int EPB>
constexpr size_t stage_offset() {
  const size_t o = Q * P + Q * Q + (size_t)EPB * ((KIND == FEM_DIFFUSION) ? 3 : 2) * Q * Q * Q;
  const size_t per16 = 16 / sizeof(T);
  return (o + per16 - 1) / per16 * per16;
}

template <typename T, int Q, int P, int KIND, int EPB, bool COLLOC = false>
constexpr size_t apply_smem_bytes() {
  return sizeof(T) * (stage_offset<T, Q, P, KIND, EPB>() +
                      (StageQ<T, KIND, COLLOC>::value ? (size_t)EPB * 6 * Q * Q * Q : 0));
}

// Row `row` of a shared table with `stride` between entries, into registers.
// (Loaded once per stage: the compiler cannot hoist these loads out of the
// stage loops itself because the loops also store to shared memory.)
template <int N, typename T>
__device__ __forceinline__ void load_row(const T *base, int stride, T (&out)[N]) {
#pragma unroll
  for (int m = 0; m < N; m++) out[m] = base[m * stride];
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Bulk prefetch of [p, p + bytes) into L2 (one instruction, nothing to wait
// for).  The range is shrunk to whole 16-byte units inside it (start rounded
// up, end rounded down), so that it never leaves the buffer it came from.
__device__ __forceinline__ void prefetch_l2(const void *p, size_t bytes) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uintptr_t lo = (a + 15) & ~(uintptr_t)15, hi = (a + bytes) & ~(uintptr_t)15;
  if (hi <= lo) return;
  size_t n = hi - lo;
  uintptr_t s = lo;
  // in pieces of at most 64 KB
  while (n > 0) {
    const unsigned piece = n > 65536 ? 65536u : (unsigned)n;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(s), "r"(piece) : "memory");
    s += piece;
    n -= piece;
  }
}

template <typename T>
__device__ __forceinline__ void atomic_add(T *a, T v) { atomicAdd(a, v); }
__device__ __forceinline__ void atomic_add(double *a, dw v) { atomicAdd(a, dw_to_double_int(v)); }

// Thread-local view of one block: slot, slab coordinates and shared buffers.
template <typename T, int P, int Q, int KIND, int EPB>
struct Slab {
  int slot_raw, slot, tx, ty;
  bool live;
  T *sB, *sD, *su, *sv, *sw;
  T *sq;   // staged qdata of the group [EPB][6][q^3] (FP32 diffusion)
  __device__ Slab(unsigned char *smem_raw) {
    constexpr int Q2 = Q * Q, Q3 = Q * Q * Q;
    constexpr int NCUBE = (KIND == FEM_DIFFUSION) ? 3 : 2;
    sB = reinterpret_cast<T *>(smem_raw);
    sD = sB + Q * P;
    T *cube = sD + Q * Q;
    slot_raw = threadIdx.x / Q2;
    live = slot_raw < EPB;
    slot = live ? slot_raw : EPB - 1;
    const int t = threadIdx.x - slot_raw * Q2;
    tx = t % Q; ty = t / Q;
    su = cube + slot * NCUBE * Q3;
    sv = su + Q3;
    sw = (NCUBE == 3) ? sv + Q3 : sv;
    sq = reinterpret_cast<T *>(smem_raw) + stage_offset<T, Q, P, KIND, EPB>();
  }
  __device__ void load_tables(const T *B, const T *Dq) {
    for (int i = threadIdx.x; i < Q * P; i += blockDim.x) sB[i] = B[i];
    for (int i = threadIdx.x; i < Q * Q; i += blockDim.x) sD[i] = Dq[i];
  }
};

// One group of EPB elements (elements g*EPB .. g*EPB + EPB - 1 of the
// selection), all components.  Every thread of the block calls it (it
// synchronizes the block).  Adds this thread's share of x.y to `dot`.
template <typename T, int P, int Q, int KIND, bool COLLOC, int EPB>
__device__ __forceinline__ void apply_group(const ApplyParams<T> &prm, int64_t g,
                                            const Slab<T, P, Q, KIND, EPB> &sl, double &dot) {
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q, P2 = P * P, P3 = P * P * P;
  constexpr int ND = (KIND == FEM_DIFFUSION) ? 6 : 1;
  const int tx = sl.tx, ty = sl.ty;
  const bool live = sl.live;
  const T *sB = sl.sB;
  const T *sD = sl.sD;
  T *su = sl.su, *sv = sl.sv, *sw = sl.sw;
  (void)sw;
  const int64_t N = prm.N;
  const int64_t k_el = g * EPB + sl.slot_raw;
  const bool valid = live && (k_el < prm.nsel);
  int64_t e = 0;
  if (valid) e = prm.list ? (int64_t)prm.list[k_el] : k_el;
  const int32_t *en = prm.elem_nodes + e * P3;
  constexpr bool STAGE = StageQ<T, KIND, COLLOC>::value;
  const T *qd = prm.qdata + e * (int64_t)(ND * Q3) + (ty * Q + tx);
  if constexpr (STAGE) {
    // all threads copy the group's qdata (8-byte chunks: 6 q^3 is even)
    for (int s_ = 0; s_ < EPB; s_++) {
      const int64_t ks = g * EPB + s_;
      if (ks >= prm.nsel) break;
      const int64_t es = prm.list ? (int64_t)prm.list[ks] : ks;
      const T *src = prm.qdata + es * (int64_t)(6 * Q3);
      T *dst = sl.sq + s_ * 6 * Q3;
      for (int ch = threadIdx.x; ch < 3 * Q3; ch += blockDim.x) cp_async8(dst + 2 * ch, src + 2 * ch);
    }
    cp_async_commit();
    qd = sl.sq + sl.slot * 6 * Q3 + (ty * Q + tx);
  }
  // this thread's share of x.y over the group (see DotAcc), added to the
  // FP64 `dot` once
  DotAcc<T> dl;
    for (int c = 0; c < prm.ncomp; c++) {
      const T *xc = prm.x + c * N;
      T *yc = prm.y + c * N;
      if constexpr (COLLOC && KIND == FEM_MASS) {
        // B = I and D diagonal: y_e = (w det J) x_e
        if (valid) {
#pragma unroll
          for (int k = 0; k < Q; k++) {
            const int64_t gi = en[tx + P * ty + P2 * k];
            const T xv = gather_load(&xc[gi], prm.x_l2_only);
            const T v = qd[k * Q2] * xv;
            atomic_add(&yc[gi], v);
            dl.add(v, xv);
          }
        }
      } else if constexpr (COLLOC) {
        // ---- BP5/BP6: gradients directly on the Gauss-Lobatto nodes
        T u[Q];
#pragma unroll
        for (int k = 0; k < Q; k++) u[k] = valid ? gather_load(&xc[en[tx + P * ty + P2 * k]], prm.x_l2_only) : T(0);
        if (live) {
#pragma unroll
          for (int k = 0; k < Q; k++) su[(k * Q + ty) * Q + tx] = u[k];
        }
        __syncthreads();
        T gx[Q], gy[Q], gz[Q];
        {
          T dX[Q], dY[Q];
          load_row<Q>(sD + tx * Q, 1, dX);
          load_row<Q>(sD + ty * Q, 1, dY);
#pragma unroll
          for (int k = 0; k < Q; k++) {
            T sx = 0, sy = 0, sz = 0;
#pragma unroll
            for (int m = 0; m < Q; m++) {
              sx += dX[m] * su[(k * Q + ty) * Q + m];
              sy += dY[m] * su[(k * Q + m) * Q + tx];
              sz += sD[k * Q + m] * u[m];
            }
            gx[k] = sx; gy[k] = sy; gz[k] = sz;
          }
        }
        if constexpr (STAGE) {
          if (c == 0) { cp_async_wait_all(); __syncthreads(); }
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
        T dXT[Q], dYT[Q];
        load_row<Q>(sD + tx, Q, dXT);
        load_row<Q>(sD + ty, Q, dYT);
#pragma unroll
        for (int k = 0; k < Q; k++) {
          T s = 0;
#pragma unroll
          for (int m = 0; m < Q; m++) {
            s += dXT[m] * sv[(k * Q + ty) * Q + m];
            s += dYT[m] * sw[(k * Q + m) * Q + tx];
            s += sD[m * Q + k] * gz[m];
          }
          if (valid) {
            const int64_t gi = en[tx + P * ty + P2 * k];
            atomic_add(&yc[gi], s);
            dl.add(s, u[k]);
          }
        }
      } else {
        // ---- Gauss-Legendre: interpolate, (gradient), D, transposes
        const bool own = (tx < P) && (ty < P);
        T r[P];
#pragma unroll
        for (int k = 0; k < P; k++) r[k] = (valid && own) ? gather_load(&xc[en[tx + P * ty + P2 * k]], prm.x_l2_only) : T(0);
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
          T bY[P];
          load_row<P>(sB + ty * P, 1, bY);
#pragma unroll
          for (int kq = 0; kq < Q; kq++) {
            T s = 0;
#pragma unroll
            for (int j = 0; j < P; j++) s += bY[j] * su[(kq * Q + j) * Q + tx];
            sv[(kq * Q + ty) * Q + tx] = s;
          }
        }
        __syncthreads();
        // B along x: thread (iq, jq) -> values at its column of quadrature points
        {
          T bX[P];
          load_row<P>(sB + tx * P, 1, bX);
#pragma unroll
          for (int kq = 0; kq < Q; kq++) {
            T s = 0;
#pragma unroll
            for (int i = 0; i < P; i++) s += bX[i] * sv[(kq * Q + ty) * Q + i];
            tq[kq] = s;
          }
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
          {
            T dX[Q], dY[Q];
            load_row<Q>(sD + tx * Q, 1, dX);
            load_row<Q>(sD + ty * Q, 1, dY);
#pragma unroll
            for (int kq = 0; kq < Q; kq++) {
              T sx = 0, sy = 0, sz = 0;
#pragma unroll
              for (int m = 0; m < Q; m++) {
                sx += dX[m] * su[(kq * Q + ty) * Q + m];
                sy += dY[m] * su[(kq * Q + m) * Q + tx];
                sz += sD[kq * Q + m] * tq[m];
              }
              gx[kq] = sx; gy[kq] = sy; gz[kq] = sz;
            }
          }
          if constexpr (STAGE) {
            if (c == 0) { cp_async_wait_all(); __syncthreads(); }
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
          {
            T dXT[Q], dYT[Q];
            load_row<Q>(sD + tx, Q, dXT);
            load_row<Q>(sD + ty, Q, dYT);
#pragma unroll
            for (int kq = 0; kq < Q; kq++) {
              T s = 0;
#pragma unroll
              for (int m = 0; m < Q; m++) {
                s += dXT[m] * sv[(kq * Q + ty) * Q + m];
                s += dYT[m] * sw[(kq * Q + m) * Q + tx];
                s += sD[m * Q + kq] * gz[m];
              }
              tq[kq] = s;
            }
          }
          if (live) {
#pragma unroll
            for (int kq = 0; kq < Q; kq++) su[(kq * Q + ty) * Q + tx] = tq[kq];
          }
          __syncthreads();
        }
        // B^T along x: thread (i < P, jq)
        if (tx < P && live) {
          T bXT[Q];
          load_row<Q>(sB + tx, P, bXT);
#pragma unroll
          for (int kq = 0; kq < Q; kq++) {
            T s = 0;
#pragma unroll
            for (int m = 0; m < Q; m++) s += bXT[m] * su[(kq * Q + ty) * Q + m];
            sv[(kq * Q + ty) * Q + tx] = s;
          }
        }
        __syncthreads();
        if (own) {
          // B^T along y: thread (i, j)
          {
            T bYT[Q];
            load_row<Q>(sB + ty, P, bYT);
#pragma unroll
            for (int kq = 0; kq < Q; kq++) {
              T s = 0;
#pragma unroll
              for (int m = 0; m < Q; m++) s += bYT[m] * sv[(kq * Q + m) * Q + tx];
              tq[kq] = s;
            }
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
              dl.add(s, r[k]);
            }
          }
        }
      }
    }
  if (prm.dot_out || prm.want_dot) dot += dl.get();
}

template <typename T, int P, int Q, int KIND, bool COLLOC, int EPB>
__global__ void __launch_bounds__(ApplyShape<Q, EPB>::NT)
    fem_apply_kernel(const ApplyParams<T> prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (apply_skipped(prm)) return;
  Slab<T, P, Q, KIND, EPB> sl(smem_raw);
  sl.load_tables(prm.B, prm.Dq);
  __syncthreads();
  double dot = 0.0;
  const int64_t ngroups = (prm.nsel + EPB - 1) / EPB;
  for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x)
    apply_group<T, P, Q, KIND, COLLOC, EPB>(prm, g, sl, dot);
  if (prm.dot_out) {
    double v[1] = {dot};
    __shared__ double tot[1];
    if (fem_grid_sum<1>(v, prm.partials, prm.counter, tot) && threadIdx.x == 0)
      *prm.dot_out = tot[0];
  }
}

}  // namespace fem_apply
