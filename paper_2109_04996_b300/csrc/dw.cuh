// Double-word ("double-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum h + l of two FP32 numbers with |l| small
// against |h|.  Sums use Knuth's TwoSum, products the exact FMA residual of
// h*h (Dekker 1971; the double-word building blocks and their error bounds:
// Joldes, Muller & Popescu, ACM TOMS 44(2), 2017).  The operations here are
// the "sloppy" forms of those building blocks without the final
// renormalization:
//   a + b : (s, e) = TwoSum(a.h, b.h);           (s, e + (a.l + b.l))
//   a * b : p = a.h b.h, e = fma(a.h, b.h, -p) + a.h b.l + a.l b.h;  (p, e)
// Their error is a few u^2 (u = 2^-24) times the magnitudes of the
// operands, i.e. relative to sum |terms| like FP64 summation itself (a
// value whose h cancelled keeps the absolute accuracy of its operands), and
// l stays within a small multiple of u |h| + the operands' l without a
// renormalizing Fast2Sum.  With 48 bits against FP64's 53 this carries an
// FP64-accurate operator apply (relative error of order 1e-14) at FP32
// rates: B300 runs FP32 at 64 times its FP64 rate, and one double-word
// multiply-add costs 12 FP32 instructions.
//
// The __fadd_rn / __fmul_rn / __fmaf_rn intrinsics are never contracted or
// reassociated by the compiler, which the error-free transforms rely on.
#pragma once
#include <cuda_runtime.h>

struct dw {
  float h, l;
  dw() = default;
  __host__ __device__ constexpr dw(float hh, float ll = 0.0f) : h(hh), l(ll) {}
};

// Host: split an FP64 value, h = fl32(d), l = fl32(d - h).
inline dw dw_split_host(double d) {
  const float h = (float)d;
  return dw(h, (float)(d - (double)h));
}

#ifdef __CUDACC__
// s + e = a + b exactly (Knuth's TwoSum, 6 FP32 additions, no ordering
// condition on |a|, |b|).
__device__ __forceinline__ void dw_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// FEM_DW_ADD_ORDERED (set per translation unit before this header): the
// exact error of s = a.h + b.h by Fast2Sum on the operands ordered by
// magnitude (Dekker 1971) instead of TwoSum -- the same e, hence the same
// result bit for bit, from 3 FP32 additions instead of 6 plus a compare and
// two selects on the ALU pipe.  Measured on the headline sweep (5e7 DOFs,
// ms): the line bodies at p = 3..8 faster (5.32 -> 5.18, 4.91 -> 4.57 with
// another launch shape, 4.34 -> 4.30, 4.05 -> 3.95, 4.11 -> 3.99, 5.40 ->
// 5.32), the stencil and the element matrices at p = 1, 2 slower (2.27 ->
// 2.41, 5.03 -> 5.10), and the collocated bodies (BP5) no faster or slower
// (p = 3: 0.36 -> 0.38 ms at 8e6 DOFs), so each translation unit chooses.
#ifndef FEM_DW_ADD_ORDERED
#define FEM_DW_ADD_ORDERED 0
#endif
__device__ __forceinline__ dw operator+(dw a, dw b) {
#if FEM_DW_ADD_ORDERED
  const float s = __fadd_rn(a.h, b.h);
  const bool big = fabsf(a.h) >= fabsf(b.h);
  const float x = big ? a.h : b.h, y = big ? b.h : a.h;
  const float e = __fsub_rn(y, __fsub_rn(s, x));
#else
  float s, e;
  dw_two_sum(a.h, b.h, s, e);
#endif
  return dw(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dw operator-(dw a) { return dw(-a.h, -a.l); }
__device__ __forceinline__ dw operator-(dw a, dw b) { return a + (-b); }

// Product: p = fl(a.h b.h) with its exact residual from the FMA, plus the
// cross terms (a.l b.l is below the double-word precision).
__device__ __forceinline__ dw operator*(dw a, dw b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return dw(p, e);
}
__device__ __forceinline__ dw &operator+=(dw &a, dw b) { return a = a + b; }
__device__ __forceinline__ dw &operator-=(dw &a, dw b) { return a = a - b; }
__device__ __forceinline__ dw &operator*=(dw &a, dw b) { return a = a * b; }
__device__ __forceinline__ dw fma(dw a, dw b, dw c) { return c + a * b; }

// Packed pairs of FP32 values for the f32x2 instructions (two FP32
// operations per issue slot; same FMA rate per clock as scalar FP32 on
// B300): element 0 in the low 32 bits.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(f32x2 v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// TwoSum on both halves: s + e = a + b exactly, element by element.
__device__ __forceinline__ void two_sum2(f32x2 a, f32x2 b, f32x2 &s, f32x2 &e) {
  s = add2(a, b);
  const f32x2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}

// FP64 <-> double word.  The split is exact up to the 48 bits kept:
// h = fl32(d), l = fl32(d - h) (d - h is exact in FP64).  Conversions
// between FP64 and FP32 run at the FP64 rate on B300, so these two serve
// set-up kernels and once-per-thread results; the hot loops use the integer
// forms below.
__device__ __forceinline__ dw dw_from_double(double d) {
  const float h = __double2float_rn(d);
  return dw(h, __double2float_rn(d - (double)h));
}
__device__ __forceinline__ double dw_to_double(dw a) { return (double)a.h + (double)a.l; }

// Split of an FP64 value by integer operations on its bits (no FP64 or
// conversion instruction), rounding to nearest at both steps.  With
// d = s 2^(e-1023) 1.m (52-bit m), low 29 bits of m dropped for h:
//   h = d rounded to 24 significant bits: 2^28 added to the bit pattern
//       (a carry out of the mantissa correctly bumps the exponent), then the
//       float with exponent field e' - 896 and the top 23 mantissa bits;
//   r = d - h in units of 2^(e-1075): the low 29 bits of d sign-extended
//       from bit 28 (exactly the remainder after that rounding), an integer
//       in [-2^28, 2^28);
//   l = RN(r) 2^(e-1075): r split into r_hi 2^14 + r_lo, both converted
//       exactly by the magic-number trick (Hecker, "Let's get to the
//       (floating) point", 1996), one FMA rounds their sum, two exact
//       multiplies scale it (underflowing gracefully).
// |d - (h + l)| <= 2^-49 |d| for 2^-74 <= |d| < 2^128; below 2^-74 the low
// word leaves FP32's range (the error grows to 2^-24 |d| at 2^-126),
// |d| < 2^-126 (zeros included) gives 0 and |d| >= 2^128 saturates to
// infinity.  The double-word bodies share this range: inputs scaled far
// outside it need the FP64-arithmetic bodies.
__device__ __forceinline__ dw dw_from_double_int(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned e = (hi >> 20) & 0x7ffu;
  const unsigned long long br = b + (1ull << 28);
  const unsigned hir = (unsigned)(br >> 32), lor = (unsigned)br;
  // (hi << 3) | (lo >> 29): exponent bits e[8:0] at 31..23, top 23 mantissa
  // bits below; the FP32 exponent field e - 896 = e[7:0] with bit 7 flipped
  const unsigned wr = __funnelshift_l(lor, hir, 3);
  const unsigned hb = ((wr ^ 0x40000000u) & 0x7fffffffu) | (hi & 0x80000000u);
  const int r = ((int)(lo << 3)) >> 3;
  const float f_hi = __fsub_rn(__int_as_float(0x4b400000 + (r >> 14)), 12582912.0f);
  const float f_lo = __fsub_rn(__int_as_float(0x4b000000u | ((unsigned)r & 0x3fffu)), 8388608.0f);
  const float rn = __fmaf_rn(f_hi, 16384.0f, f_lo);
  // 2^(e-1023) with d's sign (from the unrounded pattern), times 2^-52
  const unsigned w = __funnelshift_l(lo, hi, 3);
  const float sc = __fmul_rn(__int_as_float(((w ^ 0x40000000u) & 0x7f800000u) | (hi & 0x80000000u)),
                             2.220446049250313e-16f);
  float h = __int_as_float(hb), l = __fmul_rn(rn, sc);
  if (e < 897u) { h = 0.0f; l = 0.0f; }
  if (e > 1150u) { h = __int_as_float((hi & 0x80000000u) | 0x7f800000u); l = 0.0f; }
  return dw(h, l);
}

// FP32 -> FP64 by integer operations (exact for normal floats; zeros and
// FP32 subnormals give 0).
__device__ __forceinline__ double f32_to_f64_int(float f) {
  const unsigned fb = (unsigned)__float_as_int(f);
  const unsigned hi = (fb & 0x80000000u) | (((fb >> 3) & 0x0fffffffu) + 0x38000000u);
  const unsigned long long b = ((unsigned long long)hi << 32) | (unsigned long long)(fb << 29);
  return (fb & 0x7f800000u) ? __longlong_as_double((long long)b) : 0.0;
}

// h + l rounded to FP64 with one FP64 addition (the conversions of h and l
// are integer operations).
__device__ __forceinline__ double dw_to_double_int(dw a) {
  return __dadd_rn(f32_to_f64_int(a.h), f32_to_f64_int(a.l));
}
#endif
