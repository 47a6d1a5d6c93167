// Line-based element body of the fused diffusion apply, with even-odd
// split 1D operators.
//
// The 1D tables are symmetric under reversal of both indices because the
// Gauss and Gauss-Lobatto points are symmetric about 0:
//   interpolation  B[q-1-k][P-1-a] =  B[k][a]
//   derivative     D[q-1-k][q-1-m] = -D[k][m]
// so a 1D contraction out = M in over a whole line splits into its even and
// odd parts (Solomonoff, J. Comput. Phys. 98, 1992): with
//   ie[a] = in[a] + in[NI-1-a],  io[a] = in[a] - in[NI-1-a]   (a < NI/2)
// every pair (out[k], out[NO-1-k]) costs about NI FMAs instead of 2 NI.
// That saving needs one thread to own a whole line, so here every stage
// assigns lines to threads (rotating the axis from stage to stage) and the
// stages exchange their results through shared-memory cubes:
//   z-interp (registers) -> y-interp -> x-interp -> x/y/z derivatives ->
//   pointwise D -> transposed derivatives (in place) -> transposed x, y, z
//   interpolation -> scatter.
// Collocated Gauss-Lobatto (BP5/BP6) skips the interpolation stages.  The
// split tables are kernel parameters: every lane reads the same entry, which
// the constant bank broadcasts.
#pragma once
#include <cstring>

#include "apply_kernel.cuh"

namespace fem_apply {

// Split table of an NI -> NO contraction M[NO][NI] with reversal symmetry S.
template <typename T, int NI, int NO>
struct SymTab {
  static constexpr int HI = NI / 2, HO = NO / 2;
  T e[HO + 1][HI > 0 ? HI : 1];  // (M[k][a] + M[k][NI-1-a]) / 2
  T o[HO + 1][HI > 0 ? HI : 1];  // (M[k][a] - M[k][NI-1-a]) / 2
  T mid[HO + 1];                 // M[k][NI/2] (NI odd)
};

// Double words: the even and odd tables also as packed pairs for the f32x2
// path of sym_apply: (e.h, o.h), (-e.h, -o.h), (-e.l, -o.l).
template <int NI, int NO>
struct SymTab<dw, NI, NO> {
  static constexpr int HI = NI / 2, HO = NO / 2;
  dw e[HO + 1][HI > 0 ? HI : 1];
  dw o[HO + 1][HI > 0 ? HI : 1];
  dw mid[HO + 1];
  unsigned long long ph[HO > 0 ? HO : 1][HI > 0 ? HI : 1];
  unsigned long long pnh[HO > 0 ? HO : 1][HI > 0 ? HI : 1];
  unsigned long long pnl[HO > 0 ? HO : 1][HI > 0 ? HI : 1];
};

// out = M in over one line.  S = +1: M[NO-1-k][NI-1-a] = M[k][a];
// S = -1: M[NO-1-k][NI-1-a] = -M[k][a].
template <int S, typename T, int NI, int NO>
__device__ __forceinline__ void sym_apply(const SymTab<T, NI, NO> &M, const T (&in)[NI],
                                          T (&out)[NO]) {
  constexpr int HI = NI / 2, HO = NO / 2;
  T ie[HI > 0 ? HI : 1], io[HI > 0 ? HI : 1];
#pragma unroll
  for (int a = 0; a < HI; a++) {
    ie[a] = in[a] + in[NI - 1 - a];
    io[a] = in[a] - in[NI - 1 - a];
  }
#pragma unroll
  for (int k = 0; k < HO; k++) {
    T A = 0, Bv = 0;
#pragma unroll
    for (int a = 0; a < HI; a++) {
      A += M.e[k][a] * ie[a];
      Bv += M.o[k][a] * io[a];
    }
    if constexpr (NI % 2 == 1) A += M.mid[k] * in[HI];
    out[k] = A + Bv;
    out[NO - 1 - k] = (S > 0) ? A - Bv : Bv - A;
  }
  if constexpr (NO % 2 == 1) {
    T v = 0;
    if constexpr (S > 0) {
#pragma unroll
      for (int a = 0; a < HI; a++) v += M.e[HO][a] * ie[a];
      if constexpr (NI % 2 == 1) v += M.mid[HO] * in[HI];
    } else {
#pragma unroll
      for (int a = 0; a < HI; a++) v += M.o[HO][a] * io[a];
    }
    out[HO] = v;
  }
}

// Double words: every output starts from its first product rather than a
// TwoSum with zero (the generic form above spends 6 instructions on that).
template <int S, int NI, int NO>
__device__ __forceinline__ void sym_apply(const SymTab<dw, NI, NO> &M, const dw (&in)[NI],
                                          dw (&out)[NO]) {
  constexpr int HI = NI / 2, HO = NO / 2;
  static_assert(HI > 0, "lines have at least two entries");
  dw ie[HI], io[HI];
#pragma unroll
  for (int a = 0; a < HI; a++) {
    ie[a] = in[a] + in[NI - 1 - a];
    io[a] = in[a] - in[NI - 1 - a];
  }
#pragma unroll
  for (int k = 0; k < HO; k++) {
    dw A = M.e[k][0] * ie[0], Bv = M.o[k][0] * io[0];
#pragma unroll
    for (int a = 1; a < HI; a++) {
      A += M.e[k][a] * ie[a];
      Bv += M.o[k][a] * io[a];
    }
    if constexpr (NI % 2 == 1) A += M.mid[k] * in[HI];
    out[k] = A + Bv;
    out[NO - 1 - k] = (S > 0) ? A - Bv : Bv - A;
  }
  if constexpr (NO % 2 == 1) {
    if constexpr (S > 0) {
      dw v = M.e[HO][0] * ie[0];
#pragma unroll
      for (int a = 1; a < HI; a++) v += M.e[HO][a] * ie[a];
      if constexpr (NI % 2 == 1) v += M.mid[HO] * in[HI];
      out[HO] = v;
    } else {
      dw v = M.o[HO][0] * io[0];
#pragma unroll
      for (int a = 1; a < HI; a++) v += M.o[HO][a] * io[a];
      out[HO] = v;
    }
  }
}

// Double words: the even and odd accumulations of an output pair run the
// same double-word instruction sequence, so they are carried as f32x2 pairs
// (A, B): each packed instruction does the step for both, halving the
// issue slots of the contraction.  The pair's value is h - nl (the low
// words kept negated, so that the FMA-exact product error needs no
// negation: with the negated tables, fma(-m.h, x.h, p) = -(m.h x.h - p)).
// Per term: p = m.h x.h; ne = -(exact error of p) - m.h x.l - m.l x.h (three
// FMAs); (h, e) = TwoSum(h, p); nl = nl + ne - e.  The first term starts
// the pair (h, nl) = (p, ne).  The pre-sums ie = x + y, io = x - y are one
// packed double-word sum of (x, x) and (y, -y).
template <int S, int NI, int NO>
__device__ __forceinline__ void sym_apply_packed(const SymTab<dw, NI, NO> &M, const dw (&in)[NI],
                                                 dw (&out)[NO]) {
  constexpr int HI = NI / 2, HO = NO / 2;
  static_assert(HI > 0, "lines have at least two entries");
  f32x2 xh[HI], xl[HI];   // (ie, io) high and low words
#pragma unroll
  for (int a = 0; a < HI; a++) {
    const dw x = in[a], y = in[NI - 1 - a];
    f32x2 s, e;
    two_sum2(pk2(x.h, x.h), pk2(y.h, -y.h), s, e);
    xh[a] = s;
    xl[a] = add2(e, add2(pk2(x.l, x.l), pk2(y.l, -y.l)));
  }
#pragma unroll
  for (int k = 0; k < HO; k++) {
    f32x2 h = 0ull, nl = 0ull;
#pragma unroll
    for (int a = 0; a < HI; a++) {
      const f32x2 mh = M.ph[k][a], nmh = M.pnh[k][a], nml = M.pnl[k][a];
      const f32x2 p = mul2(mh, xh[a]);
      f32x2 ne = fma2(nmh, xh[a], p);
      ne = fma2(nmh, xl[a], ne);
      ne = fma2(nml, xh[a], ne);
      if (a == 0) {
        h = p;
        nl = ne;
      } else {
        f32x2 s, e;
        two_sum2(h, p, s, e);
        h = s;
        nl = sub2(add2(nl, ne), e);
      }
    }
    float Ah, Bh, Anl, Bnl;
    upk2(h, Ah, Bh);
    upk2(nl, Anl, Bnl);
    dw A(Ah, -Anl), Bv(Bh, -Bnl);
    if constexpr (NI % 2 == 1) A += M.mid[k] * in[HI];
    out[k] = A + Bv;
    out[NO - 1 - k] = (S > 0) ? A - Bv : Bv - A;
  }
  if constexpr (NO % 2 == 1) {
    // the middle output: one chain, scalar double words
    float xeh[HI], xoh[HI], xel[HI], xol[HI];
#pragma unroll
    for (int a = 0; a < HI; a++) {
      upk2(xh[a], xeh[a], xoh[a]);
      upk2(xl[a], xel[a], xol[a]);
    }
    if constexpr (S > 0) {
      dw v = M.e[HO][0] * dw(xeh[0], xel[0]);
#pragma unroll
      for (int a = 1; a < HI; a++) v += M.e[HO][a] * dw(xeh[a], xel[a]);
      if constexpr (NI % 2 == 1) v += M.mid[HO] * in[HI];
      out[HO] = v;
    } else {
      dw v = M.o[HO][0] * dw(xoh[0], xol[0]);
#pragma unroll
      for (int a = 1; a < HI; a++) v += M.o[HO][a] * dw(xoh[a], xol[a]);
      out[HO] = v;
    }
  }
}

// The line body's contractions: PK selects the packed form (double words).
template <int S, bool PK, typename T, int NI, int NO>
__device__ __forceinline__ void sym(const SymTab<T, NI, NO> &M, const T (&in)[NI], T (&out)[NO]) {
  if constexpr (PK) sym_apply_packed<S>(M, in, out);
  else sym_apply<S>(M, in, out);
}

template <typename T, int P, int Q>
struct LineTables {
  static constexpr int kP = P, kQ = Q;
  SymTab<T, P, Q> Bf;  // interpolation, nodes -> quadrature points
  SymTab<T, Q, P> Bt;  // its transpose
  SymTab<T, Q, Q> Df;  // collocated derivative
  SymTab<T, Q, Q> Dt;  // its transpose
};

template <typename T, int P, int Q>
struct LineParams {
  ApplyParams<T> a;
  LineTables<T, P, Q> t;
};

// Host: a table entry in arithmetic type T (double words split the FP64
// value, h = fl32(v), l = fl32(v - h)).
template <typename T>
inline T tab_value(double v) {
  if constexpr (std::is_same<T, dw>::value) return dw_split_host(v);
  else return (T)v;
}

// Host: split a row-major M[NO][NI] (FP64) into the table.
template <typename T, int NI, int NO>
inline void make_symtab(const double *M, SymTab<T, NI, NO> &s) {
  constexpr int HI = NI / 2, HO = NO / 2;
  for (int k = 0; k <= HO && k < NO; k++) {
    for (int a = 0; a < (HI > 0 ? HI : 1); a++) {
      if (a < HI) {
        s.e[k][a] = tab_value<T>(0.5 * (M[k * NI + a] + M[k * NI + NI - 1 - a]));
        s.o[k][a] = tab_value<T>(0.5 * (M[k * NI + a] - M[k * NI + NI - 1 - a]));
      } else {
        s.e[k][a] = tab_value<T>(0.0);
        s.o[k][a] = tab_value<T>(0.0);
      }
    }
    s.mid[k] = tab_value<T>((NI % 2 == 1) ? M[k * NI + HI] : 0.0);
  }
  if constexpr (std::is_same<T, dw>::value) {
    auto bits = [](float f) -> unsigned long long {
      unsigned u;
      memcpy(&u, &f, 4);
      return u;
    };
    auto pack = [&](float lo, float hi) { return bits(lo) | (bits(hi) << 32); };
    for (int k = 0; k < HO; k++)
      for (int a = 0; a < (HI > 0 ? HI : 1); a++) {
        s.ph[k][a] = pack(s.e[k][a].h, s.o[k][a].h);
        s.pnh[k][a] = pack(-s.e[k][a].h, -s.o[k][a].h);
        s.pnl[k][a] = pack(-s.e[k][a].l, -s.o[k][a].l);
      }
  }
}

// One cube of q^3 values in shared memory, x-contiguous: entry (k, j, i) at
// i + sj j + sk k, cubes `size` words apart.  The stages read and write
// whole lines along x, y and z with the warp's threads spread over the other
// two directions (and over the elements of the group), so the strides decide
// how many of a warp's accesses share a bank.  Plain layout: sj = q, sk =
// q^2.  For q a multiple of 4 the pitch is q + 1 (a pitch of 4 or 8 words
// puts 4 or 8 of an x-line stage's threads on one bank; BP5/BP6 p=7 +3-15 %).
// FP32 at q = 4 and q = 10 uses the strides that minimize the words per bank
// over every access instruction of both element bodies and the three
// elements-per-block choices (counted on the host), measured faster at 8e6
// DOFs: BP3 p=2 651 -> 515 us, BP5 p=3 185 -> 171 us, BP1 p=2 280 -> 242
// us, BP3 p=8 226 -> 203 us.  (The same count favoured odd k-strides at q =
// 5, 6, 7, 8, which measured 1-22 % slower: even strides let the compiler
// pair the x-line accesses into 8-byte shared loads.)  PAD = false keeps
// the plain layout (the batched kernel, which holds every order in one
// kernel and is register-bound).
template <int Q, bool PAD = true, int TSZ = 4>
struct LineCube {
  static constexpr bool tuned = PAD && TSZ == 4 && (Q == 4 || Q == 10);
  static constexpr bool pitch1 = PAD && !tuned && Q % 4 == 0;
  static constexpr int sj = tuned ? Q : (pitch1 ? Q + 1 : Q);
  static constexpr int sk = tuned ? (Q == 4 ? 19 : 105) : Q * sj;
  static constexpr int size = tuned ? (Q == 4 ? 76 : 1049) : Q * Q * sj;
  static_assert(size >= (Q - 1) * (1 + sj + sk) + 1, "cube entries must fit");
};

// Index of cube entry (k, j, i).  (A function, not a lambda: with a lambda
// here the batched kernel, which inlines every order, took 119 registers
// instead of 72.)
template <int SJ, int SK>
__device__ __forceinline__ int cube_ix(int k, int j, int i) {
  return i + SJ * j + SK * k;
}

// Shared memory: 4 cubes per element slot.
template <typename T, int Q, int EPB, bool PAD = true>
constexpr size_t lines_smem_bytes() {
  return sizeof(T) * (size_t)EPB * 4 * LineCube<Q, PAD, (int)sizeof(T)>::size;
}

// One thread's z-column of an element: its P node ids and gathered values.
// The pipelined loop carries the next group's column across iterations so
// that its loads overlap the current group's stages.
template <typename T, int P>
struct Column {
  int32_t idx[P];
  T u[P];
  int32_t idx0;   // the element's local node 0 (shifted double-word bodies)
};

// Column of element group g for the calling thread (a P x P line set
// thread); zeros where the element does not exist.
template <typename T, int P, int Q, int EPB>
__device__ __forceinline__ void column_indices(const ApplyParams<T> &prm, int64_t g, Column<T, P> &col) {
  constexpr int Q2 = Q * Q, P2 = P * P, P3 = P * P * P;
  const int slot_raw = threadIdx.x / Q2, t = threadIdx.x - slot_raw * Q2;
  const int64_t k_el = g * EPB + slot_raw;
  const bool ok = slot_raw < EPB && t < P2 && k_el < prm.nsel;
  const int32_t *en = prm.elem_nodes + (ok ? k_el : 0) * P3 + (t % P) + P * (t / P);
#pragma unroll
  for (int k = 0; k < P; k++) col.idx[k] = ok ? en[P2 * k] : -1;
  col.idx0 = ok ? prm.elem_nodes[k_el * P3] : -1;
}

// SH: values shifted by x at the element's node 0 (ShiftX).
template <typename T, int P, bool SH = false>
__device__ __forceinline__ void column_values(const ApplyParams<T> &prm, Column<T, P> &col) {
  const double c0 = (SH && col.idx0 >= 0) ? (double)gather_load(&prm.x[col.idx0], prm.x_l2_only) : 0.0;
#pragma unroll
  for (int k = 0; k < P; k++)
    col.u[k] = col.idx[k] >= 0 ? gather_shifted<T, SH>(&prm.x[col.idx[k]], prm.x_l2_only, c0) : T(0);
}

// PIPE (scalar operator, contiguous elements): the column of this group is
// given in `cur` (ids and values loaded by the previous iteration) and the
// next group's (g + gridDim.x) is loaded into `nxt`: its ids at the start,
// its values after the gradient stage.
// KIND: FEM_DIFFUSION (gradients, 6 qdata per point) or FEM_MASS (values,
// 1 qdata per point: the interpolation stages only; not collocated).
// PF (contiguous elements): thread 0 starts an L2 bulk prefetch of the
// next group's qdata (and of its element node ids, two groups ahead when
// PIPE loads the next group's ids here), so that the pointwise stage's
// qdata loads hit L2.
template <typename T, int P, int Q, bool COLLOC, int EPB, bool PIPE = false, bool PAD = true,
          int KIND = FEM_DIFFUSION, bool PK = false, bool PF = false>
__device__ __forceinline__ void apply_group_lines(const ApplyParams<T> &prm,
                                                  const LineTables<T, P, Q> &tb, int64_t g,
                                                  T *cubes, double &dot,
                                                  const Column<T, P> *cur = nullptr,
                                                  Column<T, P> *nxt = nullptr) {
  constexpr bool DIFF = KIND == FEM_DIFFUSION;
  constexpr bool SH = ShiftX<T, KIND>::value;
  static_assert(DIFF || !COLLOC, "the collocated mass operator is pointwise: slab body");
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q, P2 = P * P, P3 = P * P * P;
  using Cube = LineCube<Q, PAD, (int)sizeof(T)>;
  constexpr int CS = Cube::size, SJ = Cube::sj, SK = Cube::sk;
  const int slot_raw = threadIdx.x / Q2;
  const bool live = slot_raw < EPB;
  const int slot = live ? slot_raw : EPB - 1;
  const int t = threadIdx.x - slot_raw * Q2;   // thread within the element
  T *c1 = cubes + (size_t)slot * 4 * CS, *c2 = c1 + CS, *c3 = c2 + CS, *c4 = c3 + CS;
  const int64_t N = prm.N;
  const int64_t k_el = g * EPB + slot_raw;
  const bool valid = live && (k_el < prm.nsel);
  int64_t e = 0;
  if (valid) e = prm.list ? (int64_t)prm.list[k_el] : k_el;
  const int32_t *en = prm.elem_nodes + e * P3;
  const auto *qd = prm.qdata + e * (int64_t)((DIFF ? 6 : 1) * Q3);
  // line coordinates of this thread: (t % Q, t / Q) for q-by-q line sets,
  // (t % P, t / P) for P-by-q, (t % P, t / P) for P-by-P
  const int lq0 = t % Q, lq1 = t / Q;
  const int lp0 = t % P, lp1 = t / P;
  const bool on_qq = live;                  // t < Q^2 always
  const bool on_pq = live && t < P * Q;
  const bool on_pp = live && t < P2;
  // this thread's share of x.y over the group (see DotAcc), added to the
  // FP64 `dot` once
  DotAcc<T> dl;
  if constexpr (PF) {
    if (threadIdx.x == 0 && !prm.list) {
      constexpr int NQD = DIFF ? 6 : 1;
      const int64_t eq = (g + gridDim.x) * EPB, ei = (g + (PIPE ? 2 : 1) * (int64_t)gridDim.x) * EPB;
      if (eq < prm.nsel) {
        const int64_t ne = prm.nsel - eq < EPB ? prm.nsel - eq : EPB;
        prefetch_l2(prm.qdata + eq * NQD * Q3, (size_t)ne * NQD * Q3 * sizeof(*prm.qdata));
      }
      if (ei < prm.nsel) {
        const int64_t ne = prm.nsel - ei < EPB ? prm.nsel - ei : EPB;
        prefetch_l2(prm.elem_nodes + ei * P3, (size_t)ne * P3 * sizeof(int32_t));
      }
    }
  }
  if constexpr (PIPE) column_indices<T, P, Q, EPB>(prm, g + gridDim.x, *nxt);
  for (int c = 0; c < prm.ncomp; c++) {
    const auto *xc = prm.x + c * N;
    auto *yc = prm.y + c * N;
    // ---- gather the z-column (a, b) = (lp0, lp1) of the element
    T u[P];
    if constexpr (PIPE) {
#pragma unroll
      for (int k = 0; k < P; k++) u[k] = cur->u[k];
    } else {
      const double c0 = (SH && valid) ? (double)gather_load(&xc[en[0]], prm.x_l2_only) : 0.0;
#pragma unroll
      for (int k = 0; k < P; k++)
        u[k] = (valid && on_pp) ? gather_shifted<T, SH>(&xc[en[lp0 + P * lp1 + P2 * k]], prm.x_l2_only, c0)
                                : T(0);
    }
    // c3 holds the values at the quadrature points, x-contiguous [k][j][i]
    if constexpr (COLLOC) {
      if (on_pp) {
#pragma unroll
        for (int k = 0; k < Q; k++) c3[cube_ix<SJ, SK>(k, lp1, lp0)] = u[k];
      }
    } else {
      // z-interpolation of the column (a, b)
      if (on_pp) {
        T w[Q];
        sym<+1, PK>(tb.Bf, u, w);
#pragma unroll
        for (int k = 0; k < Q; k++) c1[cube_ix<SJ, SK>(k, lp1, lp0)] = w[k];
      }
      __syncthreads();
      // y-lines (a, kq): c1[kq][0..P)[a] -> c2[kq][0..Q)[a]
      if (on_pq) {
        T in[P], out[Q];
#pragma unroll
        for (int j = 0; j < P; j++) in[j] = c1[cube_ix<SJ, SK>(lp1, j, lp0)];
        sym<+1, PK>(tb.Bf, in, out);
#pragma unroll
        for (int j = 0; j < Q; j++) c2[cube_ix<SJ, SK>(lp1, j, lp0)] = out[j];
      }
      __syncthreads();
      // x-lines (jq, kq): c2[kq][jq][0..P) -> c3[kq][jq][0..Q)
      if (on_qq) {
        T in[P], out[Q];
#pragma unroll
        for (int i = 0; i < P; i++) in[i] = c2[cube_ix<SJ, SK>(lq1, lq0, i)];
        sym<+1, PK>(tb.Bf, in, out);
#pragma unroll
        for (int i = 0; i < Q; i++) c3[cube_ix<SJ, SK>(lq1, lq0, i)] = out[i];
      }
    }
    __syncthreads();
    if constexpr (!DIFF) {
      if constexpr (PIPE) column_values<T, P, SH>(prm, *nxt);
      // ---- mass: values at the quadrature points times w detJ, in place
      if (on_qq) {
#pragma unroll
        for (int kq = 0; kq < Q; kq++) {
          const int pt = cube_ix<SJ, SK>(kq, lq1, lq0);
          const T w = valid ? ld_qdata<T>(qd + (kq * Q + lq1) * Q + lq0) : T(0);
          c3[pt] *= w;
        }
      }
      __syncthreads();
    } else {
    // ---- reference gradients: x into c1, y into c2, z into c4
    if (on_qq) {
      T in[Q], out[Q];
      // x-line (jq, kq) = (lq0, lq1)
#pragma unroll
      for (int m = 0; m < Q; m++) in[m] = c3[cube_ix<SJ, SK>(lq1, lq0, m)];
      sym<-1, PK>(tb.Df, in, out);
#pragma unroll
      for (int m = 0; m < Q; m++) c1[cube_ix<SJ, SK>(lq1, lq0, m)] = out[m];
      // y-line (iq, kq) = (lq0, lq1)
#pragma unroll
      for (int m = 0; m < Q; m++) in[m] = c3[cube_ix<SJ, SK>(lq1, m, lq0)];
      sym<-1, PK>(tb.Df, in, out);
#pragma unroll
      for (int m = 0; m < Q; m++) c2[cube_ix<SJ, SK>(lq1, m, lq0)] = out[m];
      // z-line (iq, jq) = (lq0, lq1)
#pragma unroll
      for (int m = 0; m < Q; m++) in[m] = c3[cube_ix<SJ, SK>(m, lq1, lq0)];
      sym<-1, PK>(tb.Df, in, out);
#pragma unroll
      for (int m = 0; m < Q; m++) c4[cube_ix<SJ, SK>(m, lq1, lq0)] = out[m];
    }
    __syncthreads();
    if constexpr (PIPE) column_values<T, P, SH>(prm, *nxt);
    // ---- pointwise D at the column (iq, jq) = (lq0, lq1), in place
    if (on_qq) {
#pragma unroll
      for (int kq = 0; kq < Q; kq++) {
        const int pt = cube_ix<SJ, SK>(kq, lq1, lq0);
        T G00 = 0, G11 = 0, G22 = 0, G12 = 0, G02 = 0, G01 = 0;
        if (valid) {
          // qdata is unpadded: the cube index unless the cube is padded
          const auto *qk = qd + ((SJ == Q && SK == Q * Q) ? pt : (kq * Q + lq1) * Q + lq0);
          G00 = ld_qdata<T>(qk); G11 = ld_qdata<T>(qk + Q3); G22 = ld_qdata<T>(qk + 2 * Q3);
          G12 = ld_qdata<T>(qk + 3 * Q3); G02 = ld_qdata<T>(qk + 4 * Q3); G01 = ld_qdata<T>(qk + 5 * Q3);
        }
        const T gx = c1[pt], gy = c2[pt], gz = c4[pt];
        c1[pt] = G00 * gx + G01 * gy + G02 * gz;
        c2[pt] = G01 * gx + G11 * gy + G12 * gz;
        c4[pt] = G02 * gx + G12 * gy + G22 * gz;
      }
    }
    __syncthreads();
    // ---- transposed derivatives, each line in place (disjoint cubes)
    if (on_qq) {
      T in[Q], out[Q];
#pragma unroll
      for (int m = 0; m < Q; m++) in[m] = c1[cube_ix<SJ, SK>(lq1, lq0, m)];
      sym<-1, PK>(tb.Dt, in, out);
#pragma unroll
      for (int m = 0; m < Q; m++) c1[cube_ix<SJ, SK>(lq1, lq0, m)] = out[m];
#pragma unroll
      for (int m = 0; m < Q; m++) in[m] = c2[cube_ix<SJ, SK>(lq1, m, lq0)];
      sym<-1, PK>(tb.Dt, in, out);
#pragma unroll
      for (int m = 0; m < Q; m++) c2[cube_ix<SJ, SK>(lq1, m, lq0)] = out[m];
#pragma unroll
      for (int m = 0; m < Q; m++) in[m] = c4[cube_ix<SJ, SK>(m, lq1, lq0)];
      sym<-1, PK>(tb.Dt, in, out);
#pragma unroll
      for (int m = 0; m < Q; m++) c4[cube_ix<SJ, SK>(m, lq1, lq0)] = out[m];
    }
    __syncthreads();
    }  // DIFF
    if constexpr (COLLOC) {
      // sum of the three contributions at the node column (a, b), scatter
      if (on_pp) {
#pragma unroll
        for (int k = 0; k < P; k++) {
          const int pt = cube_ix<SJ, SK>(k, lp1, lp0);
          const T s = c1[pt] + c2[pt] + c4[pt];
          if (valid) {
            const int64_t gi = PIPE ? cur->idx[k] : en[lp0 + P * lp1 + P2 * k];
            atomic_add(&yc[gi], s);
            dl.add(s, u[k]);
          }
        }
      }
      // the next component's first writes (c3) and the next gradients
      // (c1, c2, c4) must not pass these reads
      __syncthreads();
    } else {
      // x-lines (jq, kq): sum of the three, transposed interpolation -> c3[kq][jq][0..P)
      if (on_qq) {
        T in[Q], out[P];
#pragma unroll
        for (int m = 0; m < Q; m++) {
          const int pt = cube_ix<SJ, SK>(lq1, lq0, m);
          in[m] = DIFF ? c1[pt] + c2[pt] + c4[pt] : c3[pt];
        }
        sym<+1, PK>(tb.Bt, in, out);
#pragma unroll
        for (int i = 0; i < P; i++) c3[cube_ix<SJ, SK>(lq1, lq0, i)] = out[i];
      }
      __syncthreads();
      // y-lines (a, kq): c3[kq][0..Q)[a] -> c1[kq][0..P)[a]
      if (on_pq) {
        T in[Q], out[P];
#pragma unroll
        for (int j = 0; j < Q; j++) in[j] = c3[cube_ix<SJ, SK>(lp1, j, lp0)];
        sym<+1, PK>(tb.Bt, in, out);
#pragma unroll
        for (int j = 0; j < P; j++) c1[cube_ix<SJ, SK>(lp1, j, lp0)] = out[j];
      }
      __syncthreads();
      // z-lines (a, b): c1[0..Q)[b][a] -> nodes, scatter
      if (on_pp) {
        T in[Q], out[P];
#pragma unroll
        for (int k = 0; k < Q; k++) in[k] = c1[cube_ix<SJ, SK>(k, lp1, lp0)];
        sym<+1, PK>(tb.Bt, in, out);
#pragma unroll
        for (int k = 0; k < P; k++) {
          if (valid) {
            const int64_t gi = PIPE ? cur->idx[k] : en[lp0 + P * lp1 + P2 * k];
            atomic_add(&yc[gi], out[k]);
            dl.add(out[k], u[k]);
          }
        }
      }
      // c1 is the next component's first target
      __syncthreads();
    }
  }
  if (prm.dot_out || prm.want_dot) dot += dl.get();
}

// PIPE: the group loop carries each group's column gather one group ahead
// (scalar operators over contiguous elements; the launcher picks it for FP32,
// whose time is load latency); a separate instantiation, so that the others
// keep their lower register count.
// The kernel body, shared by the two entry points below.
template <typename T, int P, int Q, bool COLLOC, int EPB, bool PIPE, int KIND, bool PK, bool PF>
__device__ __forceinline__ void lines_kernel_body(const LineParams<T, P, Q> &lp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *cubes = reinterpret_cast<T *>(smem_raw);
  const ApplyParams<T> &prm = lp.a;
  if (apply_skipped(prm)) return;
  double dot = 0.0;
  const int64_t ngroups = (prm.nsel + EPB - 1) / EPB;
  if constexpr (PIPE) {
    Column<T, P> cur, nxt;
    column_indices<T, P, Q, EPB>(prm, blockIdx.x, cur);
    column_values<T, P, ShiftX<T, KIND>::value>(prm, cur);
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
      apply_group_lines<T, P, Q, COLLOC, EPB, true, true, KIND, PK, PF>(prm, lp.t, g, cubes, dot, &cur, &nxt);
      cur = nxt;
    }
  } else {
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x)
      apply_group_lines<T, P, Q, COLLOC, EPB, false, true, KIND, PK, PF>(prm, lp.t, g, cubes, dot);
  }
  if (prm.dot_out) {
    double v[1] = {dot};
    __shared__ double tot[1];
    if (fem_grid_sum<1>(v, prm.partials, prm.counter, tot) && threadIdx.x == 0)
      *prm.dot_out = tot[0];
  }
}

template <typename T, int P, int Q, bool COLLOC, int EPB, bool PIPE, int KIND, bool PK = false,
          bool PF = false>
__global__ void __launch_bounds__(ApplyShape<Q, EPB>::NT)
    fem_apply_lines_kernel(const LineParams<T, P, Q> lp) {
  lines_kernel_body<T, P, Q, COLLOC, EPB, PIPE, KIND, PK, PF>(lp);
}

// The same body held to MINB blocks per SM (LinesMinBlocks; 0: the
// unbounded entry point above), for the shapes where that measured faster
// (5e7 DOFs, the best bounded against the best unbounded shape):
//   q = 10 (p = 8, Gauss), at most two elements per block: three blocks,
//     80 registers, some spilled; BP3 p = 8 6.21 -> 5.39 ms (BP1 p = 8 at
//     8e6: 0.50 -> 0.44 ms);
//   double-word diffusion with the pipelined gather, packed contractions and
//   the L2 prefetch at q = 7 (5 elements per block) and q = 8 (4): two
//     blocks; BP3 p = 5 4.44 -> 4.33 ms, p = 6 4.19 -> 4.04 ms, BP5 p = 7
//     (q = 8, collocated) 1.26 -> 1.19 ms;
//   the pipelined gather alone at q = 9 (3 elements per block): two blocks;
//     BP3 p = 7 4.15 -> 4.10 ms (BP5 p = 8 at 8e6: 0.40 -> 0.36 ms).
// The other shapes lost 10-60 % under the same bounds, and so did q = 9
// held to three blocks (4.16 -> 4.40 ms) and four elements per block at
// q = 10 held to two; a minimum of one block, which the entry point above
// leaves out, changes the register allocation of every shape: p = 3..7
// 25-50 % slower.
template <typename T, int Q, int EPB, bool PIPE = false, int KIND = FEM_DIFFUSION, bool PK = false,
          bool PF = false>
struct LinesMinBlocks {
  static constexpr bool DW = std::is_same<T, dw>::value, DIFF = KIND == FEM_DIFFUSION;
  static constexpr int value =
      !DW ? 0
      : (Q == 10 && EPB <= 2) ? 3
      : (DIFF && PIPE && PK && PF && ((Q == 7 && EPB == 5) || (Q == 8 && EPB == 4))) ? 2
      : (DIFF && PIPE && !PK && !PF && Q == 9 && EPB == 3) ? 2
      : 0;
};

template <int MINB, typename T, int P, int Q, bool COLLOC, int EPB, bool PIPE, int KIND, bool PK = false,
          bool PF = false>
__global__ void __launch_bounds__(ApplyShape<Q, EPB>::NT, MINB)
    fem_apply_lines_kernel_mb(const LineParams<T, P, Q> lp) {
  lines_kernel_body<T, P, Q, COLLOC, EPB, PIPE, KIND, PK, PF>(lp);
}

}  // namespace fem_apply
