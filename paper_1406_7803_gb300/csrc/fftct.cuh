// fftct.cuh -- compile-time specialised mixed-radix Stockham transforms of many lines held
// in shared memory, executed by a whole CTA.
//
// The length N of a line, its radix sequence (9, 3, 5, then 8, 4, 2 by default) and the
// register budget of a stage are template constants, so every index division and twiddle
// stride folds at compile time.
// A stage works on the flattened set of (line, butterfly) items of a batch of lines: each
// thread loads up to IPT butterflies into registers, the CTA synchronises, the permuted
// outputs are written back, and the CTA synchronises again (in place, one buffer).
// Stage s (radix R, Ns = product of the earlier radices): butterfly j of a line reads
// x_r = a[j + r N/R], multiplies x_r by W_N^{r (j mod Ns) N/(Ns R)}, takes the R-point
// DFT y_q = sum_r x_r W_R^{rq} and writes a'[(j div Ns) Ns R + (j mod Ns) + q Ns] = y_q,
// with W_m = exp(sign 2 pi i / m).
#pragma once

#include <type_traits>

#include "fft.cuh"

namespace fde {

// Placeholder for the optional global-memory input / output of a stage (ct_stage).
struct NoIO {};

struct CtPlan {
  int n, ns;
  int r[8];
};

// Radix order 0: the odd radices (9, 3, 5) first, then 8, 4, 2.  The first stage writes its
// outputs R complex values apart; an odd R spreads a warp's stores over every shared-memory
// bank, where R = 8 put them on 2 (float2) or 4 (double2) banks.  Later stages write runs of
// Ns contiguous values.  Order 1: largest radix first (8, 9, 4, 3, 5, 2).
__host__ __device__ constexpr CtPlan ct_factor(int n, int order = 0) {
  CtPlan p{n, 0, {0, 0, 0, 0, 0, 0, 0, 0}};
  int m = n;
  if (order == 1) {
    while (m % 8 == 0 && p.ns < 8) { p.r[p.ns++] = 8; m /= 8; }
  }
  while (m % 9 == 0 && p.ns < 8) { p.r[p.ns++] = 9; m /= 9; }
  if (order == 1) {
    while (m % 4 == 0 && p.ns < 8) { p.r[p.ns++] = 4; m /= 4; }
  }
  while (m % 3 == 0 && p.ns < 8) { p.r[p.ns++] = 3; m /= 3; }
  while (m % 5 == 0 && p.ns < 8) { p.r[p.ns++] = 5; m /= 5; }
  while (m % 8 == 0 && p.ns < 8) { p.r[p.ns++] = 8; m /= 8; }
  while (m % 4 == 0 && p.ns < 8) { p.r[p.ns++] = 4; m /= 4; }
  while (m % 2 == 0 && p.ns < 8) { p.r[p.ns++] = 2; m /= 2; }
  if (m != 1) p.ns = -1;
  return p;
}

// Variant V of the staged transform: bits 0-3 the register budget (0: 16 complex values per
// thread for FP32 data, 9 for FP64; 1: 18 / 9), bit 4 the radix order of ct_factor, bit 5 the
// thread mapping of unit-stride lines (ct_stage).
__host__ __device__ constexpr int ct_order(int V) { return (V >> 4) & 1; }
__host__ __device__ constexpr bool ct_linefast(int V) { return ((V >> 5) & 1) != 0; }

// The same radices in the opposite order: the plan of a forward transform that starts where an
// inverse transform of plan p ended (its first stage reads the groups p's last stage wrote).
__host__ __device__ constexpr CtPlan ct_reverse(CtPlan p) {
  CtPlan q = p;
  for (int s = 0; s < p.ns; ++s) q.r[s] = p.r[p.ns - 1 - s];
  return q;
}
template <int N, int V, bool REV> __host__ __device__ constexpr CtPlan ct_plan() {
  return REV ? ct_reverse(ct_factor(N, ct_order(V))) : ct_factor(N, ct_order(V));
}

// 8- and 9-point DFTs as 2 x 4 and 3 x 3 Cooley-Tukey in registers.
template <typename C> __device__ __forceinline__ void dft8(C* v, int sign) {
  using T = decltype(v[0].x);
  constexpr T h = T(0.70710678118654752440);  // cos(pi/4)
  C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
  dft4(e, sign);
  dft4(o, sign);
  // o_k *= W_8^k
  C t1 = o[1], t3 = o[3];
  o[1] = cscale(cadd(t1, cmuli(t1, sign)), h);           // (1 + sign i)/sqrt2
  o[2] = cmuli(o[2], sign);                              // sign i
  o[3] = cscale(csub(cmuli(t3, sign), t3), h);           // (-1 + sign i)/sqrt2
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = cadd(e[k], o[k]);
    v[k + 4] = csub(e[k], o[k]);
  }
}

template <typename C> __device__ __forceinline__ void dft9(C* v, int sign) {
  using T = decltype(v[0].x);
  // W_9^1, W_9^2, W_9^4 for sign = -1 (conjugated for sign = +1)
  constexpr T c1 = T(0.76604444311897803520), s1 = T(0.64278760968653932632);   // 2 pi / 9
  constexpr T c2 = T(0.17364817766693034885), s2 = T(0.98480775301220805936);   // 4 pi / 9
  constexpr T c4 = T(-0.93969262078590838405), s4 = T(0.34202014332566873304);  // 8 pi / 9
  C a[3][3];
#pragma unroll
  for (int n2 = 0; n2 < 3; ++n2) {
    a[n2][0] = v[n2];
    a[n2][1] = v[n2 + 3];
    a[n2][2] = v[n2 + 6];
    dft3(a[n2], sign);
  }
  const T sg = (T)sign;
  // a[1][1] *= W^1, a[1][2] *= W^2, a[2][1] *= W^2, a[2][2] *= W^4 with W = exp(sign 2 pi i/9)
  a[1][1] = cmul(a[1][1], mk<T>(c1, sg * s1));
  a[1][2] = cmul(a[1][2], mk<T>(c2, sg * s2));
  a[2][1] = cmul(a[2][1], mk<T>(c2, sg * s2));
  a[2][2] = cmul(a[2][2], mk<T>(c4, sg * s4));
#pragma unroll
  for (int k1 = 0; k1 < 3; ++k1) {
    C b[3] = {a[0][k1], a[1][k1], a[2][k1]};
    dft3(b, sign);
    v[k1] = b[0];
    v[k1 + 3] = b[1];
    v[k1 + 6] = b[2];
  }
}

template <int R, typename C> __device__ __forceinline__ void dft_ct(C* v, int sign) {
  if constexpr (R == 2) dft2(v, sign);
  else if constexpr (R == 3) dft3(v, sign);
  else if constexpr (R == 4) dft4(v, sign);
  else if constexpr (R == 5) dft5(v, sign);
  else if constexpr (R == 8) dft8(v, sign);
  else dft9(v, sign);
}

// Register budget (complex values per thread) of one stage.
template <typename T, int V = 0> __host__ __device__ constexpr int ct_budget() {
  return sizeof(T) == 4 ? ((V & 15) == 1 ? 18 : 16) : 9;
}
template <typename T, int R, int V = 0> __host__ __device__ constexpr int ct_ipt() {
  return ct_budget<T, V>() / R > 0 ? ct_budget<T, V>() / R : 1;
}

template <typename T, int N, int NT, int V = 0, int S = 0>
__host__ __device__ constexpr int ct_lines_per_batch() {
  constexpr CtPlan P = ct_factor(N, ct_order(V));
  if constexpr (S >= P.ns) {
    return 1 << 20;
  } else {
    constexpr int R = P.r[S];
    constexpr int here = NT * ct_ipt<T, R, V>() / (N / R);
    constexpr int rest = ct_lines_per_batch<T, N, NT, V, S + 1>();
    return here < rest ? here : rest;
  }
}

// Line addressing: line l of the batch starts at base(l); elements are es apart.
struct LinesContig {  // line l at l * pitch, unit element stride
  int pitch;
  __device__ __forceinline__ int base(int l) const { return l * pitch; }
  static constexpr bool kUnit = true;
};
struct LinesRows {  // line l at rows[l] * pitch, unit element stride
  const int* rows;
  int pitch;
  __device__ __forceinline__ int base(int l) const { return rows[l] * pitch; }
  static constexpr bool kUnit = true;
};
struct LinesCols {  // line l at l, element stride pitch (columns of a plane)
  int pitch;
  __device__ __forceinline__ int base(int l) const { return l; }
  static constexpr bool kUnit = false;
};

// Thread mapping of the (line, butterfly) items: strided lines (plane columns) and, when
// ct_linefast(V), unit-stride lines too: consecutive threads take the same butterfly of
// neighbouring lines, so a half-warp touches 16 lines one pitch (an odd number of complex
// values) apart -- every bank once, in every stage, for reads and for the stride-R writes of
// the first stages alike.  Unit-stride lines batches may then be partial (l < nl checked).
// Otherwise unit-stride lines are walked by consecutive threads (contiguous reads; the stride-R
// writes of a stage with Ns = 1 conflict 2-way on 16-line planes).
// LD / ST (optional): a stage that reads its inputs through ld(line, element) instead of the
// buffer (the first stage of a transform fed straight from global memory), or hands its outputs
// to st(line, element, value) instead of writing the buffer (the last stage of one whose result
// leaves the CTA).
template <typename T, int N, int R, int NS, int NT, int NL, int V, typename A, typename LD = NoIO,
          typename ST = NoIO>
__device__ __forceinline__ void ct_stage(cplx<T>* buf, const A& addr, int l0, int nl,
                                         const cplx<T>* __restrict__ tw, int sign, const LD& ld = LD(),
                                         const ST& stf = ST()) {
  using C = cplx<T>;
  constexpr int NB = N / R;
  constexpr int TWS = N / (NS * R);
  constexpr int IPT = ct_ipt<T, R, V>();
  constexpr bool LF = !A::kUnit || ct_linefast(V);
  const int es = A::kUnit ? 1 : addr.pitch;
  const int items = (A::kUnit && LF) ? NL * NB : nl * NB;
  C v[IPT][R];
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int w = threadIdx.x + it * NT;
    int l = 0, j = 0;
    if (LF) { j = w / NL; l = w - j * NL; } else { l = w / NB; j = w - l * NB; }
    if (w < items && l < nl) {
      const int k = j % NS;
      const C* a = buf + addr.base(l0 + l);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C x;
        if constexpr (std::is_same<LD, NoIO>::value) x = a[(j + r * NB) * es];
        else x = ld(l0 + l, j + r * NB);
        if (r > 0 && NS > 1) {
          C t = tw[r * k * TWS];
          if (sign > 0) t.y = -t.y;
          x = cmul(x, t);
        }
        v[it][r] = x;
      }
      dft_ct<R>(v[it], sign);
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int w = threadIdx.x + it * NT;
    int l = 0, j = 0;
    if (LF) { j = w / NL; l = w - j * NL; } else { l = w / NB; j = w - l * NB; }
    if (w < items && l < nl) {
      const int k = j % NS;
      const int d = (j / NS) * NS * R + k;
      C* a = buf + addr.base(l0 + l);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        if constexpr (std::is_same<ST, NoIO>::value) a[(d + q * NS) * es] = v[it][q];
        else stf(l0 + l, d + q * NS, v[it][q]);
      }
    }
  }
  __syncthreads();
}

template <typename T, int N, int NT, int NL, int S, int NS, int V, typename A>
__device__ __forceinline__ void ct_stages(cplx<T>* buf, const A& addr, int l0, int nl, const cplx<T>* tw, int sign) {
  constexpr CtPlan P = ct_factor(N, ct_order(V));
  if constexpr (S < P.ns) {
    constexpr int R = P.r[S];
    ct_stage<T, N, R, NS, NT, NL, V>(buf, addr, l0, nl, tw, sign);
    ct_stages<T, N, NT, NL, S + 1, NS * R, V>(buf, addr, l0, nl, tw, sign);
  }
}

// Stages S .. SE - 1 of the plan, reversed radix order when REV; NS = product of the radices
// of the stages before S.
template <typename T, int N, int NT, int NL, int S, int SE, int NS, int V, bool REV, typename A>
__device__ __forceinline__ void ct_stage_range(cplx<T>* buf, const A& addr, int l0, int nl, const cplx<T>* tw,
                                               int sign) {
  constexpr CtPlan P = ct_plan<N, V, REV>();
  if constexpr (S < SE) {
    constexpr int R = P.r[S];
    ct_stage<T, N, R, NS, NT, NL, V>(buf, addr, l0, nl, tw, sign);
    ct_stage_range<T, N, NT, NL, S + 1, SE, NS * R, V, REV>(buf, addr, l0, nl, tw, sign);
  }
}

// Strided lines (plane columns, element stride pitch): the last stage of the inverse transform
// (radix R, Ns = N / R), the product with a real potential and the first stage of the forward
// transform in the reversed radix order (radix R, Ns = 1), on the same registers.  Butterfly j
// ends the inverse holding the outputs j + q N/R, which are exactly the inputs j + r N/R of the
// forward stage's butterfly j; it writes the forward stage's outputs to j R + q.  The potential
// of element i of line l is vp[i * vpitch + l].  Saves one exchange through shared memory and
// the separate multiply pass.
template <typename T, int N, int R, int NT, int NL, int V>
__device__ __forceinline__ void ct_stage_vmul(cplx<T>* buf, int pitch, int l0, int nl,
                                              const cplx<T>* __restrict__ tw, const T* __restrict__ vp,
                                              int vpitch) {
  using C = cplx<T>;
  constexpr int NB = N / R;
  constexpr int IPT = ct_ipt<T, R, V>();
  const int items = nl * NB;
  C v[IPT][R];
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int w = threadIdx.x + it * NT;
    if (w < items) {
      const int j = w / NL, l = w - j * NL;
      const C* a = buf + (l0 + l);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C x = a[(j + r * NB) * pitch];
        if (r > 0 && NB > 1) {
          C t = tw[r * j];  // W_N^{r j} of the last stage, conjugated for the inverse sign
          t.y = -t.y;
          x = cmul(x, t);
        }
        v[it][r] = x;
      }
      dft_ct<R>(v[it], +1);
      const T* vl = vp + (l0 + l);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const T s = vl[(j + q * NB) * vpitch];
        v[it][q].x *= s;
        v[it][q].y *= s;
      }
      dft_ct<R>(v[it], -1);
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int w = threadIdx.x + it * NT;
    if (w < items) {
      const int j = w / NL, l = w - j * NL;
      C* a = buf + (l0 + l);
#pragma unroll
      for (int q = 0; q < R; ++q) a[(j * R + q) * pitch] = v[it][q];
    }
  }
  __syncthreads();
}

// Largest divisor of N not above LB (batch size of strided lines, so every batch is full).
template <int N, int LB> __host__ __device__ constexpr int ct_full_batch() {
  int b = LB < N ? LB : N;
  while (N % b) --b;
  return b;
}

// Transform nlines lines of length N with the whole CTA (NT threads; all must call).
// Strided (column) lines must come N at a time: nlines == N.
template <typename T, int N, int NT, typename A, int V = 0>
__device__ __forceinline__ void ct_lines(cplx<T>* buf, const A& addr, int nlines, const cplx<T>* tw, int sign) {
  static_assert(ct_factor(N, ct_order(V)).ns > 0, "length must factor into 2, 3, 5");
  constexpr int LB0 = ct_lines_per_batch<T, N, NT, V>();
  static_assert(LB0 >= 1, "register budget too small for this length");
  constexpr int LB = A::kUnit ? LB0 : ct_full_batch<N, LB0>();
  for (int l0 = 0; l0 < nlines; l0 += LB) {
    const int nl = nlines - l0 < LB ? nlines - l0 : LB;
    ct_stages<T, N, NT, LB, 0, 1, V>(buf, addr, l0, nl, tw, sign);
  }
}

// Stages S .. ns - 1 with the first stage reading through ld and the last writing through st.
template <typename T, int N, int NT, int NL, int S, int NS, int V, typename A, typename LD, typename ST>
__device__ __forceinline__ void ct_stages_io(cplx<T>* buf, const A& addr, int l0, int nl, const cplx<T>* tw, int sign,
                                             const LD& ld, const ST& st) {
  constexpr CtPlan P = ct_factor(N, ct_order(V));
  if constexpr (S < P.ns) {
    constexpr int R = P.r[S];
    if constexpr (S == 0 && S == P.ns - 1)
      ct_stage<T, N, R, NS, NT, NL, V, A, LD, ST>(buf, addr, l0, nl, tw, sign, ld, st);
    else if constexpr (S == 0)
      ct_stage<T, N, R, NS, NT, NL, V, A, LD, NoIO>(buf, addr, l0, nl, tw, sign, ld, NoIO());
    else if constexpr (S == P.ns - 1)
      ct_stage<T, N, R, NS, NT, NL, V, A, NoIO, ST>(buf, addr, l0, nl, tw, sign, NoIO(), st);
    else
      ct_stage<T, N, R, NS, NT, NL, V, A>(buf, addr, l0, nl, tw, sign);
    ct_stages_io<T, N, NT, NL, S + 1, NS * R, V, A, LD, ST>(buf, addr, l0, nl, tw, sign, ld, st);
  }
}
// ct_lines for unit-stride lines with global-memory input (ld) or output (st) of the transform.
template <typename T, int N, int NT, typename A, int V, typename LD, typename ST>
__device__ __forceinline__ void ct_lines_io(cplx<T>* buf, const A& addr, int nlines, const cplx<T>* tw, int sign,
                                            const LD& ld, const ST& st) {
  static_assert(A::kUnit, "row transforms only");
  constexpr int LB = ct_lines_per_batch<T, N, NT, V>();
  for (int l0 = 0; l0 < nlines; l0 += LB) {
    const int nl = nlines - l0 < LB ? nlines - l0 : LB;
    ct_stages_io<T, N, NT, LB, 0, 1, V, A, LD, ST>(buf, addr, l0, nl, tw, sign, ld, st);
  }
}

// The N columns of an N x N plane (element stride pitch): inverse transform (sign +1), product
// with the potential vp[i * N + l] and forward transform (sign -1), batch by batch, with the
// inverse's last stage and the forward's first fused (ct_stage_vmul).
template <typename T, int N, int NT, int V = 0>
__device__ __forceinline__ void ct_cols_vmul(cplx<T>* buf, int pitch, const cplx<T>* tw, const T* vp) {
  constexpr CtPlan P = ct_factor(N, ct_order(V));
  static_assert(P.ns > 0, "length must factor into 2, 3, 5");
  constexpr int RL = P.r[P.ns - 1];
  constexpr int LB = ct_full_batch<N, ct_lines_per_batch<T, N, NT, V>()>();
  for (int l0 = 0; l0 < N; l0 += LB) {
    ct_stage_range<T, N, NT, LB, 0, P.ns - 1, 1, V, false>(buf, LinesCols{pitch}, l0, LB, tw, +1);
    ct_stage_vmul<T, N, RL, NT, LB, V>(buf, pitch, l0, LB, tw, vp, N);
    ct_stage_range<T, N, NT, LB, 1, P.ns, RL, V, true>(buf, LinesCols{pitch}, l0, LB, tw, -1);
  }
}

}  // namespace fde
