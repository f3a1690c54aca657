// fft.cuh -- mixed-radix (2, 3, 4, 5) Stockham transforms of lines held in shared memory.
//
// One warp transforms one line in place: every stage loads its butterflies into
// registers, synchronises the warp, writes the permuted outputs and synchronises again,
// so no second buffer is needed.  A line is n complex values at shared-memory element
// stride `es` (1 for contiguous lines, the padded row pitch for strided ones).
//
// Stage s with radix R and Ns = product of the earlier radices: butterfly j in [0, n/R)
// with k = j mod Ns reads x_r = a[j + r n/R], multiplies x_r by W_n^{r k n/(Ns R)},
// takes the R-point DFT y_q = sum_r x_r W_R^{r q}, and writes
// a'[(j div Ns) Ns R + k + q Ns] = y_q.  W_m = exp(sign 2 pi i / m); sign = -1 for the
// forward transform f(G) ~ sum_r f(r) e^{-iG.r} and +1 for the inverse (unnormalised).
#pragma once

#include "common.cuh"

namespace fde {

// R-point DFTs in registers; constants are exact trigonometric values.
template <typename C> __device__ __forceinline__ void dft2(C* v, int) {
  C a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

// Constants are constexpr so that every arithmetic type (float, double, double-float) gets them
// folded at compile time.
template <typename C> __device__ __forceinline__ void dft3(C* v, int sign) {
  using T = decltype(v[0].x);
  constexpr T h = T(0.86602540378443864676);  // sin(2 pi / 3)
  constexpr T half = T(0.5);
  C t1 = cadd(v[1], v[2]);
  C t2 = cmuli(cscale(csub(v[1], v[2]), h), sign);
  C m = csub(v[0], cscale(t1, half));
  v[0] = cadd(v[0], t1);
  v[1] = cadd(m, t2);
  v[2] = csub(m, t2);
}

template <typename C> __device__ __forceinline__ void dft4(C* v, int sign) {
  C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
  C c = cadd(v[1], v[3]), d = cmuli(csub(v[1], v[3]), sign);
  v[0] = cadd(a, c);
  v[2] = csub(a, c);
  v[1] = cadd(b, d);
  v[3] = csub(b, d);
}

template <typename C> __device__ __forceinline__ void dft5(C* v, int sign) {
  using T = decltype(v[0].x);
  constexpr T c1 = T(0.30901699437494742410);   // cos(2 pi / 5)
  constexpr T c2 = T(-0.80901699437494742410);  // cos(4 pi / 5)
  constexpr T s1 = T(0.95105651629515357212);   // sin(2 pi / 5)
  constexpr T s2 = T(0.58778525229247312917);   // sin(4 pi / 5)
  C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  C t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  C a1 = cadd(v[0], cadd(cscale(t1, c1), cscale(t2, c2)));
  C a2 = cadd(v[0], cadd(cscale(t1, c2), cscale(t2, c1)));
  C b1 = cmuli(cadd(cscale(t3, s1), cscale(t4, s2)), sign);
  C b2 = cmuli(csub(cscale(t3, s2), cscale(t4, s1)), sign);
  v[0] = cadd(v[0], cadd(t1, t2));
  v[1] = cadd(a1, b1);
  v[4] = csub(a1, b1);
  v[2] = cadd(a2, b2);
  v[3] = csub(a2, b2);
}

template <int R, typename C> __device__ __forceinline__ void dftR(C* v, int sign) {
  if (R == 2) dft2(v, sign);
  else if (R == 3) dft3(v, sign);
  else if (R == 4) dft4(v, sign);
  else dft5(v, sign);
}

template <typename T, int R, int NMAX>
__device__ __forceinline__ void stage(cplx<T>* a, int es, int n, int Ns, const cplx<T>* __restrict__ tw,
                                      int lane, int sign) {
  using C = cplx<T>;
  constexpr int MAXB = (NMAX / R + 31) / 32;
  const int nb = n / R;
  const int tws = n / (Ns * R);
  C v[MAXB][R];
#pragma unroll
  for (int b = 0; b < MAXB; ++b) {
    const int j = lane + 32 * b;
    if (j < nb) {
      const int k = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C x = a[(j + r * nb) * es];
        if (r > 0 && k > 0) {
          C w = tw[r * k * tws];
          if (sign > 0) w.y = -w.y;
          x = cmul(x, w);
        }
        v[b][r] = x;
      }
      dftR<R>(v[b], sign);
    }
  }
  __syncwarp();
#pragma unroll
  for (int b = 0; b < MAXB; ++b) {
    const int j = lane + 32 * b;
    if (j < nb) {
      const int k = j % Ns;
      const int d = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) a[(d + r * Ns) * es] = v[b][r];
    }
  }
  __syncwarp();
}

// Transform one line with the calling warp (all 32 lanes must call).
template <typename T, int NMAX = kMaxLine>
__device__ __forceinline__ void fft_line(cplx<T>* a, int es, const LinePlan<T>& p, int lane, int sign) {
  int Ns = 1;
  for (int s = 0; s < p.nstages; ++s) {
    const int R = p.radix[s];
    if (R == 4) stage<T, 4, NMAX>(a, es, p.n, Ns, p.tw, lane, sign);
    else if (R == 2) stage<T, 2, NMAX>(a, es, p.n, Ns, p.tw, lane, sign);
    else if (R == 3) stage<T, 3, NMAX>(a, es, p.n, Ns, p.tw, lane, sign);
    else stage<T, 5, NMAX>(a, es, p.n, Ns, p.tw, lane, sign);
    Ns *= R;
  }
}

}  // namespace fde
