// fft_dd.cu -- full-grid 3D transforms of FP64 grids in double-float arithmetic (dd.cuh).
//
// The same staged mixed-radix transforms as the FP64 axis passes (fftct.cuh), instantiated on
// the double-float type: each value is two floats, so the arithmetic runs on the FP32 pipes
// (64x the FP64 rate on this part) at about 48 significant bits.  The first axis pass reads the
// FP64 grid and splits each value, the middle pass keeps the split form in global memory (the
// same 16 bytes per complex value), and the last pass adds the parts back into FP64.
#include "fftct.cuh"
#include "kernels.h"
#include "prof.h"

namespace fde {

namespace {

constexpr int kDdThreads = 256;
template <int N> __host__ __device__ constexpr int dd_axis_lines() { return ct_lines_per_batch<dd, N, kDdThreads>(); }

// Element (o, e, t) of a pass sits at (o * N + e) * I + t.  in_dd / out_dd: the global grid
// holds split values (ddc) rather than FP64 (double2).
template <int N>
__global__ void __launch_bounds__(kDdThreads)
k_fft_axis_dd(void* __restrict__ data, int nlines, int I, const ddc* __restrict__ tw, int sign, int in_dd,
              int out_dd) {
  constexpr int LP = N + 1;
  constexpr int LPC = dd_axis_lines<N>();
  __shared__ __align__(16) ddc lines[LPC * LP];
  __shared__ int base[LPC];
  const int l0 = blockIdx.x * LPC;
  const int nl = min(LPC, nlines - l0);
  if ((int)threadIdx.x < LPC) {
    const int l = l0 + (int)threadIdx.x, o = l / I, t = l - o * I;
    base[threadIdx.x] = o * N * I + t;
  }
  __syncthreads();
  const double2* d64 = reinterpret_cast<const double2*>(data);
  const ddc* dsp = reinterpret_cast<const ddc*>(data);
  for (int idx = threadIdx.x; idx < LPC * N; idx += kDdThreads) {
    int tl, e;
    if (I == 1) { tl = idx / N; e = idx - tl * N; } else { e = idx / LPC; tl = idx - e * LPC; }
    ddc v;
    if (tl < nl) {
      const int g = base[tl] + e * I;
      if (in_dd) {
        v = dsp[g];
      } else {
        const double2 x = d64[g];
        v.x = dd_from_double(x.x);
        v.y = dd_from_double(x.y);
      }
    } else {
      v.x = dd(0);
      v.y = dd(0);
    }
    lines[tl * LP + e] = v;
  }
  __syncthreads();
  ct_lines<dd, N, kDdThreads>(lines, LinesContig{LP}, LPC, tw, sign);
  double2* o64 = reinterpret_cast<double2*>(data);
  ddc* osp = reinterpret_cast<ddc*>(data);
  for (int idx = threadIdx.x; idx < LPC * N; idx += kDdThreads) {
    int tl, e;
    if (I == 1) { tl = idx / N; e = idx - tl * N; } else { e = idx / LPC; tl = idx - e * LPC; }
    if (tl < nl) {
      const int g = base[tl] + e * I;
      const ddc v = lines[tl * LP + e];
      if (out_dd) osp[g] = v;
      else o64[g] = make_double2(dd_to_double(v.x), dd_to_double(v.y));
    }
  }
}

bool dd_axis(int n, long long nlines, long long I, cudaStream_t st, void* data, const ddc* tw, int sign, int in_dd,
             int out_dd) {
  switch (n) {
#define FDE_CASE(N)                                                                                       \
  case N:                                                                                                 \
    count_launches(1);                                                                                    \
    k_fft_axis_dd<N><<<(unsigned)ceil_div(nlines, dd_axis_lines<N>()), kDdThreads, 0, st>>>(             \
        data, (int)nlines, (int)I, tw, sign, in_dd, out_dd);                                              \
    return true;
    FDE_CASE(24) FDE_CASE(32) FDE_CASE(60) FDE_CASE(72) FDE_CASE(96) FDE_CASE(144) FDE_CASE(180) FDE_CASE(288)
#undef FDE_CASE
  }
  return false;
}

bool dd_length_ok(int n) {
  return n == 24 || n == 32 || n == 60 || n == 72 || n == 96 || n == 144 || n == 180 || n == 288;
}

}  // namespace

bool launch_fft3d_dd(double2* data, const GridDims& g, const FftPlans<dd>& fp, int sign, cudaStream_t st) {
  if (!dd_length_ok(g.n1) || !dd_length_ok(g.n2) || !dd_length_ok(g.n3)) return false;
  const long long nr = (long long)g.n1 * g.n2 * g.n3;
  if (nr >= (1ll << 31)) return false;
  ProfScope prof_("k_fft_axis_dd", st);
  dd_axis(g.n3, nr / g.n3, 1, st, data, fp.p3.tw, sign, 0, 1);
  dd_axis(g.n2, nr / g.n2, g.n3, st, data, fp.p2.tw, sign, 1, 1);
  dd_axis(g.n1, nr / g.n1, (long long)g.n2 * g.n3, st, data, fp.p1.tw, sign, 1, 0);
  return true;
}

}  // namespace fde
