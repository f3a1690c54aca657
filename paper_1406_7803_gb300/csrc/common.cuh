// common.cuh -- types and small device helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fde {

// Interleaved complex type of a real type.
template <typename T> struct cx;
template <> struct cx<float> { using t = float2; };
template <> struct cx<double> { using t = double2; };
template <typename T> using cplx = typename cx<T>::t;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T re, T im) {
  cplx<T> z; z.x = re; z.y = im; return z;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z;
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  C z; z.x = a.x * b.x + a.y * b.y; z.y = a.x * b.y - a.y * b.x; return z;
}
template <typename C, typename T> __host__ __device__ __forceinline__ C cscale(C a, T s) { a.x *= s; a.y *= s; return a; }
// multiply by sign * i
template <typename C> __host__ __device__ __forceinline__ C cmuli(C a, int sign) {
  C z; if (sign > 0) { z.x = -a.y; z.y = a.x; } else { z.x = a.y; z.y = -a.x; } return z;
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }

// Device status word bits (checked by the host after synchronising calls).
enum : unsigned { ST_NONFINITE = 1u, ST_CHOLESKY = 2u, ST_NOCONV = 4u, ST_TIMEOUT = 8u, ST_TMEM_HELD = 16u };

// Largest supported 1D transform length (one line held by one warp in shared memory).
constexpr int kMaxLine = 320;
// Largest (x, y) plane side transformed inside one CTA.
constexpr int kMaxPlane = 160;
constexpr int kMaxStages = 8;

// One 1D transform length: its radix factorisation and twiddle table
// tw[m] = exp(-2 pi i m / n), m in [0, n).
template <typename T> struct LinePlan {
  int n;
  int nstages;
  int radix[kMaxStages];
  const cplx<T>* tw;
};

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace fde
