// small.cu -- products of small dense FP64 complex matrices (subspace size <= a few hundred)
// used by the Rayleigh-Ritz step: C = op(A) op(B) with op = identity or conjugate transpose.
#include "kernels.h"
#include "prof.h"
#include "small.h"

namespace fde {

__global__ void k_small_gemm(const double2* __restrict__ A, int lda, int opA, const double2* __restrict__ B, int ldb,
                             int opB, int m, int n, int k, double2* __restrict__ C, int ldc) {
  __shared__ double2 As[16][17], Bs[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
  double re = 0, im = 0;
  for (int k0 = 0; k0 < k; k0 += 16) {
    {
      const int kk = k0 + tx;
      double2 a = make_double2(0, 0);
      if (i < m && kk < k) a = opA ? cconj(A[(size_t)kk * lda + i]) : A[(size_t)i * lda + kk];
      As[ty][tx] = a;
    }
    {
      const int kk = k0 + ty;
      double2 b = make_double2(0, 0);
      if (j < n && kk < k) b = opB ? cconj(B[(size_t)j * ldb + kk]) : B[(size_t)kk * ldb + j];
      Bs[ty][tx] = b;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const double2 a = As[ty][q], b = Bs[q][tx];
      re += a.x * b.x - a.y * b.y;
      im += a.x * b.y + a.y * b.x;
    }
    __syncthreads();
  }
  if (i < m && j < n) C[(size_t)i * ldc + j] = make_double2(re, im);
}

void launch_small_gemm(const double2* A, int lda, int opA, const double2* B, int ldb, int opB, int m, int n, int k,
                       double2* C, int ldc, cudaStream_t st) {
  dim3 grid(ceil_div(n, 16), ceil_div(m, 16));
  count_launches(1);
  k_small_gemm<<<grid, dim3(16, 16), 0, st>>>(A, lda, opA, B, ldb, opB, m, n, k, C, ldc);
}

// Copy selected rows: dst[r] = src[idx[r]] for r < nrows (complex T, row length K).
template <typename T>
__global__ void k_gather_rows(const cplx<T>* __restrict__ src, int lds, const int* __restrict__ idx, int K,
                              cplx<T>* __restrict__ dst, int ldd) {
  const int r = blockIdx.y;
  const int s = idx[r];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x)
    dst[(size_t)r * ldd + g] = src[(size_t)s * lds + g];
}

template <typename T>
void launch_gather_rows(const cplx<T>* src, int lds, const int* idx, int nrows, int K, cplx<T>* dst, int ldd,
                        cudaStream_t st) {
  if (nrows <= 0) return;
  count_launches(1);
  k_gather_rows<T><<<dim3(ceil_div(K, 1024), nrows), 256, 0, st>>>(src, lds, idx, K, dst, ldd);
}

template void launch_gather_rows<float>(const float2*, int, const int*, int, int, float2*, int, cudaStream_t);
template void launch_gather_rows<double>(const double2*, int, const int*, int, int, double2*, int, cudaStream_t);

}  // namespace fde
