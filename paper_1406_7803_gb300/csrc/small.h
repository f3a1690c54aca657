// small.h -- launch wrappers of small.cu.
#pragma once

#include "kernels.h"

namespace fde {

// C[m][n] = op(A) op(B), op = 0 identity, 1 conjugate transpose (row-major, FP64 complex).
void launch_small_gemm(const double2* A, int lda, int opA, const double2* B, int ldb, int opB, int m, int n, int k,
                       double2* C, int ldc, cudaStream_t st);

template <typename T>
void launch_gather_rows(const cplx<T>* src, int lds, const int* idx, int nrows, int K, cplx<T>* dst, int ldd,
                        cudaStream_t st);

}  // namespace fde
