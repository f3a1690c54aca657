// dense.h -- cluster-distributed FP64 dense kernels of the Rayleigh-Ritz step (dense.cu).
#pragma once

#include "kernels.h"

namespace fde {

// Largest n the cluster kernels take (0 when thread-block clusters are unavailable).
int dense_cluster_max_n();

// S = L L^H and Li = L^{-1} (n x n FP64 complex, row-major, lower); ST_CHOLESKY in *status on
// a pivot not above rel_pivot times the input diagonal entry.  Returns false (nothing
// launched) when n is out of range.
bool launch_cholesky_cluster(const double2* S, int n, double2* L, double2* Li, unsigned* status, double rel_pivot,
                             cudaStream_t st);

// Eigenvalues w[n] ascending and eigenvectors of the lowest nvec (column j of the row-major V)
// of the Hermitian A (not modified); columns nvec.. of V are zero.  work: at least
// heev_cluster_work_doubles(n, nvec) doubles.  Returns false when n is out of range.
size_t heev_cluster_work_doubles(int n, int nvec);
bool launch_heev_cluster(const double2* A, int n, int nvec, double* w, double2* V, double* work, cudaStream_t st);

}  // namespace fde
