// grid_kernels.h -- launch wrappers of the grid kernels (grid.cu).
#pragma once

#include "kernels.h"

namespace fde {

int grid_red_blocks();
template <typename T>
void grid_poisson(const cplx<T>* F, cplx<T>* V, const GridDims& g, const CellDev& c, double* partial, cudaStream_t st);
template <typename T>
void grid_gradient_g(const cplx<T>* F, cplx<T>* ox, cplx<T>* oy, cplx<T>* oz, const GridDims& g, const CellDev& c,
                     cudaStream_t st);
template <typename T>
void grid_divergence_g(cplx<T>* hx, const cplx<T>* hy, const cplx<T>* hz, const GridDims& g, const CellDev& c,
                       cudaStream_t st);
void grid_vloc_g(double2* V, const GridDims& g, const CellDev& c, const double* pos, const double* Z, int natoms,
                 double rc, cudaStream_t st);
template <typename T>
void grid_pointwise(const double* rho, cplx<T>* gx, cplx<T>* gy, cplx<T>* gz, long long nr, int xc_mode, int xc_pot,
                    int kedf, double rho_cut, double* vpart, double* partial, cudaStream_t st);
template <typename T>
void grid_real_to_c(const double* a, cplx<T>* c, long long n, cudaStream_t st);
template <typename T>
void grid_c_to_real(const cplx<T>* c, double* a, long long n, cudaStream_t st);
template <typename T>
void grid_combine(const double* a, const double* b, const double* c, const cplx<T>* d, double sd, double* out,
                  long long n, cudaStream_t st);
template <typename T>
void grid_scale_c(cplx<T>* a, double s, long long n, cudaStream_t st);
void grid_sum_rows(const double* a, int nrows, long long n, double* out, cudaStream_t st);
void grid_dot_partial(const double* a, const double* b, long long n, int mode, double* partial, cudaStream_t st);
void grid_finalize(const double* partial, int nq, double scale, double* out, cudaStream_t st);
void grid_lincomb(const double* const* ins, const double* const* res, const double* coef, int m, double beta,
                  long long n, double* out, cudaStream_t st);
void grid_axpy(double* a, const double* b, double alpha, long long n, cudaStream_t st);
void grid_nonfinite(const double* a, long long n, unsigned* status, cudaStream_t st);

}  // namespace fde
