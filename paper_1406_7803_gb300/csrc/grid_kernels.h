// grid_kernels.h -- launch wrappers of the grid kernels (grid.cu).
#pragma once

#include "kernels.h"

namespace fde {

int grid_red_blocks();
void grid_vloc_g(double2* V, const GridDims& g, const CellDev& c, const double* pos, const double* Z, int natoms,
                 double rc, cudaStream_t st);
template <typename T>
void grid_c_to_real(const cplx<T>* c, double* a, long long n, cudaStream_t st);
template <typename T>
void grid_combine(const double* a, const double* b, const double* c, const cplx<T>* d, double sd, double* out,
                  long long n, cudaStream_t st);
template <typename T>
void grid_scale_c(cplx<T>* a, double s, long long n, cudaStream_t st);
void grid_dot_partial(const double* a, const double* b, long long n, int mode, double* partial, cudaStream_t st);
void grid_finalize(const double* partial, int nq, double scale, double* out, cudaStream_t st);
void grid_lincomb(const double* const* ins, const double* const* res, const double* coef, int m, double beta,
                  long long n, double* out, cudaStream_t st);
void grid_axpy(double* a, const double* b, double alpha, long long n, cudaStream_t st);
void grid_nonfinite(const double* a, long long n, unsigned* status, cudaStream_t st);
// out(r) = (1 / nops) sum_o in(R_o r), R_o = diag(+-1) from the 3-bit masks (r -> -r mod grid on
// the flipped axes); in and out must not overlap.
struct SymOps {
  int n;
  int mask[8];
};
void grid_symmetrize(const double* in, double* out, const GridDims& g, const SymOps& ops, cudaStream_t st);

// ---- ultrasoft-like augmentation: charges q_ij g_a(r), g_a a normalised Gaussian of width sigma ----
// A = sum_a coef_a g_a(G) (complex grid; its inverse transform is the augmentation density).
void grid_aug_density_g(double2* A, const GridDims& g, const CellDev& c, const double* pos, const double* coef,
                        int natoms, double sigma, cudaStream_t st);
// Dscr[a] = D + q int v g_a for every atom (VG: v's forward transform, scaled by 1/N_r).
void grid_aug_screening(const double2* VG, const GridDims& g, const CellDev& c, const double* pos, int natoms,
                        double sigma, const KbBlock& D, const KbBlock& q, double* Dscr, cudaStream_t st);

// ---- packed pairs of real fields (two real grids in one complex transform) ----
constexpr int kMaxPairs = 32;
struct GradPacks {  // real-space gradients of the subsystem densities, pairwise packed
  const double2* a[kMaxPairs];  // d/dx + i d/dy of the first density of pair q
  const double2* b[kMaxPairs];  // the same for the second density (when has_b)
  const double2* z[kMaxPairs];  // d/dz of the first + i d/dz of the second
  int has_b[kMaxPairs];
  int npairs;
};
void grid_pack2(const double* a, const double* b, double2* c, long long n, cudaStream_t st);
void grid_unpack_density(const double2* C, int has_b, double2* RT, int accumulate, double2* Pa, double2* Pb,
                         double2* Pz, const GridDims& g, const CellDev& c, double* partial, cudaStream_t st);
// fp32: the pointwise functionals in FP32 arithmetic (mixed path), else FP64.
void grid_pw_total(const double* rho, const GradPacks& gp, int xc_mode, int kedf, double rho_cut, double* vpart,
                   double* hx, double* hy, double* hz, long long nr, double* partial, bool fp32, cudaStream_t st);
// The divergence arguments (Da, Db, Dz), the reciprocal-space potentials F and their transforms
// are in precision TD: FP64 in FP64 contexts (Da.. may alias Pa..), FP32 in mixed ones.
template <typename TD>
void grid_pw_pair(const double* ra, const double* rb, const double2* Pa, const double2* Pb, const double2* Pz,
                  cplx<TD>* Da, cplx<TD>* Db, cplx<TD>* Dz, const double* hx, const double* hy, const double* hz,
                  const double* vtot, int xc_mode, int kedf, double rho_cut, double* wa, double* wb, int write_d,
                  long long nr, double* partial, cudaStream_t st);
template <typename TD>
void grid_assemble_pair(const double2* RT, const cplx<TD>* Da, const cplx<TD>* Db, const cplx<TD>* Dz, int has_b,
                        cplx<TD>* F, const GridDims& g, const CellDev& c, double* partial, cudaStream_t st);
template <typename TD>
void grid_finish_pair(const cplx<TD>* F, const double* vloc, double* va, double* vb, long long n, cudaStream_t st);

}  // namespace fde
