// kernels.h -- launch wrappers of the library's CUDA kernels (internal interface between
// the host orchestration in fde_host.cu and the kernel translation units).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "dd.cuh"

namespace fde {

// Columns of one plane-wave sphere on the FFT grid.  A column is a fixed (m1, m2) with a
// contiguous run of m3 values; sphere order puts each column's run contiguously.
struct SphereDev {
  int npw, ncol, nrow;
  const int* col_start;  // [ncol + 1] offsets into the sphere
  const int* col_m3lo;   // [ncol] signed m3 of the first point
  const int* col_i1;     // [ncol] grid index i1 = m1 mod n1
  const int* col_i2;     // [ncol] grid index i2 = m2 mod n2
  const int* row_i1;     // [nrow] distinct i1 holding at least one column
};

struct GridDims {
  int n1, n2, n3;
};

template <typename T> struct FftPlans {
  LinePlan<T> p1, p2, p3;
};

// ---- H psi local part and densities (hpsi.cu) -----------------------------------------
// scratch: [nb][n3][ncol] complex T.  vplane: [n3][n1][n2] real T.
template <typename T>
void launch_hpsi_local(const cplx<T>* psi, int ldpsi, cplx<T>* hpsi, int ldh, int nb,
                       const T* kin, const T* vplane, cplx<T>* scratch, const SphereDev& sp,
                       const GridDims& g, const FftPlans<T>& fp, cudaStream_t st);

// rho_plane[n3][n1][n2] (+)= sum_b weight[b] |u_b(r)|^2 for the block of nb orbitals.
template <typename T>
void launch_density(const cplx<T>* psi, int ldpsi, int nb, const double* weight,
                    cplx<T>* scratch, double* rho_plane, int accumulate, const SphereDev& sp,
                    const GridDims& g, const FftPlans<T>& fp, cudaStream_t st);

// One (subsystem, k) block of bands of a batched H psi launch.
template <typename T> struct HpsiItemDesc {
  SphereDev sp;
  const cplx<T>* psi;
  cplx<T>* hpsi;
  const T* kin;
  const T* vplane;
  cplx<T>* scratch;  // [nb][n3][ncol] of this item
  int ld, nb;
};
// Local H psi of many items in three launches (batches of up to 24 items each).
template <typename T>
bool launch_hpsi_batch_ct(const HpsiItemDesc<T>* items, int nitems, const GridDims& g, const FftPlans<T>& fp,
                          cudaStream_t st);

// Variant of the FP32 plane pass the tuner chose for plane side n1 and z length n3 (-1: none
// tuned yet).
int query_plane_variant(int n1, int n3);
// Pin the variant (0 .. count - 1) or return to tuning (-1); false for other values.
bool pin_plane_variant(int v);

// Compile-time-length variants (hpsi_ct.cuh); return false when the grid sizes are not
// among the instantiated ones, and the runtime-length kernels run instead.
template <typename T>
bool launch_hpsi_local_ct(const cplx<T>* psi, int ldpsi, cplx<T>* hpsi, int ldh, int nb, const T* kin,
                          const T* vplane, cplx<T>* scratch, const SphereDev& sp, const GridDims& g,
                          const FftPlans<T>& fp, cudaStream_t st);
template <typename T>
bool launch_density_ct(const cplx<T>* psi, int ldpsi, int nb, const double* weight, cplx<T>* scratch,
                       double* rho_plane, int accumulate, const SphereDev& sp, const GridDims& g,
                       const FftPlans<T>& fp, cudaStream_t st);
template <typename T>
bool launch_fft3d_ct(cplx<T>* data, const GridDims& g, const FftPlans<T>& fp, int sign, cudaStream_t st);

// out[j][i] = (Tout) in[i][j], in is [rows][cols]; with optional accumulate.
template <typename Tin, typename Tout>
void launch_transpose(const Tin* in, Tout* out, int rows, int cols, int accumulate, cudaStream_t st);

// ---- dense complex algebra (linalg.cu) --------------------------------------------------
// C[i][j] = sum_g conj(A[i][g]) B[j][g], A [m][K] (lda), B [n][K] (ldb); C [m][n] FP64
// complex (ldc).  work: at least gemm_hn_work(m, n, K) double2 elements.
size_t gemm_hn_work(int m, int n, int K);
// Path of the FP32 products C = A^H B: 0 CUDA cores (FP32 FMA), 1 tensor cores with TF32
// operands, 3 tensor cores with split-TF32 operands (hi*hi + hi*lo + lo*hi, FP32 accuracy).
// Process-wide; the default is 3.
void set_gemm_hn_path(int path);
int gemm_hn_path();
// The tensor-core kernel itself (gemm_tc.cu): partial tiles into part[nsplit][m][n];
// returns nsplit, or 0 when the kernel could not be configured (nothing launched).
int gemm_hn_tc_splits(int m, int n, int K);
int launch_gemm_hn_tc(const float2* A, int lda, const float2* B, int ldb, int m, int n, int K, int passes,
                      double2* part, cudaStream_t st);
// Y = alpha U^T-combination of the rows of X + beta Y on the tensor cores (gemm_tc.cu), with
// the same passes as launch_gemm_hn_tc; false when the kernel could not be configured.
bool launch_gemm_rot_tc(const float2* X, int ldx, const double2* U, int ldu, int m, int n, int K, float2* Y,
                        int ldy, double alpha, double beta, int passes, cudaStream_t st);
// ST_* bits raised by the tensor-core kernels since the last call (read, cleared; syncs).
unsigned gemm_tc_take_status(cudaStream_t st);
bool set_tc_stage_spin(long long polls);
void disable_tensor_cores();
bool tensor_cores_disabled();
void launch_gemm_hn_reduce(const double2* part, int nsplit, int m, int n, double2* C, int ldc, cudaStream_t st);
template <typename T>
void launch_gemm_hn(const cplx<T>* A, int lda, const cplx<T>* B, int ldb, int m, int n, int K,
                    double2* C, int ldc, double2* work, cudaStream_t st);

// Y[j][g] = alpha * sum_i U[i][j] X[i][g] + beta * Y[j][g]; X [m][K] (ldx), U [m][n] FP64
// complex (ldu), Y [n][K] (ldy).  alpha/beta real.  tensor: FP32 data may take the tensor-core
// kernel (the gemm_hn path's split TF32, ~2^-20 relative per product) -- used for the projector
// expansion of H psi; the eigensolver's rotations, whose errors accumulate in the orbitals
// from one iteration to the next, keep FP32 fused multiply-adds (2^-24).
template <typename T>
void launch_gemm_rot(const cplx<T>* X, int ldx, const double2* U, int ldu, int m, int n, int K,
                     cplx<T>* Y, int ldy, double alpha, double beta, cudaStream_t st, bool tensor = false);

// Per-atom block of the projector coupling (np x np, row-major, np <= 8).
struct KbBlock {
  double d[64];
  int np;
};
// Q[a np + i][b] = sum_j D[i][j] P[a np + j][b] for natoms atoms and nb columns (FP64 complex,
// leading dimension nb).
void launch_kb_couple(const double2* P, const KbBlock& D, int natoms, int nb, double2* Q, cudaStream_t st);
// The same with its own np x np block for every atom: D [natoms][np][np] (device).
void launch_kb_couple_atoms(const double2* P, const double* D, int np, int natoms, int nb, double2* Q, cudaStream_t st);

// Cholesky S = L L^H (n x n, FP64 complex, lower, in place into L) and Linv = L^{-1};
// sets status bit ST_CHOLESKY on a pivot not above rel_pivot S_jj (the squared norm of a
// vector's part orthogonal to the earlier ones, relative to its own squared norm: below the
// rounding level of the vectors' precision they are numerically dependent).
void launch_cholesky_inv(const double2* S, int n, double2* L, double2* Linv, unsigned* status, double rel_pivot,
                         cudaStream_t st);

// Hermitian eigenproblem (FP64): A (n x n) -> eigenvalues w[n] ascending and the eigenvectors
// of the lowest nvec eigenvalues in the columns of V (other columns zero), by
// tridiagonalisation, bisection and inverse iteration (dense.cu, heev.cu).
size_t heev_work_doubles(int n, int nvec);
void launch_heev(double2* A, int n, int nvec, double* w, double2* V, double* work, cudaStream_t st);

// Row-wise helpers on [nb][K] blocks.
template <typename T>
void launch_residual(const cplx<T>* HX, const cplx<T>* X, const double* eps, int nb, int K, int ld,
                     cplx<T>* R, int ldr, cudaStream_t st);
template <typename T>
void launch_row_norms(const cplx<T>* X, int ld, int nb, int K, const T* weight, double* out,
                      double* work, cudaStream_t st);
template <typename T>
void launch_tpa(const cplx<T>* R, int ldr, const T* kin, const double* tband, int nb, int K,
                cplx<T>* W, int ldw, cudaStream_t st);
template <typename T>
void launch_scale_rows(cplx<T>* X, int ld, int nb, int K, const double* s, cudaStream_t st);
template <typename Ta, typename Tb>
void launch_convert_c(const cplx<Ta>* a, cplx<Tb>* b, size_t n, cudaStream_t st);
template <typename T>
void launch_shape_init(cplx<T>* X, int ld, const T* kin, int nb, int K, cudaStream_t st);
void launch_hermitize(double2* A, int n, cudaStream_t st);

// ---- grid kernels (grid.cu) -------------------------------------------------------------
// Full 3D transforms of complex grids [n1][n2][n3] in place: sign -1 forward (scaled by
// 1/N_r), +1 inverse (unscaled).
template <typename T>
void launch_fft3d(cplx<T>* data, const GridDims& g, const FftPlans<T>& fp, int sign, cudaStream_t st);
// The same 3D transform of an FP64 grid computed in double-float arithmetic on the FP32 pipes
// (fft_dd.cu): converted on the first axis pass, converted back on the last.  False (nothing
// launched) when an axis length has no compiled kernel.
bool launch_fft3d_dd(double2* data, const GridDims& g, const FftPlans<dd>& fp, int sign, cudaStream_t st);

struct CellDev {
  double b[3][3];  // reciprocal rows
  double omega;
};

}  // namespace fde
