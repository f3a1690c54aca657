// linalg.cu -- dense complex algebra of the subspace eigensolver (Eq. KS solved by block
// Davidson): band-block inner products (Gram / subspace Hamiltonian / projector
// contractions), band-block rotations, FP64 Cholesky with triangular inverse, and the
// row-wise residual / preconditioner helpers.
#include <math.h>
#include <stdlib.h>

#include <algorithm>

#include "dense.h"
#include "kernels.h"
#include "prof.h"

namespace fde {

// ---- C = A^H B over a long K ------------------------------------------------------------
// 32 x 32 output tile per CTA (256 threads, 2 x 2 outputs each), K split over gridDim.z;
// each split writes its partial tile, a second kernel sums the splits in a fixed order.
constexpr int kGT = 32, kGK = 32;

template <typename T, typename Acc>
__global__ void __launch_bounds__(256)
k_gemm_hn_partial(const cplx<T>* __restrict__ A, int lda, const cplx<T>* __restrict__ B, int ldb, int m, int n,
                  int K, int kchunk, double2* __restrict__ part) {
  using C = cplx<T>;
  __shared__ C As[kGT][kGK + 1];
  __shared__ C Bs[kGT][kGK + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.x * kGT, j0 = blockIdx.y * kGT;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  Acc re[2][2] = {{0, 0}, {0, 0}}, im[2][2] = {{0, 0}, {0, 0}};
  for (int k0 = kb; k0 < ke; k0 += kGK) {
    for (int idx = threadIdx.x; idx < kGT * kGK; idx += 256) {
      const int r = idx / kGK, kk = idx % kGK;
      const int g = k0 + kk;
      const bool ok = g < ke;
      As[r][kk] = (ok && i0 + r < m) ? A[(size_t)(i0 + r) * lda + g] : mk<T>(0, 0);
      Bs[r][kk] = (ok && j0 + r < n) ? B[(size_t)(j0 + r) * ldb + g] : mk<T>(0, 0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kGK; ++kk) {
      C a0 = As[ty][kk], a1 = As[ty + 16][kk];
      C b0 = Bs[tx][kk], b1 = Bs[tx + 16][kk];
      // conj(a) * b
      re[0][0] += (Acc)a0.x * b0.x + (Acc)a0.y * b0.y; im[0][0] += (Acc)a0.x * b0.y - (Acc)a0.y * b0.x;
      re[0][1] += (Acc)a0.x * b1.x + (Acc)a0.y * b1.y; im[0][1] += (Acc)a0.x * b1.y - (Acc)a0.y * b1.x;
      re[1][0] += (Acc)a1.x * b0.x + (Acc)a1.y * b0.y; im[1][0] += (Acc)a1.x * b0.y - (Acc)a1.y * b0.x;
      re[1][1] += (Acc)a1.x * b1.x + (Acc)a1.y * b1.y; im[1][1] += (Acc)a1.x * b1.y - (Acc)a1.y * b1.x;
    }
    __syncthreads();
  }
  double2* P = part + (size_t)blockIdx.z * m * n;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
      if (i < m && j < n) P[(size_t)i * n + j] = make_double2((double)re[a][b], (double)im[a][b]);
    }
}

// Sum of the K-split partial tiles: a CTA owns 32 consecutive outputs (one per lane, so
// every split's row segment is one coalesced 512-byte read); warp w sums the splits
// s = w, w + 8, ..., and the eight warp sums are added in warp order (fixed order: the
// result does not depend on scheduling).
__global__ void __launch_bounds__(256)
k_gemm_hn_reduce(const double2* __restrict__ part, int nsplit, int m, int n, double2* C, int ldc) {
  __shared__ double2 acc[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long mn = (long long)m * n;
  const long long idx = (long long)blockIdx.x * 32 + lane;
  double re = 0, im = 0;
  if (idx < mn)
    for (int s = w; s < nsplit; s += 8) {
      const double2 v = part[(size_t)s * mn + idx];
      re += v.x;
      im += v.y;
    }
  acc[w][lane] = make_double2(re, im);
  __syncthreads();
  if (w == 0 && idx < mn) {
    double2 t = acc[0][lane];
#pragma unroll
    for (int q = 1; q < 8; ++q) {
      t.x += acc[q][lane].x;
      t.y += acc[q][lane].y;
    }
    const int i = (int)(idx / n), j = (int)(idx % n);
    C[(size_t)i * ldc + j] = t;
  }
}

static int gemm_hn_splits(int m, int n, int K) {
  const int tiles = ceil_div(m, kGT) * ceil_div(n, kGT);
  int s = ceil_div(4 * 152, tiles);
  const int smax = ceil_div(K, 512);
  if (s > smax) s = smax;
  if (s < 1) s = 1;
  return s;
}

size_t gemm_hn_work(int m, int n, int K) {
  return (size_t)std::max(gemm_hn_splits(m, n, K), gemm_hn_tc_splits(m, n, K)) * m * n;
}

// FDE_GEMM_PATH (0, 1 or 3) in the environment sets the initial path.
static int initial_gemm_path() {
  const char* e = getenv("FDE_GEMM_PATH");
  const int p = e ? atoi(e) : 3;
  return (p == 0 || p == 1) ? p : 3;
}
static int g_gemm_path = initial_gemm_path();
void set_gemm_hn_path(int path) { g_gemm_path = (path == 0 || path == 1) ? path : 3; }
int gemm_hn_path() { return g_gemm_path; }
// Set once a tensor-core kernel kept its tensor memory (its MMAs could not be confirmed
// complete): every later product of the process takes the CUDA-core path.
static bool g_tc_disabled = false;
void disable_tensor_cores() { g_tc_disabled = true; }
bool tensor_cores_disabled() { return g_tc_disabled; }

void launch_gemm_hn_reduce(const double2* part, int nsplit, int m, int n, double2* C, int ldc, cudaStream_t st) {
  count_launches(1);
  ProfScope prof_r("k_gemm_hn_reduce", st);
  k_gemm_hn_reduce<<<ceil_div((long long)m * n, 32), 256, 0, st>>>(part, nsplit, m, n, C, ldc);
}

template <typename T>
static bool gemm_hn_tensor(const cplx<T>*, int, const cplx<T>*, int, int, int, int, double2*, int, double2*,
                           cudaStream_t) {
  return false;  // FP64 products stay on the CUDA cores (the part's FP64 tensor rate is no faster)
}
template <>
bool gemm_hn_tensor<float>(const float2* A, int lda, const float2* B, int ldb, int m, int n, int K, double2* C,
                           int ldc, double2* work, cudaStream_t st) {
  if (g_gemm_path == 0 || g_tc_disabled || K <= 0) return false;
  const int ns = launch_gemm_hn_tc(A, lda, B, ldb, m, n, K, g_gemm_path, work, st);
  if (ns == 0) return false;
  launch_gemm_hn_reduce(work, ns, m, n, C, ldc, st);
  return true;
}

template <typename T>
void launch_gemm_hn(const cplx<T>* A, int lda, const cplx<T>* B, int ldb, int m, int n, int K, double2* C,
                    int ldc, double2* work, cudaStream_t st) {
  if (m <= 0 || n <= 0) return;
  if (gemm_hn_tensor<T>(A, lda, B, ldb, m, n, K, C, ldc, work, st)) return;
  const int s = gemm_hn_splits(m, n, K);
  int kchunk = ceil_div(K, s);
  kchunk = ((kchunk + kGK - 1) / kGK) * kGK;
  const int ns = ceil_div(K, kchunk > 0 ? kchunk : 1);
  const dim3 grid(ceil_div(m, kGT), ceil_div(n, kGT), ns > 0 ? ns : 1);
  count_launches(1);
  ProfScope prof_("k_gemm_hn_partial", st);
  k_gemm_hn_partial<T, T><<<grid, 256, 0, st>>>(A, lda, B, ldb, m, n, K, kchunk, work);
  count_launches(1);
  ProfScope prof_r("k_gemm_hn_reduce", st);
  k_gemm_hn_reduce<<<ceil_div((long long)m * n, 32), 256, 0, st>>>(work, grid.z, m, n, C, ldc);
}

// ---- Y = alpha * U^T-combination of rows of X + beta * Y -----------------------------------
// CTA: 64 columns g x 32 output rows j; each of the 256 threads owns one g and 8 rows.
template <typename T>
__global__ void __launch_bounds__(256)
k_gemm_rot(const cplx<T>* __restrict__ X, int ldx, const double2* __restrict__ U, int ldu, int m, int n, int K,
           cplx<T>* __restrict__ Y, int ldy, T alpha, T beta) {
  using C = cplx<T>;
  __shared__ C Xs[16][64];
  __shared__ C Us[16][32];
  const int tg = threadIdx.x & 63, tj = threadIdx.x >> 6;
  const int g0 = blockIdx.x * 64, j0 = blockIdx.y * 32;
  const int g = g0 + tg;
  T re[8], im[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) re[q] = im[q] = 0;
  for (int i0 = 0; i0 < m; i0 += 16) {
    for (int idx = threadIdx.x; idx < 16 * 64; idx += 256) {
      const int ii = idx / 64, gg = idx % 64;
      Xs[ii][gg] = (i0 + ii < m && g0 + gg < K) ? X[(size_t)(i0 + ii) * ldx + g0 + gg] : mk<T>(0, 0);
    }
    for (int idx = threadIdx.x; idx < 16 * 32; idx += 256) {
      const int ii = idx / 32, jj = idx % 32;
      if (i0 + ii < m && j0 + jj < n) {
        const double2 u = U[(size_t)(i0 + ii) * ldu + j0 + jj];
        Us[ii][jj] = mk<T>((T)u.x, (T)u.y);
      } else {
        Us[ii][jj] = mk<T>(0, 0);
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int ii = 0; ii < 16; ++ii) {
      const C x = Xs[ii][tg];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const C u = Us[ii][tj + 4 * q];
        re[q] += u.x * x.x - u.y * x.y;
        im[q] += u.x * x.y + u.y * x.x;
      }
    }
    __syncthreads();
  }
  if (g >= K) return;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int j = j0 + tj + 4 * q;
    if (j < n) {
      C* y = Y + (size_t)j * ldy + g;
      C o;
      if (beta != (T)0) {
        const C old = *y;
        o.x = alpha * re[q] + beta * old.x;
        o.y = alpha * im[q] + beta * old.y;
      } else {
        o.x = alpha * re[q];
        o.y = alpha * im[q];
      }
      *y = o;
    }
  }
}

template <typename T>
static bool gemm_rot_tensor(const cplx<T>*, int, const double2*, int, int, int, int, cplx<T>*, int, double, double,
                            cudaStream_t) {
  return false;
}
template <>
bool gemm_rot_tensor<float>(const float2* X, int ldx, const double2* U, int ldu, int m, int n, int K, float2* Y,
                            int ldy, double alpha, double beta, cudaStream_t st) {
  if (g_gemm_path == 0 || g_tc_disabled || m <= 0) return false;
  return launch_gemm_rot_tc(X, ldx, U, ldu, m, n, K, Y, ldy, alpha, beta, g_gemm_path, st);
}

template <typename T>
void launch_gemm_rot(const cplx<T>* X, int ldx, const double2* U, int ldu, int m, int n, int K, cplx<T>* Y,
                     int ldy, double alpha, double beta, cudaStream_t st, bool tensor) {
  if (n <= 0 || K <= 0) return;
  if (tensor && gemm_rot_tensor<T>(X, ldx, U, ldu, m, n, K, Y, ldy, alpha, beta, st)) return;
  const dim3 grid(ceil_div(K, 64), ceil_div(n, 32));
  count_launches(1);
  ProfScope prof_("k_gemm_rot", st);
  k_gemm_rot<T><<<grid, 256, 0, st>>>(X, ldx, U, ldu, m, n, K, Y, ldy, (T)alpha, (T)beta);
}

// ---- Cholesky and triangular inverse (one CTA) -------------------------------------------
__global__ void __launch_bounds__(512)
k_cholesky_inv(const double2* __restrict__ S, int n, double2* __restrict__ L, double2* __restrict__ Li,
               unsigned* status, double rel_pivot) {
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    L[idx] = (j <= i) ? S[idx] : make_double2(0, 0);
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const double d = L[(size_t)j * n + j].x;
    if (!(d > rel_pivot * S[(size_t)j * n + j].x)) {
      if (threadIdx.x == 0) { fail = 1; atomicOr(status, ST_CHOLESKY); }
      break;
    }
    const double sd = sqrt(d);
    const double inv = 1.0 / sd;
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      double2 v = L[(size_t)i * n + j];
      v.x *= inv;
      v.y *= inv;
      L[(size_t)i * n + j] = v;
    }
    if (threadIdx.x == 0) L[(size_t)j * n + j] = make_double2(sd, 0.0);
    __syncthreads();
    const int rem = n - j - 1;
    for (int idx = threadIdx.x; idx < rem * rem; idx += blockDim.x) {
      const int i = j + 1 + idx / rem, k = j + 1 + idx % rem;
      if (k <= i) {
        const double2 a = L[(size_t)i * n + j], b = L[(size_t)k * n + j];
        double2 v = L[(size_t)i * n + k];
        // v -= a * conj(b)
        v.x -= a.x * b.x + a.y * b.y;
        v.y -= a.y * b.x - a.x * b.y;
        L[(size_t)i * n + k] = v;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  if (fail) return;
  // Li = L^{-1}: column c by forward substitution, one warp per column (lanes share the
  // inner products).
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = threadIdx.x >> 5; c < n; c += nw) {
    for (int i = lane; i < c; i += 32) Li[(size_t)i * n + c] = make_double2(0, 0);
    for (int i = c; i < n; ++i) {
      double re = 0.0, im = 0.0;
      for (int k = c + lane; k < i; k += 32) {
        const double2 l = L[(size_t)i * n + k], x = Li[(size_t)k * n + c];
        re += l.x * x.x - l.y * x.y;
        im += l.x * x.y + l.y * x.x;
      }
      for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (lane == 0) {
        const double dd = L[(size_t)i * n + i].x;
        Li[(size_t)i * n + c] = make_double2(((i == c) ? 1.0 : 0.0) - re, -im);
        Li[(size_t)i * n + c].x /= dd;
        Li[(size_t)i * n + c].y /= dd;
      }
      __syncwarp();
    }
  }
}

// The cluster-distributed factorisation (dense.cu) when n fits it, else one CTA.
void launch_cholesky_inv(const double2* S, int n, double2* L, double2* Linv, unsigned* status, double rel_pivot,
                         cudaStream_t st) {
  if (launch_cholesky_cluster(S, n, L, Linv, status, rel_pivot, st)) return;
  count_launches(1);
  k_cholesky_inv<<<1, 512, 0, st>>>(S, n, L, Linv, status, rel_pivot);
}

// ---- per-atom projector coupling ------------------------------------------------------------
// Q[a np + i][b] = sum_j D[i][j] P[a np + j][b]: D is the same small block for every atom, so
// the coupling of Eq. KB (nonlocal part) is block diagonal and needs no dense product.
__global__ void k_kb_couple(const double2* __restrict__ P, KbBlock D, int natoms, int nb, double2* __restrict__ Q) {
  const long long n = (long long)natoms * D.np * nb;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n; idx += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(idx % nb);
    const long long r = idx / nb;
    const int i = (int)(r % D.np);
    const long long base = (r - i) * nb + b;
    double re = 0, im = 0;
    for (int j = 0; j < D.np; ++j) {
      const double d = D.d[i * D.np + j];
      const double2 p = P[base + (long long)j * nb];
      re += d * p.x;
      im += d * p.y;
    }
    Q[idx] = make_double2(re, im);
  }
}

void launch_kb_couple(const double2* P, const KbBlock& D, int natoms, int nb, double2* Q, cudaStream_t st) {
  const long long n = (long long)natoms * D.np * nb;
  if (n <= 0) return;
  count_launches(1);
  ProfScope prof_("k_kb_couple", st);
  const int blocks = (int)std::min<long long>((n + 255) / 256, 1024);
  k_kb_couple<<<blocks, 256, 0, st>>>(P, D, natoms, nb, Q);
}

// The same with a different block for every atom: D [natoms][np][np] in device memory (the
// screened couplings of ultrasoft-like atoms).
__global__ void k_kb_couple_atoms(const double2* __restrict__ P, const double* __restrict__ D, int np, int natoms,
                                  int nb, double2* __restrict__ Q) {
  const long long n = (long long)natoms * np * nb;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n; idx += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(idx % nb);
    const long long r = idx / nb;
    const int i = (int)(r % np);
    const int a = (int)(r / np);
    const long long base = (r - i) * nb + b;
    const double* Da = D + (size_t)a * np * np;
    double re = 0, im = 0;
    for (int j = 0; j < np; ++j) {
      const double d = Da[i * np + j];
      const double2 p = P[base + (long long)j * nb];
      re += d * p.x;
      im += d * p.y;
    }
    Q[idx] = make_double2(re, im);
  }
}

void launch_kb_couple_atoms(const double2* P, const double* D, int np, int natoms, int nb, double2* Q, cudaStream_t st) {
  const long long n = (long long)natoms * np * nb;
  if (n <= 0) return;
  count_launches(1);
  ProfScope prof_("k_kb_couple", st);
  const int blocks = (int)std::min<long long>((n + 255) / 256, 1024);
  k_kb_couple_atoms<<<blocks, 256, 0, st>>>(P, D, np, natoms, nb, Q);
}

__global__ void k_hermitize(double2* A, int n) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int i = idx / n, j = idx % n;
  if (j < i) return;
  const double2 a = A[(size_t)i * n + j], b = A[(size_t)j * n + i];
  const double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
  A[(size_t)i * n + j] = h;
  A[(size_t)j * n + i] = make_double2(h.x, -h.y);
  if (i == j) A[(size_t)i * n + i].y = 0.0;
}

void launch_hermitize(double2* A, int n, cudaStream_t st) {
  count_launches(1);
  k_hermitize<<<ceil_div((long long)n * n, 256), 256, 0, st>>>(A, n);
}

// ---- row-wise helpers ----------------------------------------------------------------------
template <typename T>
__global__ void k_residual(const cplx<T>* __restrict__ HX, const cplx<T>* __restrict__ X, const double* eps, int K,
                           int ld, cplx<T>* __restrict__ R, int ldr) {
  const int j = blockIdx.y;
  const T e = (T)eps[j];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    const cplx<T> h = HX[(size_t)j * ld + g], x = X[(size_t)j * ld + g];
    R[(size_t)j * ldr + g] = mk<T>(h.x - e * x.x, h.y - e * x.y);
  }
}

template <typename T>
void launch_residual(const cplx<T>* HX, const cplx<T>* X, const double* eps, int nb, int K, int ld, cplx<T>* R,
                     int ldr, cudaStream_t st) {
  if (nb <= 0) return;
  count_launches(1);
  k_residual<T><<<dim3(ceil_div(K, 256 * 4), nb), 256, 0, st>>>(HX, X, eps, K, ld, R, ldr);
}

// out[j] = sum_g weight[g] |X[j][g]|^2 (weight NULL: 1); one CTA per row, fixed order.
template <typename T>
__global__ void k_row_norms(const cplx<T>* __restrict__ X, int ld, int K, const T* __restrict__ weight,
                            double* out) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  double acc = 0;
  for (int g = threadIdx.x; g < K; g += blockDim.x) {
    const cplx<T> x = X[(size_t)j * ld + g];
    const double m2 = (double)x.x * x.x + (double)x.y * x.y;
    acc += weight ? (double)weight[g] * m2 : m2;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    out[j] = t;
  }
}

template <typename T>
void launch_row_norms(const cplx<T>* X, int ld, int nb, int K, const T* weight, double* out, double*,
                      cudaStream_t st) {
  if (nb <= 0) return;
  count_launches(1);
  k_row_norms<T><<<nb, 512, 0, st>>>(X, ld, K, weight, out);
}

// Teter-Payne-Allan kinetic preconditioner: W = K(x) R with x = |k+G|^2/2 / T_band,
// K(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4).
template <typename T>
__global__ void k_tpa(const cplx<T>* __restrict__ R, int ldr, const T* __restrict__ kin, const double* tband, int K,
                      cplx<T>* __restrict__ W, int ldw) {
  const int j = blockIdx.y;
  const T tb = (T)fmax(tband[j], 1e-12);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    const T x = kin[g] / tb;
    const T p = (T)27 + x * ((T)18 + x * ((T)12 + x * (T)8));
    const T f = p / (p + (T)16 * x * x * x * x);
    const cplx<T> r = R[(size_t)j * ldr + g];
    W[(size_t)j * ldw + g] = mk<T>(f * r.x, f * r.y);
  }
}

template <typename T>
void launch_tpa(const cplx<T>* R, int ldr, const T* kin, const double* tband, int nb, int K, cplx<T>* W, int ldw,
                cudaStream_t st) {
  if (nb <= 0) return;
  count_launches(1);
  k_tpa<T><<<dim3(ceil_div(K, 256 * 4), nb), 256, 0, st>>>(R, ldr, kin, tband, K, W, ldw);
}

template <typename T>
__global__ void k_scale_rows(cplx<T>* X, int ld, int K, const double* s) {
  const int j = blockIdx.y;
  const T f = (T)s[j];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    cplx<T> x = X[(size_t)j * ld + g];
    x.x *= f;
    x.y *= f;
    X[(size_t)j * ld + g] = x;
  }
}

template <typename T>
void launch_scale_rows(cplx<T>* X, int ld, int nb, int K, const double* s, cudaStream_t st) {
  if (nb <= 0) return;
  count_launches(1);
  k_scale_rows<T><<<dim3(ceil_div(K, 256 * 4), nb), 256, 0, st>>>(X, ld, K, s);
}

template <typename Ta, typename Tb>
__global__ void k_convert_c(const cplx<Ta>* a, cplx<Tb>* b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = mk<Tb>((Tb)a[i].x, (Tb)a[i].y);
}

template <typename Ta, typename Tb>
void launch_convert_c(const cplx<Ta>* a, cplx<Tb>* b, size_t n, cudaStream_t st) {
  if (!n) return;
  count_launches(1);
  k_convert_c<Ta, Tb><<<(int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, st>>>(a, b, n);
}

template <typename T>
__global__ void k_shape_init(cplx<T>* X, int ld, const T* kin, int K) {
  const int j = blockIdx.y;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    cplx<T> x = X[(size_t)j * ld + g];
    const T f = (T)1 / ((T)1 + kin[g]);
    x.x *= f;
    x.y *= f;
    X[(size_t)j * ld + g] = x;
  }
}

template <typename T>
void launch_shape_init(cplx<T>* X, int ld, const T* kin, int nb, int K, cudaStream_t st) {
  if (nb <= 0) return;
  count_launches(1);
  k_shape_init<T><<<dim3(ceil_div(K, 256 * 4), nb), 256, 0, st>>>(X, ld, kin, K);
}

#define FDE_INST_T(T)                                                                                            \
  template void launch_gemm_hn<T>(const cplx<T>*, int, const cplx<T>*, int, int, int, int, double2*, int,        \
                                  double2*, cudaStream_t);                                                       \
  template void launch_gemm_rot<T>(const cplx<T>*, int, const double2*, int, int, int, int, cplx<T>*, int,       \
                                   double, double, cudaStream_t, bool);                                          \
  template void launch_residual<T>(const cplx<T>*, const cplx<T>*, const double*, int, int, int, cplx<T>*, int,  \
                                   cudaStream_t);                                                                \
  template void launch_row_norms<T>(const cplx<T>*, int, int, int, const T*, double*, double*, cudaStream_t);    \
  template void launch_tpa<T>(const cplx<T>*, int, const T*, const double*, int, int, cplx<T>*, int,             \
                              cudaStream_t);                                                                     \
  template void launch_scale_rows<T>(cplx<T>*, int, int, int, const double*, cudaStream_t);                      \
  template void launch_shape_init<T>(cplx<T>*, int, const T*, int, int, cudaStream_t);
FDE_INST_T(float)
FDE_INST_T(double)
template void launch_convert_c<double, float>(const double2*, float2*, size_t, cudaStream_t);
template void launch_convert_c<float, double>(const float2*, double2*, size_t, cudaStream_t);
template void launch_convert_c<double, double>(const double2*, double2*, size_t, cudaStream_t);

}  // namespace fde
