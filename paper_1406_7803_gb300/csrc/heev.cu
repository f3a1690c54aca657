// heev.cu -- FP64 Hermitian eigenproblem of the Rayleigh-Ritz step (Eq. KS, block solver):
// the one-CTA solver for sizes beyond the cluster-distributed one of dense.cu.
//
// One CTA of 1024 threads:
//   1. Householder reduction of the Hermitian A (n x n) to a real symmetric tridiagonal
//      T = Q^H A Q, Q = H_0 H_1 ... H_{n-2}, H_k = I - tau_k v_k v_k^H; each reflector
//      zeroes column k below the subdiagonal and makes the subdiagonal element real.
//   2. Every eigenvalue of T by bisection on Sturm counts (one thread per eigenvalue), so
//      they come out in ascending order.
//   3. Eigenvectors of T for the lowest nvec eigenvalues by inverse iteration with a
//      partially pivoted tridiagonal LU; eigenvalues closer than 1e-3 ||T|| form a cluster
//      whose vectors are orthogonalised against each other (one warp per cluster).
//   4. Back-transformation v = Q z (one warp per vector).
#include <math.h>

#include <algorithm>

#include "dense.h"
#include "kernels.h"
#include "prof.h"

namespace fde {

constexpr int kHeevThreads = 1024;
constexpr int kHeevWarps = kHeevThreads / 32;

__device__ __forceinline__ double block_sum_heev(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0;
  for (int k = 0; k < kHeevWarps; ++k) t += red[k];
  return t;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sturm count: number of eigenvalues of T below x.
__device__ int sturm_count(const double* d, const double* e, int n, double x, double pivmin) {
  int c = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++c;
  for (int j = 1; j < n; ++j) {
    q = d[j] - x - e[j - 1] * e[j - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++c;
  }
  return c;
}

// Solve (T - lambda I) x = b in place (b -> x) with partial pivoting; work: 4n doubles.
__device__ void tridiag_solve(const double* d, const double* e, int n, double lambda, double tiny, double* b,
                              double* work) {
  double* a = work;         // diagonal after elimination
  double* u1 = work + n;    // first superdiagonal
  double* u2 = work + 2 * n;  // second superdiagonal (fill from pivoting)
  double* l = work + 3 * n;   // multipliers; sign bit of the stored value codes nothing
  int* piv = reinterpret_cast<int*>(work + 4 * n);  // needs n ints (n/2 doubles)
  for (int j = 0; j < n; ++j) {
    a[j] = d[j] - lambda;
    u1[j] = (j < n - 1) ? e[j] : 0.0;
    u2[j] = 0.0;
  }
  for (int j = 0; j < n - 1; ++j) {
    const double sub = e[j];
    if (fabs(a[j]) >= fabs(sub)) {
      piv[j] = 0;
      const double aj = (a[j] == 0.0) ? tiny : a[j];
      const double m = sub / aj;
      l[j] = m;
      a[j + 1] -= m * u1[j];
      // u2 row j stays 0
    } else {
      piv[j] = 1;
      // swap rows j and j+1: row j+1 = [sub, a_{j+1}, u1_{j+1}], row j = [a_j, u1_j, 0]
      const double m = a[j] / sub;
      l[j] = m;
      const double nj0 = sub, nj1 = a[j + 1], nj2 = (j + 1 < n - 1) ? u1[j + 1] : 0.0;
      const double oj1 = u1[j];
      a[j] = nj0;
      u1[j] = nj1;
      u2[j] = nj2;
      a[j + 1] = oj1 - m * nj1;
      if (j + 1 < n - 1) u1[j + 1] = -m * nj2;
    }
  }
  if (a[n - 1] == 0.0) a[n - 1] = tiny;
  // forward: apply the row operations to b
  for (int j = 0; j < n - 1; ++j) {
    if (piv[j]) {
      const double t = b[j];
      b[j] = b[j + 1];
      b[j + 1] = t - l[j] * b[j];
    } else {
      b[j + 1] -= l[j] * b[j];
    }
  }
  // back substitution
  for (int j = n - 1; j >= 0; --j) {
    double s = b[j];
    if (j + 1 < n) s -= u1[j] * b[j + 1];
    if (j + 2 < n) s -= u2[j] * b[j + 2];
    const double aj = (a[j] == 0.0) ? tiny : a[j];
    b[j] = s / aj;
  }
}

__device__ __forceinline__ double start_value(int i, int j) {
  unsigned h = (unsigned)(i * 2654435761u) ^ (unsigned)(j * 40503u + 0x9e3779b9u);
  h ^= h >> 15;
  h *= 2246822519u;
  h ^= h >> 13;
  return 0.5 + (double)(h & 0xffff) / 65536.0;
}

// A: n x n Hermitian (full, row-major), destroyed.  w[n] ascending eigenvalues; V: column j
// (j < nvec) the eigenvector of w[j] (V[r * n + j]); columns >= nvec are zero.
// work: heev_work_doubles(n, nvec) doubles.
__global__ void __launch_bounds__(kHeevThreads)
k_heev(double2* __restrict__ A, int n, int nvec, double* __restrict__ w, double2* __restrict__ V,
       double* __restrict__ work) {
  __shared__ double red[kHeevWarps];
  __shared__ double2 s_tau, s_scale;
  __shared__ int s_cl_start[1025];
  __shared__ int s_ncl;
  __shared__ double s_tnorm, s_lo, s_hi;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* d = work;
  double* e = d + n;
  double2* tau = reinterpret_cast<double2*>(e + n);
  double2* p = tau + n;
  double* Z = reinterpret_cast<double*>(p + n);  // nvec x n
  double* lu = Z + (size_t)nvec * n;             // kHeevWarps x 6n

  // ---- 1. tridiagonalisation ----
  for (int k = 0; k < n - 1; ++k) {
    const int L = n - k - 1;
    double2* col = A + (size_t)(k + 1) * n + k;  // A[k+1+i][k] = col[i * n]
    double acc = 0;
    for (int i = tid + 1; i < L; i += kHeevThreads) {
      const double2 x = col[(size_t)i * n];
      acc += x.x * x.x + x.y * x.y;
    }
    const double xn2 = block_sum_heev(acc, red);
    if (tid == 0) {
      const double2 alpha = col[0];
      double2 t = make_double2(0, 0), sc = make_double2(0, 0);
      double beta = alpha.x;
      if (!(xn2 == 0.0 && alpha.y == 0.0)) {
        beta = -copysign(sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2), alpha.x);
        t = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
        // sc = 1 / (alpha - beta)
        const double ar = alpha.x - beta, ai = alpha.y, den = ar * ar + ai * ai;
        sc = make_double2(ar / den, -ai / den);
      }
      s_tau = t;
      s_scale = sc;
      e[k] = beta;
      d[k] = A[(size_t)k * n + k].x;
      tau[k] = t;
    }
    __syncthreads();
    const double2 tk = s_tau, sc = s_scale;
    if (tk.x == 0.0 && tk.y == 0.0) {
      if (tid == 0) col[0] = make_double2(1.0, 0.0);
      __syncthreads();
      continue;
    }
    for (int i = tid + 1; i < L; i += kHeevThreads) col[(size_t)i * n] = cmul(col[(size_t)i * n], sc);
    if (tid == 0) col[0] = make_double2(1.0, 0.0);
    __syncthreads();
    // p = tau * A22 v  (warp per row)
    for (int i = warp; i < L; i += kHeevWarps) {
      const double2* row = A + (size_t)(k + 1 + i) * n + (k + 1);
      double sr = 0, si = 0;
      for (int j = lane; j < L; j += 32) {
        const double2 a = row[j], v = col[(size_t)j * n];
        sr += a.x * v.x - a.y * v.y;
        si += a.x * v.y + a.y * v.x;
      }
      sr = warp_sum(sr);
      si = warp_sum(si);
      if (lane == 0) p[i] = cmul(tk, make_double2(sr, si));
    }
    __syncthreads();
    // alpha2 = -1/2 tau (p^H v)
    double dr = 0, di = 0;
    for (int i = tid; i < L; i += kHeevThreads) {
      const double2 pp = p[i], v = col[(size_t)i * n];
      dr += pp.x * v.x + pp.y * v.y;
      di += pp.x * v.y - pp.y * v.x;
    }
    dr = block_sum_heev(dr, red);
    di = block_sum_heev(di, red);
    const double2 al = cmul(make_double2(-0.5 * tk.x, -0.5 * tk.y), make_double2(dr, di));
    for (int i = tid; i < L; i += kHeevThreads) {
      const double2 v = col[(size_t)i * n];
      p[i] = cadd(p[i], cmul(al, v));
    }
    __syncthreads();
    // A22 -= v w^H + w v^H
    for (int idx = tid; idx < L * L; idx += kHeevThreads) {
      const int i = idx / L, j = idx - i * L;
      const double2 vi = col[(size_t)i * n], vj = col[(size_t)j * n], wi = p[i], wj = p[j];
      double2& a = A[(size_t)(k + 1 + i) * n + (k + 1 + j)];
      // v_i conj(w_j) + w_i conj(v_j)
      a.x -= (vi.x * wj.x + vi.y * wj.y) + (wi.x * vj.x + wi.y * vj.y);
      a.y -= (vi.y * wj.x - vi.x * wj.y) + (wi.y * vj.x - wi.x * vj.y);
    }
    __syncthreads();
  }
  if (tid == 0) {
    d[n - 1] = A[(size_t)(n - 1) * n + (n - 1)].x;
    e[n - 1] = 0.0;
    double tn = 0, lo = 1e300, hi = -1e300;
    for (int j = 0; j < n; ++j) {
      const double r = fabs(e[j]) + (j > 0 ? fabs(e[j - 1]) : 0.0);
      tn = fmax(tn, fabs(d[j]) + r);
      lo = fmin(lo, d[j] - r);
      hi = fmax(hi, d[j] + r);
    }
    s_tnorm = tn;
    s_lo = lo;
    s_hi = hi;
  }
  __syncthreads();
  const double tnorm = fmax(s_tnorm, 1e-300);
  double emax2 = 0;
  for (int j = 0; j < n - 1; ++j) emax2 = fmax(emax2, e[j] * e[j]);
  const double pivmin = fmax(1e-300, 2.2e-308 * fmax(1.0, emax2));

  // ---- 2. eigenvalues by bisection ----
  for (int i = tid; i < n; i += kHeevThreads) {
    double lo = s_lo - 1e-12 * tnorm - 1e-300, hi = s_hi + 1e-12 * tnorm + 1e-300;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (hi - lo <= 2.2e-16 * fmax(fabs(lo), fabs(hi)) + 1e-300) break;
      if (sturm_count(d, e, n, mid, pivmin) > i) hi = mid;
      else lo = mid;
    }
    w[i] = 0.5 * (lo + hi);
  }
  __syncthreads();

  // ---- 3. eigenvectors of T by inverse iteration ----
  if (tid == 0) {
    int nc = 0;
    for (int i = 0; i < nvec; ++i)
      if (i == 0 || w[i] - w[i - 1] > 1e-3 * tnorm) s_cl_start[nc++] = i;
    s_cl_start[nc] = nvec;
    s_ncl = nc;
  }
  __syncthreads();
  const double tiny = 2.2e-16 * tnorm;
  for (int c = warp; c < s_ncl; c += kHeevWarps) {
    double* wk = lu + (size_t)warp * 6 * n;
    for (int i = s_cl_start[c]; i < s_cl_start[c + 1]; ++i) {
      double* z = Z + (size_t)i * n;
      for (int j = lane; j < n; j += 32) z[j] = start_value(i, j);
      __syncwarp();
      for (int it = 0; it < 3; ++it) {
        if (lane == 0) tridiag_solve(d, e, n, w[i], tiny, z, wk);
        __syncwarp();
        // orthogonalise against the earlier vectors of the cluster, then normalise
        for (int q = s_cl_start[c]; q < i; ++q) {
          const double* zq = Z + (size_t)q * n;
          double s = 0;
          for (int j = lane; j < n; j += 32) s += zq[j] * z[j];
          s = warp_sum(s);
          for (int j = lane; j < n; j += 32) z[j] -= s * zq[j];
          __syncwarp();
        }
        double nn = 0;
        for (int j = lane; j < n; j += 32) nn += z[j] * z[j];
        nn = warp_sum(nn);
        const double inv = 1.0 / sqrt(fmax(nn, 1e-300));
        for (int j = lane; j < n; j += 32) z[j] *= inv;
        __syncwarp();
      }
    }
  }
  __syncthreads();

  // ---- 4. back-transformation v = H_0 ... H_{n-2} z ----
  for (int i = warp; i < nvec; i += kHeevWarps) {
    const double* z = Z + (size_t)i * n;
    // complex vector held in V column i
    for (int j = lane; j < n; j += 32) V[(size_t)j * n + i] = make_double2(z[j], 0.0);
    __syncwarp();
    for (int k = n - 2; k >= 0; --k) {
      const double2 tk = tau[k];
      if (tk.x == 0.0 && tk.y == 0.0) continue;
      const int L = n - k - 1;
      const double2* col = A + (size_t)(k + 1) * n + k;
      double sr = 0, si = 0;  // v^H z over rows k+1 ..
      for (int j = lane; j < L; j += 32) {
        const double2 v = col[(size_t)j * n], x = V[(size_t)(k + 1 + j) * n + i];
        sr += v.x * x.x + v.y * x.y;
        si += v.x * x.y - v.y * x.x;
      }
      sr = warp_sum(sr);
      si = warp_sum(si);
      const double2 f = cmul(tk, make_double2(sr, si));
      for (int j = lane; j < L; j += 32) {
        const double2 v = col[(size_t)j * n];
        double2& x = V[(size_t)(k + 1 + j) * n + i];
        x = csub(x, cmul(f, v));
      }
      __syncwarp();
    }
  }
  // zero the unused columns
  for (int idx = tid; idx < n * (n - nvec); idx += kHeevThreads) {
    const int r = idx / (n - nvec), j = nvec + idx % (n - nvec);
    V[(size_t)r * n + j] = make_double2(0, 0);
  }
}

size_t heev_work_doubles(int n, int nvec) {
  const size_t one_cta = (size_t)n * (2 + 4) + (size_t)nvec * n + (size_t)kHeevWarps * 6 * n + 64;
  return std::max(one_cta, heev_cluster_work_doubles(n, nvec));
}

// The cluster-distributed solver (dense.cu) when n fits it, else this one-CTA kernel.
void launch_heev(double2* A, int n, int nvec, double* w, double2* V, double* work, cudaStream_t st) {
  if (launch_heev_cluster(A, n, nvec, w, V, work, st)) return;
  count_launches(1);
  k_heev<<<1, kHeevThreads, 0, st>>>(A, n, nvec, w, V, work);
}

}  // namespace fde
