// dense.cu -- FP64 dense kernels of the Rayleigh-Ritz step (Eq. KS, block solver) spread over
// many SMs.  FP64 arithmetic on this part runs at a small fraction of the FP32 rate per SM, so
// the O(n^3) factorisations are distributed over a thread-block cluster of P CTAs that hold
// the matrix rows cyclically in shared memory (row i in CTA i % P) and synchronise with the
// hardware cluster barrier; the embarrassingly parallel phases run as ordinary launches.
//
//   k_cl_cholesky   S = L L^H (right-looking, 2 cluster barriers per column)
//   k_tri_inverse   L^{-1}, one warp per column
//   k_cl_tridiag    Householder reduction A = Q T Q^H (3 cluster barriers per column)
//   k_tri_eigvals   eigenvalues of T by 32-point multisection on Sturm counts (warp each)
//   k_tri_solve     inverse iteration, one thread per eigenvector
//   k_tri_orth      modified Gram-Schmidt inside clusters of close eigenvalues
//   k_backtransform v = H_0 ... H_{n-2} z, one warp per eigenvector
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>

#include "dense.h"
#include "prof.h"

namespace cg = cooperative_groups;

namespace fde {

constexpr int kClThreads = 256;
constexpr int kClWarps = kClThreads / 32;

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (all threads receive it); red holds kClWarps doubles.
__device__ __forceinline__ double block_sum_cl(double v, double* red) {
  v = warp_sum_d(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0;
  for (int k = 0; k < kClWarps; ++k) t += red[k];
  return t;
}

struct ClusterLayout {
  int P, rank, nloc, ld;
};

__device__ __forceinline__ ClusterLayout cluster_layout(int n) {
  ClusterLayout c;
  c.P = (int)cg::this_cluster().num_blocks();
  c.rank = (int)cg::this_cluster().block_rank();
  c.nloc = (n + c.P - 1) / c.P;
  c.ld = n;
  return c;
}

// ---- Cholesky --------------------------------------------------------------------------------
// Shared memory: rows [nloc][n] double2, col [n] double2, red.
__global__ void __launch_bounds__(kClThreads)
k_cl_cholesky(const double2* __restrict__ S, int n, double2* __restrict__ L, unsigned* status, double rel_pivot) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  const ClusterLayout c = cluster_layout(n);
  double2* rows = reinterpret_cast<double2*>(smem);
  double2* col = rows + (size_t)c.nloc * n;
  __shared__ double s_diag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int idx = tid; idx < c.nloc * n; idx += kClThreads) {
    const int li = idx / n, j = idx - li * n, i = li * c.P + c.rank;
    rows[idx] = (i < n && j <= i) ? S[(size_t)i * n + j] : make_double2(0, 0);
  }
  cl.sync();
  bool failed = false;
  for (int j = 0; j < n; ++j) {
    const int oj = j % c.P, lj = j / c.P;
    if (tid == 0) {
      const double2* rj = cl.map_shared_rank(rows, oj);
      s_diag = rj[(size_t)lj * n + j].x;
    }
    __syncthreads();
    const double d = s_diag;
    if (!(d > rel_pivot * S[(size_t)j * n + j].x)) {  // identical values in every CTA: a uniform exit
      failed = true;
      break;
    }
    const double sd = sqrt(d), inv = 1.0 / sd;
    // scale column j of the own rows below the diagonal
    for (int li = tid; li < c.nloc; li += kClThreads) {
      const int i = li * c.P + c.rank;
      if (i > j && i < n) {
        double2& v = rows[(size_t)li * n + j];
        v.x *= inv;
        v.y *= inv;
      }
    }
    cl.sync();
    if (c.rank == oj && tid == 0) rows[(size_t)lj * n + j] = make_double2(sd, 0.0);
    // gather column j (rows > j) and update the own rows: A[i][k] -= L[i][j] conj(L[k][j])
    for (int k = j + 1 + tid; k < n; k += kClThreads) {
      const double2* rk = cl.map_shared_rank(rows, k % c.P);
      col[k] = rk[(size_t)(k / c.P) * n + j];
    }
    __syncthreads();
    for (int li = warp; li < c.nloc; li += kClWarps) {
      const int i = li * c.P + c.rank;
      if (i <= j || i >= n) continue;
      const double2 a = rows[(size_t)li * n + j];
      double2* ri = rows + (size_t)li * n;
      for (int k = j + 1 + lane; k <= i; k += 32) {
        const double2 b = col[k];
        double2 v = ri[k];
        v.x -= a.x * b.x + a.y * b.y;
        v.y -= a.y * b.x - a.x * b.y;
        ri[k] = v;
      }
    }
    cl.sync();
  }
  if (failed) {
    if (c.rank == 0 && tid == 0) atomicOr(status, ST_CHOLESKY);
  } else {
    for (int idx = tid; idx < c.nloc * n; idx += kClThreads) {
      const int li = idx / n, j = idx - li * n, i = li * c.P + c.rank;
      if (i < n) L[(size_t)i * n + j] = (j <= i) ? rows[idx] : make_double2(0, 0);
    }
  }
  cl.sync();  // no CTA leaves while others may still read its shared memory
}

// ---- triangular inverse ------------------------------------------------------------------------
// Li = L^{-1} (lower); column c by forward substitution, one warp per column.
__global__ void k_tri_inverse(const double2* __restrict__ L, int n, double2* __restrict__ Li, const unsigned* status) {
  if (*status & ST_CHOLESKY) return;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= n) return;
  for (int i = lane; i < c; i += 32) Li[(size_t)i * n + c] = make_double2(0, 0);
  for (int i = c; i < n; ++i) {
    double re = 0.0, im = 0.0;
    const double2* li = L + (size_t)i * n;
    for (int k = c + lane; k < i; k += 32) {
      const double2 l = li[k], x = Li[(size_t)k * n + c];
      re += l.x * x.x - l.y * x.y;
      im += l.x * x.y + l.y * x.x;
    }
    re = warp_sum_d(re);
    im = warp_sum_d(im);
    if (lane == 0) {
      const double dd = li[i].x;
      Li[(size_t)i * n + c] = make_double2((((i == c) ? 1.0 : 0.0) - re) / dd, -im / dd);
    }
    __syncwarp();
  }
}

// ---- Householder tridiagonalisation ----------------------------------------------------------
// A (n x n Hermitian, full storage) -> d[n], e[n] (T = Q^H A Q real symmetric tridiagonal),
// tau[n] and the reflector vectors Vh[k][j] (j > k; Vh[k][k+1] = 1) with
// H_k = I - tau_k v_k v_k^H.
// Shared memory: rows [nloc][n], vfull [n], wfull [n], wown [nloc] (double2), pub (2 double2).
__global__ void __launch_bounds__(kClThreads)
k_cl_tridiag(const double2* __restrict__ A, int n, double* __restrict__ d, double* __restrict__ e,
             double2* __restrict__ tau, double2* __restrict__ Vh) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  const ClusterLayout c = cluster_layout(n);
  double2* rows = reinterpret_cast<double2*>(smem);
  double2* vfull = rows + (size_t)c.nloc * n;
  double2* wfull = vfull + n;
  double2* wown = wfull + n;
  double2* pub = wown + c.nloc;  // pub[0].x: partial |x|^2, pub[1]: partial p^H v
  __shared__ double red[kClWarps];
  __shared__ double2 s_tau, s_sc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int idx = tid; idx < c.nloc * n; idx += kClThreads) {
    const int li = idx / n, j = idx - li * n, i = li * c.P + c.rank;
    rows[idx] = (i < n) ? A[(size_t)i * n + j] : make_double2(0, 0);
  }
  __syncthreads();
  for (int k = 0; k < n - 1; ++k) {
    // (1) partial |x|^2 of the column below the subdiagonal
    double acc = 0;
    for (int li = tid; li < c.nloc; li += kClThreads) {
      const int i = li * c.P + c.rank;
      if (i >= k + 2 && i < n) {
        const double2 x = rows[(size_t)li * n + k];
        acc += x.x * x.x + x.y * x.y;
      }
    }
    acc = block_sum_cl(acc, red);
    if (tid == 0) pub[0] = make_double2(acc, 0.0);
    cl.sync();
    // (2) reflector (every CTA computes the same one)
    if (tid == 0) {
      double xn2 = 0;
      for (int r = 0; r < c.P; ++r) xn2 += cl.map_shared_rank(pub, r)[0].x;
      const double2 alpha = cl.map_shared_rank(rows, (k + 1) % c.P)[(size_t)((k + 1) / c.P) * n + k];
      double2 t = make_double2(0, 0), sc = make_double2(0, 0);
      double beta = alpha.x;
      if (!(xn2 == 0.0 && alpha.y == 0.0)) {
        beta = -copysign(sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2), alpha.x);
        t = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
        const double ar = alpha.x - beta, ai = alpha.y, den = ar * ar + ai * ai;
        sc = make_double2(ar / den, -ai / den);
      }
      s_tau = t;
      s_sc = sc;
      if (c.rank == 0) {
        e[k] = beta;
        tau[k] = t;
      }
      if (c.rank == k % c.P) d[k] = rows[(size_t)(k / c.P) * n + k].x;
    }
    __syncthreads();
    const double2 tk = s_tau, sc = s_sc;
    const bool skip = (tk.x == 0.0 && tk.y == 0.0);  // uniform over the cluster
    for (int j = k + 1 + tid; j < n; j += kClThreads) {
      double2 v;
      if (j == k + 1) {
        v = make_double2(1.0, 0.0);
      } else if (skip) {
        v = make_double2(0.0, 0.0);
      } else {
        v = cmul(cl.map_shared_rank(rows, j % c.P)[(size_t)(j / c.P) * n + k], sc);
      }
      vfull[j] = v;
      if (c.rank == 0) Vh[(size_t)k * n + j] = v;
    }
    __syncthreads();
    if (skip) {
      cl.sync();
      cl.sync();
      continue;
    }
    // p_i = tau (A22 v)_i for the own trailing rows (warp per row); partial p^H v
    double dr = 0, di = 0;
    for (int li = warp; li < c.nloc; li += kClWarps) {
      const int i = li * c.P + c.rank;
      if (i <= k || i >= n) continue;
      const double2* ri = rows + (size_t)li * n;
      double sr = 0, si = 0;
      for (int j = k + 1 + lane; j < n; j += 32) {
        const double2 a = ri[j], v = vfull[j];
        sr += a.x * v.x - a.y * v.y;
        si += a.x * v.y + a.y * v.x;
      }
      sr = warp_sum_d(sr);
      si = warp_sum_d(si);
      const double2 p = cmul(tk, make_double2(sr, si));
      if (lane == 0) {
        wown[li] = p;
        const double2 v = vfull[i];
        dr += p.x * v.x + p.y * v.y;
        di += p.x * v.y - p.y * v.x;
      }
    }
    dr = block_sum_cl(dr, red);
    di = block_sum_cl(di, red);
    if (tid == 0) pub[1] = make_double2(dr, di);
    cl.sync();
    // (3) w = p + alpha2 v with alpha2 = -tau (p^H v) / 2
    if (tid == 0) {
      double tr = 0, ti = 0;
      for (int r = 0; r < c.P; ++r) {
        const double2 q = cl.map_shared_rank(pub, r)[1];
        tr += q.x;
        ti += q.y;
      }
      red[0] = tr;
      red[1] = ti;
    }
    __syncthreads();
    const double2 al = cmul(make_double2(-0.5 * tk.x, -0.5 * tk.y), make_double2(red[0], red[1]));
    for (int li = tid; li < c.nloc; li += kClThreads) {
      const int i = li * c.P + c.rank;
      if (i > k && i < n) wown[li] = cadd(wown[li], cmul(al, vfull[i]));
    }
    cl.sync();
    // (4) full w, then A22 -= v w^H + w v^H on the own rows
    for (int j = k + 1 + tid; j < n; j += kClThreads) wfull[j] = cl.map_shared_rank(wown, j % c.P)[j / c.P];
    __syncthreads();
    for (int li = warp; li < c.nloc; li += kClWarps) {
      const int i = li * c.P + c.rank;
      if (i <= k || i >= n) continue;
      const double2 vi = vfull[i], wi = wfull[i];
      double2* ri = rows + (size_t)li * n;
      for (int j = k + 1 + lane; j < n; j += 32) {
        const double2 vj = vfull[j], wj = wfull[j];
        double2 a = ri[j];
        a.x -= (vi.x * wj.x + vi.y * wj.y) + (wi.x * vj.x + wi.y * vj.y);
        a.y -= (vi.y * wj.x - vi.x * wj.y) + (wi.y * vj.x - wi.x * vj.y);
        ri[j] = a;
      }
    }
    __syncthreads();
  }
  if (tid == 0 && c.rank == (n - 1) % c.P) d[n - 1] = rows[(size_t)((n - 1) / c.P) * n + (n - 1)].x;
  if (tid == 0 && c.rank == 0) {
    e[n - 1] = 0.0;
    tau[n - 1] = make_double2(0, 0);
  }
  cl.sync();
}

// ---- eigenvalues of T -------------------------------------------------------------------------
__device__ __forceinline__ int sturm_count_s(const double* d, const double* e, int n, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int j = 1; j < n; ++j) {
    q = d[j] - x - e[j - 1] * e[j - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// Gershgorin interval and scale of T; pivmin for the Sturm recurrences.
struct TriBounds {
  double lo, hi, tnorm, pivmin;
};
__device__ TriBounds tri_bounds(const double* d, const double* e, int n) {
  TriBounds b;
  double tn = 0, lo = 1e300, hi = -1e300, emax2 = 0;
  for (int j = 0; j < n; ++j) {
    const double r = (j < n - 1 ? fabs(e[j]) : 0.0) + (j > 0 ? fabs(e[j - 1]) : 0.0);
    tn = fmax(tn, fabs(d[j]) + r);
    lo = fmin(lo, d[j] - r);
    hi = fmax(hi, d[j] + r);
    if (j < n - 1) emax2 = fmax(emax2, e[j] * e[j]);
  }
  b.tnorm = fmax(tn, 1e-300);
  b.lo = lo - 1e-12 * b.tnorm - 1e-300;
  b.hi = hi + 1e-12 * b.tnorm + 1e-300;
  b.pivmin = fmax(1e-300, 2.2e-308 * fmax(1.0, emax2));
  return b;
}

// w[i] = i-th smallest eigenvalue; one warp per i, 32 Sturm counts per step (the interval
// shrinks 33-fold per step).
__global__ void k_tri_eigvals(const double* __restrict__ dg, const double* __restrict__ eg, int n, double* w) {
  extern __shared__ double sde[];
  double* d = sde;
  double* e = sde + n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    d[j] = dg[j];
    e[j] = eg[j];
  }
  __syncthreads();
  const TriBounds b = tri_bounds(d, e, n);
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  double lo = b.lo, hi = b.hi;
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= 2.2e-16 * fmax(fabs(lo), fabs(hi)) + 1e-300) break;
    const double step = (hi - lo) / 33.0;
    const double x = lo + step * (double)(lane + 1);
    const bool above = sturm_count_s(d, e, n, x, b.pivmin) > i;
    const unsigned m = __ballot_sync(0xffffffffu, above);
    double nlo, nhi;
    if (m == 0) {
      nlo = __shfl_sync(0xffffffffu, x, 31);
      nhi = hi;
    } else {
      const int f = __ffs(m) - 1;
      nhi = __shfl_sync(0xffffffffu, x, f);
      const double xl = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
      nlo = (f > 0) ? xl : lo;
    }
    if (!(nlo > lo || nhi < hi)) break;  // no representable progress
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) w[i] = 0.5 * (lo + hi);
}

// ---- eigenvectors of T by inverse iteration -----------------------------------------------
__device__ __forceinline__ double start_value_s(int i, int j) {
  unsigned h = (unsigned)(i * 2654435761u) ^ (unsigned)(j * 40503u + 0x9e3779b9u);
  h ^= h >> 15;
  h *= 2246822519u;
  h ^= h >> 13;
  return 0.5 + (double)(h & 0xffff) / 65536.0;
}

// Inverse iteration for vectors i < nvec: `iters` solves of (T - w_i I) z_new = z with the
// partially pivoted LU of T - w_i I (factorised once), normalising after each; starts from
// the current Z (fresh = 0) or a fixed pseudo-random vector (fresh = 1).  Z[i][n] (row per
// vector); work: 5 n nvec doubles, interleaved by vector so that the threads of a warp touch
// consecutive addresses.
__global__ void k_tri_solve(const double* __restrict__ d, const double* __restrict__ e, int n, const double* w,
                            int nvec, int fresh, int iters, double* __restrict__ Z, double* __restrict__ work) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvec) return;
  double tn = 0;
  for (int j = 0; j < n; ++j) {
    const double r = (j < n - 1 ? fabs(e[j]) : 0.0) + (j > 0 ? fabs(e[j - 1]) : 0.0);
    tn = fmax(tn, fabs(d[j]) + r);
  }
  const double tiny = 2.2e-16 * fmax(tn, 1e-300);
  const double lam = w[i];
  double* z = Z + (size_t)i * n;
  const size_t nv = (size_t)nvec;
  double* wa = work;                 // pivots
  double* wu1 = work + n * nv;       // first superdiagonal
  double* wu2 = work + 2 * n * nv;   // second superdiagonal (fill-in)
  double* wl = work + 3 * n * nv;    // multipliers
  double* wp = work + 4 * n * nv;    // 1 where rows j and j+1 were interchanged
  if (fresh)
    for (int j = 0; j < n; ++j) z[j] = start_value_s(i, j);
  {
    double a = d[0] - lam, u1 = (n > 1) ? e[0] : 0.0;
    for (int j = 0; j < n - 1; ++j) {
      const double sub = e[j], dn = d[j + 1] - lam, en = (j + 1 < n - 1) ? e[j + 1] : 0.0;
      if (fabs(a) >= fabs(sub)) {
        const double m = sub / ((a == 0.0) ? tiny : a);
        wa[j * nv + i] = a;
        wu1[j * nv + i] = u1;
        wu2[j * nv + i] = 0.0;
        wl[j * nv + i] = m;
        wp[j * nv + i] = 0.0;
        a = dn - m * u1;
        u1 = en;
      } else {
        const double m = a / sub;
        wa[j * nv + i] = sub;
        wu1[j * nv + i] = dn;
        wu2[j * nv + i] = en;
        wl[j * nv + i] = m;
        wp[j * nv + i] = 1.0;
        a = u1 - m * dn;
        u1 = -m * en;
      }
    }
    wa[(size_t)(n - 1) * nv + i] = a;
    wu1[(size_t)(n - 1) * nv + i] = 0.0;
    wu2[(size_t)(n - 1) * nv + i] = 0.0;
  }
  for (int it = 0; it < iters; ++it) {
    // forward: apply the row operations
    for (int j = 0; j < n - 1; ++j) {
      const double m = wl[j * nv + i];
      if (wp[j * nv + i] != 0.0) {
        const double t = z[j];
        z[j] = z[j + 1];
        z[j + 1] = t - m * z[j];
      } else {
        z[j + 1] -= m * z[j];
      }
    }
    // back substitution
    double b1 = 0.0, b2 = 0.0, nn = 0.0;
    for (int j = n - 1; j >= 0; --j) {
      const double aj = wa[j * nv + i];
      const double x = (z[j] - wu1[j * nv + i] * b1 - wu2[j * nv + i] * b2) / ((aj == 0.0) ? tiny : aj);
      z[j] = x;
      b2 = b1;
      b1 = x;
      nn += x * x;
    }
    const double inv = 1.0 / sqrt(fmax(nn, 1e-300));
    for (int j = 0; j < n; ++j) z[j] *= inv;
  }
}

// Modified Gram-Schmidt inside each cluster of eigenvalues closer than gap_rel * ||T||
// (one CTA per cluster; CTAs beyond the number of clusters return).  Z[i][n].
__global__ void k_tri_orth(const double* __restrict__ d, const double* __restrict__ e, int n, const double* w,
                           int nvec, double gap_rel, double* __restrict__ Z) {
  __shared__ double red[32];
  __shared__ int s_lo, s_hi;
  if (threadIdx.x == 0) {
    double tn = 0;
    for (int j = 0; j < n; ++j) {
      const double r = (j < n - 1 ? fabs(e[j]) : 0.0) + (j > 0 ? fabs(e[j - 1]) : 0.0);
      tn = fmax(tn, fabs(d[j]) + r);
    }
    const double gap = gap_rel * fmax(tn, 1e-300);
    int c = -1, lo = 0, hi = 0;
    for (int q = 0; q < nvec; ++q) {
      if (q == 0 || w[q] - w[q - 1] > gap) {
        ++c;
        if (c == (int)blockIdx.x) lo = q;
        if (c == (int)blockIdx.x + 1) break;
      }
      if (c == (int)blockIdx.x) hi = q + 1;
    }
    s_lo = lo;
    s_hi = (c >= (int)blockIdx.x) ? hi : lo;
  }
  __syncthreads();
  const int lo = s_lo, hi = s_hi;
  if (hi - lo < 2) return;  // a single vector is already normalised
  const int nw = blockDim.x >> 5, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = lo; q < hi; ++q) {
    double* zq = Z + (size_t)q * n;
    double acc = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) acc += zq[j] * zq[j];
    acc = warp_sum_d(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    double t = 0;
    for (int k = 0; k < nw; ++k) t += red[k];
    const double inv = 1.0 / sqrt(fmax(t, 1e-300));
    for (int j = threadIdx.x; j < n; j += blockDim.x) zq[j] *= inv;
    __syncthreads();
    for (int r = q + 1 + warp; r < hi; r += nw) {
      double* zr = Z + (size_t)r * n;
      double s = 0;
      for (int j = lane; j < n; j += 32) s += zq[j] * zr[j];
      s = warp_sum_d(s);
      for (int j = lane; j < n; j += 32) zr[j] -= s * zq[j];
    }
    __syncthreads();
  }
}

// V[:, i] = H_0 H_1 ... H_{n-2} z_i (column i of the row-major n x n V; one warp per vector);
// columns nvec..n-1 of V are zeroed.
__global__ void k_backtransform(const double2* __restrict__ Vh, const double2* __restrict__ tau, int n, int nvec,
                                const double* __restrict__ Z, double2* __restrict__ V) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  if (i >= nvec) {
    for (int r = lane; r < n; r += 32) V[(size_t)r * n + i] = make_double2(0, 0);
    return;
  }
  const double* z = Z + (size_t)i * n;
  for (int r = lane; r < n; r += 32) V[(size_t)r * n + i] = make_double2(z[r], 0.0);
  __syncwarp();
  for (int k = n - 2; k >= 0; --k) {
    const double2 tk = tau[k];
    if (tk.x == 0.0 && tk.y == 0.0) continue;
    const double2* v = Vh + (size_t)k * n;
    double sr = 0, si = 0;  // v^H x over rows k+1 ..
    for (int j = k + 1 + lane; j < n; j += 32) {
      const double2 a = v[j], x = V[(size_t)j * n + i];
      sr += a.x * x.x + a.y * x.y;
      si += a.x * x.y - a.y * x.x;
    }
    sr = warp_sum_d(sr);
    si = warp_sum_d(si);
    const double2 f = cmul(tk, make_double2(sr, si));
    for (int j = k + 1 + lane; j < n; j += 32) {
      const double2 a = v[j];
      double2& x = V[(size_t)j * n + i];
      x = csub(x, cmul(f, a));
    }
    __syncwarp();
  }
}

// ---- host side -----------------------------------------------------------------------------
static int g_cluster_p = -1;  // CTAs per cluster (16, else 8; 0: clusters unusable)

static size_t tridiag_smem(int n, int P) {
  const int nloc = (n + P - 1) / P;
  return ((size_t)nloc * n + 2 * (size_t)n + nloc + 2) * sizeof(double2);
}
static size_t chol_smem(int n, int P) {
  const int nloc = (n + P - 1) / P;
  return ((size_t)nloc * n + n) * sizeof(double2);
}

static int cluster_size() {
  if (g_cluster_p >= 0) return g_cluster_p;
  int dev = 0;
  cudaGetDevice(&dev);
  int cc = 0;
  cudaDeviceGetAttribute(&cc, cudaDevAttrComputeCapabilityMajor, dev);
  g_cluster_p = 0;
  if (cc < 9) return g_cluster_p;
  const size_t smax = 200 * 1024;
  for (int P : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smax;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = P;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    bool ok = true;
    for (const void* f : {(const void*)k_cl_tridiag, (const void*)k_cl_cholesky}) {
      if (P > 8 && cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) ok = false;
      if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax) != cudaSuccess) ok = false;
      int ncl = 0;
      if (ok && (cudaOccupancyMaxActiveClusters(&ncl, f, &cfg) != cudaSuccess || ncl < 1)) ok = false;
    }
    cudaGetLastError();
    if (ok) {
      g_cluster_p = P;
      break;
    }
  }
  return g_cluster_p;
}

int dense_cluster_max_n() {
  static int nmax = -1;
  if (nmax >= 0) return nmax;
  const int P = cluster_size();
  int n = 0;
  if (P > 0)
    while (tridiag_smem(n + 1, P) <= 200 * 1024 && chol_smem(n + 1, P) <= 200 * 1024) ++n;
  nmax = n;
  return nmax;
}

static cudaLaunchConfig_t cluster_cfg(int P, size_t smem, cudaStream_t st, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P);
  cfg.blockDim = dim3(kClThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = P;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

bool launch_cholesky_cluster(const double2* S, int n, double2* L, double2* Li, unsigned* status, double rel_pivot,
                             cudaStream_t st) {
  if (n < 1 || n > dense_cluster_max_n()) return false;
  const int P = cluster_size();
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = cluster_cfg(P, chol_smem(n, P), st, at);
  count_launches(2);
  if (cudaLaunchKernelEx(&cfg, k_cl_cholesky, S, n, L, status, rel_pivot) != cudaSuccess) return false;
  const int wpb = 4;
  k_tri_inverse<<<(n + wpb - 1) / wpb, 32 * wpb, 0, st>>>(L, n, Li, status);
  return true;
}

size_t heev_cluster_work_doubles(int n, int nvec) {
  // d, e, w copies | tau (2n) | Vh (2 n^2) | Z (nvec n) | solve work (5 n nvec)
  return (size_t)2 * n + 2 * (size_t)n + 2 * (size_t)n * n + (size_t)nvec * n + 5 * (size_t)n * nvec + 64;
}

bool launch_heev_cluster(const double2* A, int n, int nvec, double* w, double2* V, double* work, cudaStream_t st) {
  if (n < 2 || n > dense_cluster_max_n() || nvec < 1 || nvec > n) return false;
  const int P = cluster_size();
  double* d = work;
  double* e = d + n;
  double2* tau = reinterpret_cast<double2*>(e + n);
  double2* Vh = tau + n;
  double* Z = reinterpret_cast<double*>(Vh + (size_t)n * n);
  double* sw = Z + (size_t)nvec * n;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = cluster_cfg(P, tridiag_smem(n, P), st, at);
  count_launches(1);
  if (cudaLaunchKernelEx(&cfg, k_cl_tridiag, A, n, d, e, tau, Vh) != cudaSuccess) return false;
  const int wpb = 4;
  count_launches(7);
  k_tri_eigvals<<<(n + wpb - 1) / wpb, 32 * wpb, 2 * n * sizeof(double), st>>>(d, e, n, w);
  const int tpb = 64;
  // Two rounds of (inverse iteration, Gram-Schmidt inside clusters of close eigenvalues).
  const double gap_rel = 1e-3;
  k_tri_solve<<<(nvec + tpb - 1) / tpb, tpb, 0, st>>>(d, e, n, w, nvec, 1, 2, Z, sw);
  k_tri_orth<<<nvec, 128, 0, st>>>(d, e, n, w, nvec, gap_rel, Z);
  k_tri_solve<<<(nvec + tpb - 1) / tpb, tpb, 0, st>>>(d, e, n, w, nvec, 0, 1, Z, sw);
  k_tri_orth<<<nvec, 128, 0, st>>>(d, e, n, w, nvec, gap_rel, Z);
  k_backtransform<<<n, 32, 0, st>>>(Vh, tau, n, nvec, Z, V);
  return true;
}

}  // namespace fde
