// hpsi_static.cu -- the local part of H psi for callers that cannot allocate device memory.
//
// Some callers run where cudaMalloc is not available to them: code inside another
// framework's memory pool or allocator hooks, an embedding host that owns every device
// allocation, or a library entry point that must not grow the process's device footprint
// at call time.  For them, fde_apply_h_local_static takes every input as a caller buffer,
// builds nothing with cudaMalloc and keeps its working memory in the fixed-size device
// arrays below, which every GPU that loads the library holds until the process exits.
//
// Set-up: the first call on a device (with that device current) resolves the device
// addresses of these arrays with cudaGetSymbolAddress and caches them per device, so that
// first call must come before any stream capture.  All calls share the arrays and they keep
// the previous call's contents (every value a call reads is written by that call first);
// calls that overlap on the GPU -- from two streams, or two host threads -- race on them.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "fde.h"
#include "kernels.h"
#include "prof.h"

namespace fde {

// Capacities of the static working memory (about 26 MB per device in total).
constexpr int kStMaxNpw = 65536;        // plane waves of one sphere
constexpr int kStMaxCols = 8192;        // (m1, m2) columns of one sphere
constexpr long long kStMaxGrid = 1 << 20;  // grid points n1 n2 n3
constexpr long long kStScratch = 1 << 20;  // complex values of the column scratch

static __device__ __align__(256) double2 st_scratch[kStScratch];
static __device__ __align__(256) double st_vplane[kStMaxGrid];
static __device__ __align__(256) double st_kin[kStMaxNpw];
static __device__ __align__(256) int st_cols[4 * kStMaxCols + 1 + kMaxPlane];
static __device__ __align__(256) int st_ncols[2];
static __device__ __align__(256) double2 st_tw[3][kMaxLine];

struct StaticPtrs {
  double2* scratch;
  double* vplane;
  double* kin;
  int* cols;
  int* ncols;
  double2* tw;
};

static std::mutex st_mutex;
static StaticPtrs st_ptrs[64];
static bool st_ready[64];

static fde_status static_setup(int dev, StaticPtrs* out) {
  std::lock_guard<std::mutex> lock(st_mutex);
  if (dev < 0 || dev >= 64) return FDE_EUNSUPPORTED;
  if (!st_ready[dev]) {
    StaticPtrs p;
    if (cudaGetSymbolAddress((void**)&p.scratch, st_scratch) != cudaSuccess) return FDE_ECUDA;
    if (cudaGetSymbolAddress((void**)&p.vplane, st_vplane) != cudaSuccess) return FDE_ECUDA;
    if (cudaGetSymbolAddress((void**)&p.kin, st_kin) != cudaSuccess) return FDE_ECUDA;
    if (cudaGetSymbolAddress((void**)&p.cols, st_cols) != cudaSuccess) return FDE_ECUDA;
    if (cudaGetSymbolAddress((void**)&p.ncols, st_ncols) != cudaSuccess) return FDE_ECUDA;
    if (cudaGetSymbolAddress((void**)&p.tw, st_tw) != cudaSuccess) return FDE_ECUDA;
    st_ptrs[dev] = p;
    st_ready[dev] = true;
  }
  *out = st_ptrs[dev];
  return FDE_OK;
}

// Column map of a sphere (one CTA): cols = [start(ncol+1) | m3lo | i1 | i2 | rows];
// ncols = {ncol, nrow}.  A column starts where (m1, m2) changes; rows are the distinct i1.
// The caller's list is checked on the way, because the transforms index shared-memory lines
// by it: (m1, m2) keys strictly increasing from column to column (sorted, no repeats), m3
// contiguous inside a column, every m3 in [-n3, n3), every column at most n3 long, and the
// m1 and m2 spans at most n1 and n2 (so no two columns land on one (i1, i2) slot of a
// plane).  A list that breaks any of these gives ncols = {0, -2}; more than kStMaxCols
// columns gives {ncol, -1}.
__global__ void __launch_bounds__(1024)
k_static_columns(const int* __restrict__ mil, int npw, int n1, int n2, int n3, int* cols, int* ncols) {
  __shared__ int warp_sums[32];
  __shared__ int base, bad;
  __shared__ int lo1, hi1, lo2, hi2;
  __shared__ int rowflag[kMaxPlane];
  if (threadIdx.x == 0) {
    base = 0;
    bad = 0;
    lo1 = lo2 = 1 << 30;
    hi1 = hi2 = -(1 << 30);
  }
  for (int i = threadIdx.x; i < kMaxPlane; i += blockDim.x) rowflag[i] = 0;
  __syncthreads();
  // pass 1: validate every point and count columns (block-wide scan over chunks of points)
  int* start = cols;
  int mylo1 = 1 << 30, myhi1 = -(1 << 30), mylo2 = 1 << 30, myhi2 = -(1 << 30), mybad = 0;
  for (int c0 = 0; c0 < npw; c0 += blockDim.x) {
    const int p = c0 + threadIdx.x;
    int f = 0;
    if (p < npw) {
      const int m1 = mil[3 * p], m2 = mil[3 * p + 1], m3 = mil[3 * p + 2];
      mylo1 = min(mylo1, m1);
      myhi1 = max(myhi1, m1);
      mylo2 = min(mylo2, m2);
      myhi2 = max(myhi2, m2);
      if (m3 < -n3 || m3 >= n3) mybad = 1;
      if (p == 0) {
        f = 1;
      } else {
        const int q1 = mil[3 * (p - 1)], q2 = mil[3 * (p - 1) + 1], q3 = mil[3 * (p - 1) + 2];
        f = (m1 != q1) || (m2 != q2);
        if (f && (m1 < q1 || (m1 == q1 && m2 < q2))) mybad = 1;  // keys must increase
        if (!f && m3 != q3 + 1) mybad = 1;                      // m3 contiguous in a column
      }
    }
    int x = f;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
      int s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;
    }
    __syncthreads();
    const int incl = x + (w > 0 ? warp_sums[w - 1] : 0);
    if (f) {
      const int c = base + incl - 1;
      if (c < kStMaxCols) start[c] = p;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) base += incl;
    __syncthreads();
  }
  atomicMin(&lo1, mylo1);
  atomicMax(&hi1, myhi1);
  atomicMin(&lo2, mylo2);
  atomicMax(&hi2, myhi2);
  if (mybad) atomicOr(&bad, 1);
  __syncthreads();
  const int ncol = base;
  if (ncol > kStMaxCols) {
    if (threadIdx.x == 0) { ncols[0] = ncol; ncols[1] = -1; }
    return;
  }
  if (threadIdx.x == 0) start[ncol] = npw;
  __syncthreads();
  for (int c = threadIdx.x; c < ncol; c += blockDim.x)
    if (start[c + 1] - start[c] > n3) atomicOr(&bad, 1);
  __syncthreads();
  if (bad || hi1 - lo1 + 1 > n1 || hi2 - lo2 + 1 > n2) {
    if (threadIdx.x == 0) { ncols[0] = 0; ncols[1] = -2; }
    return;
  }
  int* m3lo = cols + ncol + 1;
  int* ci1 = m3lo + ncol;
  int* ci2 = ci1 + ncol;
  int* rows = ci2 + ncol;
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
    const int p = start[c];
    const int m1 = mil[3 * p], m2 = mil[3 * p + 1];
    m3lo[c] = mil[3 * p + 2];
    const int i1 = ((m1 % n1) + n1) % n1;
    ci1[c] = i1;
    ci2[c] = ((m2 % n2) + n2) % n2;
    rowflag[i1] = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int r = 0;
    for (int i = 0; i < n1; ++i)
      if (rowflag[i]) rows[r++] = i;
    ncols[0] = ncol;
    ncols[1] = r;
  }
}

// Twiddles exp(-2 pi i m / n) of the three axes, kinetic energies and the plane-major
// potential, all into the static arrays.
__global__ void k_static_tables(int n1, int n2, int n3, double2* tw) {
  const int ns[3] = {n1, n2, n3};
  for (int a = 0; a < 3; ++a)
    for (int m = threadIdx.x + blockIdx.x * blockDim.x; m < ns[a]; m += blockDim.x * gridDim.x) {
      double s, c;
      sincospi(2.0 * (double)m / (double)ns[a], &s, &c);
      tw[a * kMaxLine + m] = make_double2(c, -s);
    }
}

__global__ void k_static_kin(const int* __restrict__ mil, int npw, double b0, double b1, double b2, double k0,
                             double k1, double k2, double* kin) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npw; p += gridDim.x * blockDim.x) {
    const double qx = k0 + (double)mil[3 * p] * b0;
    const double qy = k1 + (double)mil[3 * p + 1] * b1;
    const double qz = k2 + (double)mil[3 * p + 2] * b2;
    kin[p] = 0.5 * (qx * qx + qy * qy + qz * qz);
  }
}

static void factor_line(int n, LinePlan<double>& p) {
  int m = n, k = 0;
  while (m % 4 == 0) { p.radix[k++] = 4; m /= 4; }
  while (m % 2 == 0) { p.radix[k++] = 2; m /= 2; }
  while (m % 3 == 0) { p.radix[k++] = 3; m /= 3; }
  while (m % 5 == 0) { p.radix[k++] = 5; m /= 5; }
  p.n = n;
  p.nstages = (m == 1) ? k : -1;
}

}  // namespace fde

extern "C" fde_status fde_apply_h_local_static(const fde_cell_desc* cell, const double* kfrac, int npw,
                                               const int* d_miller, const double* d_veff, const double* d_psi,
                                               double* d_hpsi, int nb, void* cuda_stream) {
  using namespace fde;
  if (!cell || !kfrac || !d_miller || !d_veff || !d_psi || !d_hpsi || npw <= 0 || nb <= 0) return FDE_EINVAL;
  const int n1 = cell->grid[0], n2 = cell->grid[1], n3 = cell->grid[2];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (i != j && cell->lattice[i][j] != 0.0) return FDE_EUNSUPPORTED;
  if (n1 < 2 || n2 < 2 || n3 < 2 || n1 > kMaxPlane || n2 > kMaxPlane || n3 > kMaxLine) return FDE_EUNSUPPORTED;
  const long long nr = (long long)n1 * n2 * n3;
  if (nr > kStMaxGrid || npw > kStMaxNpw) return FDE_EUNSUPPORTED;
  LinePlan<double> lp[3];
  factor_line(n1, lp[0]);
  factor_line(n2, lp[1]);
  factor_line(n3, lp[2]);
  if (lp[0].nstages < 0 || lp[1].nstages < 0 || lp[2].nstages < 0) return FDE_EUNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FDE_ECUDA;
  StaticPtrs P;
  const fde_status s = static_setup(dev, &P);
  if (s != FDE_OK) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  for (int a = 0; a < 3; ++a) lp[a].tw = P.tw + a * kMaxLine;
  const double b[3] = {2.0 * M_PI * (1.0 / cell->lattice[0][0]), 2.0 * M_PI * (1.0 / cell->lattice[1][1]),
                       2.0 * M_PI * (1.0 / cell->lattice[2][2])};
  k_static_columns<<<1, 1024, 0, st>>>(d_miller, npw, n1, n2, n3, P.cols, P.ncols);
  k_static_tables<<<1, 320, 0, st>>>(n1, n2, n3, P.tw);
  k_static_kin<<<ceil_div(npw, 256), 256, 0, st>>>(d_miller, npw, b[0], b[1], b[2], kfrac[0] * b[0],
                                                   kfrac[1] * b[1], kfrac[2] * b[2], P.kin);
  launch_transpose<double, double>(d_veff, P.vplane, n1 * n2, n3, 0, st);
  int hc[2] = {0, 0};
  if (cudaMemcpyAsync(hc, P.ncols, sizeof(hc), cudaMemcpyDeviceToHost, st) != cudaSuccess) return FDE_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FDE_ECUDA;
  const int ncol = hc[0], nrow = hc[1];
  if (nrow == -2) return FDE_EINVAL;  // the sphere list is unsorted or does not fit the grid
  if (nrow < 0 || ncol <= 0 || ncol > kStMaxCols) return FDE_EUNSUPPORTED;
  // the column scratch holds n3 x ncol complex values of at least one band
  if ((long long)n3 * ncol > kStScratch) return FDE_EUNSUPPORTED;
  SphereDev sp;
  sp.npw = npw;
  sp.ncol = ncol;
  sp.nrow = nrow;
  sp.col_start = P.cols;
  sp.col_m3lo = P.cols + ncol + 1;
  sp.col_i1 = sp.col_m3lo + ncol;
  sp.col_i2 = sp.col_i1 + ncol;
  sp.row_i1 = sp.col_i2 + ncol;
  FftPlans<double> fp;
  fp.p1 = lp[0];
  fp.p2 = lp[1];
  fp.p3 = lp[2];
  const GridDims g{n1, n2, n3};
  const long long per_band = (long long)n3 * ncol;
  const int chunk = (int)std::min<long long>(nb, kStScratch / per_band);
  for (int b0 = 0; b0 < nb; b0 += chunk) {
    const int nbc = std::min(chunk, nb - b0);
    launch_hpsi_local<double>((const double2*)d_psi + (size_t)b0 * npw, npw, (double2*)d_hpsi + (size_t)b0 * npw,
                              npw, nbc, P.kin, P.vplane, P.scratch, sp, g, fp, st);
  }
  if (cudaGetLastError() != cudaSuccess) return FDE_ECUDA;
  return FDE_OK;
}
