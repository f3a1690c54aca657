// hpsi.cu -- local part of the embedded Kohn-Sham apply (Eq. KS) and band densities.
//
// (H psi)_loc(G) = |k+G|^2/2 psi(G) + P_sphere FFT[ v_eff(r) . IFFT psi ](G)
//
// The 3D transforms are split so that only the z-lines that hold sphere points ("columns")
// are ever transformed along z, and the (x, y) planes are transformed whole in shared
// memory with the potential multiply fused between the inverse and forward 2D passes:
//
//   k_zinv     : gather each column's sphere run into a zero z-line, inverse FFT along z,
//                write scratch[b][i3][col]                 (reads psi, writes scratch)
//   k_plane    : per (band, i3): scatter the columns into the plane, inverse FFT along y
//                (rows holding columns only) and x, multiply by v_eff, forward FFT along x
//                and y, gather the columns back                (scratch -> scratch)
//   k_zfwd     : forward FFT along z, pick the sphere run, scale by 1/N_r and add the
//                kinetic term                                (scratch, psi -> hpsi)
//
// Only the sphere columns (a disk of the (x, y) plane) travel through global memory, so
// a band-apply moves about 4 x n3 x ncol complex values plus the potential plane instead
// of the 4 x N_r of a plain 3D transform pair.
#include "fft.cuh"
#include "kernels.h"
#include "prof.h"

namespace fde {

constexpr int kColsPerCta = 8;     // z-lines (one warp each) per CTA in the z passes
constexpr int kPlaneThreads = 256;  // threads of a plane CTA

template <typename T>
__global__ void __launch_bounds__(kColsPerCta * 32)
k_zinv(const cplx<T>* __restrict__ psi, int ldpsi, cplx<T>* __restrict__ scratch, SphereDev sp,
       int n3, LinePlan<T> pz) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* lines = reinterpret_cast<C*>(smem_raw);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = blockIdx.x * kColsPerCta, b = blockIdx.y;
  const int lp = n3 + 1;
  C* L = lines + w * lp;
  const int c = c0 + w;
  for (int i = lane; i < n3; i += 32) L[i] = mk<T>(0, 0);
  __syncwarp();
  if (c < sp.ncol) {
    const int s = sp.col_start[c], e = sp.col_start[c + 1], m3 = sp.col_m3lo[c];
    const C* src = psi + (size_t)b * ldpsi + s;
    for (int t = lane; t < e - s; t += 32) {
      int i3 = m3 + t;
      i3 += (i3 < 0) ? n3 : 0;
      L[i3] = src[t];
    }
    __syncwarp();
    fft_line<T>(L, 1, pz, lane, +1);
  }
  __syncthreads();
  const int nc = min(kColsPerCta, sp.ncol - c0);
  C* dst = scratch + (size_t)b * n3 * sp.ncol + c0;
  for (int idx = threadIdx.x; idx < n3 * kColsPerCta; idx += blockDim.x) {
    const int i3 = idx / kColsPerCta, ww = idx % kColsPerCta;
    if (ww < nc) dst[(size_t)i3 * sp.ncol + ww] = lines[ww * lp + i3];
  }
}

template <typename T>
__global__ void __launch_bounds__(kPlaneThreads)
k_plane(cplx<T>* __restrict__ scratch, SphereDev sp, const T* __restrict__ vplane, GridDims g,
        LinePlan<T> p1, LinePlan<T> p2) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* P = reinterpret_cast<C*>(smem_raw);
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3, pitch = n2 + 1;
  const int i3 = blockIdx.x, b = blockIdx.y;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  C* S = scratch + ((size_t)b * n3 + i3) * sp.ncol;
  for (int idx = threadIdx.x; idx < n1 * pitch; idx += blockDim.x) P[idx] = mk<T>(0, 0);
  __syncthreads();
  for (int c = threadIdx.x; c < sp.ncol; c += blockDim.x) P[sp.col_i1[c] * pitch + sp.col_i2[c]] = S[c];
  __syncthreads();
  for (int r = w; r < sp.nrow; r += nw) fft_line<T, kMaxPlane>(P +sp.row_i1[r] * pitch, 1, p2, lane, +1);
  __syncthreads();
  for (int i2 = w; i2 < n2; i2 += nw) fft_line<T, kMaxPlane>(P +i2, pitch, p1, lane, +1);
  __syncthreads();
  const T* V = vplane + (size_t)i3 * n1 * n2;
  for (int idx = threadIdx.x; idx < n1 * n2; idx += blockDim.x) {
    const int i1 = idx / n2, i2 = idx - i1 * n2;
    C& z = P[i1 * pitch + i2];
    const T v = V[idx];
    z.x *= v;
    z.y *= v;
  }
  __syncthreads();
  for (int i2 = w; i2 < n2; i2 += nw) fft_line<T, kMaxPlane>(P +i2, pitch, p1, lane, -1);
  __syncthreads();
  for (int r = w; r < sp.nrow; r += nw) fft_line<T, kMaxPlane>(P +sp.row_i1[r] * pitch, 1, p2, lane, -1);
  __syncthreads();
  for (int c = threadIdx.x; c < sp.ncol; c += blockDim.x) S[c] = P[sp.col_i1[c] * pitch + sp.col_i2[c]];
}

template <typename T>
__global__ void __launch_bounds__(kColsPerCta * 32)
k_zfwd(const cplx<T>* __restrict__ scratch, const cplx<T>* __restrict__ psi, int ldpsi,
       cplx<T>* __restrict__ hpsi, int ldh, const T* __restrict__ kin, SphereDev sp, int n3,
       T inv_nr, LinePlan<T> pz) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* lines = reinterpret_cast<C*>(smem_raw);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = blockIdx.x * kColsPerCta, b = blockIdx.y;
  const int lp = n3 + 1;
  const int nc = min(kColsPerCta, sp.ncol - c0);
  const C* src = scratch + (size_t)b * n3 * sp.ncol + c0;
  for (int idx = threadIdx.x; idx < n3 * kColsPerCta; idx += blockDim.x) {
    const int i3 = idx / kColsPerCta, ww = idx % kColsPerCta;
    lines[ww * lp + i3] = (ww < nc) ? src[(size_t)i3 * sp.ncol + ww] : mk<T>(0, 0);
  }
  __syncthreads();
  const int c = c0 + w;
  if (c >= sp.ncol) return;
  C* L = lines + w * lp;
  fft_line<T>(L, 1, pz, lane, -1);
  const int s = sp.col_start[c], e = sp.col_start[c + 1], m3 = sp.col_m3lo[c];
  const C* ps = psi + (size_t)b * ldpsi;
  C* hs = hpsi + (size_t)b * ldh;
  for (int t = lane; t < e - s; t += 32) {
    int i3 = m3 + t;
    i3 += (i3 < 0) ? n3 : 0;
    const int gidx = s + t;
    const C x = ps[gidx];
    const T kk = kin[gidx];
    C o = L[i3];
    o.x = o.x * inv_nr + kk * x.x;
    o.y = o.y * inv_nr + kk * x.y;
    hs[gidx] = o;
  }
}

template <typename T> static size_t zpass_smem(int n3) {
  return (size_t)kColsPerCta * (n3 + 1) * sizeof(cplx<T>);
}
template <typename T> static size_t plane_smem(const GridDims& g) {
  return (size_t)g.n1 * (g.n2 + 1) * sizeof(cplx<T>);
}

template <typename K> static void allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
void launch_hpsi_local(const cplx<T>* psi, int ldpsi, cplx<T>* hpsi, int ldh, int nb,
                       const T* kin, const T* vplane, cplx<T>* scratch, const SphereDev& sp,
                       const GridDims& g, const FftPlans<T>& fp, cudaStream_t st) {
  if (nb <= 0) return;
  if (launch_hpsi_local_ct<T>(psi, ldpsi, hpsi, ldh, nb, kin, vplane, scratch, sp, g, fp, st)) return;
  const dim3 gz(ceil_div(sp.ncol, kColsPerCta), nb);
  const size_t zs = zpass_smem<T>(g.n3), ps = plane_smem<T>(g);
  allow_smem(k_zinv<T>, zs);
  allow_smem(k_zfwd<T>, zs);
  allow_smem(k_plane<T>, ps);
  {
    ProfScope p("k_zinv", st, 1);
    count_launches(1);
    k_zinv<T><<<gz, kColsPerCta * 32, zs, st>>>(psi, ldpsi, scratch, sp, g.n3, fp.p3);
  }
  {
    ProfScope p("k_plane", st, 1);
    count_launches(1);
    k_plane<T><<<dim3(g.n3, nb), kPlaneThreads, ps, st>>>(scratch, sp, vplane, g, fp.p1, fp.p2);
  }
  const T inv_nr = (T)(1.0 / ((double)g.n1 * g.n2 * g.n3));
  {
    ProfScope p("k_zfwd", st, 1);
    count_launches(1);
    k_zfwd<T><<<gz, kColsPerCta * 32, zs, st>>>(scratch, psi, ldpsi, hpsi, ldh, kin, sp, g.n3, inv_nr, fp.p3);
  }
}

// ---- densities ---------------------------------------------------------------------------
// One CTA owns one z-plane of the density and walks the bands, so the accumulation needs
// no atomics and its order is fixed (bitwise reproducible).
template <typename T>
__global__ void __launch_bounds__(kPlaneThreads)
k_plane_density(const cplx<T>* __restrict__ scratch, SphereDev sp, int nb, const double* __restrict__ weight,
                double* __restrict__ rho_plane, int accumulate, GridDims g, LinePlan<T> p1, LinePlan<T> p2) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* P = reinterpret_cast<C*>(smem_raw);
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3, pitch = n2 + 1, npl = n1 * n2;
  const int i3 = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double* R = rho_plane + (size_t)i3 * npl;
  for (int b = 0; b < nb; ++b) {
    const C* S = scratch + ((size_t)b * n3 + i3) * sp.ncol;
    for (int idx = threadIdx.x; idx < n1 * pitch; idx += blockDim.x) P[idx] = mk<T>(0, 0);
    __syncthreads();
    for (int c = threadIdx.x; c < sp.ncol; c += blockDim.x) P[sp.col_i1[c] * pitch + sp.col_i2[c]] = S[c];
    __syncthreads();
    for (int r = w; r < sp.nrow; r += nw) fft_line<T, kMaxPlane>(P +sp.row_i1[r] * pitch, 1, p2, lane, +1);
    __syncthreads();
    for (int i2 = w; i2 < n2; i2 += nw) fft_line<T, kMaxPlane>(P +i2, pitch, p1, lane, +1);
    __syncthreads();
    const double wb = weight[b];
    const bool first = (b == 0) && !accumulate;
    for (int idx = threadIdx.x; idx < npl; idx += blockDim.x) {
      const int i1 = idx / n2, i2 = idx - i1 * n2;
      const C z = P[i1 * pitch + i2];
      const double d = wb * ((double)z.x * (double)z.x + (double)z.y * (double)z.y);
      R[idx] = first ? d : R[idx] + d;
    }
    __syncthreads();
  }
}

template <typename T>
void launch_density(const cplx<T>* psi, int ldpsi, int nb, const double* weight, cplx<T>* scratch,
                    double* rho_plane, int accumulate, const SphereDev& sp, const GridDims& g,
                    const FftPlans<T>& fp, cudaStream_t st) {
  if (nb <= 0) return;
  if (launch_density_ct<T>(psi, ldpsi, nb, weight, scratch, rho_plane, accumulate, sp, g, fp, st)) return;
  const dim3 gz(ceil_div(sp.ncol, kColsPerCta), nb);
  const size_t zs = zpass_smem<T>(g.n3), ps = plane_smem<T>(g);
  allow_smem(k_zinv<T>, zs);
  allow_smem(k_plane_density<T>, ps);
  count_launches(1);
  k_zinv<T><<<gz, kColsPerCta * 32, zs, st>>>(psi, ldpsi, scratch, sp, g.n3, fp.p3);
  count_launches(1);
  k_plane_density<T><<<g.n3, kPlaneThreads, ps, st>>>(scratch, sp, nb, weight, rho_plane, accumulate, g, fp.p1, fp.p2);
}

// ---- transposes ----------------------------------------------------------------------------
template <typename Tin, typename Tout>
__global__ void k_transpose(const Tin* __restrict__ in, Tout* __restrict__ out, int rows, int cols, int accumulate) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = by + j, c = bx + threadIdx.x;
    if (r < rows && c < cols) tile[j][threadIdx.x] = (double)in[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = bx + j, r = by + threadIdx.x;
    if (r < rows && c < cols) {
      Tout v = (Tout)tile[threadIdx.x][j];
      size_t o = (size_t)c * rows + r;
      out[o] = accumulate ? (Tout)(out[o] + v) : v;
    }
  }
}

template <typename Tin, typename Tout>
void launch_transpose(const Tin* in, Tout* out, int rows, int cols, int accumulate, cudaStream_t st) {
  dim3 grid(ceil_div(cols, 32), ceil_div(rows, 32));
  count_launches(1);
  k_transpose<Tin, Tout><<<grid, dim3(32, 8), 0, st>>>(in, out, rows, cols, accumulate);
}

template void launch_hpsi_local<float>(const float2*, int, float2*, int, int, const float*, const float*, float2*,
                                       const SphereDev&, const GridDims&, const FftPlans<float>&, cudaStream_t);
template void launch_hpsi_local<double>(const double2*, int, double2*, int, int, const double*, const double*,
                                        double2*, const SphereDev&, const GridDims&, const FftPlans<double>&,
                                        cudaStream_t);
template void launch_density<float>(const float2*, int, int, const double*, float2*, double*, int, const SphereDev&,
                                    const GridDims&, const FftPlans<float>&, cudaStream_t);
template void launch_density<double>(const double2*, int, int, const double*, double2*, double*, int,
                                     const SphereDev&, const GridDims&, const FftPlans<double>&, cudaStream_t);
template void launch_transpose<double, double>(const double*, double*, int, int, int, cudaStream_t);
template void launch_transpose<double, float>(const double*, float*, int, int, int, cudaStream_t);

}  // namespace fde
