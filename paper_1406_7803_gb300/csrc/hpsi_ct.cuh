// hpsi_ct.cuh -- H psi, band-density and full-grid transform kernels with compile-time
// transform lengths (fftct.cuh).  Same data flow as hpsi.cu / grid.cu; included by one
// translation unit per precision, which instantiates the supported lengths.
#pragma once

#include "fftct.cuh"
#include "kernels.h"
#include "prof.h"

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

namespace fde {

constexpr int kCtThreads = 256;
// Sphere columns (z-lines) per CTA in the z passes: 8 (one warp gathers or scatters each
// column), fewer when one staged batch holds fewer lines.  Measured on the 72 x 72 x 180 cell:
// 12 columns of 180 points (the full FP32 batch) made the forward pass 17 % slower (fewer
// CTAs, two columns per warp in the epilogue) for a 4 % faster inverse pass.
template <typename T, int N3> __host__ __device__ constexpr int ct_zcols() {
  return ct_lines_per_batch<T, N3, kCtThreads>() < 8 ? ct_lines_per_batch<T, N3, kCtThreads>() : 8;
}

// Every (subsystem, k) block of bands is an item; the kernels below run a batch of items in
// one launch (the batch travels as a kernel parameter), so subsystems of uneven size share
// the GPU instead of taking one small launch each.  The first z-block and the first plane
// block of each item are prefix offsets; a CTA finds its item by scanning the table.
template <typename T> struct HpsiItem {
  SphereDev sp;
  const cplx<T>* psi;
  cplx<T>* hpsi;
  const T* kin;
  const T* vplane;
  cplx<T>* scratch;  // [nb][n3][ncol]
  int ld, nb, zstart, pstart;
};
constexpr int kBatchMax = 24;
template <typename T> struct HpsiBatch {
  int n;
  HpsiItem<T> it[kBatchMax];
};

template <typename T>
__device__ __forceinline__ int batch_item(const HpsiBatch<T>& B, int blk, bool plane) {
  int i = 0;
  for (int j = 1; j < B.n; ++j)
    if ((plane ? B.it[j].pstart : B.it[j].zstart) <= blk) i = j;
  return i;
}

template <typename T, int N3>
__global__ void __launch_bounds__(kCtThreads)
k_zinv_ct(const __grid_constant__ HpsiBatch<T> B, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int LP = N3 + 1;
  constexpr int ZC = ct_zcols<T, N3>();
  __shared__ __align__(16) C lines[ZC * LP];
  const HpsiItem<T>& I = B.it[batch_item(B, blockIdx.x, false)];
  const SphereDev& sp = I.sp;
  const int ntile = (sp.ncol + ZC - 1) / ZC;
  const int local = blockIdx.x - I.zstart;
  const int b = local / ntile, c0 = (local - b * ntile) * ZC;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < ZC * LP; i += kCtThreads) lines[i] = mk<T>(0, 0);
  __syncthreads();
  for (int cc = w; cc < ZC; cc += kCtThreads / 32) {  // one warp per column
    const int c = c0 + cc;
    if (c >= sp.ncol) break;
    const int s = sp.col_start[c], e = sp.col_start[c + 1], m3 = sp.col_m3lo[c];
    const C* src = I.psi + (size_t)b * I.ld + s;
    C* L = lines + cc * LP;
    for (int t = lane; t < e - s; t += 32) {
      int i3 = m3 + t;
      i3 += (i3 < 0) ? N3 : 0;
      L[i3] = src[t];
    }
  }
  __syncthreads();
  ct_lines<T, N3, kCtThreads>(lines, LinesContig{LP}, ZC, tw, +1);
  const int nc = min(ZC, sp.ncol - c0);
  C* dst = I.scratch + (size_t)b * N3 * sp.ncol + c0;
  for (int idx = threadIdx.x; idx < N3 * ZC; idx += kCtThreads) {
    const int i3 = idx / ZC, ww = idx % ZC;
    if (ww < nc) dst[(size_t)i3 * sp.ncol + ww] = lines[ww * LP + i3];
  }
}

template <typename T, int N3>
__global__ void __launch_bounds__(kCtThreads)
k_zfwd_ct(const __grid_constant__ HpsiBatch<T> B, T inv_nr, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int LP = N3 + 1;
  constexpr int ZC = ct_zcols<T, N3>();
  __shared__ __align__(16) C lines[ZC * LP];
  const HpsiItem<T>& I = B.it[batch_item(B, blockIdx.x, false)];
  const SphereDev& sp = I.sp;
  const int ntile = (sp.ncol + ZC - 1) / ZC;
  const int local = blockIdx.x - I.zstart;
  const int b = local / ntile, c0 = (local - b * ntile) * ZC;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nc = min(ZC, sp.ncol - c0);
  const C* src = I.scratch + (size_t)b * N3 * sp.ncol + c0;
  for (int idx = threadIdx.x; idx < N3 * ZC; idx += kCtThreads) {
    const int i3 = idx / ZC, ww = idx % ZC;
    lines[ww * LP + i3] = (ww < nc) ? src[(size_t)i3 * sp.ncol + ww] : mk<T>(0, 0);
  }
  __syncthreads();
  ct_lines<T, N3, kCtThreads>(lines, LinesContig{LP}, ZC, tw, -1);
  const C* ps = I.psi + (size_t)b * I.ld;
  C* hs = I.hpsi + (size_t)b * I.ld;
  for (int cc = w; cc < ZC; cc += kCtThreads / 32) {  // one warp per column
    const int c = c0 + cc;
    if (c >= sp.ncol) break;
    const C* L = lines + cc * LP;
    const int s = sp.col_start[c], e = sp.col_start[c + 1], m3 = sp.col_m3lo[c];
    for (int t = lane; t < e - s; t += 32) {
      int i3 = m3 + t;
      i3 += (i3 < 0) ? N3 : 0;
      const int gidx = s + t;
      const C x = ps[gidx];
      const T kk = I.kin[gidx];
      C o = L[i3];
      o.x = o.x * inv_nr + kk * x.x;
      o.y = o.y * inv_nr + kk * x.y;
      hs[gidx] = o;
    }
  }
}

// Row r of a plane's data rows holds the sphere columns S[rs[r] .. rs[r] + rl[r]) at consecutive
// signed m2 from m2lo[r] (i2 = m2 mod N): element i2 of the row is column rs + m2(i2) - m2lo
// when that lies in the row, else zero.  RowIn feeds the first stage of the inverse y transform
// straight from the columns; RowOut takes the last stage of the forward y transform's outputs
// at the sphere columns back to them.
__device__ __forceinline__ int row_offset(int i2, int n, int m2lo, int len) {
  const int d = (i2 <= n / 2 ? i2 : i2 - n) - m2lo;
  return (d >= 0 && d < len) ? d : -1;
}
template <typename T> struct RowIn {
  const cplx<T>* S;
  const int *rs, *rl, *m2lo;
  int n;
  __device__ __forceinline__ cplx<T> operator()(int r, int i2) const {
    const int d = row_offset(i2, n, m2lo[r], rl[r]);
    return d >= 0 ? S[rs[r] + d] : mk<T>(0, 0);
  }
};
template <typename T> struct RowOut {
  cplx<T>* S;
  const int *rs, *rl, *m2lo;
  int n;
  __device__ __forceinline__ void operator()(int r, int i2, cplx<T> v) const {
    const int d = row_offset(i2, n, m2lo[r], rl[r]);
    if (d >= 0) S[rs[r] + d] = v;
  }
};

// One CTA per (item, band, z-plane): columns in, 2D inverse FFT (y on the rows holding
// columns, then x), potential multiply, 2D forward FFT, columns out.  n1 = n2 = N; the plane is
// P[i1][i2] (pitch N + 1) and the potential plane vplane[i3][i1][i2].
// Variants of the plane pass: V selects the staged transform's register budget, radix order
// and row thread mapping (fftct.cuh), MINB the CTAs per SM the registers are bounded for (four
// FP32 CTAs of 42 KB for a 72 x 72 plane need <= 64 registers; FP64 planes of 84 KB fit two),
// FX fuses the x pass: the inverse's last stage, the potential multiply and the forward's first
// stage run on the same registers (ct_cols_vmul), one shared-memory round trip and one barrier
// pair fewer per column batch and no separate multiply pass.  SG fuses the sphere scatter and
// gather into the y transforms: the first inverse stage reads the columns from global memory
// and the last forward stage writes them back, so only the rows without columns are
// zero-filled and neither the scatter nor the gather pass goes through shared memory.
template <typename T, int N, int V = 0, int MINB = (sizeof(T) == 4 ? 4 : 2), bool FX = false, bool SG = false>
__global__ void __launch_bounds__(kCtThreads, MINB)
k_plane_ct(const __grid_constant__ HpsiBatch<T> B, int n3, const cplx<T>* __restrict__ tw1,
           const cplx<T>* __restrict__ tw2) {
  using C = cplx<T>;
  constexpr int PITCH = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* P = reinterpret_cast<C*>(smem_raw);
  __shared__ int rows[N];
  const HpsiItem<T>& I = B.it[batch_item(B, blockIdx.x, true)];
  const SphereDev& sp = I.sp;
  const int local = blockIdx.x - I.pstart;
  const int b = local / n3, i3 = local - b * n3;
  C* S = I.scratch + ((size_t)b * n3 + i3) * sp.ncol;
  const T* vp = I.vplane + (size_t)i3 * N * N;
  if constexpr (SG) {
    __shared__ int rowof[N], rs[N], re[N], rm2[N];
    for (int i = threadIdx.x; i < N; i += kCtThreads) rowof[i] = -1;
    __syncthreads();
    for (int r = threadIdx.x; r < sp.nrow; r += kCtThreads) {
      rows[r] = sp.row_i1[r];
      rowof[rows[r]] = r;
    }
    __syncthreads();
    // the columns of a row are consecutive in the sphere order (sorted by m1, then m2)
    for (int c = threadIdx.x; c < sp.ncol; c += kCtThreads) {
      const int i1 = sp.col_i1[c];
      if (c == 0 || sp.col_i1[c - 1] != i1) {
        const int r = rowof[i1], i2 = sp.col_i2[c];
        rs[r] = c;
        rm2[r] = i2 <= N / 2 ? i2 : i2 - N;
      }
      if (c == sp.ncol - 1 || sp.col_i1[c + 1] != i1) re[rowof[i1]] = c + 1;
    }
    for (int idx = threadIdx.x; idx < N * PITCH; idx += kCtThreads)
      if (rowof[idx / PITCH] < 0) P[idx] = mk<T>(0, 0);
    __syncthreads();
    for (int r = threadIdx.x; r < sp.nrow; r += kCtThreads) re[r] -= rs[r];  // now the row lengths
    __syncthreads();
    ct_lines_io<T, N, kCtThreads, LinesRows, V>(P, LinesRows{rows, PITCH}, sp.nrow, tw2, +1,
                                                RowIn<T>{S, rs, re, rm2, N}, NoIO());
    ct_cols_vmul<T, N, kCtThreads, V>(P, PITCH, tw1, vp);
    ct_lines_io<T, N, kCtThreads, LinesRows, V>(P, LinesRows{rows, PITCH}, sp.nrow, tw2, -1, NoIO(),
                                                RowOut<T>{S, rs, re, rm2, N});
  } else {
    for (int idx = threadIdx.x; idx < N * PITCH; idx += kCtThreads) P[idx] = mk<T>(0, 0);
    for (int r = threadIdx.x; r < sp.nrow; r += kCtThreads) rows[r] = sp.row_i1[r];
    __syncthreads();
    for (int c = threadIdx.x; c < sp.ncol; c += kCtThreads) P[sp.col_i1[c] * PITCH + sp.col_i2[c]] = S[c];
    __syncthreads();
    ct_lines<T, N, kCtThreads, LinesRows, V>(P, LinesRows{rows, PITCH}, sp.nrow, tw2, +1);
    if constexpr (FX) {
      ct_cols_vmul<T, N, kCtThreads, V>(P, PITCH, tw1, vp);
    } else {
      ct_lines<T, N, kCtThreads, LinesCols, V>(P, LinesCols{PITCH}, N, tw1, +1);
      for (int idx = threadIdx.x; idx < N * N; idx += kCtThreads) {
        const int a = idx / N, c = idx - a * N;
        C& z = P[a * PITCH + c];
        const T v = vp[idx];
        z.x *= v;
        z.y *= v;
      }
      __syncthreads();
      ct_lines<T, N, kCtThreads, LinesCols, V>(P, LinesCols{PITCH}, N, tw1, -1);
    }
    ct_lines<T, N, kCtThreads, LinesRows, V>(P, LinesRows{rows, PITCH}, sp.nrow, tw2, -1);
    for (int c = threadIdx.x; c < sp.ncol; c += kCtThreads) S[c] = P[sp.col_i1[c] * PITCH + sp.col_i2[c]];
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(kCtThreads)
k_plane_density_ct(const cplx<T>* __restrict__ scratch, SphereDev sp, int nb, const double* __restrict__ weight,
                   double* __restrict__ rho_plane, int accumulate, int n3, const cplx<T>* __restrict__ tw1,
                   const cplx<T>* __restrict__ tw2) {
  using C = cplx<T>;
  constexpr int PITCH = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* P = reinterpret_cast<C*>(smem_raw);
  __shared__ int rows[N];
  const int i3 = blockIdx.x;
  for (int r = threadIdx.x; r < sp.nrow; r += kCtThreads) rows[r] = sp.row_i1[r];
  double* R = rho_plane + (size_t)i3 * N * N;
  for (int b = 0; b < nb; ++b) {
    const C* S = scratch + ((size_t)b * n3 + i3) * sp.ncol;
    for (int idx = threadIdx.x; idx < N * PITCH; idx += kCtThreads) P[idx] = mk<T>(0, 0);
    __syncthreads();
    for (int c = threadIdx.x; c < sp.ncol; c += kCtThreads) P[sp.col_i1[c] * PITCH + sp.col_i2[c]] = S[c];
    __syncthreads();
    ct_lines<T, N, kCtThreads>(P, LinesRows{rows, PITCH}, sp.nrow, tw2, +1);
    ct_lines<T, N, kCtThreads>(P, LinesCols{PITCH}, N, tw1, +1);
    const double wb = weight[b];
    const bool first = (b == 0) && !accumulate;
    for (int idx = threadIdx.x; idx < N * N; idx += kCtThreads) {
      const int i1 = idx / N, i2 = idx - i1 * N;
      const C z = P[i1 * PITCH + i2];
      const double d = wb * ((double)z.x * (double)z.x + (double)z.y * (double)z.y);
      R[idx] = first ? d : R[idx] + d;
    }
    __syncthreads();
  }
}

// One axis of a full 3D transform: element (o, e, t) at (o * N + e) * I + t.  A CTA holds as
// many lines as one batch of the staged transform keeps every thread busy with
// (ct_lines_per_batch), so all stages run in a single pass over the CTA's lines; each line's
// base offset is computed once (32-bit: the grid has fewer than 2^31 points).
template <typename T, int N> __host__ __device__ constexpr int ct_axis_lines() {
  return ct_lines_per_batch<T, N, kCtThreads>();
}
template <typename T, int N>
__global__ void __launch_bounds__(kCtThreads)
k_fft_axis_ct(cplx<T>* __restrict__ data, int nlines, int I, const cplx<T>* __restrict__ tw, int sign) {
  using C = cplx<T>;
  constexpr int LP = N + 1;
  constexpr int LPC = ct_axis_lines<T, N>();
  __shared__ __align__(16) C lines[LPC * LP];
  __shared__ int base[LPC];
  const int l0 = blockIdx.x * LPC;
  const int nl = min(LPC, nlines - l0);
  if ((int)threadIdx.x < LPC) {
    const int l = l0 + (int)threadIdx.x, o = l / I, t = l - o * I;
    base[threadIdx.x] = o * N * I + t;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < LPC * N; idx += kCtThreads) {
    int tl, e;
    if (I == 1) { tl = idx / N; e = idx - tl * N; } else { e = idx / LPC; tl = idx - e * LPC; }
    lines[tl * LP + e] = (tl < nl) ? data[base[tl] + e * I] : mk<T>(0, 0);
  }
  __syncthreads();
  ct_lines<T, N, kCtThreads>(lines, LinesContig{LP}, LPC, tw, sign);
  for (int idx = threadIdx.x; idx < LPC * N; idx += kCtThreads) {
    int tl, e;
    if (I == 1) { tl = idx / N; e = idx - tl * N; } else { e = idx / LPC; tl = idx - e * LPC; }
    if (tl < nl) data[base[tl] + e * I] = lines[tl * LP + e];
  }
}

template <typename K> static inline void ct_allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define FDE_CT_LINES(X) X(24) X(32) X(60) X(72) X(96) X(144) X(180) X(288)
#define FDE_CT_PLANES(X) X(24) X(32) X(72) X(96) X(144)

template <typename T> bool ct_line_ok(int n) {
  switch (n) {
#define FDE_CASE(N) case N:
    FDE_CT_LINES(FDE_CASE)
#undef FDE_CASE
    return true;
    default: return false;
  }
}
template <typename T> bool ct_plane_ok(int n1, int n2) {
  if (n1 != n2) return false;
  if ((size_t)n1 * (n1 + 1) * sizeof(cplx<T>) > 200 * 1024) return false;
  switch (n1) {
#define FDE_CASE(N) case N:
    FDE_CT_PLANES(FDE_CASE)
#undef FDE_CASE
    return true;
    default: return false;
  }
}

template <typename T> static int ct_zcols_host(int n3) {
  switch (n3) {
#define FDE_CASE(N) \
  case N:           \
    return ct_zcols<T, N>();
    FDE_CT_LINES(FDE_CASE)
#undef FDE_CASE
  }
  return 8;
}

template <typename T>
static void ct_zinv(int n3, unsigned blocks, cudaStream_t st, const HpsiBatch<T>& B, const cplx<T>* tw) {
  switch (n3) {
#define FDE_CASE(N)                                                    \
  case N:                                                              \
    count_launches(1);                                                 \
    k_zinv_ct<T, N><<<blocks, kCtThreads, 0, st>>>(B, tw);            \
    break;
    FDE_CT_LINES(FDE_CASE)
#undef FDE_CASE
  }
}

template <typename T>
static void ct_zfwd(int n3, unsigned blocks, cudaStream_t st, const HpsiBatch<T>& B, T inv_nr, const cplx<T>* tw) {
  switch (n3) {
#define FDE_CASE(N)                                                    \
  case N:                                                              \
    count_launches(1);                                                 \
    k_zfwd_ct<T, N><<<blocks, kCtThreads, 0, st>>>(B, inv_nr, tw);    \
    break;
    FDE_CT_LINES(FDE_CASE)
#undef FDE_CASE
  }
}

// Plane-pass variants tried by the tuner (FP32; FP64 tries 0, 2, 4 and 6):
//   0: register budget 16, odd radices first, 4 CTAs/SM    1: largest radix first, 4 CTAs/SM
//   2: fused x pass (FX), 4 CTAs/SM                         3: fused x pass, 3 CTAs/SM
//   4: fused x pass, line-fastest row mapping, 4 CTAs/SM    5: the same, 3 CTAs/SM
// Measured on the 72 x 72 x 180 cell: variant 0 1.49 ms, largest-first 1.56 ms, budget 18 at
// 3 / 2 CTAs/SM 1.75 / 2.00 ms (dropped), fused x at 3 CTAs/SM 1.35 ms.  Also dropped:
// 288-thread CTAs (1.75 / 2.30 ms); warp-local line transforms, each line owned by one warp so
// that a stage synchronises only that warp (2.21 ms: the pass is bound by shared-memory
// bandwidth, not by its barriers, and the transposed layout conflicts on more banks).
//   6: fused x pass and fused scatter / gather (SG), 3 CTAs/SM    7: the same with the row mapping
constexpr int kPlaneVariants = 8;
template <typename T> constexpr bool plane_variant_ok(int v) {
  return sizeof(T) == 4 ? (v >= 0 && v < kPlaneVariants) : (v == 0 || v == 2 || v == 4 || v == 6);
}

template <typename T, int N, int V, int MINB, bool FX = false, bool SG = false>
static void ct_plane_launch(unsigned blocks, cudaStream_t st, const HpsiBatch<T>& B, int n3, const cplx<T>* tw1,
                            const cplx<T>* tw2) {
  const size_t sm = (size_t)N * (N + 1) * sizeof(cplx<T>);
  ct_allow_smem(k_plane_ct<T, N, V, MINB, FX, SG>, sm);
  count_launches(1);
  k_plane_ct<T, N, V, MINB, FX, SG><<<blocks, kCtThreads, sm, st>>>(B, n3, tw1, tw2);
}

// CTAs of the plane pass that fit an SM's 228 KB of shared memory (the plane plus ~2 KB of
// static and reserved memory per CTA): the register bound of a variant is never set for more
// CTAs than can be resident (a 144 x 144 FP32 plane, 167 KB, runs one CTA per SM with the full
// register file instead of spilling under a 64-register bound).
template <typename T, int N> constexpr int ct_plane_fit() {
  return (int)(233472 / ((size_t)N * (N + 1) * sizeof(cplx<T>) + 2048));
}

template <typename T, int N>
static void ct_plane_variant(int variant, unsigned blocks, cudaStream_t st, const HpsiBatch<T>& B, int n3,
                             const cplx<T>* tw1, const cplx<T>* tw2) {
  constexpr int FIT = ct_plane_fit<T, N>() > 0 ? ct_plane_fit<T, N>() : 1;
  constexpr int HI = (sizeof(T) == 4 ? 4 : 2) < FIT ? (sizeof(T) == 4 ? 4 : 2) : FIT;
  // the lower-occupancy variants: 3 CTAs/SM, or one fewer than fit when that is at most 3
  constexpr int LO = FIT > 3 ? 3 : (FIT > 1 ? FIT - 1 : 1);
  constexpr int M4 = HI, M3 = sizeof(T) == 4 ? LO : HI;
  switch (variant) {
    case 1:
      if constexpr (sizeof(T) == 4) return ct_plane_launch<T, N, 16, M4>(blocks, st, B, n3, tw1, tw2);
      break;
    case 2: return ct_plane_launch<T, N, 0, M4, true>(blocks, st, B, n3, tw1, tw2);
    case 3:
      if constexpr (sizeof(T) == 4) return ct_plane_launch<T, N, 0, M3, true>(blocks, st, B, n3, tw1, tw2);
      break;
    case 4: return ct_plane_launch<T, N, 32, M4, true>(blocks, st, B, n3, tw1, tw2);
    case 5:
      if constexpr (sizeof(T) == 4) return ct_plane_launch<T, N, 32, M3, true>(blocks, st, B, n3, tw1, tw2);
      break;
    case 6: return ct_plane_launch<T, N, 0, M3, true, true>(blocks, st, B, n3, tw1, tw2);
    case 7:
      if constexpr (sizeof(T) == 4) return ct_plane_launch<T, N, 32, M3, true, true>(blocks, st, B, n3, tw1, tw2);
      break;
  }
  ct_plane_launch<T, N, 0, M4>(blocks, st, B, n3, tw1, tw2);
}

template <typename T>
static void ct_plane(int n, unsigned blocks, cudaStream_t st, const HpsiBatch<T>& B, int n3, const cplx<T>* tw1,
                     const cplx<T>* tw2, int variant) {
  switch (n) {
#define FDE_CASE(N)                                                          \
  case N:                                                                    \
    ct_plane_variant<T, N>(variant, blocks, st, B, n3, tw1, tw2);            \
    break;
    FDE_CT_PLANES(FDE_CASE)
#undef FDE_CASE
  }
}

// Plane-pass tuner: the first large batch (>= kTuneMinPlanes planes) of a grid shape (plane
// side, z length) times every variant once on the batch itself -- the z pass is rerun before
// each trial, so the scratch it transforms in place is regenerated -- and keeps the fastest
// for that shape.  Smaller batches (the eigensolver's residual blocks) use the tuned choice
// when there is one, else variant 0.  Never runs while the stream is being captured.
// FDE_PLANE_VARIANT=<v> in the environment pins the variant (reproducible rounding across
// machines); an FP64 plane pass runs a pinned 0, 2, 4 or 6 as it is and every other pin as 0.
constexpr unsigned kTuneMinPlanes = 4096;
struct PlaneTuner {
  std::mutex mu;
  std::map<std::tuple<int, int, int>, int> best;
};
inline PlaneTuner& plane_tuner() {
  static PlaneTuner t;
  return t;
}
// Pinned variant (-1: tune); FDE_PLANE_VARIANT in the environment sets the initial value.
inline std::atomic<int>& plane_pin() {
  static std::atomic<int> pin([] {
    const char* e = getenv("FDE_PLANE_VARIANT");
    const int v = e ? atoi(e) : -1;
    return (v >= 0 && v < kPlaneVariants) ? v : -1;
  }());
  return pin;
}
// Tuned variant of the FP32 plane pass for a grid shape, or -1 if none was tuned yet.
inline int tuned_plane_variant(int n, int n3) {
  PlaneTuner& tuner = plane_tuner();
  std::lock_guard<std::mutex> lock(tuner.mu);
  auto it = tuner.best.find(std::make_tuple(n, n3, 4));
  return it == tuner.best.end() ? -1 : it->second;
}
template <typename T>
static int plane_variant(int n, int n3, unsigned zb, unsigned pb, cudaStream_t st, const HpsiBatch<T>& B,
                         const FftPlans<T>& fp) {
  const int pinned = plane_pin().load();
  if (pinned >= 0) return plane_variant_ok<T>(pinned) ? pinned : 0;
  const auto key = std::make_tuple(n, n3, (int)sizeof(T));
  PlaneTuner& tuner = plane_tuner();
  std::lock_guard<std::mutex> lock(tuner.mu);
  auto& tab = tuner.best;
  auto it = tab.find(key);
  if (it != tab.end()) return it->second;
  if (pb < kTuneMinPlanes) return 0;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return 0;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return 0;
  if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return 0; }
  int bestv = 0;
  float bestt = 1e30f;
  for (int v = 0; v < kPlaneVariants; ++v) {
    if (!plane_variant_ok<T>(v)) continue;
    ct_zinv<T>(n3, zb, st, B, fp.p3.tw);
    cudaEventRecord(a, st);
    ct_plane<T>(n, pb, st, B, n3, fp.p1.tw, fp.p2.tw, v);
    cudaEventRecord(b, st);
    float ms = 1e30f;
    if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms < bestt) {
      bestt = ms;
      bestv = v;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  tab[key] = bestv;
  return bestv;
}

template <typename T>
static void ct_plane_density(int n, int n3, cudaStream_t st, const cplx<T>* scr, const SphereDev& sp, int nb,
                             const double* weight, double* rho_plane, int acc, const cplx<T>* tw1,
                             const cplx<T>* tw2) {
  const size_t sm = (size_t)n * (n + 1) * sizeof(cplx<T>);
  switch (n) {
#define FDE_CASE(N)                                                                                      \
  case N:                                                                                                \
    ct_allow_smem(k_plane_density_ct<T, N>, sm);                                                         \
    count_launches(1);                                                                                   \
    k_plane_density_ct<T, N><<<n3, kCtThreads, sm, st>>>(scr, sp, nb, weight, rho_plane, acc, n3, tw1, tw2); \
    break;
    FDE_CT_PLANES(FDE_CASE)
#undef FDE_CASE
  }
}

template <typename T>
static void ct_axis(int n, long long nlines, long long I, cudaStream_t st, cplx<T>* data, const cplx<T>* tw, int sign) {
  ProfScope prof_(sizeof(T) == 8 ? "k_fft_axis_f64" : "k_fft_axis_f32", st);
  switch (n) {
#define FDE_CASE(N)                                                                                    \
  case N:                                                                                              \
    count_launches(1);                                                                                 \
    k_fft_axis_ct<T, N><<<(unsigned)ceil_div(nlines, ct_axis_lines<T, N>()), kCtThreads, 0, st>>>(   \
        data, (int)nlines, (int)I, tw, sign);                                                          \
    break;
    FDE_CT_LINES(FDE_CASE)
#undef FDE_CASE
  }
}

// Run up to kBatchMax items per launch; items[i].zstart / pstart are filled here.
template <typename T>
bool launch_hpsi_batch_ct(const HpsiItemDesc<T>* items, int nitems, const GridDims& g, const FftPlans<T>& fp,
                          cudaStream_t st) {
  if (!ct_plane_ok<T>(g.n1, g.n2) || !ct_line_ok<T>(g.n3)) return false;
  const T inv_nr = (T)(1.0 / ((double)g.n1 * g.n2 * g.n3));
  for (int i0 = 0; i0 < nitems; i0 += kBatchMax) {
    HpsiBatch<T> B;
    B.n = std::min(kBatchMax, nitems - i0);
    int zb = 0, pb = 0;
    for (int j = 0; j < B.n; ++j) {
      const HpsiItemDesc<T>& d = items[i0 + j];
      HpsiItem<T>& it = B.it[j];
      it.sp = d.sp;
      it.psi = d.psi;
      it.hpsi = d.hpsi;
      it.kin = d.kin;
      it.vplane = d.vplane;
      it.scratch = d.scratch;
      it.ld = d.ld;
      it.nb = d.nb;
      it.zstart = zb;
      it.pstart = pb;
      zb += ceil_div(d.sp.ncol, ct_zcols_host<T>(g.n3)) * d.nb;
      pb += g.n3 * d.nb;
    }
    if (zb == 0) continue;
    const int variant = plane_variant<T>(g.n1, g.n3, (unsigned)zb, (unsigned)pb, st, B, fp);
    {
      ProfScope p("k_zinv", st, 1);
      ct_zinv<T>(g.n3, (unsigned)zb, st, B, fp.p3.tw);
    }
    {
      ProfScope p("k_plane", st, 1);
      ct_plane<T>(g.n1, (unsigned)pb, st, B, g.n3, fp.p1.tw, fp.p2.tw, variant);
    }
    {
      ProfScope p("k_zfwd", st, 1);
      ct_zfwd<T>(g.n3, (unsigned)zb, st, B, inv_nr, fp.p3.tw);
    }
  }
  return true;
}

template <typename T>
bool launch_hpsi_local_ct(const cplx<T>* psi, int ldpsi, cplx<T>* hpsi, int ldh, int nb, const T* kin,
                          const T* vplane, cplx<T>* scratch, const SphereDev& sp, const GridDims& g,
                          const FftPlans<T>& fp, cudaStream_t st) {
  if (ldpsi != ldh) return false;
  HpsiItemDesc<T> d{sp, psi, hpsi, kin, vplane, scratch, ldpsi, nb};
  return launch_hpsi_batch_ct<T>(&d, 1, g, fp, st);
}

template <typename T>
bool launch_density_ct(const cplx<T>* psi, int ldpsi, int nb, const double* weight, cplx<T>* scratch,
                       double* rho_plane, int accumulate, const SphereDev& sp, const GridDims& g,
                       const FftPlans<T>& fp, cudaStream_t st) {
  if (!ct_plane_ok<T>(g.n1, g.n2) || !ct_line_ok<T>(g.n3)) return false;
  HpsiBatch<T> B;
  B.n = 1;
  B.it[0] = HpsiItem<T>{sp, psi, nullptr, nullptr, nullptr, scratch, ldpsi, nb, 0, 0};
  {
    ProfScope prof_("k_zinv_density", st);
    ct_zinv<T>(g.n3, (unsigned)(ceil_div(sp.ncol, ct_zcols_host<T>(g.n3)) * nb), st, B, fp.p3.tw);
  }
  ProfScope prof_("k_plane_density", st);
  ct_plane_density<T>(g.n1, g.n3, st, scratch, sp, nb, weight, rho_plane, accumulate, fp.p1.tw, fp.p2.tw);
  return true;
}

template <typename T>
bool launch_fft3d_ct(cplx<T>* data, const GridDims& g, const FftPlans<T>& fp, int sign, cudaStream_t st) {
  if (!ct_line_ok<T>(g.n1) || !ct_line_ok<T>(g.n2) || !ct_line_ok<T>(g.n3)) return false;
  const long long nr = (long long)g.n1 * g.n2 * g.n3;
  if (nr >= (1ll << 31)) return false;  // the compile-time kernels index in 32 bits
  ct_axis<T>(g.n3, nr / g.n3, 1, st, data, fp.p3.tw, sign);
  ct_axis<T>(g.n2, nr / g.n2, g.n3, st, data, fp.p2.tw, sign);
  ct_axis<T>(g.n1, nr / g.n1, (long long)g.n2 * g.n3, st, data, fp.p1.tw, sign);
  return true;
}

}  // namespace fde
