// grid.cu -- the embedding-potential build on the shared real-space grid:
//   rho = sum_I rho_I (Eq. meth:1), full 3D FFTs, the FFT Poisson solve for v_H, the
//   erf local potential of all nuclei, gradients and divergences through FFTs, and the
//   pointwise exchange-correlation and GGA kinetic functionals (Appendix: kinetic energy
//   functional and potential), with FP64 energy reductions in a fixed order.
#include <math.h>

#include "fft.cuh"
#include "grid_kernels.h"
#include "prof.h"

namespace fde {

// ---- full 3D transforms, one axis per pass ---------------------------------------------
// Element (o, e, t) of a pass sits at (o * N + e) * I + t: N is the transformed length, I
// the product of the faster axes.  A CTA holds kLinesPerCta lines (one warp each).
constexpr int kLinesPerCta = 8;

template <typename T>
__global__ void __launch_bounds__(kLinesPerCta * 32)
k_fft_axis(cplx<T>* __restrict__ data, long long nlines, int N, long long I, LinePlan<T> p, int sign) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* lines = reinterpret_cast<C*>(smem_raw);
  const int lp = N + 1;
  const long long l0 = (long long)blockIdx.x * kLinesPerCta;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nl = (int)min((long long)kLinesPerCta, nlines - l0);
  for (int idx = threadIdx.x; idx < kLinesPerCta * N; idx += blockDim.x) {
    int tl, e;
    if (I == 1) { tl = idx / N; e = idx - tl * N; } else { e = idx / kLinesPerCta; tl = idx - e * kLinesPerCta; }
    if (tl < nl) {
      const long long l = l0 + tl, o = l / I, t = l - o * I;
      lines[tl * lp + e] = data[(o * N + e) * I + t];
    }
  }
  __syncthreads();
  if (w < nl) fft_line<T>(lines + w * lp, 1, p, lane, sign);
  __syncthreads();
  for (int idx = threadIdx.x; idx < kLinesPerCta * N; idx += blockDim.x) {
    int tl, e;
    if (I == 1) { tl = idx / N; e = idx - tl * N; } else { e = idx / kLinesPerCta; tl = idx - e * kLinesPerCta; }
    if (tl < nl) {
      const long long l = l0 + tl, o = l / I, t = l - o * I;
      data[(o * N + e) * I + t] = lines[tl * lp + e];
    }
  }
}

template <typename T>
void launch_fft3d(cplx<T>* data, const GridDims& g, const FftPlans<T>& fp, int sign, cudaStream_t st) {
  if (launch_fft3d_ct<T>(data, g, fp, sign, st)) return;
  const long long nr = (long long)g.n1 * g.n2 * g.n3;
  struct Ax { int N; long long I; const LinePlan<T>* p; } ax[3] = {
      {g.n3, 1, &fp.p3}, {g.n2, g.n3, &fp.p2}, {g.n1, (long long)g.n2 * g.n3, &fp.p1}};
  for (int a = 0; a < 3; ++a) {
    const long long nlines = nr / ax[a].N;
    const size_t sm = (size_t)kLinesPerCta * (ax[a].N + 1) * sizeof(cplx<T>);
    count_launches(1);
    k_fft_axis<T><<<(unsigned)((nlines + kLinesPerCta - 1) / kLinesPerCta), kLinesPerCta * 32, sm, st>>>(
        data, nlines, ax[a].N, ax[a].I, *ax[a].p, sign);
  }
}

// ---- reciprocal-space helpers -----------------------------------------------------------
struct Gpt {
  double gx, gy, gz, g2;
  bool nyq;
};

// Grid points are indexed in 32 bits here: the context accepts at most 320 points per axis,
// so a grid has fewer than 2^31 points.
__device__ __forceinline__ Gpt gvec(long long idx, const GridDims& g, const CellDev& c) {
  const int id = (int)idx;
  const int i3 = id % g.n3;
  const int r = id / g.n3;
  const int i2 = r % g.n2, i1 = r / g.n2;
  const int m1 = (i1 < (g.n1 + 1) / 2) ? i1 : i1 - g.n1;
  const int m2 = (i2 < (g.n2 + 1) / 2) ? i2 : i2 - g.n2;
  const int m3 = (i3 < (g.n3 + 1) / 2) ? i3 : i3 - g.n3;
  Gpt p;
  p.gx = m1 * c.b[0][0] + m2 * c.b[1][0] + m3 * c.b[2][0];
  p.gy = m1 * c.b[0][1] + m2 * c.b[1][1] + m3 * c.b[2][1];
  p.gz = m1 * c.b[0][2] + m2 * c.b[1][2] + m3 * c.b[2][2];
  p.g2 = p.gx * p.gx + p.gy * p.gy + p.gz * p.gz;
  p.nyq = ((g.n1 % 2 == 0) && m1 == -g.n1 / 2) || ((g.n2 % 2 == 0) && m2 == -g.n2 / 2) ||
          ((g.n3 % 2 == 0) && m3 == -g.n3 / 2);
  return p;
}

constexpr int kRedBlocks = 304;  // 2 x 152 SMs
constexpr int kRedThreads = 256;

__device__ __forceinline__ void block_sum_store(double v, double* out_slot) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    *out_slot = t;
  }
  __syncthreads();
}

// Local potential of all nuclei in reciprocal space (FP64):
// v(G) = (1/Omega) sum_a -4 pi Z_a / G^2 exp(-G^2 rc^2/4) exp(-i G.R_a), G != 0;
// v(0) = (1/Omega) sum_a pi Z_a rc^2; Nyquist planes zero.
__global__ void k_vloc_g(double2* __restrict__ V, GridDims g, CellDev c, const double* __restrict__ pos,
                         const double* __restrict__ Z, int natoms, double rc) {
  const long long nr = (long long)g.n1 * g.n2 * g.n3;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nr; idx += (long long)gridDim.x * blockDim.x) {
    const Gpt p = gvec(idx, g, c);
    double re = 0, im = 0;
    if (p.g2 == 0) {
      for (int a = 0; a < natoms; ++a) re += M_PI * Z[a] * rc * rc;
    } else if (!p.nyq) {
      const double f = -4.0 * M_PI / p.g2 * exp(-p.g2 * rc * rc / 4.0);
      for (int a = 0; a < natoms; ++a) {
        const double ph = p.gx * pos[3 * a] + p.gy * pos[3 * a + 1] + p.gz * pos[3 * a + 2];
        double sn, cs;
        sincos(ph, &sn, &cs);
        re += f * Z[a] * cs;
        im -= f * Z[a] * sn;
      }
    }
    V[idx] = make_double2(re / c.omega, im / c.omega);
  }
}

// ---- pointwise functionals ------------------------------------------------------------------
// Energy densities with their partial derivatives along rho and sigma = |grad rho|^2, in
// closed form, in the arithmetic type R (FP64 in FP64 contexts; FP32 in the mixed path, where
// the density and its gradients come from the double-float transforms and only the pointwise
// evaluation is single precision).  Every rho power comes from one cube root (rho^{1/3},
// 1/rho^{1/3} = rho^{2/3} / rho), and each chain-rule factor is written next to the quantity
// it differentiates, so the potentials are the exact derivatives of the coded energy
// densities.  Forms that would overflow FP32 at low density with noisy gradients (A^2 t^4 in
// PBE's H, t^4 in its A derivative) are written in the reciprocal variable there.
template <typename R> struct Pt {
  R rho, ir, r13, ir13;  // rho, 1/rho, rho^{1/3}, rho^{-1/3}
};
template <typename R> __device__ __forceinline__ Pt<R> make_pt(R rho) {
  Pt<R> p;
  p.rho = rho;
  p.ir = R(1) / rho;
  p.r13 = cbrt(rho);
  p.ir13 = p.r13 * p.r13 * p.ir;
  return p;
}

// Slater exchange of the uniform gas per volume, e_x = C_x rho^{4/3}, and its rho derivative.
constexpr double kCx = -0.75 * 0.98474502184269654;  // -(3/4)(3/pi)^{1/3}
template <typename R> __device__ __forceinline__ void slater(const Pt<R>& p, R* e, R* de) {
  *e = R(kCx) * p.rho * p.r13;
  *de = R(4.0 / 3.0 * kCx) * p.r13;
}

// PW92 correlation energy per particle of the unpolarised gas, eps_c(r_s), and d eps_c / d rho.
// r_s = (3 / (4 pi rho))^{1/3};  eps_c = -2A (1 + a1 r_s) ln(1 + 1/D),
// D = 2A (b1 r_s^{1/2} + b2 r_s + b3 r_s^{3/2} + b4 r_s^2).
template <typename R> __device__ __forceinline__ void pw92(const Pt<R>& p, R* ec, R* dec) {
  const R A = R(0.031091), a1 = R(0.21370), b1 = R(7.5957), b2 = R(3.5876), b3 = R(1.6382), b4 = R(0.49294);
  const R rs = R(0.62035049089940001667) * p.ir13;  // (3/(4 pi))^{1/3}
  const R srs = sqrt(rs);
  const R D = R(2) * A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs);
  const R dD = R(2) * A * (R(0.5) * b1 / srs + b2 + R(1.5) * b3 * srs + R(2) * b4 * rs);  // dD/dr_s
  const R iD = R(1) / D;
  const R L = log1p(iD);
  const R dL = -iD * iD / (R(1) + iD);  // d ln(1 + 1/D) / dD
  *ec = R(-2) * A * (R(1) + a1 * rs) * L;
  const R dec_drs = R(-2) * A * (a1 * L + (R(1) + a1 * rs) * dL * dD);
  *dec = dec_drs * (-rs * p.ir / R(3));  // d r_s / d rho = -r_s / (3 rho)
}

// PBE exchange-correlation energy per volume e(rho, sigma) with e_rho, e_sigma:
//   e = e_x^unif F_x(s) + rho (eps_c + H),  F_x = 1 + kappa - kappa / (1 + mu s^2 / kappa),
//   s^2 = sigma / (4 k_F^2 rho^2),  k_F = (3 pi^2 rho)^{1/3},
//   H = gamma ln(1 + (beta/gamma) t^2 P(A t^2)),  P(x) = (1 + x) / (1 + x + x^2),
//   t^2 = sigma / (4 k_s^2 rho^2),  k_s^2 = 4 k_F / pi,  A = (beta/gamma) / (exp(-eps_c/gamma) - 1).
// With x = A t^2: P, x P'(x) and x^2 P'(x) for x <= 1 directly, for x > 1 in y = 1/x
// (P = y (1 + y) / (1 + y + y^2), x P' = -y (1 + 2y) / (1 + y + y^2)^2,
// x^2 P' = -(1 + 2y) / (1 + y + y^2)^2); then dQ/dt^2 = (beta/gamma)(P + x P') and
// dQ/dA = (beta/gamma) x^2 P' / A^2 need no t^4.
template <typename R> __device__ __forceinline__ void pbe(const Pt<R>& p, R sig, R* e, R* er, R* es) {
  const R kappa = R(0.804), mu = R(0.2195149727645171);
  const R gamma = R((1.0 - 0.69314718055994530942) / (M_PI * M_PI));
  const R bg = R(0.06672455060314922 / ((1.0 - 0.69314718055994530942) / (M_PI * M_PI)));
  const double ckf = 3.0936677262801359310;  // (3 pi^2)^{1/3}
  R ex, dex, ec, dec;
  slater(p, &ex, &dex);
  pw92(p, &ec, &dec);
  const R ir2 = p.ir * p.ir;
  // s^2 = sigma / (4 ckf^2) rho^{-8/3}
  const R s2_s = ir2 * p.ir13 * p.ir13 * R(1.0 / (4.0 * ckf * ckf));  // d s^2 / d sigma
  const R s2 = sig * s2_s;
  const R u = R(1) + mu * s2 / kappa, iu = R(1) / u;
  const R Fx = R(1) + kappa - kappa * iu;
  const R dFx = mu * iu * iu;  // dF_x / d s^2
  // t^2 = sigma pi / (16 ckf) rho^{-7/3}
  const R t2_s = ir2 * p.ir13 * R(M_PI / (16.0 * ckf));  // d t^2 / d sigma
  const R t2 = sig * t2_s;
  const R em1 = expm1(-ec / gamma);
  const R Aa = bg / em1;
  const R dA = Aa * Aa * (em1 + R(1)) / (bg * gamma);  // dA / d eps_c
  const R x = Aa * t2;
  R P, xdP, x2dP;
  if (x <= R(1)) {
    const R iDn = R(1) / (R(1) + x + x * x);
    P = (R(1) + x) * iDn;
    const R dP = -x * (R(2) + x) * iDn * iDn;
    xdP = x * dP;
    x2dP = x * xdP;
  } else {
    const R y = R(1) / x, iDy = R(1) / (R(1) + y + y * y);
    P = y * (R(1) + y) * iDy;
    x2dP = -(R(1) + R(2) * y) * iDy * iDy;
    xdP = y * x2dP;
  }
  const R Q = bg * t2 * P;
  const R H = gamma * log1p(Q);
  const R dHdQ = gamma / (R(1) + Q);
  const R dQ_t2 = bg * (P + xdP);           // dQ / dt^2 at fixed A
  const R dQ_A = bg * x2dP / (Aa * Aa);     // dQ / dA at fixed t^2
  *e = ex * Fx + p.rho * (ec + H);
  // rho derivatives: d s^2/d rho = -(8/3) s^2 / rho, d t^2/d rho = -(7/3) t^2 / rho
  const R dH_r = dHdQ * (dQ_t2 * R(-7.0 / 3.0) * t2 * p.ir + dQ_A * dA * dec);
  *er = dex * Fx + ex * dFx * R(-8.0 / 3.0) * s2 * p.ir + ec + H + p.rho * (dec + dH_r);
  *es = ex * dFx * s2_s + p.rho * dHdQ * dQ_t2 * t2_s;
}

// Kinetic enhancement factors F(s) and F'(s).
template <typename R> __device__ __forceinline__ void kedf_F(int kind, R s, R* F, R* dF) {
  if (kind == 0) { *F = 1; *dF = 0; return; }
  if (kind == 1) {  // revAPBEK
    const R k = R(1.245), mu = R(0.23889);
    const R id = R(1) / (R(1) + mu * s * s / k);
    *F = R(1) + k - k * id;
    *dF = R(2) * mu * s * id * id;
    return;
  }
  // LC94 (PW91 form); at very large s (noisy gradients of a vanishing density) the s^4 term
  // overflows FP32 to infinity, and F and F' correctly go to zero
  const R a = R(0.093907), b = R(76.32), c = R(0.26608), dd = R(-0.0809615), al = R(100), f = R(0.000057767);
  const R ash = asinh(b * s), ex = exp(-al * s * s);
  const R num = R(1) + a * s * ash + (c + dd * ex) * s * s;
  const R den = R(1) + a * s * ash + f * s * s * s * s;
  const R dash = a * ash + a * s * b / sqrt(R(1) + b * b * s * s);
  const R dnum = dash + R(2) * s * (c + dd * ex) - R(2) * al * dd * s * s * s * ex;
  const R dden = dash + R(4) * f * s * s * s;
  const R iden = R(1) / den;
  *F = num * iden;
  *dF = (dnum - num * iden * dden) * iden;
}

// FP64 grid values into and out of the arithmetic type R: for FP32 the conversions work on the
// bit patterns (dd.cuh), so the mixed path's pointwise kernels stay off the FP64 pipe.
template <typename R> __device__ __forceinline__ R narrow(double v);
template <> __device__ __forceinline__ double narrow<double>(double v) { return v; }
template <> __device__ __forceinline__ float narrow<float>(double v) { return float_of_double_bits(v); }
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) { return float_to_double_bits(v); }

// One point of a functional evaluation.  xc_mode: -1 none, 0 LDA, 1 PBE.  kedf: -1 none,
// 0 TF, 1 revAPBEK, 2 LC94.  Returns the local potential part (d e/d rho of both), the
// coefficient multiplying grad rho in the divergence term, and the two energy densities.
template <typename R>
__device__ __forceinline__ void point_functional(R rho, R gx, R gy, R gz, int xc_mode, int xc_pot, int kedf,
                                                 R rho_cut, R* vloc, R* hcoef, R* exc, R* ekin) {
  *vloc = 0; *hcoef = 0; *exc = 0; *ekin = 0;
  if (!(rho >= rho_cut)) return;
  const R sig = gx * gx + gy * gy + gz * gz;
  const Pt<R> p = make_pt(rho);
  if (xc_mode == 0) {
    R ex, dex, ec, dec;
    slater(p, &ex, &dex);
    pw92(p, &ec, &dec);
    if (xc_pot) *vloc += dex + ec + rho * dec;
    *exc = ex + rho * ec;
  } else if (xc_mode == 1) {
    R e, er, es;
    pbe(p, sig, &e, &er, &es);
    if (xc_pot) {
      *vloc += er;
      *hcoef += R(2) * es;
    }
    *exc = e;
  }
  if (kedf >= 0) {
    const R ctf = R(2.8712340001881918);   // (3/10)(3 pi^2)^{2/3}
    const R cs = R(0.16162045967399548);   // 1 / (2 (3 pi^2)^{1/3})
    const R r23 = p.r13 * p.r13;
    const R gn = sqrt(sig);
    const R s = cs * gn * p.ir * p.ir13;  // cs |grad rho| / rho^{4/3}
    R F, dF;
    kedf_F(kedf, s, &F, &dF);
    *ekin = ctf * rho * r23 * F;
    *vloc += ctf * r23 * (R(5.0 / 3.0) * F - R(4.0 / 3.0) * s * dF);
    if (kedf > 0) *hcoef += ctf * cs * p.r13 * dF / (gn > R(1e-30) ? gn : R(1e-30));
  }
}

// ---- small elementwise kernels -----------------------------------------------------------
template <typename T>
__global__ void k_c_to_real(const cplx<T>* __restrict__ c, double* __restrict__ a, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a[i] = (double)c[i].x;
}

// out = a + b + c - Re(d) (any of b, c, d may be NULL).
template <typename T>
__global__ void k_combine(const double* a, const double* b, const double* c, const cplx<T>* d, double sd,
                          double* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = a ? a[i] : 0.0;
    if (b) v += b[i];
    if (c) v += c[i];
    if (d) v += sd * (double)d[i].x;
    out[i] = v;
  }
}

template <typename T>
__global__ void k_scale_c(cplx<T>* __restrict__ a, double s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    a[i].x = (T)(a[i].x * s);
    a[i].y = (T)(a[i].y * s);
  }
}

// partial sums of a[i] * b[i] (b NULL: a[i]; absdiff: |a - b|)
__global__ void k_dot_partial(const double* __restrict__ a, const double* __restrict__ b, long long n, int mode,
                              double* partial) {
  double acc = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (mode == 0) acc += b ? a[i] * b[i] : a[i];
    else acc += fabs(a[i] - b[i]);
  }
  block_sum_store(acc, partial + blockIdx.x);
}

// out[q] = scale * sum_b partial[q][b]: warp q, lane l sums b = l, l + 32, ... and the lane
// sums are combined by a fixed butterfly (deterministic; the block count is a launch constant).
__global__ void k_finalize(const double* __restrict__ partial, int nblk, int nq, double scale, double* out) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= nq) return;
  double t = 0;
  for (int b = lane; b < nblk; b += 32) t += partial[(size_t)q * nblk + b];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) out[q] = t * scale;
}

// out = sum_k c[k] * (a_k + beta * r_k) for the Pulay step; coefs on the device.
__global__ void k_lincomb(const double* const* __restrict__ ins, const double* const* __restrict__ res,
                          const double* __restrict__ coef, int m, double beta, long long n, double* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = 0;
    for (int k = 0; k < m; ++k) v += coef[k] * (ins[k][i] + beta * res[k][i]);
    out[i] = v;
  }
}

__global__ void k_axpy(double* __restrict__ a, const double* __restrict__ b, double alpha, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a[i] += alpha * b[i];
}

__global__ void k_nonfinite(const double* __restrict__ a, long long n, unsigned* status) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(a[i])) { atomicOr(status, ST_NONFINITE); return; }
}

// ---- packed pairs of real fields ------------------------------------------------------------
// One complex transform carries two real fields a and b: with C = FFT(a + i b),
// a(G) = (C(G) + conj C(-G)) / 2 and b(G) = (C(G) - conj C(-G)) / (2 i).  The potential build
// packs the subsystem densities, gradient components and divergence arguments in pairs, so
// that it needs half the FP64 transforms while computing the same quantities.
__device__ __forceinline__ long long neg_index(long long idx, const GridDims& g) {
  const int id = (int)idx;
  const int i3 = id % g.n3;
  const int r = id / g.n3;
  const int i2 = r % g.n2, i1 = r / g.n2;
  const int j1 = i1 ? g.n1 - i1 : 0, j2 = i2 ? g.n2 - i2 : 0, j3 = i3 ? g.n3 - i3 : 0;
  return (long long)((j1 * g.n2 + j2) * g.n3 + j3);
}
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2((double)v.x, (double)v.y); }
__device__ __forceinline__ void unpack2(double2 c, double2 cn, double2* a, double2* b) {
  *a = make_double2(0.5 * (c.x + cn.x), 0.5 * (c.y - cn.y));
  *b = make_double2(0.5 * (c.y + cn.y), -0.5 * (c.x - cn.x));
}
// u + i v for complex u, v
__device__ __forceinline__ double2 pack2(double2 u, double2 v) { return make_double2(u.x - v.y, u.y + v.x); }
// i g f
__device__ __forceinline__ double2 ig_mul(double gc, double2 f) { return make_double2(-gc * f.y, gc * f.x); }

__global__ void k_pack2(const double* __restrict__ a, const double* __restrict__ b, double2* __restrict__ c,
                        long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    c[i] = make_double2(a[i], b ? b[i] : 0.0);
}

// From C = FFT(rho_a + i rho_b) (unscaled): RT (+)= rho_a(G) + rho_b(G); Hartree sums
// sum 4 pi |rho_x(G)|^2 / G^2 of both into partial rows 0 and 1; packed gradient transforms
// Pa = iGx a + i iGy a, Pb = iGx b + i iGy b, Pz = iGz a + i iGz b (Nyquist planes zero).
// Without b, C is rho_a's transform itself, Pb is not written and Pz carries iGz a alone.
__global__ void k_unpack_density(const double2* __restrict__ C, int has_b, double2* __restrict__ RT, int accumulate,
                                 double2* __restrict__ Pa, double2* __restrict__ Pb, double2* __restrict__ Pz,
                                 GridDims g, CellDev c, double inv_nr, double* partial) {
  const long long nr = (long long)g.n1 * g.n2 * g.n3;
  double ea = 0, eb = 0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nr; idx += (long long)gridDim.x * blockDim.x) {
    const Gpt p = gvec(idx, g, c);
    const double2 cv = C[idx];
    double2 a, b;
    if (has_b) {
      unpack2(cv, C[neg_index(idx, g)], &a, &b);
    } else {
      a = cv;
      b = make_double2(0, 0);
    }
    a.x *= inv_nr; a.y *= inv_nr;
    b.x *= inv_nr; b.y *= inv_nr;
    double2 t = make_double2(a.x + b.x, a.y + b.y);
    if (accumulate) t = make_double2(RT[idx].x + t.x, RT[idx].y + t.y);
    RT[idx] = t;
    if (p.g2 > 0 && !p.nyq) {
      const double f = 4.0 * M_PI / p.g2;
      ea += f * (a.x * a.x + a.y * a.y);
      eb += f * (b.x * b.x + b.y * b.y);
    }
    if (Pa) {
      if (p.nyq) {
        Pa[idx] = Pz[idx] = make_double2(0, 0);
        if (has_b) Pb[idx] = make_double2(0, 0);
      } else {
        Pa[idx] = pack2(ig_mul(p.gx, a), ig_mul(p.gy, a));
        if (has_b) Pb[idx] = pack2(ig_mul(p.gx, b), ig_mul(p.gy, b));
        Pz[idx] = pack2(ig_mul(p.gz, a), ig_mul(p.gz, b));
      }
    }
  }
  if (partial) {
    block_sum_store(ea, partial + blockIdx.x);
    block_sum_store(eb, partial + kRedBlocks + blockIdx.x);
  }
}

// Functional of the total density rho_tot = sum_I rho_I whose gradient is the sum of the
// subsystem gradients held in the packed grids of each pair.  Writes vpart (d f / d rho) and
// h = (d f / d grad rho) in hx, hy, hz (real; when there are gradients); energy partial rows
// 0 (xc) and 1 (kinetic).
template <typename R>
__global__ void k_pw_total(const double* __restrict__ rho, GradPacks gp, int xc_mode, int kedf, double rho_cut,
                           double* __restrict__ vpart, double* __restrict__ hx, double* __restrict__ hy,
                           double* __restrict__ hz, long long nr, double* partial) {
  double ax = 0, ak = 0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nr; idx += (long long)gridDim.x * blockDim.x) {
    R x = 0, y = 0, z = 0;
    for (int q = 0; q < gp.npairs; ++q) {
      const double2 pa = gp.a[q][idx], pz = gp.z[q][idx];
      x += narrow<R>(pa.x);
      y += narrow<R>(pa.y);
      z += narrow<R>(pz.x);
      if (gp.has_b[q]) {
        const double2 pb = gp.b[q][idx];
        x += narrow<R>(pb.x);
        y += narrow<R>(pb.y);
        z += narrow<R>(pz.y);
      }
    }
    R v, h, ex, ek;
    point_functional<R>(narrow<R>(rho[idx]), x, y, z, xc_mode, 1, kedf, (R)rho_cut, &v, &h, &ex, &ek);
    if (vpart) vpart[idx] = widen(v);
    if (hx) {
      hx[idx] = widen(h * x);
      hy[idx] = widen(h * y);
      hz[idx] = widen(h * z);
    }
    ax += widen(ex);
    ak += widen(ek);
  }
  block_sum_store(ax, partial + blockIdx.x);
  block_sum_store(ak, partial + kRedBlocks + blockIdx.x);
}

// The kinetic functional (and, for energies, the xc functional) of the two densities of a
// pair: w_x = vpart_tot - d f_kin / d rho_x (the pointwise part of v~_kin[rho] - v~_kin[rho_x]
// with the xc part of the total), and, in place of the packed gradients, the packed
// divergence arguments d_x = h_tot - h_x.  Energy partial rows 0/1 (xc/kin of a), 2/3 (b).
// The divergence arguments go to Da, Db, Dz in precision TD (FP64: in place over Pa, Pb, Pz;
// FP32: separate grids for the single-precision transforms of the mixed path).
template <typename TD>
__global__ void k_pw_pair(const double* __restrict__ ra, const double* __restrict__ rb, const double2* Pa,
                          const double2* Pb, const double2* Pz, cplx<TD>* Da, cplx<TD>* Db, cplx<TD>* Dz,
                          const double* __restrict__ hx, const double* __restrict__ hy,
                          const double* __restrict__ hz, const double* __restrict__ vtot, int xc_mode, int kedf,
                          double rho_cut, double* __restrict__ wa, double* __restrict__ wb, int write_d, long long nr,
                          double* partial) {
  double xa = 0, ka = 0, xb = 0, kb = 0;
  const bool has_b = rb != nullptr;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nr; idx += (long long)gridDim.x * blockDim.x) {
    double2 pa = make_double2(0, 0), pb = make_double2(0, 0), pz = make_double2(0, 0);
    if (Pa) {
      pa = Pa[idx];
      pz = Pz[idx];
      if (has_b) pb = Pb[idx];
    }
    const TD pax = narrow<TD>(pa.x), pay = narrow<TD>(pa.y), pzx = narrow<TD>(pz.x);
    const TD pbx = narrow<TD>(pb.x), pby = narrow<TD>(pb.y), pzy = narrow<TD>(pz.y);
    TD va, ha, ex, ek;
    point_functional<TD>(narrow<TD>(ra[idx]), pax, pay, pzx, xc_mode, 0, kedf, (TD)rho_cut, &va, &ha, &ex, &ek);
    xa += widen(ex);
    ka += widen(ek);
    TD vb = 0, hb = 0;
    if (has_b) {
      point_functional<TD>(narrow<TD>(rb[idx]), pbx, pby, pzy, xc_mode, 0, kedf, (TD)rho_cut, &vb, &hb, &ex, &ek);
      xb += widen(ex);
      kb += widen(ek);
    }
    const TD vt = vtot ? narrow<TD>(vtot[idx]) : TD(0);
    if (wa) wa[idx] = widen(vt - va);
    if (wb) wb[idx] = widen(vt - vb);
    if (write_d) {
      const TD tx = narrow<TD>(hx[idx]), ty = narrow<TD>(hy[idx]), tz = narrow<TD>(hz[idx]);
      Da[idx] = mk<TD>(tx - ha * pax, ty - ha * pay);
      if (has_b) Db[idx] = mk<TD>(tx - hb * pbx, ty - hb * pby);
      Dz[idx] = mk<TD>(tz - ha * pzx, has_b ? tz - hb * pzy : TD(0));
    }
  }
  block_sum_store(xa, partial + blockIdx.x);
  block_sum_store(ka, partial + kRedBlocks + blockIdx.x);
  block_sum_store(xb, partial + 2 * kRedBlocks + blockIdx.x);
  block_sum_store(kb, partial + 3 * kRedBlocks + blockIdx.x);
}

// Reciprocal-space part of the potentials of a pair: F = Va + i Vb with
// Vx(G) = v_H(G) - i G . d_x(G), v_H = 4 pi RT / G^2 (RT = rho_tot(G), scaled), the d_x
// unpacked from the forward transforms Da (x, y of a), Db (x, y of b), Dz (z of a and b),
// unscaled; without gradients Va = Vb = v_H.  Hartree sum of rho_tot into partial row 0.
template <typename TD>
__global__ void k_assemble_pair(const double2* __restrict__ RT, const cplx<TD>* __restrict__ Da,
                                const cplx<TD>* __restrict__ Db, const cplx<TD>* __restrict__ Dz, int has_b,
                                cplx<TD>* __restrict__ F, GridDims g, CellDev c, double inv_nr, double* partial) {
  const long long nr = (long long)g.n1 * g.n2 * g.n3;
  double eh = 0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nr; idx += (long long)gridDim.x * blockDim.x) {
    const Gpt p = gvec(idx, g, c);
    double2 vh = make_double2(0, 0);
    if (p.g2 > 0 && !p.nyq) {
      const double f = 4.0 * M_PI / p.g2;
      const double2 r = RT[idx];
      vh = make_double2(f * r.x, f * r.y);
      eh += f * (r.x * r.x + r.y * r.y);
    }
    double2 va = vh, vb = vh;
    if (Da && !p.nyq) {
      const long long jn = neg_index(idx, g);
      double2 ax, ay, az, bx = make_double2(0, 0), by = make_double2(0, 0), bz = make_double2(0, 0);
      unpack2(to_d2(Da[idx]), to_d2(Da[jn]), &ax, &ay);
      if (has_b) {
        unpack2(to_d2(Db[idx]), to_d2(Db[jn]), &bx, &by);
        unpack2(to_d2(Dz[idx]), to_d2(Dz[jn]), &az, &bz);
      } else {
        const double2 t = to_d2(Dz[idx]), tn = to_d2(Dz[jn]);
        az = make_double2(0.5 * (t.x + tn.x), 0.5 * (t.y - tn.y));
      }
      // i G . d / N_r
      const double dar = p.gx * ax.x + p.gy * ay.x + p.gz * az.x, dai = p.gx * ax.y + p.gy * ay.y + p.gz * az.y;
      const double dbr = p.gx * bx.x + p.gy * by.x + p.gz * bz.x, dbi = p.gx * bx.y + p.gy * by.y + p.gz * bz.y;
      va = make_double2(vh.x + dai * inv_nr, vh.y - dar * inv_nr);
      vb = make_double2(vh.x + dbi * inv_nr, vh.y - dbr * inv_nr);
    }
    if (F) {
      const double2 o = has_b ? pack2(va, vb) : va;
      F[idx] = mk<TD>((TD)o.x, (TD)o.y);
    }
  }
  if (partial) block_sum_store(eh, partial + blockIdx.x);
}

// veff_x = vloc + Re/Im F (inverse-transformed reciprocal part) + w_x for the pair's
// subsystems (either output may be NULL).
template <typename TD>
__global__ void k_finish_pair(const cplx<TD>* __restrict__ F, const double* __restrict__ vloc, double* va,
                              double* vb, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 f = to_d2(F[i]);
    const double vl = vloc[i];
    if (va) va[i] = vl + f.x + va[i];
    if (vb) vb[i] = vl + f.y + vb[i];
  }
}

// ---- ultrasoft-like augmentation (Appendix: subsystem-specific projectors) -------------------
// Augmentation charges q_ij g_a(r) with g_a the normalised Gaussian (pi s^2)^{-3/2}
// exp(-|r - R_a|^2 / s^2): g_a(G) = (1/Omega) exp(-G^2 s^2 / 4) exp(-i G.R_a), Nyquist planes zero.

// rho_aug(G) = sum_a c_a g_a(G) into A (complex grid), for the inverse transform.
__global__ void k_aug_density_g(double2* __restrict__ A, GridDims g, CellDev c, const double* __restrict__ pos,
                                const double* __restrict__ coef, int natoms, double sigma) {
  const long long nr = (long long)g.n1 * g.n2 * g.n3;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nr; idx += (long long)gridDim.x * blockDim.x) {
    const Gpt p = gvec(idx, g, c);
    double re = 0, im = 0;
    if (!p.nyq) {
      const double f = exp(-p.g2 * sigma * sigma / 4.0) / c.omega;
      for (int a = 0; a < natoms; ++a) {
        double sn, cs;
        sincos(p.gx * pos[3 * a] + p.gy * pos[3 * a + 1] + p.gz * pos[3 * a + 2], &sn, &cs);
        re += f * coef[a] * cs;
        im -= f * coef[a] * sn;
      }
    }
    A[idx] = make_double2(re, im);
  }
}

// Screened coupling of each atom: Dscr_a = D + q int v g_a, with
// int v g_a = Re sum_G v(G) exp(-G^2 s^2 / 4) exp(+i G.R_a) (Parseval; VG = v's forward transform
// scaled by 1/N_r).  One CTA per atom; D and q are np x np (row-major).
__global__ void k_aug_screening(const double2* __restrict__ VG, GridDims g, CellDev c, const double* __restrict__ pos,
                                double sigma, KbBlock D, KbBlock q, double* __restrict__ Dscr) {
  const long long nr = (long long)g.n1 * g.n2 * g.n3;
  const int a = blockIdx.x;
  const double x = pos[3 * a], y = pos[3 * a + 1], z = pos[3 * a + 2];
  double acc = 0;
  for (long long idx = threadIdx.x; idx < nr; idx += blockDim.x) {
    const Gpt p = gvec(idx, g, c);
    if (p.nyq) continue;
    double sn, cs;
    sincos(p.gx * x + p.gy * y + p.gz * z, &sn, &cs);
    const double2 v = VG[idx];
    acc += exp(-p.g2 * sigma * sigma / 4.0) * (v.x * cs - v.y * sn);
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    red[0] = t;
  }
  __syncthreads();
  const double ov = red[0];
  for (int e = threadIdx.x; e < D.np * D.np; e += blockDim.x) Dscr[(size_t)a * D.np * D.np + e] = D.d[e] + q.d[e] * ov;
}

// ---- launch wrappers ------------------------------------------------------------------------
__global__ void k_symmetrize(const double* __restrict__ in, double* __restrict__ out, GridDims g, SymOps ops) {
  const long long nr = (long long)g.n1 * g.n2 * g.n3;
  const double w = 1.0 / (double)ops.n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nr; i += (long long)gridDim.x * blockDim.x) {
    const int i3 = (int)(i % g.n3);
    const long long t = i / g.n3;
    const int i2 = (int)(t % g.n2), i1 = (int)(t / g.n2);
    double acc = 0;
    for (int o = 0; o < ops.n; ++o) {
      const int m = ops.mask[o];
      const int j1 = (m & 1) ? (g.n1 - i1) % g.n1 : i1;
      const int j2 = (m & 2) ? (g.n2 - i2) % g.n2 : i2;
      const int j3 = (m & 4) ? (g.n3 - i3) % g.n3 : i3;
      acc += in[((long long)j1 * g.n2 + j2) * g.n3 + j3];
    }
    out[i] = acc * w;
  }
}

static int gs(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

void grid_aug_density_g(double2* A, const GridDims& g, const CellDev& c, const double* pos, const double* coef,
                        int natoms, double sigma, cudaStream_t st) {
  const long long nr = (long long)g.n1 * g.n2 * g.n3;
  count_launches(1);
  ProfScope prof_("k_aug_density_g", st);
  k_aug_density_g<<<gs(nr), 256, 0, st>>>(A, g, c, pos, coef, natoms, sigma);
}
void grid_aug_screening(const double2* VG, const GridDims& g, const CellDev& c, const double* pos, int natoms,
                        double sigma, const KbBlock& D, const KbBlock& q, double* Dscr, cudaStream_t st) {
  if (natoms <= 0) return;
  count_launches(1);
  ProfScope prof_("k_aug_screening", st);
  k_aug_screening<<<natoms, 512, 0, st>>>(VG, g, c, pos, sigma, D, q, Dscr);
}

void grid_vloc_g(double2* V, const GridDims& g, const CellDev& c, const double* pos, const double* Z, int natoms,
                 double rc, cudaStream_t st) {
  const long long nr = (long long)g.n1 * g.n2 * g.n3;
  count_launches(1);
  k_vloc_g<<<gs(nr), 256, 0, st>>>(V, g, c, pos, Z, natoms, rc);
}
template <typename T>
void grid_c_to_real(const cplx<T>* c, double* a, long long n, cudaStream_t st) {
  count_launches(1);
  k_c_to_real<T><<<gs(n), 256, 0, st>>>(c, a, n);
}
template <typename T>
void grid_combine(const double* a, const double* b, const double* c, const cplx<T>* d, double sd, double* out,
                  long long n, cudaStream_t st) {
  count_launches(1);
  ProfScope prof_("k_combine", st);
  k_combine<T><<<gs(n), 256, 0, st>>>(a, b, c, d, sd, out, n);
}
template <typename T>
void grid_scale_c(cplx<T>* a, double s, long long n, cudaStream_t st) {
  count_launches(1);
  k_scale_c<T><<<gs(n), 256, 0, st>>>(a, s, n);
}
template void grid_scale_c<float>(float2*, double, long long, cudaStream_t);
template void grid_scale_c<double>(double2*, double, long long, cudaStream_t);
void grid_dot_partial(const double* a, const double* b, long long n, int mode, double* partial, cudaStream_t st) {
  count_launches(1);
  k_dot_partial<<<kRedBlocks, kRedThreads, 0, st>>>(a, b, n, mode, partial);
}
void grid_finalize(const double* partial, int nq, double scale, double* out, cudaStream_t st) {
  count_launches(1);
  k_finalize<<<1, 32 * nq, 0, st>>>(partial, kRedBlocks, nq, scale, out);
}
void grid_lincomb(const double* const* ins, const double* const* res, const double* coef, int m, double beta,
                  long long n, double* out, cudaStream_t st) {
  count_launches(1);
  k_lincomb<<<gs(n), 256, 0, st>>>(ins, res, coef, m, beta, n, out);
}
void grid_axpy(double* a, const double* b, double alpha, long long n, cudaStream_t st) {
  count_launches(1);
  k_axpy<<<gs(n), 256, 0, st>>>(a, b, alpha, n);
}
void grid_symmetrize(const double* in, double* out, const GridDims& g, const SymOps& ops, cudaStream_t st) {
  const long long nr = (long long)g.n1 * g.n2 * g.n3;
  count_launches(1);
  k_symmetrize<<<gs(nr), 256, 0, st>>>(in, out, g, ops);
}
void grid_nonfinite(const double* a, long long n, unsigned* status, cudaStream_t st) {
  count_launches(1);
  ProfScope prof_("k_nonfinite", st);
  k_nonfinite<<<gs(n), 256, 0, st>>>(a, n, status);
}
void grid_pack2(const double* a, const double* b, double2* c, long long n, cudaStream_t st) {
  count_launches(1);
  ProfScope prof_("k_pack2", st);
  k_pack2<<<gs(n), 256, 0, st>>>(a, b, c, n);
}
void grid_unpack_density(const double2* C, int has_b, double2* RT, int accumulate, double2* Pa, double2* Pb,
                         double2* Pz, const GridDims& g, const CellDev& c, double* partial, cudaStream_t st) {
  count_launches(1);
  ProfScope prof_("k_unpack_density", st);
  k_unpack_density<<<kRedBlocks, kRedThreads, 0, st>>>(C, has_b, RT, accumulate, Pa, Pb, Pz, g, c,
                                                       1.0 / ((double)g.n1 * g.n2 * g.n3), partial);
}
void grid_pw_total(const double* rho, const GradPacks& gp, int xc_mode, int kedf, double rho_cut, double* vpart,
                   double* hx, double* hy, double* hz, long long nr, double* partial, bool fp32, cudaStream_t st) {
  count_launches(1);
  ProfScope prof_("k_pw_total", st);
  if (fp32)
    k_pw_total<float><<<kRedBlocks, kRedThreads, 0, st>>>(rho, gp, xc_mode, kedf, rho_cut, vpart, hx, hy, hz, nr,
                                                          partial);
  else
    k_pw_total<double><<<kRedBlocks, kRedThreads, 0, st>>>(rho, gp, xc_mode, kedf, rho_cut, vpart, hx, hy, hz, nr,
                                                           partial);
}
template <typename TD>
void grid_pw_pair(const double* ra, const double* rb, const double2* Pa, const double2* Pb, const double2* Pz,
                  cplx<TD>* Da, cplx<TD>* Db, cplx<TD>* Dz, const double* hx, const double* hy, const double* hz,
                  const double* vtot, int xc_mode, int kedf, double rho_cut, double* wa, double* wb, int write_d,
                  long long nr, double* partial, cudaStream_t st) {
  count_launches(1);
  ProfScope prof_("k_pw_pair", st);
  k_pw_pair<TD><<<kRedBlocks, kRedThreads, 0, st>>>(ra, rb, Pa, Pb, Pz, Da, Db, Dz, hx, hy, hz, vtot, xc_mode, kedf,
                                                    rho_cut, wa, wb, write_d, nr, partial);
}
template <typename TD>
void grid_assemble_pair(const double2* RT, const cplx<TD>* Da, const cplx<TD>* Db, const cplx<TD>* Dz, int has_b,
                        cplx<TD>* F, const GridDims& g, const CellDev& c, double* partial, cudaStream_t st) {
  count_launches(1);
  ProfScope prof_("k_assemble_pair", st);
  k_assemble_pair<TD><<<kRedBlocks, kRedThreads, 0, st>>>(RT, Da, Db, Dz, has_b, F, g, c,
                                                          1.0 / ((double)g.n1 * g.n2 * g.n3), partial);
}
template <typename TD>
void grid_finish_pair(const cplx<TD>* F, const double* vloc, double* va, double* vb, long long n, cudaStream_t st) {
  count_launches(1);
  ProfScope prof_("k_finish_pair", st);
  k_finish_pair<TD><<<gs(n), 256, 0, st>>>(F, vloc, va, vb, n);
}
int grid_red_blocks() { return kRedBlocks; }

#define FDE_GRID_INST(T)                                                                                       \
  template void launch_fft3d<T>(cplx<T>*, const GridDims&, const FftPlans<T>&, int, cudaStream_t);             \
  template void grid_c_to_real<T>(const cplx<T>*, double*, long long, cudaStream_t);                           \
  template void grid_combine<T>(const double*, const double*, const double*, const cplx<T>*, double, double*,   \
                                long long, cudaStream_t);                                                      \
  template void grid_pw_pair<T>(const double*, const double*, const double2*, const double2*, const double2*,   \
                                cplx<T>*, cplx<T>*, cplx<T>*, const double*, const double*, const double*,       \
                                const double*, int, int, double, double*, double*, int, long long, double*,      \
                                cudaStream_t);                                                                 \
  template void grid_assemble_pair<T>(const double2*, const cplx<T>*, const cplx<T>*, const cplx<T>*, int,      \
                                      cplx<T>*, const GridDims&, const CellDev&, double*, cudaStream_t);        \
  template void grid_finish_pair<T>(const cplx<T>*, const double*, double*, double*, long long, cudaStream_t);
FDE_GRID_INST(float)
FDE_GRID_INST(double)

}  // namespace fde
