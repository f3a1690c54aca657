// precond.cu -- learned per-G preconditioner of the block eigensolver (Eq. KS).
//
// W_jG = K(y) exp(o_jG) R_jG, K the kinetic (Teter-Payne-Allan) preconditioner,
// y = |k+G|^2/2 / T_j, and o = MLP(f) a per-G network of three tanh layers of width 64 and
// a linear output on f = (log(1 + y), log T_j, |R_jG| / rms_G |R_j|).  Inference reads
// bfloat16 weights and accumulates in FP32; training keeps FP32 master weights, evaluates
// the loss sum_j min_a |a m R_j - D_j|^2 / |D_j|^2 (a complex: the eigensolver's Rayleigh-Ritz
// step rescales each preconditioned residual, so only its direction counts) and its gradient
// with per-block partial sums reduced in a fixed order, and takes Adam steps.  The optimal
// a_j = <m R_j, D_j> / |m R_j|^2 comes from a first pass; by the envelope theorem the
// gradient of the minimised loss is that of |a m R - D|^2 at fixed a.
#include <cuda_bf16.h>
#include <algorithm>
#include <math.h>

#include "precond.h"
#include "prof.h"
#include "tc.cuh"

namespace fde {

// parameter layout (floats): W1[64][3] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[64] b4[1]
constexpr int kH = kPrecondWidth;
constexpr int oW1 = 0, ob1 = oW1 + kH * 3, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kH * kH, oW4 = ob3 + kH, ob4 = oW4 + kH;
static_assert(ob4 + 1 == kPrecondParams, "parameter count");

__device__ __forceinline__ float tpa_f(float y) {
  const float p = 27.f + y * (18.f + y * (12.f + y * 8.f));
  return p / (p + 16.f * y * y * y * y);
}

// Load the weights (bf16 or fp32 source) into shared memory as float.
__device__ __forceinline__ void load_weights(float* s, const __nv_bfloat16* wb, const float* wf) {
  for (int i = threadIdx.x; i < kPrecondParams; i += blockDim.x) s[i] = wb ? __bfloat162float(wb[i]) : wf[i];
  __syncthreads();
}

__device__ __forceinline__ void features(float kin, float tb, float amp, float rms, float f[3], float* y) {
  *y = kin / fmaxf(tb, 1e-12f);
  f[0] = log1pf(*y);
  f[1] = logf(fmaxf(tb, 1e-12f));
  f[2] = amp / fmaxf(rms, 1e-30f);
}

// Forward pass of one element; keeps the three hidden layers.
__device__ __forceinline__ float mlp_forward(const float* w, const float f[3], float h1[kH], float h2[kH], float h3[kH]) {
#pragma unroll
  for (int i = 0; i < kH; ++i) {
    float a = w[ob1 + i] + w[oW1 + 3 * i] * f[0] + w[oW1 + 3 * i + 1] * f[1] + w[oW1 + 3 * i + 2] * f[2];
    h1[i] = tanhf(a);
  }
#pragma unroll
  for (int i = 0; i < kH; ++i) {
    float a = w[ob2 + i];
    const float4* row = reinterpret_cast<const float4*>(w + oW2 + kH * i);
#pragma unroll
    for (int q = 0; q < kH / 4; ++q) {
      const float4 v = row[q];
      a += v.x * h1[4 * q] + v.y * h1[4 * q + 1] + v.z * h1[4 * q + 2] + v.w * h1[4 * q + 3];
    }
    h2[i] = tanhf(a);
  }
#pragma unroll
  for (int i = 0; i < kH; ++i) {
    float a = w[ob3 + i];
    const float4* row = reinterpret_cast<const float4*>(w + oW3 + kH * i);
#pragma unroll
    for (int q = 0; q < kH / 4; ++q) {
      const float4 v = row[q];
      a += v.x * h2[4 * q] + v.y * h2[4 * q + 1] + v.z * h2[4 * q + 2] + v.w * h2[4 * q + 3];
    }
    h3[i] = tanhf(a);
  }
  float o = w[ob4];
#pragma unroll
  for (int k = 0; k < kH; ++k) o += w[oW4 + k] * h3[k];
  return o;
}

// W[j][g] = m_jg R[j][g] for nb rows; tband[j] band kinetic energy, sumsq[j] = sum_g |R_jg|^2.
template <typename T>
__global__ void __launch_bounds__(128)
k_precond_apply(const cplx<T>* __restrict__ R, int ldr, const T* __restrict__ kin, const double* __restrict__ tband,
                const double* __restrict__ sumsq, int K, const __nv_bfloat16* __restrict__ wb, cplx<T>* __restrict__ W,
                int ldw) {
  __shared__ __align__(16) float w[kPrecondParams + 3];
  load_weights(w, wb, nullptr);
  const int j = blockIdx.y;
  const float tb = (float)tband[j];
  const float rms = (float)sqrt(sumsq[j] / (double)K);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    const cplx<T> r = R[(size_t)j * ldr + g];
    const float amp = sqrtf((float)r.x * (float)r.x + (float)r.y * (float)r.y);
    float f[3], y;
    features((float)kin[g], tb, amp, rms, f, &y);
    float ha[kH], hb[kH];
    const float o = mlp_forward(w, f, ha, hb, ha);  // the third layer reuses the first's registers
    const float m = tpa_f(y) * expf(o);
    W[(size_t)j * ldw + g] = mk<T>((T)(m * (float)r.x), (T)(m * (float)r.y));
  }
}

// ---- inference on the tensor cores ----------------------------------------------------------
// The two 64 x 64 hidden layers as BF16 tcgen05 MMAs (kind::f16, M = 128 points, N = 64
// neurons, K = 16 per MMA, FP32 accumulation in tensor memory).  The weights are the bf16
// inference weights, so only the activations are rounded: each is split h = hi + lo with
// hi = bf16(h) and lo = bf16(h - hi) (|h - hi - lo| <= 2^-18 |h|), and a layer is W hi + W lo,
// two passes of four MMAs.  The first layer (three inputs), the tanh of every layer, the
// output layer and the multiplier run on the CUDA cores, one thread per point.  Persistent
// CTAs of 128 threads loop over tiles of 128 points (consecutive G of one band); thread t owns
// point t of a tile, which is row t of the A operand and lane t of the accumulator.
// tanh(x) = (e^{2x} - 1) / (e^{2x} + 1) with the hardware exponential and division
// (absolute error ~2e-7), the argument clamped to |x| <= 15 where tanh is 1 in FP32.
constexpr int kPcThreads = 128;
constexpr int kPcCtasPerSm = 4;
constexpr int kPcAct = kPcThreads * 128;  // bytes of one 128 x 64 bf16 activation tile
constexpr int kPcW = kH * 128;            // bytes of one 64 x 64 bf16 weight tile
constexpr int kPcSmem = 1024 + 2 * kPcAct + 2 * kPcW;
constexpr int kPcTmemCols = 64;
// kind::f16 instruction descriptor: D f32 (bits 4-5 = 1), A and B bf16 (bits 7-9, 10-12 = 1),
// both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kPcIdesc =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kH / 8) << 17) | ((uint32_t)(kPcThreads / 16) << 24);
// small parameters in shared memory (float): W1, b1, b2, b3, W4, b4
constexpr int sW1 = 0, sb1 = sW1 + 3 * kH, sb2 = sb1 + kH, sb3 = sb2 + kH, sW4 = sb3 + kH, sb4 = sW4 + kH,
              sEnd = sb4 + 1;

__device__ unsigned g_pc_status;
__device__ long long g_pc_spin = kTcSpin;

__device__ __forceinline__ float tanh_tc(float x) {
  const float t = __expf(2.f * fminf(fmaxf(x, -15.f), 15.f));
  return __fdividef(t - 1.f, t + 1.f);
}
__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) {  // a in the low half
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}
// Row t of the hi and lo activation tiles (128-byte rows, 16-byte chunks swizzled by t mod 8).
__device__ __forceinline__ void store_split(uint32_t a_hi, uint32_t a_lo, int t, const float* h) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    uint32_t hb[4], lb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float x0 = h[8 * c + 2 * q], x1 = h[8 * c + 2 * q + 1];
      hb[q] = bf16x2_bits(x0, x1);
      const __nv_bfloat162 hv = *reinterpret_cast<const __nv_bfloat162*>(&hb[q]);
      lb[q] = bf16x2_bits(x0 - __low2float(hv), x1 - __high2float(hv));
    }
    const uint32_t off = (uint32_t)(t * 128 + ((c ^ (t & 7)) << 4));
    st_shared_v4(a_hi + off, make_uint4(hb[0], hb[1], hb[2], hb[3]));
    st_shared_v4(a_lo + off, make_uint4(lb[0], lb[1], lb[2], lb[3]));
  }
}
__device__ __forceinline__ void mma_bf16(uint32_t dt, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
      "l"(a), "l"(b), "r"(kPcIdesc), "r"(acc)
      : "memory");
}

template <typename T>
__global__ void __launch_bounds__(kPcThreads, kPcCtasPerSm)
k_precond_apply_tc(const cplx<T>* __restrict__ R, int ldr, const T* __restrict__ kin, const double* __restrict__ tband,
                   const double* __restrict__ sumsq, int nb, int K, const __nv_bfloat16* __restrict__ wb,
                   cplx<T>* __restrict__ W, int ldw) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ float ws[sEnd];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag, drained;
  const int t = threadIdx.x, warp = t >> 5;
  const uint32_t base = (su32(smem_raw) + 1023u) & ~1023u;
  const uint32_t a_hi = base, a_lo = base + kPcAct, w2s = base + 2 * kPcAct, w3s = w2s + kPcW;
  for (int i = t; i < 3 * kH; i += kPcThreads) ws[sW1 + i] = __bfloat162float(wb[oW1 + i]);
  for (int i = t; i < kH; i += kPcThreads) {
    ws[sb1 + i] = __bfloat162float(wb[ob1 + i]);
    ws[sb2 + i] = __bfloat162float(wb[ob2 + i]);
    ws[sb3 + i] = __bfloat162float(wb[ob3 + i]);
    ws[sW4 + i] = __bfloat162float(wb[oW4 + i]);
  }
  if (t == 0) ws[sb4] = __bfloat162float(wb[ob4]);
  // B operands: row i of W2 / W3 (the weights into neuron i), K-major, 128-byte swizzle
  for (int q = t; q < 2 * kH * 8; q += kPcThreads) {
    const int m = q / (kH * 8), r = (q >> 3) % kH, c = q & 7;
    const uint4 v = reinterpret_cast<const uint4*>(wb + (m ? oW3 : oW2) + r * kH)[c];
    st_shared_v4((m ? w3s : w2s) + (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)), v);
  }
  if (t == 0) {
    mbar_init(su32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                 "r"(kPcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
  const int tiles_per_band = (K + kPcThreads - 1) / kPcThreads;
  const long long ntiles = (long long)nb * tiles_per_band;
  unsigned phase = 0;
  bool ok = true;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = (int)(tile / tiles_per_band);
    const int g = (int)(tile - (long long)j * tiles_per_band) * kPcThreads + t;
    const bool valid = g < K;
    const cplx<T> r = valid ? R[(size_t)j * ldr + g] : mk<T>(0, 0);
    const float rx = (float)r.x, ry = (float)r.y;
    float f[3], y;
    features(valid ? (float)kin[g] : 0.f, (float)tband[j], sqrtf(rx * rx + ry * ry),
             (float)sqrt(sumsq[j] / (double)K), f, &y);
    float h[kH];
#pragma unroll
    for (int i = 0; i < kH; ++i)
      h[i] = tanh_tc(ws[sb1 + i] + ws[sW1 + 3 * i] * f[0] + ws[sW1 + 3 * i + 1] * f[1] + ws[sW1 + 3 * i + 2] * f[2]);
    store_split(a_hi, a_lo, t, h);
#pragma unroll 1
    for (int layer = 0; layer < 2; ++layer) {
      tc_fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      if (t == 0) {
        tc_fence_after();
        const uint32_t wsm = layer ? w3s : w2s;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) mma_bf16(tmem, sdesc(a_hi + 32u * kk), sdesc(wsm + 32u * kk), kk > 0 ? 1u : 0u);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) mma_bf16(tmem, sdesc(a_lo + 32u * kk), sdesc(wsm + 32u * kk), 1u);
        mma_commit(su32(&bar));
        if (!mbar_wait(su32(&bar), phase, g_pc_spin)) abort_flag = 1;
      }
      __syncthreads();
      phase ^= 1u;
      if (abort_flag) {
        ok = false;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int c = 0; c < kH; c += 16) tmem_ld16(trow + (uint32_t)c, h + c);
      const float* bl = ws + (layer ? sb3 : sb2);
#pragma unroll
      for (int i = 0; i < kH; ++i) h[i] = tanh_tc(h[i] + bl[i]);
      if (layer == 0) store_split(a_hi, a_lo, t, h);  // the MMAs that read the tile have completed
    }
    if (!ok) break;
    float o = ws[sb4];
#pragma unroll
    for (int k = 0; k < kH; ++k) o += ws[sW4 + k] * h[k];
    const float m = tpa_f(y) * expf(o);
    if (valid) W[(size_t)j * ldw + g] = mk<T>((T)(m * rx), (T)(m * ry));
  }
  // after a timeout: wait (bounded) for the outstanding MMAs before tensor memory is released
  if (t == 0) drained = ok ? 1 : (mbar_wait(su32(&bar), phase ^ 1u) ? 1 : 0);
  tc_fence_before();
  __syncthreads();
  if (!ok && t == 0) atomicOr(&g_pc_status, drained ? ST_TIMEOUT : (ST_TIMEOUT | ST_TMEM_HELD));
  if (warp == 0 && drained) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPcTmemCols) : "memory");
  }
}

// Per-band sums for the optimal scale a_j: <m R_j, D_j> (re, im) and |m R_j|^2 with the FP32
// master weights; CTA (b, j) strides over G, block sums in a fixed order into
// part[(j * kAlphaBlocks + b) * 3 + {0, 1, 2}].
constexpr int kAlphaBlocks = 32;
constexpr int kAlphaThreads = 128;
template <typename T>
__global__ void __launch_bounds__(kAlphaThreads)
k_precond_alpha(const cplx<T>* __restrict__ R, const cplx<T>* __restrict__ D, int K, const T* __restrict__ kin,
                const double* __restrict__ tband, const double* __restrict__ sumsq, const float* __restrict__ wf,
                double* __restrict__ part) {
  __shared__ __align__(16) float w[kPrecondParams + 3];
  __shared__ double red[3][kAlphaThreads];
  load_weights(w, nullptr, wf);
  const int j = blockIdx.y;
  const float tb = (float)tband[j];
  const float rms = (float)sqrt(sumsq[j] / (double)K);
  double cr = 0, ci = 0, nn = 0;
  for (int g = blockIdx.x * kAlphaThreads + threadIdx.x; g < K; g += kAlphaBlocks * kAlphaThreads) {
    const cplx<T> r = R[(size_t)j * K + g], d = D[(size_t)j * K + g];
    const float rx = (float)r.x, ry = (float)r.y;
    float f[3], y;
    features((float)kin[g], tb, sqrtf(rx * rx + ry * ry), rms, f, &y);
    float ha[kH], hb[kH];
    const float m = tpa_f(y) * expf(mlp_forward(w, f, ha, hb, ha));
    cr += (double)(m * (rx * (float)d.x + ry * (float)d.y));
    ci += (double)(m * (rx * (float)d.y - ry * (float)d.x));
    nn += (double)(m * m * (rx * rx + ry * ry));
  }
  red[0][threadIdx.x] = cr;
  red[1][threadIdx.x] = ci;
  red[2][threadIdx.x] = nn;
  __syncthreads();
  for (int h = kAlphaThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 3) part[((size_t)j * kAlphaBlocks + blockIdx.x) * 3 + threadIdx.x] = red[threadIdx.x][0];
}
// a_j = <m R_j, D_j> / |m R_j|^2 (0 when m R_j vanishes); alpha[2 j], alpha[2 j + 1].
__global__ void k_precond_alpha_fin(const double* __restrict__ part, int nb, double* __restrict__ alpha) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  double cr = 0, ci = 0, nn = 0;
  for (int b = 0; b < kAlphaBlocks; ++b) {
    const double* q = part + ((size_t)j * kAlphaBlocks + b) * 3;
    cr += q[0];
    ci += q[1];
    nn += q[2];
  }
  alpha[2 * j] = nn > 0 ? cr / nn : 0.0;
  alpha[2 * j + 1] = nn > 0 ? ci / nn : 0.0;
}

// Loss and gradient: one CTA of kGradBlock threads handles kGradBlock elements (rows of
// (band j, G)); per-block partial gradients go to part[blk][0..kPrecondParams), the partial
// loss to part[blk][kPrecondParams].  Activations and back-propagated errors live in
// dynamic shared memory, [kGradBlock][kH + 1] each.
constexpr int kGradBlock = 64;
constexpr int kGradPitch = kH + 1;
constexpr size_t kGradSmem =
    sizeof(float) * ((size_t)kPrecondParams + 3 + 6 * (size_t)kGradBlock * kGradPitch + 6 * (size_t)kGradBlock);

template <typename T>
__global__ void __launch_bounds__(kGradBlock)
k_precond_grad(const cplx<T>* __restrict__ R, const cplx<T>* __restrict__ D, int K, int nb,
               const T* __restrict__ kin, const double* __restrict__ tband, const double* __restrict__ sumsq,
               const double* __restrict__ dnorm2, const double* __restrict__ alpha, const float* __restrict__ wf,
               float* __restrict__ part) {
  extern __shared__ __align__(16) float smem[];
  float* w = smem;
  float* base = smem + ((kPrecondParams + 3 + 3) / 4) * 4;
  float* sh1 = base;
  float* sh2 = sh1 + kGradBlock * kGradPitch;
  float* sh3 = sh2 + kGradBlock * kGradPitch;
  float* sd1 = sh3 + kGradBlock * kGradPitch;
  float* sd2 = sd1 + kGradBlock * kGradPitch;
  float* sd3 = sd2 + kGradBlock * kGradPitch;
  float* sf = sd3 + kGradBlock * kGradPitch;  // [kGradBlock][4]
  float* sgo = sf + 4 * kGradBlock;
  float* sloss = sgo + kGradBlock;
  load_weights(w, nullptr, wf);
  const long long e = (long long)blockIdx.x * kGradBlock + threadIdx.x;
  const long long total = (long long)nb * K;
  const int t = threadIdx.x;
  float* h1 = sh1 + t * kGradPitch;
  float* h2 = sh2 + t * kGradPitch;
  float* h3 = sh3 + t * kGradPitch;
  float go = 0.f, lo = 0.f;
  float f[3] = {0.f, 0.f, 0.f};
  if (e < total) {
    const int j = (int)(e / K), g = (int)(e - (long long)j * K);
    const cplx<T> r = R[e], d = D[e];
    const float rx = (float)r.x, ry = (float)r.y;
    const float amp = sqrtf(rx * rx + ry * ry);
    float y;
    features((float)kin[g], (float)tband[j], amp, (float)sqrt(sumsq[j] / (double)K), f, &y);
    for (int i = 0; i < kH; ++i)
      h1[i] = tanhf(w[ob1 + i] + w[oW1 + 3 * i] * f[0] + w[oW1 + 3 * i + 1] * f[1] + w[oW1 + 3 * i + 2] * f[2]);
    for (int i = 0; i < kH; ++i) {
      float a = w[ob2 + i];
      for (int k = 0; k < kH; ++k) a += w[oW2 + kH * i + k] * h1[k];
      h2[i] = tanhf(a);
    }
    for (int i = 0; i < kH; ++i) {
      float a = w[ob3 + i];
      for (int k = 0; k < kH; ++k) a += w[oW3 + kH * i + k] * h2[k];
      h3[i] = tanhf(a);
    }
    float o = w[ob4];
    for (int k = 0; k < kH; ++k) o += w[oW4 + k] * h3[k];
    const float m = tpa_f(y) * expf(o);
    // a r (complex product), e = m a r - d; dL/dm = 2 Re(conj(e) a r) / |d_j|^2
    const float ax = (float)alpha[2 * j], ay = (float)alpha[2 * j + 1];
    const float qx = ax * rx - ay * ry, qy = ax * ry + ay * rx;
    const float ex = m * qx - (float)d.x, ey = m * qy - (float)d.y;
    const float nd = (float)dnorm2[j];
    lo = (ex * ex + ey * ey) / nd;
    go = 2.f * (ex * qx + ey * qy) / nd * m;
  } else {
    for (int i = 0; i < kH; ++i) h1[i] = h2[i] = h3[i] = 0.f;
  }
  sf[4 * t] = f[0];
  sf[4 * t + 1] = f[1];
  sf[4 * t + 2] = f[2];
  sgo[t] = go;
  sloss[t] = lo;
  float* d3 = sd3 + t * kGradPitch;
  float* d2 = sd2 + t * kGradPitch;
  float* d1 = sd1 + t * kGradPitch;
  for (int i = 0; i < kH; ++i) d3[i] = go * w[oW4 + i] * (1.f - h3[i] * h3[i]);
  for (int k = 0; k < kH; ++k) {
    float a = 0.f;
    for (int i = 0; i < kH; ++i) a += w[oW3 + kH * i + k] * d3[i];
    d2[k] = a * (1.f - h2[k] * h2[k]);
  }
  for (int k = 0; k < kH; ++k) {
    float a = 0.f;
    for (int i = 0; i < kH; ++i) a += w[oW2 + kH * i + k] * d2[i];
    d1[k] = a * (1.f - h1[k] * h1[k]);
  }
  __syncthreads();
  // block sums of the weight gradients (fixed order over the block's elements)
  float* P = part + (size_t)blockIdx.x * (kPrecondParams + 1);
  for (int p = t; p < kPrecondParams + 1; p += kGradBlock) {
    float acc = 0.f;
    if (p < ob1) {
      const int i = (p - oW1) / 3, c = (p - oW1) % 3;
      for (int q = 0; q < kGradBlock; ++q) acc += sd1[q * kGradPitch + i] * sf[4 * q + c];
    } else if (p < oW2) {
      const int i = p - ob1;
      for (int q = 0; q < kGradBlock; ++q) acc += sd1[q * kGradPitch + i];
    } else if (p < ob2) {
      const int i = (p - oW2) / kH, k = (p - oW2) % kH;
      for (int q = 0; q < kGradBlock; ++q) acc += sd2[q * kGradPitch + i] * sh1[q * kGradPitch + k];
    } else if (p < oW3) {
      const int i = p - ob2;
      for (int q = 0; q < kGradBlock; ++q) acc += sd2[q * kGradPitch + i];
    } else if (p < ob3) {
      const int i = (p - oW3) / kH, k = (p - oW3) % kH;
      for (int q = 0; q < kGradBlock; ++q) acc += sd3[q * kGradPitch + i] * sh2[q * kGradPitch + k];
    } else if (p < oW4) {
      const int i = p - ob3;
      for (int q = 0; q < kGradBlock; ++q) acc += sd3[q * kGradPitch + i];
    } else if (p < ob4) {
      const int k = p - oW4;
      for (int q = 0; q < kGradBlock; ++q) acc += sgo[q] * sh3[q * kGradPitch + k];
    } else if (p == ob4) {
      for (int q = 0; q < kGradBlock; ++q) acc += sgo[q];
    } else {
      for (int q = 0; q < kGradBlock; ++q) acc += sloss[q];
    }
    P[p] = acc;
  }
}

__global__ void k_precond_reduce(const float* __restrict__ part, int nblk, double* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kPrecondParams) return;
  double acc = 0;
  for (int b = 0; b < nblk; ++b) acc += (double)part[(size_t)b * (kPrecondParams + 1) + p];
  out[p] = acc;
}

// Adam step on the FP32 master weights; refreshes the bf16 copy.
__global__ void k_precond_adam(float* __restrict__ wf, __nv_bfloat16* __restrict__ wb, const double* __restrict__ grad,
                               float* __restrict__ m1, float* __restrict__ m2, float lr, float b1, float b2, float eps,
                               float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kPrecondParams) return;
  const float g = (float)grad[p];
  m1[p] = b1 * m1[p] + (1.f - b1) * g;
  m2[p] = b2 * m2[p] + (1.f - b2) * g * g;
  const float mh = m1[p] / c1, vh = m2[p] / c2;
  wf[p] -= lr * mh / (sqrtf(vh) + eps);
  wb[p] = __float2bfloat16_rn(wf[p]);
}

__global__ void k_precond_to_bf16(const float* __restrict__ wf, __nv_bfloat16* __restrict__ wb, float* rounded) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kPrecondParams) return;
  wb[p] = __float2bfloat16_rn(wf[p]);
  if (rounded) rounded[p] = __bfloat162float(wb[p]);
}

static bool g_pc_tc = true;  // tensor-core inference (default) or the CUDA-core kernel
void set_precond_tensor_cores(bool on) { g_pc_tc = on; }
bool precond_tensor_cores() { return g_pc_tc && !tensor_cores_disabled(); }

template <typename T>
void launch_precond_apply(const cplx<T>* R, int ldr, const T* kin, const double* tband, const double* sumsq, int nb,
                          int K, const void* wb, cplx<T>* W, int ldw, cudaStream_t st) {
  if (nb <= 0 || K <= 0) return;
  if (precond_tensor_cores()) {
    static int attr = 0, sms = 0;  // 1 configured, -1 failed
    if (attr == 0) {
      int dev = 0;
      const bool ok = cudaGetDevice(&dev) == cudaSuccess &&
                      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                      cudaFuncSetAttribute(k_precond_apply_tc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           kPcSmem) == cudaSuccess &&
                      cudaFuncSetAttribute(k_precond_apply_tc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           kPcSmem) == cudaSuccess;
      attr = ok ? 1 : -1;
    }
    if (attr > 0) {
      const long long tiles = (long long)nb * ceil_div(K, kPcThreads);
      const int grid = (int)std::min<long long>(tiles, (long long)sms * kPcCtasPerSm);
      count_launches(1);
      ProfScope p("k_precond_apply_tc", st);
      k_precond_apply_tc<T><<<grid, kPcThreads, kPcSmem, st>>>(R, ldr, kin, tband, sumsq, nb, K,
                                                               (const __nv_bfloat16*)wb, W, ldw);
      return;
    }
  }
  count_launches(1);
  ProfScope p("k_precond_apply", st);
  k_precond_apply<T><<<dim3(ceil_div(K, 128 * 4), nb), 128, 0, st>>>(R, ldr, kin, tband, sumsq, K,
                                                                      (const __nv_bfloat16*)wb, W, ldw);
}

// Status bits raised by the tensor-core inference since the last call (read and cleared;
// synchronises the stream); a kernel that kept its tensor memory turns the tensor cores off.
unsigned precond_tc_take_status(cudaStream_t st) {
  unsigned h = 0, z = 0;
  if (cudaMemcpyFromSymbolAsync(&h, g_pc_status, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return 0;
  if (h) cudaMemcpyToSymbolAsync(g_pc_status, &z, sizeof(unsigned), 0, cudaMemcpyHostToDevice, st);
  if (h & ST_TMEM_HELD) disable_tensor_cores();
  return h;
}
bool set_precond_tc_spin(long long polls) {
  const long long v = polls < 0 ? kTcSpin : std::min(polls, kTcSpin);
  return cudaMemcpyToSymbol(g_pc_spin, &v, sizeof(v)) == cudaSuccess;
}

int precond_grad_blocks(int nb, int K) { return ceil_div((long long)nb * K, kGradBlock); }

size_t precond_alpha_work(int nb) { return (size_t)nb * kAlphaBlocks * 3 + 2 * (size_t)nb; }
template <typename T>
void launch_precond_grad(const cplx<T>* R, const cplx<T>* D, int nb, int K, const T* kin, const double* tband,
                         const double* sumsq, const double* dnorm2, const float* wf, float* part, double* awork,
                         double* out, cudaStream_t st) {
  const int nblk = precond_grad_blocks(nb, K);
  double* alpha = awork + (size_t)nb * kAlphaBlocks * 3;
  cudaFuncSetAttribute(k_precond_grad<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem);
  count_launches(4);
  k_precond_alpha<T><<<dim3(kAlphaBlocks, nb), kAlphaThreads, 0, st>>>(R, D, K, kin, tband, sumsq, wf, awork);
  k_precond_alpha_fin<<<ceil_div(nb, 128), 128, 0, st>>>(awork, nb, alpha);
  k_precond_grad<T><<<nblk, kGradBlock, kGradSmem, st>>>(R, D, K, nb, kin, tband, sumsq, dnorm2, alpha, wf, part);
  k_precond_reduce<<<ceil_div(kPrecondParams + 1, 256), 256, 0, st>>>(part, nblk, out);
}

void launch_precond_adam(float* wf, void* wb, const double* grad, float* m1, float* m2, float lr, int step,
                         cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  count_launches(1);
  k_precond_adam<<<ceil_div(kPrecondParams, 256), 256, 0, st>>>(wf, (__nv_bfloat16*)wb, grad, m1, m2, lr, b1, b2,
                                                                1e-8f, c1, c2);
}

void launch_precond_to_bf16(const float* wf, void* wb, float* rounded, cudaStream_t st) {
  count_launches(1);
  k_precond_to_bf16<<<ceil_div(kPrecondParams, 256), 256, 0, st>>>(wf, (__nv_bfloat16*)wb, rounded);
}

template void launch_precond_apply<float>(const float2*, int, const float*, const double*, const double*, int, int,
                                          const void*, float2*, int, cudaStream_t);
template void launch_precond_apply<double>(const double2*, int, const double*, const double*, const double*, int, int,
                                           const void*, double2*, int, cudaStream_t);
template void launch_precond_grad<float>(const float2*, const float2*, int, int, const float*, const double*,
                                         const double*, const double*, const float*, float*, double*, double*,
                                         cudaStream_t);
template void launch_precond_grad<double>(const double2*, const double2*, int, int, const double*, const double*,
                                          const double*, const double*, const float*, float*, double*, double*,
                                          cudaStream_t);

}  // namespace fde
