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
#include <math.h>

#include "precond.h"
#include "prof.h"

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

template <typename T>
void launch_precond_apply(const cplx<T>* R, int ldr, const T* kin, const double* tband, const double* sumsq, int nb,
                          int K, const void* wb, cplx<T>* W, int ldw, cudaStream_t st) {
  if (nb <= 0) return;
  count_launches(1);
  k_precond_apply<T><<<dim3(ceil_div(K, 128 * 4), nb), 128, 0, st>>>(R, ldr, kin, tband, sumsq, K,
                                                                      (const __nv_bfloat16*)wb, W, ldw);
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
