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

// ---- the network on the tensor cores ----------------------------------------------------------
// The two 64 x 64 hidden layers as BF16 tcgen05 MMAs (kind::f16, M = 128 points, N = 64
// neurons, K = 16 per MMA, FP32 accumulation in tensor memory).  Activations are split
// h = hi + lo with hi = bf16(h) and lo = bf16(h - hi) (|h - hi - lo| <= 2^-18 |h|).  With the
// bf16 inference weights a layer is W hi + W lo (two passes of four MMAs); with the FP32
// master weights (training) the weights are split the same way and a layer is
// Whi hi + Wlo hi + Whi lo (three passes; the dropped Wlo lo term is below 2^-16 relative).
// The first layer (three inputs), the tanh of every layer, the output layer and the
// multiplier run on the CUDA cores, one thread per point.  Persistent CTAs of 128 threads loop
// over tiles of 128 points; thread t owns point t of a tile, which is row t of the A operand
// and lane t of the accumulator.
// tanh(x) = (e^{2x} - 1) / (e^{2x} + 1) with the hardware exponential and division
// (absolute error ~2e-7), the argument clamped to |x| <= 15 where tanh is 1 in FP32.
constexpr int kPcThreads = 128;
constexpr int kPcCtasPerSm = 3;
constexpr int kPcAct = kPcThreads * 128;  // bytes of one 128 x 64 bf16 activation tile
constexpr int kPcW = kH * 128;            // bytes of one 64 x 64 bf16 weight tile
template <bool MASTER> constexpr int pc_smem() { return 1024 + 2 * kPcAct + (MASTER ? 4 : 2) * kPcW; }
constexpr int kPcTmemCols = 64;
// kind::f16 instruction descriptor: D f32 (bits 4-5 = 1), A and B bf16 (bits 7-9, 10-12 = 1),
// both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28 (M = 128).
__host__ __device__ constexpr uint32_t pc_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n / 8) << 17) | ((uint32_t)(128 / 16) << 24);
}
// small parameters in shared memory (float): W1, b1, b2, b3, W4, b4
constexpr int sW1 = 0, sb1 = sW1 + 3 * kH, sb2 = sb1 + kH, sb3 = sb2 + kH, sW4 = sb3 + kH, sb4 = sW4 + kH,
              sEnd = sb4 + 1;

__device__ unsigned g_pc_status;
__device__ long long g_pc_spin = kTcSpin;

// Operands of the tensor-core kernels to FP32 on the bit patterns (dd.cuh), keeping their
// per-point work off the FP64 pipe.
__device__ __forceinline__ float tof(float v) { return v; }
__device__ __forceinline__ float tof(double v) { return float_of_double_bits(v); }

__device__ __forceinline__ float tanh_tc(float x) {
  const float t = __expf(2.f * fminf(fmaxf(x, -15.f), 15.f));
  return __fdividef(t - 1.f, t + 1.f);
}
__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) {  // a in the low half
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}
// Row t of the hi and lo tiles of a 64-wide K-major operand (128-byte rows, 16-byte chunks
// swizzled by t mod 8).
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
__device__ __forceinline__ void mma_bf16(uint32_t dt, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// B operand of a 64 x 64 layer: row i = the weights into neuron i (W[i][k]), or with TRANS the
// transposed matrix (row k = W[.][k], for back-propagation), as bf16 hi (and lo) tiles.
template <bool TRANS>
__device__ __forceinline__ void stage_weights(uint32_t hi, uint32_t lo, const float* __restrict__ wf,
                                              const __nv_bfloat16* __restrict__ wb, int t) {
  for (int q = t; q < kH * 8; q += kPcThreads) {
    const int r = q >> 3, c = q & 7;
    uint32_t hb[4], lb[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float x[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int k = 8 * c + 2 * u + e;
        const int idx = TRANS ? k * kH + r : r * kH + k;
        x[e] = wf ? wf[idx] : __bfloat162float(wb[idx]);
      }
      hb[u] = bf16x2_bits(x[0], x[1]);
      const __nv_bfloat162 hv = *reinterpret_cast<const __nv_bfloat162*>(&hb[u]);
      lb[u] = bf16x2_bits(x[0] - __low2float(hv), x[1] - __high2float(hv));
    }
    const uint32_t off = (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
    st_shared_v4(hi + off, make_uint4(hb[0], hb[1], hb[2], hb[3]));
    if (lo) st_shared_v4(lo + off, make_uint4(lb[0], lb[1], lb[2], lb[3]));
  }
}
__device__ __forceinline__ void load_small(float* ws, const float* __restrict__ wf, const __nv_bfloat16* __restrict__ wb,
                                           int t) {
  auto w = [&](int i) { return wf ? wf[i] : __bfloat162float(wb[i]); };
  for (int i = t; i < 3 * kH; i += kPcThreads) ws[sW1 + i] = w(oW1 + i);
  for (int i = t; i < kH; i += kPcThreads) {
    ws[sb1 + i] = w(ob1 + i);
    ws[sb2 + i] = w(ob2 + i);
    ws[sb3 + i] = w(ob3 + i);
    ws[sW4 + i] = w(oW4 + i);
  }
  if (t == 0) ws[sb4] = w(ob4);
}
// One layer's MMAs: D = A W^T over K = 64 (four K-steps of 16) for each split pass.
__device__ __forceinline__ void layer_mmas(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t w_hi, uint32_t w_lo,
                                           uint32_t idesc) {
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) mma_bf16(d, sdesc(a_hi + 32u * kk), sdesc(w_hi + 32u * kk), idesc, kk > 0 ? 1u : 0u);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) mma_bf16(d, sdesc(a_lo + 32u * kk), sdesc(w_hi + 32u * kk), idesc, 1u);
  if (w_lo) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) mma_bf16(d, sdesc(a_hi + 32u * kk), sdesc(w_lo + 32u * kk), idesc, 1u);
  }
}
// Commit the issued MMAs to bar and wait for them (thread 0, bounded); every thread returns
// false after a timeout.  phase flips on every call.
__device__ __forceinline__ bool commit_wait(uint64_t* bar, unsigned& phase, int* abort_flag) {
  if (threadIdx.x == 0) {
    mma_commit(su32(bar));
    if (!mbar_wait(su32(bar), phase, g_pc_spin)) *abort_flag = 1;
  }
  __syncthreads();
  phase ^= 1u;
  if (*abort_flag) return false;
  tc_fence_after();
  return true;
}
// After a timeout: wait (bounded) for the outstanding MMAs, raise the status and release the
// tensor memory only if they completed.
__device__ __forceinline__ void tc_finish(bool ok, uint64_t* bar, unsigned phase, int* drained, uint32_t tmem,
                                          uint32_t cols) {
  if (threadIdx.x == 0) *drained = ok ? 1 : (mbar_wait(su32(bar), phase ^ 1u) ? 1 : 0);
  tc_fence_before();
  __syncthreads();
  if (!ok && threadIdx.x == 0) atomicOr(&g_pc_status, *drained ? ST_TIMEOUT : (ST_TIMEOUT | ST_TMEM_HELD));
  if ((threadIdx.x >> 5) == 0 && *drained) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
  }
}
__device__ __forceinline__ uint32_t tmem_alloc(uint32_t* slot, uint32_t cols) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *slot;
}

// W[j][g] = m_jg R[j][g] for nb rows: the bf16 inference weights (wf null) or the FP32 master
// weights (MASTER, training's scale pass).
template <typename T, bool MASTER>
__global__ void __launch_bounds__(kPcThreads, kPcCtasPerSm)
k_precond_apply_tc(const cplx<T>* __restrict__ R, int ldr, const T* __restrict__ kin, const double* __restrict__ tband,
                   const double* __restrict__ sumsq, int nb, int K, const __nv_bfloat16* __restrict__ wb,
                   const float* __restrict__ wf, cplx<T>* __restrict__ W, int ldw) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ float ws[sEnd];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag, drained;
  const int t = threadIdx.x, warp = t >> 5;
  const uint32_t base = (su32(smem_raw) + 1023u) & ~1023u;
  const uint32_t a_hi = base, a_lo = base + kPcAct, w2h = base + 2 * kPcAct, w3h = w2h + kPcW;
  const uint32_t w2l = MASTER ? w3h + kPcW : 0u, w3l = MASTER ? w3h + 2 * kPcW : 0u;
  const float* wsrc = MASTER ? wf : nullptr;
  load_small(ws, wsrc, wb, t);
  stage_weights<false>(w2h, w2l, wsrc ? wsrc + oW2 : nullptr, wb + oW2, t);
  stage_weights<false>(w3h, w3l, wsrc ? wsrc + oW3 : nullptr, wb + oW3, t);
  if (t == 0) {
    mbar_init(su32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const uint32_t tmem = tmem_alloc(&tmem_slot, kPcTmemCols);
  const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
  const int tiles_per_band = (K + kPcThreads - 1) / kPcThreads;
  const long long ntiles = (long long)nb * tiles_per_band;
  unsigned phase = 0;
  bool ok = true;
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int j = (int)(tile / tiles_per_band);
    const int g = (int)(tile - (long long)j * tiles_per_band) * kPcThreads + t;
    const bool valid = g < K;
    const cplx<T> r = valid ? R[(size_t)j * ldr + g] : mk<T>(0, 0);
    const float rx = tof(r.x), ry = tof(r.y);
    float f[3], y;
    features(valid ? tof(kin[g]) : 0.f, tof(tband[j]), sqrtf(rx * rx + ry * ry), sqrtf(tof(sumsq[j]) / (float)K), f,
             &y);
    float h[kH];
#pragma unroll
    for (int i = 0; i < kH; ++i)
      h[i] = tanh_tc(ws[sb1 + i] + ws[sW1 + 3 * i] * f[0] + ws[sW1 + 3 * i + 1] * f[1] + ws[sW1 + 3 * i + 2] * f[2]);
    store_split(a_hi, a_lo, t, h);
#pragma unroll 1
    for (int layer = 0; layer < 2 && ok; ++layer) {
      tc_fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      if (t == 0) {
        tc_fence_after();
        layer_mmas(tmem, a_hi, a_lo, layer ? w3h : w2h, layer ? w3l : w2l, pc_idesc(kH));
      }
      if (!commit_wait(&bar, phase, &abort_flag)) {
        ok = false;
        break;
      }
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
  tc_finish(ok, &bar, phase, &drained, tmem, kPcTmemCols);
}

// ---- loss gradient on the tensor cores ---------------------------------------------------------
// Per tile of 128 elements (band, G) with thread t on element t:
//   forward   h1 = tanh(W1 f + b1) (CUDA cores); h2, h3 by the layer MMAs (master weights);
//             o, m, the loss and g_o = dL/do per element;
//   backward  d3 = g_o W4 (1 - h3^2); d2 = (W3^T d3) (1 - h2^2); d1 = (W2^T d2) (1 - h1^2),
//             the products W^T d as MMAs against the transposed weight tiles;
//   gradients dW3 = sum d3 h2^T, db3 = sum d3 (and the same for layers 2 and 1) as MMAs with
//             the 128 elements as K: A = [d^T hi ; d^T lo] (M = 128: neurons, then their low
//             parts), B = [x^T ; ones] (N = 80: the 64 inputs, a row of ones for the bias, zero
//             pad; N = 16 for layer 1: f0, f1, f2, ones), hi and lo passes, so the product
//             (d_hi + d_lo)(x_hi + x_lo) is kept whole; the two 64-row halves of the
//             accumulator are added at the end.  These accumulate in tensor memory over all
//             tiles of the CTA; dW4, db4 and the loss in registers.
// Each CTA writes its partial gradient to part[blockIdx.x]; k_precond_reduce sums them in a
// fixed order.  One CTA per SM (217 KB of operand tiles); 240 tensor-memory columns.
constexpr int kPgN = 80;                 // rows of the layer-2/3 gradient B operands
constexpr int kPgN1 = 16;                // rows of the layer-1 gradient B operand
constexpr int kPgAg = 2 * 128 * 128;     // A of the weight gradients, two K halves (32 KB)
constexpr int kPgBg = 2 * kPgN * 128;    // B of a layer-2/3 weight gradient, two K halves (20 KB)
constexpr int kPgBg1 = 2 * kPgN1 * 128;  // B of the layer-1 weight gradient (4 KB)
constexpr int gAh = 0, gAl = gAh + kPcAct, gW2h = gAl + kPcAct, gW2l = gW2h + kPcW, gW3h = gW2l + kPcW,
              gW3l = gW3h + kPcW, gT3h = gW3l + kPcW, gT3l = gT3h + kPcW, gT2h = gT3l + kPcW, gT2l = gT2h + kPcW,
              gAg = gT2l + kPcW, gB3h = gAg + kPgAg, gB3l = gB3h + kPgBg, gB2h = gB3l + kPgBg, gB2l = gB2h + kPgBg,
              gB1h = gB2l + kPgBg, gB1l = gB1h + kPgBg1, gEnd = gB1l + kPgBg1;
constexpr int kPgSmem = 1024 + gEnd;
constexpr int cAct = 0, cG3 = 64, cG2 = cG3 + kPgN, cG1 = cG2 + kPgN;
constexpr int kPgTmemCols = 256;
static_assert(cG1 + kPgN1 <= kPgTmemCols, "tensor-memory columns");
static_assert(kPgSmem <= 227 * 1024 - 4096, "operand tiles fit one CTA's shared memory");

// Byte offset of element (r, p) of a K-major operand whose K (the tile's 128 elements) is
// split into two 64-element halves of `rows` rows each.
__device__ __forceinline__ uint32_t tswz(int r, int p, int rows) {
  const int h = p >> 6, kk = p & 63;
  return (uint32_t)(h * rows * 128 + r * 128 + ((((kk >> 3) ^ (r & 7)) << 4) | ((kk & 7) << 1)));
}
__device__ __forceinline__ void st_b16(uint32_t addr, uint16_t v) {
  asm volatile("st.shared.b16 [%0], %1;" ::"r"(addr), "h"(v) : "memory");
}
__device__ __forceinline__ uint16_t ld_b16(uint32_t addr) {
  uint16_t v;
  asm volatile("ld.shared.b16 %0, [%1];" : "=h"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ uint16_t bf16_bits(float x) {
  const __nv_bfloat16 b = __float2bfloat16_rn(x);
  return *reinterpret_cast<const uint16_t*>(&b);
}
__device__ __forceinline__ float bf16_val(uint16_t v) {
  return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(&v));
}
// Column p of rows r0 .. r0 + n - 1 of a hi / lo pair of K-split tiles: the split of x[0 .. n).
__device__ __forceinline__ void store_col(uint32_t hi, uint32_t lo, int rows, int r0, int p, const float* x, int n,
                                          int lo_row_shift) {
  for (int i = 0; i < n; ++i) {
    const uint16_t hb = bf16_bits(x[i]);
    const uint16_t lb = bf16_bits(x[i] - bf16_val(hb));
    st_b16(hi + tswz(r0 + i, p, rows), hb);
    st_b16(lo + tswz(r0 + i + lo_row_shift, p, rows), lb);
  }
}
// h[i] = hi + lo of column p (rows 0 .. 63) of a hi / lo pair of K-split tiles.
__device__ __forceinline__ void load_col(uint32_t hi, uint32_t lo, int rows, int p, float* h) {
#pragma unroll 8
  for (int i = 0; i < kH; ++i) h[i] = bf16_val(ld_b16(hi + tswz(i, p, rows))) + bf16_val(ld_b16(lo + tswz(i, p, rows)));
}
// The weight-gradient MMAs of one layer: D += A_g B^T over the tile's 128 elements.
__device__ __forceinline__ void grad_mmas(uint32_t d, uint32_t ag, uint32_t bh, uint32_t bl, int nrows,
                                          uint32_t idesc, uint32_t acc0) {
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    const uint32_t half = (uint32_t)(kk >> 2), off = 32u * (kk & 3);
    const uint64_t a = sdesc(ag + half * 128u * 128u + off);
    mma_bf16(d, a, sdesc(bh + half * (uint32_t)nrows * 128u + off), idesc, (kk > 0 || acc0) ? 1u : 0u);
    mma_bf16(d, a, sdesc(bl + half * (uint32_t)nrows * 128u + off), idesc, 1u);
  }
}

template <typename T>
__global__ void __launch_bounds__(kPcThreads, 1)
k_precond_grad_tc(const cplx<T>* __restrict__ R, const cplx<T>* __restrict__ D, int K, int nb,
                  const T* __restrict__ kin, const double* __restrict__ tband, const double* __restrict__ sumsq,
                  const double* __restrict__ dnorm2, const double* __restrict__ alpha, const float* __restrict__ wf,
                  float* __restrict__ part) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ float ws[sEnd];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag, drained;
  const int t = threadIdx.x, warp = t >> 5;
  const uint32_t base = (su32(smem_raw) + 1023u) & ~1023u;
  load_small(ws, wf, nullptr, t);
  stage_weights<false>(base + gW2h, base + gW2l, wf + oW2, nullptr, t);
  stage_weights<false>(base + gW3h, base + gW3l, wf + oW3, nullptr, t);
  stage_weights<true>(base + gT3h, base + gT3l, wf + oW3, nullptr, t);
  stage_weights<true>(base + gT2h, base + gT2l, wf + oW2, nullptr, t);
  // constant rows of the gradient B operands: ones (hi) for the biases, zero padding
  for (int p = t; p < 128; p += kPcThreads) {
    for (int r = kH; r < kPgN; ++r) {
      const uint16_t one = (r == kH) ? bf16_bits(1.f) : (uint16_t)0;
      st_b16(base + gB3h + tswz(r, p, kPgN), one);
      st_b16(base + gB3l + tswz(r, p, kPgN), 0);
      st_b16(base + gB2h + tswz(r, p, kPgN), one);
      st_b16(base + gB2l + tswz(r, p, kPgN), 0);
    }
    for (int r = 3; r < kPgN1; ++r) {
      st_b16(base + gB1h + tswz(r, p, kPgN1), r == 3 ? bf16_bits(1.f) : (uint16_t)0);
      st_b16(base + gB1l + tswz(r, p, kPgN1), 0);
    }
  }
  if (t == 0) {
    mbar_init(su32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const uint32_t tmem = tmem_alloc(&tmem_slot, kPgTmemCols);
  const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
  const uint32_t idAct = pc_idesc(kH), idG = pc_idesc(kPgN), idG1 = pc_idesc(kPgN1);
  const long long total = (long long)nb * K;
  const long long ntiles = (total + kPcThreads - 1) / kPcThreads;
  float acc4[kH], accb4 = 0.f, accl = 0.f;
#pragma unroll
  for (int k = 0; k < kH; ++k) acc4[k] = 0.f;
  unsigned phase = 0;
  bool ok = true, first = true;
  auto sync_issue = [&]() {
    tc_fence_proxy_async();
    tc_fence_before();
    __syncthreads();
  };
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long long e = tile * kPcThreads + t;
    const bool valid = e < total;
    const int j = valid ? (int)(e / K) : 0, g = valid ? (int)(e - (long long)j * K) : 0;
    const cplx<T> r = valid ? R[e] : mk<T>(0, 0), dv = valid ? D[e] : mk<T>(0, 0);
    const float rx = tof(r.x), ry = tof(r.y);
    float f[3], y;
    features(valid ? tof(kin[g]) : 0.f, tof(tband[j]), sqrtf(rx * rx + ry * ry), sqrtf(tof(sumsq[j]) / (float)K), f,
             &y);
    float h[kH];
#pragma unroll
    for (int i = 0; i < kH; ++i)
      h[i] = tanh_tc(ws[sb1 + i] + ws[sW1 + 3 * i] * f[0] + ws[sW1 + 3 * i + 1] * f[1] + ws[sW1 + 3 * i + 2] * f[2]);
    store_split(base + gAh, base + gAl, t, h);
    {
      float x[kH];
#pragma unroll
      for (int i = 0; i < kH; ++i) x[i] = valid ? h[i] : 0.f;
      store_col(base + gB2h, base + gB2l, kPgN, 0, t, x, kH, 0);
      float fv[3] = {valid ? f[0] : 0.f, valid ? f[1] : 0.f, valid ? f[2] : 0.f};
      store_col(base + gB1h, base + gB1l, kPgN1, 0, t, fv, 3, 0);
    }
    // layers 2 and 3
#pragma unroll 1
    for (int layer = 0; layer < 2 && ok; ++layer) {
      sync_issue();
      if (t == 0) {
        tc_fence_after();
        layer_mmas(tmem + cAct, base + gAh, base + gAl, base + (layer ? gW3h : gW2h), base + (layer ? gW3l : gW2l),
                   idAct);
      }
      if (!commit_wait(&bar, phase, &abort_flag)) { ok = false; break; }
#pragma unroll
      for (int c = 0; c < kH; c += 16) tmem_ld16(trow + (uint32_t)(cAct + c), h + c);
      const float* bl = ws + (layer ? sb3 : sb2);
#pragma unroll
      for (int i = 0; i < kH; ++i) h[i] = tanh_tc(h[i] + bl[i]);
      if (layer == 0) {
        store_split(base + gAh, base + gAl, t, h);
        float x[kH];
#pragma unroll
        for (int i = 0; i < kH; ++i) x[i] = valid ? h[i] : 0.f;
        store_col(base + gB3h, base + gB3l, kPgN, 0, t, x, kH, 0);
      }
    }
    if (!ok) break;
    // output, loss and g_o = dL/do (a_j the band's optimal complex scale)
    float o = ws[sb4];
#pragma unroll
    for (int k = 0; k < kH; ++k) o += ws[sW4 + k] * h[k];
    const float m = tpa_f(y) * expf(o);
    float go = 0.f;
    if (valid) {
      const float ax = tof(alpha[2 * j]), ay = tof(alpha[2 * j + 1]);
      const float qx = ax * rx - ay * ry, qy = ax * ry + ay * rx;
      const float ex = m * qx - tof(dv.x), ey = m * qy - tof(dv.y);
      const float nd = tof(dnorm2[j]);
      accl += (ex * ex + ey * ey) / nd;
      go = 2.f * (ex * qx + ey * qy) / nd * m;
    }
    accb4 += go;
    // d3 = g_o W4 (1 - h3^2)
#pragma unroll
    for (int k = 0; k < kH; ++k) {
      acc4[k] += go * h[k];
      h[k] = go * ws[sW4 + k] * (1.f - h[k] * h[k]);
    }
    store_split(base + gAh, base + gAl, t, h);
    store_col(base + gAg, base + gAg, 128, 0, t, h, kH, kH);
    // d2 pre = W3^T d3, and dW3 / db3 += d3 [h2; 1]^T
    sync_issue();
    if (t == 0) {
      tc_fence_after();
      layer_mmas(tmem + cAct, base + gAh, base + gAl, base + gT3h, base + gT3l, idAct);
      grad_mmas(tmem + cG3, base + gAg, base + gB3h, base + gB3l, kPgN, idG, first ? 0u : 1u);
    }
    if (!commit_wait(&bar, phase, &abort_flag)) { ok = false; break; }
    {
      float hp[kH];
#pragma unroll
      for (int c = 0; c < kH; c += 16) tmem_ld16(trow + (uint32_t)(cAct + c), h + c);
      load_col(base + gB3h, base + gB3l, kPgN, t, hp);
#pragma unroll
      for (int k = 0; k < kH; ++k) h[k] *= 1.f - hp[k] * hp[k];
    }
    store_split(base + gAh, base + gAl, t, h);
    store_col(base + gAg, base + gAg, 128, 0, t, h, kH, kH);
    // d1 pre = W2^T d2, and dW2 / db2 += d2 [h1; 1]^T
    sync_issue();
    if (t == 0) {
      tc_fence_after();
      layer_mmas(tmem + cAct, base + gAh, base + gAl, base + gT2h, base + gT2l, idAct);
      grad_mmas(tmem + cG2, base + gAg, base + gB2h, base + gB2l, kPgN, idG, first ? 0u : 1u);
    }
    if (!commit_wait(&bar, phase, &abort_flag)) { ok = false; break; }
    {
      float hp[kH];
#pragma unroll
      for (int c = 0; c < kH; c += 16) tmem_ld16(trow + (uint32_t)(cAct + c), h + c);
      load_col(base + gB2h, base + gB2l, kPgN, t, hp);
#pragma unroll
      for (int k = 0; k < kH; ++k) h[k] *= 1.f - hp[k] * hp[k];
    }
    store_col(base + gAg, base + gAg, 128, 0, t, h, kH, kH);
    // dW1 / db1 += d1 [f; 1]^T
    sync_issue();
    if (t == 0) {
      tc_fence_after();
      grad_mmas(tmem + cG1, base + gAg, base + gB1h, base + gB1l, kPgN1, idG1, first ? 0u : 1u);
    }
    if (!commit_wait(&bar, phase, &abort_flag)) { ok = false; break; }
    first = false;
  }
  // read the accumulators (nothing was accumulated when the CTA had no tile: write zeros)
  float* P = part + (size_t)blockIdx.x * (kPrecondParams + 1);
  float* buf = reinterpret_cast<float*>(smem_raw + (base - su32(smem_raw)));  // the operand tiles are free now
  constexpr int BP = kPgN + 1;  // pitch of the staged accumulator rows
  if (ok) {
    const int nl[3] = {kPgN, kPgN, kPgN1};
    const int col[3] = {cG3, cG2, cG1};
#pragma unroll 1
    for (int q = 0; q < 3; ++q) {
      float v[kPgN];
      if (!first) {
        for (int c = 0; c < nl[q]; c += 16) tmem_ld16(trow + (uint32_t)(col[q] + c), v + c);
      } else {
        for (int c = 0; c < nl[q]; ++c) v[c] = 0.f;
      }
      __syncthreads();
      for (int c = 0; c < nl[q]; ++c) buf[t * BP + c] = v[c];
      __syncthreads();
      if (t < kH) {
        // neuron i = t: its hi row t plus its lo row 64 + t
        auto gsum = [&](int c) { return buf[t * BP + c] + buf[(t + kH) * BP + c]; };
        if (q == 0) {
          for (int k = 0; k < kH; ++k) P[oW3 + t * kH + k] = gsum(k);
          P[ob3 + t] = gsum(kH);
        } else if (q == 1) {
          for (int k = 0; k < kH; ++k) P[oW2 + t * kH + k] = gsum(k);
          P[ob2 + t] = gsum(kH);
        } else {
          for (int c = 0; c < 3; ++c) P[oW1 + 3 * t + c] = gsum(c);
          P[ob1 + t] = gsum(3);
        }
      }
    }
    // dW4, db4 and the loss: sums over the CTA's threads in a fixed order
    __syncthreads();
    for (int k = 0; k < kH; ++k) buf[t * BP + k] = acc4[k];
    buf[t * BP + kH] = accb4;
    buf[t * BP + kH + 1] = accl;
    __syncthreads();
    for (int c = t; c < kH + 2; c += kPcThreads) {
      float sacc = 0.f;
      for (int q = 0; q < kPcThreads; ++q) sacc += buf[q * BP + c];
      if (c < kH) P[oW4 + c] = sacc;
      else if (c == kH) P[ob4] = sacc;
      else P[kPrecondParams] = sacc;
    }
  }
  tc_finish(ok, &bar, phase, &drained, tmem, kPgTmemCols);
}

// Per-band sums for the optimal scale from W = m R (the master-weight multiplier applied):
// <W_j, D_j> (re, im) and |W_j|^2; CTA (b, j), the same partial layout as k_precond_alpha.
constexpr int kAlphaBlocksW = 32;
template <typename T>
__global__ void __launch_bounds__(128)
k_precond_alpha_w(const cplx<T>* __restrict__ Wm, const cplx<T>* __restrict__ D, int K, double* __restrict__ part) {
  __shared__ double red[3][128];
  const int j = blockIdx.y;
  double cr = 0, ci = 0, nn = 0;
  for (int g = blockIdx.x * 128 + threadIdx.x; g < K; g += kAlphaBlocksW * 128) {
    const cplx<T> w = Wm[(size_t)j * K + g], d = D[(size_t)j * K + g];
    const double wx = (double)w.x, wy = (double)w.y;
    cr += wx * (double)d.x + wy * (double)d.y;
    ci += wx * (double)d.y - wy * (double)d.x;
    nn += wx * wx + wy * wy;
  }
  red[0][threadIdx.x] = cr;
  red[1][threadIdx.x] = ci;
  red[2][threadIdx.x] = nn;
  __syncthreads();
  for (int hh = 64; hh > 0; hh >>= 1) {
    if ((int)threadIdx.x < hh)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + hh];
    __syncthreads();
  }
  if (threadIdx.x < 3) part[((size_t)j * kAlphaBlocksW + blockIdx.x) * 3 + threadIdx.x] = red[threadIdx.x][0];
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

static bool g_pc_tc = true;  // tensor cores (default) or the CUDA-core kernels
void set_precond_tensor_cores(bool on) { g_pc_tc = on; }
bool precond_tensor_cores() { return g_pc_tc && !tensor_cores_disabled(); }

// Dynamic shared memory of the tensor-core kernels configured once per process; the SM count
// of the current device sizes their persistent grids.  False if a kernel cannot be configured.
static int pc_sms() {
  static int sms = -1;
  if (sms < 0) {
    int dev = 0, n = 0;
    sms = (cudaGetDevice(&dev) == cudaSuccess &&
           cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
              ? n
              : 0;
  }
  return sms;
}
static bool pc_configure() {
  static int attr = 0;  // 1 configured, -1 failed
  if (attr == 0) {
    const bool ok =
        pc_sms() > 0 &&
        cudaFuncSetAttribute(k_precond_apply_tc<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             pc_smem<false>()) == cudaSuccess &&
        cudaFuncSetAttribute(k_precond_apply_tc<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             pc_smem<false>()) == cudaSuccess &&
        cudaFuncSetAttribute(k_precond_apply_tc<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             pc_smem<true>()) == cudaSuccess &&
        cudaFuncSetAttribute(k_precond_apply_tc<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             pc_smem<true>()) == cudaSuccess &&
        cudaFuncSetAttribute(k_precond_grad_tc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPgSmem) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_precond_grad_tc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPgSmem) ==
            cudaSuccess;
    attr = ok ? 1 : -1;
  }
  return attr > 0;
}
static bool pc_tc_path() { return precond_tensor_cores() && pc_configure(); }

template <typename T, bool MASTER>
static void launch_apply_tc(const cplx<T>* R, int ldr, const T* kin, const double* tband, const double* sumsq, int nb,
                            int K, const void* wb, const float* wf, cplx<T>* W, int ldw, cudaStream_t st) {
  const long long tiles = (long long)nb * ceil_div(K, kPcThreads);
  const int grid = (int)std::min<long long>(tiles, (long long)pc_sms() * kPcCtasPerSm);
  count_launches(1);
  ProfScope p("k_precond_apply_tc", st);
  k_precond_apply_tc<T, MASTER><<<grid, kPcThreads, pc_smem<MASTER>(), st>>>(
      R, ldr, kin, tband, sumsq, nb, K, (const __nv_bfloat16*)wb, wf, W, ldw);
}

template <typename T>
void launch_precond_apply(const cplx<T>* R, int ldr, const T* kin, const double* tband, const double* sumsq, int nb,
                          int K, const void* wb, cplx<T>* W, int ldw, cudaStream_t st) {
  if (nb <= 0 || K <= 0) return;
  if (pc_tc_path()) return launch_apply_tc<T, false>(R, ldr, kin, tband, sumsq, nb, K, wb, nullptr, W, ldw, st);
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

int precond_grad_blocks(int nb, int K) {
  if (pc_tc_path()) return (int)std::min<long long>(ceil_div((long long)nb * K, kPcThreads), pc_sms());
  return ceil_div((long long)nb * K, kGradBlock);
}

size_t precond_alpha_work(int nb) { return (size_t)nb * kAlphaBlocks * 3 + 2 * (size_t)nb; }
static_assert(kAlphaBlocksW == kAlphaBlocks, "one partial layout for both scale passes");
template <typename T>
void launch_precond_grad(const cplx<T>* R, const cplx<T>* D, int nb, int K, const T* kin, const double* tband,
                         const double* sumsq, const double* dnorm2, const float* wf, float* part, double* awork,
                         cplx<T>* wtmp, double* out, cudaStream_t st) {
  const int nblk = precond_grad_blocks(nb, K);
  double* alpha = awork + (size_t)nb * kAlphaBlocks * 3;
  if (pc_tc_path()) {
    ProfScope p("k_precond_grad_tc", st);
    launch_apply_tc<T, true>(R, K, kin, tband, sumsq, nb, K, nullptr, wf, wtmp, K, st);
    count_launches(4);
    k_precond_alpha_w<T><<<dim3(kAlphaBlocks, nb), 128, 0, st>>>(wtmp, D, K, awork);
    k_precond_alpha_fin<<<ceil_div(nb, 128), 128, 0, st>>>(awork, nb, alpha);
    k_precond_grad_tc<T><<<nblk, kPcThreads, kPgSmem, st>>>(R, D, K, nb, kin, tband, sumsq, dnorm2, alpha, wf, part);
    k_precond_reduce<<<ceil_div(kPrecondParams + 1, 256), 256, 0, st>>>(part, nblk, out);
    return;
  }
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
                                         const double*, const double*, const float*, float*, double*, float2*,
                                         double*, cudaStream_t);
template void launch_precond_grad<double>(const double2*, const double2*, int, int, const double*, const double*,
                                          const double*, const double*, const float*, float*, double*, double2*,
                                          double*, cudaStream_t);

}  // namespace fde
