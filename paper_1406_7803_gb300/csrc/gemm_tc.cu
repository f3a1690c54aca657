// gemm_tc.cu -- C = A^H B over a long K on the 5th-generation tensor cores (tcgen05, TF32
// inputs, FP32 accumulation in tensor memory): the subspace Gram / subspace-Hamiltonian
// products of the block eigensolver and the projector contraction <beta|psi> of the
// Kleinman-Bylander term (Eq. KS; Appendix, subsystem-specific projectors).
//
// Complex to real.  With a = (Re a_0, Im a_0, Re a_1, ...) the interleaved row of A and
// b~ = (Im b_0, -Re b_0, Im b_1, ...) the "rotated" row of B,
//   Re (A^H B)_ij = a_i . b_j,   Im (A^H B)_ij = a_i . b~_j,
// so one real GEMM with the B tile stacked as [b_0..b_63 ; b~_0..b~_63] (N = 128) yields
// both parts: D[i][j] = Re, D[i][64 + j] = Im.
//
// Precision.  TF32 keeps 10 mantissa bits.  Each operand is split x = hi + lo with hi = x
// truncated to TF32 (exact) and lo = x - hi (exact in FP32); D += Ahi Bhi + Ahi Blo + Alo Bhi
// (three MMAs per k-step) carries ~21 bits, the accuracy of the FP32 CUDA-core product.
// passes = 1 keeps only Ahi Bhi.
//
// Data flow per CTA (256 threads, one 128 x 64 complex output tile, one K-chunk):
//   registers <- global (8-byte loads, one k-tile of 16 complex ahead) ; split, rotate and
//   store into the 128-byte-swizzled K-major shared-memory layout the MMA descriptors
//   describe ; fence.proxy.async ; one elected thread issues 4 k-steps x passes MMAs of
//   M = 128, N = 128, K = 8 and commits them to the stage's mbarrier ; one stage per CTA,
//   two CTAs per SM.
//   Epilogue: tcgen05.ld of the 128 x 128 FP32 accumulator, FP64 partial tile to global;
//   k_gemm_hn_reduce (linalg.cu) sums the K-splits in a fixed order.
// Every wait is bounded; on timeout the kernel sets ST_TIMEOUT, waits (bounded) for its
// issued MMAs, frees its tensor memory and returns.
#include <stdint.h>

#include <algorithm>

#include "kernels.h"
#include "prof.h"
#include "tc.cuh"

namespace fde {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcM = 128;      // output rows (A rows) per CTA
constexpr int kTcN = 64;       // complex output columns (B rows) per CTA
constexpr int kTcKc = 16;      // complex K per k-tile (32 floats = one 128-byte row)
constexpr int kTile = 16384;   // bytes of one 128-row x 128-byte operand tile
constexpr int kStage = 4 * kTile;  // A hi, A lo, B hi, B lo
// One shared-memory stage per CTA and two CTAs per SM: twice the warps issuing the next
// k-tile's loads (the kernel is latency-bound) for the same buffering per SM.
constexpr int kStages = 1;
constexpr int kCtasPerSm = 2;
constexpr int kTmemCols = 128;
constexpr long long kSpin = kTcSpin;

__device__ unsigned g_tc_status;
// Poll limit of the waits for a shared-memory stage inside the K loop (settable from the host
// so that the timeout path can be exercised; the final drain always uses kSpin).
__device__ long long g_tc_stage_spin = kSpin;

// Instruction descriptor, kind::tf32: D f32 (bits 4-5 = 1), A and B tf32 (bits 7-9, 10-12
// = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(2 * kTcN / 8) << 17) |
                            ((uint32_t)(kTcM / 16) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t dt, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Byte offset of floats (c, c + 1) of row r in a 128-byte-swizzled tile (c even).
__device__ __forceinline__ uint32_t swz(int r, int c) {
  return (uint32_t)(r * 128 + ((((c >> 2) ^ (r & 7)) << 4) | ((c & 3) << 2)));
}
__device__ __forceinline__ void st2(uint32_t addr, float a, float b) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(a), "f"(b) : "memory");
}

constexpr int kAld = kTcM * kTcKc / kTcThreads;  // A elements per thread per k-tile (8)
constexpr int kBld = kTcN * kTcKc / kTcThreads;  // B elements per thread per k-tile (4)

__global__ void __launch_bounds__(kTcThreads, kCtasPerSm)
k_gemm_hn_tc(const float2* __restrict__ A, int lda, const float2* __restrict__ B, int ldb, int m, int n, int K,
             int kchunk, int passes, double2* __restrict__ part) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t base = (su32(smem_raw) + 1023u) & ~1023u;
  const int i0 = blockIdx.x * kTcM, j0 = blockIdx.y * kTcN;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  const int nt = ke > kb ? (ke - kb + kTcKc - 1) / kTcKc : 0;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(su32(&bars[s]), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  float2 ra[kAld], rb[kBld];
  auto load = [&](int t) {
    const int k0 = kb + t * kTcKc;
#pragma unroll
    for (int q = 0; q < kAld; ++q) {
      const int idx = tid + kTcThreads * q, r = idx >> 4, kc = idx & 15;
      const int i = i0 + r, k = k0 + kc;
      ra[q] = (i < m && k < ke) ? __ldg(A + (size_t)i * lda + k) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < kBld; ++q) {
      const int idx = tid + kTcThreads * q, r = idx >> 4, kc = idx & 15;
      const int j = j0 + r, k = k0 + kc;
      rb[q] = (j < n && k < ke) ? __ldg(B + (size_t)j * ldb + k) : make_float2(0.f, 0.f);
    }
  };
  auto store = [&](uint32_t st) {
#pragma unroll
    for (int q = 0; q < kAld; ++q) {
      const int idx = tid + kTcThreads * q, r = idx >> 4, c = 2 * (idx & 15);
      const float hx = tf32_hi(ra[q].x), hy = tf32_hi(ra[q].y);
      st2(st + swz(r, c), hx, hy);
      if (passes > 1) st2(st + kTile + swz(r, c), ra[q].x - hx, ra[q].y - hy);
    }
#pragma unroll
    for (int q = 0; q < kBld; ++q) {
      const int idx = tid + kTcThreads * q, r = idx >> 4, c = 2 * (idx & 15);
      const float hx = tf32_hi(rb[q].x), hy = tf32_hi(rb[q].y);
      st2(st + 2 * kTile + swz(r, c), hx, hy);                // b
      st2(st + 2 * kTile + swz(r + kTcN, c), hy, -hx);        // b~ = (Im b, -Re b)
      if (passes > 1) {
        const float lx = rb[q].x - hx, ly = rb[q].y - hy;
        st2(st + 3 * kTile + swz(r, c), lx, ly);
        st2(st + 3 * kTile + swz(r + kTcN, c), ly, -lx);
      }
    }
  };

  int issued = 0;  // k-tiles whose MMAs were committed (meaningful in thread 0)
  if (nt > 0) load(0);
  for (int t = 0; t < nt; ++t) {
    const int s = t % kStages;
    const uint32_t st = base + (uint32_t)s * kStage;
    if (t >= kStages) {
      // stage s is free once the MMAs of tile t - kStages have completed
      if (tid == 0 && !mbar_wait(su32(&bars[s]), (unsigned)(((t - kStages) / kStages) & 1), g_tc_stage_spin))
        abort_flag = 1;
      __syncthreads();
      if (abort_flag) break;
    }
    store(st);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < kTcKc * 2 / 8; ++kk) {
        const uint32_t off = (uint32_t)kk * 32u;
        const uint64_t ah = sdesc(st + off), bh = sdesc(st + 2 * kTile + off);
        mma_tf32(tmem, ah, bh, (t > 0 || kk > 0) ? 1u : 0u);
        if (passes > 1) {
          const uint64_t al = sdesc(st + kTile + off), bl = sdesc(st + 3 * kTile + off);
          mma_tf32(tmem, ah, bl, 1u);
          mma_tf32(tmem, al, bh, 1u);
        }
      }
      mma_commit(su32(&bars[s]));
      ++issued;
    }
    if (t + 1 < nt) load(t + 1);
  }

  // wait for the last commit of each stage: every issued MMA has completed
  __shared__ int drained;
  if (tid == 0) {
    drained = 1;
    for (int s = 0; s < kStages && s < issued; ++s) {
      const int uses = (issued - s + kStages - 1) / kStages;
      if (!mbar_wait(su32(&bars[s]), (unsigned)((uses - 1) & 1))) drained = 0;
    }
  }
  __syncthreads();
  const bool ok = !abort_flag && drained;
  if (!ok && tid == 0) atomicOr(&g_tc_status, drained ? ST_TIMEOUT : (ST_TIMEOUT | ST_TMEM_HELD));
  tc_fence_after();
  if (ok) {
    // warp w reads accumulator lanes 32 (w % 4) .. + 31 (its rows); warps 0-3 take the
    // complex columns 0..31, warps 4-7 the columns 32..63
    const int q = warp & 3, h = warp >> 2;
    const int r = 32 * q + lane, i = i0 + r;
    const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
    double2* P = part + ((size_t)blockIdx.z * m + (size_t)(i < m ? i : 0)) * n;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int jc = 32 * h + 16 * half;
      float re[16], im[16];
      if (nt > 0) {
        tmem_ld16(trow + (uint32_t)jc, re);
        tmem_ld16(trow + (uint32_t)(kTcN + jc), im);
      } else {
#pragma unroll
        for (int x = 0; x < 16; ++x) re[x] = im[x] = 0.f;
      }
      if (i < m) {
#pragma unroll
        for (int x = 0; x < 16; ++x) {
          const int j = j0 + jc + x;
          if (j < n) P[j] = make_double2((double)re[x], (double)im[x]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  // Tensor memory is released only once every issued MMA is known to have completed; if the
  // drain ran out, the columns stay allocated (an MMA may still write them) and the host,
  // seeing ST_TMEM_HELD, stops using the tensor-core kernels in this process.
  if (warp == 0 && drained) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}


// ---- Y = alpha sum_i U[i][j] X_i + beta Y (band-block rotation, projector expansion) ------------
// One real GEMM per CTA: D[j][p] = sum_(i, c) A[j][(i, c)] B[p][(i, c)] over the interleaved
// K index (i, c), c in {re, im}, with A[j][(i, 0)] = Re U_ij, A[j][(i, 1)] = Im U_ij and, for
// the 128 plane waves g of the tile, rows p = g (real part of Y) and p = 128 + g (imaginary
// part):  B[g][(i, 0)] = Re X_ig, B[g][(i, 1)] = -Im X_ig;  B[128 + g][(i, 0)] = Im X_ig,
// B[128 + g][(i, 1)] = Re X_ig.  M = 128 output rows j, N = 256, K = 8 per MMA; the same
// split-TF32 passes as the inner product; 128 x 256 FP32 accumulator in tensor memory.
constexpr int kRotJ = 128;             // output rows per CTA
constexpr int kRotG = 128;             // complex plane waves per CTA
constexpr int kRotKi = 16;             // input rows i per k-tile (32 floats)
constexpr int kRotA = kRotJ * 128;     // bytes of one A tile (16 KB)
constexpr int kRotB = 2 * kRotG * 128; // bytes of one B tile (32 KB)
constexpr int kRotStage = 2 * kRotA + 2 * kRotB;
constexpr int kRotStages = 2;
constexpr int kRotTmemCols = 256;
constexpr int kRotPitch = 2 * kRotG + 4;  // floats per row of the staged accumulator
static_assert((size_t)kRotJ * kRotPitch * 4 <= (size_t)kRotStages * (2 * kRotJ * 128 + 4 * kRotG * 128),
              "staged accumulator fits the stage buffers");
constexpr uint32_t kIdescRot = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(2 * kRotG / 8) << 17) |
                               ((uint32_t)(kRotJ / 16) << 24);

__device__ __forceinline__ void mma_tf32_rot(uint32_t dt, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
      "l"(a), "l"(b), "r"(kIdescRot), "r"(acc)
      : "memory");
}

constexpr int kRotXld = kRotKi * kRotG / kTcThreads;  // X elements per thread per k-tile (8)
constexpr int kRotUld = kRotKi * kRotJ / kTcThreads;  // U elements per thread per k-tile (8)

__global__ void __launch_bounds__(kTcThreads, 1)
k_gemm_rot_tc(const float2* __restrict__ X, int ldx, const double2* __restrict__ U, int ldu, int m, int n, int K,
              float2* __restrict__ Y, int ldy, float alpha, float beta, int passes) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kRotStages];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t base = (su32(smem_raw) + 1023u) & ~1023u;
  const int g0 = blockIdx.x * kRotG, j0 = blockIdx.y * kRotJ;
  const int nt = (m + kRotKi - 1) / kRotKi;

  if (tid == 0) {
    for (int q = 0; q < kRotStages; ++q) mbar_init(su32(&bars[q]), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                 "r"(kRotTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // element q of a thread: input row ii = 2 (q) + (tid & 1), plane wave (or output row) tid >> 1,
  // so pairs of threads read two rows at the same column (coalesced 8-byte runs) and a warp's
  // shared-memory stores cover 16 swizzled rows without conflicts beyond the 2 wavefronts
  float2 rx[kRotXld];
  double2 ru[kRotUld];
  auto load = [&](int t) {
    const int i0 = t * kRotKi;
#pragma unroll
    for (int q = 0; q < kRotXld; ++q) {
      const int ii = 2 * q + (tid & 1), gg = tid >> 1;
      const int i = i0 + ii, g = g0 + gg;
      rx[q] = (i < m && g < K) ? __ldg(X + (size_t)i * ldx + g) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < kRotUld; ++q) {
      const int ii = 2 * q + (tid & 1), jj = tid >> 1;
      const int i = i0 + ii, j = j0 + jj;
      ru[q] = (i < m && j < n) ? __ldg(U + (size_t)i * ldu + j) : make_double2(0.0, 0.0);
    }
  };
  auto store = [&](uint32_t st) {
#pragma unroll
    for (int q = 0; q < kRotUld; ++q) {
      const int ii = 2 * q + (tid & 1), jj = tid >> 1, c = 2 * ii;
      const float ur = (float)ru[q].x, ui = (float)ru[q].y;
      const float hr = tf32_hi(ur), hi = tf32_hi(ui);
      st2(st + swz(jj, c), hr, hi);
      if (passes > 1) st2(st + kRotA + swz(jj, c), ur - hr, ui - hi);
    }
#pragma unroll
    for (int q = 0; q < kRotXld; ++q) {
      const int ii = 2 * q + (tid & 1), gg = tid >> 1, c = 2 * ii;
      const float xr = rx[q].x, xi = rx[q].y;
      const float hr = tf32_hi(xr), hi = tf32_hi(xi);
      const uint32_t b = st + 2 * kRotA;
      st2(b + swz(gg, c), hr, -hi);
      st2(b + swz(kRotG + gg, c), hi, hr);
      if (passes > 1) {
        const float lr = xr - hr, li = xi - hi;
        st2(b + kRotB + swz(gg, c), lr, -li);
        st2(b + kRotB + swz(kRotG + gg, c), li, lr);
      }
    }
  };

  int issued = 0;
  if (nt > 0) load(0);
  for (int t = 0; t < nt; ++t) {
    const int s = t % kRotStages;
    const uint32_t st = base + (uint32_t)s * kRotStage;
    if (t >= kRotStages) {
      if (tid == 0 && !mbar_wait(su32(&bars[s]), (unsigned)(((t - kRotStages) / kRotStages) & 1), g_tc_stage_spin))
        abort_flag = 1;
      __syncthreads();
      if (abort_flag) break;
    }
    store(st);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < kRotKi * 2 / 8; ++kk) {
        const uint32_t off = (uint32_t)kk * 32u;
        const uint64_t ah = sdesc(st + off), bh = sdesc(st + 2 * kRotA + off);
        mma_tf32_rot(tmem, ah, bh, (t > 0 || kk > 0) ? 1u : 0u);
        if (passes > 1) {
          const uint64_t al = sdesc(st + kRotA + off), bl = sdesc(st + 2 * kRotA + kRotB + off);
          mma_tf32_rot(tmem, ah, bl, 1u);
          mma_tf32_rot(tmem, al, bh, 1u);
        }
      }
      mma_commit(su32(&bars[s]));
      ++issued;
    }
    if (t + 1 < nt) load(t + 1);
  }
  __shared__ int drained;
  if (tid == 0) {
    drained = 1;
    for (int s = 0; s < kRotStages && s < issued; ++s) {
      const int uses = (issued - s + kRotStages - 1) / kRotStages;
      if (!mbar_wait(su32(&bars[s]), (unsigned)((uses - 1) & 1))) drained = 0;
    }
  }
  __syncthreads();
  const bool ok = !abort_flag && drained;
  if (!ok && tid == 0) atomicOr(&g_tc_status, drained ? ST_TIMEOUT : (ST_TIMEOUT | ST_TMEM_HELD));
  tc_fence_after();
  if (ok) {
    // Accumulator -> shared memory (the stage buffers are free: every MMA has completed), then a
    // read-modify-write of Y with consecutive threads on consecutive plane waves.
    // Ds[j][p], row pitch kRotPitch floats (a pitch of 4 mod 32 words keeps the 16-byte stores
    // of eight consecutive rows on distinct banks).
    float* Ds = reinterpret_cast<float*>(smem_raw + (base - su32(smem_raw)));
    {
      const int q = warp & 3, h = warp >> 2;
      const int r = 32 * q + lane;
      const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
#pragma unroll 1
      for (int c16 = 0; c16 < 8; ++c16) {
        const int pc = 128 * h + 16 * c16;
        float v[16];
        if (nt > 0) {
          tmem_ld16(trow + (uint32_t)pc, v);
        } else {
#pragma unroll
          for (int x = 0; x < 16; ++x) v[x] = 0.f;
        }
        float4* dst = reinterpret_cast<float4*>(Ds + (size_t)r * kRotPitch + pc);
#pragma unroll
        for (int x = 0; x < 4; ++x) dst[x] = make_float4(v[4 * x], v[4 * x + 1], v[4 * x + 2], v[4 * x + 3]);
      }
    }
    __syncthreads();
    const int gg = tid & (kRotG - 1), jr = tid >> 7;  // 128 plane waves x 2 rows per pass
    const int g = g0 + gg;
    if (g < K) {
#pragma unroll 4
      for (int jj = jr; jj < kRotJ; jj += kTcThreads / kRotG) {
        const int j = j0 + jj;
        if (j >= n) break;
        float2 o = make_float2(alpha * Ds[(size_t)jj * kRotPitch + gg], alpha * Ds[(size_t)jj * kRotPitch + kRotG + gg]);
        float2* y = Y + (size_t)j * ldy + g;
        if (beta != 0.f) {
          const float2 old = *y;
          o.x += beta * old.x;
          o.y += beta * old.y;
        }
        *y = o;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0 && drained) {  // as in k_gemm_hn_tc: held if the drain ran out
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kRotTmemCols) : "memory");
  }
}

}  // namespace

// K-splits of the tensor-core product: about two resident CTAs per SM over the grid, at
// least eight k-tiles per split.
int gemm_hn_tc_splits(int m, int n, int K) {
  const int tiles = ceil_div(m, kTcM) * ceil_div(n, kTcN);
  int s = ceil_div(2 * 152, tiles);
  const int smax = std::max(1, ceil_div(K, 8 * kTcKc));
  return std::max(1, std::min(s, smax));
}

size_t gemm_hn_tc_smem() { return (size_t)kStages * kStage + 1024; }

// Partial tiles of C = A^H B into part[nsplit][m][n]; returns the number of splits (0 if the
// kernel could not be configured; nothing is launched then).
int launch_gemm_hn_tc(const float2* A, int lda, const float2* B, int ldb, int m, int n, int K, int passes,
                      double2* part, cudaStream_t st) {
  static int attr = 0;  // 1 configured, -1 failed
  if (attr == 0)
    attr = cudaFuncSetAttribute(k_gemm_hn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)gemm_hn_tc_smem()) == cudaSuccess ? 1 : -1;
  if (attr < 0) return 0;
  const int s = gemm_hn_tc_splits(m, n, K);
  int kchunk = ceil_div(K, s);
  kchunk = ((kchunk + kTcKc - 1) / kTcKc) * kTcKc;
  const int ns = std::max(1, ceil_div(K, std::max(kchunk, 1)));
  const dim3 grid(ceil_div(m, kTcM), ceil_div(n, kTcN), ns);
  count_launches(1);
  ProfScope p("k_gemm_hn_tc", st);
  k_gemm_hn_tc<<<grid, kTcThreads, gemm_hn_tc_smem(), st>>>(A, lda, B, ldb, m, n, K, kchunk, passes, part);
  return ns;
}

// Status bits raised by the tensor-core kernels since the last call (read and cleared;
// synchronises the stream).  A kernel that could not confirm its MMAs complete kept its
// tensor memory (ST_TMEM_HELD): from then on the products run on the CUDA cores.
unsigned gemm_tc_take_status(cudaStream_t st) {
  unsigned h = 0, z = 0;
  if (cudaMemcpyFromSymbolAsync(&h, g_tc_status, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return 0;  // the stream's own error surfaces at the caller's next check
  if (h) cudaMemcpyToSymbolAsync(g_tc_status, &z, sizeof(unsigned), 0, cudaMemcpyHostToDevice, st);
  if (h & ST_TMEM_HELD) disable_tensor_cores();
  return h;
}

// Poll limit of the tensor-core kernels' stage waits (polls < 0: the default bound).
bool set_tc_stage_spin(long long polls) {
  const long long v = polls < 0 ? kSpin : std::min(polls, kSpin);
  return cudaMemcpyToSymbol(g_tc_stage_spin, &v, sizeof(v)) == cudaSuccess;
}

}  // namespace fde

namespace fde {

size_t gemm_rot_tc_smem() { return (size_t)kRotStages * kRotStage + 1024; }

// Y = alpha U^T-combination of the rows of X + beta Y on the tensor cores; returns false if the
// kernel could not be configured (nothing launched).
bool launch_gemm_rot_tc(const float2* X, int ldx, const double2* U, int ldu, int m, int n, int K, float2* Y,
                        int ldy, double alpha, double beta, int passes, cudaStream_t st) {
  static int attr = 0;
  if (attr == 0)
    attr = cudaFuncSetAttribute(k_gemm_rot_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)gemm_rot_tc_smem()) == cudaSuccess ? 1 : -1;
  if (attr < 0) return false;
  const dim3 grid(ceil_div(K, kRotG), ceil_div(n, kRotJ));
  count_launches(1);
  ProfScope p("k_gemm_rot_tc", st);
  k_gemm_rot_tc<<<grid, kTcThreads, gemm_rot_tc_smem(), st>>>(X, ldx, U, ldu, m, n, K, Y, ldy, (float)alpha,
                                                               (float)beta, passes);
  return true;
}

}  // namespace fde
