// sg_mlp.cu -- the dense contractions of the learned one-day emulator on the
// fifth-generation tensor cores (tcgen05, accumulators in tensor memory), and
// the small element-wise kernels around them (loss, optimiser, features,
// sampling).  The emulator is an extension of the method, not part of the
// paper.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "sg_common.h"
#include "sg_device.cuh"
#include "sg_mlp.h"
#include "sg_tc.cuh"

using namespace sg;

namespace {

constexpr int kBM = 128;              // rows per tile (tensor-core M)
constexpr int kBK = 64;               // K per pipeline stage
constexpr uint32_t kWaitLimit = 1u << 24;  // mbarrier polls before giving up

// Byte offset of element (row, k) of a rows x 64 BF16 stage in the
// no-swizzle K-major core-matrix layout: 8-row x 8-element (16 byte) core
// matrices, the 8 core matrices of an 8-row group consecutive along K.
__device__ __forceinline__ uint32_t stage_off(int row, int kgroup) {
  return (uint32_t)(((row >> 3) * 8 + kgroup) * 128 + (row & 7) * 16);
}

// 16-byte asynchronous global-to-shared copy; src_bytes = 0 zero-fills.
__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *gsrc, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(gsrc),
               "r"(src_bytes)
               : "memory");
}

// GELU in its tanh form, 0.5 x (1 + tanh(sqrt(2 / pi) (x + 0.044715 x^3))),
// with the hardware tanh approximation (relative error ~2^-11, below the
// BF16 rounding of the activations).
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float gelu(float x) {
  const float u = 0.7978845608028654f * (x + 0.044715f * x * x * x);
  return 0.5f * x * (1.0f + tanh_fast(u));
}

// C = act(A . Bt^T + bias) for one 128 x BN tile.  A: M x K, Bt: N x K, both
// row-major BF16 with K contiguous (K % 8 == 0, rows 16-byte aligned).
// 256 threads: all load the double-buffered K stages into shared memory
// (cp.async, overlapping the previous stage's MMAs), thread 0 issues the MMAs
// (4 per stage, K = 16 each) and commits them to the stage's mbarrier; in the
// epilogue warp w reads TMEM lane quarter w % 4 (32 tile rows), columns of
// half w / 4 of the tile.
//
// F8: A and B are FP8 E4M3 bytes instead (K = 128 per stage, the same 128
// bytes per row; tcgen05.mma kind::f8f6f4 with K = 32 per instruction, the
// same 32 bytes), and the accumulator is scaled by a_scale * b_scale[n].
// Optional outputs: FP32 before the activation, BF16 after it, FP8 E4M3
// after it (scaled by c8_inv_scale, saturated to the finite range).
constexpr int kGemmThreads = 256;
template <int BN, bool F8>
__global__ void __launch_bounds__(kGemmThreads) k_gemm_tc(const GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int kStageK = F8 ? 2 * kBK : kBK;    // elements of K per stage
  constexpr uint32_t kAStage = kBM * kBK * 2;  // 16 KB (128 bytes per row)
  constexpr uint32_t kBStage = BN * kBK * 2;
  unsigned char *sA[2] = {smem, smem + kAStage};
  unsigned char *sB[2] = {smem + 2 * kAStage, smem + 2 * kAStage + kBStage};
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_mbar_init();
    s_fail = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tmem_slot, BN);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  constexpr uint32_t idesc = F8 ? tc::idesc_e4m3_f32(kBM, BN) : tc::idesc_bf16_f32(kBM, BN);
  const int stages = (g.K + kStageK - 1) / kStageK;
  uint32_t uses[2] = {0, 0};
  bool ok = true;

  // Stage loader: every thread issues its 16-byte asynchronous copies
  // (cp.async) for stage s into buffer s & 1, rows past M / N and columns
  // past K are zero-filled.
  auto load_stage = [&](int s) {
    const int b = s & 1, k0 = s * kStageK;
    constexpr int kChunk = F8 ? 16 : 8;  // elements per 16-byte chunk
    const uint32_t a0 = tc::smem_u32(sA[b]), b0 = tc::smem_u32(sB[b]);
    for (int idx = tid; idx < kBM * 8; idx += kGemmThreads) {
      const int r = idx >> 3, kg = idx & 7;
      const int m = m0 + r, k = k0 + kg * kChunk;
      const bool in = m < g.M && k < g.K;
      const void *src;
      if constexpr (F8)
        src = in ? (const void *)(g.A8 + (long long)m * g.lda + k) : (const void *)g.A8;
      else
        src = in ? (const void *)(g.A + (long long)m * g.lda + k) : (const void *)g.A;
      cp_async16(a0 + stage_off(r, kg), src, in ? 16 : 0);
    }
    for (int idx = tid; idx < BN * 8; idx += kGemmThreads) {
      const int r = idx >> 3, kg = idx & 7;
      const int n = n0 + r, k = k0 + kg * kChunk;
      const bool in = n < g.N && k < g.K;
      const void *src;
      if constexpr (F8)
        src = in ? (const void *)(g.B8 + (long long)n * g.ldb + k) : (const void *)g.B8;
      else
        src = in ? (const void *)(g.Bt + (long long)n * g.ldb + k) : (const void *)g.Bt;
      cp_async16(b0 + stage_off(r, kg), src, in ? 16 : 0);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  if (stages > 0) load_stage(0);
  for (int s = 0; s < stages && ok; ++s) {
    const int b = s & 1;
    // stage s has landed in shared memory
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::tc_fence_after();
      const uint32_t a0 = tc::smem_u32(sA[b]), b0 = tc::smem_u32(sB[b]);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        // two core matrices along K per MMA: +256 bytes per K step of 16
        const uint64_t ad = tc::smem_desc(a0 + kk * 256, 128, 1024);
        const uint64_t bd = tc::smem_desc(b0 + kk * 256, 128, 1024);
        if constexpr (F8)
          tc::mma_e4m3(tmem, ad, bd, idesc, (s > 0 || kk > 0) ? 1u : 0u);
        else
          tc::mma_bf16(tmem, ad, bd, idesc, (s > 0 || kk > 0) ? 1u : 0u);
      }
      tc::mma_commit(&bar[b]);
    }
    ++uses[b];
    if (s + 1 < stages) {
      // the other buffer is free once the MMAs of stage s - 1 are done; its
      // loads then overlap the MMAs of stage s
      const int nb = (s + 1) & 1;
      if (uses[nb] > 0 && !tc::mbar_wait(&bar[nb], (uses[nb] - 1) & 1, kWaitLimit)) s_fail = 1;
      __syncthreads();
      if (s_fail) {
        ok = false;
        break;
      }
      load_stage(s + 1);
    }
  }
  // all MMAs done: the last stage's commit completes after every earlier one
  if (ok && stages > 0) {
    const int b = (stages - 1) & 1;
    if (!tc::mbar_wait(&bar[b], (uses[b] - 1) & 1, kWaitLimit)) ok = false;
  }
  if (!ok) {
    if (tid == 0) atomicExch(g.err, SG_ERR_TIMEOUT);
    // let MMAs still in flight finish (bounded) before the TMEM is freed
    for (int b = 0; b < 2; ++b)
      if (uses[b]) tc::mbar_wait(&bar[b], (uses[b] - 1) & 1, kWaitLimit);
  } else {
    // Epilogue.  Warp w reads TMEM lanes 32 (w % 4) .. + 31 (tile rows) and
    // the columns of half w / 4.  FP32 results go out as 16-byte vectors;
    // BF16 results are staged in shared memory (the stage buffers are free
    // now) and then written row by row, each warp storing whole rows.
    tc::tc_fence_after();
    constexpr int kPitch = BN * 2 + 16;  // bytes per staged row (bank offset)
    unsigned char *stage = smem;
    const int q = warp & 3, half = warp >> 2;
    const int lr = q * 32 + lane;
    const int row = m0 + lr;
    const bool vec32 = g.C32 && (g.ldc32 % 4) == 0 && (((uintptr_t)g.C32) & 15) == 0;
    for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
      const int nb = n0 + c;
      if constexpr (F8) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          v[i] *= g.a_scale * ((nb + i < g.N) ? __ldg(g.b_scale + nb + i) : 0.0f);
      }
      if (g.bias) {
        if (nb + 16 <= g.N && (((uintptr_t)(g.bias + nb)) & 15) == 0) {
#pragma unroll
          for (int i = 0; i < 16; i += 4) {
            const float4 b4 = __ldg(reinterpret_cast<const float4 *>(g.bias + nb + i));
            v[i] += b4.x;
            v[i + 1] += b4.y;
            v[i + 2] += b4.z;
            v[i + 3] += b4.w;
          }
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] += (nb + i < g.N) ? __ldg(g.bias + nb + i) : 0.0f;
        }
      }
      if (g.C32 && row < g.M) {
        float *dst = g.C32 + (long long)row * g.ldc32 + nb;
        if (vec32 && nb + 16 <= g.N) {
#pragma unroll
          for (int i = 0; i < 16; i += 4)
            *reinterpret_cast<float4 *>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        } else {
          for (int i = 0; i < 16 && nb + i < g.N; ++i) dst[i] = v[i];
        }
      }
      if (g.C16 || g.C8) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (g.act == 1) v[i] = gelu(v[i]);
      }
      if (g.C16) {
        uint32_t packed[8];
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[i], v[i + 1]);
          packed[i / 2] = *reinterpret_cast<const uint32_t *>(&h2);
        }
        uint4 *sp = reinterpret_cast<uint4 *>(stage + lr * kPitch + c * 2);
        sp[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        sp[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
      }
      if (g.C8 && row < g.M) {
        // 16 E4M3 values of this row, one 16-byte store when it fits
        uint32_t packed[4];
#pragma unroll
        for (int i = 0; i < 16; i += 4) {
          const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(
              make_float2(v[i] * g.c8_inv_scale, v[i + 1] * g.c8_inv_scale), __NV_SATFINITE,
              __NV_E4M3);
          const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(
              make_float2(v[i + 2] * g.c8_inv_scale, v[i + 3] * g.c8_inv_scale), __NV_SATFINITE,
              __NV_E4M3);
          packed[i / 4] = (uint32_t)lo | ((uint32_t)hi << 16);
        }
        uint8_t *dst = g.C8 + (long long)row * g.ldc8 + nb;
        if (nb + 16 <= g.N && (((uintptr_t)dst) & 15) == 0) {
          *reinterpret_cast<uint4 *>(dst) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        } else {
          const uint8_t *bytes = reinterpret_cast<const uint8_t *>(packed);
          for (int i = 0; i < 16 && nb + i < g.N; ++i) dst[i] = bytes[i];
        }
      }
    }
    if (g.C16) {
      __syncthreads();
      constexpr int kVecPerRow = BN * 2 / 16;
      const bool vec16 = (g.ldc16 % 8) == 0 && (((uintptr_t)g.C16) & 15) == 0;
      for (int idx = tid; idx < kBM * kVecPerRow; idx += kGemmThreads) {
        const int r = idx / kVecPerRow, j = idx - r * kVecPerRow;
        const int grow = m0 + r, col = n0 + j * 8;
        if (grow >= g.M || col >= g.N) continue;
        const uint4 val = *reinterpret_cast<const uint4 *>(stage + r * kPitch + j * 16);
        __nv_bfloat16 *dst = g.C16 + (long long)grow * g.ldc16 + col;
        if (vec16 && col + 8 <= g.N) {
          *reinterpret_cast<uint4 *>(dst) = val;
        } else {
          const __nv_bfloat16 *hv = reinterpret_cast<const __nv_bfloat16 *>(&val);
          for (int i = 0; i < 8 && col + i < g.N; ++i) dst[i] = hv[i];
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, BN);
}

std::mutex g_err_mu;
int *g_err_buf[64] = {};

int gemm_err_buf(int **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_err_mu);
  if (!g_err_buf[dev]) {
    if (cudaMalloc(&g_err_buf[dev], sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return SG_ERR_NOMEM;
    }
    cudaMemset(g_err_buf[dev], 0, sizeof(int));
  }
  *out = g_err_buf[dev];
  return SG_OK;
}

template <int BN, bool F8>
void launch_gemm(const GemmArgs &g, cudaStream_t st) {
  const size_t smem = 2 * ((size_t)kBM * kBK * 2 + (size_t)BN * kBK * 2);
  static unsigned long long attr_set = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !((attr_set >> dev) & 1ull)) {
    cudaFuncSetAttribute(k_gemm_tc<BN, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr_set |= 1ull << dev;
  }
  const dim3 grid((unsigned)((g.M + kBM - 1) / kBM), (unsigned)((g.N + BN - 1) / BN));
  k_gemm_tc<BN, F8><<<grid, kGemmThreads, smem, st>>>(g);
}

}  // namespace

namespace sg {

int gemm_bf16(const GemmArgs &g0, cudaStream_t st) {
  GemmArgs g = g0;
  const bool f8 = g.f8 != 0;
  const int align = f8 ? 16 : 8;  // elements per 16 bytes
  const void *A = f8 ? (const void *)g.A8 : (const void *)g.A;
  const void *B = f8 ? (const void *)g.B8 : (const void *)g.Bt;
  if (g.M < 0 || g.N < 0 || g.K < 0 || (g.K % align) != 0 || g.lda < g.K || g.ldb < g.K ||
      (g.lda % align) != 0 || (g.ldb % align) != 0 || !A || !B ||
      (!g.C32 && !g.C16 && !g.C8) || (((uintptr_t)A | (uintptr_t)B) & 15) != 0 ||
      (f8 && !g.b_scale) || (g.C8 && g.ldc8 < g.N))
    return SG_ERR_ARG;
  if (g.M == 0 || g.N == 0) return SG_OK;
  if (!g.err) {
    int rc = gemm_err_buf(&g.err);
    if (rc) return rc;
  }
  if (f8) {
    if (g.N <= 64)
      launch_gemm<64, true>(g, st);
    else if (g.N <= 128)
      launch_gemm<128, true>(g, st);
    else
      launch_gemm<256, true>(g, st);
  } else {
    if (g.N <= 64)
      launch_gemm<64, false>(g, st);
    else if (g.N <= 128)
      launch_gemm<128, false>(g, st);
    else
      launch_gemm<256, false>(g, st);
  }
  return SG_OK;
}

int gemm_prepare() {
  int *e = nullptr;
  return gemm_err_buf(&e);
}

int gemm_check(cudaStream_t st) {
  int *e = nullptr;
  int rc = gemm_err_buf(&e);
  if (rc) return rc;
  int h = 0;
  if (cudaMemcpyAsync(&h, e, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  if (h) {
    cudaMemsetAsync(e, 0, sizeof(int), st);
    return h;
  }
  return SG_OK;
}

}  // namespace sg

extern "C" int sg_gemm_bf16(const void *A, int32_t lda, const void *Bt, int32_t ldb, int32_t M,
                            int32_t N, int32_t K, const float *bias, int32_t act, float *C32,
                            int32_t ldc32, void *C16, int32_t ldc16, void *stream) {
  GemmArgs g{};
  g.A = (const __nv_bfloat16 *)A;
  g.lda = lda;
  g.Bt = (const __nv_bfloat16 *)Bt;
  g.ldb = ldb;
  g.M = M;
  g.N = N;
  g.K = K;
  g.bias = bias;
  g.act = act;
  g.C32 = C32;
  g.ldc32 = ldc32;
  g.C16 = (__nv_bfloat16 *)C16;
  g.ldc16 = ldc16;
  g.err = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  const int rc = sg::gemm_bf16(g, st);
  if (rc) return rc;
  return sg::gemm_check(st);
}

extern "C" int sg_gemm_bf16_to_fp8(const void *A, int32_t lda, const void *Bt, int32_t ldb,
                                   int32_t M, int32_t N, int32_t K, const float *bias,
                                   int32_t act, void *C8, int32_t ldc8, float c8_inv_scale,
                                   void *stream) {
  GemmArgs g{};
  g.A = (const __nv_bfloat16 *)A;
  g.lda = lda;
  g.Bt = (const __nv_bfloat16 *)Bt;
  g.ldb = ldb;
  g.M = M;
  g.N = N;
  g.K = K;
  g.bias = bias;
  g.act = act;
  g.C8 = (uint8_t *)C8;
  g.ldc8 = ldc8;
  g.c8_inv_scale = c8_inv_scale;
  g.err = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  const int rc = sg::gemm_bf16(g, st);
  if (rc) return rc;
  return sg::gemm_check(st);
}

extern "C" int sg_gemm_fp8(const void *A8, int32_t lda, const void *B8, int32_t ldb, int32_t M,
                           int32_t N, int32_t K, float a_scale, const float *b_scale,
                           const float *bias, int32_t act, float *C32, int32_t ldc32,
                           void *C16, int32_t ldc16, void *C8, int32_t ldc8,
                           float c8_inv_scale, void *stream) {
  GemmArgs g{};
  g.f8 = 1;
  g.A8 = (const uint8_t *)A8;
  g.lda = lda;
  g.B8 = (const uint8_t *)B8;
  g.ldb = ldb;
  g.M = M;
  g.N = N;
  g.K = K;
  g.a_scale = a_scale;
  g.b_scale = b_scale;
  g.bias = bias;
  g.act = act;
  g.C32 = C32;
  g.ldc32 = ldc32;
  g.C16 = (__nv_bfloat16 *)C16;
  g.ldc16 = ldc16;
  g.C8 = (uint8_t *)C8;
  g.ldc8 = ldc8;
  g.c8_inv_scale = c8_inv_scale;
  g.err = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  const int rc = sg::gemm_bf16(g, st);
  if (rc) return rc;
  return sg::gemm_check(st);
}

// ---------------------------------------------------------------------------
// Element-wise kernels of the emulator: training loss, GELU backward,
// transposes, bias gradients, Adam, input features, output sampling.
// ---------------------------------------------------------------------------

namespace {

constexpr int kHeads = 3;    // one head per age class
constexpr int kBins = 129;   // increments -64 .. 64
constexpr int kHalf = 64;

// d/dx of the tanh-form GELU: 0.5 (1 + t) + 0.5 x (1 - t^2) c (1 + 3 a x^2)
__device__ __forceinline__ float gelu_grad(float x) {
  const float c = 0.7978845608028654f, a = 0.044715f;
  const float t = tanh_fast(c * (x + a * x * x * x));
  return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * c * (1.0f + 3.0f * a * x * x);
}

// Cross-entropy over the three 129-way heads, one warp per row: loss and
// d loss / d logits (scaled by 1 / B, BF16; padding columns get 0).
__global__ void k_ce_loss(const float *__restrict__ logits, int ldl,
                          const int32_t *__restrict__ tgt, int B, __nv_bfloat16 *dlog, int ldd,
                          int ncols_grad, double *loss_sum) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= B) return;
  const float *row = logits + (long long)warp * ldl;
  __nv_bfloat16 *grow = dlog + (long long)warp * ldd;
  const float invB = 1.0f / (float)B;
  float loss = 0.0f;
  for (int h = 0; h < kHeads; ++h) {
    const float *lg = row + h * kBins;
    float mx = -INFINITY;
    for (int c = lane; c < kBins; c += 32) mx = fmaxf(mx, lg[c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float se = 0.0f;
    for (int c = lane; c < kBins; c += 32) se += expf(lg[c] - mx);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    const float lz = mx + logf(se);
    const int t = tgt[(long long)warp * kHeads + h];
    if (lane == 0) loss += lz - lg[t];
    for (int c = lane; c < kBins; c += 32) {
      const float p = expf(lg[c] - lz) - (c == t ? 1.0f : 0.0f);
      grow[h * kBins + c] = __float2bfloat16_rn(p * invB);
    }
  }
  for (int c = kHeads * kBins + lane; c < ncols_grad; c += 32) grow[c] = __float2bfloat16_rn(0.0f);
  if (lane == 0) atomicAdd(loss_sum, (double)loss);
}

__global__ void k_gelu_bwd(const float *__restrict__ dpost, const float *__restrict__ pre,
                           long long n, __nv_bfloat16 *dpre) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dpre[i] = __float2bfloat16_rn(dpost[i] * gelu_grad(pre[i]));
}

// dst[c][r] = src[r][c] through 32 x 32 shared-memory tiles.
__global__ void k_transpose(const __nv_bfloat16 *__restrict__ src, int rows, int cols,
                            __nv_bfloat16 *dst) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = src[(long long)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[(long long)c * rows + r] = tile[threadIdx.x][i];
  }
}

// FP8 quantisation.  Per row of W (rows x cols, FP32): scale = max |w| /
// 448 (the largest finite E4M3 value; 1 for a zero row), W8 = e4m3(w /
// scale) rounded to nearest even and saturated.  One block per row.
__global__ void k_quant_rows_fp8(const float *__restrict__ W, int rows, int cols, uint8_t *W8,
                                 float *scale) {
  __shared__ float s_max[8];
  const int r = blockIdx.x;
  const float *w = W + (long long)r * cols;
  float m = 0.0f;
  for (int k = threadIdx.x; k < cols; k += blockDim.x) m = fmaxf(m, fabsf(w[k]));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = m;
  __syncthreads();
  float mx = 0.0f;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mx = fmaxf(mx, s_max[i]);
  const float sc = mx > 0.0f ? mx / 448.0f : 1.0f;
  if (threadIdx.x == 0) scale[r] = sc;
  for (int k = threadIdx.x; k < cols; k += blockDim.x)
    W8[(long long)r * cols + k] =
        (uint8_t)__nv_cvt_float_to_fp8(w[k] / sc, __NV_SATFINITE, __NV_E4M3);
}

// x8 = e4m3(x * inv_scale) for BF16 x, saturated.
__global__ void k_quant_bf16_fp8(const __nv_bfloat16 *__restrict__ x, long long n, float inv_scale,
                                 uint8_t *out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (uint8_t)__nv_cvt_float_to_fp8(__bfloat162float(x[i]) * inv_scale, __NV_SATFINITE,
                                            __NV_E4M3);
}

// *out = max |x_i| over BF16 x (out starts at 0; non-negative floats order
// like their bit patterns).
__global__ void k_absmax_bf16(const __nv_bfloat16 *__restrict__ x, long long n, float *out) {
  float m = 0.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(__bfloat162float(x[i])));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(out), __float_as_int(m));
}

__global__ void k_colsum(const __nv_bfloat16 *__restrict__ src, int rows, int cols, float *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.0f;
  for (int r = 0; r < rows; ++r) s += __bfloat162float(src[(long long)r * cols + c]);
  out[c] = s;
}

__global__ void k_adam(float *p, const float *__restrict__ g, float *m, float *v, long long n,
                       float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16 *p16) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (p16) p16[i] = __float2bfloat16_rn(pi);
  }
}

}  // namespace

namespace sg {

// Input features of one SISe3 node for the emulator, and whether the node is
// in the emulator's range (herd <= max_herd and phi_lo <= phi <= phi_hi).
__global__ void k_emu_features(const int32_t *__restrict__ u, const double *__restrict__ v,
                               long long units, EmuParams ep, __nv_bfloat16 *feat,
                               int32_t *flag) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < units;
       i += (long long)gridDim.x * blockDim.x) {
    const int32_t *un = u + i * 6;
    int herd = 0;
#pragma unroll
    for (int p = 0; p < 6; ++p) herd += un[p];
    const double phi = v[i];
    const bool in = herd <= ep.max_herd && phi >= ep.phi_lo && phi <= ep.phi_hi;
    flag[i] = in ? 1 : 0;
    float f[16];
#pragma unroll
    for (int p = 0; p < 6; ++p) f[p] = log1pf((float)max(un[p], 0));
    f[6] = (float)phi;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      f[7 + a] = 50.0f * (float)ep.gdata[a];
      f[10 + a] = 10.0f * (float)ep.gdata[3 + a];
    }
    f[13] = f[14] = f[15] = 0.0f;
    __nv_bfloat16 *row = feat + i * 16;
#pragma unroll
    for (int k = 0; k < 16; ++k) row[k] = __float2bfloat16_rn(f[k]);
  }
}

// Sample each in-range node's increments from the emulator's three heads:
// softmax over the 129 bins, inverse CDF at a uniform from the emulator's
// Philox stream (seed, replicate, node, day), and clamp so that neither S_a
// nor I_a becomes negative (each age class keeps its size within the day).
// One warp per node; lane l holds bins 5 l .. 5 l + 4.
__global__ void k_emu_sample(const float *__restrict__ logits, int ldl,
                             const int32_t *__restrict__ u, const int32_t *__restrict__ flag,
                             long long units, int n_nodes, uint32_t k0, uint32_t k1, int T,
                             int32_t *delta) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= units) return;
  int32_t *out = delta + w * 4;
  if (!flag[w]) {
    if (lane == 0) out[3] = 0;
    return;
  }
  const int rep = (int)(w / n_nodes), node = (int)(w - (long long)rep * n_nodes);
  const U4 x = philox10(U4{0u, (uint32_t)node, (uint32_t)T, (SG_STREAM_EMU << 24) | (uint32_t)rep},
                        k0, k1);
  const uint32_t words[3] = {x.x, x.y, x.z};
  const float *row = logits + w * ldl;
  for (int h = 0; h < kHeads; ++h) {
    const float *lg = row + h * kBins;
    float vals[5];
    float mx = -INFINITY;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const int c = lane * 5 + j;
      vals[j] = c < kBins ? lg[c] : -INFINITY;
      mx = fmaxf(mx, vals[j]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float part = 0.0f;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      vals[j] = lane * 5 + j < kBins ? expf(vals[j] - mx) : 0.0f;
      part += vals[j];
    }
    // inclusive scan of the lane sums
    float incl = part;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const float total = __shfl_sync(0xffffffffu, incl, 31);
    const float target = ((float)(words[h] >> 8) + 0.5f) * (1.0f / 16777216.0f) * total;
    // the lane whose range holds the target, then the bin inside it
    const unsigned ge = __ballot_sync(0xffffffffu, incl >= target);
    const int owner = ge ? __ffs(ge) - 1 : 31;
    int bin = kBins - 1;
    if (lane == owner) {
      float acc = incl - part;
      bin = min(lane * 5 + 4, kBins - 1);
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        acc += vals[j];
        if (acc >= target && lane * 5 + j < kBins) {
          bin = lane * 5 + j;
          break;
        }
      }
    }
    bin = __shfl_sync(0xffffffffu, bin, owner);
    if (lane == 0) {
      const int S = u[w * 6 + 2 * h], I = u[w * 6 + 2 * h + 1];
      int d = bin - kHalf;
      d = max(d, -I);
      d = min(d, S);
      out[h] = d;
    }
  }
  if (lane == 0) out[3] = 1;
}

// Training targets: the one-day increment of I_a, as a bin index in 0..128
// (clamped to the edge bins).
__global__ void k_emu_targets(const int32_t *__restrict__ u0, const int32_t *__restrict__ u1,
                              long long units, int32_t *tgt) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < units;
       i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int d = u1[i * 6 + 2 * a + 1] - u0[i * 6 + 2 * a + 1];
      tgt[i * 3 + a] = min(max(d + kHalf, 0), kBins - 1);
    }
  }
}

}  // namespace sg

static unsigned grid_n(long long n, int block) {
  return (unsigned)std::max<long long>(1, std::min<long long>(16384, (n + block - 1) / block));
}

static int finish(cudaStream_t st) {
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  return SG_OK;
}

extern "C" int sg_mlp_ce_loss(const float *logits, int32_t ldl, const int32_t *targets,
                              int32_t B, void *dlogits, int32_t ldd, double *loss_sum,
                              void *stream) {
  if (B < 0 || ldl < 387 || ldd < 387 || !logits || !targets || !dlogits || !loss_sum)
    return SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (B) k_ce_loss<<<grid_n((long long)B * 32, 256), 256, 0, st>>>(
      logits, ldl, targets, B, (__nv_bfloat16 *)dlogits, ldd, ldd, loss_sum);
  return finish(st);
}

extern "C" int sg_gelu_backward(const float *dpost, const float *pre, int64_t n, void *dpre,
                                void *stream) {
  if (n < 0 || (n && (!dpost || !pre || !dpre))) return SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (n) k_gelu_bwd<<<grid_n(n, 256), 256, 0, st>>>(dpost, pre, n, (__nv_bfloat16 *)dpre);
  return finish(st);
}

extern "C" int sg_transpose_bf16(const void *src, int32_t rows, int32_t cols, void *dst,
                                 void *stream) {
  if (rows < 0 || cols < 0 || (rows && cols && (!src || !dst))) return SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (rows && cols)
    k_transpose<<<dim3((cols + 31) / 32, (rows + 31) / 32), dim3(32, 8), 0, st>>>(
        (const __nv_bfloat16 *)src, rows, cols, (__nv_bfloat16 *)dst);
  return finish(st);
}

extern "C" int sg_colsum_bf16(const void *src, int32_t rows, int32_t cols, float *out,
                              void *stream) {
  if (rows < 0 || cols < 0 || (cols && (!src || !out))) return SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cols) k_colsum<<<(cols + 127) / 128, 128, 0, st>>>((const __nv_bfloat16 *)src, rows, cols, out);
  return finish(st);
}

extern "C" int sg_quant_fp8_rows(const float *W, int32_t rows, int32_t cols, void *W8,
                                 float *scale, void *stream) {
  if (rows < 0 || cols < 0 || (rows && (!W || !W8 || !scale))) return SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (rows) k_quant_rows_fp8<<<rows, 256, 0, st>>>(W, rows, cols, (uint8_t *)W8, scale);
  return finish(st);
}

extern "C" int sg_quant_fp8_bf16(const void *x, int64_t n, float inv_scale, void *out8,
                                 void *stream) {
  if (n < 0 || (n && (!x || !out8))) return SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (n) {
    const unsigned g = (unsigned)std::min<long long>(4096, (n + 255) / 256);
    k_quant_bf16_fp8<<<g, 256, 0, st>>>((const __nv_bfloat16 *)x, n, inv_scale, (uint8_t *)out8);
  }
  return finish(st);
}

extern "C" int sg_absmax_bf16(const void *x, int64_t n, float *out, void *stream) {
  if (n < 0 || !out || (n && !x)) return SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemsetAsync(out, 0, sizeof(float), st);
  if (n) {
    const unsigned g = (unsigned)std::min<long long>(4096, (n + 255) / 256);
    k_absmax_bf16<<<g, 256, 0, st>>>((const __nv_bfloat16 *)x, n, out);
  }
  return finish(st);
}

extern "C" int sg_adam_step(float *params, const float *grads, float *m, float *v, int64_t n,
                            float lr, float beta1, float beta2, float eps, int32_t step,
                            void *params_bf16, void *stream) {
  if (n < 0 || step < 1 || (n && (!params || !grads || !m || !v))) return SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  if (n)
    k_adam<<<grid_n(n, 256), 256, 0, st>>>(params, grads, m, v, n, lr, beta1, beta2, eps, c1, c2,
                                           (__nv_bfloat16 *)params_bf16);
  return finish(st);
}

extern "C" int sg_emu_features(const int32_t *u, const double *v, int64_t units,
                               const double *gdata, int32_t max_herd, double phi_lo,
                               double phi_hi, void *feat, int32_t *flag, void *stream) {
  if (units < 0 || !gdata || (units && (!u || !v || !feat || !flag))) return SG_ERR_ARG;
  EmuParams ep{};
  for (int i = 0; i < 11; ++i) ep.gdata[i] = gdata[i];
  ep.max_herd = max_herd;
  ep.phi_lo = phi_lo;
  ep.phi_hi = phi_hi;
  cudaStream_t st = (cudaStream_t)stream;
  if (units)
    k_emu_features<<<grid_n(units, 256), 256, 0, st>>>(u, v, units, ep, (__nv_bfloat16 *)feat,
                                                       flag);
  return finish(st);
}

extern "C" int sg_emu_targets(const int32_t *u_before, const int32_t *u_after, int64_t units,
                              int32_t *targets, void *stream) {
  if (units < 0 || (units && (!u_before || !u_after || !targets))) return SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (units) k_emu_targets<<<grid_n(units, 256), 256, 0, st>>>(u_before, u_after, units, targets);
  return finish(st);
}

extern "C" int sg_emu_sample(const float *logits, int32_t ldl, const int32_t *u,
                             const int32_t *flag, int64_t units, int32_t n_nodes, uint64_t seed,
                             int32_t day, int32_t *delta, void *stream) {
  if (units < 0 || n_nodes < 1 || ldl < 387 || (units && (!logits || !u || !flag || !delta)))
    return SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (units)
    k_emu_sample<<<grid_n(units * 32, 256), 256, 0, st>>>(
        logits, ldl, u, flag, units, n_nodes, (uint32_t)seed, (uint32_t)(seed >> 32), day, delta);
  return finish(st);
}
