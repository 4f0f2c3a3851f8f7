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

// s GELU(x), given hs = s / 2: h (1 + tanh(u)) with h = hs x and u = x
// (sqrt(2 / pi) + 0.044715 sqrt(2 / pi) x^2), in fused multiply-adds (s
// folds an output scale into the activation).
__device__ __forceinline__ float gelu_scaled(float x, float hs) {
  const float u = x * __fmaf_rn(0.0356774081f, x * x, 0.7978845608f);
  const float h = hs * x;
  return __fmaf_rn(h, tanh_fast(u), h);
}

// 2^x with the hardware approximation (the sampler's softmax weights).
__device__ __forceinline__ float ex2_fast(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr float kLog2e = 1.44269504088896341f;

// 16 E4M3 bytes of y[0..15] (nearest even, saturated), y[0] in the lowest.
__device__ __forceinline__ uint4 pack_e4m3_16(const float *y) {
  uint32_t packed[4];
#pragma unroll
  for (int j = 0; j < 16; j += 4) {
    const __nv_fp8x2_storage_t lo =
        __nv_cvt_float2_to_fp8x2(make_float2(y[j], y[j + 1]), __NV_SATFINITE, __NV_E4M3);
    const __nv_fp8x2_storage_t hi =
        __nv_cvt_float2_to_fp8x2(make_float2(y[j + 2], y[j + 3]), __NV_SATFINITE, __NV_E4M3);
    packed[j / 4] = (uint32_t)lo | ((uint32_t)hi << 16);
  }
  return make_uint4(packed[0], packed[1], packed[2], packed[3]);
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
      // pre-activation: accumulator x a_scale b_scale[n] (E4M3) + bias[n],
      // one fused multiply-add
      float bs[16];
      if (g.bias && nb + 16 <= g.N && (((uintptr_t)(g.bias + nb)) & 15) == 0) {
#pragma unroll
        for (int i = 0; i < 16; i += 4) {
          const float4 b4 = __ldg(reinterpret_cast<const float4 *>(g.bias + nb + i));
          bs[i] = b4.x;
          bs[i + 1] = b4.y;
          bs[i + 2] = b4.z;
          bs[i + 3] = b4.w;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) bs[i] = (g.bias && nb + i < g.N) ? __ldg(g.bias + nb + i) : 0.0f;
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        float cs = 1.0f;
        if constexpr (F8) cs = g.a_scale * ((nb + i < g.N) ? __ldg(g.b_scale + nb + i) : 0.0f);
        v[i] = __fmaf_rn(v[i], cs, bs[i]);
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
      if (g.C16) {
        float y[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) y[i] = g.act == 1 ? gelu_scaled(v[i], 0.5f) : v[i];
        uint32_t packed[8];
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(y[i], y[i + 1]);
          packed[i / 2] = *reinterpret_cast<const uint32_t *>(&h2);
        }
        uint4 *sp = reinterpret_cast<uint4 *>(stage + lr * kPitch + c * 2);
        sp[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        sp[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
      }
      if (g.C8 && row < g.M) {
        // 16 E4M3 values of this row (the output scale folded into the
        // activation), one 16-byte store when it fits
        const float hs = 0.5f * g.c8_inv_scale;
        float y[16];
#pragma unroll
        for (int i = 0; i < 16; ++i)
          y[i] = g.act == 1 ? gelu_scaled(v[i], hs) : v[i] * g.c8_inv_scale;
        const uint4 pk = pack_e4m3_16(y);
        const uint32_t packed[4] = {pk.x, pk.y, pk.z, pk.w};
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

// Input features of one SISe3 node for the emulator (the BF16 values of the
// 16 inputs), and whether the node is in the emulator's range (herd <=
// max_herd, phi_lo <= phi <= phi_hi, total transition rate >= min_rate).
__device__ __forceinline__ bool emu_feature_row(const int32_t *un, double phi,
                                                const EmuParams &ep, __nv_bfloat16 *row) {
  int herd = 0;
#pragma unroll
  for (int p = 0; p < 6; ++p) herd += un[p];
  // total transition rate: S_a -> I_a at upsilon_a phi S_a, I_a -> S_a at
  // gamma_a I_a
  double a0 = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    a0 += ep.gdata[a] * phi * (double)un[2 * a] + ep.gdata[3 + a] * (double)un[2 * a + 1];
  const bool in = herd <= ep.max_herd && phi >= ep.phi_lo && phi <= ep.phi_hi &&
                  a0 >= ep.min_rate;
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
#pragma unroll
  for (int k = 0; k < 16; ++k) row[k] = __float2bfloat16_rn(f[k]);
  return in;
}

__global__ void k_emu_features(const int32_t *__restrict__ u, const double *__restrict__ v,
                               long long units, EmuParams ep, __nv_bfloat16 *feat,
                               int32_t *flag) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < units;
       i += (long long)gridDim.x * blockDim.x)
    flag[i] = emu_feature_row(u + i * 6, v[i], ep, feat + i * 16) ? 1 : 0;
}

// Sample each in-range node's increments from the emulator's three heads:
// softmax over the 129 bins (weights 2^(z - max z) with z = logit log2 e, the
// hardware 2^x), inverse CDF at a uniform from the emulator's
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
      vals[j] = c < kBins ? lg[c] * kLog2e : -INFINITY;
      mx = fmaxf(mx, vals[j]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float part = 0.0f;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      vals[j] = lane * 5 + j < kBins ? ex2_fast(vals[j] - mx) : 0.0f;
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

// ---------------------------------------------------------------------------
// The engine's FP8 inference chain: one persistent kernel per layer (one CTA
// per SM), the layer's weights resident in shared memory, activations in a
// tiled layout that one bulk copy moves, and (hidden layers) two tensor-memory
// accumulators, so that the epilogue of one 128-row tile overlaps the MMAs of
// the next.  Warp roles: producer warps (bulk copies, or the input features
// computed in place), one MMA warp (one elected thread issues tcgen05.mma),
// epilogue warps (tcgen05.ld, scale, bias, activation, store).
//
// Tiled layout of a matrix with rows padded to a multiple of 128 and Kb bytes
// per row: tile t (rows 128 t .. 128 t + 127) occupies bytes [128 Kb t,
// 128 Kb (t + 1)), as Kb / 16 chunks of 128 rows x 16 bytes (chunk c at
// 2048 c, row r of it at 16 r).  Copied to shared memory this is the
// no-swizzle K-major operand layout with 8-row core matrices 128 bytes apart
// along M and 2048 bytes apart along K.  A weight image uses the same layout
// with all of its N rows in one tile (chunk c at 16 N c).
//
// Layer kinds: 0, the input layer: features computed from the node states in
// the kernel (BF16, K = 16), 256 outputs, GELU, E4M3 out; 1, a hidden layer:
// E4M3 in (K = 256), 256 outputs, GELU, E4M3 out; 2, the output layer fused
// with the sampler: E4M3 in, head h's 129 logits at accumulator columns
// 144 h .. 144 h + 128, sampled as k_emu_sample samples them, bit for bit.
// Every layer's arithmetic is that of k_gemm_tc on the same operands.
// ---------------------------------------------------------------------------
constexpr int kEmuHeadPitch = 144;               // accumulator columns per head
constexpr int kEmuHeadCols = 3 * kEmuHeadPitch;  // 432 (MMAs of N = 256 and 176)
constexpr uint32_t kEmuTmemCols = 512;
constexpr uint32_t kEmuMinSmem = 120u * 1024u;   // one CTA per SM (its TMEM is 512 columns)

template <int L>
struct EmuLayerCfg;
template <>
struct EmuLayerCfg<0> {
  static constexpr bool kF8 = false;
  static constexpr int kKb = 32, kN = 256, kStages = 4, kAcc = 2, kProdWarps = 4,
                       kEpiWarps = 16;
};
template <>
struct EmuLayerCfg<1> {
  static constexpr bool kF8 = true;
  static constexpr int kKb = 256, kN = 256, kStages = 2, kAcc = 2, kProdWarps = 1,
                       kEpiWarps = 16;
};
template <>
struct EmuLayerCfg<2> {
  static constexpr bool kF8 = true;
  static constexpr int kKb = 256, kN = kEmuHeadCols, kStages = 2, kAcc = 1, kProdWarps = 1,
                       kEpiWarps = 12;
};

template <int L>
constexpr int emu_layer_threads() {
  return (EmuLayerCfg<L>::kProdWarps + 1 + EmuLayerCfg<L>::kEpiWarps) * 32;
}

// weight image, A stages, per-column accumulator factor and bias
template <int L>
constexpr uint32_t emu_layer_smem() {
  using C = EmuLayerCfg<L>;
  return (uint32_t)C::kN * C::kKb + (uint32_t)C::kStages * 128u * C::kKb + 8u * C::kN;
}

__device__ __forceinline__ void emu_fail(volatile int *s_fail, int *err) {
  *s_fail = 1;
  atomicExch(err, SG_ERR_TIMEOUT);
}

template <int L>
__global__ void __launch_bounds__(emu_layer_threads<L>(), 1) k_emu_layer(const EmuChainArgs a) {
  using C = EmuLayerCfg<L>;
  constexpr uint32_t kATile = 128u * C::kKb;
  constexpr uint32_t kWBytes = (uint32_t)C::kN * C::kKb;
  constexpr int kKSteps = C::kKb / 32;  // 32 bytes of K per MMA
  constexpr int kMmaWarp = C::kProdWarps, kEpi0 = C::kProdWarps + 1;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *sW = smem;
  unsigned char *sA = smem + kWBytes;
  float *sScale = reinterpret_cast<float *>(sA + C::kStages * kATile);
  float *sBias = sScale + C::kN;
  __shared__ __align__(8) uint64_t bar_w, bar_full[C::kStages], bar_empty[C::kStages],
      bar_tfull[C::kAcc], bar_tempty[C::kAcc];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar_w, 1);
    for (int s = 0; s < C::kStages; ++s) {
      tc::mbar_init(&bar_full[s], L == 0 ? 128 : 1);
      tc::mbar_init(&bar_empty[s], 1);
    }
    for (int b = 0; b < C::kAcc; ++b) {
      tc::mbar_init(&bar_tfull[b], 1);
      tc::mbar_init(&bar_tempty[b], C::kEpiWarps);
    }
    tc::fence_mbar_init();
    s_fail = 0;
  }
  // the accumulator's factor a_scale * w_scale[n] (E4M3 layers), the bias
  for (int n = threadIdx.x; n < C::kN; n += blockDim.x) {
    sScale[n] = C::kF8 ? a.a_scale * a.wscale[n] : 1.0f;
    sBias[n] = a.bias[n];
  }
  if (warp == kMmaWarp) tc::tmem_alloc(&tmem_slot, kEmuTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const int my_tiles = (a.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1;

  if (warp < C::kProdWarps) {
    // ---- producer ----
    if (threadIdx.x == 0) {
      tc::mbar_arrive_expect_tx(&bar_w, kWBytes);
      for (uint32_t off = 0; off < kWBytes; off += 16384u)
        tc::bulk_g2s(sW + off, a.W + off, kWBytes - off < 16384u ? kWBytes - off : 16384u, &bar_w);
    }
    if constexpr (L == 0) {
      // four warps, thread p writes row p of each tile: its 16 BF16
      // features as two 16-byte pieces (chunks 0 and 1)
      const int p = threadIdx.x;
      for (int i = 0; i < my_tiles; ++i) {
        const int s = i % C::kStages, k = i / C::kStages;
        if (k > 0 && !tc::mbar_wait(&bar_empty[s], (k - 1) & 1, kWaitLimit)) {
          emu_fail(&s_fail, a.err);
          break;
        }
        if (s_fail) break;
        const long long w = ((long long)blockIdx.x + (long long)i * gridDim.x) * 128 + p;
        __align__(16) __nv_bfloat16 row[16];
        if (w < a.units) {
          a.flag[w] = emu_feature_row(a.u + w * 6, a.v[w], a.ep, row) ? 1 : 0;
        } else {
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) row[k2] = __float2bfloat16_rn(0.0f);
        }
        const uint4 *r4 = reinterpret_cast<const uint4 *>(row);
        unsigned char *stage = sA + s * kATile;
        *reinterpret_cast<uint4 *>(stage + p * 16) = r4[0];
        *reinterpret_cast<uint4 *>(stage + 2048 + p * 16) = r4[1];
        tc::fence_async_smem();
        tc::mbar_arrive(&bar_full[s]);
      }
      if (threadIdx.x == 0) tc::mbar_wait(&bar_w, 0, kWaitLimit);
    } else {
      if (lane == 0) {
        int last[C::kStages];
#pragma unroll
        for (int s = 0; s < C::kStages; ++s) last[s] = -1;
        for (int i = 0; i < my_tiles; ++i) {
          const int s = i % C::kStages, k = i / C::kStages;
          if (k > 0 && !tc::mbar_wait(&bar_empty[s], (k - 1) & 1, kWaitLimit)) {
            emu_fail(&s_fail, a.err);
            break;
          }
          if (s_fail) break;
          const long long t = (long long)blockIdx.x + (long long)i * gridDim.x;
          tc::mbar_arrive_expect_tx(&bar_full[s], kATile);
          tc::bulk_g2s(sA + s * kATile, a.A + t * kATile, kATile, &bar_full[s]);
          last[s] = k;
        }
        // no copy of ours may still be landing in shared memory at exit
        tc::mbar_wait(&bar_w, 0, kWaitLimit);
#pragma unroll
        for (int s = 0; s < C::kStages; ++s)
          if (last[s] >= 0) tc::mbar_wait(&bar_full[s], last[s] & 1, kWaitLimit);
      }
      __syncwarp();
    }
  } else if (warp == kMmaWarp) {
    // ---- MMA issue ----
    if (lane == 0) {
      int last_b = -1, last_kb = 0;
      bool ok = tc::mbar_wait(&bar_w, 0, kWaitLimit);
      const uint32_t a0 = tc::smem_u32(sA), w0 = tc::smem_u32(sW);
      for (int i = 0; ok && i < my_tiles; ++i) {
        const int s = i % C::kStages, k = i / C::kStages;
        const int b = i % C::kAcc, kb = i / C::kAcc;
        if (!tc::mbar_wait(&bar_full[s], k & 1, kWaitLimit) ||
            (kb > 0 && !tc::mbar_wait(&bar_tempty[b], (kb - 1) & 1, kWaitLimit))) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * 256);
        const uint32_t as = a0 + (uint32_t)s * kATile;
#pragma unroll
        for (int ks = 0; ks < kKSteps; ++ks) {
          const uint64_t ad = tc::smem_desc(as + ks * 4096, 2048, 128);
          const uint64_t bd = tc::smem_desc(w0 + ks * 32 * C::kN, 16 * C::kN, 128);
          if constexpr (L == 0) {
            tc::mma_bf16(d, ad, bd, tc::idesc_bf16_f32(128, 256), ks > 0 ? 1u : 0u);
          } else {
            tc::mma_e4m3(d, ad, bd, tc::idesc_e4m3_f32(128, 256), ks > 0 ? 1u : 0u);
            if constexpr (L == 2) {
              const uint64_t bd2 = tc::smem_desc(w0 + 256 * 16 + ks * 32 * C::kN, 16 * C::kN, 128);
              tc::mma_e4m3(d + 256, ad, bd2, tc::idesc_e4m3_f32(128, C::kN - 256),
                           ks > 0 ? 1u : 0u);
            }
          }
        }
        tc::mma_commit(&bar_empty[s]);
        tc::mma_commit(&bar_tfull[b]);
        last_b = b;
        last_kb = kb;
      }
      if (!ok) emu_fail(&s_fail, a.err);
      // the tensor memory is freed only after our MMAs are done
      if (last_b >= 0) tc::mbar_wait(&bar_tfull[last_b], last_kb & 1, kWaitLimit);
    }
    __syncwarp();
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 ----
    const int ew = warp - kEpi0;
    const int q = warp & 3;
    const int r = q * 32 + lane;  // tile row of this thread
    if constexpr (L < 2) {
      const int c0 = (ew >> 2) * 64;  // column quarter
      const float hs = 0.5f * a.inv_out;
      for (int i = 0; i < my_tiles; ++i) {
        const int b = i % C::kAcc, kb = i / C::kAcc;
        if (!tc::mbar_wait(&bar_tfull[b], kb & 1, kWaitLimit)) {
          emu_fail(&s_fail, a.err);
          break;
        }
        tc::tc_fence_after();
        const long long t = (long long)blockIdx.x + (long long)i * gridDim.x;
        const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 256);
        unsigned char *orow = a.out + t * (128 * 256) + r * 16;
        tc::tmem_stream16<4>(tb + (uint32_t)c0, [&](int k, float *v) {
          const int c = c0 + 16 * k;
          const float4 *s4 = reinterpret_cast<const float4 *>(sScale + c);
          const float4 *b4 = reinterpret_cast<const float4 *>(sBias + c);
#pragma unroll
          for (int j4 = 0; j4 < 4; ++j4) {
            const float4 sc = s4[j4], bi = b4[j4];
            float *x = v + 4 * j4;
            x[0] = __fmaf_rn(x[0], sc.x, bi.x);
            x[1] = __fmaf_rn(x[1], sc.y, bi.y);
            x[2] = __fmaf_rn(x[2], sc.z, bi.z);
            x[3] = __fmaf_rn(x[3], sc.w, bi.w);
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = gelu_scaled(v[j], hs);
          *reinterpret_cast<uint4 *>(orow + (c / 16) * 2048) = pack_e4m3_16(v);
        });
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bar_tempty[b]);
      }
    } else {
      const int h = ew >> 2;  // head (age class) of this warp
      const int col0 = h * kEmuHeadPitch;
      for (int i = 0; i < my_tiles; ++i) {
        if (!tc::mbar_wait(&bar_tfull[0], i & 1, kWaitLimit)) {
          emu_fail(&s_fail, a.err);
          break;
        }
        tc::tc_fence_after();
        const long long w = ((long long)blockIdx.x + (long long)i * gridDim.x) * 128 + r;
        const bool live = w < a.units;
        const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col0;
        // pass 1: the logits (accumulator x a_scale w_scale + bias) times
        // log2 e, written back to the tensor memory, and their maximum
        float mx = -INFINITY;
        tc::tmem_stream16<kEmuHeadPitch / 16>(tb, [&](int k, float *x) {
          const int c = 16 * k;
          const float4 *s4 = reinterpret_cast<const float4 *>(sScale + col0 + c);
          const float4 *b4 = reinterpret_cast<const float4 *>(sBias + col0 + c);
#pragma unroll
          for (int j4 = 0; j4 < 4; ++j4) {
            const float4 sc = s4[j4], bi = b4[j4];
            float *y = x + 4 * j4;
            y[0] = __fmaf_rn(y[0], sc.x, bi.x) * kLog2e;
            y[1] = __fmaf_rn(y[1], sc.y, bi.y) * kLog2e;
            y[2] = __fmaf_rn(y[2], sc.z, bi.z) * kLog2e;
            y[3] = __fmaf_rn(y[3], sc.w, bi.w) * kLog2e;
          }
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c + j < kBins) mx = fmaxf(mx, x[j]);
          tc::tmem_st16(tb + (uint32_t)c, x);
        });
        tc::tmem_wait_st();
        // pass 2: the 32 partial sums of 5 bins' softmax weights 2^(z - max z)
        float p[32];
#pragma unroll
        for (int l = 0; l < 32; ++l) p[l] = 0.0f;
        tc::tmem_stream16<kEmuHeadPitch / 16>(tb, [&](int k, float *x) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (16 * k + j < kBins) p[(16 * k + j) / 5] += ex2_fast(x[j] - mx);
        });
        // inclusive scan of the partial sums in the order of the warp's
        // shuffle scan in k_emu_sample (steps 1, 2, 4, 8, 16)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1)
#pragma unroll
          for (int l = 31; l >= o; --l) p[l] += p[l - o];
        const float total = p[31];
        const long long rep = live ? w / a.n_nodes : 0;
        const long long node = live ? w - rep * a.n_nodes : 0;
        const U4 x4 = philox10(
            U4{0u, (uint32_t)node, (uint32_t)a.T, (SG_STREAM_EMU << 24) | (uint32_t)rep}, a.k0,
            a.k1);
        const uint32_t word = h == 0 ? x4.x : (h == 1 ? x4.y : x4.z);
        const float target = ((float)(word >> 8) + 0.5f) * (1.0f / 16777216.0f) * total;
        // the first partial range that reaches the target, then the bin in it
        int owner = 31;
        float incl_o = p[31];
#pragma unroll
        for (int l = 30; l >= 0; --l)
          if (p[l] >= target) {
            owner = l;
            incl_o = p[l];
          }
        // pass 3: the five values of that range, then their weights
        float xo[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        tc::tmem_stream16<kEmuHeadPitch / 16>(tb, [&](int k, float *x) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (16 * k + j < kBins && (16 * k + j) / 5 == owner) xo[(16 * k + j) % 5] = x[j];
        });
        // the range's own partial sum, added in the same order as in pass 2
        float e[5], part_o = 0.0f;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          e[j] = owner * 5 + j < kBins ? ex2_fast(xo[j] - mx) : 0.0f;
          part_o += e[j];
        }
        float acc = incl_o - part_o;
        int bin = min(owner * 5 + 4, kBins - 1);
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          acc += e[j];
          if (acc >= target && owner * 5 + j < kBins) {
            bin = owner * 5 + j;
            break;
          }
        }
        if (live) {
          int32_t *o = a.delta + w * 4;
          if (a.flag[w]) {
            const int S = a.u[w * 6 + 2 * h], I = a.u[w * 6 + 2 * h + 1];
            int d = bin - kHalf;
            d = max(d, -I);
            d = min(d, S);
            o[h] = d;
            if (h == 0) o[3] = 1;
          } else if (h == 0) {
            o[3] = 0;
          }
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bar_tempty[0]);
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) tc::tmem_dealloc(tmem, kEmuTmemCols);
}

// Weight image of the chain: row n of the image is row n of W (src_rows x
// Kb bytes, row-major), or with head_pad row 129 h + j for image row 144 h + j
// (j < 129); other image rows are zero.
__global__ void k_emu_image(const uint8_t *__restrict__ W, int src_rows, int Kb, int n_img,
                            int head_pad, uint8_t *img) {
  const int chunks = Kb / 16;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n_img * chunks;
       idx += gridDim.x * blockDim.x) {
    const int c = idx / n_img, n = idx - c * n_img;
    int src = n;
    if (head_pad) {
      const int h = n / kEmuHeadPitch, j = n - h * kEmuHeadPitch;
      src = j < kBins ? h * kBins + j : -1;
    }
    uint4 val = make_uint4(0u, 0u, 0u, 0u);
    if (src >= 0 && src < src_rows)
      val = *reinterpret_cast<const uint4 *>(W + (size_t)src * Kb + c * 16);
    *reinterpret_cast<uint4 *>(img + (size_t)idx * 16) = val;
  }
}

// Bias and weight scales of the output layer in the head-padded order.
__global__ void k_emu_head_vec(const float *__restrict__ b, const float *__restrict__ ws,
                               float *bimg, float *wimg) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < kEmuHeadCols;
       n += gridDim.x * blockDim.x) {
    const int h = n / kEmuHeadPitch, j = n - h * kEmuHeadPitch;
    const bool in = j < kBins;
    bimg[n] = in ? b[h * kBins + j] : 0.0f;
    wimg[n] = in ? ws[h * kBins + j] : 0.0f;
  }
}

template <int L>
static void launch_emu_layer(const EmuChainArgs &a, int grid, cudaStream_t st) {
  const uint32_t smem = std::max(emu_layer_smem<L>(), kEmuMinSmem);
  static bool attr_set = false;  // guarded by the caller's lock
  if (!attr_set) {
    cudaFuncSetAttribute(k_emu_layer<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  k_emu_layer<L><<<grid, emu_layer_threads<L>(), smem, st>>>(a);
}

int emu_chain_images(const EmuChainWeights &cw, uint8_t *img, float *hvec, cudaStream_t st) {
  k_emu_image<<<16, 256, 0, st>>>(reinterpret_cast<const uint8_t *>(cw.W0), kEmuHidden, 32,
                                  kEmuHidden, 0, img + kEmuImgOff[0]);
  k_emu_image<<<64, 256, 0, st>>>(cw.W8[0], kEmuHidden, 256, kEmuHidden, 0, img + kEmuImgOff[1]);
  k_emu_image<<<64, 256, 0, st>>>(cw.W8[1], kEmuHidden, 256, kEmuHidden, 0, img + kEmuImgOff[2]);
  k_emu_image<<<64, 256, 0, st>>>(cw.W8[2], kEmuOut, 256, kEmuHeadCols, 1, img + kEmuImgOff[3]);
  k_emu_head_vec<<<2, 256, 0, st>>>(cw.b[3], cw.wscale[2], hvec, hvec + kEmuHeadCols);
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

int emu_chain_day(const EmuChainWeights &cw, const uint8_t *img, const float *hvec,
                  uint8_t *act0, uint8_t *act1, const int32_t *u, const double *v,
                  const EmuParams &ep, long long units, int n_nodes, uint32_t k0, uint32_t k1,
                  int T, int32_t *flag, int32_t *delta, cudaStream_t st, int part) {
  if (units <= 0) return SG_OK;
  static std::mutex mu;
  static int n_sm = 0;
  std::lock_guard<std::mutex> lock(mu);
  if (!n_sm) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n_sm <= 0) {
      cudaGetLastError();
      n_sm = 0;
      return SG_ERR_CUDA;
    }
  }
  int *err = nullptr;
  int rc = gemm_err_buf(&err);
  if (rc) return rc;
  const long long tiles = (units + 127) / 128;
  if (tiles > (1ll << 30)) return SG_ERR_ARG;
  const int grid = (int)std::min<long long>(tiles, n_sm);
  EmuChainArgs a{};
  a.u = u;
  a.v = v;
  a.flag = flag;
  a.delta = delta;
  a.ep = ep;
  a.units = units;
  a.n_nodes = n_nodes;
  a.k0 = k0;
  a.k1 = k1;
  a.T = T;
  a.n_tiles = (int)tiles;
  a.err = err;
  if (part == 0) {
    // layer 1: features -> E4M3 activations (act0), range flags
    a.W = img + kEmuImgOff[0];
    a.bias = cw.b[0];
    a.inv_out = 1.0f / cw.act_scale[0];
    a.out = act0;
    launch_emu_layer<0>(a, grid, st);
    return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
  }
  // layers 2 and 3: act0 -> act1 -> act0
  for (int l = 1; l <= 2; ++l) {
    a.A = l == 1 ? act0 : act1;
    a.out = l == 1 ? act1 : act0;
    a.W = img + kEmuImgOff[l];
    a.bias = cw.b[l];
    a.wscale = cw.wscale[l - 1];
    a.a_scale = cw.act_scale[l - 1];
    a.inv_out = 1.0f / cw.act_scale[l];
    launch_emu_layer<1>(a, grid, st);
  }
  // layer 4 and sampling: act0 -> delta
  a.A = act0;
  a.out = nullptr;
  a.W = img + kEmuImgOff[3];
  a.bias = hvec;
  a.wscale = hvec + kEmuHeadCols;
  a.a_scale = cw.act_scale[2];
  launch_emu_layer<2>(a, grid, st);
  return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
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
                               double phi_hi, double min_rate, void *feat, int32_t *flag,
                               void *stream) {
  if (units < 0 || !gdata || (units && (!u || !v || !feat || !flag))) return SG_ERR_ARG;
  EmuParams ep{};
  for (int i = 0; i < 11; ++i) ep.gdata[i] = gdata[i];
  ep.max_herd = max_herd;
  ep.phi_lo = phi_lo;
  ep.phi_hi = phi_hi;
  ep.min_rate = min_rate;
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
