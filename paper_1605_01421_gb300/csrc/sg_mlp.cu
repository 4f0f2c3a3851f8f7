// sg_mlp.cu -- the dense contractions of the learned one-day emulator on the
// fifth-generation tensor cores (tcgen05, accumulators in tensor memory), and
// the small element-wise kernels around them (loss, optimiser, features,
// sampling).  The emulator is an extension of the method, not part of the
// paper.
#include <cuda_bf16.h>
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

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}

// C = act(A . Bt^T + bias) for one 128 x BN tile.  A: M x K, Bt: N x K, both
// row-major BF16 with K contiguous (K % 8 == 0, rows 16-byte aligned).
// 128 threads: all load the double-buffered K stages into shared memory,
// thread 0 issues the MMAs (4 per stage, K = 16 each) and commits them to the
// stage's mbarrier; the 4 warps then read the FP32 accumulator rows of their
// TMEM lanes for the epilogue.
template <int BN>
__global__ void __launch_bounds__(128) k_gemm_tc(const GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr uint32_t kAStage = kBM * kBK * 2;  // 16 KB
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
  constexpr uint32_t idesc = tc::idesc_bf16_f32(kBM, BN);
  const int stages = (g.K + kBK - 1) / kBK;
  uint32_t uses[2] = {0, 0};
  bool ok = true;

  for (int s = 0; s < stages && ok; ++s) {
    const int b = s & 1;
    if (s >= 2) {  // buffer b is free once the MMAs of stage s - 2 are done
      if (!tc::mbar_wait(&bar[b], (uses[b] - 1) & 1, kWaitLimit)) s_fail = 1;
    }
    __syncthreads();
    if (s_fail) {
      ok = false;
      break;
    }
    const int k0 = s * kBK;
    // A stage: 128 rows x 64
    for (int idx = tid; idx < kBM * 8; idx += 128) {
      const int r = idx >> 3, kg = idx & 7;
      const int m = m0 + r, k = k0 + kg * 8;
      int4 val = make_int4(0, 0, 0, 0);
      if (m < g.M && k < g.K)
        val = *reinterpret_cast<const int4 *>(g.A + (long long)m * g.lda + k);
      *reinterpret_cast<int4 *>(sA[b] + stage_off(r, kg)) = val;
    }
    // B stage: BN rows x 64
    for (int idx = tid; idx < BN * 8; idx += 128) {
      const int r = idx >> 3, kg = idx & 7;
      const int n = n0 + r, k = k0 + kg * 8;
      int4 val = make_int4(0, 0, 0, 0);
      if (n < g.N && k < g.K)
        val = *reinterpret_cast<const int4 *>(g.Bt + (long long)n * g.ldb + k);
      *reinterpret_cast<int4 *>(sB[b] + stage_off(r, kg)) = val;
    }
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
        tc::mma_bf16(tmem, ad, bd, idesc, (s > 0 || kk > 0) ? 1u : 0u);
      }
      tc::mma_commit(&bar[b]);
    }
    ++uses[b];
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
    tc::tc_fence_after();
    const int row = m0 + warp * 32 + lane;
    for (int c = 0; c < BN; c += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
      if (row < g.M) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int n = n0 + c + i;
          if (n >= g.N) break;
          float x = v[i] + (g.bias ? g.bias[n] : 0.0f);
          if (g.C32) g.C32[(long long)row * g.ldc32 + n] = x;
          if (g.act == 1) x = gelu(x);
          if (g.C16) g.C16[(long long)row * g.ldc16 + n] = __float2bfloat16_rn(x);
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

template <int BN>
void launch_gemm(const GemmArgs &g, cudaStream_t st) {
  const size_t smem = 2 * ((size_t)kBM * kBK * 2 + (size_t)BN * kBK * 2);
  static unsigned long long attr_set = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !((attr_set >> dev) & 1ull)) {
    cudaFuncSetAttribute(k_gemm_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set |= 1ull << dev;
  }
  const dim3 grid((unsigned)((g.M + kBM - 1) / kBM), (unsigned)((g.N + BN - 1) / BN));
  k_gemm_tc<BN><<<grid, 128, smem, st>>>(g);
}

}  // namespace

namespace sg {

int gemm_bf16(const GemmArgs &g0, cudaStream_t st) {
  GemmArgs g = g0;
  if (g.M < 0 || g.N < 0 || g.K < 0 || (g.K % 8) != 0 || g.lda < g.K || g.ldb < g.K ||
      (g.lda % 8) != 0 || (g.ldb % 8) != 0 || !g.A || !g.Bt || (!g.C32 && !g.C16) ||
      (((uintptr_t)g.A | (uintptr_t)g.Bt) & 15) != 0)
    return SG_ERR_ARG;
  if (g.M == 0 || g.N == 0) return SG_OK;
  if (!g.err) {
    int rc = gemm_err_buf(&g.err);
    if (rc) return rc;
  }
  if (g.N <= 64)
    launch_gemm<64>(g, st);
  else if (g.N <= 128)
    launch_gemm<128>(g, st);
  else
    launch_gemm<256>(g, st);
  return SG_OK;
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
