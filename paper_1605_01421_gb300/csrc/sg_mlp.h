// sg_mlp.h -- internal interface of the emulator's tensor-core kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "siminf_gpu.h"

namespace sg {

// C = act(A . Bt^T + bias): A is M x K, Bt is N x K (row-major BF16, K
// contiguous); C32 (FP32, before the activation) and / or C16 (BF16, after
// it) are written.  act: 0 identity, 1 GELU.
struct GemmArgs {
  const __nv_bfloat16 *A;
  int lda;
  const __nv_bfloat16 *Bt;
  int ldb;
  int M, N, K;
  const float *bias;
  int act;
  float *C32;
  int ldc32;
  __nv_bfloat16 *C16;
  int ldc16;
  int *err;  // device error word (SG_ERR_TIMEOUT if a wait gave up)
  // FP8 operands (f8 != 0): A8 (M x K) and B8 (N x K) hold E4M3 bytes, K
  // contiguous (K % 16 == 0); the accumulator is multiplied by a_scale *
  // b_scale[n] before the bias.
  int f8;
  const uint8_t *A8, *B8;
  float a_scale;
  const float *b_scale;
  // FP8 output after the activation: C8 = e4m3(act(..) * c8_inv_scale),
  // saturated to the finite range (null: none)
  uint8_t *C8;
  int ldc8;
  float c8_inv_scale;
};

int gemm_bf16(const GemmArgs &g, cudaStream_t st);
int gemm_check(cudaStream_t st);
int gemm_prepare();  // allocates the error word (call before stream capture)

constexpr int kEmuIn = 16, kEmuHidden = 256, kEmuOut = 392;  // 3 x 129 used

// What the emulator's feature kernel needs of an SISe3 model.
struct EmuParams {
  double gdata[11];
  int32_t max_herd;
  double phi_lo, phi_hi;
};

__global__ void k_emu_features(const int32_t *u, const double *v, long long units, EmuParams ep,
                               __nv_bfloat16 *feat, int32_t *flag);
__global__ void k_emu_sample(const float *logits, int ldl, const int32_t *u, const int32_t *flag,
                             long long units, int n_nodes, uint32_t k0, uint32_t k1, int T,
                             int32_t *delta);

}  // namespace sg
