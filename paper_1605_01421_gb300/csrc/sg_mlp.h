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
  double min_rate;  // least total transition rate (per day) of an emulated node
};

// The engine's FP8 inference chain (layers 2-4 with E4M3 operands, the
// sampler fused into the output layer); see sg_mlp.cu.
struct EmuChainArgs {
  const uint8_t *A;      // tiled E4M3 input (hidden and output layers)
  const uint8_t *W;      // weight image
  const float *bias;     // per output column
  const float *wscale;   // per output column (E4M3 layers)
  float a_scale;         // dequantisation factor of A (E4M3 layers)
  float inv_out;         // E4M3 output scale (input and hidden layers)
  uint8_t *out;          // tiled E4M3 output (input and hidden layers)
  const int32_t *u;      // node states, units x 6
  const double *v;       // phi per unit (input layer)
  int32_t *flag;         // written by the input layer, read by the output layer
  int32_t *delta;        // (dI_1, dI_2, dI_3, used) per unit (output layer)
  EmuParams ep;          // input layer
  long long units;
  int n_nodes;
  uint32_t k0, k1;
  int T;
  int n_tiles;
  int *err;
};

// Caller-owned weights of the chain (device pointers): W0 BF16 256 x 16,
// W8[l] E4M3 rows x 256 (256, 256, 392) with per-row scales wscale[l],
// biases b[0..3], static activation scales act_scale[0..2].
struct EmuChainWeights {
  const __nv_bfloat16 *W0;
  const uint8_t *W8[3];
  const float *wscale[3];
  const float *b[4];
  float act_scale[3];
};

// Byte offsets of the four weight images in the chain's image buffer, its
// size, and the floats of its head-padded output-layer vectors.
constexpr size_t kEmuImgOff[4] = {0, 8192, 8192 + 65536, 8192 + 2 * 65536};
constexpr size_t kEmuImgBytes = 8192 + 2 * 65536 + 432 * 256;
constexpr size_t kEmuHeadVecFloats = 2 * 432;
constexpr size_t kEmuTileBytes = 128 * 256;  // one tile of tiled E4M3 activations

int emu_chain_images(const EmuChainWeights &cw, uint8_t *img, float *hvec, cudaStream_t st);
// One emulator day in two parts: part 0 computes the features and range
// flags of every unit from the day-start state (the input layer), part 1 the
// other layers and the sampled increments; the SSA of the units outside the
// range may run between them on another stream (it never touches a flagged
// unit, and part 1 reads only flagged units' state).
int emu_chain_day(const EmuChainWeights &cw, const uint8_t *img, const float *hvec,
                  uint8_t *act0, uint8_t *act1, const int32_t *u, const double *v,
                  const EmuParams &ep, long long units, int n_nodes, uint32_t k0, uint32_t k1,
                  int T, int32_t *flag, int32_t *delta, cudaStream_t st, int part);

__global__ void k_emu_features(const int32_t *u, const double *v, long long units, EmuParams ep,
                               __nv_bfloat16 *feat, int32_t *flag);
__global__ void k_emu_sample(const float *logits, int ldl, const int32_t *u, const int32_t *flag,
                             long long units, int n_nodes, uint32_t k0, uint32_t k1, int T,
                             int32_t *delta);

}  // namespace sg
