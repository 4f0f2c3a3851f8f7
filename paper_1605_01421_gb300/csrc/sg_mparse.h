// sg_mparse.h -- internal interface of the model parser (transition strings
// of Sec. 3.5) and of the run-time compilation of its kernels.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "sg_common.h"

namespace sg {

// A parsed model: S column-major (S[j * C + p] = change of compartment p by
// transition j), G column-major (G[j * T + k] = 1: recompute propensity k
// after transition j), and the CUDA expression of each propensity over
// u (counts), g (global data).
struct ParsedModel {
  int C = 0, T = 0;
  std::vector<int> S, G;
  std::vector<std::string> rate_code;
};

// The engine's kernels compiled for one parsed model.
struct JitKernels {
  enum { kDaysSsm, kDaysAem, kE2, kE2Smem, kRecord0, kCount };
  cudaLibrary_t lib = nullptr;
  cudaKernel_t k[kCount] = {};
  int device = -1;
};

// Returns SG_OK, SG_ERR_ARG or SG_ERR_PARSE (message in err).
int mparse(const char *const *transitions, int n_trans, const char *const *compartments,
           int n_comp, const char *const *gdata_names, int n_gdata, ParsedModel &out,
           std::string &err);
// The CUDA source of ModelTraits<SG_GENERIC> plus the kernel headers.
std::string generic_source(const ParsedModel &pm);
// Compiles with NVRTC for sm_103a and loads on the current device.  Returns
// SG_OK or SG_ERR_JIT (message in err).
int jit_build(const ParsedModel &pm, JitKernels &out, std::string &err);
void jit_release(JitKernels &k);

}  // namespace sg
