// Internal interfaces of the network kernels (tensor-core convolutions, depthwise,
// implicit layer, Green's function, BatchNorm, projection) and the network executor.
#pragma once

#include <cuda_bf16.h>

#include "problem.h"

namespace helm {

// channels per tap staged in shared memory (K of one tap, multiple of 16)
inline int conv_cs(int ci) { return ci <= 16 ? 16 : ((ci + 15) / 16) * 16; }

struct ConvLaunch {
  const __nv_bfloat16* x = nullptr;
  int B = 0, Hi = 0, Wi = 0, Ci = 0, Co = 0, taps = 9, mode = HELM_CONV_S1;
  const __nv_bfloat16* wpk = nullptr;
  const float* scale = nullptr;
  const float* shift = nullptr;
  int act = 0;
  const __nv_bfloat16* add1 = nullptr;
  const __nv_bfloat16* add2 = nullptr;
  int add2_div = 1;   // consecutive samples sharing one add2 entry
  __nv_bfloat16* y = nullptr;
  float* yraw = nullptr;
};

int conv_tc(const ConvLaunch& c, cudaStream_t st);
int pack_conv_weights(const float* w, int Ci, int Co, int taps, int transposed, __nv_bfloat16* out, cudaStream_t st);

}  // namespace helm
