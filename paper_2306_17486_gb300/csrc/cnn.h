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

// Evaluation-mode inverted bottleneck in one kernel (ib_fused.cu):
// y = x + BN2(P softplus(BN1(dw(softplus(BN0(E x)))))), x, y BF16 NHWC [B][H][W][C].
struct IbLaunch {
  const __nv_bfloat16* x = nullptr;
  int B = 0, H = 0, W = 0, C = 0, expansion = 6;
  const __nv_bfloat16* we = nullptr;   // packed 1x1 expansion weights (conv packing, CS = C)
  const __nv_bfloat16* wp = nullptr;   // packed 1x1 projection weights (CS = expansion C)
  const float* wdw = nullptr;          // depthwise weights [expansion C][3][3], FP32
  const float* bn0 = nullptr;          // folded BN (scale | shift) after each stage
  const float* bn1 = nullptr;
  const float* bn2 = nullptr;
  // 16 and 32 channels: the 1x1 weights with BN0 / BN2 folded in (pack_ib_folded)
  const __nv_bfloat16* wef = nullptr;  // [C/8 + 2][6C][8]
  const void* wpf = nullptr;           // [6C/8 + 2][C][8], FP16
  __nv_bfloat16* y = nullptr;
};
int ib_fused(const IbLaunch& l, cudaStream_t st);
int ib_strip(const IbLaunch& l, cudaStream_t st);   // C = 16, 32 (ib_strip.cu)
// 1x1 weights w [Co][Ci] with a folded BatchNorm (fold: scale [Co] then shift [Co]) for
// the strip kernel: [Ci/8 + 2][Co][8] in BF16 (fp16 = 0) or FP16 (fp16 = 1), the last two
// 8-channel groups holding the shift (channel 0 for BF16, 1 for FP16) and zeros; Ci a
// multiple of 16
size_t ib_folded_elems(int Ci, int Co);
int pack_ib_folded(const float* w, const float* fold, int Ci, int Co, int fp16, void* out, cudaStream_t st);
int pack_conv_weights(const float* w, int Ci, int Co, int taps, int transposed, __nv_bfloat16* out, cudaStream_t st);

}  // namespace helm
