// Launchers of the CUDA-core network kernels (cnn_kernels.cu, cnn_train.cu).
#pragma once

#include <cuda_bf16.h>

#include "cnn.h"

namespace helm {

int launch_kfeat(const float* kappa, const float* gamma, long n, __nv_bfloat16* out, cudaStream_t st);
// grids are Ny x Nx (rows x columns); the paper's grids are square
int launch_prep(const float2* r, int Ny, int Nx, int B, double* part, float* s, float* inv, __nv_bfloat16* x0,
                cudaStream_t st);
int launch_dw(const __nv_bfloat16* x, int B, int H, int W, int C, const float* w, const float* scale,
              const float* shift, int act, __nv_bfloat16* y, float* yraw, cudaStream_t st);
size_t implicit_smem(int m);
// one CTA per (sample, complex channel) when the m_y x 2m_x intermediate fits shared
// memory; otherwise (or when the tuning table asks) three passes through `scratch`
// (implicit_3pass_bytes; null: the one-CTA form only, HELM_ESHAPE if it does not fit)
int launch_implicit_bf16(const __nv_bfloat16* x, int B, int my, int mx, int C, const float2* ghat,
                         __nv_bfloat16* y, cudaStream_t st, float2* scratch = nullptr);
size_t implicit_3pass_bytes(int B, int my, int mx, int C);
int launch_implicit_adjoint(const float* gy, int B, int m, int C, const float2* ghat, float* gx, cudaStream_t st);
size_t greens_scratch_elems(int my, int mx, int nk);
int launch_greens(const float* Kpar, int nk, int my, int mx, float eps, int literal, float2* scratch, float2* ghat,
                  cudaStream_t st);
int launch_proj(const __nv_bfloat16* u, int B, int Ncy, int Ncx, int C, const float* w, const float* bias, const float* s,
                float2* e, cudaStream_t st);

}  // namespace helm
