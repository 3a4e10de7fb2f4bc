// Training of the encoder-solver network (Section 4.3, Eq. 16; Section 5.3):
// forward with batch-statistics BatchNorm (convolutions on the tensor cores write
// their raw FP32 accumulators, BN statistics and the normalise/softplus/skip epilogue
// follow), and the hand-written backward pass:
//   BN + softplus + additive skips, 3x3 / 1x1 convolutions in every mode (input and
//   weight gradients), depthwise 3x3, the implicit layer (adjoint = the same layer with
//   conj(G_hat); kernel gradient through G_hat -> crop -> G -> H(K_hat) -> K, the
//   Wirtinger chain of Eq. 15), and the final projection + bilinear P.
// Also the MSE loss (Eq. 16) and the Adam update.
// All backward arithmetic is FP32 on CUDA cores, with deterministic two-stage
// reductions for every parameter gradient.
#include <cmath>

#include "cnn_impl.h"

namespace helm {

using bf16 = __nv_bfloat16;

namespace {

constexpr float BN_EPS = 1e-5f;
constexpr float BN_MOM = 0.1f;

__device__ __forceinline__ float sigmoidf(float x) { return 1.f / (1.f + __expf(-x)); }
__device__ __forceinline__ float spf(float x) { return fmaxf(x, 0.f) + log1pf(__expf(-fabsf(x))); }

int gridn(long n, int t = 256) { return static_cast<int>(std::min<long>(div_up(n, t), 8192)); }

// ---- BatchNorm statistics: per-channel sum / sum of squares -------------------------
// pixels per reduction block: enough blocks to fill the GPU, at most kMaxChunks
inline long bn_chunk(long P) { return std::max<long>(32, (P + 1023) / 1024); }

// block (C, k): thread (c, j) sums pixels j, j+k, ... of the chunk for channel c
// (coalesced, no atomics, deterministic); the k partials are combined in shared memory
__global__ void k_chan_sums(const float* __restrict__ z, long P, int C, long chunk, double* __restrict__ part) {
  extern __shared__ double dsum[];  // [2][k][C]
  const int c = threadIdx.x, j = threadIdx.y, k = blockDim.y;
  const long p0 = static_cast<long>(blockIdx.x) * chunk, p1 = min(p0 + chunk, P);
  float s1 = 0.f, s2 = 0.f;
  for (long p = p0 + j; p < p1; p += k) {
    const float v = z[p * C + c];
    s1 += v;
    s2 = fmaf(v, v, s2);
  }
  dsum[j * C + c] = s1;
  dsum[(k + j) * C + c] = s2;
  __syncthreads();
  if (j == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < k; ++q) {
      a += dsum[q * C + c];
      b += dsum[(k + q) * C + c];
    }
    part[static_cast<long>(blockIdx.x) * 2 * C + c] = a;
    part[static_cast<long>(blockIdx.x) * 2 * C + C + c] = b;
  }
}

inline dim3 chan_block(int C) { return dim3(C, std::max(1, 256 / C)); }
inline size_t chan_smem(int C) { return 2 * sizeof(double) * C * std::max(1, 256 / C); }

// mean, 1/sqrt(var + eps) (biased var); running stats: momentum 0.1, unbiased var
__global__ void k_bn_finalize(const double* __restrict__ part, int nblk, int C, long P, float* __restrict__ mean,
                              float* __restrict__ istd, float* __restrict__ running_mean,
                              float* __restrict__ running_var) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
    double s = 0, q = 0;
    for (int i = 0; i < nblk; ++i) {
      s += part[static_cast<long>(i) * 2 * C + c];
      q += part[static_cast<long>(i) * 2 * C + C + c];
    }
    const double mu = s / P;
    const double var = fmax(q / P - mu * mu, 0.0);
    mean[c] = static_cast<float>(mu);
    istd[c] = static_cast<float>(1.0 / sqrt(var + BN_EPS));
    if (running_mean) {
      running_mean[c] = (1.f - BN_MOM) * running_mean[c] + BN_MOM * static_cast<float>(mu);
      running_var[c] = (1.f - BN_MOM) * running_var[c] + BN_MOM * static_cast<float>(var * P / fmax(P - 1.0, 1.0));
    }
  }
}

// y = act(g (z - mu) istd + b) + add1 + add2 -> bf16; add2 has one entry per group of
// `div` consecutive samples (sample_elems elements per sample)
__global__ void k_bn_apply(const float* __restrict__ z, long P, int C, const float* __restrict__ mean,
                           const float* __restrict__ istd, const float* __restrict__ g, const float* __restrict__ b,
                           int act, const bf16* __restrict__ add1, const bf16* __restrict__ add2, long sample_elems,
                           int div, bf16* __restrict__ y) {
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < P * C;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(i % C);
    float v = g[c] * (z[i] - mean[c]) * istd[c] + b[c];
    if (act) v = spf(v);
    if (add1) v += __bfloat162float(add1[i]);
    if (add2) {
      const long smp = i / sample_elems;
      v += __bfloat162float(add2[(smp / div) * sample_elems + (i - smp * sample_elems)]);
    }
    y[i] = __float2bfloat16_rn(v);
  }
}

// ---- BN + activation backward ---------------------------------------------------------
// dA = dY * act'(a), a = g zhat + b; per-channel sums S1 = sum dA, S2 = sum dA zhat
__global__ void k_bn_bwd_sums(const float* __restrict__ dY, const float* __restrict__ z, long P, int C,
                              const float* __restrict__ mean, const float* __restrict__ istd,
                              const float* __restrict__ g, const float* __restrict__ b, int act, long chunk,
                              double* __restrict__ part) {
  extern __shared__ double dsum[];  // [2][k][C]
  const int c = threadIdx.x, j = threadIdx.y, k = blockDim.y;
  const long p0 = static_cast<long>(blockIdx.x) * chunk, p1 = min(p0 + chunk, P);
  const float mu = mean[c], is = istd[c], gc = g[c], bc = b[c];
  float s1 = 0.f, s2 = 0.f;
  for (long p = p0 + j; p < p1; p += k) {
    const long i = p * C + c;
    const float zh = (z[i] - mu) * is;
    float dA = dY[i];
    if (act) dA *= sigmoidf(gc * zh + bc);
    s1 += dA;
    s2 = fmaf(dA, zh, s2);
  }
  dsum[j * C + c] = s1;
  dsum[(k + j) * C + c] = s2;
  __syncthreads();
  if (j == 0) {
    double a = 0.0, bb = 0.0;
    for (int q = 0; q < k; ++q) {
      a += dsum[q * C + c];
      bb += dsum[(k + q) * C + c];
    }
    part[static_cast<long>(blockIdx.x) * 2 * C + c] = a;
    part[static_cast<long>(blockIdx.x) * 2 * C + C + c] = bb;
  }
}

__global__ void k_bn_bwd_final(const double* __restrict__ part, int nblk, int C, float* __restrict__ S,
                               float* __restrict__ dg, float* __restrict__ db) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
    double s1 = 0, s2 = 0;
    for (int i = 0; i < nblk; ++i) {
      s1 += part[static_cast<long>(i) * 2 * C + c];
      s2 += part[static_cast<long>(i) * 2 * C + C + c];
    }
    S[c] = static_cast<float>(s1);
    S[C + c] = static_cast<float>(s2);
    dg[c] += static_cast<float>(s2);
    db[c] += static_cast<float>(s1);
  }
}

// dz = g istd (dA - S1/P - zhat S2/P)
__global__ void k_bn_bwd_apply(const float* __restrict__ dY, const float* __restrict__ z, long P, int C,
                               const float* __restrict__ mean, const float* __restrict__ istd,
                               const float* __restrict__ g, const float* __restrict__ b, int act,
                               const float* __restrict__ S, float* __restrict__ dz) {
  const float invP = 1.f / static_cast<float>(P);
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < P * C;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(i % C);
    const float zh = (z[i] - mean[c]) * istd[c];
    float dA = dY[i];
    if (act) dA *= sigmoidf(g[c] * zh + b[c]);
    dz[i] = g[c] * istd[c] * (dA - S[c] * invP - zh * S[C + c] * invP);
  }
}

// dT += dY summed over each group of `div` consecutive samples (div = 1: same shape)
__global__ void k_add_grad(const float* __restrict__ dY, long n_t, long sample_elems, int div,
                           float* __restrict__ dT) {
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n_t;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const long grp = i / sample_elems, off = i - grp * sample_elems;
    float s = 0.f;
    for (int q = 0; q < div; ++q) s += dY[(grp * div + q) * sample_elems + off];
    dT[i] += s;
  }
}

// ---- convolution backward -------------------------------------------------------------
struct ConvGeo {
  int B, Hi, Wi, Ci, Ho, Wo, Co, taps, mode;  // mode: S1, S2, T2, (T1 treated as transposed S1)
  int transposed;
};

// input pixel read by output (oy, ox) through tap (ty, tx); false if zero padding
__device__ __forceinline__ bool tap_src(const ConvGeo& g, int oy, int ox, int ty, int tx, int* iy, int* ix) {
  if (g.taps == 1) {
    *iy = oy;
    *ix = ox;
    return true;
  }
  const int dy = ty - 1, dx = tx - 1;
  if (g.mode == HELM_CONV_S2) {
    *iy = 2 * oy + dy;
    *ix = 2 * ox + dx;
  } else if (g.mode == HELM_CONV_T2) {
    const int Y = oy + dy, X = ox + dx;
    if (Y < 0 || X < 0 || (Y & 1) || (X & 1)) return false;
    *iy = Y >> 1;
    *ix = X >> 1;
  } else {
    *iy = oy + dy;
    *ix = ox + dx;
  }
  return *iy >= 0 && *iy < g.Hi && *ix >= 0 && *ix < g.Wi;
}

// weight of tap (ty, tx), output co, input ci in the master layout
__device__ __forceinline__ long widx(const ConvGeo& g, int ty, int tx, int co, int ci) {
  if (g.taps == 1) return static_cast<long>(co) * g.Ci + ci;
  if (g.transposed) return ((static_cast<long>(ci) * g.Co + co) * 3 + (2 - ty)) * 3 + (2 - tx);
  return ((static_cast<long>(co) * g.Ci + ci) * 3 + ty) * 3 + tx;
}

// FP32 weights repacked as [tap][co][ci] (ci contiguous) for the input-gradient kernel
__global__ void k_pack_dgrad_w(ConvGeo g, const float* __restrict__ w, float* __restrict__ out) {
  const long n = static_cast<long>(g.taps) * g.Co * g.Ci;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const int ci = static_cast<int>(i % g.Ci), co = static_cast<int>((i / g.Ci) % g.Co);
    const int tap = static_cast<int>(i / (static_cast<long>(g.Ci) * g.Co));
    const int ty = g.taps == 1 ? 1 : tap / 3, tx = g.taps == 1 ? 1 : tap % 3;
    out[i] = w[widx(g, ty, tx, co, ci)];
  }
}

// dX[b][iy][ix][8q..8q+7] += sum over (tap, co) of outputs reading (iy, ix); Ci % 8 == 0
__global__ void k_conv_dgrad(ConvGeo g, const float* __restrict__ dz, const float* __restrict__ wp,
                             float* __restrict__ dX) {
  const int G = g.Ci / 8;
  const long total = static_cast<long>(g.B) * g.Hi * g.Wi * G;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const int q = static_cast<int>(i % G);
    const long pix = i / G;
    const int ix = static_cast<int>(pix % g.Wi), iy = static_cast<int>((pix / g.Wi) % g.Hi);
    const int b = static_cast<int>(pix / (static_cast<long>(g.Wi) * g.Hi));
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int tap = 0; tap < g.taps; ++tap) {
      const int ty = g.taps == 1 ? 1 : tap / 3, tx = g.taps == 1 ? 1 : tap % 3;
      const int dy = ty - 1, dx = tx - 1;
      int oy, ox;
      if (g.taps == 1) {
        oy = iy;
        ox = ix;
      } else if (g.mode == HELM_CONV_S2) {
        if ((iy - dy) & 1 || (ix - dx) & 1) continue;
        oy = (iy - dy) >> 1;
        ox = (ix - dx) >> 1;
      } else if (g.mode == HELM_CONV_T2) {
        oy = 2 * iy - dy;
        ox = 2 * ix - dx;
      } else {
        oy = iy - dy;
        ox = ix - dx;
      }
      if (oy < 0 || oy >= g.Ho || ox < 0 || ox >= g.Wo) continue;
      const float* dzp = dz + ((static_cast<long>(b) * g.Ho + oy) * g.Wo + ox) * g.Co;
      const float* wt = wp + (static_cast<long>(tap) * g.Co) * g.Ci + 8 * q;
      for (int co = 0; co < g.Co; ++co) {
        const float d = dzp[co];
        const float4 w0 = *reinterpret_cast<const float4*>(wt + static_cast<long>(co) * g.Ci);
        const float4 w1 = *reinterpret_cast<const float4*>(wt + static_cast<long>(co) * g.Ci + 4);
        acc[0] = fmaf(w0.x, d, acc[0]);
        acc[1] = fmaf(w0.y, d, acc[1]);
        acc[2] = fmaf(w0.z, d, acc[2]);
        acc[3] = fmaf(w0.w, d, acc[3]);
        acc[4] = fmaf(w1.x, d, acc[4]);
        acc[5] = fmaf(w1.y, d, acc[5]);
        acc[6] = fmaf(w1.z, d, acc[6]);
        acc[7] = fmaf(w1.w, d, acc[7]);
      }
    }
    float* o = dX + pix * g.Ci + 8 * q;
#pragma unroll
    for (int e = 0; e < 8; ++e) o[e] += acc[e];
  }
}

// the same for inputs with fewer than 8 channels (the network's 2-channel input):
// thread per (pixel, channel)
__global__ void k_conv_dgrad_narrow(ConvGeo g, const float* __restrict__ dz, const float* __restrict__ wp,
                                    float* __restrict__ dX) {
  const long total = static_cast<long>(g.B) * g.Hi * g.Wi * g.Ci;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const int ci = static_cast<int>(i % g.Ci);
    const long pix = i / g.Ci;
    const int ix = static_cast<int>(pix % g.Wi), iy = static_cast<int>((pix / g.Wi) % g.Hi);
    const int b = static_cast<int>(pix / (static_cast<long>(g.Wi) * g.Hi));
    float acc = 0.f;
    for (int tap = 0; tap < g.taps; ++tap) {
      const int ty = g.taps == 1 ? 1 : tap / 3, tx = g.taps == 1 ? 1 : tap % 3;
      const int dy = ty - 1, dx = tx - 1;
      int oy, ox;
      if (g.taps == 1) {
        oy = iy;
        ox = ix;
      } else if (g.mode == HELM_CONV_S2) {
        if ((iy - dy) & 1 || (ix - dx) & 1) continue;
        oy = (iy - dy) >> 1;
        ox = (ix - dx) >> 1;
      } else if (g.mode == HELM_CONV_T2) {
        oy = 2 * iy - dy;
        ox = 2 * ix - dx;
      } else {
        oy = iy - dy;
        ox = ix - dx;
      }
      if (oy < 0 || oy >= g.Ho || ox < 0 || ox >= g.Wo) continue;
      const float* dzp = dz + ((static_cast<long>(b) * g.Ho + oy) * g.Wo + ox) * g.Co;
      const float* wt = wp + static_cast<long>(tap) * g.Co * g.Ci + ci;
      for (int co = 0; co < g.Co; ++co) acc = fmaf(wt[static_cast<long>(co) * g.Ci], dzp[co], acc);
    }
    dX[i] += acc;
  }
}

// ---- input gradient of e = s P(Net(R(r / s))), s = RMS(r) ----------------------------
// With x0 = R(r/s) and g0 = dL/dx0 (complex view of its two channels), the gradient is
//   t = P(g0) / (4 s)                          (through u = r / s, R^T = P / 4)
//   grad_r = t + r (<grad_e, e> - <t, r>) / (n s^2)
// (<a, b> = Re sum conj(a) b over the n grid points); the second term is the scale's
// dependence on r, fixed by e being positively homogeneous of degree 1 in r.
// Stage 1: t at every fine point (bilinear P: even fine index = coarse value, odd =
// mean of its two coarse neighbours, zero beyond the last coarse row / column).
__global__ void k_gradr_t(const float* __restrict__ g0, int N, int B, const float* __restrict__ s,
                          float2* __restrict__ t) {
  const int Nc = N / 2;
  const long total = static_cast<long>(B) * N * N;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const int b = static_cast<int>(i / (static_cast<long>(N) * N));
    const int y = static_cast<int>((i / N) % N), x = static_cast<int>(i % N);
    const float* gb = g0 + static_cast<long>(b) * Nc * Nc * 2;
    auto at = [&](int J, int K) -> float2 {
      if (J >= Nc || K >= Nc) return make_float2(0.f, 0.f);
      const float* q = gb + (static_cast<long>(J) * Nc + K) * 2;
      return make_float2(q[0], q[1]);
    };
    const int J = y >> 1, K = x >> 1;
    float2 v;
    if (!(y & 1) && !(x & 1)) v = at(J, K);
    else if (!(y & 1)) v = cscale(cadd(at(J, K), at(J, K + 1)), 0.5f);
    else if (!(x & 1)) v = cscale(cadd(at(J, K), at(J + 1, K)), 0.5f);
    else v = cscale(cadd(cadd(at(J, K), at(J, K + 1)), cadd(at(J + 1, K), at(J + 1, K + 1))), 0.25f);
    const float sb = s[b];
    t[i] = sb > 0.f ? cscale(v, 0.25f / sb) : make_float2(0.f, 0.f);
  }
}

// Stage 2: per-block partial sums of <grad_e, e> and <t, r> per sample (FP64 across
// threads, deterministic order)
__global__ void k_gradr_dots(const float2* __restrict__ ge, const float2* __restrict__ e,
                             const float2* __restrict__ t, const float2* __restrict__ r, long n, int nblk,
                             double* __restrict__ part /*[B][nblk][2]*/) {
  const int b = blockIdx.y;
  const long chunk = (n + nblk - 1) / nblk;
  const long p0 = blockIdx.x * chunk, p1 = min(p0 + chunk, n);
  double a0 = 0.0, a1 = 0.0;
  for (long p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const long q = static_cast<long>(b) * n + p;
    const float2 g = ge[q], ev = e[q], tv = t[q], rv = r[q];
    a0 += static_cast<double>(fmaf(g.x, ev.x, g.y * ev.y));
    a1 += static_cast<double>(fmaf(tv.x, rv.x, tv.y * rv.y));
  }
  a0 = warp_sum(a0);
  a1 = warp_sum(a1);
  __shared__ double red[2][32];
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a0;
    red[1][threadIdx.x >> 5] = a1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < (blockDim.x >> 5); ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    part[(static_cast<long>(b) * nblk + blockIdx.x) * 2] = s0;
    part[(static_cast<long>(b) * nblk + blockIdx.x) * 2 + 1] = s1;
  }
}

// Stage 3: grad_r = t + c_b r, c_b = (<grad_e, e> - <t, r>) / (n s_b^2); zero where s_b = 0
__global__ void k_gradr_fix(const double* __restrict__ part, int nblk, const float* __restrict__ s, long n,
                            const float2* __restrict__ r, float2* __restrict__ gr) {
  const int b = blockIdx.y;
  __shared__ float cb;
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int k = 0; k < nblk; ++k) {
      a0 += part[(static_cast<long>(b) * nblk + k) * 2];
      a1 += part[(static_cast<long>(b) * nblk + k) * 2 + 1];
    }
    const double sb = s[b];
    cb = sb > 0.0 ? static_cast<float>((a0 - a1) / (static_cast<double>(n) * sb * sb)) : 0.f;
  }
  __syncthreads();
  const float c = cb;
  for (long p = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; p < n;
       p += static_cast<long>(gridDim.x) * blockDim.x) {
    const long q = static_cast<long>(b) * n + p;
    const float2 rv = r[q], tv = gr[q];
    gr[q] = make_float2(fmaf(c, rv.x, tv.x), fmaf(c, rv.y, tv.y));
  }
}

// dW partials: block (tap, TCO x TCI output tile, pixel chunk) -> [chunk][tap][co][ci].
// 256 threads, each a (TCO/16) x (TCI/16) register tile; 32 pixels staged per pass
// (the pixel's source index is computed once per pixel, shared by the whole tile).
constexpr int WG_PIX = 2048;
template <int TCO, int TCI>
__global__ void __launch_bounds__(256) k_conv_wgrad(ConvGeo g, const bf16* __restrict__ x, const float* __restrict__ dz,
                                                    float* __restrict__ part) {
  constexpr int RO = TCO / 16, RI = TCI / 16;
  const int nco = (g.Co + TCO - 1) / TCO;
  const int tap = blockIdx.x % g.taps;
  const int cot = (blockIdx.x / g.taps) % nco;
  const int cit = blockIdx.x / (g.taps * nco);
  const int chunk = blockIdx.y;
  const int ty = g.taps == 1 ? 1 : tap / 3, tx = g.taps == 1 ? 1 : tap % 3;
  const int to = threadIdx.x >> 4, ti = threadIdx.x & 15;
  __shared__ float sdz[32][TCO + 1];
  __shared__ float sx[32][TCI + 1];
  __shared__ long ssrc[32];
  const long P = static_cast<long>(g.B) * g.Ho * g.Wo;
  const long p0 = static_cast<long>(chunk) * WG_PIX, p1 = min(p0 + WG_PIX, P);
  float acc[RO][RI];
#pragma unroll
  for (int a = 0; a < RO; ++a)
#pragma unroll
    for (int b = 0; b < RI; ++b) acc[a][b] = 0.f;
  for (long pb = p0; pb < p1; pb += 32) {
    if (threadIdx.x < 32) {
      const long p = pb + threadIdx.x;
      long src = -1;
      if (p < p1) {
        const int ox = static_cast<int>(p % g.Wo), oy = static_cast<int>((p / g.Wo) % g.Ho);
        const int b = static_cast<int>(p / (static_cast<long>(g.Wo) * g.Ho));
        int iy, ix;
        if (tap_src(g, oy, ox, ty, tx, &iy, &ix)) src = ((static_cast<long>(b) * g.Hi + iy) * g.Wi + ix) * g.Ci;
      }
      ssrc[threadIdx.x] = src;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * TCO; e += 256) {
      const int pl = e / TCO, c = e % TCO;
      const long p = pb + pl;
      const int cz = cot * TCO + c;
      sdz[pl][c] = (p < p1 && cz < g.Co) ? dz[p * g.Co + cz] : 0.f;
    }
    for (int e = threadIdx.x; e < 32 * TCI; e += 256) {
      const int pl = e / TCI, c = e % TCI;
      const int cx = cit * TCI + c;
      const long src = ssrc[pl];
      sx[pl][c] = (src >= 0 && cx < g.Ci) ? __bfloat162float(x[src + cx]) : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int pl = 0; pl < 32; ++pl) {
      float dv[RO], xv[RI];
#pragma unroll
      for (int a = 0; a < RO; ++a) dv[a] = sdz[pl][to + 16 * a];
#pragma unroll
      for (int b = 0; b < RI; ++b) xv[b] = sx[pl][ti + 16 * b];
#pragma unroll
      for (int a = 0; a < RO; ++a)
#pragma unroll
        for (int b = 0; b < RI; ++b) acc[a][b] = fmaf(dv[a], xv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < RO; ++a)
#pragma unroll
    for (int b = 0; b < RI; ++b) {
      const int co = cot * TCO + to + 16 * a, ci = cit * TCI + ti + 16 * b;
      if (co < g.Co && ci < g.Ci)
        part[((static_cast<long>(chunk) * g.taps + tap) * g.Co + co) * g.Ci + ci] = acc[a][b];
    }
}

template <int TCO, int TCI>
void launch_wgrad(const ConvGeo& g, const bf16* x, const float* dz, float* part, int nch, cudaStream_t st) {
  const int tiles = g.taps * ((g.Co + TCO - 1) / TCO) * ((g.Ci + TCI - 1) / TCI);
  k_conv_wgrad<TCO, TCI><<<dim3(tiles, nch), 256, 0, st>>>(g, x, dz, part);
}

// sum the partials over chunks, add into the master-layout gradient
__global__ void k_wgrad_reduce(ConvGeo g, const float* __restrict__ part, int nchunk, float* __restrict__ dw) {
  const long n = static_cast<long>(g.taps) * g.Co * g.Ci;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < nchunk; ++k) s += part[k * n + i];
    const int ci = static_cast<int>(i % g.Ci), co = static_cast<int>((i / g.Ci) % g.Co);
    const int tap = static_cast<int>(i / (static_cast<long>(g.Ci) * g.Co));
    const int ty = g.taps == 1 ? 1 : tap / 3, tx = g.taps == 1 ? 1 : tap % 3;
    dw[widx(g, ty, tx, co, ci)] += s;
  }
}

// ---- depthwise backward ----------------------------------------------------------------
__global__ void k_dw_dgrad(const float* __restrict__ dz, int B, int H, int W, int C, const float* __restrict__ w,
                           float* __restrict__ dX) {
  const long total = static_cast<long>(B) * H * W * C;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(i % C);
    const long pix = i / C;
    const int xx = static_cast<int>(pix % W), yy = static_cast<int>((pix / W) % H);
    const int b = static_cast<int>(pix / (static_cast<long>(W) * H));
    float acc = 0.f;
    for (int ty = 0; ty < 3; ++ty)
      for (int tx = 0; tx < 3; ++tx) {
        const int oy = yy - (ty - 1), ox = xx - (tx - 1);
        if (oy < 0 || oy >= H || ox < 0 || ox >= W) continue;
        acc = fmaf(w[c * 9 + ty * 3 + tx], dz[((static_cast<long>(b) * H + oy) * W + ox) * C + c], acc);
      }
    dX[i] += acc;
  }
}

// partials [chunk][C][9]: thread per channel (coalesced), the 9 taps in registers
constexpr int DW_PIX = 256;
__global__ void k_dw_wgrad(const bf16* __restrict__ x, const float* __restrict__ dz, int B, int H, int W, int C,
                           float* __restrict__ part) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const long P = static_cast<long>(B) * H * W;
  const long p0 = static_cast<long>(blockIdx.y) * DW_PIX, p1 = min(p0 + DW_PIX, P);
  float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (long p = p0; p < p1; ++p) {
    const int xx = static_cast<int>(p % W), yy = static_cast<int>((p / W) % H);
    const int b = static_cast<int>(p / (static_cast<long>(W) * H));
    const float d = dz[p * C + c];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int sy = yy + tap / 3 - 1, sx = xx + tap % 3 - 1;
      if (sy < 0 || sy >= H || sx < 0 || sx >= W) continue;
      acc[tap] = fmaf(d, __bfloat162float(x[((static_cast<long>(b) * H + sy) * W + sx) * C + c]), acc[tap]);
    }
  }
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) part[(static_cast<long>(blockIdx.y) * C + c) * 9 + tap] = acc[tap];
}

__global__ void k_sum_chunks_add(const float* __restrict__ part, int nchunk, long n, float* __restrict__ out) {
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < nchunk; ++k) s += part[k * n + i];
    out[i] += s;
  }
}

// ---- implicit layer kernel gradient ------------------------------------------------------
// per (b, k): contribution conj(X_hat) . F(pad(gy)) / (2m)^2 to grad G_hat_k
__global__ void k_implicit_kgrad(const bf16* __restrict__ x, const float* __restrict__ gy, int m, int C,
                                 float2* __restrict__ contrib) {
  const int b = blockIdx.y, k = blockIdx.x;
  const int n = 2 * m;
  extern __shared__ float2 ism[];
  float2* Wt = ism;
  float2* X = Wt + n;
  float2* R = X + m * m;
  float2* F1 = R + m * n;
  float2* F2 = F1 + n * n;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    float s, c;
    sincospif(-2.f * e / n, &s, &c);
    Wt[e] = make_float2(c, s);
  }
  const long base = static_cast<long>(b) * m * m;
  for (int i = threadIdx.x; i < m * m; i += blockDim.x)
    X[i] = make_float2(__bfloat162float(x[(base + i) * C + k]), __bfloat162float(x[(base + i) * C + k + C / 2]));
  __syncthreads();
  // forward DFT of pad(x) into F1
  for (int i = threadIdx.x; i < m * n; i += blockDim.x) {
    const int r = i / n, u = i % n;
    float2 acc = make_float2(0.f, 0.f);
    for (int c = 0, e = 0; c < m; ++c, e = (e + u >= n ? e + u - n : e + u))
      acc = cadd(acc, cmul(X[r * m + c], Wt[e]));
    R[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int v = i / n, u = i % n;
    float2 acc = make_float2(0.f, 0.f);
    for (int r = 0, e = 0; r < m; ++r, e = (e + v >= n ? e + v - n : e + v))
      acc = cadd(acc, cmul(R[r * n + u], Wt[e]));
    F1[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m * m; i += blockDim.x)
    X[i] = make_float2(gy[(base + i) * C + k], gy[(base + i) * C + k + C / 2]);
  __syncthreads();
  for (int i = threadIdx.x; i < m * n; i += blockDim.x) {
    const int r = i / n, u = i % n;
    float2 acc = make_float2(0.f, 0.f);
    for (int c = 0, e = 0; c < m; ++c, e = (e + u >= n ? e + u - n : e + u))
      acc = cadd(acc, cmul(X[r * m + c], Wt[e]));
    R[i] = acc;
  }
  __syncthreads();
  const float sc = 1.f / static_cast<float>(n * n);
  float2* out = contrib + (static_cast<long>(b) * gridDim.x + k) * n * n;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int v = i / n, u = i % n;
    float2 acc = make_float2(0.f, 0.f);
    for (int r = 0, e = 0; r < m; ++r, e = (e + v >= n ? e + v - n : e + v))
      acc = cadd(acc, cmul(R[r * n + u], Wt[e]));
    F2[i] = acc;
    out[i] = cscale(cmulc(F1[i], acc), sc);  // conj(X_hat) * F(pad gy) / n^2
  }
}

// g_ghat[k] = sum_b contrib[b][k]
__global__ void k_sum_batch_c(const float2* __restrict__ contrib, int B, long n, float2* __restrict__ out) {
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    float2 s = make_float2(0.f, 0.f);
    for (int b = 0; b < B; ++b) s = cadd(s, contrib[b * n + i]);
    out[i] = s;
  }
}

// grad G_hat -> grad K (one CTA per channel), following the adjoints of Eq. (15):
//   g_Gc = sum_{p,q} g_ghat e^{+2 pi i (p i + q j)/2m}             (F^H of the 2m DFT)
//   g_H[u][v] = (1/n6^2) sum_{offsets d} g_Gc(d) e^{-2 pi i (u dy + v dx)/n6}
//   g_Kh = g_H conj(a) + conj(g_H) b,  a = dH/dKh, b = dH/dconj(Kh)
//   g_K[a][b] = sum_{u,v} g_Kh e^{+2 pi i (u a + v b)/n6}            (F^H of the n6 DFT)
__global__ void k_greens_bwd(const float* __restrict__ Kpar, int nk, int m, float eps, int literal,
                             const float2* __restrict__ gghat, float2* __restrict__ scratch,
                             float* __restrict__ gK /*[2][nk][9] += */) {
  const int k = blockIdx.x;
  const int n6 = 6 * m, n = 2 * m;
  float2* gGc = scratch + static_cast<long>(k) * (n * n + n * n6 + n6 * n6);
  float2* T = gGc + n * n;
  float2* gKh = T + n * n6;
  const float2* gg = gghat + static_cast<long>(k) * n * n;
  // g_Gc = F^H g_ghat: rows then columns (T as scratch, layout [n][n])
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int p = i / n, j = i % n;
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < n; ++q) {
      float s, c;
      sincospif(2.f * ((q * j) % n) / n, &s, &c);
      acc = cadd(acc, cmul(gg[p * n + q], make_float2(c, s)));
    }
    T[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int ii = i / n, j = i % n;
    float2 acc = make_float2(0.f, 0.f);
    for (int p = 0; p < n; ++p) {
      float s, c;
      sincospif(2.f * ((p * ii) % n) / n, &s, &c);
      acc = cadd(acc, cmul(T[p * n + j], make_float2(c, s)));
    }
    gGc[i] = acc;
  }
  __syncthreads();
  // T2[i][v] = sum_j gGc[i][j] e^{-2 pi i v dx_j / n6}  (layout [n][n6])
  for (int i = threadIdx.x; i < n * n6; i += blockDim.x) {
    const int ii = i / n6, v = i % n6;
    float2 acc = make_float2(0.f, 0.f);
    for (int j = 0; j < n; ++j) {
      const int dx = j < m ? j : j - n;
      float s, c;
      const int e = ((v * dx) % n6 + n6) % n6;
      sincospif(-2.f * e / n6, &s, &c);
      acc = cadd(acc, cmul(gGc[ii * n + j], make_float2(c, s)));
    }
    T[i] = acc;
  }
  __syncthreads();
  float Kr[9], Ki[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    Kr[t] = Kpar[k * 9 + t];
    Ki[t] = Kpar[(nk + k) * 9 + t];
  }
  const float sc = 1.f / (static_cast<float>(n6) * n6);
  for (int i = threadIdx.x; i < n6 * n6; i += blockDim.x) {
    const int u = i / n6, v = i % n6;
    float2 gH = make_float2(0.f, 0.f);
    for (int ii = 0; ii < n; ++ii) {
      const int dy = ii < m ? ii : ii - n;
      float s, c;
      const int e = ((u * dy) % n6 + n6) % n6;
      sincospif(-2.f * e / n6, &s, &c);
      gH = cadd(gH, cmul(T[ii * n6 + v], make_float2(c, s)));
    }
    gH = cscale(gH, sc);
    float2 kh = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = -1; a <= 1; ++a)
#pragma unroll
      for (int c2 = -1; c2 <= 1; ++c2) {
        float s, c;
        const int e = ((u * a + v * c2) % n6 + n6) % n6;
        sincospif(-2.f * e / n6, &s, &c);
        const int t = (a + 1) * 3 + (c2 + 1);
        kh = cadd(kh, cmul(make_float2(Kr[t], Ki[t]), make_float2(c, s)));
      }
    float2 gk;
    if (literal) {
      // H = Kh / (Kh^2 + eps), holomorphic: a = (eps - Kh^2)/(Kh^2 + eps)^2, b = 0
      const float2 k2 = cmul(kh, kh);
      const float2 den = make_float2(k2.x + eps, k2.y);
      const float2 den2 = cmul(den, den);
      const float2 num = make_float2(eps - k2.x, -k2.y);
      const float d2 = den2.x * den2.x + den2.y * den2.y;
      const float2 a = make_float2((num.x * den2.x + num.y * den2.y) / d2, (num.y * den2.x - num.x * den2.y) / d2);
      gk = cmul(gH, make_float2(a.x, -a.y));
    } else {
      const float mag2 = kh.x * kh.x + kh.y * kh.y;
      const float den = (mag2 + eps) * (mag2 + eps);
      // a = -conj(Kh)^2 / den, b = eps / den; g_Kh = gH conj(a) + conj(gH) b
      const float2 ck = make_float2(kh.x, -kh.y);
      const float2 ck2 = cmul(ck, ck);
      const float2 a = make_float2(-ck2.x / den, -ck2.y / den);
      gk = cadd(cmul(gH, make_float2(a.x, -a.y)), cscale(make_float2(gH.x, -gH.y), eps / den));
    }
    gKh[i] = gk;
  }
  __syncthreads();
  // g_K[t] = sum_{u,v} g_Kh e^{+2 pi i (u a + v b)/n6}: 9 outputs, block reduction each
  __shared__ float red[2][256];
  for (int t = 0; t < 9; ++t) {
    const int a = t / 3 - 1, c2 = t % 3 - 1;
    float sr = 0.f, si = 0.f;
    for (int i = threadIdx.x; i < n6 * n6; i += blockDim.x) {
      const int u = i / n6, v = i % n6;
      float s, c;
      const int e = ((u * a + v * c2) % n6 + n6) % n6;
      sincospif(2.f * e / n6, &s, &c);
      const float2 z = cmul(gKh[i], make_float2(c, s));
      sr += z.x;
      si += z.y;
    }
    red[0][threadIdx.x] = sr;
    red[1][threadIdx.x] = si;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        red[0][threadIdx.x] += red[0][threadIdx.x + o];
        red[1][threadIdx.x] += red[1][threadIdx.x + o];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      gK[k * 9 + t] += red[0][0];
      gK[(nk + k) * 9 + t] += red[1][0];
    }
    __syncthreads();
  }
}

// ---- projection + P backward ----------------------------------------------------------
// g_p = s * P^T g_e = s * 4 R(g_e) at I/2; du[c] = sum_o w[o][c] g_p[o]; dW, db partials
__global__ void __launch_bounds__(256) k_proj_bwd(const float2* __restrict__ ge, const bf16* __restrict__ u, int B,
                                                  int Nc, int C, const float* __restrict__ w,
                                                  const float* __restrict__ s, float* __restrict__ du,
                                                  float* __restrict__ part /*[nblk][2*C + 2]*/) {
  const int N = 2 * Nc;
  constexpr int MAXC = 16;
  float pw[2 * MAXC + 2];
#pragma unroll
  for (int i = 0; i < 2 * MAXC + 2; ++i) pw[i] = 0.f;
  const long total = static_cast<long>(B) * Nc * Nc;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const int b = static_cast<int>(i / (static_cast<long>(Nc) * Nc));
    const int J = static_cast<int>((i / Nc) % Nc), K = static_cast<int>(i % Nc);
    float2 acc = make_float2(0.f, 0.f);
    for (int a = -1; a <= 1; ++a)
      for (int c = -1; c <= 1; ++c) {
        const int y = 2 * J + a, x = 2 * K + c;
        if (y < 0 || y >= N || x < 0 || x >= N) continue;
        const float wt = (a == 0 ? 2.f : 1.f) * (c == 0 ? 2.f : 1.f) * 0.25f;
        const float2 gv = ge[(static_cast<long>(b) * N + y) * N + x];
        acc.x += wt * gv.x;
        acc.y += wt * gv.y;
      }
    acc = cscale(acc, s[b]);
    const bf16* up = u + i * C;
#pragma unroll
    for (int ch = 0; ch < MAXC; ++ch) {
      if (ch >= C) break;
      du[i * C + ch] += w[ch] * acc.x + w[C + ch] * acc.y;
      const float v = __bfloat162float(up[ch]);
      pw[ch] = fmaf(acc.x, v, pw[ch]);
      pw[MAXC + ch] = fmaf(acc.y, v, pw[MAXC + ch]);
    }
    pw[2 * MAXC] += acc.x;
    pw[2 * MAXC + 1] += acc.y;
  }
  __shared__ float red[8][2 * MAXC + 2];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 2 * MAXC + 2; ++i) {
    const float v = warp_sum(pw[i]);
    if (lane == 0) red[wp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2 * C + 2) {
    // output order: w0[0..C), w1[0..C), b0, b1
    const int t = threadIdx.x;
    const int src = t < C ? t : (t < 2 * C ? MAXC + (t - C) : 2 * MAXC + (t - 2 * C));
    float v = 0.f;
    for (int q = 0; q < (blockDim.x >> 5); ++q) v += red[q][src];
    part[static_cast<long>(blockIdx.x) * (2 * C + 2) + t] = v;
  }
}

// out[i] += sum_k part[k * stride + off + i], i < n
__global__ void k_strided_reduce(const float* __restrict__ part, int nchunk, int stride, int off, int n,
                                 float* __restrict__ out) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < nchunk; ++k) s += part[static_cast<long>(k) * stride + off + i];
    out[i] += s;
  }
}

// ---- loss and optimiser ---------------------------------------------------------------
// loss = (1/B) sum |e - t|^2, grad = 2 (e - t) / B; loss via per-block partials
__global__ void k_mse(const float2* __restrict__ e, const float2* __restrict__ t, long n, int B,
                      float2* __restrict__ grad, double* __restrict__ part) {
  double acc = 0.0;
  const float sc = 2.f / B;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const float2 d = csub(e[i], t[i]);
    acc += static_cast<double>(d.x) * d.x + static_cast<double>(d.y) * d.y;
    if (grad) grad[i] = cscale(d, sc);
  }
  acc = warp_sum(acc);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < (blockDim.x >> 5); ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

__global__ void k_mse_final(const double* __restrict__ part, int nblk, int B, double* __restrict__ loss) {
  double s = 0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += part[i];
  s = warp_sum(s);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (blockDim.x >> 5); ++w) t += red[w];
    *loss = t / B;
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace

// =====================================================================================
// training state carved from the caller's workspace (same order in forward/backward)
struct TrainState {
  Plan enc, sol;
  int enc_out[3], kf, x0, u3, enc_ids[3];
  std::vector<void*> eptr, sptr;     // activation pointers
  std::vector<float*> eraw, sraw;    // raw z per layer (null if no BN)
  std::vector<float*> emean, eistd, smean, sistd;
  float *s, *inv;
  double* part;
  float2* esave;   // the forward's output e, for the input gradient
  // backward
  float* gx0;      // dL/dx0 of the network input (only when the input gradient is asked for)
  std::vector<float*> egrad, sgrad;  // dT per tensor
  float* dz;
  float* wpart;
  double* bnpart;
  float* S;
  float2 *kcontrib, *gghat, *gscr;
  float* ppart;
  size_t dz_elems, wpart_elems;
  bool overflow;
};

static const int kMaxChunks = 2048;   // BN / projection reduction blocks
static const int kMaxWChunks = 512;   // weight-gradient pixel chunks

static void carve_train(const helm_cnn* c, int I, int B, int nprob, Carve& cv, TrainState* T, bool with_backward) {
  build_encoder_plan(c, I, I, &T->enc, T->enc_out, &T->kf, nprob);
  build_solver_plan(c, I, I, B, skip_for(c, I, I), &T->sol, &T->x0, &T->u3, T->enc_ids, nprob);
  char* ea = cv.take<char>(T->enc.arena);
  char* sa = cv.take<char>(T->sol.arena);
  T->eptr.resize(T->enc.t.size());
  T->sptr.resize(T->sol.t.size());
  for (size_t i = 0; i < T->enc.t.size(); ++i) T->eptr[i] = ea ? ea + T->enc.t[i].off : nullptr;
  for (size_t i = 0; i < T->sol.t.size(); ++i)
    T->sptr[i] = (sa && T->sol.t[i].off != ~size_t(0)) ? sa + T->sol.t[i].off : nullptr;
  for (int k = 0; k < 3; ++k) T->sptr[T->enc_ids[k]] = T->eptr[T->enc_out[k]];
  auto raws = [&](const Plan& pl, std::vector<float*>& raw, std::vector<float*>& mean, std::vector<float*>& istd) {
    for (const Layer& L : pl.layers) {
      if (L.bn < 0) {
        raw.push_back(nullptr);
        mean.push_back(nullptr);
        istd.push_back(nullptr);
        continue;
      }
      const TensorDesc& o = pl.t[L.out];
      raw.push_back(cv.take<float>(static_cast<size_t>(o.B) * o.H * o.W * o.C));
      mean.push_back(cv.take<float>(o.C));
      istd.push_back(cv.take<float>(o.C));
    }
  };
  raws(T->enc, T->eraw, T->emean, T->eistd);
  raws(T->sol, T->sraw, T->smean, T->sistd);
  T->s = cv.take<float>(B);
  T->inv = cv.take<float>(B);
  T->part = cv.take<double>(static_cast<size_t>(B) * 256 + 2 * 384 * kMaxChunks);
  T->esave = cv.take<float2>(static_cast<size_t>(B) * I * I);
  if (with_backward) {
    size_t maxel = 0;
    auto grads = [&](const Plan& pl, std::vector<float*>& g) {
      for (const TensorDesc& t : pl.t) {
        if (t.off == ~size_t(0)) {
          g.push_back(nullptr);
          continue;
        }
        const size_t el = static_cast<size_t>(t.B) * t.H * t.W * t.C;
        maxel = std::max(maxel, el);
        g.push_back(cv.take<float>(el));
      }
    };
    grads(T->enc, T->egrad);
    grads(T->sol, T->sgrad);
    for (int k = 0; k < 3; ++k) T->sgrad[T->enc_ids[k]] = T->egrad[T->enc_out[k]];
    T->egrad[T->kf] = nullptr;   // no gradient needed for the network inputs
    T->sgrad[T->x0] = nullptr;
    T->dz_elems = maxel;
    T->dz = cv.take<float>(maxel);
    T->wpart_elems = static_cast<size_t>(kMaxWChunks) * 9 * 64 * 64;
    T->wpart = cv.take<float>(T->wpart_elems);
    T->bnpart = T->part;
    T->S = cv.take<float>(2 * 384);
    const int m = T->sol.m, n = 2 * m, n6 = 6 * m;
    const int nk = c->desc.c0 * 2;
    T->kcontrib = cv.take<float2>(static_cast<size_t>(B) * nk * n * n);
    T->gghat = cv.take<float2>(static_cast<size_t>(nk) * n * n);
    T->gscr = cv.take<float2>(static_cast<size_t>(nk) * (n * n + n * n6 + n6 * n6));
    T->ppart = cv.take<float>(static_cast<size_t>(kMaxChunks) * (2 * 16 + 2));
    T->gx0 = cv.take<float>(static_cast<size_t>(B) * (I / 2) * (I / 2) * 2);
  }
  T->overflow = cv.overflow;
}

size_t cnn_train_bytes(const helm_cnn* c, int I, int B, int nprob) {
  Carve cv(nullptr, ~size_t(0));
  TrainState T;
  carve_train(c, I, B, nprob, cv, &T, true);
  return cv.off + 4096;
}

static const float* PP(const helm_cnn* c, int idx) { return c->params_dev + c->params[idx].offset; }

// forward of one plan in training mode
static int run_layers_train(helm_cnn* c, const Plan& pl, const std::vector<void*>& ptr, const std::vector<float*>& raw,
                            const std::vector<float*>& mean, const std::vector<float*>& istd, double* part,
                            cudaStream_t st) {
  for (size_t li = 0; li < pl.layers.size(); ++li) {
    const Layer& L = pl.layers[li];
    const TensorDesc& in = pl.t[L.in];
    const TensorDesc& out = pl.t[L.out];
    int rc = HELM_OK;
    if (L.kind == L_IMPL) {
      rc = launch_implicit_bf16(static_cast<const bf16*>(ptr[L.in]), in.B, in.H, in.W, in.C, c->ghat.at(pl.m),
                                static_cast<bf16*>(ptr[L.out]), st);
      if (rc) return rc;
      continue;
    }
    if (L.kind == L_CONV) {
      ConvLaunch cl;
      cl.x = static_cast<const bf16*>(ptr[L.in]);
      cl.B = in.B;
      cl.Hi = in.H;
      cl.Wi = in.W;
      cl.Ci = L.ci;
      cl.Co = L.co;
      cl.taps = L.taps;
      cl.mode = L.mode == HELM_CONV_T1 ? HELM_CONV_S1 : L.mode;
      cl.wpk = c->wpk + wpk_offset(c, L.wparam);
      cl.yraw = raw[li];
      rc = conv_tc(cl, st);
    } else {
      rc = launch_dw(static_cast<const bf16*>(ptr[L.in]), in.B, in.H, in.W, in.C, PP(c, L.wparam), nullptr, nullptr, 0,
                     nullptr, raw[li], st);
    }
    if (rc) return rc;
    // BN statistics and the epilogue
    const BnInfo& bn = c->bns[L.bn];
    const long P = static_cast<long>(out.B) * out.H * out.W;
    const long chunk = bn_chunk(P);
    const int nblk = div_up(P, chunk);
    if (nblk > kMaxChunks) {
      set_error("cnn training: activation too large for the BN reduction");
      return HELM_ESHAPE;
    }
    HELM_LAUNCH("k_chan_sums", st, k_chan_sums<<<nblk, chan_block(bn.C), chan_smem(bn.C), st>>>(raw[li], P, bn.C, chunk, part));
    HELM_LAUNCH("k_bn_finalize", st,
                k_bn_finalize<<<div_up(bn.C, 128), 128, 0, st>>>(part, nblk, bn.C, P, mean[li], istd[li],
                                                                 c->running + bn.roff, c->running + bn.roff + bn.C));
    const int div2 = L.add2 >= 0 ? out.B / pl.t[L.add2].B : 1;
    HELM_LAUNCH("k_bn_apply", st,
                k_bn_apply<<<gridn(P * bn.C), 256, 0, st>>>(
                    raw[li], P, bn.C, mean[li], istd[li], PP(c, bn.pg), PP(c, bn.pb), L.act,
                    L.add1 >= 0 ? static_cast<const bf16*>(ptr[L.add1]) : nullptr,
                    L.add2 >= 0 ? static_cast<const bf16*>(ptr[L.add2]) : nullptr,
                    static_cast<long>(out.H) * out.W * bn.C, div2, static_cast<bf16*>(ptr[L.out])));
    HELM_CHECK_LAUNCH("bn train");
  }
  return HELM_OK;
}

int cnn_forward_train(helm_cnn* c, const helm_problem* const* probs, int nprob, const float2* r, float2* e, int B,
                      Carve& cv, cudaStream_t st) {
  const helm_problem* p = probs[0];
  const int I = p->nx;
  if (p->nx != p->ny || I % 16) {
    set_error("cnn: the network needs a square grid divisible by 16");
    return HELM_ESHAPE;
  }
  if (nprob < 1 || B % nprob) {
    set_error("cnn training: batch %d not divisible by the %d slowness models", B, nprob);
    return HELM_EINVAL;
  }
  for (int k = 1; k < nprob; ++k)
    if (probs[k]->nx != I || probs[k]->ny != I) {
      set_error("cnn training: all slowness models of a batch need the same grid");
      return HELM_ESHAPE;
    }
  TrainState T;
  carve_train(c, I, B, nprob, cv, &T, true);
  if (T.overflow) {
    set_error("cnn training: workspace too small (helm_cnn_train_workspace_size)");
    return HELM_EWORKSPACE;
  }
  int rc = cnn_derive(c, T.sol.m, st);
  if (rc) return rc;
  for (int k = 0; k < nprob; ++k)
    if ((rc = launch_kfeat(probs[k]->kappa, probs[k]->gamma, p->npts(0),
                           static_cast<bf16*>(T.eptr[T.kf]) + static_cast<size_t>(k) * p->npts(0) * 2, st)))
      return rc;
  if ((rc = run_layers_train(c, T.enc, T.eptr, T.eraw, T.emean, T.eistd, T.part, st))) return rc;
  if ((rc = launch_prep(r, I, I, B, T.part, T.s, T.inv, static_cast<bf16*>(T.sptr[T.x0]), st))) return rc;
  if ((rc = run_layers_train(c, T.sol, T.sptr, T.sraw, T.smean, T.sistd, T.part, st))) return rc;
  const ParamInfo& pw = c->params[c->pidx.at("s.proj.w")];
  const ParamInfo& pb = c->params[c->pidx.at("s.proj.b")];
  rc = launch_proj(static_cast<const bf16*>(T.sptr[T.u3]), B, I / 2, I / 2, T.sol.t[T.u3].C, c->params_dev + pw.offset,
                   c->params_dev + pb.offset, T.s, e, st);
  if (rc) return rc;
  HELM_CUDA(cudaMemcpyAsync(T.esave, e, static_cast<size_t>(B) * I * I * sizeof(float2), cudaMemcpyDeviceToDevice,
                            st));
  c->enc_prob = nullptr;  // the cached evaluation-mode encodings are stale now
  c->dirty = true;        // running statistics moved: refold before the next inference
  c->train_nprob = nprob;
  return HELM_OK;
}

// backward through one plan
static int run_layers_backward(helm_cnn* c, const Plan& pl, const TrainState& T, const std::vector<void*>& ptr,
                               const std::vector<float*>& raw, const std::vector<float*>& mean,
                               const std::vector<float*>& istd, const std::vector<float*>& grad, float* gparams,
                               cudaStream_t st) {
  for (int li = static_cast<int>(pl.layers.size()) - 1; li >= 0; --li) {
    const Layer& L = pl.layers[li];
    const TensorDesc& in = pl.t[L.in];
    const TensorDesc& out = pl.t[L.out];
    float* dY = grad[L.out];
    if (L.kind == L_IMPL) {
      int rc = launch_implicit_adjoint(dY, in.B, in.H, in.C, c->ghat.at(pl.m), grad[L.in], st);
      if (rc) return rc;
      const int m = pl.m, n = 2 * m, nk = in.C / 2;
      const size_t sm = implicit_smem(m) + static_cast<size_t>(n) * n * sizeof(float2);
      static std::atomic<unsigned long long> attr_done{0};
      if ((rc = smem_attr_once(k_implicit_kgrad, 200 * 1024, &attr_done))) return rc;
      HELM_LAUNCH("k_implicit_kgrad", st,
                  k_implicit_kgrad<<<dim3(nk, in.B), 256, sm, st>>>(static_cast<const bf16*>(ptr[L.in]), dY, m, in.C,
                                                                   T.kcontrib));
      HELM_LAUNCH("k_sum_batch_c", st,
                  k_sum_batch_c<<<gridn(static_cast<long>(nk) * n * n), 256, 0, st>>>(T.kcontrib, in.B,
                                                                                      static_cast<long>(nk) * n * n,
                                                                                      T.gghat));
      HELM_LAUNCH("k_greens_bwd", st,
                  k_greens_bwd<<<nk, 256, 0, st>>>(PP(c, L.wparam), nk, m, 1e-5f, c->desc.literal_green, T.gghat,
                                                    T.gscr, gparams + c->params[L.wparam].offset));
      HELM_CHECK_LAUNCH("implicit backward");
      continue;
    }
    const BnInfo& bn = c->bns[L.bn];
    const long P = static_cast<long>(out.B) * out.H * out.W;
    const long n_out = P * bn.C;
    // additive skips receive dY unchanged (batch-summed for a broadcast encoding)
    const long selem = static_cast<long>(out.H) * out.W * bn.C;
    if (L.add1 >= 0 && grad[L.add1])
      HELM_LAUNCH("k_add_grad", st, k_add_grad<<<gridn(n_out), 256, 0, st>>>(dY, n_out, selem, 1, grad[L.add1]));
    if (L.add2 >= 0 && grad[L.add2]) {
      const TensorDesc& a2 = pl.t[L.add2];
      const long n_t = static_cast<long>(a2.B) * a2.H * a2.W * a2.C;
      HELM_LAUNCH("k_add_grad", st,
                  k_add_grad<<<gridn(n_t), 256, 0, st>>>(dY, n_t, selem, out.B / a2.B, grad[L.add2]));
    }
    // BN + activation
    const long chunk = bn_chunk(P);
    const int nblk = div_up(P, chunk);
    HELM_LAUNCH("k_bn_bwd_sums", st,
                k_bn_bwd_sums<<<nblk, chan_block(bn.C), chan_smem(bn.C), st>>>(dY, raw[li], P, bn.C, mean[li], istd[li],
                                                                           PP(c, bn.pg), PP(c, bn.pb), L.act,
                                                                           chunk, T.bnpart));
    HELM_LAUNCH("k_bn_bwd_final", st,
                k_bn_bwd_final<<<div_up(bn.C, 128), 128, 0, st>>>(T.bnpart, nblk, bn.C, T.S,
                                                                  gparams + c->params[bn.pg].offset,
                                                                  gparams + c->params[bn.pb].offset));
    HELM_LAUNCH("k_bn_bwd_apply", st,
                k_bn_bwd_apply<<<gridn(n_out), 256, 0, st>>>(dY, raw[li], P, bn.C, mean[li], istd[li], PP(c, bn.pg),
                                                             PP(c, bn.pb), L.act, T.S, T.dz));
    HELM_CHECK_LAUNCH("bn backward");
    // convolution / depthwise backward
    if (L.kind == L_DW) {
      if (grad[L.in])
        HELM_LAUNCH("k_dw_dgrad", st,
                    k_dw_dgrad<<<gridn(n_out), 256, 0, st>>>(T.dz, in.B, in.H, in.W, in.C, PP(c, L.wparam), grad[L.in]));
      const int nch = div_up(P, DW_PIX);
      if (static_cast<size_t>(nch) * in.C * 9 > T.wpart_elems) {
        set_error("cnn training: depthwise weight-gradient partials exceed the workspace");
        return HELM_ESHAPE;
      }
      HELM_LAUNCH("k_dw_wgrad", st,
                  k_dw_wgrad<<<dim3(div_up(in.C, 64), nch), 64, 0, st>>>(static_cast<const bf16*>(ptr[L.in]),
                                                                              T.dz, in.B, in.H, in.W, in.C, T.wpart));
      HELM_LAUNCH("k_sum_chunks_add", st,
                  k_sum_chunks_add<<<gridn(in.C * 9), 256, 0, st>>>(T.wpart, nch, in.C * 9,
                                                                    gparams + c->params[L.wparam].offset));
      HELM_CHECK_LAUNCH("dw backward");
      continue;
    }
    ConvGeo g;
    g.B = in.B;
    g.Hi = in.H;
    g.Wi = in.W;
    g.Ci = L.ci;
    g.Ho = out.H;
    g.Wo = out.W;
    g.Co = L.co;
    g.taps = L.taps;
    g.mode = L.mode == HELM_CONV_T1 ? HELM_CONV_S1 : L.mode;
    g.transposed = (L.mode == HELM_CONV_T1 || L.mode == HELM_CONV_T2) ? 1 : 0;
    if (grad[L.in]) {
      const long nw = static_cast<long>(g.taps) * g.Co * g.Ci;
      HELM_LAUNCH("k_pack_dgrad_w", st, k_pack_dgrad_w<<<gridn(nw), 256, 0, st>>>(g, PP(c, L.wparam), T.wpart));
      if (in.C % 8 == 0) {
        const long nin = static_cast<long>(in.B) * in.H * in.W * (in.C / 8);
        HELM_LAUNCH("k_conv_dgrad", st, k_conv_dgrad<<<gridn(nin), 256, 0, st>>>(g, T.dz, T.wpart, grad[L.in]));
      } else {
        const long nin = static_cast<long>(in.B) * in.H * in.W * in.C;
        HELM_LAUNCH("k_conv_dgrad_narrow", st,
                    k_conv_dgrad_narrow<<<gridn(nin), 256, 0, st>>>(g, T.dz, T.wpart, grad[L.in]));
      }
    }
    const int nch = div_up(P, WG_PIX);
    if (static_cast<size_t>(nch) * g.taps * g.Co * g.Ci > T.wpart_elems) {
      set_error("cnn training: weight-gradient partials exceed the workspace");
      return HELM_ESHAPE;
    }
    {
      const bf16* xin = static_cast<const bf16*>(ptr[L.in]);
      const int tco = g.Co >= 64 ? 64 : (g.Co >= 32 ? 32 : 16);
      const int tci = g.Ci >= 64 ? 64 : (g.Ci >= 32 ? 32 : 16);
      if (tco == 64 && tci == 64) HELM_LAUNCH("k_conv_wgrad", st, launch_wgrad<64, 64>(g, xin, T.dz, T.wpart, nch, st));
      else if (tco == 64 && tci == 32) HELM_LAUNCH("k_conv_wgrad", st, launch_wgrad<64, 32>(g, xin, T.dz, T.wpart, nch, st));
      else if (tco == 32 && tci == 64) HELM_LAUNCH("k_conv_wgrad", st, launch_wgrad<32, 64>(g, xin, T.dz, T.wpart, nch, st));
      else if (tco == 32 && tci == 32) HELM_LAUNCH("k_conv_wgrad", st, launch_wgrad<32, 32>(g, xin, T.dz, T.wpart, nch, st));
      else if (tco == 64) HELM_LAUNCH("k_conv_wgrad", st, launch_wgrad<64, 16>(g, xin, T.dz, T.wpart, nch, st));
      else if (tci == 64) HELM_LAUNCH("k_conv_wgrad", st, launch_wgrad<16, 64>(g, xin, T.dz, T.wpart, nch, st));
      else if (tco == 32) HELM_LAUNCH("k_conv_wgrad", st, launch_wgrad<32, 16>(g, xin, T.dz, T.wpart, nch, st));
      else if (tci == 32) HELM_LAUNCH("k_conv_wgrad", st, launch_wgrad<16, 32>(g, xin, T.dz, T.wpart, nch, st));
      else HELM_LAUNCH("k_conv_wgrad", st, launch_wgrad<16, 16>(g, xin, T.dz, T.wpart, nch, st));
    }
    HELM_LAUNCH("k_wgrad_reduce", st,
                k_wgrad_reduce<<<gridn(static_cast<long>(g.taps) * g.Co * g.Ci), 256, 0, st>>>(
                    g, T.wpart, nch, gparams + c->params[L.wparam].offset));
    HELM_CHECK_LAUNCH("conv backward");
  }
  return HELM_OK;
}

int cnn_backward(helm_cnn* c, const helm_problem* p, const float2* r, const float2* ge, float2* grad_r,
                 float* gparams, int B, Carve& cv, cudaStream_t st) {
  const int I = p->nx;
  if (c->train_nprob < 1) {
    set_error("cnn backward: no training forward to differentiate");
    return HELM_ESTATE;
  }
  TrainState T;
  carve_train(c, I, B, c->train_nprob, cv, &T, true);
  if (T.overflow) {
    set_error("cnn backward: workspace too small");
    return HELM_EWORKSPACE;
  }
  if (grad_r) T.sgrad[T.x0] = T.gx0;   // the network input's gradient is needed too
  // zero the activation gradients and the parameter gradients
  for (size_t i = 0; i < T.egrad.size(); ++i)
    if (T.egrad[i])
      HELM_CUDA(cudaMemsetAsync(T.egrad[i], 0,
                                static_cast<size_t>(T.enc.t[i].B) * T.enc.t[i].H * T.enc.t[i].W * T.enc.t[i].C * 4, st));
  for (size_t i = 0; i < T.sgrad.size(); ++i)
    if (T.sgrad[i])
      HELM_CUDA(cudaMemsetAsync(T.sgrad[i], 0,
                                static_cast<size_t>(T.sol.t[i].B) * T.sol.t[i].H * T.sol.t[i].W * T.sol.t[i].C * 4, st));
  HELM_CUDA(cudaMemsetAsync(gparams, 0, c->nparams * sizeof(float), st));
  // solver output: projection + P
  {
    const int Nc = I / 2, C = T.sol.t[T.u3].C;
    const ParamInfo& pw = c->params[c->pidx.at("s.proj.w")];
    const ParamInfo& pb = c->params[c->pidx.at("s.proj.b")];
    const long tot = static_cast<long>(B) * Nc * Nc;
    const int nblk = std::min<int>(kMaxChunks, gridn(tot));
    HELM_LAUNCH("k_proj_bwd", st,
                k_proj_bwd<<<nblk, 256, 0, st>>>(ge, static_cast<const bf16*>(T.sptr[T.u3]),
                                                                         B, Nc, C, c->params_dev + pw.offset, T.s,
                                                                         T.sgrad[T.u3], T.ppart));
    HELM_LAUNCH("k_strided_reduce", st,
                k_strided_reduce<<<1, 64, 0, st>>>(T.ppart, nblk, 2 * C + 2, 0, 2 * C, gparams + pw.offset));
    HELM_LAUNCH("k_strided_reduce", st,
                k_strided_reduce<<<1, 32, 0, st>>>(T.ppart, nblk, 2 * C + 2, 2 * C, 2, gparams + pb.offset));
    HELM_CHECK_LAUNCH("proj backward");
  }
  // the solver accumulates the encodings' gradients directly into the encoder's
  // output-tensor gradients (aliased in carve_train), then the encoder runs backward
  int rc = run_layers_backward(c, T.sol, T, T.sptr, T.sraw, T.smean, T.sistd, T.sgrad, gparams, st);
  if (rc) return rc;
  if (grad_r) {
    const long n = static_cast<long>(I) * I;
    const int nblk = std::max(1, std::min(128, div_up(n, 8192)));
    HELM_LAUNCH("k_gradr_t", st, k_gradr_t<<<gridn(static_cast<long>(B) * n), 256, 0, st>>>(T.gx0, I, B, T.s, grad_r));
    HELM_LAUNCH("k_gradr_dots", st,
                k_gradr_dots<<<dim3(nblk, B), 256, 0, st>>>(ge, T.esave, grad_r, r, n, nblk, T.part));
    HELM_LAUNCH("k_gradr_fix", st,
                k_gradr_fix<<<dim3(std::min<long>(div_up(n, 256), 512), B), 256, 0, st>>>(T.part, nblk, T.s, n, r,
                                                                                          grad_r));
    HELM_CHECK_LAUNCH("input gradient");
  }
  return run_layers_backward(c, T.enc, T, T.eptr, T.eraw, T.emean, T.eistd, T.egrad, gparams, st);
}

}  // namespace helm

extern "C" {

int helm_cnn_train_workspace_size(const helm_problem* p, const helm_cnn* c, int batch, int nprob, size_t* bytes) {
  if (!p || !c || !bytes || batch <= 0 || nprob < 1) {
    helm::set_error("helm_cnn_train_workspace_size: invalid argument");
    return HELM_EINVAL;
  }
  *bytes = helm::cnn_train_bytes(c, p->nx, batch, nprob);
  return HELM_OK;
}

int helm_cnn_train_forward(const helm_problem* const* probs, int nprob, helm_cnn* c, const void* r, void* e,
                           int batch, void* ws, size_t ws_bytes, void* stream) {
  if (!probs || nprob < 1 || !c || !r || !e || batch <= 0 || !ws) {
    helm::set_error("helm_cnn_train_forward: invalid argument");
    return HELM_EINVAL;
  }
  for (int k = 0; k < nprob; ++k)
    if (!probs[k]) {
      helm::set_error("helm_cnn_train_forward: null problem %d", k);
      return HELM_EINVAL;
    }
  helm::Carve cv(ws, ws_bytes);
  return helm::cnn_forward_train(c, probs, nprob, static_cast<const float2*>(r), static_cast<float2*>(e), batch, cv,
                                 static_cast<cudaStream_t>(stream));
}

int helm_cnn_precond_backward(const helm_problem* p, helm_cnn* c, const void* r, const void* grad_e, void* grad_r,
                              float* grad_params, int batch, void* ws, size_t ws_bytes, void* stream) {
  if (!p || !c || !grad_e || !grad_params || batch <= 0 || !ws || (grad_r && (!r || r == grad_r))) {
    helm::set_error("helm_cnn_precond_backward: invalid argument (grad_r needs the forward's input r, distinct)");
    return HELM_EINVAL;
  }
  helm::Carve cv(ws, ws_bytes);
  return helm::cnn_backward(c, p, static_cast<const float2*>(r), static_cast<const float2*>(grad_e),
                            static_cast<float2*>(grad_r), grad_params, batch, cv, static_cast<cudaStream_t>(stream));
}

int helm_mse_loss(const void* e_pred, const void* e_true, long n, int batch, double* loss_dev, void* grad,
                  void* ws, void* stream) {
  if (!e_pred || !e_true || n <= 0 || batch <= 0 || !loss_dev || !ws) {
    helm::set_error("helm_mse_loss: invalid argument");
    return HELM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* part = static_cast<double*>(ws);
  const int nblk = 512;
  HELM_LAUNCH("k_mse", st,
              helm::k_mse<<<nblk, 256, 0, st>>>(static_cast<const float2*>(e_pred), static_cast<const float2*>(e_true), n,
                                                batch, static_cast<float2*>(grad), part));
  HELM_LAUNCH("k_mse_final", st, helm::k_mse_final<<<1, 256, 0, st>>>(part, nblk, batch, loss_dev));
  HELM_CHECK_LAUNCH("mse");
  return HELM_OK;
}

int helm_adam_step(float* params, const float* grads, float* m, float* v, long n, double lr, double beta1,
                   double beta2, double eps, int step, void* stream) {
  if (!params || !grads || !m || !v || n <= 0 || step < 1) {
    helm::set_error("helm_adam_step: invalid argument");
    return HELM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const float c1 = static_cast<float>(1.0 - std::pow(beta1, step));
  const float c2 = static_cast<float>(1.0 - std::pow(beta2, step));
  HELM_LAUNCH("k_adam", st,
              helm::k_adam<<<std::min<long>(helm::div_up(n, 256), 4096), 256, 0, st>>>(
                  params, grads, m, v, n, static_cast<float>(lr), static_cast<float>(beta1),
                  static_cast<float>(beta2), static_cast<float>(eps), c1, c2));
  HELM_CHECK_LAUNCH("adam");
  return HELM_OK;
}

}  // extern "C"
