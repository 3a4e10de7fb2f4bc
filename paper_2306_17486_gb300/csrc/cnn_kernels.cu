// CUDA-core kernels of the encoder-solver network (forward): encoder input
// features, residual normalisation and fixed restriction, depthwise 3x3, the
// implicit layer (Eq. 14) in shared memory, the Green's function of a learned kernel
// (Eq. 15), and the projection + bilinear upsampling that ends the solver.
#include <cuda_bf16.h>

#include "cnn_kern.h"

namespace helm {

using bf16 = __nv_bfloat16;

// ---- encoder input: (Re, Im) of kappa^2 (1 - gamma i) ------------------------------
__global__ void k_kfeat(const float* __restrict__ kappa, const float* __restrict__ gamma, long n,
                        bf16* __restrict__ out) {
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const float k2 = kappa[i] * kappa[i];
    out[2 * i] = __float2bfloat16_rn(k2);
    out[2 * i + 1] = __float2bfloat16_rn(-k2 * gamma[i]);
  }
}

// ---- ||r_b||^2 partial sums and the input scale s_b = RMS(r_b) -------------------
__global__ void k_norm_partial(const float2* __restrict__ r, long n, int nblk, double* __restrict__ part) {
  const int b = blockIdx.y;
  const long chunk = (n + nblk - 1) / nblk;
  const long p0 = blockIdx.x * chunk, p1 = min(p0 + chunk, n);
  // FP32 per thread (a few dozen terms; FP64 arithmetic is slow on this part), FP64
  // across threads and blocks
  float accf = 0.f;
  for (long p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const float2 v = r[b * n + p];
    accf = fmaf(v.x, v.x, fmaf(v.y, v.y, accf));
  }
  double acc = warp_sum(static_cast<double>(accf));
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (blockDim.x >> 5); ++w) t += red[w];
    part[static_cast<long>(b) * nblk + blockIdx.x] = t;
  }
}

// s_b = RMS of r_b over the grid (the network's input scale; the paper leaves it unstated)
__global__ void k_norm_final(const double* __restrict__ part, int nblk, int B, long n, float* __restrict__ s,
                             float* __restrict__ inv) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double t = 0;
  for (int i = 0; i < nblk; ++i) t += part[static_cast<long>(b) * nblk + i];
  const double v = sqrt(t / static_cast<double>(n));
  s[b] = static_cast<float>(v);
  inv[b] = v > 0.0 ? static_cast<float>(1.0 / v) : 0.f;
}

// x0[b][J][K][0..1] = (Re, Im) of I_h^H (r_b / s_b): full weighting, zero padding
// (s_b the RMS of r_b)
__global__ void k_prep_restrict(const float2* __restrict__ r, int Ny, int Nx, int B, const float* __restrict__ inv,
                                bf16* __restrict__ x0) {
  const int Ncy = Ny / 2, Ncx = Nx / 2;
  const long total = static_cast<long>(B) * Ncy * Ncx;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const int b = static_cast<int>(i / (static_cast<long>(Ncy) * Ncx));
    const int J = static_cast<int>((i / Ncx) % Ncy), K = static_cast<int>(i % Ncx);
    const float2* rb = r + static_cast<long>(b) * Ny * Nx;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = -1; a <= 1; ++a)
#pragma unroll
      for (int c = -1; c <= 1; ++c) {
        const int y = 2 * J + a, x = 2 * K + c;
        if (y < 0 || y >= Ny || x < 0 || x >= Nx) continue;
        const float w = (a == 0 ? 2.f : 1.f) * (c == 0 ? 2.f : 1.f) * (1.f / 16.f);
        const float2 v = rb[static_cast<long>(y) * Nx + x];
        acc.x += w * v.x;
        acc.y += w * v.y;
      }
    const float sc = inv[b];
    x0[2 * i] = __float2bfloat16_rn(acc.x * sc);
    x0[2 * i + 1] = __float2bfloat16_rn(acc.y * sc);
  }
}

// ---- depthwise 3x3 (stride 1, zero padding): thread per (pixel, 8-channel group) ----
// y = act(scale * acc + shift) (bf16) and/or the raw accumulator (fp32).  Weights and
// the per-channel affine are staged in shared memory once per CTA.
constexpr int DW_MAXC = 384;
__global__ void __launch_bounds__(256) k_dw3x3(const bf16* __restrict__ x, int B, int H, int W, int C,
                                               const float* __restrict__ w, const float* __restrict__ scale,
                                               const float* __restrict__ shift, int act, bf16* __restrict__ y,
                                               float* __restrict__ yraw) {
  __shared__ float sw[9][DW_MAXC];
  __shared__ float ssc[DW_MAXC], ssh[DW_MAXC];
  for (int i = threadIdx.x; i < C * 9; i += blockDim.x) sw[i % 9][i / 9] = w[i];
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    ssc[c] = scale ? scale[c] : 1.f;
    ssh[c] = shift ? shift[c] : 0.f;
  }
  __syncthreads();
  const int G = C / 8;
  const long total = static_cast<long>(B) * H * W * G;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const int g = static_cast<int>(i % G);
    const long pix = i / G;
    const int xx = static_cast<int>(pix % W), yy = static_cast<int>((pix / W) % H);
    const int b = static_cast<int>(pix / (static_cast<long>(W) * H));
    float acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = 0.f;
#pragma unroll
    for (int ty = 0; ty < 3; ++ty) {
      const int sy = yy + ty - 1;
      if (sy < 0 || sy >= H) continue;
#pragma unroll
      for (int tx = 0; tx < 3; ++tx) {
        const int sx = xx + tx - 1;
        if (sx < 0 || sx >= W) continue;
        uint4 u = *reinterpret_cast<const uint4*>(x + ((static_cast<long>(b) * H + sy) * W + sx) * C + 8 * g);
        const bf16* e8 = reinterpret_cast<const bf16*>(&u);
        const float* wt = &sw[ty * 3 + tx][8 * g];
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[e] = fmaf(wt[e], __bfloat162float(e8[e]), acc[e]);
      }
    }
    if (yraw) {
      float4* o = reinterpret_cast<float4*>(yraw + pix * C + 8 * g);
      o[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
      o[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
    }
    if (y) {
      uint4 o;
      bf16* ob = reinterpret_cast<bf16*>(&o);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int c = 8 * g + e;
        float t = fmaf(acc[e], ssc[c], ssh[c]);
        if (act) t = fmaxf(t, 0.f) + log1pf(__expf(-fabsf(t)));
        ob[e] = __float2bfloat16_rn(t);
      }
      *reinterpret_cast<uint4*>(y + pix * C + 8 * g) = o;
    }
  }
}

// Depthwise 3x3 for the expanded widths of the inverted bottlenecks (C = 6 c), one CTA
// per output row: thread (strip, g) holds the 72 weights of channel group g in registers
// and slides along a strip of DW_XS pixels, so each input vector is loaded once per
// row of taps and reused by up to three outputs.
constexpr int DW_XS = 4;
template <int C>
__global__ void __launch_bounds__(256) k_dw3x3_row(const bf16* __restrict__ x, int H, int W,
                                                   const float* __restrict__ w, const float* __restrict__ scale,
                                                   const float* __restrict__ shift, int act, bf16* __restrict__ y,
                                                   float* __restrict__ yraw) {
  constexpr int G = C / 8;
  __shared__ float4 sw[9][C / 4];
  __shared__ float ssc[C], ssh[C];
  float* swf = reinterpret_cast<float*>(sw);
  for (int i = threadIdx.x; i < C * 9; i += blockDim.x) swf[(i % 9) * C + i / 9] = w[i];
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    ssc[c] = scale ? scale[c] : 1.f;
    ssh[c] = shift ? shift[c] : 0.f;
  }
  __syncthreads();
  const int row = blockIdx.y;                 // b * H + yy
  const int yy = row % H;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nstrip = (W + DW_XS - 1) / DW_XS;
  if (t >= nstrip * G) return;
  const int g = t % G, x0 = (t / G) * DW_XS;
  float wr[9][8];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float4 lo = sw[k][2 * g], hi = sw[k][2 * g + 1];
    wr[k][0] = lo.x; wr[k][1] = lo.y; wr[k][2] = lo.z; wr[k][3] = lo.w;
    wr[k][4] = hi.x; wr[k][5] = hi.y; wr[k][6] = hi.z; wr[k][7] = hi.w;
  }
  float acc[DW_XS][8];
#pragma unroll
  for (int o = 0; o < DW_XS; ++o)
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[o][e] = 0.f;
#pragma unroll
  for (int ty = 0; ty < 3; ++ty) {
    const int sy = yy + ty - 1;
    if (sy < 0 || sy >= H) continue;
    const bf16* rp = x + (static_cast<long>(row + ty - 1) * W) * C + 8 * g;
#pragma unroll
    for (int c = 0; c < DW_XS + 2; ++c) {
      const int sx = x0 + c - 1;
      if (sx < 0 || sx >= W) continue;
      const uint4 u = __ldg(reinterpret_cast<const uint4*>(rp + static_cast<long>(sx) * C));
      const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&u);
      float f[8];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 v = __bfloat1622float2(h2[e]);
        f[2 * e] = v.x;
        f[2 * e + 1] = v.y;
      }
#pragma unroll
      for (int tx = 0; tx < 3; ++tx) {
        const int o = c - tx;   // output strip position that this tap of this column feeds
        if (o < 0 || o >= DW_XS) continue;
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[o][e] = fmaf(wr[ty * 3 + tx][e], f[e], acc[o][e]);
      }
    }
  }
#pragma unroll
  for (int o = 0; o < DW_XS; ++o) {
    const int xx = x0 + o;
    if (xx >= W) break;
    const long pix = static_cast<long>(row) * W + xx;
    if (yraw) {
      float4* op = reinterpret_cast<float4*>(yraw + pix * C + 8 * g);
      op[0] = make_float4(acc[o][0], acc[o][1], acc[o][2], acc[o][3]);
      op[1] = make_float4(acc[o][4], acc[o][5], acc[o][6], acc[o][7]);
    }
    if (y) {
      uint4 u;
      __nv_bfloat162* ob = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = 8 * g + 2 * e;
        float t0 = fmaf(acc[o][2 * e], ssc[c], ssh[c]);
        float t1 = fmaf(acc[o][2 * e + 1], ssc[c + 1], ssh[c + 1]);
        if (act) {
          t0 = fmaxf(t0, 0.f) + __logf(1.f + __expf(-fabsf(t0)));
          t1 = fmaxf(t1, 0.f) + __logf(1.f + __expf(-fabsf(t1)));
        }
        ob[e] = __floats2bfloat162_rn(t0, t1);
      }
      *reinterpret_cast<uint4*>(y + pix * C + 8 * g) = u;
    }
  }
}

// ---- implicit layer (Eq. 14), one CTA per (sample, complex channel) -----------------
// x: channels k (Re) and k + C/2 (Im) of an m x m map; zero-pad to 2m x 2m, DFT,
// multiply by G_hat_k, inverse DFT, keep the top-left m x m block.
template <typename TIn>
__device__ __forceinline__ float2 load_pair(const TIn* p, long idx, int C, int k) {
  return make_float2(static_cast<float>(p[idx * C + k]), static_cast<float>(p[idx * C + k + C / 2]));
}
template <>
__device__ __forceinline__ float2 load_pair<bf16>(const bf16* p, long idx, int C, int k) {
  return make_float2(__bfloat162float(p[idx * C + k]), __bfloat162float(p[idx * C + k + C / 2]));
}

// The 2m_y x 2m_x transforms of the implicit layer (an m_y x m_x coarsest map; m_y = m_x
// = m on the paper's square grids) run as mixed-radix FFTs (Stockham autosort: every
// stage reads one buffer and writes the other in natural order, so no digit reversal is
// needed), batched over the lines of a phase and spread over the CTA's threads:
//   rows     R[r][.]  = FFT(pad(X[r][.]))                     r < m_y, length 2m_x
//   columns  R[.][u]  = IFFT(G_hat[.][u] . FFT(pad(R[.][u])))  length 2m_y, kept for r < m_y
//   rows     Y[r][c]  = IFFT(R[r][.])[c] / (4 m_y m_x)         r < m_y, c < m_x
// Each phase runs in chunks of cw lines, so that shared memory holds R (m_y x 2m_x) and
// two line buffers of cw lines of the longer length.
// Each length is factored into radices 8, 9, 4, 2, 3, 5 (8 and 9 as in-register 4 x 2 and
// 3 x 3 decompositions) and any other prime up to FFT_PMAX (direct DFT of that size);
// twiddles come from one table per length, W[e] = exp(-2 pi i e / n) (one shared table
// when the two lengths are equal).
constexpr int FFT_MAXF = 16;
constexpr int FFT_PMAX = 17;
struct FftPlan {
  int nf;              // stages
  int f[FFT_MAXF];     // radix of each stage
};

__device__ __forceinline__ float2 tw(const float2* Wt, int e, bool inv) {
  const float2 w = Wt[e];
  return inv ? make_float2(w.x, -w.y) : w;
}
// multiply by -i (forward) or +i (inverse)
__device__ __forceinline__ float2 rot_i(float2 v, bool inv) {
  return inv ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
}
// length-4 DFT in place (forward: W4 = -i)
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3, bool inv) {
  const float2 a0 = cadd(x0, x2), a1 = csub(x0, x2), b0 = cadd(x1, x3), b1 = rot_i(csub(x1, x3), inv);
  x0 = cadd(a0, b0);
  x1 = cadd(a1, b1);
  x2 = csub(a0, b0);
  x3 = csub(a1, b1);
}
// length-3 DFT in place (forward: W3 = exp(-2 pi i / 3))
__device__ __forceinline__ void dft3(float2& x0, float2& x1, float2& x2, bool inv) {
  const float2 t1 = cadd(x1, x2);
  const float2 t2 = make_float2(x0.x - 0.5f * t1.x, x0.y - 0.5f * t1.y);
  // sqrt(3)/2 (x1 - x2) turned by -i (forward) or +i (inverse)
  const float2 t3 = rot_i(cscale(csub(x1, x2), 0.86602540378443865f), inv);
  x0 = cadd(x0, t1);
  x1 = cadd(t2, t3);
  x2 = csub(t2, t3);
}

// One Stockham stage of radix p over L lines of length n: butterfly j of a line reads
// x[j + r n/p] (r < p), multiplies input r by W_n^(k r n/(Ns p)) with k = j mod Ns, takes
// the length-p DFT and writes output r to y[(j / Ns) Ns p + k + r Ns].
__device__ void fft_stage(const float2* __restrict__ src, float2* __restrict__ dst, int L, int n, int p, int Ns,
                          const float2* __restrict__ Wt, bool inv) {
  const int q = n / p;                 // butterflies per line
  const int tws = n / (Ns * p);        // twiddle index step per unit of k r
  const int total = L * q;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int line = t / q, j = t - line * q;
    const float2* s = src + static_cast<long>(line) * n + j;
    const int k = j % Ns;
    float2* d = dst + static_cast<long>(line) * n + (j / Ns) * Ns * p + k;
    const int ek = k * tws;            // twiddle index of input 1; input r takes r ek (< n)
    if (p == 8) {
      // two length-4 DFTs of the even and odd inputs, then W8^k on the odd half
      float2 v[8];
      v[0] = s[0];
#pragma unroll
      for (int r = 1; r < 8; ++r) v[r] = cmul(s[r * q], tw(Wt, r * ek, inv));
      dft4(v[0], v[2], v[4], v[6], inv);
      dft4(v[1], v[3], v[5], v[7], inv);
      const float h = 0.70710678118654752f;
      const float2 o1 = cscale(cadd(v[3], rot_i(v[3], inv)), h);       // W8^1 = (1 -+ i)/sqrt(2)
      const float2 o2 = rot_i(v[5], inv);                               // W8^2 = -+ i
      const float2 o3 = cscale(csub(rot_i(v[7], inv), v[7]), h);       // W8^3 = (-1 -+ i)/sqrt(2)
      d[0] = cadd(v[0], v[1]);
      d[4 * Ns] = csub(v[0], v[1]);
      d[Ns] = cadd(v[2], o1);
      d[5 * Ns] = csub(v[2], o1);
      d[2 * Ns] = cadd(v[4], o2);
      d[6 * Ns] = csub(v[4], o2);
      d[3 * Ns] = cadd(v[6], o3);
      d[7 * Ns] = csub(v[6], o3);
    } else if (p == 9) {
      // 3 x 3: length-3 DFTs over n1 for each n2, twiddles W9^(n2 k1), length-3 DFTs over n2
      float2 v[9];
      v[0] = s[0];
#pragma unroll
      for (int r = 1; r < 9; ++r) v[r] = cmul(s[r * q], tw(Wt, r * ek, inv));
#pragma unroll
      for (int n2 = 0; n2 < 3; ++n2) dft3(v[n2], v[3 + n2], v[6 + n2], inv);
      const int e9 = n / 9;
      v[4] = cmul(v[4], tw(Wt, e9, inv));        // n2 = 1, k1 = 1
      v[7] = cmul(v[7], tw(Wt, 2 * e9, inv));    // n2 = 1, k1 = 2
      v[5] = cmul(v[5], tw(Wt, 2 * e9, inv));    // n2 = 2, k1 = 1
      v[8] = cmul(v[8], tw(Wt, 4 * e9, inv));    // n2 = 2, k1 = 2
#pragma unroll
      for (int k1 = 0; k1 < 3; ++k1) {
        dft3(v[3 * k1], v[3 * k1 + 1], v[3 * k1 + 2], inv);
        d[k1 * Ns] = v[3 * k1];
        d[(k1 + 3) * Ns] = v[3 * k1 + 1];
        d[(k1 + 6) * Ns] = v[3 * k1 + 2];
      }
    } else if (p == 4) {
      float2 v0 = s[0], v1 = cmul(s[q], tw(Wt, ek, inv)), v2 = cmul(s[2 * q], tw(Wt, 2 * ek, inv)),
             v3 = cmul(s[3 * q], tw(Wt, 3 * ek, inv));
      dft4(v0, v1, v2, v3, inv);
      d[0] = v0;
      d[Ns] = v1;
      d[2 * Ns] = v2;
      d[3 * Ns] = v3;
    } else if (p == 2) {
      const float2 v0 = s[0], v1 = cmul(s[q], tw(Wt, ek, inv));
      d[0] = cadd(v0, v1);
      d[Ns] = csub(v0, v1);
    } else if (p == 3) {
      float2 v0 = s[0], v1 = cmul(s[q], tw(Wt, ek, inv)), v2 = cmul(s[2 * q], tw(Wt, 2 * ek, inv));
      dft3(v0, v1, v2, inv);
      d[0] = v0;
      d[Ns] = v1;
      d[2 * Ns] = v2;
    } else {
      // any other radix: direct DFT of length p with W_p^(a b) = W_n^((a b mod p) q)
      float2 v[FFT_PMAX];
      for (int r = 0; r < p; ++r) v[r] = r ? cmul(s[r * q], tw(Wt, r * ek, inv)) : s[0];
      for (int a = 0; a < p; ++a) {
        float2 acc = v[0];
        for (int r = 1; r < p; ++r) acc = cadd(acc, cmul(v[r], tw(Wt, ((a * r) % p) * q, inv)));
        d[a * Ns] = acc;
      }
    }
  }
}

// All stages over L lines, ping-ponging between a and b; returns the buffer holding the
// result.  Callers synchronise the CTA before the first stage.
__device__ float2* fft_lines(float2* a, float2* b, int L, int n, const FftPlan& plan, const float2* Wt, bool inv) {
  int Ns = 1;
  for (int s = 0; s < plan.nf; ++s) {
    fft_stage(a, b, L, n, plan.f[s], Ns, Wt, inv);
    __syncthreads();
    Ns *= plan.f[s];
    float2* t = a;
    a = b;
    b = t;
  }
  return a;
}

// Eq. 14 for one (sample b, complex channel k) of an m_y x m_x map:
// y = crop(IFFT(G_hat_k . FFT(pad(x)))), or with conj_g the adjoint (conj(G_hat_k));
// accumulate adds into y (FP32 output only).  G_hat_k is [2m_y][2m_x].
// Registers are capped so that three CTAs share an SM at m = 36 (62.8 KB each).
template <typename TIn, typename TOut>
__global__ void __launch_bounds__(256, 3) k_implicit(const TIn* __restrict__ x, int my, int mx, int C,
                                                  const float2* __restrict__ ghat, int conj_g, TOut* __restrict__ y,
                                                  int accumulate, int cw, FftPlan planx, FftPlan plany) {
  const int b = blockIdx.y, k = blockIdx.x;
  const int nx = 2 * mx, ny = 2 * my;      // row and column lengths of the padded map
  const int nl = max(nx, ny);
  extern __shared__ float2 ism[];
  float2* Wx = ism;                          // nx
  float2* Wy = ny == nx ? Wx : Wx + nx;      // ny (the same table on a square map)
  float2* R = Wx + nx + (ny == nx ? 0 : ny); // m_y x nx: the rows' spectra, later the columns' results
  float2* P0 = R + my * nx;                  // cw x nl ping-pong buffers of the line transforms
  float2* P1 = P0 + cw * nl;
  for (int e = threadIdx.x; e < nx; e += blockDim.x) {
    float s, c;
    sincospif(-2.f * e / nx, &s, &c);
    Wx[e] = make_float2(c, s);
  }
  if (ny != nx)
    for (int e = threadIdx.x; e < ny; e += blockDim.x) {
      float s, c;
      sincospif(-2.f * e / ny, &s, &c);
      Wy[e] = make_float2(c, s);
    }
  const long base = static_cast<long>(b) * my * mx;
  for (int r0 = 0; r0 < my; r0 += cw) {
    const int w = min(cw, my - r0);
    for (int i = threadIdx.x; i < w * nx; i += blockDim.x) {
      const int r = i / nx, c = i - r * nx;
      P0[i] = c < mx ? load_pair<TIn>(x, base + (r0 + r) * mx + c, C, k) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2* rs = fft_lines(P0, P1, w, nx, planx, Wx, false);
    for (int i = threadIdx.x; i < w * nx; i += blockDim.x) R[r0 * nx + i] = rs[i];
    __syncthreads();
  }
  const float2* G = ghat + static_cast<long>(k) * ny * nx;
  for (int u0 = 0; u0 < nx; u0 += cw) {
    const int w = min(cw, nx - u0);
    for (int i = threadIdx.x; i < w * ny; i += blockDim.x) {
      const int l = i / ny, v = i - l * ny;
      P0[i] = v < my ? R[v * nx + u0 + l] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* fs = fft_lines(P0, P1, w, ny, plany, Wy, false);
    for (int i = threadIdx.x; i < w * ny; i += blockDim.x) {
      const int l = i / ny, v = i - l * ny;
      float2 g = G[static_cast<long>(v) * nx + u0 + l];
      if (conj_g) g.y = -g.y;
      fs[i] = cmul(fs[i], g);
    }
    __syncthreads();
    const float2* is = fft_lines(fs, fs == P0 ? P1 : P0, w, ny, plany, Wy, true);
    for (int i = threadIdx.x; i < w * my; i += blockDim.x) {
      const int l = i / my, v = i - l * my;
      R[v * nx + u0 + l] = is[l * ny + v];
    }
    __syncthreads();
  }
  const float sc = 1.f / static_cast<float>(nx * ny);
  for (int r0 = 0; r0 < my; r0 += cw) {
    const int w = min(cw, my - r0);
    // the chunk's rows of R are consumed here, so they serve as one of the two buffers
    const float2* ys = fft_lines(R + r0 * nx, P0, w, nx, planx, Wx, true);
    for (int i = threadIdx.x; i < w * mx; i += blockDim.x) {
      const int r = i / mx, c = i - r * mx;
      const float2 v = cscale(ys[r * nx + c], sc);
      const long idx = (base + (r0 + r) * mx + c) * C;
      if constexpr (sizeof(TOut) == 2) {
        y[idx + k] = __float2bfloat16_rn(v.x);
        y[idx + k + C / 2] = __float2bfloat16_rn(v.y);
      } else {
        if (accumulate) {
          y[idx + k] += v.x;
          y[idx + k + C / 2] += v.y;
        } else {
          y[idx + k] = v.x;
          y[idx + k + C / 2] = v.y;
        }
      }
    }
    __syncthreads();
  }
}

// The same layer in three passes through a global intermediate Rg [B][C/2][m_y][2m_x]
// (complex), for maps whose m_y x 2m_x intermediate exceeds a CTA's shared memory.
// blockIdx = (complex channel k, sample b, chunk of cw lines):
//   pass 0  rows r0..r0+cw of the zero-padded input: FFT (length 2m_x) -> Rg
//   pass 1  columns u0..u0+cw of Rg: FFT (length 2m_y, rows >= m_y zero), times G_hat,
//           inverse FFT, rows < m_y back into Rg
//   pass 2  rows r0..r0+cw of Rg: inverse FFT, scale 1/(4 m_y m_x), crop to m_x -> y
// Shared memory: the pass's twiddle table (n) and two cw x n line buffers.
template <typename TIn, typename TOut>
__global__ void __launch_bounds__(256) k_implicit_pass(const TIn* __restrict__ x, int my, int mx, int C,
                                                       const float2* __restrict__ ghat, int conj_g,
                                                       float2* __restrict__ Rg, TOut* __restrict__ y, int accumulate,
                                                       int pass, int cw, FftPlan plan) {
  const int k = blockIdx.x, b = blockIdx.y, nk = C / 2;
  const int nx = 2 * mx, ny = 2 * my;
  const int n = pass == 1 ? ny : nx;        // line length of this pass
  const int lines = pass == 1 ? nx : my;
  const int l0 = blockIdx.z * cw;
  if (l0 >= lines) return;
  const int w = min(cw, lines - l0);
  extern __shared__ float2 ism[];
  float2* Wt = ism;
  float2* P0 = Wt + n;
  float2* P1 = P0 + cw * n;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    float s, c;
    sincospif(-2.f * e / n, &s, &c);
    Wt[e] = make_float2(c, s);
  }
  float2* Rb = Rg + (static_cast<long>(b) * nk + k) * my * nx;   // this (sample, channel)'s m_y x 2m_x block
  if (pass == 0) {
    const long base = static_cast<long>(b) * my * mx;
    for (int i = threadIdx.x; i < w * nx; i += blockDim.x) {
      const int r = i / nx, c = i - r * nx;
      P0[i] = c < mx ? load_pair<TIn>(x, base + static_cast<long>(l0 + r) * mx + c, C, k) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2* rs = fft_lines(P0, P1, w, nx, plan, Wt, false);
    for (int i = threadIdx.x; i < w * nx; i += blockDim.x) Rb[static_cast<long>(l0) * nx + i] = rs[i];
  } else if (pass == 1) {
    // column l of the chunk is column l0 + l of Rb; consecutive threads take consecutive
    // columns of one row, so the global reads and writes are contiguous runs of w
    for (int i = threadIdx.x; i < w * ny; i += blockDim.x) {
      const int v = i / w, l = i - v * w;
      P0[l * ny + v] = v < my ? Rb[static_cast<long>(v) * nx + l0 + l] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* fs = fft_lines(P0, P1, w, ny, plan, Wt, false);
    const float2* G = ghat + static_cast<long>(k) * ny * nx;
    for (int i = threadIdx.x; i < w * ny; i += blockDim.x) {
      const int v = i / w, l = i - v * w;
      float2 g = G[static_cast<long>(v) * nx + l0 + l];
      if (conj_g) g.y = -g.y;
      fs[l * ny + v] = cmul(fs[l * ny + v], g);
    }
    __syncthreads();
    const float2* is = fft_lines(fs, fs == P0 ? P1 : P0, w, ny, plan, Wt, true);
    for (int i = threadIdx.x; i < w * my; i += blockDim.x) {
      const int v = i / w, l = i - v * w;
      Rb[static_cast<long>(v) * nx + l0 + l] = is[l * ny + v];
    }
  } else {
    for (int i = threadIdx.x; i < w * nx; i += blockDim.x) P0[i] = Rb[static_cast<long>(l0) * nx + i];
    __syncthreads();
    const float2* ys = fft_lines(P0, P1, w, nx, plan, Wt, true);
    const float sc = 1.f / static_cast<float>(nx * ny);
    const long base = static_cast<long>(b) * my * mx;
    for (int i = threadIdx.x; i < w * mx; i += blockDim.x) {
      const int r = i / mx, c = i - r * mx;
      const float2 v = cscale(ys[r * nx + c], sc);
      const long idx = (base + static_cast<long>(l0 + r) * mx + c) * C;
      if constexpr (sizeof(TOut) == 2) {
        y[idx + k] = __float2bfloat16_rn(v.x);
        y[idx + k + C / 2] = __float2bfloat16_rn(v.y);
      } else {
        if (accumulate) {
          y[idx + k] += v.x;
          y[idx + k + C / 2] += v.y;
        } else {
          y[idx + k] = v.x;
          y[idx + k + C / 2] = v.y;
        }
      }
    }
  }
}

// Radices of n (8s first, then 9, 4, 2, 3, 5, other primes); false if a prime factor exceeds
// FFT_PMAX or there are too many stages.
static bool fft_plan(int n, FftPlan* p) {
  p->nf = 0;
  const int pref[] = {8, 9, 4, 2, 3, 5};
  for (int r : pref)
    while (n % r == 0) {
      if (p->nf == FFT_MAXF) return false;
      p->f[p->nf++] = r;
      n /= r;
    }
  for (int r = 7; n > 1; r += 2)
    while (n % r == 0) {
      if (r > FFT_PMAX || p->nf == FFT_MAXF) return false;
      p->f[p->nf++] = r;
      n /= r;
    }
  return true;
}

// shared memory of k_implicit on an m_y x m_x map with chunks of cw lines
static size_t implicit_chunk_smem(int my, int mx, int cw) {
  const size_t nx = 2 * mx, ny = 2 * my, nl = std::max(nx, ny);
  return (nx + (ny == nx ? 0 : ny) + my * nx + 2 * static_cast<size_t>(cw) * nl) * sizeof(float2);
}
// the widest chunk (in equal parts of the 2m_x columns) whose CTA fits 76 KB (three CTAs
// per SM), else 200 KB; 0 if none does
static int implicit_chunk(int my, int mx) {
  const int n = 2 * mx;
  for (size_t cap : {size_t(76) * 1024, size_t(200) * 1024})
    for (int parts = 1; parts <= n; ++parts) {
      const int cw = (n + parts - 1) / parts;
      if (implicit_chunk_smem(my, mx, cw) <= cap) return cw;
    }
  return 0;
}

// ---- Green's function of a learned 3x3 kernel (Eq. 15), one CTA per channel ---------
// Kpar: [2][nk][3][3] (real, imaginary parts).  An m_y x m_x coarsest map takes the
// 6m_y x 6m_x periodic grid, source at the centre: G at offsets (dy, dx) (|dy| <= m_y,
// |dx| <= m_x) is (1/(36 m_y m_x)) sum_{u,v} H(u,v) e^{+2 pi i (u dy / 6m_y + v dx / 6m_x)}
// with H = conj(Kh)/(|Kh|^2 + eps) (or Kh/(Kh^2 + eps)); crop to offsets -m..m-1 per axis
// with offset 0 at index 0, then G_hat = DFT_{2m_y x 2m_x}.
// scratch per channel: 6m_y*6m_x (H) + 6m_y*2m_x (T) + 2m_y*2m_x (Gc) complex.
__global__ void k_greens(const float* __restrict__ Kpar, int nk, int my, int mx, float eps, int literal,
                         float2* __restrict__ scratch, float2* __restrict__ ghat) {
  const int k = blockIdx.x;
  const int n6y = 6 * my, n6x = 6 * mx, ny = 2 * my, nx = 2 * mx;
  // the two axes' phases over one common period (the grid's point count when the axes
  // differ; one axis' length on a square grid)
  const bool sq = n6y == n6x;
  const int per = sq ? n6x : n6y * n6x;
  const int fy = sq ? 1 : n6x, fx = sq ? 1 : n6y;
  float2* H = scratch + static_cast<long>(k) * (n6y * n6x + n6y * nx + ny * nx);
  float2* T = H + n6y * n6x;
  float2* Gc = T + n6y * nx;
  float Kr[9], Ki[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    Kr[t] = Kpar[k * 9 + t];
    Ki[t] = Kpar[(nk + k) * 9 + t];
  }
  for (int i = threadIdx.x; i < n6y * n6x; i += blockDim.x) {
    const int u = i / n6x, v = i % n6x;
    float2 kh = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = -1; a <= 1; ++a)
#pragma unroll
      for (int c = -1; c <= 1; ++c) {
        float s, co;
        // exp(-2 pi i (u a / n6y + v c / n6x)), argument reduced mod the period in integers
        const int e = ((u * a * fy + v * c * fx) % per + per) % per;
        sincospif(-2.f * e / per, &s, &co);
        const int t = (a + 1) * 3 + (c + 1);
        kh = cadd(kh, cmul(make_float2(Kr[t], Ki[t]), make_float2(co, s)));
      }
    float2 h;
    if (literal) {
      const float2 k2 = cmul(kh, kh);
      const float2 den = make_float2(k2.x + eps, k2.y);
      const float d2 = den.x * den.x + den.y * den.y;
      h = make_float2((kh.x * den.x + kh.y * den.y) / d2, (kh.y * den.x - kh.x * den.y) / d2);
    } else {
      const float d = kh.x * kh.x + kh.y * kh.y + eps;
      h = make_float2(kh.x / d, -kh.y / d);
    }
    H[i] = h;
  }
  __syncthreads();
  // T[u][j] = sum_v H[u][v] e^{+2 pi i v d_j / n6x}, d_j = j for j < m_x else j - 2m_x
  for (int i = threadIdx.x; i < n6y * nx; i += blockDim.x) {
    const int u = i / nx, j = i % nx;
    const int d = j < mx ? j : j - nx;
    float2 acc = make_float2(0.f, 0.f);
    for (int v = 0; v < n6x; ++v) {
      float s, co;
      const int e = ((v * d) % n6x + n6x) % n6x;
      sincospif(2.f * e / n6x, &s, &co);
      acc = cadd(acc, cmul(H[u * n6x + v], make_float2(co, s)));
    }
    T[i] = acc;
  }
  __syncthreads();
  // Gc[i][j] = sum_u T[u][j] e^{+2 pi i u d_i / n6y} / (n6y n6x), d_i = i for i < m_y else i - 2m_y
  const float sc = 1.f / (static_cast<float>(n6y) * n6x);
  for (int i = threadIdx.x; i < ny * nx; i += blockDim.x) {
    const int ii = i / nx, j = i % nx;
    const int d = ii < my ? ii : ii - ny;
    float2 acc = make_float2(0.f, 0.f);
    for (int u = 0; u < n6y; ++u) {
      float s, co;
      const int e = ((u * d) % n6y + n6y) % n6y;
      sincospif(2.f * e / n6y, &s, &co);
      acc = cadd(acc, cmul(T[u * nx + j], make_float2(co, s)));
    }
    Gc[i] = cscale(acc, sc);
  }
  __syncthreads();
  // G_hat = DFT(Gc): along rows (length 2m_x), then along columns (length 2m_y), T as scratch
  for (int i = threadIdx.x; i < ny * nx; i += blockDim.x) {
    const int r = i / nx, q = i % nx;
    float2 acc = make_float2(0.f, 0.f);
    for (int j = 0; j < nx; ++j) {
      float s, co;
      sincospif(-2.f * ((q * j) % nx) / nx, &s, &co);
      acc = cadd(acc, cmul(Gc[r * nx + j], make_float2(co, s)));
    }
    T[i] = acc;
  }
  __syncthreads();
  float2* out = ghat + static_cast<long>(k) * ny * nx;
  for (int i = threadIdx.x; i < ny * nx; i += blockDim.x) {
    const int p = i / nx, q = i % nx;
    float2 acc = make_float2(0.f, 0.f);
    for (int r = 0; r < ny; ++r) {
      float s, co;
      sincospif(-2.f * ((p * r) % ny) / ny, &s, &co);
      acc = cadd(acc, cmul(T[r * nx + q], make_float2(co, s)));
    }
    out[i] = acc;
  }
}

// ---- projection 1x1 (C -> 2, + bias) at I/2, bilinear prolongation to I, times s ----
// one CTA per (sample b, coarse row J) of the Ncy x Ncx coarse grid: the 1x1 projections
// of coarse rows J and J + 1 are computed once into shared memory, then the CTA writes
// fine rows 2J and 2J + 1 (bilinear P: even fine index = coarse value, odd = mean of the
// two neighbours, zero beyond the last coarse row / column)
constexpr int PJ_C = 16;
constexpr int PJ_MAXNC = 2048;
__global__ void __launch_bounds__(256) k_proj_prolong(const bf16* __restrict__ u, int B, int Ncy, int Ncx, int C,
                                                      const float* __restrict__ w, const float* __restrict__ bias,
                                                      const float* __restrict__ s, float2* __restrict__ e) {
  __shared__ float2 Pk[2][PJ_MAXNC + 1];
  const int J = blockIdx.x, b = blockIdx.y;
  float w0[PJ_C], w1[PJ_C];
#pragma unroll
  for (int ch = 0; ch < PJ_C; ++ch) {
    w0[ch] = w[ch];
    w1[ch] = w[C + ch];
  }
  const float b0 = bias[0], b1 = bias[1];
  for (int i = threadIdx.x; i < 2 * (Ncx + 1); i += blockDim.x) {
    const int a = i / (Ncx + 1), K = i - a * (Ncx + 1);
    float2 pv = make_float2(0.f, 0.f);
    if (J + a < Ncy && K < Ncx) {
      const uint4* up = reinterpret_cast<const uint4*>(u + ((static_cast<long>(b) * Ncy + J + a) * Ncx + K) * C);
      float p0 = b0, p1 = b1;
#pragma unroll
      for (int h = 0; h < PJ_C / 8; ++h) {
        const uint4 v = up[h];
        const __nv_bfloat162* e2 = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 f = __bfloat1622float2(e2[q]);
          p0 = fmaf(w0[8 * h + 2 * q], f.x, fmaf(w0[8 * h + 2 * q + 1], f.y, p0));
          p1 = fmaf(w1[8 * h + 2 * q], f.x, fmaf(w1[8 * h + 2 * q + 1], f.y, p1));
        }
      }
      pv = make_float2(p0, p1);
    }
    Pk[a][K] = pv;
  }
  __syncthreads();
  const int Ny = 2 * Ncy, Nx = 2 * Ncx;
  const float sc = s[b];
  for (int i = threadIdx.x; i < 2 * Ncx; i += blockDim.x) {
    const int af = i / Ncx, K = i - af * Ncx;   // fine row 2J + af, fine columns 2K, 2K + 1
    const float2 r0 = af ? cscale(cadd(Pk[0][K], Pk[1][K]), 0.5f) : Pk[0][K];
    const float2 r1 = af ? cscale(cadd(Pk[0][K + 1], Pk[1][K + 1]), 0.5f) : Pk[0][K + 1];
    const float2 ev = cscale(r0, sc);
    const float2 od = cscale(cscale(cadd(r0, r1), 0.5f), sc);
    float2* eo = e + (static_cast<long>(b) * Ny + 2 * J + af) * Nx + 2 * K;
    *reinterpret_cast<float4*>(eo) = make_float4(ev.x, ev.y, od.x, od.y);
  }
}

// ---- launch helpers -----------------------------------------------------------------
static int grid_for(long n, int threads = 256) { return static_cast<int>(std::min<long>(div_up(n, threads), 8192)); }

int launch_kfeat(const float* kappa, const float* gamma, long n, bf16* out, cudaStream_t st) {
  HELM_LAUNCH("k_kfeat", st, k_kfeat<<<grid_for(n), 256, 0, st>>>(kappa, gamma, n, out));
  HELM_CHECK_LAUNCH("k_kfeat");
  return HELM_OK;
}

int launch_prep(const float2* r, int Ny, int Nx, int B, double* part, float* s, float* inv, bf16* x0,
                cudaStream_t st) {
  const long n = static_cast<long>(Ny) * Nx;
  const int nblk = std::max(1, std::min(256, div_up(n, 4096)));
  HELM_LAUNCH("k_norm_partial", st, k_norm_partial<<<dim3(nblk, B), 256, 0, st>>>(r, n, nblk, part));
  HELM_LAUNCH("k_norm_final", st, k_norm_final<<<div_up(B, 64), 64, 0, st>>>(part, nblk, B, n, s, inv));
  HELM_LAUNCH("k_prep_restrict", st,
              k_prep_restrict<<<grid_for(static_cast<long>(B) * (Ny / 2) * (Nx / 2)), 256, 0, st>>>(r, Ny, Nx, B, inv,
                                                                                                    x0));
  HELM_CHECK_LAUNCH("prep");
  return HELM_OK;
}

int launch_dw(const bf16* x, int B, int H, int W, int C, const float* w, const float* scale, const float* shift,
              int act, bf16* y, float* yraw, cudaStream_t st) {
  if (C > DW_MAXC || C % 8) {
    set_error("depthwise: %d channels (kernel supports multiples of 8 up to %d)", C, DW_MAXC);
    return HELM_EINVAL;
  }
  const int nstrip = div_up(W, DW_XS);
#define HELM_DW_CASE(cc)                                                                                   \
  if (C == cc) {                                                                                         \
    dim3 grid(div_up(nstrip * (cc / 8), 256), B * H);                                                    \
    HELM_LAUNCH("k_dw3x3", st, k_dw3x3_row<cc><<<grid, 256, 0, st>>>(x, H, W, w, scale, shift, act, y, yraw)); \
    HELM_CHECK_LAUNCH("k_dw3x3");                                                                        \
    return HELM_OK;                                                                                      \
  }
  if (static_cast<long>(B) * H <= 65535) {
    HELM_DW_CASE(96)
    HELM_DW_CASE(192)
    HELM_DW_CASE(384)
  }
#undef HELM_DW_CASE
  HELM_LAUNCH("k_dw3x3", st,
              k_dw3x3<<<grid_for(static_cast<long>(B) * H * W * (C / 8)), 256, 0, st>>>(x, B, H, W, C, w, scale,
                                                                                         shift, act, y, yraw));
  HELM_CHECK_LAUNCH("k_dw3x3");
  return HELM_OK;
}

size_t implicit_smem(int m) { return static_cast<size_t>(2 * m + m * m + m * 2 * m + 4 * m * m) * sizeof(float2); }

// chunk width and FFT plans (rows of length 2m_x, columns of length 2m_y) of an
// m_y x m_x implicit layer, or an error
static int implicit_setup(int my, int mx, int* cw, FftPlan* planx, FftPlan* plany) {
  if (my <= 0 || mx <= 0) {
    set_error("implicit layer: empty %dx%d coarsest map", my, mx);
    return HELM_ESHAPE;
  }
  *cw = implicit_chunk(my, mx);
  if (!*cw) {
    set_error("implicit layer: %dx%d coarsest map exceeds shared memory", my, mx);
    return HELM_ESHAPE;
  }
  if (!fft_plan(2 * mx, planx) || !fft_plan(2 * my, plany)) {
    set_error("implicit layer: 2m_x = %d or 2m_y = %d has a prime factor above %d", 2 * mx, 2 * my, FFT_PMAX);
    return HELM_ESHAPE;
  }
  return HELM_OK;
}

// lines per CTA of a three-pass line length n: the most (up to 16) whose two buffers and
// twiddles fit 48 KB
static int pass_chunk(int n) { return std::max(1, std::min(16, (6144 - n) / (2 * n))); }

size_t implicit_3pass_bytes(int B, int my, int mx, int C) {
  return static_cast<size_t>(B) * (C / 2) * my * (2 * mx) * sizeof(float2);
}

// the three passes of k_implicit_pass; scratch holds implicit_3pass_bytes
static int launch_implicit_3pass(const bf16* x, int B, int my, int mx, int C, const float2* ghat, bf16* y,
                                 float2* scratch, cudaStream_t st) {
  FftPlan planx, plany;
  if (!fft_plan(2 * mx, &planx) || !fft_plan(2 * my, &plany)) {
    set_error("implicit layer: 2m_x = %d or 2m_y = %d has a prime factor above %d", 2 * mx, 2 * my, FFT_PMAX);
    return HELM_ESHAPE;
  }
  const int nx = 2 * mx, ny = 2 * my;
  if (nx > 2048 || ny > 2048 || B > 65535 || C / 2 > 65535) {
    set_error("implicit layer: %dx%d map or batch %d beyond the three-pass kernel's limits", my, mx, B);
    return HELM_ESHAPE;
  }
  for (int pass = 0; pass < 3; ++pass) {
    const int n = pass == 1 ? ny : nx, lines = pass == 1 ? nx : my;
    const int cw = pass_chunk(n);
    const size_t smem = static_cast<size_t>(n + 2 * cw * n) * sizeof(float2);
    const dim3 grid(C / 2, B, div_up(lines, cw));
    HELM_LAUNCH("k_implicit_pass", st,
                k_implicit_pass<bf16, bf16><<<grid, 256, smem, st>>>(x, my, mx, C, ghat, 0, scratch, y, 0, pass, cw,
                                                                      pass == 1 ? plany : planx));
  }
  HELM_CHECK_LAUNCH("k_implicit_pass");
  return HELM_OK;
}

int launch_implicit_bf16(const bf16* x, int B, int my, int mx, int C, const float2* ghat, bf16* y, cudaStream_t st,
                         float2* scratch) {
  if (my <= 0 || mx <= 0) {
    set_error("implicit layer: empty %dx%d coarsest map", my, mx);
    return HELM_ESHAPE;
  }
  // three passes when the one-CTA form does not fit shared memory, or when the tuning
  // table asks for them at this height and batch; they need the caller's scratch
  if (scratch && (!implicit_chunk(my, mx) || tune_get(HELM_TUNE_IMPLICIT_3PASS, my, B) > 0))
    return launch_implicit_3pass(x, B, my, mx, C, ghat, y, scratch, st);
  int cw;
  FftPlan planx, plany;
  if (int rc = implicit_setup(my, mx, &cw, &planx, &plany)) return rc;
  static std::atomic<unsigned long long> attr_done{0};
  if (int rc = smem_attr_once(k_implicit<bf16, bf16>, 200 * 1024, &attr_done)) return rc;
  HELM_LAUNCH("k_implicit", st,
              k_implicit<bf16, bf16><<<dim3(C / 2, B), 256, implicit_chunk_smem(my, mx, cw), st>>>(
                  x, my, mx, C, ghat, 0, y, 0, cw, planx, plany));
  HELM_CHECK_LAUNCH("k_implicit");
  return HELM_OK;
}

int launch_implicit_adjoint(const float* gy, int B, int m, int C, const float2* ghat, float* gx, cudaStream_t st) {
  int cw;
  FftPlan planx, plany;
  if (int rc = implicit_setup(m, m, &cw, &planx, &plany)) return rc;
  static std::atomic<unsigned long long> attr_done{0};
  if (int rc = smem_attr_once(k_implicit<float, float>, 200 * 1024, &attr_done)) return rc;
  HELM_LAUNCH("k_implicit_adj", st,
              k_implicit<float, float><<<dim3(C / 2, B), 256, implicit_chunk_smem(m, m, cw), st>>>(
                  gy, m, m, C, ghat, 1, gx, 1, cw, planx, plany));
  HELM_CHECK_LAUNCH("k_implicit_adj");
  return HELM_OK;
}

size_t greens_scratch_elems(int my, int mx, int nk) {
  const long n6y = 6 * my, n6x = 6 * mx, ny = 2 * my, nx = 2 * mx;
  return static_cast<size_t>(nk) * (n6y * n6x + n6y * nx + ny * nx);
}

int launch_greens(const float* Kpar, int nk, int my, int mx, float eps, int literal, float2* scratch, float2* ghat,
                  cudaStream_t st) {
  HELM_LAUNCH("k_greens", st, k_greens<<<nk, 256, 0, st>>>(Kpar, nk, my, mx, eps, literal, scratch, ghat));
  HELM_CHECK_LAUNCH("k_greens");
  return HELM_OK;
}

int launch_proj(const bf16* u, int B, int Ncy, int Ncx, int C, const float* w, const float* bias, const float* s,
                float2* e, cudaStream_t st) {
  if (C != PJ_C) {
    set_error("projection: kernel built for %d input channels", PJ_C);
    return HELM_EINVAL;
  }
  if (Ncx > PJ_MAXNC || Ncy > 65535 || B > 65535) {
    set_error("projection: coarse grid %d x %d or batch %d beyond the kernel's limits (width %d, 65535 rows and "
              "samples)", Ncy, Ncx, B, PJ_MAXNC);
    return HELM_ESHAPE;
  }
  HELM_LAUNCH("k_proj_prolong", st, k_proj_prolong<<<dim3(Ncy, B), 256, 0, st>>>(u, B, Ncy, Ncx, C, w, bias, s, e));
  HELM_CHECK_LAUNCH("k_proj_prolong");
  return HELM_OK;
}

}  // namespace helm

extern "C" int helm_implicit_bf16(const void* x, int batch, int m, int c, const void* ghat, void* y, void* stream) {
  using namespace helm;
  if (!x || !ghat || !y || x == y || batch <= 0 || m <= 0 || c <= 0 || c % 2) {
    set_error("helm_implicit_bf16: invalid argument (even channel count, distinct x and y)");
    return HELM_EINVAL;
  }
  if (c % 8) {
    set_error("helm_implicit_bf16: channels must be a multiple of 8 (NHWC groups of 8)");
    return HELM_EINVAL;
  }
  return launch_implicit_bf16(static_cast<const bf16*>(x), batch, m, m, c, static_cast<const float2*>(ghat),
                              static_cast<bf16*>(y), static_cast<cudaStream_t>(stream));
}

extern "C" int helm_implicit_3pass_bf16(const void* x, int batch, int my, int mx, int c, const void* ghat, void* y,
                                        void* ws, size_t ws_bytes, void* stream) {
  using namespace helm;
  if (!x || !ghat || !y || !ws || x == y || batch <= 0 || my <= 0 || mx <= 0 || c <= 0 || c % 8) {
    set_error("helm_implicit_3pass_bf16: invalid argument (channels a multiple of 8, distinct x and y, a workspace)");
    return HELM_EINVAL;
  }
  if (ws_bytes < implicit_3pass_bytes(batch, my, mx, c)) {
    set_error("helm_implicit_3pass_bf16: workspace of %zu bytes, %zu needed", ws_bytes,
              implicit_3pass_bytes(batch, my, mx, c));
    return HELM_EWORKSPACE;
  }
  return launch_implicit_3pass(static_cast<const bf16*>(x), batch, my, mx, c, static_cast<const float2*>(ghat),
                               static_cast<bf16*>(y), static_cast<float2*>(ws), static_cast<cudaStream_t>(stream));
}

extern "C" int helm_implicit_3pass_workspace_size(int batch, int my, int mx, int c, size_t* bytes) {
  if (batch <= 0 || my <= 0 || mx <= 0 || c <= 0 || !bytes) {
    helm::set_error("helm_implicit_3pass_workspace_size: invalid argument");
    return HELM_EINVAL;
  }
  *bytes = helm::implicit_3pass_bytes(batch, my, mx, c);
  return HELM_OK;
}

extern "C" int helm_implicit_rect_bf16(const void* x, int batch, int my, int mx, int c, const void* ghat, void* y,
                                       void* stream) {
  using namespace helm;
  if (!x || !ghat || !y || x == y || batch <= 0 || my <= 0 || mx <= 0 || c <= 0 || c % 8) {
    set_error("helm_implicit_rect_bf16: invalid argument (channels a multiple of 8, distinct x and y)");
    return HELM_EINVAL;
  }
  return launch_implicit_bf16(static_cast<const bf16*>(x), batch, my, mx, c, static_cast<const float2*>(ghat),
                              static_cast<bf16*>(y), static_cast<cudaStream_t>(stream));
}
