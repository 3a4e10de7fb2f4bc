// Inverted bottleneck of the solver network (MobileNetV2 block of Sections 4.4 and 5.3)
// in one kernel, evaluation mode:
//     y = x + BN2(P * softplus(BN1(dw3x3(softplus(BN0(E * x))))))
// with E the 1x1 expansion C -> 6C, dw3x3 the depthwise 3x3 (zero padding) and P the
// 1x1 projection 6C -> C.  The 6C-channel intermediates never leave the SM.
//
// One CTA (8 warps) per 8 x 16 output tile at a time (persistent over tiles):
//   1. the 10 x 18 halo of x is staged by cp.async (zero outside the image) as the
//      K-major A operand of the expansion (one plane of 256 rows per 8-channel group);
//   2. for each chunk of 96 expanded channels: two M = 128 tcgen05 MMAs (halo rows
//      0-127 and 128-255) into TMEM; epilogue BN0 + softplus -> BF16 halo buffer in
//      shared memory, exactly zero outside the image (the depthwise zero padding);
//      the depthwise 3x3 on CUDA cores (weights in registers) + BN1 + softplus -> BF16
//      K-major A operand of the projection; projection MMAs accumulate over the chunks;
//   3. epilogue BN2 + the identity skip read from the staged halo tile -> BF16 output.
// The expanded activations are held in FP16 (three more mantissa bits than the BF16
// tensor of the three-kernel path) so that the depthwise products run as packed HFMA2:
// each row of three taps is summed in FP16, the three row sums in FP32.  The depthwise
// output is rounded to BF16 as in the three-kernel path.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "cnn.h"
#include "tc.cuh"

namespace {

using bf16 = __nv_bfloat16;

constexpr int IB_THREADS = 256;
constexpr int IB_TH = 8, IB_TW = 16;                           // output tile
constexpr int IB_HH = IB_TH + 2, IB_HW = IB_TW + 2;            // halo tile
constexpr int IB_NH = IB_HH * IB_HW;                           // 180 halo pixels
constexpr int IB_ROWS = 256;                                   // A rows of the expansion
constexpr int IB_EC = 96;                                      // expanded channels per chunk
constexpr int IB_EG = IB_EC / 8;                               // 8-channel groups per chunk
constexpr int IB_EPITCH = IB_EC + 8;                           // halo buffer row pitch (bf16)
constexpr int IB_DW_THREADS = IB_EG * IB_TW;                   // 192: (group, column)

template <int C>
struct IbCfg {
  static constexpr int E = 6 * C;
  static constexpr int G = C / 8;
  static constexpr int NCH = E / IB_EC;
  static constexpr size_t X_BYTES = static_cast<size_t>(G) * IB_ROWS * 16;
  static constexpr size_t WE_BYTES = static_cast<size_t>(E) * C * 2;
  static constexpr size_t WP_BYTES = WE_BYTES;
  static constexpr size_t H_BYTES = static_cast<size_t>(IB_NH) * IB_EPITCH * 2;
  static constexpr size_t D_BYTES = static_cast<size_t>(IB_EG) * 128 * 16;
  static constexpr size_t DW_BYTES = static_cast<size_t>(9) * E * 4;
  static constexpr size_t BN_BYTES = static_cast<size_t>(4 * E + 2 * C) * 4;
  static constexpr size_t SMEM = X_BYTES + WE_BYTES + WP_BYTES + H_BYTES + D_BYTES + DW_BYTES + BN_BYTES + 64;
  static constexpr int TCOLS = 256;   // expansion: 2 x 96 columns; projection: C <= 64
  static_assert(E % IB_EC == 0 && C % 16 == 0 && C <= 64, "IB shape");
};

struct IbArgs {
  const bf16* x;          // [B][H][W][C]
  int B, H, W;
  const bf16* we;         // packed expansion weights [G][E][8]
  const bf16* wp;         // packed projection weights [E/8][C][8]
  const float* wdw;       // depthwise weights [E][9] (FP32)
  const float* bn0;       // folded BN after the expansion: scale [E], shift [E]
  const float* bn1;       // after the depthwise conv: scale [E], shift [E]
  const float* bn2;       // after the projection: scale [C], shift [C]
  bf16* y;                // [B][H][W][C]
  int tiles_x, tiles_y, ntiles;
};

template <int C>
__global__ void __launch_bounds__(IB_THREADS, 2) k_ib_fused(const IbArgs a) {
  using Cfg = IbCfg<C>;
  constexpr int E = Cfg::E, G = Cfg::G;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sX = smem;
  uint8_t* sWe = sX + Cfg::X_BYTES;
  uint8_t* sWp = sWe + Cfg::WE_BYTES;
  __half* sH = reinterpret_cast<__half*>(sWp + Cfg::WP_BYTES);
  uint8_t* sD = reinterpret_cast<uint8_t*>(sH) + Cfg::H_BYTES;
  float* sDW = reinterpret_cast<float*>(sD + Cfg::D_BYTES);      // [9][E]
  float* sS0 = sDW + 9 * E;
  float* sB0 = sS0 + E;
  float* sS1 = sB0 + E;
  float* sB1 = sS1 + E;
  float* sS2 = sB1 + E;
  float* sB2 = sS2 + C;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sB2 + C + (C & 1));   // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane_q = warp & 3;

  if (warp == 0) tc::tmem_alloc(tslot, Cfg::TCOLS);
  {
    const uint4* s1 = reinterpret_cast<const uint4*>(a.we);
    const uint4* s2 = reinterpret_cast<const uint4*>(a.wp);
    uint4* d1 = reinterpret_cast<uint4*>(sWe);
    uint4* d2 = reinterpret_cast<uint4*>(sWp);
    for (int i = tid; i < static_cast<int>(Cfg::WE_BYTES / 16); i += IB_THREADS) {
      d1[i] = s1[i];
      d2[i] = s2[i];
    }
    for (int i = tid; i < 9 * E; i += IB_THREADS) sDW[(i % 9) * E + i / 9] = a.wdw[i];
    for (int c = tid; c < E; c += IB_THREADS) {
      sS0[c] = a.bn0[c];
      sB0[c] = a.bn0[E + c];
      sS1[c] = a.bn1[c];
      sB1[c] = a.bn1[E + c];
    }
    for (int c = tid; c < C; c += IB_THREADS) {
      sS2[c] = a.bn2[c];
      sB2[c] = a.bn2[C + c];
    }
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t sX_u = smem_u32(sX), sWe_u = smem_u32(sWe), sWp_u = smem_u32(sWp), sD_u = smem_u32(sD);
  constexpr uint32_t idesc_e = tc::idesc_bf16(128, IB_EC);
  constexpr uint32_t idesc_p = tc::idesc_bf16(128, C);
  constexpr uint32_t TP = 2 * IB_EC;   // TMEM column of the projection accumulator
  uint32_t phase[2] = {0u, 0u};
  bool ok = true;

  for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
    const int b = tile / (a.tiles_x * a.tiles_y);
    const int rem = tile - b * a.tiles_x * a.tiles_y;
    const int y0 = (rem / a.tiles_x) * IB_TH, x0 = (rem % a.tiles_x) * IB_TW;
    const bf16* xb = a.x + static_cast<long>(b) * a.H * a.W * C;
    // ---- 1. halo tile of x: plane g, row p = halo pixel (hy, hx) ----
    for (int idx = tid; idx < IB_NH * G; idx += IB_THREADS) {
      const int g = idx % G, p = idx / G;
      const int iy = y0 - 1 + p / IB_HW, ix = x0 - 1 + p % IB_HW;
      const bool in = iy >= 0 && iy < a.H && ix >= 0 && ix < a.W;
      const bf16* src = in ? xb + (static_cast<long>(iy) * a.W + ix) * C + 8 * g : xb;
      tc::cp_async16(sX_u + static_cast<uint32_t>((g * IB_ROWS + p) * 16), src, in ? 16u : 0u);
    }
    tc::cp_async_wait_all();
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();

#pragma unroll 1
    for (int ch = 0; ch < Cfg::NCH && ok; ++ch) {
      // ---- 2a. expansion MMAs: rows 0-127 -> TMEM columns [0, 96), 128-255 -> [96, 192) ----
      if (tid == 0) {
        tc::fence_after_sync();
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
          for (int kc = 0; kc < C / 16; ++kc) {
            const uint32_t aaddr = sX_u + static_cast<uint32_t>(((2 * kc) * IB_ROWS + 128 * mt) * 16);
            const uint32_t baddr = sWe_u + static_cast<uint32_t>(((2 * kc) * E + ch * IB_EC) * 16);
            tc::mma_bf16(tmem + mt * IB_EC, tc::sdesc(aaddr, IB_ROWS * 16, 128), tc::sdesc(baddr, E * 16, 128),
                         idesc_e, kc > 0);
          }
        }
        tc::commit(&bar[0]);
      }
      ok = mbar_wait_bounded(&bar[0], phase[0], HELM_DEVERR_MMA_WAIT) && ok;
      phase[0] ^= 1u;
      tc::fence_after_sync();
      // ---- 2b. BN0 + softplus -> halo buffer; warps 0-3: halo rows 0-127, 4-7: 128-255 ----
      {
        const int p = 128 * (warp >> 2) + 32 * lane_q + (tid & 31);
        const int iy = y0 - 1 + p / IB_HW, ix = x0 - 1 + p % IB_HW;
        const bool in = p < IB_NH && iy >= 0 && iy < a.H && ix >= 0 && ix < a.W;
#pragma unroll 1
        for (int c0 = 0; c0 < IB_EC; c0 += 16) {
          float v[16];
          tc::ld16(tmem + (static_cast<uint32_t>(lane_q * 32) << 16) + (warp >> 2) * IB_EC + c0, v);
          if (p >= IB_NH) continue;
          uint4 o[2];
          __half2* ob = reinterpret_cast<__half2*>(o);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int c = ch * IB_EC + c0 + 2 * i;
            float t0 = tc::softplus_fast(fmaf(v[2 * i], sS0[c], sB0[c]));
            float t1 = tc::softplus_fast(fmaf(v[2 * i + 1], sS0[c + 1], sB0[c + 1]));
            if (!in) t0 = t1 = 0.f;
            ob[i] = __floats2half2_rn(t0, t1);
          }
          uint4* dst = reinterpret_cast<uint4*>(sH + p * IB_EPITCH + c0);
          dst[0] = o[0];
          dst[1] = o[1];
        }
      }
      tc::fence_before_sync();
      ok = __syncthreads_and(ok) != 0;   // uniform: a timed-out wait stops every thread
      // ---- 2c. depthwise 3x3 + BN1 + softplus -> projection A operand (plane g, row = pixel) ----
      if (tid < IB_DW_THREADS) {
        // column fastest: the 16-byte stores of a quarter-warp go to consecutive rows
        const int xx = tid % IB_TW, g = tid / IB_TW;
        const int cb = ch * IB_EC + 8 * g;
        __half2 w[9][4];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const float4 lo = *reinterpret_cast<const float4*>(sDW + k * E + cb);
          const float4 hi = *reinterpret_cast<const float4*>(sDW + k * E + cb + 4);
          w[k][0] = __floats2half2_rn(lo.x, lo.y);
          w[k][1] = __floats2half2_rn(lo.z, lo.w);
          w[k][2] = __floats2half2_rn(hi.x, hi.y);
          w[k][3] = __floats2half2_rn(hi.z, hi.w);
        }
#pragma unroll 1
        for (int yy = 0; yy < IB_TH; ++yy) {
          float acc[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) acc[e] = 0.f;
#pragma unroll
          for (int dy = 0; dy < 3; ++dy) {
            __half2 rs[4];   // FP16 sum of the row's three taps
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
              const uint4 u = *reinterpret_cast<const uint4*>(sH + ((yy + dy) * IB_HW + xx + dx) * IB_EPITCH + 8 * g);
              const __half2* h2 = reinterpret_cast<const __half2*>(&u);
#pragma unroll
              for (int e = 0; e < 4; ++e)
                rs[e] = dx == 0 ? __hmul2(w[dy * 3][e], h2[e]) : __hfma2(w[dy * 3 + dx][e], h2[e], rs[e]);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float2 f = __half22float2(rs[e]);
              acc[2 * e] += f.x;
              acc[2 * e + 1] += f.y;
            }
          }
          uint4 o;
          __nv_bfloat162* ob = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int c = cb + 2 * e;
            ob[e] = __floats2bfloat162_rn(tc::softplus_fast(fmaf(acc[2 * e], sS1[c], sB1[c])),
                                          tc::softplus_fast(fmaf(acc[2 * e + 1], sS1[c + 1], sB1[c + 1])));
          }
          *reinterpret_cast<uint4*>(sD + (g * 128 + yy * IB_TW + xx) * 16) = o;
        }
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      // ---- 2d. projection MMAs, accumulated over the chunks ----
      if (tid == 0) {
        tc::fence_after_sync();
#pragma unroll
        for (int kc = 0; kc < IB_EC / 16; ++kc) {
          const uint32_t aaddr = sD_u + static_cast<uint32_t>((2 * kc) * 128 * 16);
          const uint32_t baddr = sWp_u + static_cast<uint32_t>(((ch * IB_EG + 2 * kc) * C) * 16);
          tc::mma_bf16(tmem + TP, tc::sdesc(aaddr, 128 * 16, 128), tc::sdesc(baddr, C * 16, 128), idesc_p,
                       ch > 0 || kc > 0);
        }
        tc::commit(&bar[1]);
      }
      // the next chunk rewrites the projection operand: wait for these MMAs first
      ok = mbar_wait_bounded(&bar[1], phase[1], HELM_DEVERR_MMA_WAIT) && ok;
      phase[1] ^= 1u;
      tc::fence_after_sync();
      ok = __syncthreads_and(ok) != 0;
    }
    // ---- 3. BN2 + identity skip -> y; warps 0-3, TMEM lane = output pixel ----
    if (warp < 4 && ok) {
      const int q = tid;   // 0..127 = yy * 16 + xx
      const int yy = q / IB_TW, xx = q % IB_TW;
      const int oy = y0 + yy, ox = x0 + xx;
      const bool valid = oy < a.H && ox < a.W;
      const int hp = (yy + 1) * IB_HW + xx + 1;   // halo pixel of the skip value
#pragma unroll 1
      for (int c0 = 0; c0 < C; c0 += 16) {
        float v[16];
        tc::ld16(tmem + (static_cast<uint32_t>(lane_q * 32) << 16) + TP + c0, v);
        if (!valid) continue;
        uint4 o[2];
        __nv_bfloat162* ob = reinterpret_cast<__nv_bfloat162*>(o);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint4 u = *reinterpret_cast<const uint4*>(sX + ((c0 / 8 + h) * IB_ROWS + hp) * 16);
          const __nv_bfloat162* s2 = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int i = 8 * h + 2 * e, c = c0 + i;
            const float2 sk = __bfloat1622float2(s2[e]);
            ob[4 * h + e] = __floats2bfloat162_rn(fmaf(v[i], sS2[c], sB2[c]) + sk.x,
                                                  fmaf(v[i + 1], sS2[c + 1], sB2[c + 1]) + sk.y);
          }
        }
        uint4* dst = reinterpret_cast<uint4*>(a.y + ((static_cast<long>(b) * a.H + oy) * a.W + ox) * C + c0);
        dst[0] = o[0];
        dst[1] = o[1];
      }
    }
    tc::fence_before_sync();
    ok = __syncthreads_and(ok) != 0;   // the halo tile is restaged by the next tile
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, Cfg::TCOLS);
}

template <int C>
int launch_ib_t(const IbArgs& a0, cudaStream_t st) {
  using Cfg = IbCfg<C>;
  IbArgs a = a0;
  a.tiles_x = helm::div_up(a.W, IB_TW);
  a.tiles_y = helm::div_up(a.H, IB_TH);
  a.ntiles = a.tiles_x * a.tiles_y * a.B;
  static std::atomic<unsigned long long> attr_done{0};
  int rc = helm::smem_attr_once(k_ib_fused<C>, static_cast<int>(Cfg::SMEM), &attr_done);
  int nsm = 0;
  if (!rc) rc = helm::sm_count(&nsm);
  if (rc) return rc;
  // resident CTAs per SM: shared memory (228 KB per SM, 1 KB reserved per CTA) and TMEM
  const int per_sm = std::max(1, std::min(static_cast<int>((228 * 1024) / (Cfg::SMEM + 1024)), 2));
  const int grid = std::max(1, std::min(a.ntiles, nsm * per_sm));
  HELM_LAUNCH("k_ib_fused", st, k_ib_fused<C><<<grid, IB_THREADS, Cfg::SMEM, st>>>(a));
  HELM_CHECK_LAUNCH("k_ib_fused");
  return HELM_OK;
}

}  // namespace

namespace helm {

int ib_fused(const IbLaunch& l, cudaStream_t st) {
  IbArgs a{};
  a.x = l.x;
  a.B = l.B;
  a.H = l.H;
  a.W = l.W;
  a.we = l.we;
  a.wp = l.wp;
  a.wdw = l.wdw;
  a.bn0 = l.bn0;
  a.bn1 = l.bn1;
  a.bn2 = l.bn2;
  a.y = l.y;
  if (l.expansion != 6) {
    set_error("fused inverted bottleneck: expansion %d (kernels exist for 6)", l.expansion);
    return HELM_EINVAL;
  }
  if ((l.C == 16 || l.C == 32) && l.wef && l.wpf) return ib_strip(l, st);   // the row-sweeping strip kernel
  switch (l.C) {
    case 16: return launch_ib_t<16>(a, st);
    case 32: return launch_ib_t<32>(a, st);
    case 64: return launch_ib_t<64>(a, st);
    default:
      set_error("fused inverted bottleneck: %d channels (kernels exist for 16, 32, 64)", l.C);
      return HELM_EINVAL;
  }
}

}  // namespace helm

extern "C" int helm_ib_bf16(const void* x, int batch, int h, int w, int c, const float* w_exp, const float* bn0,
                            const float* w_dw, const float* bn1, const float* w_proj, const float* bn2, void* y,
                            void* ws, size_t ws_bytes, void* stream) {
  using namespace helm;
  if (!x || !w_exp || !bn0 || !w_dw || !bn1 || !w_proj || !bn2 || !y || x == y || batch <= 0 || h <= 0 || w <= 0) {
    set_error("helm_ib_bf16: invalid argument (x and y must be distinct device buffers)");
    return HELM_EINVAL;
  }
  if (c != 16 && c != 32 && c != 64) {
    set_error("helm_ib_bf16: %d channels (kernels exist for 16, 32, 64)", c);
    return HELM_EINVAL;
  }
  const int E = 6 * c;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carve cv(ws, ws_bytes);
  bf16* we = cv.take<bf16>(static_cast<size_t>(conv_cs(c)) * E);
  bf16* wp = cv.take<bf16>(static_cast<size_t>(conv_cs(E)) * c);
  bf16* wef = cv.take<bf16>(ib_folded_elems(c, E));
  bf16* wpf = cv.take<bf16>(ib_folded_elems(E, c));
  if (cv.overflow || !ws) {
    set_error("helm_ib_bf16: workspace too small (need %zu bytes)", cv.off);
    return HELM_EWORKSPACE;
  }
  int rc = pack_conv_weights(w_exp, c, E, 1, 0, we, st);
  if (!rc) rc = pack_conv_weights(w_proj, E, c, 1, 0, wp, st);
  if (!rc && c != 64) rc = pack_ib_folded(w_exp, bn0, c, E, 0, wef, st);
  if (!rc && c != 64) rc = pack_ib_folded(w_proj, bn2, E, c, 1, wpf, st);
  if (rc) return rc;
  IbLaunch l;
  l.x = static_cast<const bf16*>(x);
  l.B = batch;
  l.H = h;
  l.W = w;
  l.C = c;
  l.expansion = 6;
  l.we = we;
  l.wp = wp;
  l.wdw = w_dw;
  l.bn0 = bn0;
  l.bn1 = bn1;
  l.bn2 = bn2;
  l.wef = c != 64 ? wef : nullptr;
  l.wpf = c != 64 ? wpf : nullptr;
  l.y = static_cast<bf16*>(y);
  return ib_fused(l, st);
}
