// 3x3 and 1x1 convolutions of the encoder-solver network (Sections 4.1, 4.4, 5.3) as
// implicit GEMMs on the tcgen05 tensor cores: BF16 NHWC activations and weights,
// FP32 accumulation in TMEM, fused epilogue
//     y = act(scale[c] * acc + shift[c]) + add1 + add2      (folded BN, softplus, skips)
// or the raw FP32 accumulator (training forward, BN statistics taken afterwards).
//
// GEMM mapping: M = 128 output pixels per tile, N = output channels, K = taps x
// input channels.  The output grid is flattened with a virtual pitch Po = Wo + 1 (one
// gap column, never written), so for every 3x3 tap the 128 input rows of the A
// operand are one contiguous window of virtual pixels shifted by dy*Po + dx; in the
// K-major no-swizzle shared-memory layout (core matrices of 8 rows x 16 bytes) a
// shift of the window is just a 16-byte step of the descriptor start address.  The
// loader stages, per 8-channel group, a plane of window rows (16 B each):
//   stride 1      : the input itself (output grid = input grid)
//   stride 2      : four phase planes S_{py,px}(y,x) = in(2y+py, 2x+px); tap dy uses
//                   phase (1, 0, 1)[dy+1] and shift (-1, 0, 0)[dy+1]
//   transposed s2 : sub-pixel form: the virtual grid is the INPUT grid, the window the
//                   input itself, and each of the four output phases (oy mod 2,
//                   ox mod 2) has its own accumulator and the 1, 2, 2 or 4 taps of the
//                   flipped kernel that reach it (out(2y+py, 2x+px) sums in(y + a, x + c)
//                   over a in {0, py}, c in {0, px}); no zero-inserted copy is staged
//   1x1           : 128 consecutive pixels, Po = Wo
// A dedicated MMA warp issues all MMAs of a step and commits them to an mbarrier; 8
// epilogue warps read the accumulator with tcgen05.ld (TMEM lane t = pixel q0 + t) and
// run the epilogue (see k_conv_tc).  CTAs are persistent over segments; weights stay
// resident in shared memory.
#include <cuda_bf16.h>

#include <algorithm>

#include "cnn.h"
#include "tc.cuh"

namespace {

using bf16 = __nv_bfloat16;

struct ConvArgs {
  const bf16* x;
  int B, Hi, Wi, Cg;     // input: batch, size, channels stored in global memory
  int Ho, Wo, Po;        // virtual output grid (input grid for transposed s2), pitch
  int Hout, Wout;        // stored output size (2 Ho x 2 Wo for transposed s2)
  int mode;
  const bf16* wpk;       // packed weights [taps][G][COUT][8]
  const float* scale;    // [COUT] or null (1)
  const float* shift;    // [COUT] or null (0)
  int act;               // softplus
  const bf16* add1;      // [B][Ho][Wo][COUT] or null
  const bf16* add2;      // [B / add2_div][Ho][Wo][COUT] or null
  int add2_div;          // consecutive samples sharing one add2 entry (1: per sample)
  bf16* y;               // bf16 NHWC output or null
  float* yraw;           // fp32 NHWC raw accumulator or null
  int seg_q;             // virtual output pixels per segment (whole rows for 3x3 where
                         // a row's window fits shared memory)
  int segs_per_img, nsegs;
  int L;                 // window rows per plane (odd)
};

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

template <int CS, int COUT, int TAPS, int PH = 1, int MTR = 2>
struct ConvCfg {
  static constexpr int G = CS / 8;                          // 16-byte groups per pixel
  static constexpr int NSPLIT = COUT > 256 ? 2 : 1;
  static constexpr int NH = COUT / NSPLIT;                  // N of one MMA
  static constexpr int ACC = PH * COUT;                     // accumulator columns per M-tile
  static constexpr int BBYTES = TAPS * G * COUT * 16;
  // M-tiles per step: two (256 pixels, one per epilogue warpgroup) while the two
  // double-buffered steps fit in 256 TMEM columns (two CTAs per SM), for light-weight
  // layers whose two-tile window fits beside the weights; MTR = 1 forces one
  static constexpr int MT =
      (MTR == 2 && 4 * ACC <= 256 && BBYTES <= 40 * 1024 && (TAPS == 9 || CS <= 192)) ? 2 : 1;
  static constexpr int STEP = MT * ACC;                     // accumulator columns per step
  static constexpr int NBUF = 2 * STEP <= 512 ? 2 : 1;      // TMEM accumulators (double buffer)
  static constexpr int NEED = NBUF * STEP;
  static constexpr int NCOLS = NEED <= 32 ? 32 : NEED <= 64 ? 64 : NEED <= 128 ? 128 : NEED <= 256 ? 256 : 512;
  static_assert(CS % 16 == 0, "K per tap must be a multiple of 16");
  static_assert(NH % 16 == 0 && NH <= 256, "N per MMA");
};

// One CTA works through segments (a band of whole output rows of one image; on grids too
// wide for one row's window, a run of MMA steps within a row; for 1x1 a run of pixels): all warps stage the segment's input window with asynchronous
// 16-byte copies (zero-filled outside the image); then warp 8 alone issues the MMAs of
// every step (one or two 128-pixel M-tiles) into one of two TMEM accumulators, and
// warps 0-7 run the epilogues.  The hand-off is two mbarrier pairs: `full` (MMA
// commit -> epilogue) and `empty` (the 8 epilogue warps -> MMA warp), so steps flow
// without block-wide barriers; the block synchronises only between segments, when the
// window is restaged.  Epilogue warps w and w + 4 share TMEM lanes 32 (w mod 4) .. + 31:
// with two M-tiles per step warpgroup g takes tile g and all channels, with one the two
// warpgroups split the channels in 16-wide chunks.
constexpr int CONV_EPI_WARPS = 8;
constexpr int CONV_THREADS = 32 * (CONV_EPI_WARPS + 1);

template <int CS, int COUT, int TAPS, int PH, int MTR>
__global__ void __launch_bounds__(CONV_THREADS, 2) k_conv_tc(const ConvArgs a) {
  using Cfg = ConvCfg<CS, COUT, TAPS, PH, MTR>;
  constexpr int G = Cfg::G;
  constexpr int MT = Cfg::MT;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sB = smem;
  uint8_t* sA = smem + Cfg::BBYTES;
  const int nph = (a.mode == HELM_CONV_S2) ? 4 : 1;
  const int L = a.L;
  const size_t win_bytes = static_cast<size_t>(nph) * G * L * 16;
  float* sScale = reinterpret_cast<float*>(sA + win_bytes);
  float* sShift = sScale + COUT;
  uint64_t* full = reinterpret_cast<uint64_t*>(sShift + COUT + (COUT & 1));   // [2]
  uint64_t* empty = full + 2;                                                // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(empty + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool mma_warp = warp == CONV_EPI_WARPS;
  const int lane_q = warp & 3, chalf = (warp >> 2) & 1;

  if (warp == 0) tc::tmem_alloc(tslot, Cfg::NCOLS);
  {
    const uint4* src = reinterpret_cast<const uint4*>(a.wpk);
    uint4* dst = reinterpret_cast<uint4*>(sB);
    for (int i = tid; i < Cfg::BBYTES / 16; i += CONV_THREADS) dst[i] = src[i];
    for (int c = tid; c < COUT; c += CONV_THREADS) {
      sScale[c] = a.scale ? a.scale[c] : 1.f;
      sShift[c] = a.shift ? a.shift[c] : 0.f;
    }
  }
  const bool full_groups = (a.Cg % 8) == 0;
  // inputs of 2 or 4 channels: only the first bytes of group 0 are ever written, so the
  // window is zeroed once here and the rest of it stays zero for every segment
  const bool narrow = a.Cg == 2 || a.Cg == 4;
  if (!full_groups) {
    uint4* w4 = reinterpret_cast<uint4*>(sA);
    for (int i = tid; i < nph * G * L; i += CONV_THREADS) w4[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&empty[0], CONV_EPI_WARPS);
    mbar_init(&empty[1], CONV_EPI_WARPS);
    fence_mbar_init();
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t sA_u = smem_u32(sA), sB_u = smem_u32(sB);
  constexpr uint32_t idesc = tc::idesc_bf16(128, Cfg::NH);
  // descriptor bits other than the start address (the address field is OR-ed in)
  const uint64_t dA = tc::sdesc(0, static_cast<uint32_t>(L) * 16u, 128);
  const uint64_t dB = tc::sdesc(0, COUT * 16, 128);
  // window offset (rows) and phase plane of each tap, for the MMA warp
  int toff[9], tpl[9];
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const int ty = tap / 3, tx = tap % 3;
    if (a.mode == HELM_CONV_S2) {
      toff[tap] = (ty == 0 ? 0 : 1) * a.Po + (tx == 0 ? 0 : 1);
      tpl[tap] = (ty == 1 ? 0 : 2) + (tx == 1 ? 0 : 1);
    } else {
      toff[tap] = ty * a.Po + tx;
      tpl[tap] = 0;
    }
  }
  bool ok = true;
  uint32_t gstep = 0;   // steps of this CTA over all its segments (buffer and phase index)
  // window start (virtual output position) relative to the segment start
  const int wofs = (TAPS == 1 || PH == 4) ? 0 : -(a.Po + 1);

  for (int seg = blockIdx.x; seg < a.nsegs && ok; seg += gridDim.x) {
    const int b = seg / a.segs_per_img;
    const int qs = (seg % a.segs_per_img) * a.seg_q;
    const int qe = min(qs + a.seg_q, a.Ho * a.Po);
    const bf16* xb = a.x + static_cast<long>(b) * a.Hi * a.Wi * a.Cg;
    // ---- stage the window: group fastest (coalesced global reads); plane (ph, g)
    //      holds L rows of 16 bytes ----
    for (int ph = 0; ph < nph; ++ph) {
      const int total = (narrow ? 1 : G) * L;
      for (int idx = tid; idx < total; idx += CONV_THREADS) {
        const int g = narrow ? 0 : idx % G, t = narrow ? idx : idx / G;
        const int q = qs + wofs + t;
        int iy = -1, ix = 0;
        if (TAPS == 1) {
          if (q < qe) { iy = 0; ix = q; }   // 1x1: the virtual pixel is the linear pixel
        } else {
          const int yv = floordiv(q, a.Po), xv = q - yv * a.Po;
          if (yv >= 0 && yv < a.Ho && xv < a.Wo) {
            if (a.mode == HELM_CONV_S1 || PH == 4) {
              iy = yv; ix = xv;
            } else {   // stride 2: phase plane ph
              iy = 2 * yv + (ph >> 1); ix = 2 * xv + (ph & 1);
            }
          }
        }
        const int c0 = 8 * g;
        uint8_t* dptr = sA + static_cast<size_t>((ph * G + g) * L + t) * 16;
        const bf16* px = xb + (static_cast<long>(iy < 0 ? 0 : iy) * a.Wi + ix) * a.Cg;
        if (full_groups) {
          const bool in = iy >= 0 && c0 < a.Cg;
          tc::cp_async16(smem_u32(dptr), in ? px + c0 : xb, in ? 16u : 0u);
        } else if (narrow) {
          if (a.Cg == 2)
            tc::cp_async_small<4>(smem_u32(dptr), iy >= 0 ? px : xb, iy >= 0 ? 4u : 0u);
          else
            tc::cp_async_small<8>(smem_u32(dptr), iy >= 0 ? px : xb, iy >= 0 ? 8u : 0u);
        } else {
          uint16_t tmp[8] = {0, 0, 0, 0, 0, 0, 0, 0};
          if (iy >= 0)
            for (int e = 0; c0 + e < a.Cg && e < 8; ++e) tmp[e] = reinterpret_cast<const uint16_t*>(px)[c0 + e];
          *reinterpret_cast<uint4*>(dptr) = make_uint4(tmp[0] | (tmp[1] << 16), tmp[2] | (tmp[3] << 16),
                                                       tmp[4] | (tmp[5] << 16), tmp[6] | (tmp[7] << 16));
        }
      }
    }
    tc::cp_async_wait_all();
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const int nsteps = (qe - qs + 128 * MT - 1) / (128 * MT);

    if (mma_warp) {
      // ---- MMA issue: one thread, all steps of the segment ----
      if (lane == 0) {
        for (int j = 0; j < nsteps; ++j) {
          const uint32_t g = gstep + j, buf = g % Cfg::NBUF, use = g / Cfg::NBUF;
          if (use > 0) ok = mbar_wait_bounded(&empty[buf], (use - 1) & 1u, HELM_DEVERR_MMA_WAIT) && ok;
          tc::fence_after_sync();
#pragma unroll
          for (int mt = 0; mt < MT; ++mt) {
            const int row0 = 128 * (MT * j + mt);
            const uint32_t dcol = buf * Cfg::STEP + mt * Cfg::ACC;
            if constexpr (PH == 4) {
              // output phase ph = 2 py + px: taps (ty, tx) of the flipped kernel with ty
              // in {1} (py = 0) or {0, 2} (py = 1), likewise tx; window offset
              // (ty / 2) Po + tx / 2
#pragma unroll
              for (int ph = 0; ph < 4; ++ph) {
                const int py = ph >> 1, px = ph & 1;
                int kstep = 0;
#pragma unroll
                for (int a2 = 0; a2 <= py; ++a2)
#pragma unroll
                  for (int c2 = 0; c2 <= px; ++c2) {
                    const int tap = (py ? 2 * a2 : 1) * 3 + (px ? 2 * c2 : 1);
                    const int row = row0 + a2 * a.Po + c2;
#pragma unroll
                    for (int kc = 0; kc < CS / 16; ++kc) {
                      const uint32_t aaddr = sA_u + static_cast<uint32_t>(((2 * kc) * L + row) * 16);
                      const uint32_t baddr = sB_u + static_cast<uint32_t>(((tap * G + 2 * kc) * COUT) * 16);
                      tc::mma_bf16(tmem + dcol + ph * COUT, dA | (aaddr >> 4), dB | (baddr >> 4), idesc, kstep > 0);
                      ++kstep;
                    }
                  }
              }
            } else {
#pragma unroll
              for (int tap = 0; tap < TAPS; ++tap) {
                const int row = row0 + (TAPS == 9 ? toff[tap] : 0);
                const int pl = TAPS == 9 ? tpl[tap] : 0;
#pragma unroll
                for (int kc = 0; kc < CS / 16; ++kc) {
                  const uint32_t aaddr = sA_u + static_cast<uint32_t>(((pl * G + 2 * kc) * L + row) * 16);
#pragma unroll
                  for (int nh = 0; nh < Cfg::NSPLIT; ++nh) {
                    const uint32_t baddr =
                        sB_u + static_cast<uint32_t>(((tap * G + 2 * kc) * COUT + nh * Cfg::NH) * 16);
                    tc::mma_bf16(tmem + dcol + nh * Cfg::NH, dA | (aaddr >> 4), dB | (baddr >> 4), idesc,
                                 tap > 0 || kc > 0);
                  }
                }
              }
            }
          }
          tc::commit(&full[buf]);
        }
      }
      __syncwarp();
    } else {
      // ---- epilogues: TMEM lane (tid mod 128) <-> virtual pixel of M-tile mt ----
      const int mt = MT == 2 ? chalf : 0;
      const int cfirst = MT == 2 ? 0 : 16 * chalf, cstep = MT == 2 ? 16 : 32;
      // the residual inputs of one 16-channel chunk (two 16-byte vectors each), loaded
      // before the accumulator is read so that their latency overlaps the TMEM load
      // (and, for a step's first chunk, the wait for the MMAs)
      auto load_adds = [&](bool ok_px, long pix, long pix2, int c0, uint4 (&r1)[2], uint4 (&r2)[2]) {
        if (ok_px && a.y && a.add1) {
          const uint4* pp = reinterpret_cast<const uint4*>(a.add1 + pix * COUT + c0);
          r1[0] = pp[0];
          r1[1] = pp[1];
        }
        if (ok_px && a.y && a.add2) {
          const uint4* pp = reinterpret_cast<const uint4*>(a.add2 + pix2 * COUT + c0);
          r2[0] = pp[0];
          r2[1] = pp[1];
        }
      };
      for (int j = 0; j < nsteps; ++j) {
        const uint32_t g = gstep + j, buf = g % Cfg::NBUF, use = g / Cfg::NBUF;
        const int q = qs + 128 * (MT * j + mt) + (tid & 127);
        const int y = q / a.Po, x = q - y * a.Po;
        const bool inside = q < qe && x < a.Wo;
        auto pixel = [&](int ph, long& pix, long& pix2) {
          const int oy = PH == 4 ? 2 * y + (ph >> 1) : y, ox = PH == 4 ? 2 * x + (ph & 1) : x;
          pix = (static_cast<long>(b) * a.Hout + oy) * a.Wout + ox;
          pix2 = (static_cast<long>(b / a.add2_div) * a.Hout + oy) * a.Wout + ox;
        };
        uint4 n1[2], n2[2];
        {
          long pix, pix2;
          pixel(0, pix, pix2);
          load_adds(inside, pix, pix2, cfirst, n1, n2);
        }
        ok = mbar_wait_bounded(&full[buf], use & 1u, HELM_DEVERR_MMA_WAIT) && ok;
        tc::fence_after_sync();
        const bool valid = ok && inside;
#pragma unroll 1
        for (int ph = 0; ph < PH; ++ph) {
          long pix, pix2;
          pixel(ph, pix, pix2);
#pragma unroll 1
          for (int c0 = cfirst; c0 < COUT; c0 += cstep) {
            if (ph > 0 || c0 != cfirst) load_adds(inside, pix, pix2, c0, n1, n2);   // the first came before the wait
            float v[16];
            tc::ld16(tmem + (static_cast<uint32_t>(lane_q * 32) << 16) + buf * Cfg::STEP + mt * Cfg::ACC + ph * COUT +
                         c0,
                     v);
            if (!valid) continue;
            if (a.yraw) {
              float4* o = reinterpret_cast<float4*>(a.yraw + pix * COUT + c0);
#pragma unroll
              for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            }
            if (a.y) {
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                float t = fmaf(v[i], sScale[c0 + i], sShift[c0 + i]);
                v[i] = a.act ? tc::softplus_fast(t) : t;
              }
              if (a.add1) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const bf16* e = reinterpret_cast<const bf16*>(&n1[h]);
#pragma unroll
                  for (int i = 0; i < 8; ++i) v[8 * h + i] += __bfloat162float(e[i]);
                }
              }
              if (a.add2) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const bf16* e = reinterpret_cast<const bf16*>(&n2[h]);
#pragma unroll
                  for (int i = 0; i < 8; ++i) v[8 * h + i] += __bfloat162float(e[i]);
                }
              }
              uint4 o[2];
              __nv_bfloat162* ob = reinterpret_cast<__nv_bfloat162*>(o);
#pragma unroll
              for (int i = 0; i < 8; ++i) ob[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
              uint4* dst = reinterpret_cast<uint4*>(a.y + pix * COUT + c0);
              dst[0] = o[0];
              dst[1] = o[1];
            }
          }
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[buf]);   // this warp's reads of the buffer are done
      }
    }
    gstep += nsteps;
    tc::fence_before_sync();
    ok = __syncthreads_and(ok) != 0;   // uniform; the window is restaged by the next segment
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, Cfg::NCOLS);
}

// ---- weight packing: FP32 master layout -> BF16 [taps][G][COUT][8] ------------------
// conv (mode S1/S2): w[co][ci][ky][kx]; transposed (T1/T2): w[ci][co][ky][kx], flipped;
// 1x1: w[co][ci].
__global__ void k_pack_weights(const float* __restrict__ w, int Ci, int Co, int CS, int taps, int transposed,
                               bf16* __restrict__ out) {
  const int G = CS / 8;
  const long total = static_cast<long>(taps) * G * Co * 8;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const int e = static_cast<int>(i % 8);
    const int co = static_cast<int>((i / 8) % Co);
    const int g = static_cast<int>((i / (8L * Co)) % G);
    const int tap = static_cast<int>(i / (8L * Co * G));
    const int ci = 8 * g + e;
    float v = 0.f;
    if (ci < Ci) {
      if (taps == 1) {
        v = w[static_cast<long>(co) * Ci + ci];
      } else {
        const int ty = tap / 3, tx = tap % 3;
        if (transposed)
          v = w[((static_cast<long>(ci) * Co + co) * 3 + (2 - ty)) * 3 + (2 - tx)];
        else
          v = w[((static_cast<long>(co) * Ci + ci) * 3 + ty) * 3 + tx];
      }
    }
    out[i] = __float2bfloat16_rn(v);
  }
}

template <int CS, int COUT, int TAPS, int PH = 1, int MTR = 2>
int launch_t(const ConvArgs& a0, cudaStream_t st) {
  using Cfg = ConvCfg<CS, COUT, TAPS, PH, MTR>;
  ConvArgs a = a0;
  const int nph = a.mode == HELM_CONV_S2 ? 4 : 1;
  // window budget: one CTA per SM for the heavy-weight layers, two otherwise
  const size_t budget = Cfg::BBYTES > 40 * 1024 ? 200 * 1024 : 100 * 1024;
  const size_t fixed = Cfg::BBYTES + 2 * COUT * 4 + 128;
  const size_t plane_row = static_cast<size_t>(nph) * Cfg::G * 16;
  auto window_rows = [&](int segq) {
    const int nt = Cfg::MT * ((segq + 128 * Cfg::MT - 1) / (128 * Cfg::MT));   // whole steps
    int Lr = 128 * nt + (TAPS == 1 ? 0 : (a.mode == HELM_CONV_S2 || PH == 4 ? a.Po + 2 : 2 * a.Po + 2));
    return Lr | 1;
  };
  int nsm = 0;
  int rc = helm::sm_count(&nsm);
  if (rc) return rc;
  if (TAPS == 1) {
    int tiles = static_cast<int>((budget - std::min(budget, fixed)) / (plane_row * 128));
    tiles = std::max(1, std::min(tiles, 16));
    a.seg_q = 128 * tiles;
  } else {
    // Rows per segment: a tuned value, the most rows that fit below it; otherwise, among
    // the row counts whose window fits the budget, the one with the least work on the
    // busiest SM, counted in MMA steps plus one step of window load and epilogue per
    // segment (ties: more rows).  Large batches take the most rows that fit; small
    // ones split images until every SM has work.
    const int tuned = helm::tune_get(HELM_TUNE_CONV_ROWS, a.Ho, a.B);
    const int rmax = std::min(a.Ho, tuned > 0 ? tuned : 32);
    int R = 1;
    long best = -1;
    for (int r = 1; r <= rmax; ++r) {
      if (r > 1 && fixed + plane_row * window_rows(r * a.Po) > budget) break;
      const long segs = static_cast<long>(a.B) * helm::div_up(a.Ho, r);
      const long steps = helm::div_up(static_cast<long>(r) * a.Po, 128 * Cfg::MT);
      const long cost = helm::div_up(segs, nsm) * (steps + 1);
      if (tuned > 0 || best < 0 || cost <= best) {
        best = cost;
        R = r;
      }
    }
    a.seg_q = R * a.Po;
  }
  a.L = window_rows(a.seg_q);
  size_t smem = fixed + plane_row * a.L;
  if (TAPS != 1 && smem > 227 * 1024) {
    // one output row's window exceeds shared memory (the widest grids): segments of
    // whole MMA steps within a row, the most that fit; the window is addressed on the
    // flattened virtual grid, so a segment may start and end anywhere in a row
    int k = helm::div_up(a.Po, 128 * Cfg::MT);
    while (k > 1 && fixed + plane_row * window_rows(k * 128 * Cfg::MT) > 227 * 1024) --k;
    a.seg_q = k * 128 * Cfg::MT;
    a.L = window_rows(a.seg_q);
    smem = fixed + plane_row * a.L;
  }
  a.segs_per_img = helm::div_up(static_cast<long>(a.Ho) * a.Po, a.seg_q);
  a.nsegs = a.segs_per_img * a.B;
  if (smem > 227 * 1024) {
    helm::set_error("conv: shared memory %zu bytes exceeds the per-CTA limit (grid row too wide)", smem);
    return HELM_ESHAPE;
  }
  static std::atomic<unsigned long long> attr_done{0};
  rc = helm::smem_attr_once(k_conv_tc<CS, COUT, TAPS, PH, MTR>, 227 * 1024, &attr_done);
  if (rc) return rc;
  // resident CTAs per SM: shared memory (228 KB per SM, 1 KB reserved per CTA), TMEM
  // columns (512 per SM) and registers (at most two 288-thread CTAs below 113 registers)
  int per_sm = static_cast<int>((228 * 1024) / (smem + 1024));
  per_sm = std::max(1, std::min({per_sm, 512 / Cfg::NCOLS, 2}));
  const int grid = std::max(1, std::min(a.nsegs, nsm * per_sm));
  HELM_LAUNCH("k_conv_tc", st, k_conv_tc<CS, COUT, TAPS, PH, MTR><<<grid, CONV_THREADS, smem, st>>>(a));
  HELM_CHECK_LAUNCH("k_conv_tc");
  return HELM_OK;
}

}  // namespace

namespace helm {

int pack_conv_weights(const float* w, int Ci, int Co, int taps, int transposed, bf16* out, cudaStream_t st) {
  const int CS = conv_cs(Ci);
  const long total = static_cast<long>(taps) * (CS / 8) * Co * 8;
  HELM_LAUNCH("k_pack_weights", st,
              k_pack_weights<<<std::min<long>(div_up(total, 256), 2048), 256, 0, st>>>(w, Ci, Co, CS, taps,
                                                                                        transposed, out));
  HELM_CHECK_LAUNCH("k_pack_weights");
  return HELM_OK;
}

int conv_tc(const ConvLaunch& c, cudaStream_t st) {
  ConvArgs a;
  a.x = c.x;
  a.B = c.B;
  a.Hi = c.Hi;
  a.Wi = c.Wi;
  a.Cg = c.Ci;
  a.mode = c.mode;
  a.wpk = c.wpk;
  a.scale = c.scale;
  a.shift = c.shift;
  a.act = c.act;
  a.add1 = c.add1;
  a.add2 = c.add2;
  a.add2_div = c.add2_div > 0 ? c.add2_div : 1;
  a.y = c.y;
  a.yraw = c.yraw;
  const int taps = c.taps;
  if (taps == 1) {
    a.Ho = c.Hi;
    a.Wo = c.Wi;
    a.Po = a.Wo;
  } else if (c.mode == HELM_CONV_S2) {
    if ((c.Hi & 1) || (c.Wi & 1)) {
      set_error("conv: stride-2 input must have even size");
      return HELM_ESHAPE;
    }
    a.Ho = c.Hi / 2;
    a.Wo = c.Wi / 2;
    a.Po = a.Wo + 1;
  } else if (c.mode == HELM_CONV_T2) {
    a.Ho = c.Hi;   // virtual grid = input grid (sub-pixel form)
    a.Wo = c.Wi;
    a.Po = a.Wo + 1;
  } else {
    a.Ho = c.Hi;
    a.Wo = c.Wi;
    a.Po = a.Wo + 1;
  }
  a.Hout = c.mode == HELM_CONV_T2 ? 2 * a.Ho : a.Ho;
  a.Wout = c.mode == HELM_CONV_T2 ? 2 * a.Wo : a.Wo;
  const int CS = conv_cs(c.Ci);
  if (c.mode == HELM_CONV_T2 && taps == 9) {
#define HELM_CONV_T2_CASE(cs, co) \
  if (CS == cs && c.Co == co) return launch_t<cs, co, 9, 4>(a, st);
    HELM_CONV_T2_CASE(16, 16)
    HELM_CONV_T2_CASE(32, 16)
    HELM_CONV_T2_CASE(32, 32)
    HELM_CONV_T2_CASE(64, 32)
    HELM_CONV_T2_CASE(64, 64)
#undef HELM_CONV_T2_CASE
    set_error("conv: no transposed tensor-core kernel for Cin=%d Cout=%d", c.Ci, c.Co);
    return HELM_EINVAL;
  }
#define HELM_CONV_CASE(cs, co, tp)                                      \
  if (CS == cs && c.Co == co && taps == tp)                            \
    return c.mode == HELM_CONV_S2 ? launch_t<cs, co, tp, 1, 1>(a, st)  \
                                  : launch_t<cs, co, tp>(a, st);
  HELM_CONV_CASE(16, 16, 9)
  HELM_CONV_CASE(16, 32, 9)
  HELM_CONV_CASE(32, 32, 9)
  HELM_CONV_CASE(32, 16, 9)
  HELM_CONV_CASE(32, 64, 9)
  HELM_CONV_CASE(64, 64, 9)
  HELM_CONV_CASE(64, 32, 9)
  HELM_CONV_CASE(16, 96, 1)
  HELM_CONV_CASE(96, 16, 1)
  HELM_CONV_CASE(32, 192, 1)
  HELM_CONV_CASE(192, 32, 1)
  HELM_CONV_CASE(64, 384, 1)
  HELM_CONV_CASE(384, 64, 1)
#undef HELM_CONV_CASE
  set_error("conv: no tensor-core kernel for Cin=%d Cout=%d taps=%d", c.Ci, c.Co, taps);
  return HELM_EINVAL;
}

}  // namespace helm

extern "C" int helm_conv_bf16(const void* x, int batch, int hi, int wi, int cin, const float* w, int cout, int taps,
                              int mode, const float* scale, const float* shift, int act, const void* add1,
                              const void* add2, int add2_bcast, void* y, float* yraw, void* ws, size_t ws_bytes,
                              void* stream) {
  using namespace helm;
  if (!x || !w || batch <= 0 || hi <= 0 || wi <= 0 || cin <= 0 || cout <= 0 || (taps != 1 && taps != 9) ||
      (!y && !yraw) || mode < 0 || mode > HELM_CONV_T1) {
    set_error("helm_conv_bf16: invalid argument");
    return HELM_EINVAL;
  }
  if ((cin > 2 && cin % 8) || cout % 16) {
    set_error("helm_conv_bf16: cin must be <= 2 or a multiple of 8, cout a multiple of 16");
    return HELM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carve cv(ws, ws_bytes);
  bf16* wpk = cv.take<bf16>(static_cast<size_t>(taps) * conv_cs(cin) * cout);
  if (cv.overflow || !ws) {
    set_error("helm_conv_bf16: workspace too small (need %zu bytes)", cv.off);
    return HELM_EWORKSPACE;
  }
  int rc = pack_conv_weights(w, cin, cout, taps, mode == HELM_CONV_T2 || mode == HELM_CONV_T1, wpk, st);
  if (rc) return rc;
  ConvLaunch c;
  c.x = static_cast<const bf16*>(x);
  c.B = batch;
  c.Hi = hi;
  c.Wi = wi;
  c.Ci = cin;
  c.Co = cout;
  c.taps = taps;
  c.mode = mode == HELM_CONV_T1 ? HELM_CONV_S1 : mode;
  c.wpk = wpk;
  c.scale = scale;
  c.shift = shift;
  c.act = act;
  c.add1 = static_cast<const bf16*>(add1);
  c.add2 = static_cast<const bf16*>(add2);
  c.add2_div = add2_bcast ? batch : 1;
  c.y = static_cast<bf16*>(y);
  c.yraw = yraw;
  return conv_tc(c, st);
}
