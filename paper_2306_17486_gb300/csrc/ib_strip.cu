// Inverted bottleneck of the solver network (MobileNetV2 block of Sections 4.4 and 5.3),
// evaluation mode, for 16 and 32 channels:
//     y = x + BN2(P softplus(BN1(dw3x3(softplus(BN0(E x))))))
// E: 1x1 expansion C -> 6C, dw3x3: depthwise 3x3 with zero padding, P: 1x1 projection.
//
// Work unit: a strip of 30 output columns and SH output rows of one image.  The strip is
// swept downward 4 rows per step, so the expanded activations of a row are computed once
// (the vertical halo costs 2 rows per strip, the horizontal one 2 of 32 pixels).
// One CTA per SM, persistent over units, 17 warps:
//   warp 16 (lane 0)    TMA loads of the 4 x 32-pixel input tiles, the expansion MMAs
//                       (M = 128 pixels, N = 6C, K = C + 16) into two TMEM accumulators,
//                       the projection MMAs (M = 128, N = C, K = 6C + 16);
//   warps 0-7           expansion epilogue: softplus of step t into a ring of 10 pixel
//                       rows of FP16 activations in shared memory (zero outside the
//                       image: the depthwise zero padding); output epilogue: the
//                       projection accumulator + the identity skip -> BF16 y;
//   warps 8-15          depthwise 3x3 of the previous step's 4 output rows from the ring
//                       (a thread: 4 channels of one channel group for 3 or 6 columns,
//                       its 9 x 4 weights read once per phase), + BN1 +
//                       softplus -> FP16 K-major projection operand.
// The two compute groups work on different steps in the same phase; one CTA barrier
// per phase hands the results over.  The control warp waits for the phase's MMAs itself
// before the barrier (the epilogue warps never wait on an mbarrier); its waits, and the
// depthwise warps' one wait per phase, sleep instead of spinning, are bounded and report
// through the device error word.  A step's output is written two phases after its
// depthwise stage (its projection runs in between).
//
// BN0 and BN2 run inside the MMAs: their scales are folded into the packed 1x1 weights
// and their shifts form one more K block, multiplied by a constant operand plane that
// holds 1.0 (pack_ib_folded below); the epilogues then read finished pre-activations.  Arithmetic: BF16 x BF16 -> FP32 expansion MMA; expanded
// activations, depthwise products and sums (weights pre-scaled by BN1's scale) and both
// softplus evaluations in FP16 pairs; FP16 x FP16 -> FP32 projection MMA (the folded
// projection weights in FP16); the skip added in FP32.  softplus(x) = max(x, 0) + log(1 + e),
// e = 2^(-|x| log2 e) from one packed-FP16 exp2, and log(1 + e) = e q(e) with q a
// degree-4 polynomial on [0, 1]: the least-squares Chebyshev fit of log(1 + e)/e,
// relative error 6e-5, below FP16's 2^-11.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "cnn.h"
#include "tc.cuh"

namespace {

using bf16 = __nv_bfloat16;

constexpr int SW = 30;                      // output columns per strip
constexpr int PW = 32;                      // input pixels per row (strip + halo)
constexpr int RB = 4;                       // rows per step
constexpr int NRING = 10;                   // FP16 activation rows held (6 read + 4 written)
constexpr int NA = 8;                       // epilogue warps 0..7 (TMEM lane quarter = warp % 4)
constexpr int NB = 8;                       // depthwise warps 8..15
constexpr int CTRL = NA + NB;               // warp 16
constexpr int THREADS = (NA + NB + 1) * 32;  // 544
constexpr int NBT = 240;                    // depthwise threads with work
constexpr int PLANE = RB * PW * 16;         // one 8-channel operand plane of 128 pixels

template <int C>
struct SCfg {
  static constexpr int E = 6 * C, G = C / 8, EG = E / 8;
  static constexpr int NXBUF = C == 16 ? 3 : 2;       // input tiles in flight
  static constexpr int TPC = NBT / (2 * EG);           // depthwise threads per (group, half)
  static constexpr int COLS = SW / TPC;                // columns per depthwise thread
  static constexpr int PITCH = E + 8;  // halves per ring pixel: consecutive pixels land on distinct banks
  static constexpr size_t RING = static_cast<size_t>(NRING) * PW * PITCH * 2;
  static constexpr size_t PROJ = static_cast<size_t>(EG) * PLANE;
  static constexpr size_t XB = static_cast<size_t>(G) * PLANE;
  static constexpr size_t WE = static_cast<size_t>(G + 2) * E * 16;   // folded expansion weights + shift block
  static constexpr size_t WP = static_cast<size_t>(EG + 2) * C * 16;  // folded projection weights + shift block
  static constexpr size_t O_RING = 0;
  static constexpr size_t O_PROJ = O_RING + RING;
  static constexpr size_t O_ONES = (O_PROJ + PROJ + 127) & ~size_t(127);
  static constexpr size_t WDW = static_cast<size_t>(EG) * 9 * 16;     // depthwise weights x BN1 scale, FP16
  static constexpr size_t O_X = O_ONES + PLANE;
  static constexpr size_t O_WE = O_X + NXBUF * XB;
  static constexpr size_t O_WP = O_WE + WE;
  static constexpr size_t O_WDW = O_WP + WP;
  static constexpr size_t O_B1 = O_WDW + WDW;                            // BN1 shift, FP16 [E]
  static constexpr size_t O_BAR = (O_B1 + static_cast<size_t>(E) * 2 + 15) & ~size_t(15);
  static constexpr size_t SMEM = O_BAR + 8 * sizeof(uint64_t) + 16 + 128;   // + alignment slack
  static constexpr uint32_t TCOLS = (2 * E + 2 * C) <= 256 ? 256u : 512u;
  static_assert(C == 16 || C == 32, "strip kernel shapes");
  static_assert(TPC * 2 * EG == NBT && COLS * TPC == SW, "depthwise thread map");
  static_assert(2 * E + 2 * C <= 512, "TMEM columns");
  static_assert(SMEM <= 232448, "shared memory per block");
};

struct StripArgs {
  CUtensorMap maps[4];  // one per 8-channel input group
  const bf16* x;
  bf16* y;
  const bf16* wef;      // folded expansion weights [G + 2][E][8]
  const __half* wpf;    // folded projection weights [E/8 + 2][C][8], FP16
  const float* wdw;     // depthwise weights [E][9]
  const float* bn1;     // folded BN after the depthwise stage: scale [E] then shift [E]
  int B, H, W;
  int nsx, nsy, SH, units;
};

// packed-FP16 arithmetic on 32-bit registers
__device__ __forceinline__ uint32_t h2fma(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t h2const(float v) {
  const __half2 h = __float2half2_rn(v);
  return *reinterpret_cast<const uint32_t*>(&h);
}
// softplus of two FP16 values: max(x, 0) + e q(e), e = 2^(-|x| log2 e), q the degree-4
// least-squares Chebyshev fit of log(1 + e)/e on [0, 1]
__device__ __forceinline__ uint32_t softplus_u(uint32_t x) {
  uint32_t ax, t, e, mx;
  asm("abs.f16x2 %0, %1;" : "=r"(ax) : "r"(x));
  asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(t) : "r"(ax), "r"(h2const(-1.4426950408889634f)));
  asm("ex2.approx.f16x2 %0, %1;" : "=r"(e) : "r"(t));
  uint32_t q = h2fma(h2const(0.04155111f), e, h2const(-0.15783838f));
  q = h2fma(q, e, h2const(0.3065611f));
  q = h2fma(q, e, h2const(-0.49703084f));
  q = h2fma(q, e, h2const(0.99994499f));
  asm("max.f16x2 %0, %1, %2;" : "=r"(mx) : "r"(x), "r"(0u));
  return h2fma(e, q, mx);
}


// tcgen05.ld of 16 columns without waiting; tmem_wait16 waits for every load of the
// thread and ties the 16 registers to the wait, so no use is scheduled before it
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}
// 8 columns, load and wait
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void decode_unit(const StripArgs& a, int ul, int& b, int& x0, int& y0) {
  const int gu = static_cast<int>(blockIdx.x) + ul * static_cast<int>(gridDim.x);
  const int per = a.nsx * a.nsy;
  b = gu / per;
  const int rem = gu - b * per;
  y0 = (rem / a.nsx) * a.SH;
  x0 = (rem % a.nsx) * SW;
}

template <int C>
__global__ void __launch_bounds__(THREADS, 1) k_ib_strip(const __grid_constant__ StripArgs a) {
  using Cfg = SCfg<C>;
  constexpr int E = Cfg::E, G = Cfg::G, EG = Cfg::EG, PITCH = Cfg::PITCH, NXBUF = Cfg::NXBUF;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  __half* ring = reinterpret_cast<__half*>(smem + Cfg::O_RING);
  uint8_t* proj = smem + Cfg::O_PROJ;
  uint8_t* xbuf = smem + Cfg::O_X;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Cfg::O_BAR);   // xfull[<=3], expdone[2], projdone[2]
  uint64_t* xfull = bar;
  uint64_t* expdone = bar + 3;
  uint64_t* projdone = bar + 5;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- set-up: TMEM, weights, constant operand planes, barriers ----
  if (warp == 0) tc::tmem_alloc(tslot, Cfg::TCOLS);
  {
    const uint4* s1 = reinterpret_cast<const uint4*>(a.wef);
    const uint4* s2 = reinterpret_cast<const uint4*>(a.wpf);
    uint4* d1 = reinterpret_cast<uint4*>(smem + Cfg::O_WE);
    uint4* d2 = reinterpret_cast<uint4*>(smem + Cfg::O_WP);
    for (int i = tid; i < static_cast<int>(Cfg::WE / 16); i += THREADS) d1[i] = s1[i];
    for (int i = tid; i < static_cast<int>(Cfg::WP / 16); i += THREADS) d2[i] = s2[i];
    // constant operand plane multiplying the shift rows of the folded weights: channel 0
    // holds BF16 1.0 (the expansion's shift row), channel 1 FP16 1.0 (the projection's);
    // every other weight of the shift K block is zero, so each MMA reads its own 1.0, and
    // the block's second 8-channel group reads the same plane again against zeros
    uint4* ones = reinterpret_cast<uint4*>(smem + Cfg::O_ONES);
    for (int i = tid; i < PLANE / 16; i += THREADS) ones[i] = make_uint4(0x3C003F80u, 0u, 0u, 0u);
    __half* wh = reinterpret_cast<__half*>(smem + Cfg::O_WDW);
    for (int i = tid; i < E * 9; i += THREADS) {
      const int e = i / 9, k = i - 9 * e;
      wh[((e >> 3) * 9 + k) * 8 + (e & 7)] = __float2half_rn(a.wdw[i] * a.bn1[e]);
    }
    __half* b1h = reinterpret_cast<__half*>(smem + Cfg::O_B1);
    for (int e = tid; e < E; e += THREADS) b1h[e] = __float2half_rn(a.bn1[E + e]);
    uint4* pz = reinterpret_cast<uint4*>(proj);
    for (int i = tid; i < static_cast<int>(Cfg::PROJ / 16); i += THREADS) pz[i] = make_uint4(0, 0, 0, 0);
  }
  if (tid == 0) {
    for (int i = 0; i < 7; ++i) mbar_init(&bar[i], 1);
    fence_mbar_init();
  }
  // depthwise threads: one 4-channel half of one channel group (its weights, read once
  // per phase through L1, are the FP16 products with BN1's scale)
  const int bt = tid - NA * 32;
  const bool bthread = warp >= NA && warp < CTRL && bt < NBT;
  const int b_h = bt & 1, b_u = bt >> 1;
  const int b_eg = bthread ? b_u / Cfg::TPC : 0, b_cl = bthread ? b_u % Cfg::TPC : 0;
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  const int S = a.SH / RB;
  const int nu = static_cast<int>(blockIdx.x) < a.units ? (a.units - 1 - static_cast<int>(blockIdx.x)) / gridDim.x + 1 : 0;
  const int Texp = nu * (S + 1);

  constexpr uint32_t idesc_e = tc::idesc_bf16(128, E);
  constexpr uint32_t idesc_p = tc::idesc_f16(128, C);   // FP16 depthwise output x FP16 weights
  const uint32_t xbuf_u = smem_u32(xbuf), proj_u = smem_u32(proj), ones_u = smem_u32(smem + Cfg::O_ONES);
  const uint32_t we_u = smem_u32(smem + Cfg::O_WE), wp_u = smem_u32(smem + Cfg::O_WP);
  bool ok = true;
  // control-lane bookkeeping (meaningful in warp CTRL, lane 0 only)
  int tma_issued = 0, tma_waited = 0, last_exp = -1, last_proj = -1;

  auto issue_tma = [&](int t) {
    int b, x0, y0;
    decode_unit(a, t / (S + 1), b, x0, y0);
    const int k = t % (S + 1);
    uint64_t* fb = &xfull[t % NXBUF];
    mbar_arrive_expect_tx(fb, static_cast<uint32_t>(G * PLANE));
    uint8_t* dst = xbuf + (t % NXBUF) * Cfg::XB;
#pragma unroll
    for (int g = 0; g < G; ++g) tma_load_4d(dst + g * PLANE, &a.maps[g], 0, x0 - 1, y0 + RB * k - 3, b, fb);
    ++tma_issued;
  };
  auto issue_exp = [&](int t) {
    ok = mbar_wait_sleep(&xfull[t % NXBUF], (t / NXBUF) & 1, HELM_DEVERR_TMA_WAIT) && ok;
    ++tma_waited;
    if (!ok) return;
    tc::fence_after_sync();
    const uint32_t xb = xbuf_u + static_cast<uint32_t>((t % NXBUF) * Cfg::XB);
    const uint32_t d = tmem + (t & 1) * E;
#pragma unroll
    for (int kc = 0; kc < C / 16; ++kc)
      tc::mma_bf16(d, tc::sdesc(xb + kc * 2 * PLANE, PLANE, 128), tc::sdesc(we_u + kc * 2 * E * 16, E * 16, 128),
                   idesc_e, kc > 0);
    // the BN0 shift: constant plane (channel 0 = 1) times the shift row
    tc::mma_bf16(d, tc::sdesc(ones_u, 0, 128), tc::sdesc(we_u + G * E * 16, E * 16, 128), idesc_e, true);
    tc::commit(&expdone[t & 1]);
    last_exp = t;
  };
  auto issue_proj = [&](int dd) {
    const uint32_t d = tmem + 2 * E + (dd & 1) * C;
#pragma unroll
    for (int kc = 0; kc < E / 16; ++kc)
      tc::mma_bf16(d, tc::sdesc(proj_u + kc * 2 * PLANE, PLANE, 128), tc::sdesc(wp_u + kc * 2 * C * 16, C * 16, 128),
                   idesc_p, kc > 0);
    tc::mma_bf16(d, tc::sdesc(ones_u, 0, 128), tc::sdesc(wp_u + EG * C * 16, C * 16, 128), idesc_p, true);
    tc::commit(&projdone[dd & 1]);
    last_proj = dd;
  };

  if (warp == CTRL && lane == 0 && Texp > 0) {
    for (int t = 0; t < (Texp < NXBUF ? Texp : NXBUF); ++t) issue_tma(t);
    issue_exp(0);
    ok = mbar_wait_sleep(&expdone[0], 0, HELM_DEVERR_MMA_WAIT) && ok;
  }
  // phase 0 reads the expansion of step 0, completed above
  tc::fence_before_sync();
  ok = __syncthreads_and(ok) != 0;
  tc::fence_after_sync();

  constexpr int CH = C / 2;    // output channels per epilogue thread
  uint4 skip_cur[CH / 8], skip_next[CH / 8];   // epilogue warps: skip values (x) of their pixel
#pragma unroll
  for (int h = 0; h < CH / 8; ++h) skip_cur[h] = skip_next[h] = make_uint4(0, 0, 0, 0);
  // depthwise steps of the previous phase (its projection runs in this phase) and of the
  // phase before (its output is written in this phase); -1: none
  int dcount = 0, dprev = -1, dprev2 = -1;
  int dprev_unit = 0, dprev_d = 0, dprev2_unit = 0, dprev2_d = 0;
  for (int t = 0; t < Texp + 3; ++t) {
    // the depthwise step of this phase: unit (t-1)/(S+1), rows 4d.., d = (t-1)%(S+1) - 1
    const bool has_dw = t >= 2 && t <= Texp && ((t - 1) % (S + 1)) >= 1;
    if (warp == CTRL) {
      // Issues this phase's tensor-core work and waits for it before the phase barrier,
      // so the other warps never wait on an mbarrier for it: the projection of the
      // previous phase's depthwise output, the expansion of step t + 1 (its tile loaded
      // two or three phases ago), the tile load of step t + NXBUF into the buffer of
      // step t, whose expansion completed in the previous phase.
      if (lane == 0) {
        tc::fence_after_sync();
        if (dprev >= 0 && ok) issue_proj(dprev);
        if (t + 1 < Texp && ok) issue_exp(t + 1);
        if (t + NXBUF < Texp && ok) issue_tma(t + NXBUF);
        if (t + 1 < Texp && ok) ok = mbar_wait_sleep(&expdone[(t + 1) & 1], ((t + 1) >> 1) & 1, HELM_DEVERR_MMA_WAIT);
        if (dprev >= 0 && ok) ok = mbar_wait_sleep(&projdone[dprev & 1], (dprev >> 1) & 1, HELM_DEVERR_MMA_WAIT);
      }
      __syncwarp();
    } else if (warp < NA) {
      const int q = warp & 3, hf = warp >> 2;
      // the skip values of the next phase's output epilogue (the previous phase's
      // depthwise step): loaded now, used a phase later
      if (dprev >= 0) {
        int b, x0, y0;
        decode_unit(a, dprev_unit, b, x0, y0);
        const int oy = y0 + RB * dprev_d + q, ox = x0 + lane;
        if (lane < SW && ox < a.W && oy < a.H) {
          const uint4* sk = reinterpret_cast<const uint4*>(a.x + ((static_cast<long>(b) * a.H + oy) * a.W + ox) * C +
                                                           hf * CH);
#pragma unroll
          for (int h = 0; h < CH / 8; ++h) skip_next[h] = sk[h];
        }
      }
      // ---- expansion epilogue of step t: softplus -> ring rows (its MMA completed) ----
      if (t < Texp) {
        int b, x0, y0;
        decode_unit(a, t / (S + 1), b, x0, y0);
        const int k = t % (S + 1);
        if (k > 0 || q >= 2) {   // step 0 of a unit: only the two rows above the segment
          const int iy = y0 + RB * k - 3 + q, ix = x0 - 1 + lane;
          const bool in = iy >= 0 && iy < a.H && ix >= 0 && ix < a.W;
          const int slot = (RB * t + q) % NRING;
          __half* dst = ring + (slot * PW + lane) * PITCH + hf * (E / 2);
          const uint32_t ta = tmem + (static_cast<uint32_t>(32 * q) << 16) + (t & 1) * E + hf * (E / 2);
          // several 16-column loads per wait: the TMEM latency is paid once per round
          constexpr int NL = C == 16 ? 3 : 2;
#pragma unroll 1
          for (int c1 = 0; c1 < E / 2; c1 += 16 * NL) {
            uint32_t r[NL][16];
#pragma unroll
            for (int j = 0; j < NL; ++j) tmem_ld16_issue(ta + c1 + 16 * j, r[j]);
#pragma unroll
            for (int j = 0; j < NL; ++j) tmem_wait16(r[j]);
#pragma unroll
            for (int j = 0; j < NL; ++j) {
              uint4 o[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
              if (in) {
                uint32_t* ou = reinterpret_cast<uint32_t*>(o);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                  const __half2 hx = __floats2half2_rn(__uint_as_float(r[j][2 * i]), __uint_as_float(r[j][2 * i + 1]));
                  ou[i] = softplus_u(*reinterpret_cast<const uint32_t*>(&hx));
                }
              }
              uint4* d4 = reinterpret_cast<uint4*>(dst + c1 + 16 * j);
              d4[0] = o[0];
              d4[1] = o[1];
            }
          }
        }
      }
      // ---- output epilogue of the step before last (its projection completed) ----
      if (dprev2 >= 0) {
        int b, x0, y0;
        decode_unit(a, dprev2_unit, b, x0, y0);
        const int oy = y0 + RB * dprev2_d + q, ox = x0 + lane;
        const uint32_t ta = tmem + (static_cast<uint32_t>(32 * q) << 16) + 2 * E + (dprev2 & 1) * C + hf * CH;
        float v[CH];
        if constexpr (CH == 8) tmem_ld8(ta, v);
        else tc::ld16(ta, v);
        if (lane < SW && ox < a.W && oy < a.H) {
          const long pix = (static_cast<long>(b) * a.H + oy) * a.W + ox;
          uint4* yo = reinterpret_cast<uint4*>(a.y + pix * C + hf * CH);
#pragma unroll
          for (int h = 0; h < CH / 8; ++h) {
            const __nv_bfloat162* s2 = reinterpret_cast<const __nv_bfloat162*>(&skip_cur[h]);
            uint4 o;
            __nv_bfloat162* ob = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float2 f = __bfloat1622float2(s2[e]);
              ob[e] = __floats2bfloat162_rn(v[8 * h + 2 * e] + f.x, v[8 * h + 2 * e + 1] + f.y);
            }
            yo[h] = o;
          }
        }
      }
#pragma unroll
      for (int h = 0; h < CH / 8; ++h) skip_cur[h] = skip_next[h];
    } else if (has_dw && bthread) {
      // ---- depthwise 3x3 of 4 output rows + BN1 + softplus -> projection operand ----
      // lane pairs share a pixel: a half-warp reads 8 pixels x 16 B (conflict-free with
      // the ring's pitch) and writes 128 contiguous bytes of the operand
      int slot0 = RB * t - 6;   // running index of the first ring row read (t >= 2)
      slot0 %= NRING;
      uint32_t dw[9][2], db1[2];
      {
        const uint32_t wa = smem_u32(smem + Cfg::O_WDW) + (b_eg * 9) * 16 + b_h * 8;
#pragma unroll
        for (int k = 0; k < 9; ++k)
          asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(dw[k][0]), "=r"(dw[k][1]) : "r"(wa + k * 16));
        asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];"
                     : "=r"(db1[0]), "=r"(db1[1])
                     : "r"(smem_u32(smem + Cfg::O_B1) + (b_eg * 8 + b_h * 4) * 2));
      }
      // the projection MMA of the previous step (issued at this phase's start) reads the
      // operand: its completion is awaited just before the first store
      bool need_wait = dprev >= 0;
      const uint32_t cbase = smem_u32(ring + b_eg * 8 + b_h * 4);
#pragma unroll 1
      for (int ci = 0; ci < Cfg::COLS; ++ci) {
        const int xc = b_cl + ci * Cfg::TPC;
        uint32_t acc[RB][2];
#pragma unroll
        for (int o = 0; o < RB; ++o) acc[o][0] = acc[o][1] = 0u;
#pragma unroll
        for (int rr = 0; rr < RB + 2; ++rr) {
          int slot = slot0 + rr;
          slot = slot >= NRING ? slot - NRING : slot;
          const uint32_t rp = cbase + static_cast<uint32_t>(((slot * PW + xc) * PITCH) * 2);
          uint32_t hv[3][2];
#pragma unroll
          for (int dx = 0; dx < 3; ++dx)
            asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(hv[dx][0]), "=r"(hv[dx][1]) : "r"(rp + dx * PITCH * 2));
#pragma unroll
          for (int o = 0; o < RB; ++o) {
            const int dy = rr - o;
            if (dy < 0 || dy > 2) continue;
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
              acc[o][0] = h2fma(dw[dy * 3 + dx][0], hv[dx][0], acc[o][0]);
              acc[o][1] = h2fma(dw[dy * 3 + dx][1], hv[dx][1], acc[o][1]);
            }
          }
        }
        if (need_wait) {
          ok = mbar_wait_sleep(&projdone[dprev & 1], (dprev >> 1) & 1, HELM_DEVERR_MMA_WAIT) && ok;
          need_wait = false;
        }
#pragma unroll
        for (int o = 0; o < RB; ++o) {
          uint32_t ob[2];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            uint32_t v;
            asm("add.rn.f16x2 %0, %1, %2;" : "=r"(v) : "r"(acc[o][e]), "r"(db1[e]));
            ob[e] = softplus_u(v);
          }
          asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(smem_u32(proj) + (b_eg * 128 + o * 32 + xc) * 16 + b_h * 8),
                       "r"(ob[0]), "r"(ob[1])
                       : "memory");
        }
      }
      tc::fence_proxy_async();
    }
    tc::fence_before_sync();
    ok = __syncthreads_and(ok) != 0;
    tc::fence_after_sync();   // TMEM reads of the next phase follow the MMAs waited for above
    if (!ok) break;
    dprev2 = dprev;
    dprev2_unit = dprev_unit;
    dprev2_d = dprev_d;
    if (has_dw) {
      dprev = dcount++;
      dprev_unit = (t - 1) / (S + 1);
      dprev_d = (t - 1) % (S + 1) - 1;
    } else {
      dprev = -1;
    }
  }
  // ---- drain: nothing of this CTA may still write shared memory or TMEM ----
  if (warp == CTRL && lane == 0) {
    for (int t = tma_waited; t < tma_issued; ++t)
      mbar_wait_sleep(&xfull[t % NXBUF], (t / NXBUF) & 1, HELM_DEVERR_TMA_WAIT);
    if (last_exp >= 0) mbar_wait_sleep(&expdone[last_exp & 1], (last_exp >> 1) & 1, HELM_DEVERR_MMA_WAIT);
    if (last_proj >= 0) mbar_wait_sleep(&projdone[last_proj & 1], (last_proj >> 1) & 1, HELM_DEVERR_MMA_WAIT);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, Cfg::TCOLS);
}

// segment height: the multiple of 4 that minimises the per-CTA phase count
int choose_sh(int B, int H, int nsx, int grid) {
  int best = 4, best_cost = 1 << 30;
  const int hmax = ((H + 3) / 4) * 4;
  for (int sh = 8; sh <= hmax; sh += 4) {
    const long units = static_cast<long>(B) * nsx * ((H + sh - 1) / sh);
    const long rounds = (units + grid - 1) / grid;
    const long cost = rounds * (sh / 4 + 1);
    if (cost < best_cost || (cost == best_cost && sh > best)) {
      best_cost = static_cast<int>(cost);
      best = sh;
    }
  }
  return best;
}

template <int C>
int launch_strip(const helm::IbLaunch& l, cudaStream_t st) {
  using Cfg = SCfg<C>;
  StripArgs a{};
  for (int g = 0; g < C / 8; ++g) {
    int rc = helm::make_bf16_nhwc_map(&a.maps[g], l.x + 8 * g, C, l.W, l.H, l.B, PW, RB);
    if (rc) return rc;
  }
  a.x = l.x;
  a.y = l.y;
  a.wef = l.wef;
  a.wpf = static_cast<const __half*>(l.wpf);
  a.wdw = l.wdw;
  a.bn1 = l.bn1;
  a.B = l.B;
  a.H = l.H;
  a.W = l.W;
  int nsm = 0;
  int rc = helm::sm_count(&nsm);
  if (rc) return rc;
  a.nsx = helm::div_up(l.W, SW);
  const int tuned = helm::tune_get(HELM_TUNE_IB_SH, l.H, l.B);
  a.SH = tuned > 0 ? std::min(std::max(4, (tuned / 4) * 4), ((l.H + 3) / 4) * 4) : choose_sh(l.B, l.H, a.nsx, nsm);
  a.nsy = helm::div_up(l.H, a.SH);
  const long units = static_cast<long>(l.B) * a.nsx * a.nsy;
  if (units > (1L << 30)) {
    helm::set_error("inverted bottleneck: %ld work units exceed the kernel's index range", units);
    return HELM_ESHAPE;
  }
  a.units = static_cast<int>(units);
  static std::atomic<unsigned long long> attr_done{0};
  if ((rc = helm::smem_attr_once(k_ib_strip<C>, static_cast<int>(Cfg::SMEM), &attr_done))) return rc;
  const int grid = static_cast<int>(std::min<long>(units, nsm));
  HELM_LAUNCH("k_ib_strip", st, k_ib_strip<C><<<grid, THREADS, Cfg::SMEM, st>>>(a));
  HELM_CHECK_LAUNCH("k_ib_strip");
  return HELM_OK;
}

// out[g][n][j] ([Ci/8 + 2][Co][8], BF16 or FP16 bits): g < Ci/8: w[n][8g + j] * scale[n];
// g = Ci/8: shift[n] in channel j = 0 (BF16) or 1 (FP16), zero elsewhere; g = Ci/8 + 1:
// zero.  Against an operand whose extra channel 0 (BF16) or 1 (FP16) is 1.0 the MMA
// computes scale * (w x) + shift.
__global__ void k_pack_folded(const float* __restrict__ w, const float* __restrict__ fold, int Ci, int Co, int fp16,
                              unsigned short* __restrict__ out) {
  const int G = Ci / 8 + 2;
  const long total = static_cast<long>(G) * Co * 8;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const int j = static_cast<int>(i % 8), n = static_cast<int>((i / 8) % Co), g = static_cast<int>(i / (8L * Co));
    float v = 0.f;
    if (g < Ci / 8) v = w[static_cast<long>(n) * Ci + 8 * g + j] * fold[n];
    else if (g == Ci / 8 && j == (fp16 ? 1 : 0)) v = fold[Co + n];
    out[i] = fp16 ? __half_as_ushort(__float2half_rn(v)) : __bfloat16_as_ushort(__float2bfloat16_rn(v));
  }
}

}  // namespace

namespace helm {

size_t ib_folded_elems(int Ci, int Co) { return static_cast<size_t>(Ci / 8 + 2) * Co * 8; }

int pack_ib_folded(const float* w, const float* fold, int Ci, int Co, int fp16, void* out, cudaStream_t st) {
  if (Ci % 16) {
    set_error("folded 1x1 packing: %d input channels (a multiple of 16 is needed)", Ci);
    return HELM_EINVAL;
  }
  const long total = static_cast<long>(ib_folded_elems(Ci, Co));
  HELM_LAUNCH("k_pack_folded", st,
              k_pack_folded<<<static_cast<int>(std::min<long>(div_up(total, 256), 1024)), 256, 0, st>>>(
                  w, fold, Ci, Co, fp16, static_cast<unsigned short*>(out)));
  HELM_CHECK_LAUNCH("k_pack_folded");
  return HELM_OK;
}

// 16 and 32 channels with folded weights: the strip kernel; otherwise HELM_EINVAL
int ib_strip(const IbLaunch& l, cudaStream_t st) {
  if (l.expansion != 6 || !l.wef || !l.wpf) return HELM_EINVAL;
  if ((reinterpret_cast<uintptr_t>(l.x) & 15) || (reinterpret_cast<uintptr_t>(l.y) & 15)) return HELM_EINVAL;
  switch (l.C) {
    case 16: return launch_strip<16>(l, st);
    case 32: return launch_strip<32>(l, st);
    default: return HELM_EINVAL;
  }
}

}  // namespace helm
