// Shifted-Laplacian V(1,1) cycle (Section 3.2, Algorithm 1 applied recursively,
// Eq. 4, 6, 8; Section 3.4: one pre- and one post-relaxation, an inexact coarsest
// solve by a few Jacobi-preconditioned GMRES iterations).
//
// Per level l (h_l^2-scaled operator S_l = 4 - neighbours - m_l, D_l = 4 - m_l, the
// damped inverse diagonal dinv_l = omega_J / D_l stored by the problem):
//   pre-sweep from zero   u  = dinv_l r                       (pointwise)
//   coarse right side     rc = 4 I_h^H (r - S_l u)            (Eq. 6, h^2 scaling)
//   coarse correction     ec = V_{l+1}(rc)  or the coarsest GMRES solve
//   prolong and correct   u2 = u + I_H^h ec                   (Eq. 8)
//   post-sweep            z  = u2 + dinv_l (r - S_l u2)
// Since D_l dinv_l = omega_J, the kernels use the equivalent forms
//   r - S_l u  = (1 - omega_J) r + sum_neighbours u
//   z          = (1 - omega_J) u2 + dinv_l (r + sum_neighbours u2)
// which need no mass array.
//
// Kernels (the legs stage the fine grid into shared memory with TMA tiled loads whose
// out-of-range elements are zero-filled, which is the Dirichlet padding):
//   k_resid_restrict : u, the residual and the full-weighting restriction fused; u is
//                      recomputed from r, never stored.
//   k_prolong_smooth : u recomputed from r, prolongation, correction and the post-sweep
//                      fused.
//   k_coarse_gmres_cluster : the coarsest-grid GMRES for one right-hand side on a
//                      cluster of 8 CTAs; each CTA keeps its slab of rows of the
//                      Krylov basis in shared memory, reads the neighbouring slabs'
//                      boundary rows through distributed shared memory, and the inner
//                      products are cluster-wide reductions (classical Gram-Schmidt
//                      twice, FP32 Hessenberg and Givens, computed redundantly and
//                      identically by every CTA of the cluster).
//   k_coarse_gmres   : the same algorithm on one CTA with the basis in global memory
//                      (FP64 Hessenberg), for coarsest grids whose basis does not fit
//                      the cluster.
#include <cooperative_groups.h>

#include <type_traits>

#include "problem.h"

namespace cg = cooperative_groups;

namespace {

// ---- the two V-cycle legs -------------------------------------------------------------
// Both legs stream the fine grid in strips 64 values wide (two per lane of a warp).  A
// CTA takes a work unit = one strip for 4 right-hand sides: one TMA load brings the
// strip of dinv (one array per level, shared by all right-hand sides) and one per active
// right-hand side brings its strip of r (and, for the prolongation, of the coarse
// correction), all zero-filled outside the grid (the Dirichlet padding).  Two warps
// share a right-hand side's strip, one per half (band) of its rows, and walk their
// rows in registers: horizontal neighbours come from warp shuffles, vertical ones from
// the previous rows' registers, so every value is read once from shared memory (the
// bands overlap by the three rows of stencil context).  The row loops are unrolled
// completely, which leaves them without branches.  CTAs are persistent, take units in
// a strided order and keep the next unit's loads in flight while they process the
// current one (two buffers).
constexpr int VL_RHS = 4;                       // right-hand sides per unit
constexpr int VL_CTAS = 2;                      // CTAs per SM (shared memory)
constexpr int VL_WARPS = 2 * VL_RHS;            // two bands per right-hand side
constexpr int VL_THREADS = 32 * VL_WARPS;
constexpr int VS_W = 64;                        // strip width (fine values)
constexpr int RC_TW = 30;                       // restriction: coarse columns per strip
constexpr int RC_TH = 8;                        //   coarse rows per strip
constexpr int RS_H = 2 * RC_TH + 3;             //   strip rows: fine rows 2 J0 - 2 .. 2 J1 + 2
constexpr int RC_HB = RC_TH / 2;                //   coarse rows per band
constexpr int RB_H = 2 * RC_HB + 3;             //   strip rows a band walks
constexpr int PS_TW = 60;                       // prolongation: output columns per strip
constexpr int PS_TH = 12;                       //   output rows per strip
constexpr int PS_H = PS_TH + 2;                 //   strip rows: one halo row above and below
constexpr int PS_HB = PS_TH / 2;                //   output rows per band
constexpr int PB_H = PS_HB + 2;                 //   strip rows a band walks
constexpr int PE_W = 36;                        //   coarse strip: columns x0/2 - 2 .. x0/2 + 33
constexpr int PE_H = PS_TH / 2 + 3;             //   coarse rows y0/2 - 1 .. y0/2 + PS_TH/2 + 1
constexpr int RS_TILE = VS_W * RS_H;            // float2 per strip
constexpr int PS_TILE = VS_W * PS_H;
constexpr int PE_TILE = (PE_W * PE_H + 15) / 16 * 16;   // padded to 128 bytes
constexpr int RS_BUF = (1 + VL_RHS) * RS_TILE;                     // dinv + r strips
constexpr int PS_BUF = (1 + VL_RHS) * PS_TILE + VL_RHS * PE_TILE;  // dinv + r + ec strips
constexpr size_t RS_SMEM = 2 * RS_BUF * sizeof(float2) + 128;   // + alignment slack
constexpr size_t PS_SMEM = 2 * PS_BUF * sizeof(float2) + 128;
static_assert(VL_CTAS * (RS_SMEM + 1024) <= 228 * 1024 && VL_CTAS * (PS_SMEM + 1024) <= 228 * 1024,
              "two buffers per CTA, VL_CTAS CTAs per SM");
static_assert(PS_HB % 2 == 0, "a band starts on an odd fine row");
static_assert((RS_TILE * sizeof(float2)) % 128 == 0 && (PS_TILE * sizeof(float2)) % 128 == 0,
              "strips start on 128-byte boundaries");

// The dynamic shared memory of a leg kernel, rounded up to the 128-byte boundary that
// TMA destinations need (the launch asks for 128 bytes more than the buffers take).
__device__ __forceinline__ float2* aligned_dyn_smem() {
  extern __shared__ unsigned char vl_smem_raw[];
  return reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(vl_smem_raw) + 127) & ~static_cast<uintptr_t>(127));
}

__device__ __forceinline__ void fence_async_proxy() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ float2 shfl_up1(float2 v) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ float2 shfl_down1(float2 v) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}

// Right-hand side of warp w in group g is processed when it exists and is not masked.
__device__ __forceinline__ bool rhs_on(int b, int batch, const int* active) {
  return b < batch && (!active || active[b]);
}
__device__ __forceinline__ long next_unit(long u, long stride, long units, long per_group, int batch,
                                          const int* active) {
  for (; u < units; u += stride) {
    const int b0 = static_cast<int>(u / per_group) * VL_RHS;
    for (int w = 0; w < VL_RHS; ++w)
      if (rhs_on(b0 + w, batch, active)) return u;
  }
  return u;
}

// Persistent double-buffered walk of a CTA over its units: issue(u, k) (thread 0) starts
// the loads of unit u into buffer k and arms bars[k]; work(u, k) runs on every thread.
// A load wait that runs out anywhere in the CTA flags the device error word; the CTA
// then waits (bounded) for its other buffer's loads if any are in flight and ends.
template <class Issue, class Work>
__device__ __forceinline__ void cta_units(uint64_t* bars, long units, long per_group, int batch, const int* active,
                                          Issue issue, Work work) {
  const long stride = gridDim.x;
  long u = next_unit(blockIdx.x, stride, units, per_group, batch, active);
  uint32_t ph0 = 0, ph1 = 0;
  int k = 0;
  if (u < units && threadIdx.x == 0) issue(u, 0);
  while (u < units) {
    const long un = next_unit(u + stride, stride, units, per_group, batch, active);
    if (un < units && threadIdx.x == 0) {
      fence_async_proxy();  // the buffer was last read through the generic proxy
      issue(un, k ^ 1);
    }
    uint32_t& ph = k ? ph1 : ph0;
    const bool ok = __syncthreads_and(mbar_wait_bounded(&bars[k], ph, HELM_DEVERR_TMA_WAIT));
    if (!ok) {
      if (un < units) mbar_wait_bounded(&bars[k ^ 1], k ? ph0 : ph1, HELM_DEVERR_TMA_WAIT);
      return;
    }
    ph ^= 1;
    work(u, k);
    __syncthreads();  // every warp is done with buffer k before it is loaded again
    u = un;
    k ^= 1;
  }
}

// Residual and full-weighting restriction (Eq. 6 with the h^2 scaling of the coarse
// operator): u = dinv r (the pre-sweep from zero), q = r - S u = (1 - omega) r + the sum
// of the neighbours' u, rc = 4 I_h^H q with the [1 2 1] x [1 2 1] / 16 stencil.
// Unit: (group of VL_RHS right-hand sides, band of RC_TH coarse rows, strip of RC_TW coarse
// columns); lane l of a warp holds fine columns 2 l, 2 l + 1 of the strip and produces
// coarse column l - 1 (lanes 1 .. 30).
__global__ void __launch_bounds__(VL_THREADS) k_resid_restrict(const __grid_constant__ CUtensorMap mr,
                                                               const __grid_constant__ CUtensorMap md,
                                                               float2* __restrict__ rc, int nx, int ny, int batch,
                                                               const int* __restrict__ active, float onemw) {
  float2* vsm = aligned_dyn_smem();
  __shared__ __align__(8) uint64_t bars[2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int ncx = nx / 2, ncy = ny / 2;
  const int nsx = (ncx + RC_TW - 1) / RC_TW, nsy = (ncy + RC_TH - 1) / RC_TH;
  const long per_group = static_cast<long>(nsx) * nsy;
  const int ngroups = (batch + VL_RHS - 1) / VL_RHS;
  auto origin = [&](long u, int& g, int& xc0, int& yc0) {
    g = static_cast<int>(u / per_group);
    const int rem = static_cast<int>(u - static_cast<long>(g) * per_group);
    yc0 = (rem / nsx) * RC_TH;
    xc0 = (rem % nsx) * RC_TW;
  };
  auto issue = [&](long u, int k) {
    int g, xc0, yc0;
    origin(u, g, xc0, yc0);
    float2* buf = vsm + k * RS_BUF;
    int nact = 0;
    for (int w = 0; w < VL_RHS; ++w) nact += rhs_on(g * VL_RHS + w, batch, active);
    mbar_arrive_expect_tx(&bars[k], (1 + nact) * RS_TILE * sizeof(float2));
    const int x = 2 * (2 * xc0 - 2), y = 2 * yc0 - 2;
    tma_load_3d(buf, &md, x, y, 0, &bars[k]);
    for (int w = 0; w < VL_RHS; ++w)
      if (rhs_on(g * VL_RHS + w, batch, active)) tma_load_3d(buf + (1 + w) * RS_TILE, &mr, x, y, g * VL_RHS + w, &bars[k]);
  };
  auto work = [&](long u, int k) {
    int g, xc0, yc0;
    origin(u, g, xc0, yc0);
    const int rw = wid >> 1, band = wid & 1;
    const int b = g * VL_RHS + rw;
    if (!rhs_on(b, batch, active)) return;  // warp-uniform
    const float2* dt = vsm + k * RS_BUF + band * 2 * RC_HB * VS_W;      // the band's first row
    const float2* rt = dt + (1 + rw) * RS_TILE;
    const int gx0 = 2 * xc0 - 2, gy0 = 2 * yc0 - 2 + band * 2 * RC_HB;  // fine row of the band's first row
    const int jc0 = yc0 + band * RC_HB;                                  // the band's first coarse row
    const int xa = gx0 + 2 * lane;                 // this lane's columns xa, xa + 1 (nx is even)
    const bool colin = xa >= 0 && xa < nx;
    float2* out = rc + static_cast<long>(b) * ncx * ncy;
    const int K = xc0 + lane - 1;
    // MK: some q of the band lie outside the grid and are masked
    auto rows = [&](auto mk) {
      constexpr bool MK = decltype(mk)::value;
      float2 um2a = make_float2(0.f, 0.f), um2b = um2a, um1a = um2a, um1b = um2a, rm1a = um2a, rm1b = um2a;
      float2 hm2 = um2a, hm1 = um2a;
#pragma unroll
      for (int y = 0; y < RB_H; ++y) {
        const int gy = gy0 + y;
        const float4 dq = *reinterpret_cast<const float4*>(dt + y * VS_W + 2 * lane);
        const float4 rv = *reinterpret_cast<const float4*>(rt + y * VS_W + 2 * lane);
        const float2 ra = make_float2(rv.x, rv.y), rb = make_float2(rv.z, rv.w);
        const float2 ua = cmul(make_float2(dq.x, dq.y), ra), ub = cmul(make_float2(dq.z, dq.w), rb);
        if (y >= 2) {
          // q on row y - 1, then the [1 2 1] row weights around this lane's even column
          const float2 ul = shfl_up1(um1b), ur = shfl_down1(um1a);
          float2 qa = cadd(cscale(rm1a, onemw), cadd(cadd(um2a, ua), cadd(ul, um1b)));
          float2 qb = cadd(cscale(rm1b, onemw), cadd(cadd(um2b, ub), cadd(um1a, ur)));
          if (MK && !(colin && gy - 1 >= 0 && gy - 1 < ny)) qa = qb = make_float2(0.f, 0.f);
          const float2 ql = shfl_up1(qb);
          const float2 hq = cadd(cadd(ql, qb), cscale(qa, 2.f));
          const int yq = y - 1;
          if (yq >= 3 && (yq & 1)) {
            // coarse row centred on fine row yq - 1
            const int J = jc0 + (yq - 3) / 2;
            if (lane >= 1 && lane <= RC_TW && K < ncx && J < ncy)
              out[static_cast<long>(J) * ncx + K] = cscale(cadd(cadd(hm2, hq), cscale(hm1, 2.f)), 0.25f);
          }
          hm2 = hm1;
          hm1 = hq;
        }
        um2a = um1a;
        um2b = um1b;
        um1a = ua;
        um1b = ub;
        rm1a = ra;
        rm1b = rb;
      }
    };
    const bool inside = __all_sync(0xffffffffu, colin) && gy0 + 1 >= 0 && gy0 + RB_H - 2 < ny;
    if (inside)
      rows(std::false_type{});
    else
      rows(std::true_type{});
  };
  cta_units(bars, static_cast<long>(ngroups) * per_group, per_group, batch, active, issue, work);
}

// Prolongation, correction and post-sweep (Eq. 8 and the damped Jacobi post-sweep):
// u2 = dinv r + I_H^h ec (the pre-sweep recomputed from r), z = (1 - omega) u2 +
// dinv (r + the sum of the neighbours' u2), plus zadd when given.  Unit: (group of VL_RHS
// right-hand sides, band of PS_TH rows, strip of PS_TW columns starting at x0); lane l
// holds columns xa = x0 - 2 + 2 l and xa + 1 and writes them for lanes 1 .. 30.  The
// bilinear prolongation of the pair needs ec at coarse columns xa / 2 and xa / 2 + 1,
// which are columns l + 1 and l + 2 of the coarse strip.
__global__ void __launch_bounds__(VL_THREADS) k_prolong_smooth(const __grid_constant__ CUtensorMap mr,
                                                               const __grid_constant__ CUtensorMap me,
                                                               const __grid_constant__ CUtensorMap md,
                                                               float2* __restrict__ z, int nx, int ny, int batch,
                                                               const int* __restrict__ active,
                                                               const float2* __restrict__ zadd, float onemw) {
  float2* vsm = aligned_dyn_smem();
  __shared__ __align__(8) uint64_t bars[2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int nsx = (nx + PS_TW - 1) / PS_TW, nsy = (ny + PS_TH - 1) / PS_TH;
  const long per_group = static_cast<long>(nsx) * nsy;
  const int ngroups = (batch + VL_RHS - 1) / VL_RHS;
  const long plane = static_cast<long>(nx) * ny;
  auto origin = [&](long u, int& g, int& x0, int& y0) {
    g = static_cast<int>(u / per_group);
    const int rem = static_cast<int>(u - static_cast<long>(g) * per_group);
    y0 = (rem / nsx) * PS_TH;
    x0 = (rem % nsx) * PS_TW;
  };
  auto issue = [&](long u, int k) {
    int g, x0, y0;
    origin(u, g, x0, y0);
    float2* buf = vsm + k * PS_BUF;
    int nact = 0;
    for (int w = 0; w < VL_RHS; ++w) nact += rhs_on(g * VL_RHS + w, batch, active);
    mbar_arrive_expect_tx(&bars[k], ((1 + nact) * PS_TILE + nact * PE_W * PE_H) * sizeof(float2));
    const int x = 2 * (x0 - 2), y = y0 - 1;       // fine strip origin (float index, row)
    const int xe = 2 * (x0 / 2 - 2), ye = y0 / 2 - 1;  // coarse strip origin
    tma_load_3d(buf, &md, x, y, 0, &bars[k]);
    for (int w = 0; w < VL_RHS; ++w) {
      const int b = g * VL_RHS + w;
      if (!rhs_on(b, batch, active)) continue;
      tma_load_3d(buf + (1 + w) * PS_TILE, &mr, x, y, b, &bars[k]);
      tma_load_3d(buf + (1 + VL_RHS) * PS_TILE + w * PE_TILE, &me, xe, ye, b, &bars[k]);
    }
  };
  auto work = [&](long u, int k) {
    int g, x0, y0;
    origin(u, g, x0, y0);
    const int rw = wid >> 1, band = wid & 1;
    const int b = g * VL_RHS + rw;
    if (!rhs_on(b, batch, active)) return;  // warp-uniform
    const float2* dbase = vsm + k * PS_BUF;
    const float2* dt = dbase + band * PS_HB * VS_W;                       // the band's first row
    const float2* rt = dt + (1 + rw) * PS_TILE;
    // ec column xa / 2 of the coarse strip; the band starts between its rows 4 band and 4 band + 1
    const float2* et = dbase + (1 + VL_RHS) * PS_TILE + rw * PE_TILE + (PS_HB / 2) * band * PE_W + lane + 1;
    const int gx0 = x0 - 2, gy0 = y0 - 1 + band * PS_HB;                 // fine row of the band's first row
    const int xa = gx0 + 2 * lane;
    const bool colin = xa >= 0 && xa < nx;
    // horizontally interpolated coarse row i of the strip: (ec(xa/2), (ec(xa/2) + ec(xa/2 + 1)) / 2)
    auto erow = [&](int i, float2& ea, float2& eb) {
      const float2 e0 = et[i * PE_W], e1 = et[i * PE_W + 1];
      ea = e0;
      eb = cscale(cadd(e0, e1), 0.5f);
    };
    float2* zb = z + static_cast<long>(b) * plane;
    const float2* zab = zadd ? zadd + static_cast<long>(b) * plane : nullptr;
    const bool outcol = lane >= 1 && lane <= PS_TW / 2 && xa < nx;
    // MK: some points of the band lie outside the grid (u masked, outputs checked);
    // ZA: zadd is added, its rows loaded four rows ahead of their use
    auto rows = [&](auto mk, auto za) {
      constexpr bool MK = decltype(mk)::value, ZA = decltype(za)::value;
      // only the band's output rows gy0 + 1 .. gy0 + PB_H - 2 that lie in the grid are read
      auto zrow = [&](int row) {
        return ZA && outcol && row <= gy0 + PB_H - 2 && (!MK || row < ny)
                   ? __ldg(reinterpret_cast<const float4*>(zab + static_cast<long>(row) * nx + xa))
                   : make_float4(0.f, 0.f, 0.f, 0.f);
      };
      float4 zq0 = zrow(gy0 + 1), zq1 = zrow(gy0 + 2), zq2 = zrow(gy0 + 3), zq3 = zrow(gy0 + 4);
      // fine row gy0 (odd, or -1) lies between rows 0 and 1 of et
      int ie = 0;
      float2 ca, cb, na, nb2;
      erow(0, ca, cb);
      erow(1, na, nb2);
      float2 um2a = make_float2(0.f, 0.f), um2b = um2a, um1a = um2a, um1b = um2a, rm1a = um2a, rm1b = um2a;
      float4 dm1 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int y = 0; y < PB_H; ++y) {
        const int gy = gy0 + y;
        if (y & 1) {  // even fine row gy: coarse row ie + 1 on it
          ++ie;
          ca = na;
          cb = nb2;
          erow(ie + 1, na, nb2);
        }
        // prolongation: even rows take coarse row ie, odd rows the mean of rows ie, ie + 1
        const bool odd = (y & 1) == 0;
        const float2 pa = odd ? cscale(cadd(ca, na), 0.5f) : ca;
        const float2 pb = odd ? cscale(cadd(cb, nb2), 0.5f) : cb;
        const float4 dq = *reinterpret_cast<const float4*>(dt + y * VS_W + 2 * lane);
        const float4 rv = *reinterpret_cast<const float4*>(rt + y * VS_W + 2 * lane);
        const float2 ra = make_float2(rv.x, rv.y), rb = make_float2(rv.z, rv.w);
        float2 ua = cadd(cmul(make_float2(dq.x, dq.y), ra), pa);
        float2 ub = cadd(cmul(make_float2(dq.z, dq.w), rb), pb);
        if (MK && !(colin && gy >= 0 && gy < ny)) ua = ub = make_float2(0.f, 0.f);
        if (y >= 2) {
          // post-sweep on row gy - 1
          const float2 ul = shfl_up1(um1b), ur = shfl_down1(um1a);
          const float4 a = zq0;
          if (ZA) {
            zq0 = zq1;
            zq1 = zq2;
            zq2 = zq3;
            zq3 = zrow(gy + 3);
          }
          const int oy = gy - 1;
          if (outcol && (!MK || oy < ny)) {
            float2 z0 = cadd(cscale(um1a, onemw),
                             cmul(make_float2(dm1.x, dm1.y), cadd(cadd(rm1a, ul), cadd(cadd(um2a, ua), um1b))));
            float2 z1 = cadd(cscale(um1b, onemw),
                             cmul(make_float2(dm1.z, dm1.w), cadd(cadd(rm1b, um1a), cadd(cadd(um2b, ub), ur))));
            if (ZA) {
              z0 = cadd(z0, make_float2(a.x, a.y));
              z1 = cadd(z1, make_float2(a.z, a.w));
            }
            *reinterpret_cast<float4*>(zb + static_cast<long>(oy) * nx + xa) = make_float4(z0.x, z0.y, z1.x, z1.y);
          }
        }
        um2a = um1a;
        um2b = um1b;
        um1a = ua;
        um1b = ub;
        rm1a = ra;
        rm1b = rb;
        dm1 = dq;
      }
    };
    const bool inside = __all_sync(0xffffffffu, colin) && gy0 >= 0 && gy0 + PB_H - 1 < ny;
    if (zab) {
      if (inside) rows(std::false_type{}, std::true_type{});
      else rows(std::true_type{}, std::true_type{});
    } else {
      if (inside) rows(std::false_type{}, std::false_type{});
      else rows(std::true_type{}, std::false_type{});
    }
  };
  cta_units(bars, static_cast<long>(ngroups) * per_group, per_group, batch, active, issue, work);
}

// ---- coarsest grid: Jacobi right-preconditioned GMRES(K), one CTA per RHS -----------
constexpr int CG_THREADS = 512;
constexpr int CG_WARPS = CG_THREADS / 32;
constexpr int CG_MAXV = HELM_MAX_RESTART + 1;

// Block-wide sum of `nv` complex float accumulators (FP64 across warps). Result in out[].
__device__ void block_csum(float2* acc, int nv, double2* out, double* scratch /*[CG_WARPS*2*CG_MAXV]*/) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = 0; i < nv; ++i) {
    float vx = warp_sum(acc[i].x), vy = warp_sum(acc[i].y);
    if (lane == 0) {
      scratch[(w * CG_MAXV + i) * 2] = vx;
      scratch[(w * CG_MAXV + i) * 2 + 1] = vy;
    }
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double sx = 0.0, sy = 0.0;
    for (int q = 0; q < CG_WARPS; ++q) {
      sx += scratch[(q * CG_MAXV + threadIdx.x) * 2];
      sy += scratch[(q * CG_MAXV + threadIdx.x) * 2 + 1];
    }
    out[threadIdx.x] = make_double2(sx, sy);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(CG_THREADS) k_coarse_gmres(const float2* __restrict__ rc, float2* __restrict__ ec,
                                                             const float2* __restrict__ mass,
                                                             const float2* __restrict__ dinv, int nx, int ny,
                                                             float2* __restrict__ basis, int K,
                                                             const int* __restrict__ active) {
  const int b = blockIdx.x;
  if (active && !active[b]) return;
  const long n = static_cast<long>(nx) * ny;
  const float2* r = rc + b * n;
  float2* V = basis + static_cast<long>(b) * (K + 1) * n;
  __shared__ double scratch[CG_WARPS * 2 * CG_MAXV];
  __shared__ double2 h1[CG_MAXV], h2[CG_MAXV];
  __shared__ double2 Hm[CG_MAXV * HELM_MAX_RESTART];  // rotated Hessenberg, column-major (K+1) x K
  __shared__ double cs[HELM_MAX_RESTART];
  __shared__ double2 sn[HELM_MAX_RESTART];
  __shared__ double2 g[CG_MAXV];
  __shared__ double2 y[HELM_MAX_RESTART];
  __shared__ float sc[CG_MAXV];
  __shared__ int kdone;
  float2 acc[CG_MAXV];

  // beta = ||r||; V_0 = r stored unnormalised with scale 1/beta
  acc[0] = make_float2(0.f, 0.f);
  for (long p = threadIdx.x; p < n; p += CG_THREADS) {
    float2 v = r[p];
    V[p] = v;
    acc[0].x += v.x * v.x + v.y * v.y;
  }
  block_csum(acc, 1, h1, scratch);
  const double beta = sqrt(h1[0].x);
  if (!(beta > 0.0)) {
    for (long p = threadIdx.x; p < n; p += CG_THREADS) ec[b * n + p] = make_float2(0.f, 0.f);
    return;
  }
  if (threadIdx.x == 0) {
    sc[0] = static_cast<float>(1.0 / beta);
    g[0] = make_double2(beta, 0.0);
    kdone = K;
  }
  __syncthreads();
  for (int j = 0; j < K; ++j) {
    const float2* Vj = V + j * n;
    float2* W = V + (j + 1) * n;
    const float sj = sc[j];
    // w = S (dinv . V_j sc_j)
    for (long p = threadIdx.x; p < n; p += CG_THREADS) {
      const int iy = static_cast<int>(p / nx), ix = static_cast<int>(p % nx);
      float2 zc = cmul(dinv[p], Vj[p]);
      float2 nb = make_float2(0.f, 0.f);
      if (iy > 0) nb = cadd(nb, cmul(dinv[p - nx], Vj[p - nx]));
      if (iy + 1 < ny) nb = cadd(nb, cmul(dinv[p + nx], Vj[p + nx]));
      if (ix > 0) nb = cadd(nb, cmul(dinv[p - 1], Vj[p - 1]));
      if (ix + 1 < nx) nb = cadd(nb, cmul(dinv[p + 1], Vj[p + 1]));
      float2 m = mass[p];
      W[p] = cscale(csub(cmul(make_float2(4.f - m.x, -m.y), zc), nb), sj);
    }
    __syncthreads();
    // classical Gram-Schmidt, pass 1: h_i = sc_i <V_i, w>
    for (int i = 0; i <= j; ++i) acc[i] = make_float2(0.f, 0.f);
    for (long p = threadIdx.x; p < n; p += CG_THREADS) {
      float2 w = W[p];
      for (int i = 0; i <= j; ++i) acc[i] = cadd(acc[i], cmulc(V[i * n + p], w));
    }
    block_csum(acc, j + 1, h1, scratch);
    // pass 2 fused with the first update: w' = w - sum h_i sc_i V_i, c_i = sc_i <V_i, w'>
    for (int i = 0; i <= j; ++i) acc[i] = make_float2(0.f, 0.f);
    for (long p = threadIdx.x; p < n; p += CG_THREADS) {
      float2 w = W[p];
      for (int i = 0; i <= j; ++i) {
        const float si = sc[i];
        const float2 hi = make_float2(static_cast<float>(h1[i].x) * si * si, static_cast<float>(h1[i].y) * si * si);
        w = csub(w, cmul(hi, V[i * n + p]));
      }
      W[p] = w;
      for (int i = 0; i <= j; ++i) acc[i] = cadd(acc[i], cmulc(V[i * n + p], w));
    }
    block_csum(acc, j + 1, h2, scratch);
    // second update and the norm
    acc[0] = make_float2(0.f, 0.f);
    for (long p = threadIdx.x; p < n; p += CG_THREADS) {
      float2 w = W[p];
      for (int i = 0; i <= j; ++i) {
        const float si = sc[i];
        const float2 ci = make_float2(static_cast<float>(h2[i].x) * si * si, static_cast<float>(h2[i].y) * si * si);
        w = csub(w, cmul(ci, V[i * n + p]));
      }
      W[p] = w;
      acc[0].x += w.x * w.x + w.y * w.y;
    }
    block_csum(acc, 1, h1 + CG_MAXV - 1, scratch);   // reuse the last slot for ||w||^2
    if (threadIdx.x == 0) {
      // Hessenberg column j (entries in the normalised basis: h_i * sc_i)
      double2* col = Hm + j * CG_MAXV;
      for (int i = 0; i <= j; ++i)
        col[i] = zscale(zadd(h1[i], h2[i]), static_cast<double>(sc[i]));
      const double hn = sqrt(h1[CG_MAXV - 1].x);
      col[j + 1] = make_double2(hn, 0.0);
      for (int i = 0; i < j; ++i) {
        double2 a = col[i], c = col[i + 1];
        col[i] = zadd(zscale(a, cs[i]), zmul(sn[i], c));
        col[i + 1] = zsub(zscale(c, cs[i]), zmul(zconj(sn[i]), a));
      }
      double2 a = col[j];
      double aa = sqrt(zabs2(a));
      double t = sqrt(zabs2(a) + hn * hn);
      if (aa == 0.0) {
        cs[j] = 0.0;
        sn[j] = make_double2(1.0, 0.0);
        col[j] = make_double2(hn, 0.0);
      } else {
        double2 ph = zscale(a, 1.0 / aa);
        cs[j] = aa / t;
        sn[j] = zscale(ph, hn / t);
        col[j] = zscale(ph, t);
      }
      col[j + 1] = make_double2(0.0, 0.0);
      g[j + 1] = zscale(zmul(zconj(sn[j]), g[j]), -1.0);
      g[j] = zscale(g[j], cs[j]);
      sc[j + 1] = hn > 0.0 ? static_cast<float>(1.0 / hn) : 0.f;
      if (!(hn > 0.0)) kdone = j + 1;
    }
    __syncthreads();
    if (kdone <= j + 1 && kdone != K) break;
  }
  if (threadIdx.x == 0) {
    const int k = kdone;
    for (int i = k - 1; i >= 0; --i) {
      double2 s = g[i];
      for (int q = i + 1; q < k; ++q) s = zsub(s, zmul(Hm[q * CG_MAXV + i], y[q]));
      double2 d = Hm[i * CG_MAXV + i];
      double den = zabs2(d);
      y[i] = make_double2((s.x * d.x + s.y * d.y) / den, (s.y * d.x - s.x * d.y) / den);
    }
  }
  __syncthreads();
  const int k = kdone;
  for (long p = threadIdx.x; p < n; p += CG_THREADS) {
    float2 u = make_float2(0.f, 0.f);
    for (int i = 0; i < k; ++i) {
      const float si = sc[i];
      u = cadd(u, cmul(make_float2(static_cast<float>(y[i].x) * si, static_cast<float>(y[i].y) * si), V[i * n + p]));
    }
    ec[b * n + p] = cmul(dinv[p], u);
  }
}


// ---- coarsest grid on a thread-block cluster ----------------------------------------
// One right-hand side per cluster of CL_SIZE CTAs; CTA `rank` owns the slab of rows
// [rank * rows_per, (rank + 1) * rows_per).  Thread t of a CTA owns the slab points
// t + CL_THREADS * k (k < PPT): the Arnoldi vector w of the current step lives in its
// registers, the basis vectors V_0 .. V_{K-1} (unnormalised, with their inverse norms
// sc_i) in the CTA's shared memory; the matrix-vector product reads the neighbouring
// slabs' boundary rows through distributed shared memory.
//
// Classical Gram-Schmidt twice with two cluster reductions per step: the first gives
// h_i = <V_i, w> and ||w||^2, the second the re-orthogonalisation products c_i and
// ||w'||^2 of the once-orthogonalised w'; the norm of the final vector follows from
// Pythagoras, ||w''||^2 = ||w'||^2 - sum sc_i^2 |c_i|^2, which is accurate because the
// c_i are already at rounding level (an explicit third reduction is taken when it is
// not).  The Hessenberg column, Givens rotations and the final triangular solve are
// FP32 on one thread: this is the inexact coarsest solve of a preconditioner (a fixed
// number of iterations, no convergence test), and FP64 dependent arithmetic costs
// about a thousand cycles per rotation on this part.
constexpr int CL_SIZE = 8;
constexpr int CL_THREADS = 128;
constexpr int CL_WARPS = CL_THREADS / 32;
constexpr int CL_K = 10;

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Sums of 32 floats over the cluster.  v[f] is this thread's partial of float f; a
// butterfly of halving exchanges leaves lane l with its warp's sum of float l, the
// warps' sums are added in warp order into this CTA's slot, and after a cluster barrier
// thread f < 32 adds float f of the CTAs' slots in rank order, so every CTA obtains
// bit-identical totals in tot[0..32).  `slot` alternates between two buffers, which is
// enough: a CTA writes a buffer again only after the next barrier, which every reader
// of the previous contents reaches after its reads.
__device__ __forceinline__ void cluster_sum32(cg::cluster_group& cl, float (&v)[32], float* scratch /*[W][32]*/,
                                              float* slot /*[32]*/, float* tot /*[32]*/) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int half = 16; half >= 1; half >>= 1) {
    const bool up = (lane & half) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = up ? v[i] : v[i + half];
      const float keep = up ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, half);
    }
  }
  scratch[w * 32 + lane] = v[0];
  __syncthreads();
  if (threadIdx.x < 32) {
    float s = scratch[threadIdx.x];
#pragma unroll
    for (int q = 1; q < CL_WARPS; ++q) s += scratch[q * 32 + threadIdx.x];
    slot[threadIdx.x] = s;
  }
  cluster_arrive();
  cluster_wait();
  if (threadIdx.x < 32) {
    float part[CL_SIZE];
#pragma unroll
    for (int r = 0; r < CL_SIZE; ++r) part[r] = cl.map_shared_rank(slot, r)[threadIdx.x];
    float s = part[0];
#pragma unroll
    for (int r = 1; r < CL_SIZE; ++r) s += part[r];
    tot[threadIdx.x] = s;
  }
  __syncthreads();
}

// Jacobi right-preconditioned GMRES(K) from a zero initial guess on the coarsest grid
// (Section 3.4): with S the h^2-scaled shifted-Laplacian operator and D the inverse
// diagonal, the Krylov basis q_0 = rc / ||rc||, q_{j+1} from S D q_j; the correction
// is ec = D sum_i y_i q_i with y the least-squares solution of the Hessenberg system.
template <int K, int PPT>
__global__ void __cluster_dims__(CL_SIZE, 1, 1) __launch_bounds__(CL_THREADS, (PPT <= 6 ? 4 : 1))
    k_coarse_gmres_cluster(const float2* __restrict__ rc, float2* __restrict__ ec, const float2* __restrict__ mass,
                           const float2* __restrict__ dinv, int nx, int ny, int rows_per,
                           const int* __restrict__ active) {
  static_assert(2 * K + 1 <= 32, "a reduction carries at most 32 floats");
  cg::cluster_group cl = cg::this_cluster();
  const int crank = static_cast<int>(cl.block_rank());
  const int b = blockIdx.x / CL_SIZE;
  if (active && !active[b]) return;  // uniform over the cluster
  extern __shared__ __align__(16) float2 dsm[];
  const int cap = rows_per * nx;
  float2* Vb = dsm;                    // [K][cap] basis slab, unnormalised
  __shared__ float scratch[CL_WARPS * 32];
  __shared__ float slots[2][32];
  __shared__ float tot[32];
  __shared__ float2 Hm[(K + 1) * K];   // rotated Hessenberg, column-major
  __shared__ float cs[K];
  __shared__ float2 sn[K];
  __shared__ float2 g[K + 1];
  __shared__ float2 hf[K];
  __shared__ float sc[K + 1];          // inverse norms of the basis vectors

  const int r0 = crank * rows_per;
  const int r1 = min(r0 + rows_per, ny);
  const int nrows = max(r1 - r0, 0);
  const int nloc = nrows * nx;
  const long n = static_cast<long>(nx) * ny;
  const long g0 = static_cast<long>(r0) * nx;    // global index of the slab's first point
  const float2* r = rc + b * n + g0;

  float v[32];
  float2 w[PPT], dv[PPT], ms[PPT];
#pragma unroll
  for (int f = 0; f < 32; ++f) v[f] = 0.f;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int p = threadIdx.x + CL_THREADS * k;
    w[k] = dv[k] = ms[k] = make_float2(0.f, 0.f);
    if (p < nloc) {
      const float2 x = r[p];
      Vb[p] = x;
      dv[k] = dinv[g0 + p];
      ms[k] = mass[g0 + p];
      v[0] += x.x * x.x + x.y * x.y;
    }
  }
  int par = 0;
  cluster_sum32(cl, v, scratch, slots[par], tot);
  par ^= 1;
  const float beta2 = tot[0];
  if (!(beta2 > 0.f)) {
    for (int p = threadIdx.x; p < nloc; p += CL_THREADS) ec[b * n + g0 + p] = make_float2(0.f, 0.f);
    cl.sync();
    return;
  }
  if (threadIdx.x == 0) {
    const float beta = sqrtf(beta2);
    sc[0] = 1.f / beta;
    g[0] = make_float2(beta, 0.f);
  }
  __syncthreads();

  int nk = K;  // Hessenberg columns completed (uniform over the cluster)
  for (int j = 0; j < K; ++j) {
    if (j > 0) cluster_wait();  // pairs with the arrive after V_j was written
    const float2* Vj = Vb + j * cap;
    const float sj = sc[j];
    const float2* up = crank > 0 ? cl.map_shared_rank(Vj, crank - 1) + (rows_per - 1) * nx : nullptr;
    const float2* dn = crank + 1 < CL_SIZE ? cl.map_shared_rank(Vj, crank + 1) : nullptr;
    // w = sc_j S (D V_j) on own points; the rows above and below the slab come from
    // the neighbouring CTAs.  Branch-free: a missing neighbour (outside the grid) reads
    // the point itself with weight 0, so that every load of all PPT points can be issued
    // before the first is used.
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int p = threadIdx.x + CL_THREADS * k;
      if (p < nloc) {
        const int ly = p / nx, ix = p - ly * nx;
        const int iy = r0 + ly;
        const float2* dg = dinv + g0 + p;
        const bool hl = ix > 0, hr = ix + 1 < nx, hu = iy > 0, hd = iy + 1 < ny;
        const float2* vu = ly > 0 ? Vj + p - nx : (hu ? up + ix : Vj + p);
        const float2* vd = ly + 1 < nrows ? Vj + p + nx : (hd ? dn + ix : Vj + p);
        const float2 tl = cmul(__ldg(dg - (hl ? 1 : 0)), Vj[p - (hl ? 1 : 0)]);
        const float2 tr = cmul(__ldg(dg + (hr ? 1 : 0)), Vj[p + (hr ? 1 : 0)]);
        const float2 tu = cmul(__ldg(dg - (hu ? nx : 0)), *vu);
        const float2 td = cmul(__ldg(dg + (hd ? nx : 0)), *vd);
        const float2 nb = cadd(cadd(hl ? tl : make_float2(0.f, 0.f), hr ? tr : make_float2(0.f, 0.f)),
                               cadd(hu ? tu : make_float2(0.f, 0.f), hd ? td : make_float2(0.f, 0.f)));
        const float2 zc = cmul(dv[k], Vj[p]);
        w[k] = cscale(csub(cmul(make_float2(4.f - ms[k].x, -ms[k].y), zc), nb), sj);
      }
    }
    // first pass: h_i = <V_i, w> (floats 2i, 2i+1), ||w||^2 (float 2K)
#pragma unroll
    for (int f = 0; f < 32; ++f) v[f] = 0.f;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int p = threadIdx.x + CL_THREADS * k;
      if (p < nloc) {
#pragma unroll
        for (int i = 0; i < K; ++i)
          if (i <= j) {
            const float2 t = cmulc(Vb[i * cap + p], w[k]);
            v[2 * i] += t.x;
            v[2 * i + 1] += t.y;
          }
        v[2 * K] += w[k].x * w[k].x + w[k].y * w[k].y;
      }
    }
    cluster_sum32(cl, v, scratch, slots[par], tot);
    par ^= 1;
    const float nW2 = tot[2 * K];
    if (threadIdx.x == 0)
      for (int i = 0; i <= j; ++i) Hm[j * (K + 1) + i] = make_float2(tot[2 * i], tot[2 * i + 1]);
    // w' = w - sum sc_i^2 h_i V_i; second pass: c_i = <V_i, w'>, ||w'||^2.  Loops
    // over i outside, points inside: each coefficient is formed once.
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (i <= j) {
        const float2 a = cscale(make_float2(tot[2 * i], tot[2 * i + 1]), sc[i] * sc[i]);
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          const int p = threadIdx.x + CL_THREADS * k;
          if (p < nloc) w[k] = csub(w[k], cmul(a, Vb[i * cap + p]));
        }
      }
#pragma unroll
    for (int f = 0; f < 32; ++f) v[f] = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (i <= j) {
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          const int p = threadIdx.x + CL_THREADS * k;
          if (p < nloc) {
            const float2 t = cmulc(Vb[i * cap + p], w[k]);
            v[2 * i] += t.x;
            v[2 * i + 1] += t.y;
          }
        }
      }
#pragma unroll
    for (int k = 0; k < PPT; ++k) v[2 * K] += w[k].x * w[k].x + w[k].y * w[k].y;
    cluster_sum32(cl, v, scratch, slots[par], tot);
    par ^= 1;
    // w'' = w' - sum sc_i^2 c_i V_i; ||w''||^2 by Pythagoras
    const float nw2 = tot[2 * K];
    float corr = 0.f;
    for (int i = 0; i <= j; ++i) corr += sc[i] * sc[i] * (tot[2 * i] * tot[2 * i] + tot[2 * i + 1] * tot[2 * i + 1]);
    float hn2 = nw2 - corr;
    if (threadIdx.x == 0)
      for (int i = 0; i <= j; ++i) Hm[j * (K + 1) + i] = cadd(Hm[j * (K + 1) + i], make_float2(tot[2 * i], tot[2 * i + 1]));
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (i <= j) {
        const float2 a = cscale(make_float2(tot[2 * i], tot[2 * i + 1]), sc[i] * sc[i]);
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          const int p = threadIdx.x + CL_THREADS * k;
          if (p < nloc) w[k] = csub(w[k], cmul(a, Vb[i * cap + p]));
        }
      }
    if (!(hn2 > 1e-3f * nw2)) {
      // the second pass removed more than rounding: take the norm explicitly
#pragma unroll
      for (int f = 0; f < 32; ++f) v[f] = 0.f;
#pragma unroll
      for (int k = 0; k < PPT; ++k) v[0] += w[k].x * w[k].x + w[k].y * w[k].y;
      cluster_sum32(cl, v, scratch, slots[par], tot);
      par ^= 1;
      hn2 = tot[0];
    }
    const bool brk = !(hn2 > 1e-12f * nW2);  // w in the span of the basis: lucky breakdown
    const float hn = brk ? 0.f : sqrtf(hn2);
    if (j + 1 < K && !brk) {
      float2* Vn = Vb + (j + 1) * cap;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const int p = threadIdx.x + CL_THREADS * k;
        if (p < nloc) Vn[p] = w[k];
      }
      cluster_arrive();
    }
    if (threadIdx.x == 0) {
      // H_ij = sc_i <V_i, w>; previous rotations, then the one that zeroes H_{j+1,j}
      float2* col = Hm + j * (K + 1);
      for (int i = 0; i <= j; ++i) col[i] = cscale(col[i], sc[i]);
      for (int i = 0; i < j; ++i) {
        const float2 a = col[i], c = col[i + 1];
        col[i] = cadd(cscale(a, cs[i]), cmul(sn[i], c));
        col[i + 1] = csub(cscale(c, cs[i]), cmul(make_float2(sn[i].x, -sn[i].y), a));
      }
      const float2 a = col[j];
      const float aa = hypotf(a.x, a.y);
      const float t = hypotf(aa, hn);
      if (aa == 0.f) {
        cs[j] = 0.f;
        sn[j] = make_float2(1.f, 0.f);
        col[j] = make_float2(hn, 0.f);
      } else {
        const float2 ph = cscale(a, 1.f / aa);
        cs[j] = aa / t;
        sn[j] = cscale(ph, hn / t);
        col[j] = cscale(ph, t);
      }
      const float2 gj = g[j];
      g[j + 1] = cscale(cmul(make_float2(sn[j].x, -sn[j].y), gj), -1.f);
      g[j] = cscale(gj, cs[j]);
      sc[j + 1] = hn > 0.f ? 1.f / hn : 0.f;
    }
    __syncthreads();
    if (brk) {
      nk = j + 1;
      break;
    }
  }
  if (threadIdx.x == 0) {
    // back substitution on the nk x nk upper triangle, y_i scaled by sc_i
    float2 y[K];
    for (int i = nk - 1; i >= 0; --i) {
      float2 s = g[i];
      for (int q = i + 1; q < nk; ++q) s = csub(s, cmul(Hm[q * (K + 1) + i], y[q]));
      const float2 d = Hm[i * (K + 1) + i];
      const float den = d.x * d.x + d.y * d.y;
      y[i] = den > 0.f ? cscale(cmulc(d, s), 1.f / den) : make_float2(0.f, 0.f);
      hf[i] = cscale(y[i], sc[i]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int p = threadIdx.x + CL_THREADS * k;
    if (p < nloc) {
      float2 u = make_float2(0.f, 0.f);
      for (int i = 0; i < nk; ++i) u = cadd(u, cmul(hf[i], Vb[i * cap + p]));
      ec[b * n + g0 + p] = cmul(dv[k], u);
    }
  }
  cl.sync();  // no CTA leaves while a neighbour may still read its shared memory
}

size_t cluster_smem_bytes(int nx, int ny) {
  const int rows_per = (ny + CL_SIZE - 1) / CL_SIZE;
  return static_cast<size_t>(CL_K) * rows_per * nx * sizeof(float2);
}

// points per thread the cluster kernel is instantiated for (0: the slab is too large)
int cluster_ppt(int nx, int ny) {
  const long nloc = static_cast<long>((ny + CL_SIZE - 1) / CL_SIZE) * nx;
  return nloc <= 6 * CL_THREADS ? 6 : (nloc <= 12 * CL_THREADS ? 12 : 0);
}

template <int K, int PPT>
int launch_cluster(const helm_problem* p, const helm::VcycleScratch& s, int batch, size_t smem, const int* active,
                   cudaStream_t st) {
  const int L = p->mg.levels;
  const int cnx = p->lnx[L - 1], cny = p->lny[L - 1];
  static std::atomic<unsigned long long> attr_done{0}, carve_done{0};
  int rc = helm::smem_attr_once(k_coarse_gmres_cluster<K, PPT>, 200 * 1024, &attr_done);
  if (rc) return rc;
  // four CTAs of 128 threads and about 54 KB share an SM when the carve-out is maximal
  int dev = 0;
  HELM_CUDA(cudaGetDevice(&dev));
  if (!(carve_done.load(std::memory_order_acquire) & (1ull << (dev & 63)))) {
    HELM_CUDA(cudaFuncSetAttribute(k_coarse_gmres_cluster<K, PPT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   cudaSharedmemCarveoutMaxShared));
    carve_done.fetch_or(1ull << (dev & 63), std::memory_order_acq_rel);
  }
  const int rows_per = (cny + CL_SIZE - 1) / CL_SIZE;
  HELM_LAUNCH("k_coarse_gmres_cluster", st,
              k_coarse_gmres_cluster<K, PPT><<<batch * CL_SIZE, CL_THREADS, smem, st>>>(
                  s.rc[L - 1], s.ec[L - 1], p->massSL[L - 1], p->dinvSL[L - 1], cnx, cny, rows_per, active));
  return HELM_OK;
}

}  // namespace

namespace helm {

void carve_vcycle(Carve& c, const helm_problem* p, int batch, VcycleScratch* s) {
  const int L = p->mg.levels;
  for (int l = 1; l < L; ++l) {
    s->rc[l] = c.take<float2>(static_cast<size_t>(batch) * p->npts(l));
    s->ec[l] = c.take<float2>(static_cast<size_t>(batch) * p->npts(l));
  }
  s->basis = c.take<float2>(static_cast<size_t>(batch) * (p->mg.coarse_iters + 1) * p->npts(L - 1));
}

int launch_vcycle(const helm_problem* p, const float2* r, float2* z, int batch, const VcycleScratch& s,
                  const int* active, cudaStream_t st, const float2* zadd) {
  const int L = p->mg.levels;
  const float onemw = static_cast<float>(1.0 - p->mg.omega_jacobi);
  int nsm = 0;
  int rc = sm_count(&nsm);
  if (rc) return rc;
  static std::atomic<unsigned long long> rs_attr{0}, ps_attr{0};
  if ((rc = smem_attr_once(k_resid_restrict, static_cast<int>(RS_SMEM), &rs_attr))) return rc;
  if ((rc = smem_attr_once(k_prolong_smooth, static_cast<int>(PS_SMEM), &ps_attr))) return rc;
  for (int l = 0; l + 1 < L; ++l) {
    const float2* rin = l == 0 ? r : s.rc[l];
    CUtensorMap m, md;
    if ((rc = make_c64_map(&m, rin, p->lnx[l], p->lny[l], batch, VS_W, RS_H))) return rc;
    if ((rc = make_c64_map(&md, p->dinvSL[l], p->lnx[l], p->lny[l], 1, VS_W, RS_H))) return rc;
    const long units = static_cast<long>(div_up(batch, VL_RHS)) * div_up(p->lnx[l + 1], RC_TW) *
                       div_up(p->lny[l + 1], RC_TH);
    const int grid = static_cast<int>(std::min<long>(units, static_cast<long>(VL_CTAS) * nsm));
    HELM_LAUNCH("k_resid_restrict", st,
                k_resid_restrict<<<grid, VL_THREADS, RS_SMEM, st>>>(m, md, s.rc[l + 1], p->lnx[l], p->lny[l], batch,
                                                                    active, onemw));
    HELM_CHECK_LAUNCH("k_resid_restrict");
  }
  {
    const int cnx = p->lnx[L - 1], cny = p->lny[L - 1];
    const size_t smem = cluster_smem_bytes(cnx, cny);
    const int ppt = cluster_ppt(cnx, cny);
    if (p->mg.coarse_iters == CL_K && ppt && smem <= 200 * 1024) {
      if ((rc = ppt == 6 ? launch_cluster<CL_K, 6>(p, s, batch, smem, active, st)
                         : launch_cluster<CL_K, 12>(p, s, batch, smem, active, st)))
        return rc;
    } else {
      HELM_LAUNCH("k_coarse_gmres", st,
                  k_coarse_gmres<<<batch, CG_THREADS, 0, st>>>(s.rc[L - 1], s.ec[L - 1], p->massSL[L - 1],
                                                               p->dinvSL[L - 1], cnx, cny, s.basis,
                                                               p->mg.coarse_iters, active));
    }
  }
  HELM_CHECK_LAUNCH("k_coarse_gmres");
  for (int l = L - 2; l >= 0; --l) {
    const float2* rin = l == 0 ? r : s.rc[l];
    float2* zout = l == 0 ? z : s.ec[l];
    CUtensorMap mr, me, md;
    if ((rc = make_c64_map(&mr, rin, p->lnx[l], p->lny[l], batch, VS_W, PS_H))) return rc;
    if ((rc = make_c64_map(&me, s.ec[l + 1], p->lnx[l + 1], p->lny[l + 1], batch, PE_W, PE_H))) return rc;
    if ((rc = make_c64_map(&md, p->dinvSL[l], p->lnx[l], p->lny[l], 1, VS_W, PS_H))) return rc;
    const long units = static_cast<long>(div_up(batch, VL_RHS)) * div_up(p->lnx[l], PS_TW) * div_up(p->lny[l], PS_TH);
    const int grid = static_cast<int>(std::min<long>(units, static_cast<long>(VL_CTAS) * nsm));
    HELM_LAUNCH("k_prolong_smooth", st,
                k_prolong_smooth<<<grid, VL_THREADS, PS_SMEM, st>>>(mr, me, md, zout, p->lnx[l], p->lny[l], batch,
                                                                    active, l == 0 ? zadd : nullptr, onemw));
    HELM_CHECK_LAUNCH("k_prolong_smooth");
  }
  return HELM_OK;
}

}  // namespace helm

extern "C" int helm_slmg_vcycle(const helm_problem* p, const void* r, void* z, int batch, void* ws, size_t ws_bytes,
                                void* stream) {
  if (!p || !r || !z || batch <= 0 || r == z) {
    helm::set_error("helm_slmg_vcycle: invalid argument (r and z must be distinct device buffers)");
    return HELM_EINVAL;
  }
  helm::Carve c(ws, ws_bytes);
  helm::VcycleScratch s;
  helm::carve_vcycle(c, p, batch, &s);
  if (c.overflow || !ws) {
    helm::set_error("helm_slmg_vcycle: workspace of %zu bytes too small (need %zu)", ws_bytes, c.off);
    return HELM_EWORKSPACE;
  }
  return helm::launch_vcycle(p, static_cast<const float2*>(r), static_cast<float2*>(z), batch, s, nullptr,
                             static_cast<cudaStream_t>(stream));
}
