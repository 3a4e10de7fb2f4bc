// The 5-point Helmholtz operator (Section 3.1, Eq. 3; Section 3.4: a 3x3 stencil plus
// a pointwise complex mass term, zero padding = Dirichlet).
//
//   (h^2 A x)[i,j] = (4 - m[i,j]) x[i,j] - x[i-1,j] - x[i+1,j] - x[i,j-1] - x[i,j+1]
//
// k_apply: one CTA per 64 x 32 tile of one right-hand side; the (32+2) x (64+4) halo
// tile is staged into shared memory by a single TMA tiled load whose out-of-range
// elements are zero-filled by the copy engine (that is the Dirichlet padding).  The
// x origin of the box is two complex entries left of the tile so it stays on a
// 16-byte boundary.  Each thread produces two adjacent outputs per row (float4).
//
// k_residual_fp64: r = b - h^2 A x with x in complex128, evaluated in FP64; the true
// residual of the stopping rule.  Per-block partial sums of |r|^2 (FP64).
#include "problem.h"

namespace {

constexpr int TW = 64;   // tile width (complex entries)
constexpr int TH = 32;   // tile height
constexpr int SW = TW + 4;
constexpr int SH = TH + 2;

__global__ void __launch_bounds__(256) k_apply(const __grid_constant__ CUtensorMap mx, const float2* __restrict__ mass,
                                               const float2* __restrict__ c, float2* __restrict__ y, int nx, int ny,
                                               const int* __restrict__ active) {
  const int b = blockIdx.z;
  if (active && !active[b]) return;
  __shared__ alignas(128) float2 tile[SH * SW];
  __shared__ alignas(8) uint64_t bar;
  const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar, SH * SW * sizeof(float2));
    tma_load_3d(tile, &mx, 2 * (x0 - 2), y0 - 1, b, &bar);
  }
  if (!mbar_wait_bounded(&bar, 0, HELM_DEVERR_TMA_WAIT)) return;

  const int lx = 2 * (threadIdx.x & 31);
  const int ty = threadIdx.x >> 5;
  const int gx = x0 + lx;
  const long plane = static_cast<long>(nx) * ny;
#pragma unroll
  for (int k = 0; k < TH / 8; ++k) {
    const int ly = ty + 8 * k;
    const int gy = y0 + ly;
    if (gy >= ny || gx >= nx) continue;
    const float2* row = tile + (ly + 1) * SW;
    float4 cc = *reinterpret_cast<const float4*>(row + lx + 2);
    float4 up = *reinterpret_cast<const float4*>(row - SW + lx + 2);
    float4 dn = *reinterpret_cast<const float4*>(row + SW + lx + 2);
    float2 lf = row[lx + 1];
    float2 rt = row[lx + 4];
    const long gi = static_cast<long>(gy) * nx + gx;
    float4 mm = *reinterpret_cast<const float4*>(mass + gi);
    float2 c0 = make_float2(cc.x, cc.y), c1 = make_float2(cc.z, cc.w);
    float2 d0 = make_float2(4.f - mm.x, -mm.y), d1 = make_float2(4.f - mm.z, -mm.w);
    float2 o0 = cmul(d0, c0), o1 = cmul(d1, c1);
    o0.x -= up.x + dn.x + lf.x + c1.x;
    o0.y -= up.y + dn.y + lf.y + c1.y;
    o1.x -= up.z + dn.z + c0.x + rt.x;
    o1.y -= up.w + dn.w + c0.y + rt.y;
    const long go = b * plane + gi;
    if (c) {
      float4 cv = *reinterpret_cast<const float4*>(c + go);
      o0 = make_float2(cv.x - o0.x, cv.y - o0.y);
      o1 = make_float2(cv.z - o1.x, cv.w - o1.y);
    }
    *reinterpret_cast<float4*>(y + go) = make_float4(o0.x, o0.y, o1.x, o1.y);
  }
}

constexpr int RES_THREADS = 256;
constexpr int RES_PTS = 2048;  // points per block

__global__ void __launch_bounds__(RES_THREADS) k_residual_fp64(const float2* __restrict__ bvec,
                                                               const double2* __restrict__ x,
                                                               const double2* __restrict__ mass,
                                                               float2* __restrict__ r, double* __restrict__ partial,
                                                               int nx, int ny, int nblk, const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const long n = static_cast<long>(nx) * ny;
  const double2* xb = x + b * n;
  double acc = 0.0;
  const long p0 = static_cast<long>(blockIdx.x) * RES_PTS;
  for (long p = p0 + threadIdx.x; p < min(p0 + RES_PTS, n); p += RES_THREADS) {
    const int iy = static_cast<int>(p / nx), ix = static_cast<int>(p % nx);
    double2 xc = xb[p];
    double2 s = make_double2(0.0, 0.0);
    if (iy > 0) s = zadd(s, xb[p - nx]);
    if (iy + 1 < ny) s = zadd(s, xb[p + nx]);
    if (ix > 0) s = zadd(s, xb[p - 1]);
    if (ix + 1 < nx) s = zadd(s, xb[p + 1]);
    double2 mf = mass[p];
    double2 d = make_double2(4.0 - mf.x, -mf.y);
    double2 ax = zsub(zmul(d, xc), s);
    float2 bf = bvec[b * n + p];
    double2 rv = make_double2(static_cast<double>(bf.x) - ax.x, static_cast<double>(bf.y) - ax.y);
    r[b * n + p] = make_float2(static_cast<float>(rv.x), static_cast<float>(rv.y));
    acc += zabs2(rv);
  }
  acc = warp_sum(acc);
  __shared__ double red[RES_THREADS / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < RES_THREADS / 32 ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) partial[static_cast<long>(b) * nblk + blockIdx.x] = v;
  }
}

__global__ void k_sum_partials(const double* __restrict__ partial, int nblk, int batch, double* __restrict__ out) {
  const int b = blockIdx.x;
  double v = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) v += partial[static_cast<long>(b) * nblk + i];
  v = warp_sum(v);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) out[b] = t;
  }
}

}  // namespace

namespace helm {

int launch_apply(const helm_problem* p, const float2* mass, const float2* x, const float2* c, float2* y, int batch,
                 int level, const int* active, cudaStream_t st) {
  const int nx = p->lnx[level], ny = p->lny[level];
  CUtensorMap map;
  int rc = make_c64_map(&map, x, nx, ny, batch, SW, SH);
  if (rc) return rc;
  dim3 grid(div_up(nx, TW), div_up(ny, TH), batch);
  HELM_LAUNCH("k_apply", st, k_apply<<<grid, 256, 0, st>>>(map, mass, c, y, nx, ny, active));
  HELM_CHECK_LAUNCH("k_apply");
  return HELM_OK;
}

int residual_blocks(const helm_problem* p) { return div_up(p->npts(0), RES_PTS); }

int launch_residual_fp64(const helm_problem* p, const float2* b, const double2* x, float2* r, double* partial,
                         int nblk, int batch, const int* active, cudaStream_t st) {
  dim3 grid(nblk, batch);
  HELM_LAUNCH("k_residual_fp64", st, k_residual_fp64<<<grid, RES_THREADS, 0, st>>>(b, x, p->massA64, r, partial, p->nx, p->ny, nblk, active));
  HELM_CHECK_LAUNCH("k_residual_fp64");
  return HELM_OK;
}

int launch_sum_partials(const double* partial, int nblk, int batch, double* out, cudaStream_t st) {
  HELM_LAUNCH("k_sum_partials", st, k_sum_partials<<<batch, 256, 0, st>>>(partial, nblk, batch, out));
  HELM_CHECK_LAUNCH("k_sum_partials");
  return HELM_OK;
}

}  // namespace helm

extern "C" {

int helm_helmholtz_apply(const helm_problem* p, const void* x, void* y, int batch, void* stream) {
  if (!p || !x || !y || batch <= 0) {
    helm::set_error("helm_helmholtz_apply: invalid argument");
    return HELM_EINVAL;
  }
  if (x == y) {
    helm::set_error("helm_helmholtz_apply: x and y must be distinct buffers");
    return HELM_EINVAL;
  }
  return helm::launch_apply(p, p->massA, static_cast<const float2*>(x), nullptr, static_cast<float2*>(y), batch, 0,
                            nullptr, static_cast<cudaStream_t>(stream));
}

int helm_helmholtz_residual_fp64(const helm_problem* p, const void* b, const void* x, void* r, double* rnorm2_dev,
                                 int batch, void* ws, size_t ws_bytes, void* stream) {
  if (!p || !b || !x || !r || batch <= 0) {
    helm::set_error("helm_helmholtz_residual_fp64: invalid argument");
    return HELM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nblk = helm::residual_blocks(p);
  helm::Carve cv(ws, ws_bytes);
  double* partial = cv.take<double>(static_cast<size_t>(nblk) * batch);
  if (cv.overflow || !partial) {
    helm::set_error("helm_helmholtz_residual_fp64: workspace too small");
    return HELM_EWORKSPACE;
  }
  int rc = helm::launch_residual_fp64(p, static_cast<const float2*>(b), static_cast<const double2*>(x),
                                      static_cast<float2*>(r), partial, nblk, batch, nullptr, st);
  if (rc) return rc;
  if (rnorm2_dev) return helm::launch_sum_partials(partial, nblk, batch, rnorm2_dev, st);
  return HELM_OK;
}

}  // extern "C"
