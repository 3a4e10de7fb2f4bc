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
// Kernels (each stages its tiles into shared memory with TMA tiled loads whose
// out-of-range elements are zero-filled, which is the Dirichlet padding):
//   k_resid_restrict : u, the residual and the full-weighting restriction fused; u is
//                      recomputed from r, never stored.
//   k_prolong_smooth : u recomputed from r, prolongation, correction and the post-sweep
//                      fused.
//   k_coarse_gmres_cluster : the coarsest-grid GMRES for one right-hand side on a
//                      cluster of 8 CTAs; each CTA keeps its slab of rows of the whole
//                      Krylov basis in shared memory, reads the neighbouring slabs'
//                      boundary rows through distributed shared memory, and the inner
//                      products are cluster-wide reductions (classical Gram-Schmidt
//                      twice, FP64 Hessenberg and Givens, computed redundantly and
//                      identically by every CTA of the cluster).
//   k_coarse_gmres   : the same algorithm on one CTA with the basis in global memory,
//                      for coarsest grids whose basis does not fit the cluster.
#include <cooperative_groups.h>

#include "problem.h"

namespace cg = cooperative_groups;

namespace {

// ---- residual + restriction ---------------------------------------------------------
// The fine halo tile is 64 complex values wide (two full warps of lanes per row), so
// the coarse tile is 30 wide; the block is 32 x 8 threads and every pass walks rows
// with whole warps.
constexpr int RC_TW = 30, RC_TH = 8;                        // coarse tile
constexpr int RF_W = 2 * RC_TW + 4, RF_H = 2 * RC_TH + 4;   // fine halo tile (64 x 20)
static_assert(RF_W == 64, "two warp widths per tile row");

__global__ void __launch_bounds__(256) k_resid_restrict(const __grid_constant__ CUtensorMap mr,
                                                        const float2* __restrict__ dinv, float2* __restrict__ rc,
                                                        int nx, int ny, const int* __restrict__ active,
                                                        const float* __restrict__ rscale, float onemw) {
  const int b = blockIdx.z;
  if (active && !active[b]) return;
  __shared__ alignas(128) float2 R[RF_H * RF_W];
  __shared__ alignas(16) float2 U[RF_H * RF_W];
  __shared__ alignas(16) float2 Q[RF_H * RF_W];
  __shared__ alignas(8) uint64_t bar;
  const int xc0 = blockIdx.x * RC_TW, yc0 = blockIdx.y * RC_TH;
  const int gx0 = 2 * xc0 - 2, gy0 = 2 * yc0 - 2;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar, sizeof(R));
    tma_load_3d(R, &mr, 2 * gx0, gy0, b, &bar);
  }
  if (!mbar_wait_bounded(&bar, 0, HELM_DEVERR_TMA_WAIT)) return;
  const float s = rscale ? rscale[b] : 1.f;
  // pass 1: u = dinv r on the halo tile (warp = row, lanes = columns)
  for (int ly = ty; ly < RF_H; ly += 8) {
    const int gy = gy0 + ly;
    const bool rowin = gy >= 0 && gy < ny;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int lx = tx + 32 * h, gx = gx0 + lx;
      const int i = ly * RF_W + lx;
      float2 rv = R[i];
      if (rscale) {
        rv = cscale(rv, s);
        R[i] = rv;
      }
      U[i] = (rowin && gx >= 0 && gx < nx) ? cmul(dinv[gy * nx + gx], rv) : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  // pass 2: q = r - M u = (1 - omega) r + sum of the neighbours' u, inner rows/columns
  for (int ly = 1 + ty; ly < RF_H - 1; ly += 8) {
    const int gy = gy0 + ly;
    const bool rowin = gy >= 0 && gy < ny;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int lx = tx + 32 * h, gx = gx0 + lx;
      if (lx < 1 || lx > RF_W - 2) continue;
      const int i = ly * RF_W + lx;
      float2 q = make_float2(0.f, 0.f);
      if (rowin && gx >= 0 && gx < nx)
        q = cadd(cscale(R[i], onemw), cadd(cadd(U[i - RF_W], U[i + RF_W]), cadd(U[i - 1], U[i + 1])));
      Q[i] = q;
    }
  }
  __syncthreads();
  // pass 3: full-weighting restriction, one coarse point per thread
  const int cy = ty, cx = tx;
  const int J = yc0 + cy, K = xc0 + cx;
  const int ncx = nx / 2, ncy = ny / 2;
  if (cx < RC_TW && J < ncy && K < ncx) {
    const int fy = 2 * cy + 2, fx = 2 * cx + 2;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int a2 = -1; a2 <= 1; ++a2)
#pragma unroll
      for (int c = -1; c <= 1; ++c) {
        const float w = (a2 == 0 ? 2.f : 1.f) * (c == 0 ? 2.f : 1.f);
        acc = cadd(acc, cscale(Q[(fy + a2) * RF_W + fx + c], w));
      }
    // 4 * (1/16) * sum
    rc[static_cast<long>(b) * ncx * ncy + J * ncx + K] = cscale(acc, 0.25f);
  }
}

// ---- prolongation + correction + post-smoothing -------------------------------------
constexpr int PS_TW = 64, PS_TH = 16;
constexpr int PR_W = PS_TW + 4, PR_H = PS_TH + 2;            // fine r tile (68 x 18)
constexpr int PE_W = PS_TW / 2 + 4, PE_H = PS_TH / 2 + 2;    // coarse e tile (36 x 10)

__global__ void __launch_bounds__(256) k_prolong_smooth(const __grid_constant__ CUtensorMap mr,
                                                        const __grid_constant__ CUtensorMap me,
                                                        const float2* __restrict__ dinv, float2* __restrict__ z,
                                                        int nx, int ny, const int* __restrict__ active,
                                                        const float* __restrict__ rscale,
                                                        const float2* __restrict__ zadd, float onemw) {
  const int b = blockIdx.z;
  if (active && !active[b]) return;
  __shared__ alignas(128) float2 R[PR_H * PR_W];
  __shared__ alignas(128) float2 E[PE_H * PE_W];
  __shared__ alignas(16) float2 U[PR_H * PR_W];
  __shared__ alignas(8) uint64_t bar;
  const int x0 = blockIdx.x * PS_TW, y0 = blockIdx.y * PS_TH;
  const int gx0 = x0 - 2, gy0 = y0 - 1;            // origin of the r tile
  const int ex0 = x0 / 2 - 2, ey0 = y0 / 2 - 1;    // origin of the e tile
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar, sizeof(R) + sizeof(E));
    tma_load_3d(R, &mr, 2 * gx0, gy0, b, &bar);
    tma_load_3d(E, &me, 2 * ex0, ey0, b, &bar);
  }
  if (!mbar_wait_bounded(&bar, 0, HELM_DEVERR_TMA_WAIT)) return;
  const float s = rscale ? rscale[b] : 1.f;
  for (int i = threadIdx.x; i < PR_H * PR_W; i += blockDim.x) {
    const int ly = i / PR_W, lx = i % PR_W;
    const int gy = gy0 + ly, gx = gx0 + lx;
    float2 rv = cscale(R[i], s);
    R[i] = rv;
    float2 u = make_float2(0.f, 0.f);
    if (lx >= 1 && lx <= PR_W - 2 && gy >= 0 && gy < ny && gx >= 0 && gx < nx) {
      // bilinear prolongation I_H^h at fine (gy, gx): weights 1 at even, 1/2,1/2 at odd
      // branch-free: the parities of (gy, gx) alternate between neighbouring lanes
      const int jy = (gy >> 1) - ey0, jx = (gx >> 1) - ex0;
      const int oy = gy & 1, ox = gx & 1;
      const float2* e0 = E + jy * PE_W + jx;
      const float2* e1 = oy ? e0 + PE_W : e0;          // the second coarse row only when odd
      const float ax = ox ? 0.5f : 1.f, bx = ox ? 0.5f : 0.f;
      const float ay = oy ? 0.5f : 1.f, by = oy ? 0.5f : 0.f;
      const float2 r0 = cadd(cscale(e0[0], ax), cscale(e0[ox], bx));
      const float2 r1 = cadd(cscale(e1[0], ax), cscale(e1[ox], bx));
      const float2 pe = cadd(cscale(r0, ay), cscale(r1, by));
      u = cadd(cmul(dinv[static_cast<long>(gy) * nx + gx], rv), pe);
    }
    U[i] = u;
  }
  __syncthreads();
  const int lx = 2 + 2 * (threadIdx.x & 31);
  const int ty = threadIdx.x >> 5;
  const int gx = gx0 + lx;
  const long plane = static_cast<long>(nx) * ny;
#pragma unroll
  for (int k = 0; k < PS_TH / 8; ++k) {
    const int ly = 1 + ty + 8 * k;
    const int gy = gy0 + ly;
    if (gy >= ny || gx >= nx) continue;
    const long gi = static_cast<long>(gy) * nx + gx;
    float2 out[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = ly * PR_W + lx + q;
      const float2 nb = cadd(cadd(U[i - PR_W], U[i + PR_W]), cadd(U[i - 1], U[i + 1]));
      out[q] = cadd(cscale(U[i], onemw), cmul(dinv[gi + q], cadd(R[i], nb)));
      if (zadd) out[q] = cadd(out[q], zadd[b * plane + gi + q]);
    }
    *reinterpret_cast<float4*>(z + b * plane + gi) = make_float4(out[0].x, out[0].y, out[1].x, out[1].y);
  }
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
constexpr int CL_SIZE = 8;
constexpr int CL_THREADS = 256;
constexpr int CL_WARPS = CL_THREADS / 32;
constexpr int CL_K = 10;

// CTA-local sum of nv complex accumulators into dst[0..nv) (this CTA's shared memory).
__device__ __forceinline__ void cta_csum(const float2* acc, int nv, double2* dst, double* scratch) {
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
    for (int q = 0; q < CL_WARPS; ++q) {
      sx += scratch[(q * CG_MAXV + threadIdx.x) * 2];
      sy += scratch[(q * CG_MAXV + threadIdx.x) * 2 + 1];
    }
    dst[threadIdx.x] = make_double2(sx, sy);
  }
}

// Cluster-wide sum: every CTA adds the per-CTA partials of all ranks in rank order,
// so all CTAs obtain bit-identical totals.
__device__ __forceinline__ void cluster_csum(cg::cluster_group& cl, double2* slot, int nv, double2* tot) {
  cl.sync();
  if (threadIdx.x < nv) {
    double sx = 0.0, sy = 0.0;
    for (int r = 0; r < CL_SIZE; ++r) {
      const double2* rp = cl.map_shared_rank(slot, r);
      double2 v = rp[threadIdx.x];
      sx += v.x;
      sy += v.y;
    }
    tot[threadIdx.x] = make_double2(sx, sy);
  }
  __syncthreads();
}

template <int K>
__global__ void __cluster_dims__(CL_SIZE, 1, 1) __launch_bounds__(CL_THREADS)
    k_coarse_gmres_cluster(const float2* __restrict__ rc, float2* __restrict__ ec, const float2* __restrict__ mass,
                           const float2* __restrict__ dinv, int nx, int ny, int rows_per,
                           const int* __restrict__ active) {
  cg::cluster_group cl = cg::this_cluster();
  const int crank = static_cast<int>(cl.block_rank());
  const int b = blockIdx.x / CL_SIZE;
  if (active && !active[b]) return;  // uniform over the cluster
  extern __shared__ __align__(16) float2 dsm[];
  const int cap = rows_per * nx;
  float2* Vb = dsm;                            // [(K+1)][cap] basis slab, unnormalised
  float2* Ds = Vb + (K + 1) * cap;             // dinv rows r0-1 .. r1 (rows_per + 2 rows)
  float2* Ms = Ds + (rows_per + 2) * nx;       // mass of own rows
  __shared__ double scratch[CL_WARPS * 2 * CG_MAXV];
  __shared__ double2 red[2][CG_MAXV];
  __shared__ double2 tot[CG_MAXV];
  __shared__ double2 h1[K + 1];
  __shared__ float2 hf[K + 1];
  __shared__ double2 Hm[(K + 1) * K];
  __shared__ double cs[K];
  __shared__ double2 sn[K];
  __shared__ double2 g[K + 1];
  __shared__ double2 yv[K];
  __shared__ float sc[K + 1];
  __shared__ int kdone;

  const int r0 = crank * rows_per;
  const int r1 = min(r0 + rows_per, ny);
  const int nrows = max(r1 - r0, 0);
  const int nloc = nrows * nx;
  const long n = static_cast<long>(nx) * ny;
  const float2* r = rc + b * n + static_cast<long>(r0) * nx;

  float2 acc[K + 1];
  acc[0] = make_float2(0.f, 0.f);
  for (int p = threadIdx.x; p < nloc; p += CL_THREADS) {
    float2 v = r[p];
    Vb[p] = v;
    Ms[p] = mass[static_cast<long>(r0) * nx + p];
    acc[0].x += v.x * v.x + v.y * v.y;
  }
  for (int p = threadIdx.x; p < (rows_per + 2) * nx; p += CL_THREADS) {
    const int iy = r0 - 1 + p / nx;
    Ds[p] = (iy >= 0 && iy < ny && iy <= r1) ? dinv[static_cast<long>(iy) * nx + p % nx] : make_float2(0.f, 0.f);
  }
  int slot = 0;
  cta_csum(acc, 1, red[slot], scratch);
  cluster_csum(cl, red[slot], 1, tot);
  slot ^= 1;
  const double beta = sqrt(tot[0].x);
  if (!(beta > 0.0)) {
    for (int p = threadIdx.x; p < nloc; p += CL_THREADS) ec[b * n + static_cast<long>(r0) * nx + p] = make_float2(0.f, 0.f);
    cl.sync();
    return;
  }
  if (threadIdx.x == 0) {
    sc[0] = static_cast<float>(1.0 / beta);
    g[0] = make_double2(beta, 0.0);
    kdone = K;
  }
  __syncthreads();

#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (kdone <= j) continue;  // uniform: lucky breakdown earlier
    const float2* Vj = Vb + j * cap;
    float2* W = Vb + (j + 1) * cap;
    const float sj = sc[j];
    const float2* up = crank > 0 ? cl.map_shared_rank(Vb + j * cap, crank - 1) + (rows_per - 1) * nx : nullptr;
    const float2* dn = crank + 1 < CL_SIZE ? cl.map_shared_rank(Vb + j * cap, crank + 1) : nullptr;
    // w = S (dinv . sc_j V_j) on own rows, halo rows from the neighbouring CTAs
    for (int p = threadIdx.x; p < nloc; p += CL_THREADS) {
      const int ly = p / nx, ix = p % nx;
      const int iy = r0 + ly;
      const float2* drow = Ds + (ly + 1) * nx + ix;
      float2 zc = cmul(drow[0], Vj[p]);
      float2 nb = make_float2(0.f, 0.f);
      if (ix > 0) nb = cadd(nb, cmul(drow[-1], Vj[p - 1]));
      if (ix + 1 < nx) nb = cadd(nb, cmul(drow[1], Vj[p + 1]));
      if (ly > 0)
        nb = cadd(nb, cmul(drow[-nx], Vj[p - nx]));
      else if (iy > 0)
        nb = cadd(nb, cmul(drow[-nx], up[ix]));
      if (ly + 1 < nrows)
        nb = cadd(nb, cmul(drow[nx], Vj[p + nx]));
      else if (iy + 1 < ny)
        nb = cadd(nb, cmul(drow[nx], dn[ix]));
      float2 m = Ms[p];
      W[p] = cscale(csub(cmul(make_float2(4.f - m.x, -m.y), zc), nb), sj);
    }
    __syncthreads();
    // pass 1: h_i = sc_i <V_i, w>
#pragma unroll
    for (int i = 0; i <= j; ++i) acc[i] = make_float2(0.f, 0.f);
    for (int p = threadIdx.x; p < nloc; p += CL_THREADS) {
      float2 w = W[p];
#pragma unroll
      for (int i = 0; i <= j; ++i) acc[i] = cadd(acc[i], cmulc(Vb[i * cap + p], w));
    }
    cta_csum(acc, j + 1, red[slot], scratch);
    cluster_csum(cl, red[slot], j + 1, tot);
    slot ^= 1;
    if (threadIdx.x <= j) {
      h1[threadIdx.x] = tot[threadIdx.x];
      const float si = sc[threadIdx.x] * sc[threadIdx.x];
      hf[threadIdx.x] = make_float2(static_cast<float>(tot[threadIdx.x].x) * si,
                                    static_cast<float>(tot[threadIdx.x].y) * si);
    }
    __syncthreads();
    // pass 2 fused with the first update
#pragma unroll
    for (int i = 0; i <= j; ++i) acc[i] = make_float2(0.f, 0.f);
    for (int p = threadIdx.x; p < nloc; p += CL_THREADS) {
      float2 w = W[p];
      float2 vv[K + 1];
#pragma unroll
      for (int i = 0; i <= j; ++i) {
        vv[i] = Vb[i * cap + p];
        w = csub(w, cmul(hf[i], vv[i]));
      }
      W[p] = w;
#pragma unroll
      for (int i = 0; i <= j; ++i) acc[i] = cadd(acc[i], cmulc(vv[i], w));
    }
    cta_csum(acc, j + 1, red[slot], scratch);
    cluster_csum(cl, red[slot], j + 1, tot);
    slot ^= 1;
    // second update and the norm
    if (threadIdx.x <= j) {
      const float si = sc[threadIdx.x] * sc[threadIdx.x];
      hf[threadIdx.x] = make_float2(static_cast<float>(tot[threadIdx.x].x) * si,
                                    static_cast<float>(tot[threadIdx.x].y) * si);
      h1[threadIdx.x] = zadd(h1[threadIdx.x], tot[threadIdx.x]);
    }
    __syncthreads();
    acc[0] = make_float2(0.f, 0.f);
    for (int p = threadIdx.x; p < nloc; p += CL_THREADS) {
      float2 w = W[p];
#pragma unroll
      for (int i = 0; i <= j; ++i) w = csub(w, cmul(hf[i], Vb[i * cap + p]));
      W[p] = w;
      acc[0].x += w.x * w.x + w.y * w.y;
    }
    cta_csum(acc, 1, red[slot], scratch);
    cluster_csum(cl, red[slot], 1, tot);
    slot ^= 1;
    if (threadIdx.x == 0) {
      double2* col = Hm + j * (K + 1);
      for (int i = 0; i <= j; ++i) col[i] = zscale(h1[i], static_cast<double>(sc[i]));
      const double hn = sqrt(tot[0].x);
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
      g[j + 1] = zscale(zmul(zconj(sn[j]), g[j]), -1.0);
      g[j] = zscale(g[j], cs[j]);
      sc[j + 1] = hn > 0.0 ? static_cast<float>(1.0 / hn) : 0.f;
      if (!(hn > 0.0)) kdone = j + 1;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int k = kdone;
    for (int i = k - 1; i >= 0; --i) {
      double2 s = g[i];
      for (int q = i + 1; q < k; ++q) s = zsub(s, zmul(Hm[q * (K + 1) + i], yv[q]));
      double2 d = Hm[i * (K + 1) + i];
      double den = zabs2(d);
      yv[i] = make_double2((s.x * d.x + s.y * d.y) / den, (s.y * d.x - s.x * d.y) / den);
    }
  }
  __syncthreads();
  const int k = kdone;
  if (threadIdx.x < k)
    hf[threadIdx.x] = make_float2(static_cast<float>(yv[threadIdx.x].x) * sc[threadIdx.x],
                                  static_cast<float>(yv[threadIdx.x].y) * sc[threadIdx.x]);
  __syncthreads();
  for (int p = threadIdx.x; p < nloc; p += CL_THREADS) {
    float2 u = make_float2(0.f, 0.f);
    for (int i = 0; i < k; ++i) u = cadd(u, cmul(hf[i], Vb[i * cap + p]));
    ec[b * n + static_cast<long>(r0) * nx + p] = cmul(Ds[nx + p], u);
  }
  cl.sync();  // no CTA leaves while a neighbour may still read its shared memory
}

size_t cluster_smem_bytes(int nx, int ny) {
  const int rows_per = (ny + CL_SIZE - 1) / CL_SIZE;
  return static_cast<size_t>((CL_K + 1) * rows_per * nx + (rows_per + 2) * nx + rows_per * nx) * sizeof(float2);
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
                  const int* active, const float* rscale, cudaStream_t st, const float2* zadd) {
  const int L = p->mg.levels;
  const float onemw = static_cast<float>(1.0 - p->mg.omega_jacobi);
  int rc;
  for (int l = 0; l + 1 < L; ++l) {
    const float2* rin = l == 0 ? r : s.rc[l];
    CUtensorMap m;
    if ((rc = make_c64_map(&m, rin, p->lnx[l], p->lny[l], batch, RF_W, RF_H))) return rc;
    dim3 grid(div_up(p->lnx[l + 1], RC_TW), div_up(p->lny[l + 1], RC_TH), batch);
    HELM_LAUNCH("k_resid_restrict", st, k_resid_restrict<<<grid, 256, 0, st>>>(m, p->dinvSL[l], s.rc[l + 1], p->lnx[l], p->lny[l],
                                           active, l == 0 ? rscale : nullptr, onemw));
    HELM_CHECK_LAUNCH("k_resid_restrict");
  }
  {
    const int cnx = p->lnx[L - 1], cny = p->lny[L - 1];
    const size_t smem = cluster_smem_bytes(cnx, cny);
    if (p->mg.coarse_iters == CL_K && smem <= 200 * 1024) {
      static std::atomic<unsigned long long> attr_done{0};
      if ((rc = smem_attr_once(k_coarse_gmres_cluster<CL_K>, 200 * 1024, &attr_done))) return rc;
      const int rows_per = (cny + CL_SIZE - 1) / CL_SIZE;
      HELM_LAUNCH("k_coarse_gmres_cluster", st,
                  k_coarse_gmres_cluster<CL_K><<<batch * CL_SIZE, CL_THREADS, smem, st>>>(
                      s.rc[L - 1], s.ec[L - 1], p->massSL[L - 1], p->dinvSL[L - 1], cnx, cny, rows_per, active));
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
    CUtensorMap mr, me;
    if ((rc = make_c64_map(&mr, rin, p->lnx[l], p->lny[l], batch, PR_W, PR_H))) return rc;
    if ((rc = make_c64_map(&me, s.ec[l + 1], p->lnx[l + 1], p->lny[l + 1], batch, PE_W, PE_H))) return rc;
    dim3 grid(div_up(p->lnx[l], PS_TW), div_up(p->lny[l], PS_TH), batch);
    HELM_LAUNCH("k_prolong_smooth", st, k_prolong_smooth<<<grid, 256, 0, st>>>(mr, me, p->dinvSL[l], zout, p->lnx[l], p->lny[l], active,
                                           l == 0 ? rscale : nullptr, l == 0 ? zadd : nullptr, onemw));
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
  return helm::launch_vcycle(p, static_cast<const float2*>(r), static_cast<float2*>(z), batch, s, nullptr, nullptr,
                             static_cast<cudaStream_t>(stream));
}
