// Flexible GMRES (Saad 1993; the Krylov method of Sections 1, 4.1 and 5), batched over
// right-hand sides, right-preconditioned, restarted.
//
// Vectors are FP32 complex; the Hessenberg matrix, Givens rotations, residual
// estimates and the least-squares solution are FP64 per right-hand side, and the
// solution accumulates in FP64 (x += Z y), so the restart residual b - A x is the
// true FP64 residual.  Orthogonalisation is classical Gram-Schmidt with selective
// (or forced) re-orthogonalisation; every inner product is one pass over the data:
//   k_dots    h_i = <v_i, w> for all i <= j, plus ||w||^2, in one read of w and V
//   k_update  w -= sum h_i v_i, fused with the second-pass products <v_i, w'> and ||w'||^2
// Partial sums are per-block FP64 and reduced deterministically by one CTA per RHS,
// which also applies the Givens rotation and decides whether the RHS stays in the cycle.
// Per-RHS convergence never syncs the host: RHS that finished are masked out of every
// batched kernel; the host reads one counter per restart cycle.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cnn_impl.h"

#define MAXV (HELM_MAX_RESTART + 1)

namespace {

constexpr int KT = 256;         // threads of the streaming kernels
constexpr int KCHUNK = 4096;    // points per block (per RHS)

struct Solver {
  int B, m;            // batch, restart
  long n;              // points per RHS
  int nblk;            // blocks per RHS for reductions
  float2* V;           // [(m+1)][B][n]
  float2* Z;           // [m][B][n]
  double2* part;       // [B][nblk][MAXV+1]
  double2* hcol;       // [B][MAXV]
  double2* ccol;       // [B][MAXV]
  double2* H;          // [B][m][MAXV] rotated Hessenberg, column-major
  double* cs;          // [B][m]
  double2* sn;         // [B][m]
  double2* g;          // [B][MAXV]
  double2* y;          // [B][m]
  double* nwb;         // [B] ||w||^2 before orthogonalisation
  double* bnorm;       // [B]
  double* est;         // [B]
  double* truer;       // [B]
  float* inv;          // [B]
  int* active;         // [B] not finished
  int* cyc;            // [B] in the current cycle
  int* kcyc;           // [B] steps in the current cycle
  int* iters;          // [B]
  int* status;         // [B]
  int* reo;            // [B] needs the second pass this step
  int* maxit;          // [B]
  int* counter;        // [1]
  double* rpart;       // [B][rblk] residual partials
  int rblk;
  double* prev;        // [B] true relative residual at the previous restart
  int* fb;             // [B] 1: this RHS fell back to the plain V-cycle preconditioner
  int* sel;            // [B] indices of the RHS the network runs on this cycle
  int use_cnn;         // the composed preconditioner is in use
  int allow_fb;        // a RHS may fall back to the plain V-cycle (stall or non-finite step)
};

// ---- streaming kernels ----------------------------------------------------------

__device__ __forceinline__ void block_reduce_store(float2* acc, int nv, double2* dst, double* red) {
  // red: [KT/32][MAXV+1][2]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = 0; i < nv; ++i) {
    float vx = warp_sum(acc[i].x), vy = warp_sum(acc[i].y);
    if (lane == 0) {
      red[(w * (MAXV + 1) + i) * 2] = vx;
      red[(w * (MAXV + 1) + i) * 2 + 1] = vy;
    }
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double sx = 0, sy = 0;
    for (int q = 0; q < KT / 32; ++q) {
      sx += red[(q * (MAXV + 1) + threadIdx.x) * 2];
      sy += red[(q * (MAXV + 1) + threadIdx.x) * 2 + 1];
    }
    dst[threadIdx.x] = make_double2(sx, sy);
  }
}

// part[b][blk][i] = sum conj(V_i) w (i < NV), part[b][blk][NV] = (||w||^2, 0)
template <int NV>
__global__ void __launch_bounds__(KT) k_dots(const float2* __restrict__ V, long vstride, const float2* __restrict__ w,
                                             long n, double2* __restrict__ part, int nblk,
                                             const int* __restrict__ mask) {
  const int b = blockIdx.y;
  if (mask && !mask[b]) return;
  __shared__ double red[(KT / 32) * (MAXV + 1) * 2];
  float2 acc[NV + 1];
#pragma unroll
  for (int i = 0; i <= NV; ++i) acc[i] = make_float2(0.f, 0.f);
  const long p0 = static_cast<long>(blockIdx.x) * KCHUNK;
  const long p1 = min(p0 + KCHUNK, n);
  const float2* wb = w + b * n;
  for (long p = p0 + 2 * threadIdx.x; p < p1; p += 2 * KT) {
    float4 wv = *reinterpret_cast<const float4*>(wb + p);
    float2 w0 = make_float2(wv.x, wv.y), w1 = make_float2(wv.z, wv.w);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      float4 vv = *reinterpret_cast<const float4*>(V + i * vstride + b * n + p);
      acc[i] = cadd(acc[i], cadd(cmulc(make_float2(vv.x, vv.y), w0), cmulc(make_float2(vv.z, vv.w), w1)));
    }
    acc[NV].x += w0.x * w0.x + w0.y * w0.y + w1.x * w1.x + w1.y * w1.y;
  }
  block_reduce_store(acc, NV + 1, part + (static_cast<long>(b) * nblk + blockIdx.x) * (MAXV + 1), red);
}

// w -= sum_i h_i V_i (h from coef[b][i], FP64 -> FP32); then, if DOTS, the products
// <V_i, w'> and ||w'||^2 into part, else only ||w'||^2 at part[...][0].
template <int NV, bool DOTS>
__global__ void __launch_bounds__(KT) k_update(const float2* __restrict__ V, long vstride, float2* __restrict__ w,
                                               long n, const double2* __restrict__ coef, double2* __restrict__ part,
                                               int nblk, const int* __restrict__ mask,
                                               const int* __restrict__ mask2) {
  const int b = blockIdx.y;
  if (mask && !mask[b]) return;
  if (mask2 && !mask2[b]) return;
  __shared__ double red[(KT / 32) * (MAXV + 1) * 2];
  __shared__ float2 h[MAXV];
  if (threadIdx.x < NV) {
    double2 c = coef[static_cast<long>(b) * MAXV + threadIdx.x];
    h[threadIdx.x] = make_float2(static_cast<float>(c.x), static_cast<float>(c.y));
  }
  __syncthreads();
  constexpr int NA = DOTS ? NV + 1 : 1;
  float2 acc[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) acc[i] = make_float2(0.f, 0.f);
  const long p0 = static_cast<long>(blockIdx.x) * KCHUNK;
  const long p1 = min(p0 + KCHUNK, n);
  float2* wb = w + b * n;
  for (long p = p0 + 2 * threadIdx.x; p < p1; p += 2 * KT) {
    float4 wv = *reinterpret_cast<const float4*>(wb + p);
    float2 w0 = make_float2(wv.x, wv.y), w1 = make_float2(wv.z, wv.w);
    float4 vv[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      vv[i] = *reinterpret_cast<const float4*>(V + i * vstride + b * n + p);
      w0 = csub(w0, cmul(h[i], make_float2(vv[i].x, vv[i].y)));
      w1 = csub(w1, cmul(h[i], make_float2(vv[i].z, vv[i].w)));
    }
    *reinterpret_cast<float4*>(wb + p) = make_float4(w0.x, w0.y, w1.x, w1.y);
    if constexpr (DOTS) {
#pragma unroll
      for (int i = 0; i < NV; ++i)
        acc[i] = cadd(acc[i], cadd(cmulc(make_float2(vv[i].x, vv[i].y), w0), cmulc(make_float2(vv[i].z, vv[i].w), w1)));
    }
    acc[NA - 1].x += w0.x * w0.x + w0.y * w0.y + w1.x * w1.x + w1.y * w1.y;
  }
  block_reduce_store(acc, NA, part + (static_cast<long>(b) * nblk + blockIdx.x) * (MAXV + 1), red);
}

// v *= inv[b]
__global__ void __launch_bounds__(KT) k_scale(float2* __restrict__ v, long n, const float* __restrict__ inv,
                                              const int* __restrict__ mask) {
  const int b = blockIdx.y;
  if (mask && !mask[b]) return;
  const float s = inv[b];
  const long p0 = static_cast<long>(blockIdx.x) * KCHUNK;
  const long p1 = min(p0 + KCHUNK, n);
  float2* vb = v + b * n;
  for (long p = p0 + 2 * threadIdx.x; p < p1; p += 2 * KT) {
    float4 a = *reinterpret_cast<float4*>(vb + p);
    *reinterpret_cast<float4*>(vb + p) = make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
  }
}

// x += sum_{i < kcyc[b]} y_i Z_i  (accumulated in FP32, added in FP64)
__global__ void __launch_bounds__(KT) k_xupdate(double2* __restrict__ x, const float2* __restrict__ Z, long zstride,
                                                long n, const double2* __restrict__ y, int m,
                                                const int* __restrict__ kcyc, const int* __restrict__ mask) {
  const int b = blockIdx.y;
  if (mask && !mask[b]) return;
  const int k = kcyc[b];
  if (k <= 0) return;
  __shared__ float2 ys[HELM_MAX_RESTART];
  if (threadIdx.x < k) {
    double2 c = y[static_cast<long>(b) * m + threadIdx.x];
    ys[threadIdx.x] = make_float2(static_cast<float>(c.x), static_cast<float>(c.y));
  }
  __syncthreads();
  const long p0 = static_cast<long>(blockIdx.x) * KCHUNK;
  const long p1 = min(p0 + KCHUNK, n);
  for (long p = p0 + 2 * threadIdx.x; p < p1; p += 2 * KT) {
    float2 u0 = make_float2(0.f, 0.f), u1 = u0;
    for (int i = 0; i < k; ++i) {
      float4 zv = *reinterpret_cast<const float4*>(Z + i * zstride + b * n + p);
      u0 = cadd(u0, cmul(ys[i], make_float2(zv.x, zv.y)));
      u1 = cadd(u1, cmul(ys[i], make_float2(zv.z, zv.w)));
    }
    double2* xp = x + b * n + p;
    double2 a = xp[0], c = xp[1];
    xp[0] = make_double2(a.x + u0.x, a.y + u0.y);
    xp[1] = make_double2(c.x + u1.x, c.y + u1.y);
  }
}

__global__ void k_zero_x(double2* __restrict__ x, long n, const double* __restrict__ bnorm) {
  const int b = blockIdx.y;
  if (bnorm[b] > 0.0) return;
  for (long p = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; p < n; p += static_cast<long>(gridDim.x) * blockDim.x)
    x[b * n + p] = make_double2(0.0, 0.0);
}

// ---- per-RHS finalisation kernels (one CTA per RHS) --------------------------------

__device__ void sum_part(const double2* part, int nblk, int nv, double2* out /*smem*/) {
  // out[i] = sum_blk part[blk][i]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = w; i < nv; i += nw) {
    double sx = 0, sy = 0;
    for (int q = lane; q < nblk; q += 32) {
      double2 v = part[static_cast<long>(q) * (MAXV + 1) + i];
      sx += v.x;
      sy += v.y;
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) out[i] = make_double2(sx, sy);
  }
  __syncthreads();
}

__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// One Givens step on column j (hc[0..j], hn) for RHS b.  Single thread.
__device__ void givens_step(Solver S, int b, int j, const double2* hc, double hn, double tol) {
  double2* col = S.H + (static_cast<long>(b) * S.m + j) * MAXV;
  double* cs = S.cs + static_cast<long>(b) * S.m;
  double2* sn = S.sn + static_cast<long>(b) * S.m;
  double2* g = S.g + static_cast<long>(b) * MAXV;
  bool ok = isfinite(hn);
  for (int i = 0; i <= j; ++i) ok = ok && finite2(hc[i]);
  if (!ok) {
    if (S.use_cnn && S.allow_fb && !S.fb[b]) {
      // a non-finite column with the learned preconditioner in use: discard this step
      // (the cycle keeps its j finite steps, x is updated with them at the restart) and
      // hand the RHS to the plain V-cycle for the rest of its solve
      S.fb[b] = 1;
      S.iters[b] += 1;
      S.kcyc[b] = j;
      S.cyc[b] = 0;   // the restart residual decides CONVERGED / MAXIT as usual
      return;
    }
    S.status[b] = HELM_STATUS_NONFINITE;
    S.cyc[b] = 0;
    S.active[b] = 0;
    return;
  }
  for (int i = 0; i <= j; ++i) col[i] = hc[i];
  for (int i = 0; i < j; ++i) {
    double2 a = col[i], c = col[i + 1];
    col[i] = zadd(zscale(a, cs[i]), zmul(sn[i], c));
    col[i + 1] = zsub(zscale(c, cs[i]), zmul(zconj(sn[i]), a));
  }
  double2 a = col[j];
  double aa = sqrt(zabs2(a));
  double t = sqrt(aa * aa + hn * hn);
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
  S.iters[b] += 1;
  S.kcyc[b] = j + 1;
  const double e = sqrt(zabs2(g[j + 1])) / S.bnorm[b];
  S.est[b] = e;
  S.inv[b] = hn > 0.0 ? static_cast<float>(1.0 / hn) : 0.f;
  if (!(e > tol) || !(hn > 0.0) || S.iters[b] >= S.maxit[b]) S.cyc[b] = 0;
}

// stage 1: h = sum of pass-1 products, nwb = ||w||^2
__global__ void k_fin1(Solver S, int nv) {
  const int b = blockIdx.x;
  if (!S.cyc[b]) return;
  __shared__ double2 tot[MAXV + 1];
  sum_part(S.part + static_cast<long>(b) * S.nblk * (MAXV + 1), S.nblk, nv + 1, tot);
  if (threadIdx.x < nv) S.hcol[static_cast<long>(b) * MAXV + threadIdx.x] = tot[threadIdx.x];
  if (threadIdx.x == 0) S.nwb[b] = tot[nv].x;
}

// stage 2: c = second-pass products, ||w'||^2; decide on re-orthogonalisation; if not
// needed, finish the column with the Givens step.
__global__ void k_fin2(Solver S, int j, int reorth, double tol) {
  const int b = blockIdx.x;
  if (!S.cyc[b]) return;
  const int nv = j + 1;
  __shared__ double2 tot[MAXV + 1];
  sum_part(S.part + static_cast<long>(b) * S.nblk * (MAXV + 1), S.nblk, nv + 1, tot);
  if (threadIdx.x == 0) {
    const double nwa = tot[nv].x;
    const bool need = reorth == 2 || (reorth == 1 && nwa < 0.5 * S.nwb[b]);
    S.reo[b] = need ? 1 : 0;
    double2* cc = S.ccol + static_cast<long>(b) * MAXV;
    for (int i = 0; i < nv; ++i) cc[i] = tot[i];
    if (!need) givens_step(S, b, j, S.hcol + static_cast<long>(b) * MAXV, sqrt(nwa), tol);
  }
}

// stage 3 (only RHS that were re-orthogonalised): h += c, norm from the second update
__global__ void k_fin3(Solver S, int j, double tol) {
  const int b = blockIdx.x;
  if (!S.cyc[b] || !S.reo[b]) return;
  __shared__ double2 tot[1];
  sum_part(S.part + static_cast<long>(b) * S.nblk * (MAXV + 1), S.nblk, 1, tot);
  if (threadIdx.x == 0) {
    double2* hc = S.hcol + static_cast<long>(b) * MAXV;
    const double2* cc = S.ccol + static_cast<long>(b) * MAXV;
    for (int i = 0; i <= j; ++i) hc[i] = zadd(hc[i], cc[i]);
    givens_step(S, b, j, hc, sqrt(tot[0].x), tol);
  }
}

// ||b||: sum of the norm partials (k_dots with NV = 0 writes them at index 0)
__global__ void k_fin_bnorm(Solver S) {
  const int b = blockIdx.x;
  __shared__ double2 tot[1];
  sum_part(S.part + static_cast<long>(b) * S.nblk * (MAXV + 1), S.nblk, 1, tot);
  if (threadIdx.x == 0) {
    const double bn = sqrt(tot[0].x);
    S.bnorm[b] = bn;
    S.iters[b] = 0;
    S.kcyc[b] = 0;
    S.est[b] = bn > 0.0 ? 1.0 : 0.0;
    S.truer[b] = S.est[b];
    if (!isfinite(bn)) {
      S.status[b] = HELM_STATUS_NONFINITE;
      S.active[b] = 0;
    } else if (bn == 0.0) {
      S.status[b] = HELM_STATUS_CONVERGED;
      S.active[b] = 0;
    } else {
      S.status[b] = HELM_STATUS_ACTIVE;
      S.active[b] = 1;
    }
    S.cyc[b] = 0;
    S.fb[b] = 0;
    S.prev[b] = -1.0;
  }
}

// back substitution y = R^{-1} g (k = kcyc[b])
__global__ void k_backsolve(Solver S) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= S.B || !S.active[b]) return;
  const int k = S.kcyc[b];
  const double2* H = S.H + static_cast<long>(b) * S.m * MAXV;
  const double2* g = S.g + static_cast<long>(b) * MAXV;
  double2* y = S.y + static_cast<long>(b) * S.m;
  for (int i = k - 1; i >= 0; --i) {
    double2 s = g[i];
    for (int q = i + 1; q < k; ++q) s = zsub(s, zmul(H[q * MAXV + i], y[q]));
    double2 d = H[i * MAXV + i];
    double den = zabs2(d);
    y[i] = den > 0.0 ? make_double2((s.x * d.x + s.y * d.y) / den, (s.y * d.x - s.x * d.y) / den)
                     : make_double2(0.0, 0.0);
  }
}

// restart: beta = ||b - A x|| (true FP64 residual), status decisions, g = beta e1
__global__ void k_fin_restart(Solver S, double tol) {
  const int b = blockIdx.x;
  if (!S.active[b]) return;
  __shared__ double tot;
  double v = 0.0;
  for (int q = threadIdx.x; q < S.rblk; q += blockDim.x) v += S.rpart[static_cast<long>(b) * S.rblk + q];
  v = warp_sum(v);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (blockDim.x >> 5); ++q) t += red[q];
    tot = t;
    const double beta = sqrt(tot);
    const double rel = beta / S.bnorm[b];
    S.truer[b] = rel;
    S.kcyc[b] = 0;
    if (!isfinite(beta)) {
      S.status[b] = HELM_STATUS_NONFINITE;
      S.active[b] = 0;
      S.cyc[b] = 0;
    } else if (!(rel > tol)) {
      S.status[b] = HELM_STATUS_CONVERGED;
      S.active[b] = 0;
      S.cyc[b] = 0;
    } else if (S.iters[b] >= S.maxit[b]) {
      S.status[b] = HELM_STATUS_MAXIT;
      S.active[b] = 0;
      S.cyc[b] = 0;
    } else {
      // a cycle with the learned preconditioner that failed to reduce the residual
      // hands this RHS to the plain SL V-cycle for the rest of the solve
      if (S.use_cnn && S.allow_fb && !S.fb[b] && S.prev[b] > 0.0 && rel > 0.95 * S.prev[b]) S.fb[b] = 1;
      S.prev[b] = rel;
      S.cyc[b] = 1;
      S.inv[b] = static_cast<float>(1.0 / beta);
      S.g[static_cast<long>(b) * MAXV] = make_double2(beta, 0.0);
      S.est[b] = rel;
      atomicAdd(S.counter, 1);
    }
  }
}

__global__ void k_init_caps(Solver S, int maxit, const int* __restrict__ caps) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= S.B) return;
  S.maxit[b] = caps ? min(maxit, caps[b]) : maxit;
}

__global__ void k_write_stats(Solver S, helm_fgmres_stats* __restrict__ st) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= S.B) return;
  helm_fgmres_stats s;
  s.iters = S.iters[b];
  s.status = S.status[b] == HELM_STATUS_ACTIVE ? HELM_STATUS_MAXIT : S.status[b];
  s.rel_res_est = S.est[b];
  s.rel_res_true = S.truer[b];
  st[b] = s;
}

// ---- template dispatch ----------------------------------------------------------
template <int NV>
void launch_dots_t(dim3 g, cudaStream_t st, const float2* V, long vs, const float2* w, long n, double2* part, int nblk,
                   const int* mask) {
  HELM_LAUNCH("k_dots", st, k_dots<NV><<<g, KT, 0, st>>>(V, vs, w, n, part, nblk, mask));
}
template <int NV, bool D>
void launch_update_t(dim3 g, cudaStream_t st, const float2* V, long vs, float2* w, long n, const double2* coef,
                     double2* part, int nblk, const int* mask, const int* mask2) {
  HELM_LAUNCH("k_update", st, k_update<NV, D><<<g, KT, 0, st>>>(V, vs, w, n, coef, part, nblk, mask, mask2));
}

#define HELM_CASES(X) \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) \
  X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30) X(31) X(32)

void launch_dots(int nv, dim3 g, cudaStream_t st, const float2* V, long vs, const float2* w, long n, double2* part,
                 int nblk, const int* mask) {
  switch (nv) {
    case 0: launch_dots_t<0>(g, st, V, vs, w, n, part, nblk, mask); break;
#define X(k) \
  case k: launch_dots_t<k>(g, st, V, vs, w, n, part, nblk, mask); break;
    HELM_CASES(X)
#undef X
    default: break;
  }
}

void launch_update(int nv, bool dots, dim3 g, cudaStream_t st, const float2* V, long vs, float2* w, long n,
                   const double2* coef, double2* part, int nblk, const int* mask, const int* mask2) {
  if (dots) {
    switch (nv) {
#define X(k) \
  case k: launch_update_t<k, true>(g, st, V, vs, w, n, coef, part, nblk, mask, mask2); break;
      HELM_CASES(X)
#undef X
      default: break;
    }
  } else {
    switch (nv) {
#define X(k) \
  case k: launch_update_t<k, false>(g, st, V, vs, w, n, coef, part, nblk, mask, mask2); break;
      HELM_CASES(X)
#undef X
      default: break;
    }
  }
}

}  // namespace

namespace helm {

// preconditioner hook implemented with the CNN (cnn.cu); returns HELM_EINVAL if the
// library was built without it.
int launch_cnn_precond(const helm_problem* p, const helm_cnn* cnn, const float2* r, float2* z, int batch,
                       Carve& carve, const VcycleScratch& vs, const int* active, cudaStream_t st,
                       const int* sel_dev = nullptr, int nsel = -1, const int* zero_rows = nullptr);
size_t cnn_workspace_bytes(const helm_problem* p, const helm_cnn* cnn, int batch);

static void carve_solver(Carve& c, const helm_problem* p, int B, int m, Solver* S) {
  const long n = p->npts(0);
  S->B = B;
  S->m = m;
  S->n = n;
  S->nblk = div_up(n, KCHUNK);
  S->rblk = residual_blocks(p);
  S->V = c.take<float2>(static_cast<size_t>(m + 1) * B * n);
  S->Z = c.take<float2>(static_cast<size_t>(m) * B * n);
  S->part = c.take<double2>(static_cast<size_t>(B) * S->nblk * (MAXV + 1));
  S->hcol = c.take<double2>(static_cast<size_t>(B) * MAXV);
  S->ccol = c.take<double2>(static_cast<size_t>(B) * MAXV);
  S->H = c.take<double2>(static_cast<size_t>(B) * m * MAXV);
  S->cs = c.take<double>(static_cast<size_t>(B) * m);
  S->sn = c.take<double2>(static_cast<size_t>(B) * m);
  S->g = c.take<double2>(static_cast<size_t>(B) * MAXV);
  S->y = c.take<double2>(static_cast<size_t>(B) * m);
  S->nwb = c.take<double>(B);
  S->bnorm = c.take<double>(B);
  S->est = c.take<double>(B);
  S->truer = c.take<double>(B);
  S->inv = c.take<float>(B);
  S->active = c.take<int>(B);
  S->cyc = c.take<int>(B);
  S->kcyc = c.take<int>(B);
  S->iters = c.take<int>(B);
  S->status = c.take<int>(B);
  S->reo = c.take<int>(B);
  S->maxit = c.take<int>(B);
  S->counter = c.take<int>(1);
  S->rpart = c.take<double>(static_cast<size_t>(B) * S->rblk);
  S->prev = c.take<double>(B);
  S->fb = c.take<int>(B);
  S->sel = c.take<int>(B);
}

size_t vcycle_bytes(const helm_problem* p, int batch) {
  Carve c(nullptr, ~size_t(0));
  VcycleScratch s;
  carve_vcycle(c, p, batch, &s);
  return c.off;
}

size_t solver_bytes(const helm_problem* p, int batch, int restart) {
  Carve c(nullptr, ~size_t(0));
  Solver S;
  carve_solver(c, p, batch, restart, &S);
  return c.off;
}

}  // namespace helm

namespace helm {

// One FGMRES solve's state: the workspace carve, options and the per-RHS device arrays.
struct SolveCtx {
  const helm_problem* p = nullptr;
  const helm_cnn* cnn = nullptr;
  const float2* b = nullptr;
  double2* x = nullptr;
  int B = 0, m = 0;
  bool use_cnn = false;
  helm_fgmres_opts o{};
  Solver S{};
  VcycleScratch vs;
  Carve c{nullptr, 0};
  long n = 0, vstride = 0;
  dim3 gs;
};

static int ctx_setup(SolveCtx& x, const helm_problem* p, const helm_cnn* cnn, const float2* b, double2* xs, int B,
                     const helm_fgmres_opts* opts, void* ws, size_t ws_bytes) {
  if (opts)
    x.o = *opts;
  else
    helm_fgmres_opts_default(&x.o);
  const helm_fgmres_opts& o = x.o;
  if (o.restart < 1 || o.restart > HELM_MAX_RESTART || o.maxit < 0 || !(o.rtol >= 0.0) || o.cnn_every < 1) {
    set_error("helm_fgmres_solve: restart must be in [1,%d], maxit >= 0, rtol >= 0, cnn_every >= 1", HELM_MAX_RESTART);
    return HELM_EINVAL;
  }
  x.p = p;
  x.cnn = cnn;
  x.b = b;
  x.x = xs;
  x.B = B;
  x.m = o.restart;
  x.c = Carve(ws, ws_bytes);
  carve_solver(x.c, p, B, o.restart, &x.S);
  carve_vcycle(x.c, p, B, &x.vs);
  if (x.c.overflow || !ws) {
    set_error("helm_fgmres_solve: workspace of %zu bytes too small (need at least %zu)", ws_bytes, x.c.off);
    return HELM_EWORKSPACE;
  }
  x.n = x.S.n;
  x.vstride = static_cast<long>(B) * x.n;
  x.use_cnn = cnn != nullptr;
  x.S.use_cnn = x.use_cnn ? 1 : 0;
  x.S.allow_fb = o.fallback ? 1 : 0;
  x.gs = dim3(x.S.nblk, B);
  return HELM_OK;
}

// restart: r = b - A x in FP64, per-RHS status, the next cycle's first basis vector
static int ctx_restart(SolveCtx& x, cudaStream_t st) {
  Solver& S = x.S;
  int r2 = launch_residual_fp64(x.p, x.b, x.x, S.V, S.rpart, S.rblk, x.B, S.active, st);
  if (r2) return r2;
  HELM_CUDA(cudaMemsetAsync(S.counter, 0, sizeof(int), st));
  HELM_LAUNCH("k_fin_restart", st, k_fin_restart<<<x.B, 256, 0, st>>>(S, x.o.rtol));
  HELM_LAUNCH("k_scale", st, k_scale<<<x.gs, KT, 0, st>>>(S.V, x.n, S.inv, S.cyc));
  HELM_CHECK_LAUNCH("restart");
  return HELM_OK;
}

static int ctx_init(SolveCtx& x, const int* maxit_dev, cudaStream_t st) {
  Solver& S = x.S;
  HELM_LAUNCH("k_init_caps", st, k_init_caps<<<div_up(x.B, 128), 128, 0, st>>>(S, x.o.maxit, maxit_dev));
  launch_dots(0, x.gs, st, S.V, x.vstride, x.b, x.n, S.part, S.nblk, nullptr);
  HELM_LAUNCH("k_fin_bnorm", st, k_fin_bnorm<<<x.B, 256, 0, st>>>(S));
  HELM_LAUNCH("k_zero_x", st, k_zero_x<<<dim3(64, x.B), 256, 0, st>>>(x.x, x.n, S.bnorm));
  HELM_CHECK_LAUNCH("fgmres init");
  return ctx_restart(x, st);
}

// number of right-hand sides still in a cycle (synchronises the stream; reports device
// timeouts)
static int ctx_active(SolveCtx& x, cudaStream_t st, int* nact) {
  unsigned int derr = 0;
  HELM_CUDA(cudaMemcpyAsync(nact, x.S.counter, sizeof(int), cudaMemcpyDeviceToHost, st));
  HELM_CUDA(cudaMemcpyFromSymbolAsync(&derr, g_helm_device_error, sizeof(unsigned int), 0, cudaMemcpyDeviceToHost, st));
  HELM_CUDA(cudaStreamSynchronize(st));
  if (derr) {
    set_error("helm_fgmres_solve: device-side wait timed out (flags 0x%x)", derr);
    return HELM_ETIMEOUT;
  }
  return HELM_OK;
}

// One restart cycle: Arnoldi steps with the preconditioner, the least-squares solution,
// x += Z y and the restart residual.  `device_only`: no host decision inside the cycle
// (for graph capture): the network runs on every right-hand side of the batch and the
// output of those that fell back to the V-cycle is zeroed on the device; otherwise the
// right-hand sides that use the network are gathered into one dense batch on the host's
// reading of the fallback flags.
static int ctx_cycle(SolveCtx& x, bool warm, bool device_only, cudaStream_t st) {
  Solver& S = x.S;
  const int m = x.m, B = x.B;
  const long n = x.n, vstride = x.vstride;
  const int mlen = warm ? std::min(x.o.warmup_iters, m) : m;
  int nsel = 0;
  if (x.use_cnn && !warm && !device_only) {
    std::vector<int> act(B), fbv(B), sel;
    HELM_CUDA(cudaMemcpyAsync(act.data(), S.cyc, B * sizeof(int), cudaMemcpyDeviceToHost, st));
    HELM_CUDA(cudaMemcpyAsync(fbv.data(), S.fb, B * sizeof(int), cudaMemcpyDeviceToHost, st));
    HELM_CUDA(cudaStreamSynchronize(st));
    for (int bb = 0; bb < B; ++bb)
      if (act[bb] && !fbv[bb]) sel.push_back(bb);
    nsel = static_cast<int>(sel.size());
    if (nsel) HELM_CUDA(cudaMemcpyAsync(S.sel, sel.data(), nsel * sizeof(int), cudaMemcpyHostToDevice, st));
  }
  int rc;
  for (int j = 0; j < mlen; ++j) {
    float2* vj = S.V + j * vstride;
    float2* zj = S.Z + j * vstride;
    float2* w = S.V + (j + 1) * vstride;
    if (x.use_cnn && !warm && j % x.o.cnn_every == 0) {
      Carve cc(x.c.base + x.c.off, x.c.cap - x.c.off);
      rc = device_only ? launch_cnn_precond(x.p, x.cnn, vj, zj, B, cc, x.vs, S.cyc, st, nullptr, -1, S.fb)
                       : launch_cnn_precond(x.p, x.cnn, vj, zj, B, cc, x.vs, S.cyc, st, S.sel, nsel);
    } else {
      rc = launch_vcycle(x.p, vj, zj, B, x.vs, S.cyc, st);
    }
    if (rc) return rc;
    if ((rc = launch_apply(x.p, x.p->massA, zj, nullptr, w, B, 0, S.cyc, st))) return rc;
    launch_dots(j + 1, x.gs, st, S.V, vstride, w, n, S.part, S.nblk, S.cyc);
    HELM_LAUNCH("k_fin1", st, k_fin1<<<B, 256, 0, st>>>(S, j + 1));
    launch_update(j + 1, true, x.gs, st, S.V, vstride, w, n, S.hcol, S.part, S.nblk, S.cyc, nullptr);
    HELM_LAUNCH("k_fin2", st, k_fin2<<<B, 256, 0, st>>>(S, j, x.o.reorth, x.o.rtol));
    if (x.o.reorth) {
      launch_update(j + 1, false, x.gs, st, S.V, vstride, w, n, S.ccol, S.part, S.nblk, S.cyc, S.reo);
      HELM_LAUNCH("k_fin3", st, k_fin3<<<B, 256, 0, st>>>(S, j, x.o.rtol));
    }
    HELM_LAUNCH("k_scale", st, k_scale<<<x.gs, KT, 0, st>>>(w, n, S.inv, S.cyc));
    HELM_CHECK_LAUNCH("arnoldi step");
  }
  HELM_LAUNCH("k_backsolve", st, k_backsolve<<<div_up(B, 64), 64, 0, st>>>(S));
  HELM_LAUNCH("k_xupdate", st, k_xupdate<<<x.gs, KT, 0, st>>>(x.x, S.Z, vstride, n, S.y, m, S.kcyc, S.active));
  HELM_CHECK_LAUNCH("x update");
  return ctx_restart(x, st);
}

static int ctx_finish(SolveCtx& x, helm_fgmres_stats* stats_dev, cudaStream_t st) {
  HELM_LAUNCH("k_write_stats", st, k_write_stats<<<div_up(x.B, 128), 128, 0, st>>>(x.S, stats_dev));
  HELM_CHECK_LAUNCH("stats");
  return HELM_OK;
}

}  // namespace helm

struct helm_solver_plan {
  helm::SolveCtx ctx;
  cudaGraphExec_t gwarm = nullptr;    // the warm-up cycle (V-cycle only), with a network
  cudaGraphExec_t gcycle = nullptr;   // a regular restart cycle
  unsigned long long param_version = 0;
};

extern "C" {

void helm_fgmres_opts_default(helm_fgmres_opts* o) {
  if (!o) return;
  o->restart = 10;
  o->rtol = 1e-6;
  o->maxit = 2000;
  o->warmup_iters = 3;
  o->reorth = 1;
  o->cnn_every = 1;
  o->fallback = 1;
}

int helm_workspace_size(const helm_problem* p, const helm_cnn* cnn, int batch, int restart, size_t* bytes) {
  if (!p || !bytes || batch <= 0 || restart < 1 || restart > HELM_MAX_RESTART) {
    helm::set_error("helm_workspace_size: invalid argument (restart in [1,%d])", HELM_MAX_RESTART);
    return HELM_EINVAL;
  }
  size_t s = helm::solver_bytes(p, batch, restart) + helm::vcycle_bytes(p, batch);
  if (cnn) s += helm::cnn_workspace_bytes(p, cnn, batch);
  // the standalone residual / vcycle calls fit inside this as well
  *bytes = s + 4096;
  return HELM_OK;
}

int helm_fgmres_solve(const helm_problem* p, const helm_cnn* cnn, const void* b_, void* x_, int B,
                      const helm_fgmres_opts* opts_, const int* maxit_dev, helm_fgmres_stats* stats_dev, void* ws,
                      size_t ws_bytes, void* stream) {
  using namespace helm;
  if (!p || !b_ || !x_ || B <= 0 || !stats_dev) {
    set_error("helm_fgmres_solve: invalid argument");
    return HELM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SolveCtx ctx;
  int rc = ctx_setup(ctx, p, cnn, static_cast<const float2*>(b_), static_cast<double2*>(x_), B, opts_, ws, ws_bytes);
  if (rc) return rc;
  if ((rc = ctx_init(ctx, maxit_dev, st))) return rc;
  for (int cycle = 0;; ++cycle) {
    int nact = 0;
    if ((rc = ctx_active(ctx, st, &nact))) return rc;
    if (nact == 0) break;
    const bool warm = ctx.use_cnn && cycle == 0 && ctx.o.warmup_iters > 0;
    if ((rc = ctx_cycle(ctx, warm, false, st))) return rc;
  }
  return ctx_finish(ctx, stats_dev, st);
}

int helm_solver_plan_create(const helm_problem* p, const helm_cnn* cnn, const void* b, void* x, int batch,
                            const helm_fgmres_opts* opts, void* ws, size_t ws_bytes, void* stream,
                            helm_solver_plan** out) {
  using namespace helm;
  if (!p || !b || !x || batch <= 0 || !out) {
    set_error("helm_solver_plan_create: invalid argument");
    return HELM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!st) {
    set_error("helm_solver_plan_create: a non-default stream is needed for graph capture");
    return HELM_EINVAL;
  }
  helm_solver_plan* pl = new helm_solver_plan();
  auto fail = [&](int code) {
    helm_solver_plan_destroy(pl);
    return code;
  };
  int rc = ctx_setup(pl->ctx, p, cnn, static_cast<const float2*>(b), static_cast<double2*>(x), batch, opts, ws,
                     ws_bytes);
  if (rc) return fail(rc);
  SolveCtx& c = pl->ctx;
  if (c.use_cnn) {
    const helm_cnn* n = cnn;
    if (n->enc_prob != p || n->enc_pversion != p->version || n->enc_version != n->param_version) {
      set_error("helm_solver_plan_create: the network's encodings are not for this problem (helm_cnn_set_problem)");
      return fail(HELM_ESTATE);
    }
    pl->param_version = n->param_version;
  }
  // one eager pass of every cycle kind first: kernel attributes and the network's derived
  // state are set up outside the capture
  if ((rc = ctx_init(c, nullptr, st))) return fail(rc);
  if (c.use_cnn && c.o.warmup_iters > 0 && (rc = ctx_cycle(c, true, true, st))) return fail(rc);
  if ((rc = ctx_cycle(c, false, true, st))) return fail(rc);
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "plan warm-up"));
  for (int kind = 0; kind < 2; ++kind) {
    const bool warm = kind == 0;
    if (warm && !(c.use_cnn && c.o.warmup_iters > 0)) continue;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamBeginCapture"));
    rc = ctx_cycle(c, warm, true, st);
    e = cudaStreamEndCapture(st, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return fail(rc);
    }
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamEndCapture"));
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaGraphInstantiate"));
    (warm ? pl->gwarm : pl->gcycle) = ex;
  }
  *out = pl;
  return HELM_OK;
}

int helm_solver_plan_solve(helm_solver_plan* pl, const int* maxit_dev, helm_fgmres_stats* stats_dev, void* stream) {
  using namespace helm;
  if (!pl || !stats_dev || !pl->gcycle) {
    set_error("helm_solver_plan_solve: invalid argument");
    return HELM_EINVAL;
  }
  SolveCtx& c = pl->ctx;
  if (c.use_cnn) {
    const helm_cnn* n = c.cnn;
    if (n->param_version != pl->param_version) {
      set_error("helm_solver_plan_solve: the network's parameters changed after the plan was made");
      return HELM_ESTATE;
    }
    if (n->enc_prob != c.p || n->enc_pversion != c.p->version || n->enc_version != n->param_version) {
      set_error("helm_solver_plan_solve: the network's encodings are not for this problem (helm_cnn_set_problem)");
      return HELM_ESTATE;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // every solve starts from x = 0
  HELM_CUDA(cudaMemsetAsync(c.x, 0, static_cast<size_t>(c.B) * c.n * sizeof(double2), st));
  int rc = ctx_init(c, maxit_dev, st);
  if (rc) return rc;
  for (int cycle = 0;; ++cycle) {
    int nact = 0;
    if ((rc = ctx_active(c, st, &nact))) return rc;
    if (nact == 0) break;
    const bool warm = cycle == 0 && pl->gwarm;
    HELM_CUDA(cudaGraphLaunch(warm ? pl->gwarm : pl->gcycle, st));
  }
  return ctx_finish(c, stats_dev, st);
}

int helm_solver_plan_destroy(helm_solver_plan* pl) {
  if (!pl) return HELM_OK;
  if (pl->gwarm) cudaGraphExecDestroy(pl->gwarm);
  if (pl->gcycle) cudaGraphExecDestroy(pl->gcycle);
  delete pl;
  return HELM_OK;
}

}  // extern "C"
