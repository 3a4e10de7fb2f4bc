// Training-data generation (Section 4.3, Eq. 17) on the device: for random vectors x,
//   b = A x;  x_tilde = FGMRES(A, M = V-cycle, b, x0 = 0) for exactly iters[i] steps;
//   e = x - x_tilde;  r = b - A x_tilde (= A e, evaluated in FP64 from x_tilde);
// and, as this library reads the residual normalisation of the network, both e and r
// are scaled by 1 / RMS(r) when `normalise` is set.
#include "problem.h"

namespace {

__global__ void k_pairs_finish(const float2* __restrict__ x, const double2* __restrict__ xt,
                               float2* __restrict__ e, float2* __restrict__ r, const double* __restrict__ rn2, long n,
                               int normalise) {
  const int b = blockIdx.y;
  const double s = normalise ? (rn2[b] > 0.0 ? 1.0 / sqrt(rn2[b] / static_cast<double>(n)) : 0.0) : 1.0;
  for (long p = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; p < n;
       p += static_cast<long>(gridDim.x) * blockDim.x) {
    const long i = b * n + p;
    const float2 xv = x[i];
    const double2 t = xt[i];
    e[i] = make_float2(static_cast<float>((xv.x - t.x) * s), static_cast<float>((xv.y - t.y) * s));
    const float2 rv = r[i];
    r[i] = make_float2(static_cast<float>(rv.x * s), static_cast<float>(rv.y * s));
  }
}

// ---- random training vectors (the x of Eq. 17) ------------------------------------
// Periodic Gaussian filter of one real plane, one 32 x 32 output tile per CTA: the tile
// plus a halo of RF cells is staged in shared memory (indices wrapped), filtered along
// x into a second array, then along y.  Weights exp(-t^2 / (2 sigma^2)), |t| <= rad,
// normalised to sum 1.  Plane p of sample b goes to component p of x (p = 0: real).
constexpr int TF_T = 32;
constexpr int TF_RMAX = 24;

__global__ void __launch_bounds__(256) k_field_filter(const float* __restrict__ white, int n, float sigma, int rad,
                                                      float* __restrict__ x) {
  __shared__ float in[TF_T + 2 * TF_RMAX][TF_T + 2 * TF_RMAX];
  __shared__ float hx[TF_T + 2 * TF_RMAX][TF_T];
  __shared__ float wt[2 * TF_RMAX + 1];
  const int b = blockIdx.z >> 1, plane = blockIdx.z & 1;
  const int x0 = blockIdx.x * TF_T, y0 = blockIdx.y * TF_T;
  const int span = TF_T + 2 * rad;
  const float* src = white + (static_cast<long>(b) * 4 + plane) * n * n;
  if (threadIdx.x == 0) {
    float sum = 0.f;
    for (int t = -rad; t <= rad; ++t) {
      const float v = expf(-0.5f * (t / sigma) * (t / sigma));
      wt[t + rad] = v;
      sum += v;
    }
    for (int t = 0; t <= 2 * rad; ++t) wt[t] /= sum;
  }
  for (int i = threadIdx.x; i < span * span; i += blockDim.x) {
    const int ly = i / span, lx = i - ly * span;
    const int gy = ((y0 + ly - rad) % n + n) % n, gx = ((x0 + lx - rad) % n + n) % n;
    in[ly][lx] = src[static_cast<long>(gy) * n + gx];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < span * TF_T; i += blockDim.x) {
    const int ly = i / TF_T, lx = i - ly * TF_T;
    float acc = 0.f;
    for (int t = 0; t <= 2 * rad; ++t) acc = fmaf(wt[t], in[ly][lx + t], acc);
    hx[ly][lx] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TF_T * TF_T; i += blockDim.x) {
    const int ly = i / TF_T, lx = i - ly * TF_T;
    const int gy = y0 + ly, gx = x0 + lx;
    if (gy >= n || gx >= n) continue;
    float acc = 0.f;
    for (int t = 0; t <= 2 * rad; ++t) acc = fmaf(wt[t], hx[ly + t][lx], acc);
    x[((static_cast<long>(b) * n + gy) * n + gx) * 2 + plane] = acc;
  }
}

// x_b <- x_b / RMS(x_b) + noise (n0 + i n1), one CTA per sample (the sum of |x|^2 in a
// fixed order: per-thread FP64 partials, then a tree over the CTA)
__global__ void __launch_bounds__(1024) k_field_finish(const float* __restrict__ white, int n, float noise,
                                                       float2* __restrict__ x) {
  __shared__ double red[1024];
  const int b = blockIdx.x;
  const long nn = static_cast<long>(n) * n;
  float2* xb = x + b * nn;
  double acc = 0.0;
  for (long i = threadIdx.x; i < nn; i += blockDim.x) {
    const float2 v = xb[i];
    acc += static_cast<double>(v.x) * v.x + static_cast<double>(v.y) * v.y;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double ms = red[0] / static_cast<double>(nn);
  const float sc = ms > 0.0 ? static_cast<float>(1.0 / sqrt(ms)) : 0.f;
  const float* n0 = white + (static_cast<long>(b) * 4 + 2) * nn;
  const float* n1 = n0 + nn;
  for (long i = threadIdx.x; i < nn; i += blockDim.x) {
    const float2 v = xb[i];
    xb[i] = make_float2(fmaf(noise, n0[i], v.x * sc), fmaf(noise, n1[i], v.y * sc));
  }
}

}  // namespace

extern "C" int helm_training_field(const float* white, int batch, int n, float sigma, float noise, void* x,
                                   void* stream) {
  const int rad = static_cast<int>(ceilf(3.f * sigma));
  if (!white || !x || batch <= 0 || n <= 0 || !(sigma > 0.f) || rad > TF_RMAX || !(noise >= 0.f)) {
    helm::set_error("helm_training_field: invalid argument (sigma in (0, %d], noise >= 0)", TF_RMAX / 3);
    return HELM_EINVAL;
  }
  if (batch > 65535 / 2) {
    helm::set_error("helm_training_field: batch %d too large", batch);
    return HELM_ESHAPE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dim3 grid(helm::div_up(n, TF_T), helm::div_up(n, TF_T), 2 * batch);
  HELM_LAUNCH("k_field_filter", st, k_field_filter<<<grid, 256, 0, st>>>(white, n, sigma, rad, static_cast<float*>(x)));
  HELM_CHECK_LAUNCH("k_field_filter");
  HELM_LAUNCH("k_field_finish", st, k_field_finish<<<batch, 1024, 0, st>>>(white, n, noise, static_cast<float2*>(x)));
  HELM_CHECK_LAUNCH("k_field_finish");
  return HELM_OK;
}

extern "C" int helm_datagen_pairs(const helm_problem* p, const void* x_, const int* iters_dev, void* e_, void* r_,
                                  int batch, int max_iters, int normalise, void* ws, size_t ws_bytes, void* stream) {
  using namespace helm;
  if (!p || !x_ || !iters_dev || !e_ || !r_ || batch <= 0 || max_iters < 1 || max_iters > HELM_MAX_RESTART) {
    set_error("helm_datagen_pairs: invalid argument (max_iters in [1,%d])", HELM_MAX_RESTART);
    return HELM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long n = p->npts(0);
  Carve cv(ws, ws_bytes);
  float2* b = cv.take<float2>(static_cast<size_t>(batch) * n);
  double2* xt = cv.take<double2>(static_cast<size_t>(batch) * n);
  double* rn2 = cv.take<double>(batch);
  helm_fgmres_stats* stats = cv.take<helm_fgmres_stats>(batch);
  const int rblk = residual_blocks(p);
  double* part = cv.take<double>(static_cast<size_t>(rblk) * batch);
  if (cv.overflow || !ws) {
    set_error("helm_datagen_pairs: workspace too small");
    return HELM_EWORKSPACE;
  }
  const float2* x = static_cast<const float2*>(x_);
  int rc = launch_apply(p, p->massA, x, nullptr, b, batch, 0, nullptr, st);
  if (rc) return rc;
  HELM_CUDA(cudaMemsetAsync(xt, 0, static_cast<size_t>(batch) * n * sizeof(double2), st));
  helm_fgmres_opts o;
  helm_fgmres_opts_default(&o);
  o.restart = max_iters;
  o.rtol = 0.0;
  o.maxit = max_iters;
  o.warmup_iters = 0;
  rc = helm_fgmres_solve(p, nullptr, b, xt, batch, &o, iters_dev, stats, cv.base + cv.off, cv.cap - cv.off, stream);
  if (rc) return rc;
  float2* r = static_cast<float2*>(r_);
  if ((rc = launch_residual_fp64(p, b, xt, r, part, rblk, batch, nullptr, st))) return rc;
  if ((rc = launch_sum_partials(part, rblk, batch, rn2, st))) return rc;
  HELM_LAUNCH("k_pairs_finish", st,
              k_pairs_finish<<<dim3(std::min<long>(div_up(n, 256), 1024), batch), 256, 0, st>>>(
                  x, xt, static_cast<float2*>(e_), r, rn2, n, normalise));
  HELM_CHECK_LAUNCH("k_pairs_finish");
  return HELM_OK;
}

extern "C" int helm_datagen_workspace_size(const helm_problem* p, int batch, int max_iters, size_t* bytes) {
  if (!p || !bytes || batch <= 0) {
    helm::set_error("helm_datagen_workspace_size: invalid argument");
    return HELM_EINVAL;
  }
  size_t fg = 0;
  int rc = helm_workspace_size(p, nullptr, batch, max_iters, &fg);
  if (rc) return rc;
  const long n = p->npts(0);
  *bytes = fg + static_cast<size_t>(batch) * n * (sizeof(float2) + sizeof(double2)) +
           static_cast<size_t>(batch) * (sizeof(double) + sizeof(helm_fgmres_stats)) +
           static_cast<size_t>(helm::residual_blocks(p)) * batch * sizeof(double) + 8 * 256;
  return HELM_OK;
}
