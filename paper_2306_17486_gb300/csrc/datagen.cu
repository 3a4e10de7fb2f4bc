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

}  // namespace

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
