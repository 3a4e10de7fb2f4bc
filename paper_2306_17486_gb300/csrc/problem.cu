// Problem setup (Section 3.1 and 3.2): absorbing layer, Helmholtz mass term, the
// full-weighting kappa^2 pyramid and the shifted-Laplacian mass and damped Jacobi
// diagonals per multigrid level.  Computed on the device in FP64, stored in FP32.
// Also: library-wide error state, version, device error word, TMA descriptors.
#include <cstdarg>
#include <cstring>
#include <mutex>

#include "problem.h"

__device__ unsigned int g_helm_device_error = 0;

namespace helm {

static thread_local char g_err[512] = {0};

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error %d (%s) in %s", static_cast<int>(e), cudaGetErrorString(e), what);
  return HELM_ECUDA;
}

// --- TMA descriptor creation through the driver entry point ---------------------
typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode() {
  static PFN_encodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_encodeTiled>(f);
  });
  return fn;
}

int sm_count(int* out) {
  static int cache[64] = {};
  int dev = 0;
  HELM_CUDA(cudaGetDevice(&dev));
  int& c = cache[dev & 63];
  if (!c) HELM_CUDA(cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev));
  *out = c;
  return HELM_OK;
}

int make_c64_map(CUtensorMap* out, const void* base, int nx, int ny, int nb, int box_w, int box_h) {
  PFN_encodeTiled enc = get_encode();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return HELM_ECUDA;
  }
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (nx & 1) || (box_w & 1)) {
    set_error("TMA map: base must be 16-byte aligned and nx, box width even");
    return HELM_EINVAL;
  }
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(2 * nx), static_cast<cuuint64_t>(ny), static_cast<cuuint64_t>(nb)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(nx) * 8, static_cast<cuuint64_t>(nx) * ny * 8};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(2 * box_w), static_cast<cuuint32_t>(box_h), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) nx=%d ny=%d nb=%d box=%dx%d", static_cast<int>(r), nx, ny, nb,
              box_w, box_h);
    return HELM_ECUDA;
  }
  return HELM_OK;
}

int make_bf16_nhwc_map(CUtensorMap* out, const void* base, int C, int W, int H, int B, int box_w, int box_h) {
  PFN_encodeTiled enc = get_encode();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return HELM_ECUDA;
  }
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || C % 8 || box_w < 1 || box_w > 256 || box_h < 1 ||
      box_h > 256) {
    set_error("TMA map: base must be 16-byte aligned, channels a multiple of 8, box sides in [1, 256]");
    return HELM_EINVAL;
  }
  cuuint64_t dims[4] = {8, static_cast<cuuint64_t>(W), static_cast<cuuint64_t>(H), static_cast<cuuint64_t>(B)};
  cuuint64_t strides[3] = {static_cast<cuuint64_t>(C) * 2, static_cast<cuuint64_t>(W) * C * 2,
                           static_cast<cuuint64_t>(H) * W * C * 2};
  cuuint32_t box[4] = {8, static_cast<cuuint32_t>(box_w), static_cast<cuuint32_t>(box_h), 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for a BF16 NHWC map C=%d W=%d H=%d B=%d box=%dx%d",
              static_cast<int>(r), C, W, H, B, box_w, box_h);
    return HELM_ECUDA;
  }
  return HELM_OK;
}

}  // namespace helm

// --- setup kernels -----------------------------------------------------------------

// gamma = gamma0 + max((d_y/L)^2, (d_x/L)^2) with d the distance in cells into the layer.
__device__ __forceinline__ double abl_profile(int i, int n, int abl) {
  if (abl <= 0) return 0.0;
  int d = max(max(abl - i, i - (n - 1 - abl)), 0);
  double t = static_cast<double>(d) / abl;
  return t * t;
}

// Boundary sides of node (y, x): 0 inside, 1 on an edge, 2 at a corner.
__device__ __forceinline__ int boundary_sides(int y, int x, int ny, int nx) {
  return (y == 0) + (y == ny - 1) + (x == 0) + (x == nx - 1);
}

__global__ void k_setup_fine(const float* __restrict__ kappa, int nx, int ny, int abl, double omega_h, double gamma0,
                             int bc, float* __restrict__ gamma, float2* __restrict__ massA, double2* __restrict__ massA64,
                             double* __restrict__ k2, double* __restrict__ g64) {
  long n = static_cast<long>(nx) * ny;
  for (long idx = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; idx < n;
       idx += static_cast<long>(gridDim.x) * blockDim.x) {
    int y = static_cast<int>(idx / nx), x = static_cast<int>(idx % nx);
    double g = gamma0 + fmax(abl_profile(y, ny, abl), abl_profile(x, nx, abl));
    double kk = static_cast<double>(kappa[idx]);
    kk = kk * kk;
    double m = omega_h * omega_h * kk;
    double mr = m, mi = -m * g;
    if (bc != HELM_BC_DIRICHLET) {
      // ghost value c u_b per boundary side, folded into the mass term
      const int nb = boundary_sides(y, x, ny, nx);
      mr += nb;
      if (bc == HELM_BC_SOMMERFELD) mi -= nb * omega_h * static_cast<double>(kappa[idx]);
    }
    gamma[idx] = static_cast<float>(g);
    massA[idx] = make_float2(static_cast<float>(mr), static_cast<float>(mi));
    massA64[idx] = make_double2(mr, mi);
    k2[idx] = kk;
    g64[idx] = g;
  }
}

// Full-weighting average (Eq. 8 weights, normalised by the in-grid weight) fine -> coarse.
__global__ void k_restrict_avg(const double* __restrict__ f, int nx, int ny, double* __restrict__ c) {
  int ncx = nx / 2, ncy = ny / 2;
  long n = static_cast<long>(ncx) * ncy;
  for (long idx = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; idx < n;
       idx += static_cast<long>(gridDim.x) * blockDim.x) {
    int J = static_cast<int>(idx / ncx), K = static_cast<int>(idx % ncx);
    double s = 0.0, w = 0.0;
    for (int a = -1; a <= 1; ++a)
      for (int b = -1; b <= 1; ++b) {
        int y = 2 * J + a, x = 2 * K + b;
        if (y < 0 || y >= ny || x < 0 || x >= nx) continue;
        double wt = (a == 0 ? 2.0 : 1.0) * (b == 0 ? 2.0 : 1.0);
        s += wt * f[static_cast<long>(y) * nx + x];
        w += wt;
      }
    c[idx] = s / w;
  }
}

// SL mass (omega h_l)^2 k^2 (1 - (beta [+ gamma]) i), then the boundary condition:
// Dirichlet with the ghost-point boundary fix on the first row/column of coarse levels,
// or the level's own Neumann / Sommerfeld ghost term (omega h_l, kappa_l = sqrt(k^2));
// and the damped Jacobi inverse diagonal.
__global__ void k_sl_mass(const double* __restrict__ k2, const double* __restrict__ g, int nx, int ny, double oh,
                          double beta, int use_gamma, double fix, int bc, double omega_j, float2* __restrict__ mass,
                          float2* __restrict__ dinv) {
  const double oh2 = oh * oh;
  long n = static_cast<long>(nx) * ny;
  for (long idx = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; idx < n;
       idx += static_cast<long>(gridDim.x) * blockDim.x) {
    int y = static_cast<int>(idx / nx), x = static_cast<int>(idx % nx);
    double sh = beta + (use_gamma ? g[idx] : 0.0);
    double mr = oh2 * k2[idx], mi = -oh2 * k2[idx] * sh;
    if (bc == HELM_BC_DIRICHLET) {
      if (y == 0) mr -= fix;
      if (x == 0) mr -= fix;
    } else {
      const int nb = boundary_sides(y, x, ny, nx);
      mr += nb;
      if (bc == HELM_BC_SOMMERFELD) mi -= nb * oh * sqrt(k2[idx]);
    }
    mass[idx] = make_float2(static_cast<float>(mr), static_cast<float>(mi));
    // omega_j / (4 - m)
    double dr = 4.0 - mr, di = -mi;
    double den = dr * dr + di * di;
    dinv[idx] = make_float2(static_cast<float>(omega_j * dr / den), static_cast<float>(-omega_j * di / den));
  }
}

// ----------------------------------------------------------------------------------
namespace helm {

// The setup kernels of Section 3.1-3.2 for the problem's current kappa source and
// omega h, into the problem's own arrays (in place; the FP64 kappa^2 and gamma pyramids
// are temporary and freed again).  Synchronises `st`.
int run_setup(helm_problem* p, const float* kappa_dev, cudaStream_t st) {
  const helm_mg_opts& o = p->mg;
  const int nx = p->nx, ny = p->ny, abl = p->abl;
  const double omega_h = p->omega_h, gamma0 = p->gamma0;
  const long n0 = p->npts(0);
  auto fail = [&](int code) { return code; };
  // FP64 kappa^2 and gamma pyramids, two levels at a time, in the problem's own scratch
  // (allocated once, so an in-place update allocates nothing)
  double *k2a = p->setup64[0], *k2b = p->setup64[1], *ga = p->setup64[2], *gb = p->setup64[3];
  if (kappa_dev != p->kappa) {
    cudaError_t ce = cudaMemcpyAsync(p->kappa, kappa_dev, n0 * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (ce != cudaSuccess) return fail(cuda_fail(ce, "copy kappa"));
  }
  int nb = static_cast<int>(std::min<long>(div_up(n0, 256), 4096));
  HELM_LAUNCH("k_setup_fine", st, k_setup_fine<<<nb, 256, 0, st>>>(p->kappa, nx, ny, abl, omega_h, gamma0, o.bc, p->gamma, p->massA, p->massA64, k2a, ga));
  for (int l = 0; l < o.levels; ++l) {
    double oh = omega_h * static_cast<double>(1 << l);
    double fix = (o.boundary_fix && l > 0) ? static_cast<double>((1 << l) - 1) : 0.0;
    long nl = p->npts(l);
    int nbl = static_cast<int>(std::min<long>(div_up(nl, 256), 4096));
    HELM_LAUNCH("k_sl_mass", st, k_sl_mass<<<nbl, 256, 0, st>>>(k2a, ga, p->lnx[l], p->lny[l], oh, o.beta, o.sl_includes_gamma, fix,
                                   o.bc, o.omega_jacobi, p->massSL[l], p->dinvSL[l]));
    if (l + 1 < o.levels) {
      long nc = p->npts(l + 1);
      int nbc = static_cast<int>(std::min<long>(div_up(nc, 256), 4096));
      HELM_LAUNCH("k_restrict_avg", st, k_restrict_avg<<<nbc, 256, 0, st>>>(k2a, p->lnx[l], p->lny[l], k2b));
      HELM_LAUNCH("k_restrict_avg", st, k_restrict_avg<<<nbc, 256, 0, st>>>(ga, p->lnx[l], p->lny[l], gb));
      std::swap(k2a, k2b);
      std::swap(ga, gb);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(cuda_fail(e, "problem setup kernels"));
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(cuda_fail(e, "problem setup sync"));
  return HELM_OK;
}

}  // namespace helm

extern "C" {

void helm_mg_opts_default(helm_mg_opts* o) {
  if (!o) return;
  o->levels = 3;
  o->beta = 0.5;
  o->omega_jacobi = 0.8;
  o->coarse_iters = 10;
  o->sl_includes_gamma = 0;
  o->boundary_fix = 1;
  o->bc = HELM_BC_DIRICHLET;
}

const char* helm_last_error_string(void) { return helm::g_err; }

const char* helm_version(void) { return "helm-gb300 0.1 (sm_103a)"; }

int helm_device_errors(unsigned int* flags) {
  if (!flags) {
    helm::set_error("helm_device_errors: null flags");
    return HELM_EINVAL;
  }
  unsigned int zero = 0;
  HELM_CUDA(cudaMemcpyFromSymbol(flags, g_helm_device_error, sizeof(unsigned int)));
  HELM_CUDA(cudaMemcpyToSymbol(g_helm_device_error, &zero, sizeof(unsigned int)));
  return HELM_OK;
}

int helm_problem_create(const float* kappa_dev, int nx, int ny, int abl, double omega_h, double gamma0,
                        const helm_mg_opts* opts, void* stream_, helm_problem** out) {
  using namespace helm;
  if (!kappa_dev || !out || nx <= 0 || ny <= 0 || abl < 0) {
    set_error("helm_problem_create: invalid argument");
    return HELM_EINVAL;
  }
  helm_mg_opts o;
  if (opts)
    o = *opts;
  else
    helm_mg_opts_default(&o);
  if (o.levels < 2 || o.levels > HELM_MAX_LEVELS || o.coarse_iters < 1 || o.coarse_iters > HELM_MAX_RESTART) {
    set_error("helm_problem_create: levels must be in [2,%d], coarse_iters in [1,%d]", HELM_MAX_LEVELS,
              HELM_MAX_RESTART);
    return HELM_EINVAL;
  }
  if (o.bc != HELM_BC_DIRICHLET && o.bc != HELM_BC_NEUMANN && o.bc != HELM_BC_SOMMERFELD) {
    set_error("helm_problem_create: bc must be HELM_BC_DIRICHLET, HELM_BC_NEUMANN or HELM_BC_SOMMERFELD");
    return HELM_EINVAL;
  }
  int div = 1 << o.levels;
  if (nx % div || ny % div) {
    set_error("helm_problem_create: nx=%d, ny=%d must be divisible by 2^levels=%d", nx, ny, div);
    return HELM_ESHAPE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  helm_problem* p = new helm_problem();
  p->nx = nx;
  p->ny = ny;
  p->abl = abl;
  p->omega_h = omega_h;
  p->gamma0 = gamma0;
  p->mg = o;
  cudaGetDevice(&p->device);
  for (int l = 0; l < o.levels; ++l) {
    p->lnx[l] = nx >> l;
    p->lny[l] = ny >> l;
  }
  long n0 = p->npts(0);
  std::vector<void*> tmp;
  auto fail = [&](int code) {
    for (void* t : tmp) cudaFree(t);
    helm_problem_destroy(p);
    return code;
  };
  if (cudaMalloc(&p->kappa, n0 * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&p->gamma, n0 * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&p->massA, n0 * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&p->massA64, n0 * sizeof(double2)) != cudaSuccess) {
    set_error("helm_problem_create: out of device memory");
    return fail(HELM_ENOMEM);
  }
  for (int l = 0; l < o.levels; ++l) {
    if (cudaMalloc(&p->massSL[l], p->npts(l) * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&p->dinvSL[l], p->npts(l) * sizeof(float2)) != cudaSuccess) {
      set_error("helm_problem_create: out of device memory");
      return fail(HELM_ENOMEM);
    }
  }
  for (double*& b : p->setup64) {
    if (cudaMalloc(&b, n0 * 8) != cudaSuccess) {
      b = nullptr;
      set_error("helm_problem_create: out of device memory for the setup pyramids");
      return fail(HELM_ENOMEM);
    }
  }
  int rc = run_setup(p, kappa_dev, st);
  if (rc) return fail(rc);
  *out = p;
  return HELM_OK;
}

int helm_problem_update(helm_problem* p, const float* kappa_dev, double omega_h, void* stream) {
  using namespace helm;
  if (!p || !kappa_dev || !(omega_h > 0.0)) {
    set_error("helm_problem_update: invalid argument");
    return HELM_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) {
    set_error("helm_problem_update: the current device is not the problem's device");
    return HELM_EINVAL;
  }
  p->omega_h = omega_h;
  const int rc = run_setup(p, kappa_dev, static_cast<cudaStream_t>(stream));
  ++p->version;
  return rc;
}

int helm_problem_destroy(helm_problem* p) {
  if (!p) return HELM_OK;
  cudaFree(p->kappa);
  cudaFree(p->gamma);
  cudaFree(p->massA);
  cudaFree(p->massA64);
  for (int l = 0; l < HELM_MAX_LEVELS; ++l) {
    cudaFree(p->massSL[l]);
    cudaFree(p->dinvSL[l]);
  }
  for (double* b : p->setup64) cudaFree(b);
  delete p;
  return HELM_OK;
}

int helm_problem_level_shape(const helm_problem* p, int level, int* nx, int* ny) {
  if (!p || level < 0 || level >= p->mg.levels) {
    helm::set_error("helm_problem_level_shape: invalid argument");
    return HELM_EINVAL;
  }
  if (nx) *nx = p->lnx[level];
  if (ny) *ny = p->lny[level];
  return HELM_OK;
}

int helm_problem_get_field(const helm_problem* p, int which, int level, void* out_dev, void* stream_) {
  if (!p || !out_dev || level < 0 || level >= p->mg.levels) {
    helm::set_error("helm_problem_get_field: invalid argument");
    return HELM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  const void* src = nullptr;
  size_t bytes = 0;
  switch (which) {
    case 0: src = p->massA; bytes = p->npts(0) * sizeof(float2); break;
    case 1: src = p->massSL[level]; bytes = p->npts(level) * sizeof(float2); break;
    case 2: src = p->dinvSL[level]; bytes = p->npts(level) * sizeof(float2); break;
    case 3: src = p->gamma; bytes = p->npts(0) * sizeof(float); break;
    case 4: src = p->kappa; bytes = p->npts(0) * sizeof(float); break;
    default: helm::set_error("helm_problem_get_field: unknown field %d", which); return HELM_EINVAL;
  }
  if ((which == 0 || which >= 3) && level != 0) {
    helm::set_error("helm_problem_get_field: field %d exists on level 0 only", which);
    return HELM_EINVAL;
  }
  HELM_CUDA(cudaMemcpyAsync(out_dev, src, bytes, cudaMemcpyDeviceToDevice, st));
  return HELM_OK;
}

}  // extern "C"

// ---- launch counting and the opt-in per-kernel event profiler -----------------------
#include <atomic>
#include <map>
#include <string>
#include <vector>

namespace helm {

static std::atomic<unsigned long long> g_launches{0};

struct ProfState {
  bool on = false;
  std::mutex mu;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Rec {
    const char* name;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  cudaEvent_t pending = nullptr;
  std::map<std::string, std::pair<long, double>> totals;  // name -> (launches, ms)
};
static ProfState g_prof;

static cudaEvent_t prof_event() {
  if (g_prof.used == g_prof.pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    g_prof.pool.push_back(e);
  }
  return g_prof.pool[g_prof.used++];
}

static void prof_flush() {
  // called with the mutex held: resolve every recorded pair
  for (auto& r : g_prof.recs) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto& t = g_prof.totals[r.name];
    t.first += 1;
    t.second += ms;
  }
  g_prof.recs.clear();
  g_prof.used = 0;
}

void prof_before(const char*, cudaStream_t st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_prof.on) return;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (g_prof.used + 2 > 4096) prof_flush();
  g_prof.pending = prof_event();
  cudaEventRecord(g_prof.pending, st);
}

void prof_after(const char* name, cudaStream_t st) {
  if (!g_prof.on) return;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  cudaEvent_t b = prof_event();
  cudaEventRecord(b, st);
  g_prof.recs.push_back({name, g_prof.pending, b});
}

}  // namespace helm

extern "C" {

unsigned long long helm_launch_count(void) { return helm::g_launches.load(); }

int helm_profile_begin(void) {
  std::lock_guard<std::mutex> lk(helm::g_prof.mu);
  helm::prof_flush();
  helm::g_prof.totals.clear();
  helm::g_prof.on = true;
  return HELM_OK;
}

int helm_profile_end(int* nkernels) {
  std::lock_guard<std::mutex> lk(helm::g_prof.mu);
  helm::prof_flush();
  helm::g_prof.on = false;
  if (nkernels) *nkernels = static_cast<int>(helm::g_prof.totals.size());
  return HELM_OK;
}

int helm_profile_read(int idx, const char** name, long* launches, double* total_ms) {
  std::lock_guard<std::mutex> lk(helm::g_prof.mu);
  if (idx < 0 || idx >= static_cast<int>(helm::g_prof.totals.size())) {
    helm::set_error("helm_profile_read: index out of range");
    return HELM_EINVAL;
  }
  auto it = helm::g_prof.totals.begin();
  std::advance(it, idx);
  if (name) *name = it->first.c_str();
  if (launches) *launches = it->second.first;
  if (total_ms) *total_ms = it->second.second;
  return HELM_OK;
}

}  // extern "C"
