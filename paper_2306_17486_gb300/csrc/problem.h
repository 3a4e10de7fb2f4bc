// Internal definition of helm_problem and the workspace carve-out helpers shared by
// the translation units of the library.
#pragma once

#include <vector>

#include "common.cuh"

#define HELM_MAX_LEVELS 8
#define HELM_MAX_RESTART 32

struct helm_problem {
  int nx, ny, abl;
  double omega_h, gamma0;
  helm_mg_opts mg;
  int device;
  int lnx[HELM_MAX_LEVELS], lny[HELM_MAX_LEVELS];
  float* kappa = nullptr;                    // [ny][nx]
  float* gamma = nullptr;                    // [ny][nx]
  float2* massA = nullptr;                   // fine Helmholtz mass (omega h)^2 k^2 (1 - gamma i)
  double2* massA64 = nullptr;                // the same in FP64, for the true residual
  float2* massSL[HELM_MAX_LEVELS] = {};      // SL mass per level
  float2* dinvSL[HELM_MAX_LEVELS] = {};      // omega_J / (4 - massSL)
  unsigned long long version = 0;            // bumped by helm_problem_update
  double* setup64[4] = {};                   // FP64 kappa^2 / gamma pyramid scratch of the setup
  long npts(int l = 0) const { return static_cast<long>(lnx[l]) * lny[l]; }
};

namespace helm {

// Bump allocator over a caller-provided workspace (256-byte aligned slices).
struct Carve {
  char* base;
  size_t cap;
  size_t off = 0;
  bool overflow = false;
  Carve(void* b, size_t c) : base(static_cast<char*>(b)), cap(c) {}
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (off + bytes > cap) overflow = true;
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += bytes;
    return overflow ? nullptr : p;
  }
};

// Scratch of one V-cycle: per coarse level l >= 1 a residual and a correction
// buffer [batch][n_l], plus the coarsest GMRES basis [batch][K+1][n_c].
struct VcycleScratch {
  float2* rc[HELM_MAX_LEVELS] = {};
  float2* ec[HELM_MAX_LEVELS] = {};
  float2* basis = nullptr;
};
void carve_vcycle(Carve& c, const helm_problem* p, int batch, VcycleScratch* s);

// Launch one V-cycle (all kernels on `stream`).  `active` (nullable, device int[batch])
// masks right-hand sides that are skipped.  `zadd` (nullable) is added to the
// finest-level output (z = zadd + V(r)).
int launch_vcycle(const helm_problem* p, const float2* r, float2* z, int batch, const VcycleScratch& s,
                  const int* active, cudaStream_t stream, const float2* zadd = nullptr);

// y = c - h^2 A x (c nullable: y = h^2 A x) with the fine Helmholtz mass, masked.
int launch_apply(const helm_problem* p, const float2* mass, const float2* x, const float2* c, float2* y,
                 int batch, int level, const int* active, cudaStream_t stream);

// r = b - h^2 A x in FP64; writes r (complex64) and per-block partial ||r||^2.
int launch_residual_fp64(const helm_problem* p, const float2* b, const double2* x, float2* r, double* partial,
                         int nblk_per_rhs, int batch, const int* active, cudaStream_t stream);
int residual_blocks(const helm_problem* p);
int launch_sum_partials(const double* partial, int nblk, int batch, double* out, cudaStream_t st);

}  // namespace helm
