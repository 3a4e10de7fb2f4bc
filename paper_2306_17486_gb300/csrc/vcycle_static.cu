// The shifted-Laplacian V(1,1) cycle of helm_slmg_vcycle, with its scratch in a fixed
// device array of this file instead of a caller workspace.
//
// Some callers cannot hand the library a workspace: a preconditioner callback of an
// external Krylov package receives only (input, output), and allocating device memory
// inside such a callback would add a device-wide synchronisation (cudaMalloc/cudaFree
// serialise with all streams) to every iteration.  This entry point serves them: it
// allocates nothing and calls no allocating CUDA or library routine.  Its scratch is a
// file-scope __device__ array of HELM_VCYCLE_STATIC_BYTES, present on every device the
// library's module is loaded on; its address is taken once per device, on the first
// call, with cudaGetSymbolAddress, and kept for the life of the process.  After a
// cudaDeviceReset (which unloads the module and its array) that kept address is stale,
// so this entry point must not be used on a device that has been reset.
#include <mutex>

#include "problem.h"

namespace {

constexpr size_t kScratchBytes = HELM_VCYCLE_STATIC_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_vcycle_scratch[kScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Address of the scratch array on `dev` (set up on the first call for that device).
int scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* a = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&a, g_vcycle_scratch);
    if (e != cudaSuccess || !a) {
      helm::set_error("helm_slmg_vcycle_static: cudaGetSymbolAddress of the static scratch failed on device %d: %s",
                      dev, cudaGetErrorString(e));
      return HELM_ECUDA;
    }
    g_scratch_addr[dev] = a;
  }
  *out = g_scratch_addr[dev];
  return HELM_OK;
}

}  // namespace

extern "C" int helm_slmg_vcycle_static(const helm_problem* p, const void* r, void* z, int batch, void* stream) {
  if (!p || !r || !z || batch <= 0 || r == z) {
    helm::set_error("helm_slmg_vcycle_static: invalid argument (r and z must be distinct device buffers)");
    return HELM_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    helm::set_error("helm_slmg_vcycle_static: no usable current device (supported: ids 0..%d)", kMaxDevices - 1);
    return HELM_ECUDA;
  }
  if (dev != p->device) {
    helm::set_error("helm_slmg_vcycle_static: current device %d is not the problem's device %d", dev, p->device);
    return HELM_EINVAL;
  }
  // scratch this call needs: the V-cycle's per-level buffers, measured on a null base
  helm::Carve probe(nullptr, ~size_t(0));
  helm::VcycleScratch s;
  helm::carve_vcycle(probe, p, batch, &s);
  if (probe.off > kScratchBytes) {
    helm::set_error("helm_slmg_vcycle_static: %d right-hand sides of this grid need %zu bytes of scratch; the static "
                    "scratch holds %zu (use helm_slmg_vcycle with a workspace, or a smaller batch)",
                    batch, probe.off, kScratchBytes);
    return HELM_EWORKSPACE;
  }
  void* base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc) return rc;
  helm::Carve c(base, kScratchBytes);
  helm::carve_vcycle(c, p, batch, &s);
  return helm::launch_vcycle(p, static_cast<const float2*>(r), static_cast<float2*>(z), batch, s, nullptr,
                             static_cast<cudaStream_t>(stream));
}
