// Shared device/host helpers for the Helmholtz library: error handling, complex
// arithmetic on float2/double2, mbarrier + TMA wrappers (inline PTX, sm_103a),
// bounded waits that report instead of hanging.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <atomic>
#include <cstdio>
#include <string>

#include "../../include/helm.h"

// ----------------------------------------------------------------------------
// host-side error reporting
// ----------------------------------------------------------------------------
namespace helm {

void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

}  // namespace helm

#define HELM_CUDA(call)                                                  \
  do {                                                                   \
    cudaError_t _e = (call);                                             \
    if (_e != cudaSuccess) return helm::cuda_fail(_e, #call);            \
  } while (0)

#define HELM_CHECK_LAUNCH(what)                                          \
  do {                                                                   \
    cudaError_t _e = cudaGetLastError();                                 \
    if (_e != cudaSuccess) return helm::cuda_fail(_e, what);             \
  } while (0)

namespace helm {
// Every kernel launch of the library goes through HELM_LAUNCH: it counts the launch
// and, when profiling is switched on (helm_profile_begin), brackets it with CUDA
// events on the launching stream, accumulated per kernel name.
void prof_before(const char* name, cudaStream_t st);
void prof_after(const char* name, cudaStream_t st);
}  // namespace helm

#define HELM_LAUNCH(name, st, ...)      \
  do {                                  \
    helm::prof_before(name, st);        \
    __VA_ARGS__;                        \
    helm::prof_after(name, st);         \
  } while (0)

// Device error word (bit flags, see helm.h HELM_DEVERR_*).  Kernels OR bits in;
// the host reads and clears it through helm_device_errors().
extern __device__ unsigned int g_helm_device_error;

// ----------------------------------------------------------------------------
// complex helpers
// ----------------------------------------------------------------------------
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double zabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// ----------------------------------------------------------------------------
// mbarrier / TMA (inline PTX)
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase.  Returns false (and flags the device error
// word) if the phase did not complete within `limit` polls; never spins forever.
#define HELM_WAIT_LIMIT (1u << 24)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned flag) {
  for (uint32_t it = 0; it < HELM_WAIT_LIMIT; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
  }
  atomicOr(&g_helm_device_error, flag);
  return false;
}

// Bounded wait that lets the waiting thread sleep: each try_wait may suspend the thread
// for up to `ns` nanoseconds until the phase completes, instead of spinning on issue
// slots that the working warps of the SM need.  At most HELM_SLEEP_WAIT_LIMIT tries.
#define HELM_SLEEP_WAIT_LIMIT (1u << 16)
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* bar, uint32_t parity, unsigned flag) {
  for (uint32_t it = 0; it < HELM_SLEEP_WAIT_LIMIT; ++it) {
    if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
  }
  atomicOr(&g_helm_device_error, flag);
  return false;
}

// 3-D tiled TMA load global -> shared, completion signalled on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// 4-D tiled TMA load global -> shared, completion signalled on `bar`.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// ----------------------------------------------------------------------------
// warp / block reductions
// ----------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ----------------------------------------------------------------------------
// host: TMA descriptor creation (driver entry point fetched at run time)
// ----------------------------------------------------------------------------
namespace helm {

// Tensor map over a complex64 batch [nb][ny][nx] (viewed as float32 pairs), box of
// box_w complex x box_h rows x 1 batch item, zero fill outside the tensor.
int make_c64_map(CUtensorMap* out, const void* base, int nx, int ny, int nb, int box_w, int box_h);

// Tensor map over one 8-channel group of a BF16 NHWC tensor [nb][H][W][C]: `base` points
// at channel 8g of pixel 0; dims (8 channels, W, H, nb), box 8 x box_w x box_h x 1, zero
// fill outside the tensor.  A box lands in shared memory as box_h x box_w pixels of 16 B.
int make_bf16_nhwc_map(CUtensorMap* out, const void* base, int C, int W, int H, int B, int box_w, int box_h);

// Tuned launch-shape value of `knob` for a layer of height `height` on `batch` images
// (0: none; tune.cu).
int tune_get(int knob, int height, int batch);

inline int div_up(long a, long b) { return static_cast<int>((a + b - 1) / b); }

// Multiprocessor count of the current device (cached per device).
int sm_count(int* out);

// Raise `kernel`'s dynamic shared-memory limit to `bytes` on the current device, once
// per device: `done` is the caller's bitmask of devices already configured (the
// attribute belongs to a device, so a process using several GPUs sets it on each).
// The mask is atomic: host threads calling into the library concurrently at most
// repeat the (idempotent) attribute call.
template <class K>
inline int smem_attr_once(K* kernel, int bytes, std::atomic<unsigned long long>* done) {
  int dev = 0;
  HELM_CUDA(cudaGetDevice(&dev));
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done->load(std::memory_order_acquire) & bit)) {
    HELM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done->fetch_or(bit, std::memory_order_acq_rel);
  }
  return HELM_OK;
}

}  // namespace helm
