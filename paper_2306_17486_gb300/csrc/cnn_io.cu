// Saving and loading a network (helm_cnn_save / helm_cnn_load).  Section 4.2 notes
// that the implicit layer's Green's function G_hat (Eq. 15) is computed from the
// learned kernel once and stored as part of the network; a saved network therefore
// carries, next to its FP32 parameters and BatchNorm running statistics, the G_hat of
// every coarsest size the handle has built, and a loaded one uses them without
// rebuilding.
//
// File layout (little-endian, as written by the host):
//   char[8]  magic "HELMCNN1"
//   int32    c0, expansion, skip_threshold, literal_green, explicit_unet
//   uint64   nparams, nrunning
//   uint32   n_ghat; then n_ghat x (int32 m, int32 nk)
//   float    params[nparams], running[nrunning]
//   float2   ghat_i[nk][2m][2m] for each stored size, in header order
//   uint64   FNV-1a hash of every byte above
#include <cstdio>
#include <cstring>
#include <vector>

#include "cnn_impl.h"

namespace {

constexpr char kMagic[8] = {'H', 'E', 'L', 'M', 'C', 'N', 'N', '1'};

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  }
};

struct Writer {
  FILE* f;
  Fnv fnv;
  bool ok = true;
  void put(const void* p, size_t n) {
    if (ok && fwrite(p, 1, n, f) != n) ok = false;
    fnv.add(p, n);
  }
};

struct Reader {
  FILE* f;
  Fnv fnv;
  bool get(void* p, size_t n) {
    if (fread(p, 1, n, f) != n) return false;
    fnv.add(p, n);
    return true;
  }
};

int nk_of(const helm_cnn* c) { return c->desc.explicit_unet ? 0 : c->params[c->pidx.at("s.imp.K")].shape[1]; }

}  // namespace

extern "C" {

int helm_cnn_save(helm_cnn* c, const char* path, void* stream) {
  using namespace helm;
  if (!c || !path) {
    set_error("helm_cnn_save: invalid argument");
    return HELM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = cnn_derive(c, 0, st);   // G_hat cached for the current parameters only
  if (rc) return rc;
  std::vector<float> params(c->nparams), running(c->nrunning);
  HELM_CUDA(cudaMemcpyAsync(params.data(), c->params_dev, c->nparams * sizeof(float), cudaMemcpyDeviceToHost, st));
  HELM_CUDA(cudaMemcpyAsync(running.data(), c->running, c->nrunning * sizeof(float), cudaMemcpyDeviceToHost, st));
  const int nk = nk_of(c);
  std::vector<std::pair<int, std::vector<float2>>> gh;
  for (const auto& kv : c->ghat) {
    const int m = kv.first;
    gh.emplace_back(m, std::vector<float2>(static_cast<size_t>(nk) * 4 * m * m));
    HELM_CUDA(cudaMemcpyAsync(gh.back().second.data(), kv.second, gh.back().second.size() * sizeof(float2),
                              cudaMemcpyDeviceToHost, st));
  }
  HELM_CUDA(cudaStreamSynchronize(st));
  FILE* f = fopen(path, "wb");
  if (!f) {
    set_error("helm_cnn_save: cannot open %s for writing", path);
    return HELM_EINVAL;
  }
  Writer w{f};
  w.put(kMagic, sizeof(kMagic));
  const int32_t d[5] = {c->desc.c0, c->desc.expansion, c->desc.skip_threshold, c->desc.literal_green,
                        c->desc.explicit_unet};
  w.put(d, sizeof(d));
  const uint64_t counts[2] = {c->nparams, c->nrunning};
  w.put(counts, sizeof(counts));
  const uint32_t ng = static_cast<uint32_t>(gh.size());
  w.put(&ng, sizeof(ng));
  for (const auto& g : gh) {
    const int32_t mk[2] = {g.first, nk};
    w.put(mk, sizeof(mk));
  }
  w.put(params.data(), params.size() * sizeof(float));
  w.put(running.data(), running.size() * sizeof(float));
  for (const auto& g : gh) w.put(g.second.data(), g.second.size() * sizeof(float2));
  const uint64_t h = w.fnv.h;
  if (w.ok && fwrite(&h, 1, sizeof(h), f) != sizeof(h)) w.ok = false;
  if (fclose(f) != 0) w.ok = false;
  if (!w.ok) {
    set_error("helm_cnn_save: write to %s failed", path);
    return HELM_EINVAL;
  }
  return HELM_OK;
}

int helm_cnn_load(helm_cnn* c, const char* path, float* params_dev, void* stream) {
  using namespace helm;
  if (!c || !path || !params_dev) {
    set_error("helm_cnn_load: invalid argument");
    return HELM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FILE* f = fopen(path, "rb");
  if (!f) {
    set_error("helm_cnn_load: cannot open %s", path);
    return HELM_EINVAL;
  }
  Reader r{f};
  char magic[8];
  int32_t d[5];
  uint64_t counts[2];
  uint32_t ng = 0;
  bool ok = r.get(magic, sizeof(magic)) && memcmp(magic, kMagic, sizeof(magic)) == 0 && r.get(d, sizeof(d)) &&
            r.get(counts, sizeof(counts)) && r.get(&ng, sizeof(ng));
  const int nk = nk_of(c);
  if (ok && (d[0] != c->desc.c0 || d[1] != c->desc.expansion || d[2] != c->desc.skip_threshold ||
             d[3] != c->desc.literal_green || d[4] != c->desc.explicit_unet || counts[0] != c->nparams ||
             counts[1] != c->nrunning || ng > 64)) {
    fclose(f);
    set_error("helm_cnn_load: %s was saved from a network with another descriptor or parameter table", path);
    return HELM_EINVAL;
  }
  std::vector<int> ms;
  for (uint32_t i = 0; ok && i < ng; ++i) {
    int32_t mk[2];
    ok = r.get(mk, sizeof(mk)) && mk[0] > 0 && mk[0] <= 4096 && mk[1] == nk;
    if (ok) ms.push_back(mk[0]);
  }
  std::vector<float> params(ok ? c->nparams : 0), running(ok ? c->nrunning : 0);
  ok = ok && r.get(params.data(), params.size() * sizeof(float)) &&
       r.get(running.data(), running.size() * sizeof(float));
  std::vector<std::vector<float2>> gh;
  for (size_t i = 0; ok && i < ms.size(); ++i) {
    gh.emplace_back(static_cast<size_t>(nk) * 4 * ms[i] * ms[i]);
    ok = r.get(gh.back().data(), gh.back().size() * sizeof(float2));
  }
  uint64_t h = 0;
  const uint64_t want = r.fnv.h;
  ok = ok && fread(&h, 1, sizeof(h), f) == sizeof(h) && h == want;
  fclose(f);
  if (!ok) {
    set_error("helm_cnn_load: %s is not a complete network file of this library (bad magic, size or hash)", path);
    return HELM_EINVAL;
  }
  // parameters into the caller's vector, statistics into the handle; derive the packed
  // weights and folded BN now, then install the stored Green's functions
  HELM_CUDA(cudaMemcpyAsync(params_dev, params.data(), params.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  HELM_CUDA(cudaMemcpyAsync(c->running, running.data(), running.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  c->params_dev = params_dev;
  c->dirty = true;
  c->param_version++;
  int rc = cnn_derive(c, 0, st);
  if (rc) return rc;
  for (size_t i = 0; i < ms.size(); ++i) {
    float2* g = nullptr;
    if (cudaMalloc(&g, gh[i].size() * sizeof(float2)) != cudaSuccess) {
      set_error("helm_cnn_load: out of device memory for G_hat");
      return HELM_ENOMEM;
    }
    const cudaError_t e = cudaMemcpyAsync(g, gh[i].data(), gh[i].size() * sizeof(float2), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      cudaFree(g);
      return cuda_fail(e, "helm_cnn_load: G_hat copy");
    }
    auto it = c->ghat.find(ms[i]);
    if (it != c->ghat.end()) cudaFree(it->second);
    c->ghat[ms[i]] = g;
  }
  HELM_CUDA(cudaStreamSynchronize(st));   // the host staging vectors go out of scope
  return HELM_OK;
}

}  // extern "C"
