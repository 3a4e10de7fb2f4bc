// Internal definition of helm_cnn: the encoder-solver network's parameter table,
// derived device state (packed BF16 weights, folded BatchNorm, Green's functions per
// coarsest size, cached encodings) and the layer plan executed by cnn.cu / cnn_train.cu.
#pragma once

#include <map>
#include <string>
#include <vector>

#include "cnn_kern.h"

namespace helm {

enum LayerKind { L_CONV = 0, L_DW = 1, L_IMPL = 2, L_IB = 3 };

struct ParamInfo {
  std::string name;
  std::vector<int> shape;
  size_t offset, count;
};

struct BnInfo {
  std::string name;
  int C;
  size_t roff;  // offset of [mean C | var C] in the running-statistics buffer
  int pg, pb;   // parameter indices of gamma, beta
};

struct TensorDesc {
  int B, H, W, C;
  size_t off;   // byte offset in the activation arena
  size_t bytes() const { return static_cast<size_t>(B) * H * W * C * 2; }
};

struct Layer {
  int kind;
  int wparam;        // parameter index of the weights
  int bn;            // BatchNorm index or -1
  int mode, taps, ci, co, act;
  int in, out, add1, add2;  // tensor ids (-1: none); add2 may have batch 1 (broadcast)
  size_t wpk_off;    // element offset of this layer's packed weights
  // L_IB (fused inverted bottleneck, inference only): wparam / bn = expansion,
  // wp_dw / bn_dw = depthwise, wp_proj / bn_proj = projection
  int wp_dw = -1, bn_dw = -1, wp_proj = -1, bn_proj = -1;
};

// A plan for one (H x W grid, B, skip) configuration: tensors and layers of either the
// encoder (batch 1) or the solver (batch B).  The coarsest map is my x mx; m = my on the
// paper's square grids (training plans are square).
struct Plan {
  int H = 0, W = 0, B = 0, skip = 0, m = 0, my = 0, mx = 0;
  std::vector<TensorDesc> t;
  std::vector<Layer> layers;
  size_t arena = 0;  // bytes of all activation tensors
  int add_tensor(int B_, int H, int W, int C) {
    TensorDesc d{B_, H, W, C, arena};
    arena += (d.bytes() + 255) & ~size_t(255);
    t.push_back(d);
    return static_cast<int>(t.size()) - 1;
  }
};

}  // namespace helm

struct helm_cnn {
  helm_cnn_desc desc;
  std::vector<helm::ParamInfo> params;
  std::map<std::string, int> pidx;
  std::vector<helm::BnInfo> bns;
  std::map<std::string, int> bidx;
  size_t nparams = 0, nrunning = 0;
  const float* params_dev = nullptr;  // caller-owned FP32 master parameters
  float* running = nullptr;           // owned: BN running mean/var
  float* fold = nullptr;              // owned: folded BN scale/shift [same layout as running]
  __nv_bfloat16* wpk = nullptr;       // owned: packed conv weights
  size_t wpk_elems = 0;
  __nv_bfloat16* wfold = nullptr;     // owned: inverted-bottleneck 1x1 weights with BN folded in
                                      // (expansion BF16, projection FP16 bits)
  size_t wfold_elems = 0;
  std::map<int, size_t> wfold_off;    // parameter index -> element offset in wfold
  std::map<int, float2*> ghat;        // owned: Green's function per coarsest size m (square maps)
  std::map<std::pair<int, int>, float2*> ghat_rect;   // owned: per (m_y, m_x) of rectangular maps
  float2* gscratch = nullptr;
  size_t gscratch_elems = 0;
  bool dirty = true;                  // params/running changed since the last derive()
  // encodings cached for one problem
  const helm_problem* enc_prob = nullptr;
  unsigned long long enc_pversion = 0;  // enc_prob->version the encodings were computed for
  int enc_H = 0, enc_W = 0;
  unsigned long long enc_version = 0, param_version = 0;
  void* enc_arena = nullptr;
  size_t enc_arena_bytes = 0;
  helm::Plan enc_plan;
  int enc_out[3] = {-1, -1, -1};
  int kf = -1;
  int train_nprob = 0;  // slowness models of the last training forward
};

namespace helm {

// parameter and BN lookup
inline int P(const helm_cnn* c, const std::string& n) { return c->pidx.at(n); }
void build_encoder_plan(const helm_cnn* c, int H, int W, Plan* pl, int* outs, int* kf, int Bk);
// fuse_ib: each inverted bottleneck as one L_IB layer (inference); otherwise expansion,
// depthwise and projection as separate layers with their activations (training)
void build_solver_plan(const helm_cnn* c, int H, int W, int B, int skip, Plan* pl, int* x0, int* u3, int enc_ids[3],
                       int Bk, bool fuse_ib = false);
// pack weights, fold BN, build G_hat of the my x mx coarsest map (none when my = 0)
int cnn_derive(helm_cnn* c, int my, int mx, cudaStream_t st);
inline int cnn_derive(helm_cnn* c, int m, cudaStream_t st) { return cnn_derive(c, m, m, st); }
// G_hat of the my x mx coarsest map (derived by cnn_derive)
const float2* ghat_of(const helm_cnn* c, int my, int mx);
// skip the solver's last downsampling: the shorter side below the threshold
int skip_for(const helm_cnn* c, int H, int W);
size_t packed_elems(const helm_cnn* c, const ParamInfo& pi);
size_t wpk_offset(const helm_cnn* c, int param);
size_t cnn_train_bytes(const helm_cnn* c, int I, int B, int nprob);
int cnn_forward_infer(helm_cnn* c, const helm_problem* p, const float2* r, float2* e, int B, Carve& cv,
                      cudaStream_t st);
int cnn_forward_train(helm_cnn* c, const helm_problem* const* probs, int nprob, const float2* r, float2* e, int B,
                      Carve& cv, cudaStream_t st);

}  // namespace helm
