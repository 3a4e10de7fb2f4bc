// The encoder-solver network (Sections 4.1-4.4, 5.3) on the device: parameter table,
// derived state, the layer plans of the encoder and of the solver, inference forward,
// the composed preconditioner z = e + V(r - A e) (Section 4.1, reading: the network
// output is smoothed by a V-cycle on the residual equation), and the C ABI.
//
// Layer sequence (c0 = 16, t = 6; I = grid side incl. the absorbing layer):
//   encoder (batch 1): (Re, Im) kappa^2(1 - gamma i) at I -> 3 downsampling modules
//     [3x3 s2 conv, 3x3 conv, 3x3 conv, each + BN + softplus] -> enc1 (16, I/2),
//     enc2 (32, I/4), enc3 (64, I/8)
//   solver (batch B): x0 = R(r/s), s = RMS(r), -> level k: conv (s1, s2, s2) + BN + softplus
//     + enc_k, inverted bottleneck (1x1 expand + BN + softplus, dw 3x3 + BN + softplus,
//     1x1 project + BN, + identity) -> g_k; level 4: 3 convs (first s2, or s1 below the
//     skip threshold) -> implicit layer -> up modules (transposed conv + 2 convs, + g_{4-k})
//     -> 1x1 projection 16 -> 2 + bias -> bilinear P to I -> times s.
#include <cmath>
#include <cstring>

#include "cnn_impl.h"

namespace helm {

namespace {

void add_param(helm_cnn* c, const std::string& n, std::vector<int> shape) {
  size_t cnt = 1;
  for (int s : shape) cnt *= s;
  c->pidx[n] = static_cast<int>(c->params.size());
  c->params.push_back({n, shape, c->nparams, cnt});
  c->nparams += cnt;
}

void add_bn(helm_cnn* c, const std::string& n, int C) {
  add_param(c, n + ".g", {C});
  add_param(c, n + ".b", {C});
  c->bidx[n] = static_cast<int>(c->bns.size());
  c->bns.push_back({n, C, c->nrunning, c->pidx[n + ".g"], c->pidx[n + ".b"]});
  c->nrunning += 2 * C;
}

void build_params(helm_cnn* c) {
  const int c0 = c->desc.c0, t = c->desc.expansion;
  const int C[3] = {c0, 2 * c0, 4 * c0};
  int cin = 2;
  for (int k = 0; k < 3; ++k) {
    const std::string p = "e.dm" + std::to_string(k + 1);
    add_param(c, p + ".conv0.w", {C[k], cin, 3, 3});
    add_bn(c, p + ".bn0", C[k]);
    for (int j = 1; j <= 2; ++j) {
      add_param(c, p + ".conv" + std::to_string(j) + ".w", {C[k], C[k], 3, 3});
      add_bn(c, p + ".bn" + std::to_string(j), C[k]);
    }
    cin = C[k];
  }
  cin = 2;
  for (int k = 0; k < 3; ++k) {
    const std::string p = "s.l" + std::to_string(k + 1);
    add_param(c, p + ".conv.w", {C[k], cin, 3, 3});
    add_bn(c, p + ".bn", C[k]);
    add_param(c, p + ".ib.exp.w", {t * C[k], C[k]});
    add_bn(c, p + ".ib.bn0", t * C[k]);
    add_param(c, p + ".ib.dw.w", {t * C[k], 3, 3});
    add_bn(c, p + ".ib.bn1", t * C[k]);
    add_param(c, p + ".ib.proj.w", {C[k], t * C[k]});
    add_bn(c, p + ".ib.bn2", C[k]);
    cin = C[k];
  }
  for (int j = 0; j < 3; ++j) {
    add_param(c, "s.l4.conv" + std::to_string(j) + ".w", {C[2], C[2], 3, 3});
    add_bn(c, "s.l4.bn" + std::to_string(j), C[2]);
  }
  if (!c->desc.explicit_unet) add_param(c, "s.imp.K", {2, C[2] / 2, 3, 3});
  const int ups[3][2] = {{C[2], C[2]}, {C[2], C[1]}, {C[1], C[0]}};
  for (int k = 0; k < 3; ++k) {
    const std::string p = "s.up" + std::to_string(k + 1);
    add_param(c, p + ".convT.w", {ups[k][0], ups[k][1], 3, 3});
    add_bn(c, p + ".bn0", ups[k][1]);
    for (int j = 1; j <= 2; ++j) {
      add_param(c, p + ".conv" + std::to_string(j) + ".w", {ups[k][1], ups[k][1], 3, 3});
      add_bn(c, p + ".bn" + std::to_string(j), ups[k][1]);
    }
  }
  add_param(c, "s.proj.w", {2, C[0]});
  add_param(c, "s.proj.b", {2});
}

}  // namespace

size_t packed_elems(const helm_cnn* c, const ParamInfo& pi) {
  (void)c;
  if (pi.shape.size() == 4) {  // 3x3 conv [co][ci][3][3] or transposed [ci][co][3][3]
    const bool tr = pi.name.find("convT") != std::string::npos;
    const int ci = tr ? pi.shape[0] : pi.shape[1], co = tr ? pi.shape[1] : pi.shape[0];
    return static_cast<size_t>(9) * conv_cs(ci) * co;
  }
  if (pi.shape.size() == 2 && (pi.name.find(".exp.w") != std::string::npos ||
                               pi.name.find(".proj.w") != std::string::npos) && pi.name.rfind("s.proj", 0) != 0)
    return static_cast<size_t>(conv_cs(pi.shape[1])) * pi.shape[0];
  return 0;
}

int skip_for(const helm_cnn* c, int H, int W) { return std::min(H, W) < c->desc.skip_threshold ? 1 : 0; }

static Layer conv_layer(const helm_cnn* c, const std::string& w, const std::string& bn, int mode, int in, int out,
                        int add1, int add2, int act = 1) {
  Layer L{};
  L.kind = L_CONV;
  L.wparam = c->pidx.at(w);
  L.bn = bn.empty() ? -1 : c->bidx.at(bn);
  const ParamInfo& pi = c->params[L.wparam];
  const bool tr = mode == HELM_CONV_T2 || mode == HELM_CONV_T1;
  if (pi.shape.size() == 4) {
    L.taps = 9;
    L.ci = tr ? pi.shape[0] : pi.shape[1];
    L.co = tr ? pi.shape[1] : pi.shape[0];
  } else {
    L.taps = 1;
    L.ci = pi.shape[1];
    L.co = pi.shape[0];
  }
  L.mode = mode;
  L.act = act;
  L.in = in;
  L.out = out;
  L.add1 = add1;
  L.add2 = add2;
  L.wpk_off = 0;
  return L;
}

void build_encoder_plan(const helm_cnn* c, int Hg, int Wg, Plan* pl, int* outs, int* kf, int Bk) {
  *pl = Plan();
  pl->H = Hg;
  pl->W = Wg;
  pl->B = Bk;
  const int C[3] = {c->desc.c0, 2 * c->desc.c0, 4 * c->desc.c0};
  *kf = pl->add_tensor(Bk, Hg, Wg, 2);
  int x = *kf, H = Hg, W = Wg;
  for (int k = 0; k < 3; ++k) {
    H /= 2;
    W /= 2;
    const std::string p = "e.dm" + std::to_string(k + 1);
    const int a = pl->add_tensor(Bk, H, W, C[k]);
    const int b = pl->add_tensor(Bk, H, W, C[k]);
    const int o = pl->add_tensor(Bk, H, W, C[k]);
    pl->layers.push_back(conv_layer(c, p + ".conv0.w", p + ".bn0", HELM_CONV_S2, x, a, -1, -1));
    pl->layers.push_back(conv_layer(c, p + ".conv1.w", p + ".bn1", HELM_CONV_S1, a, b, -1, -1));
    pl->layers.push_back(conv_layer(c, p + ".conv2.w", p + ".bn2", HELM_CONV_S1, b, o, -1, -1));
    outs[k] = o;
    x = o;
  }
}

void build_solver_plan(const helm_cnn* c, int Hg, int Wg, int B, int skip, Plan* pl, int* x0, int* u3, int enc_ids[3],
                       int Bk, bool fuse_ib) {
  *pl = Plan();
  pl->H = Hg;
  pl->W = Wg;
  pl->B = B;
  pl->skip = skip;
  const int t = c->desc.expansion;
  const int C[3] = {c->desc.c0, 2 * c->desc.c0, 4 * c->desc.c0};
  int H = Hg / 2, W = Wg / 2;
  *x0 = pl->add_tensor(B, H, W, 2);
  // encodings live in the encoder's arena: placeholders, resolved at run time
  for (int k = 0; k < 3; ++k) {
    TensorDesc d{Bk, Hg >> (k + 1), Wg >> (k + 1), C[k], ~size_t(0)};
    pl->t.push_back(d);
    enc_ids[k] = static_cast<int>(pl->t.size()) - 1;
  }
  int x = *x0;
  int g[3];
  for (int k = 0; k < 3; ++k) {
    if (k > 0) {
      H /= 2;
      W /= 2;
    }
    const std::string p = "s.l" + std::to_string(k + 1);
    const int f = pl->add_tensor(B, H, W, C[k]);
    pl->layers.push_back(conv_layer(c, p + ".conv.w", p + ".bn", k == 0 ? HELM_CONV_S1 : HELM_CONV_S2, x, f, -1,
                                    enc_ids[k]));
    if (fuse_ib) {
      g[k] = pl->add_tensor(B, H, W, C[k]);
      Layer ib = conv_layer(c, p + ".ib.exp.w", p + ".ib.bn0", HELM_CONV_S1, f, g[k], -1, -1);
      ib.kind = L_IB;
      ib.wp_dw = c->pidx.at(p + ".ib.dw.w");
      ib.bn_dw = c->bidx.at(p + ".ib.bn1");
      ib.wp_proj = c->pidx.at(p + ".ib.proj.w");
      ib.bn_proj = c->bidx.at(p + ".ib.bn2");
      pl->layers.push_back(ib);
      x = g[k];
      continue;
    }
    const int a = pl->add_tensor(B, H, W, t * C[k]);
    const int d = pl->add_tensor(B, H, W, t * C[k]);
    g[k] = pl->add_tensor(B, H, W, C[k]);
    pl->layers.push_back(conv_layer(c, p + ".ib.exp.w", p + ".ib.bn0", HELM_CONV_S1, f, a, -1, -1));
    Layer dw{};
    dw.kind = L_DW;
    dw.wparam = c->pidx.at(p + ".ib.dw.w");
    dw.bn = c->bidx.at(p + ".ib.bn1");
    dw.ci = dw.co = t * C[k];
    dw.act = 1;
    dw.in = a;
    dw.out = d;
    dw.add1 = dw.add2 = -1;
    pl->layers.push_back(dw);
    pl->layers.push_back(conv_layer(c, p + ".ib.proj.w", p + ".ib.bn2", HELM_CONV_S1, d, g[k], f, -1, 0));
    x = g[k];
  }
  const int my = skip ? H : H / 2, mx = skip ? W : W / 2;
  pl->my = my;
  pl->mx = mx;
  pl->m = my;
  const int l4a = pl->add_tensor(B, my, mx, C[2]);
  const int l4b = pl->add_tensor(B, my, mx, C[2]);
  const int l4c = pl->add_tensor(B, my, mx, C[2]);
  pl->layers.push_back(conv_layer(c, "s.l4.conv0.w", "s.l4.bn0", skip ? HELM_CONV_S1 : HELM_CONV_S2, x, l4a, -1, -1));
  pl->layers.push_back(conv_layer(c, "s.l4.conv1.w", "s.l4.bn1", HELM_CONV_S1, l4a, l4b, -1, -1));
  pl->layers.push_back(conv_layer(c, "s.l4.conv2.w", "s.l4.bn2", HELM_CONV_S1, l4b, l4c, -1, -1));
  x = l4c;
  if (!c->desc.explicit_unet) {
    const int imp = pl->add_tensor(B, my, mx, C[2]);
    Layer li{};
    li.kind = L_IMPL;
    li.wparam = c->pidx.at("s.imp.K");
    li.bn = -1;
    li.ci = li.co = C[2];
    li.in = l4c;
    li.out = imp;
    li.add1 = li.add2 = -1;
    pl->layers.push_back(li);
    x = imp;
  }
  const int upc[3] = {C[2], C[1], C[0]};
  int Hu = my, Wu = mx;
  for (int k = 0; k < 3; ++k) {
    const bool s1 = (k == 0 && skip);
    if (!s1) {
      Hu *= 2;
      Wu *= 2;
    }
    const std::string p = "s.up" + std::to_string(k + 1);
    const int a = pl->add_tensor(B, Hu, Wu, upc[k]);
    const int b = pl->add_tensor(B, Hu, Wu, upc[k]);
    const int o = pl->add_tensor(B, Hu, Wu, upc[k]);
    pl->layers.push_back(conv_layer(c, p + ".convT.w", p + ".bn0", s1 ? HELM_CONV_T1 : HELM_CONV_T2, x, a, -1, -1));
    pl->layers.push_back(conv_layer(c, p + ".conv1.w", p + ".bn1", HELM_CONV_S1, a, b, -1, -1));
    pl->layers.push_back(conv_layer(c, p + ".conv2.w", p + ".bn2", HELM_CONV_S1, b, o, g[2 - k], -1));
    x = o;
  }
  *u3 = x;
}

// ---- derived state --------------------------------------------------------------

__global__ void k_fold_bn(const float* __restrict__ params, const float* __restrict__ running, const int* __restrict__ meta,
                          int nbn, float eps, float* __restrict__ fold) {
  // meta per bn: [C, roff, goff, boff]
  const int bi = blockIdx.x;
  if (bi >= nbn) return;
  const int C = meta[4 * bi], roff = meta[4 * bi + 1], goff = meta[4 * bi + 2], boff = meta[4 * bi + 3];
  for (int ch = threadIdx.x; ch < C; ch += blockDim.x) {
    const float mean = running[roff + ch], var = running[roff + C + ch];
    const float a = params[goff + ch] / sqrtf(var + eps);
    fold[roff + ch] = a;
    fold[roff + C + ch] = params[boff + ch] - mean * a;
  }
}

int cnn_derive(helm_cnn* c, int my, int mx, cudaStream_t st) {
  if (!c->params_dev) {
    set_error("cnn: parameters not set (helm_cnn_set_params)");
    return HELM_ESTATE;
  }
  if (c->dirty) {
    // pack every conv weight
    size_t off = 0;
    for (const ParamInfo& pi : c->params) {
      const size_t ne = packed_elems(c, pi);
      if (!ne) continue;
      const bool tr = pi.name.find("convT") != std::string::npos;
      int rc;
      if (pi.shape.size() == 4) {
        const int ci = tr ? pi.shape[0] : pi.shape[1], co = tr ? pi.shape[1] : pi.shape[0];
        rc = pack_conv_weights(c->params_dev + pi.offset, ci, co, 9, tr ? 1 : 0, c->wpk + off, st);
      } else {
        rc = pack_conv_weights(c->params_dev + pi.offset, pi.shape[1], pi.shape[0], 1, 0, c->wpk + off, st);
      }
      if (rc) return rc;
      off += ne;
    }
    // fold BN with the running statistics
    std::vector<int> meta;
    for (const BnInfo& b : c->bns) {
      meta.push_back(b.C);
      meta.push_back(static_cast<int>(b.roff));
      meta.push_back(static_cast<int>(c->params[b.pg].offset));
      meta.push_back(static_cast<int>(c->params[b.pb].offset));
    }
    if (!c->gscratch) {   // freed by a failed enlargement: the small table needs its head
      if (cudaMalloc(&c->gscratch, 4096 * sizeof(float2)) != cudaSuccess) {
        c->gscratch = nullptr;
        set_error("cnn: out of device memory");
        return HELM_ENOMEM;
      }
      c->gscratch_elems = 4096;
    }
    int* dmeta = reinterpret_cast<int*>(c->gscratch);  // reuse scratch head for the small table
    HELM_CUDA(cudaMemcpyAsync(dmeta, meta.data(), meta.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    HELM_LAUNCH("k_fold_bn", st,
                k_fold_bn<<<static_cast<int>(c->bns.size()), 128, 0, st>>>(c->params_dev, c->running, dmeta,
                                                                           static_cast<int>(c->bns.size()), 1e-5f,
                                                                           c->fold));
    HELM_CHECK_LAUNCH("k_fold_bn");
    // the inverted bottlenecks' 1x1 weights with BN0 / BN2 folded in (evaluation mode)
    for (const auto& kv : c->wfold_off) {
      const ParamInfo& pi = c->params[kv.first];
      const bool expw = pi.name.find(".exp.w") != std::string::npos;
      const std::string bn = pi.name.substr(0, pi.name.rfind('.', pi.name.size() - 3)) + (expw ? ".bn0" : ".bn2");
      const int rc = pack_ib_folded(c->params_dev + pi.offset, c->fold + c->bns[c->bidx.at(bn)].roff, pi.shape[1],
                                    pi.shape[0], expw ? 0 : 1, c->wfold + kv.second, st);
      if (rc) return rc;
    }
    HELM_CUDA(cudaStreamSynchronize(st));  // dmeta is scratch reused below
    for (auto& kv : c->ghat) cudaFree(kv.second);
    c->ghat.clear();
    for (auto& kv : c->ghat_rect) cudaFree(kv.second);
    c->ghat_rect.clear();
    c->dirty = false;
  }
  const bool sq = my == mx;
  if (my > 0 && mx > 0 && !c->desc.explicit_unet &&
      (sq ? !c->ghat.count(my) : !c->ghat_rect.count(std::make_pair(my, mx)))) {
    const ParamInfo& K = c->params[c->pidx.at("s.imp.K")];
    const int nk = K.shape[1];
    const size_t need = greens_scratch_elems(my, mx, nk);
    if (need > c->gscratch_elems) {
      cudaFree(c->gscratch);
      c->gscratch = nullptr;
      c->gscratch_elems = 0;
      if (cudaMalloc(&c->gscratch, need * sizeof(float2)) != cudaSuccess) {
        c->gscratch = nullptr;
        set_error("cnn: out of memory for the Green's function scratch");
        return HELM_ENOMEM;
      }
      c->gscratch_elems = need;
    }
    float2* g = nullptr;
    if (cudaMalloc(&g, static_cast<size_t>(nk) * 4 * my * mx * sizeof(float2)) != cudaSuccess) {
      set_error("cnn: out of memory for G_hat");
      return HELM_ENOMEM;
    }
    int rc = launch_greens(c->params_dev + K.offset, nk, my, mx, 1e-5f, c->desc.literal_green, c->gscratch, g, st);
    if (rc) {
      cudaFree(g);
      return rc;
    }
    if (sq)
      c->ghat[my] = g;
    else
      c->ghat_rect[std::make_pair(my, mx)] = g;
  }
  return HELM_OK;
}

const float2* ghat_of(const helm_cnn* c, int my, int mx) {
  return my == mx ? c->ghat.at(my) : c->ghat_rect.at(std::make_pair(my, mx));
}

size_t wpk_offset(const helm_cnn* c, int param) {
  size_t off = 0;
  for (int i = 0; i < param; ++i) off += packed_elems(c, c->params[i]);
  return off;
}

// Execute the layers of a plan in inference mode; `ptr[t]` = base of tensor t; iscr: the
// implicit layer's three-pass intermediate (null for the encoder)
static int run_layers_infer(helm_cnn* c, const Plan& pl, const std::vector<void*>& ptr, cudaStream_t st,
                            float2* iscr = nullptr) {
  for (const Layer& L : pl.layers) {
    const TensorDesc& in = pl.t[L.in];
    const TensorDesc& out = pl.t[L.out];
    const float* fold = L.bn >= 0 ? c->fold + c->bns[L.bn].roff : nullptr;
    const int C = L.bn >= 0 ? c->bns[L.bn].C : 0;
    int rc = HELM_OK;
    if (L.kind == L_CONV) {
      ConvLaunch cl;
      cl.x = static_cast<const __nv_bfloat16*>(ptr[L.in]);
      cl.B = in.B;
      cl.Hi = in.H;
      cl.Wi = in.W;
      cl.Ci = L.ci;
      cl.Co = L.co;
      cl.taps = L.taps;
      cl.mode = L.mode == HELM_CONV_T1 ? HELM_CONV_S1 : L.mode;
      cl.wpk = c->wpk + wpk_offset(c, L.wparam);
      cl.scale = fold;
      cl.shift = fold ? fold + C : nullptr;
      cl.act = L.act;
      cl.add1 = L.add1 >= 0 ? static_cast<const __nv_bfloat16*>(ptr[L.add1]) : nullptr;
      cl.add2 = L.add2 >= 0 ? static_cast<const __nv_bfloat16*>(ptr[L.add2]) : nullptr;
      cl.add2_div = L.add2 >= 0 ? out.B / pl.t[L.add2].B : 1;
      cl.y = static_cast<__nv_bfloat16*>(ptr[L.out]);
      rc = conv_tc(cl, st);
    } else if (L.kind == L_IB) {
      IbLaunch il;
      il.x = static_cast<const __nv_bfloat16*>(ptr[L.in]);
      il.B = in.B;
      il.H = in.H;
      il.W = in.W;
      il.C = in.C;
      il.expansion = c->desc.expansion;
      il.we = c->wpk + wpk_offset(c, L.wparam);
      il.wp = c->wpk + wpk_offset(c, L.wp_proj);
      il.wdw = c->params_dev + c->params[L.wp_dw].offset;
      il.bn0 = fold;
      il.bn1 = c->fold + c->bns[L.bn_dw].roff;
      il.bn2 = c->fold + c->bns[L.bn_proj].roff;
      il.wef = c->wfold + c->wfold_off.at(L.wparam);
      il.wpf = c->wfold + c->wfold_off.at(L.wp_proj);
      il.y = static_cast<__nv_bfloat16*>(ptr[L.out]);
      rc = ib_fused(il, st);
    } else if (L.kind == L_DW) {
      rc = launch_dw(static_cast<const __nv_bfloat16*>(ptr[L.in]), in.B, in.H, in.W, in.C,
                     c->params_dev + c->params[L.wparam].offset, fold, fold + C, L.act,
                     static_cast<__nv_bfloat16*>(ptr[L.out]), nullptr, st);
    } else {
      rc = launch_implicit_bf16(static_cast<const __nv_bfloat16*>(ptr[L.in]), in.B, in.H, in.W, in.C,
                                ghat_of(c, pl.my, pl.mx), static_cast<__nv_bfloat16*>(ptr[L.out]), st, iscr);
    }
    if (rc) return rc;
  }
  return HELM_OK;
}

// workspace of one network forward at batch B: activation arena + norms
size_t cnn_forward_bytes(const helm_cnn* c, int H, int W, int B) {
  Plan pl;
  int x0, u3, e[3];
  build_solver_plan(c, H, W, B, skip_for(c, H, W), &pl, &x0, &u3, e, 1, true);
  return pl.arena + static_cast<size_t>(B) * 256 * sizeof(double) + 2 * 256 * B * sizeof(float) +
         implicit_3pass_bytes(B, pl.my, pl.mx, 4 * c->desc.c0) + 4096;
}

// e = s Net(r / s), s = RMS(r), in inference mode, scratch from `cv`
int cnn_forward_infer(helm_cnn* c, const helm_problem* p, const float2* r, float2* e, int B, Carve& cv,
                      cudaStream_t st) {
  if (c->enc_prob != p || c->enc_version != c->param_version || c->enc_pversion != p->version) {
    set_error("cnn: encodings not computed for this problem (call helm_cnn_set_problem)");
    return HELM_ESTATE;
  }
  const int H = p->ny, W = p->nx;
  Plan pl;
  int x0, u3, enc[3];
  build_solver_plan(c, H, W, B, skip_for(c, H, W), &pl, &x0, &u3, enc, 1, true);
  int rc = cnn_derive(c, pl.my, pl.mx, st);
  if (rc) return rc;
  char* arena = cv.take<char>(pl.arena);
  double* part = cv.take<double>(static_cast<size_t>(B) * 256);
  float* s = cv.take<float>(B);
  float* inv = cv.take<float>(B);
  float2* iscr = cv.take<float2>(implicit_3pass_bytes(B, pl.my, pl.mx, 4 * c->desc.c0) / sizeof(float2));
  if (cv.overflow) {
    set_error("cnn: workspace too small");
    return HELM_EWORKSPACE;
  }
  std::vector<void*> ptr(pl.t.size());
  for (size_t i = 0; i < pl.t.size(); ++i) ptr[i] = arena + pl.t[i].off;
  for (int k = 0; k < 3; ++k)
    ptr[enc[k]] = static_cast<char*>(c->enc_arena) + c->enc_plan.t[c->enc_out[k]].off;
  if ((rc = launch_prep(r, H, W, B, part, s, inv, static_cast<__nv_bfloat16*>(ptr[x0]), st))) return rc;
  if ((rc = run_layers_infer(c, pl, ptr, st, iscr))) return rc;
  const ParamInfo& pw = c->params[c->pidx.at("s.proj.w")];
  const ParamInfo& pb = c->params[c->pidx.at("s.proj.b")];
  return launch_proj(static_cast<const __nv_bfloat16*>(ptr[u3]), B, H / 2, W / 2, pl.t[u3].C, c->params_dev + pw.offset,
                     c->params_dev + pb.offset, s, e, st);
}

int run_encoder(helm_cnn* c, const helm_problem* p, cudaStream_t st) {
  const int H = p->ny, W = p->nx;
  if (H % 16 || W % 16) {
    set_error("cnn: the network needs grid sides divisible by 16 (got %d x %d)", p->nx, p->ny);
    return HELM_ESHAPE;
  }
  int rc = cnn_derive(c, 0, st);
  if (rc) return rc;
  if (c->enc_H != H || c->enc_W != W || !c->enc_arena) {
    build_encoder_plan(c, H, W, &c->enc_plan, c->enc_out, &c->kf, 1);
    cudaFree(c->enc_arena);
    c->enc_arena = nullptr;
    if (cudaMalloc(&c->enc_arena, c->enc_plan.arena) != cudaSuccess) {
      c->enc_arena = nullptr;
      c->enc_H = c->enc_W = 0;
      set_error("cnn: out of memory for the encodings");
      return HELM_ENOMEM;
    }
    c->enc_H = H;
    c->enc_W = W;
  }
  std::vector<void*> ptr(c->enc_plan.t.size());
  for (size_t i = 0; i < ptr.size(); ++i) ptr[i] = static_cast<char*>(c->enc_arena) + c->enc_plan.t[i].off;
  if ((rc = launch_kfeat(p->kappa, p->gamma, p->npts(0), static_cast<__nv_bfloat16*>(ptr[c->kf]), st))) return rc;
  if ((rc = run_layers_infer(c, c->enc_plan, ptr, st))) return rc;
  c->enc_prob = p;
  c->enc_pversion = p->version;
  c->enc_version = c->param_version;
  return HELM_OK;
}

size_t cnn_workspace_bytes(const helm_problem* p, const helm_cnn* cnn, int batch) {
  // forward + e, r' and the compacted input / output of the network
  return cnn_forward_bytes(cnn, p->ny, p->nx, batch) + 4 * static_cast<size_t>(batch) * p->npts(0) * sizeof(float2) +
         2048;
}

// out[b] = in[sel[b]] (gather, b < nsel) or out[sel[b]] = in[b] (scatter); n points each
__global__ void k_gather_rows(const float2* __restrict__ in, float2* __restrict__ out, const int* __restrict__ sel,
                              long n, int scatter) {
  const int b = blockIdx.y;
  const long src = scatter ? b : sel[b];
  const long dst = scatter ? sel[b] : b;
  const float4* s4 = reinterpret_cast<const float4*>(in + src * n);
  float4* d4 = reinterpret_cast<float4*>(out + dst * n);
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n / 2;
       i += static_cast<long>(gridDim.x) * blockDim.x)
    d4[i] = s4[i];
}

// e[b] = 0 where zero_rows[b] != 0 (the right-hand sides that fell back to the V-cycle)
__global__ void k_zero_rows(float2* __restrict__ e, const int* __restrict__ zero_rows, long n) {
  const int b = blockIdx.y;
  if (!zero_rows[b]) return;
  float4* e4 = reinterpret_cast<float4*>(e + b * n);
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n / 2;
       i += static_cast<long>(gridDim.x) * blockDim.x)
    e4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

int launch_cnn_precond(const helm_problem* p, const helm_cnn* cnn_, const float2* r, float2* z, int batch,
                       Carve& cv, const VcycleScratch& vs, const int* active, cudaStream_t st, const int* sel,
                       int nsel, const int* zero_rows) {
  helm_cnn* cnn = const_cast<helm_cnn*>(cnn_);
  const long n = p->npts(0);
  float2* e = cv.take<float2>(static_cast<size_t>(batch) * n);
  float2* rp = cv.take<float2>(static_cast<size_t>(batch) * n);
  float2* rs = cv.take<float2>(static_cast<size_t>(batch) * n);
  float2* es = cv.take<float2>(static_cast<size_t>(batch) * n);
  if (cv.overflow) {
    set_error("cnn precond: workspace too small");
    return HELM_EWORKSPACE;
  }
  int rc;
  if (sel == nullptr || nsel < 0) {
    // every RHS goes through the network; those flagged in zero_rows then use the plain
    // V-cycle (e = 0, z = V(r))
    if ((rc = cnn_forward_infer(cnn, p, r, e, batch, cv, st))) return rc;
    if (zero_rows) {
      const dim3 g(static_cast<unsigned>(std::min<long>(div_up(n / 2, 256), 512)), batch);
      HELM_LAUNCH("k_zero_rows", st, k_zero_rows<<<g, 256, 0, st>>>(e, zero_rows, n));
      HELM_CHECK_LAUNCH("k_zero_rows");
    }
  } else {
    // only the selected RHS: gather, forward on the compact batch, scatter; e = 0 for
    // the others, whose preconditioner is then the plain V-cycle (z = V(r))
    HELM_CUDA(cudaMemsetAsync(e, 0, static_cast<size_t>(batch) * n * sizeof(float2), st));
    if (nsel > 0) {
      const dim3 g(static_cast<unsigned>(std::min<long>(div_up(n / 2, 256), 512)), nsel);
      HELM_LAUNCH("k_gather_rows", st, k_gather_rows<<<g, 256, 0, st>>>(r, rs, sel, n, 0));
      if ((rc = cnn_forward_infer(cnn, p, rs, es, nsel, cv, st))) return rc;
      HELM_LAUNCH("k_gather_rows", st, k_gather_rows<<<g, 256, 0, st>>>(es, e, sel, n, 1));
      HELM_CHECK_LAUNCH("k_gather_rows");
    }
  }
  if ((rc = launch_apply(p, p->massA, e, r, rp, batch, 0, active, st))) return rc;   // r' = r - A e
  return launch_vcycle(p, rp, z, batch, vs, active, st, e);                // z = e + V(r')
}

}  // namespace helm

// ------------------------------------------------------------------------------------
extern "C" {

int helm_cnn_create(const helm_cnn_desc* desc, helm_cnn** out) {
  using namespace helm;
  if (!out) {
    set_error("helm_cnn_create: null output");
    return HELM_EINVAL;
  }
  helm_cnn_desc d = {16, 6, 512, 0, 0};
  if (desc) d = *desc;
  if (d.c0 != 16 || d.expansion != 6) {
    set_error("helm_cnn_create: kernels are instantiated for c0 = 16, expansion = 6");
    return HELM_EINVAL;
  }
  if (d.explicit_unet != 0 && d.explicit_unet != 1) {
    set_error("helm_cnn_create: explicit_unet must be 0 or 1");
    return HELM_EINVAL;
  }
  helm_cnn* c = new helm_cnn();
  c->desc = d;
  build_params(c);
  size_t wp = 0;
  for (const ParamInfo& pi : c->params) wp += packed_elems(c, pi);
  c->wpk_elems = wp;
  size_t wf = 0;
  for (size_t i = 0; i < c->params.size(); ++i) {
    const ParamInfo& pi = c->params[i];
    if (pi.name.find(".ib.exp.w") == std::string::npos && pi.name.find(".ib.proj.w") == std::string::npos) continue;
    c->wfold_off[static_cast<int>(i)] = wf;
    wf += ib_folded_elems(pi.shape[1], pi.shape[0]);
  }
  c->wfold_elems = wf;
  if (cudaMalloc(&c->wpk, wp * sizeof(__nv_bfloat16)) != cudaSuccess ||
      cudaMalloc(&c->wfold, wf * sizeof(__nv_bfloat16)) != cudaSuccess ||
      cudaMalloc(&c->running, c->nrunning * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&c->fold, c->nrunning * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&c->gscratch, 4096 * sizeof(float2)) != cudaSuccess) {
    helm_cnn_destroy(c);
    set_error("helm_cnn_create: out of device memory");
    return HELM_ENOMEM;
  }
  c->gscratch_elems = 4096;
  // running statistics start at mean 0, var 1
  std::vector<float> run(c->nrunning);
  for (const BnInfo& b : c->bns) {
    for (int i = 0; i < b.C; ++i) {
      run[b.roff + i] = 0.f;
      run[b.roff + b.C + i] = 1.f;
    }
  }
  cudaMemcpy(c->running, run.data(), run.size() * sizeof(float), cudaMemcpyHostToDevice);
  *out = c;
  return HELM_OK;
}

int helm_cnn_destroy(helm_cnn* c) {
  if (!c) return HELM_OK;
  cudaFree(c->wpk);
  cudaFree(c->wfold);
  cudaFree(c->running);
  cudaFree(c->fold);
  cudaFree(c->gscratch);
  cudaFree(c->enc_arena);
  for (auto& kv : c->ghat) cudaFree(kv.second);
  for (auto& kv : c->ghat_rect) cudaFree(kv.second);
  delete c;
  return HELM_OK;
}

int helm_cnn_num_params(const helm_cnn* c, size_t* n) {
  if (!c || !n) {
    helm::set_error("helm_cnn_num_params: invalid argument");
    return HELM_EINVAL;
  }
  *n = c->nparams;
  return HELM_OK;
}

int helm_cnn_param_info(const helm_cnn* c, int idx, const char** name, int* ndim, int* shape, size_t* offset) {
  if (!c || idx < 0 || idx >= static_cast<int>(c->params.size())) {
    helm::set_error("helm_cnn_param_info: index out of range");
    return HELM_EINVAL;
  }
  const helm::ParamInfo& p = c->params[idx];
  if (name) *name = p.name.c_str();
  if (ndim) *ndim = static_cast<int>(p.shape.size());
  if (shape)
    for (size_t i = 0; i < p.shape.size(); ++i) shape[i] = p.shape[i];
  if (offset) *offset = p.offset;
  return HELM_OK;
}

int helm_cnn_num_bn(const helm_cnn* c, int* n) {
  if (!c || !n) {
    helm::set_error("helm_cnn_num_bn: invalid argument");
    return HELM_EINVAL;
  }
  *n = static_cast<int>(c->bns.size());
  return HELM_OK;
}

int helm_cnn_bn_info(const helm_cnn* c, int idx, const char** name, int* C, size_t* roff) {
  if (!c || idx < 0 || idx >= static_cast<int>(c->bns.size())) {
    helm::set_error("helm_cnn_bn_info: index out of range");
    return HELM_EINVAL;
  }
  if (name) *name = c->bns[idx].name.c_str();
  if (C) *C = c->bns[idx].C;
  if (roff) *roff = c->bns[idx].roff;
  return HELM_OK;
}

int helm_cnn_set_params(helm_cnn* c, const float* params_dev, void* stream) {
  (void)stream;
  if (!c || !params_dev) {
    helm::set_error("helm_cnn_set_params: invalid argument");
    return HELM_EINVAL;
  }
  c->params_dev = params_dev;
  c->dirty = true;
  c->param_version++;
  return HELM_OK;
}

int helm_cnn_set_running(helm_cnn* c, const float* running_dev, void* stream) {
  if (!c || !running_dev) {
    helm::set_error("helm_cnn_set_running: invalid argument");
    return HELM_EINVAL;
  }
  HELM_CUDA(cudaMemcpyAsync(c->running, running_dev, c->nrunning * sizeof(float), cudaMemcpyDeviceToDevice,
                            static_cast<cudaStream_t>(stream)));
  c->dirty = true;
  c->param_version++;
  return HELM_OK;
}

int helm_cnn_get_running(helm_cnn* c, float* out_dev, void* stream) {
  if (!c || !out_dev) {
    helm::set_error("helm_cnn_get_running: invalid argument");
    return HELM_EINVAL;
  }
  HELM_CUDA(cudaMemcpyAsync(out_dev, c->running, c->nrunning * sizeof(float), cudaMemcpyDeviceToDevice,
                            static_cast<cudaStream_t>(stream)));
  return HELM_OK;
}

int helm_cnn_set_problem(helm_cnn* c, const helm_problem* p, void* ws, size_t ws_bytes, void* stream) {
  (void)ws;
  (void)ws_bytes;
  if (!c || !p) {
    helm::set_error("helm_cnn_set_problem: invalid argument");
    return HELM_EINVAL;
  }
  return helm::run_encoder(c, p, static_cast<cudaStream_t>(stream));
}

int helm_cnn_apply(const helm_problem* p, helm_cnn* c, const void* r, void* e, int batch, int train, void* ws,
                   size_t ws_bytes, void* stream) {
  if (!p || !c || !r || !e || batch <= 0) {
    helm::set_error("helm_cnn_apply: invalid argument");
    return HELM_EINVAL;
  }
  helm::Carve cv(ws, ws_bytes);
  if (train) return helm::cnn_forward_train(c, &p, 1, static_cast<const float2*>(r), static_cast<float2*>(e), batch, cv,
                                            static_cast<cudaStream_t>(stream));
  return helm::cnn_forward_infer(c, p, static_cast<const float2*>(r), static_cast<float2*>(e), batch, cv,
                                 static_cast<cudaStream_t>(stream));
}

int helm_cnn_get_ghat(helm_cnn* c, int m, void* out_dev, void* stream) {
  if (!c || m <= 0 || !out_dev) {
    helm::set_error("helm_cnn_get_ghat: invalid argument");
    return HELM_EINVAL;
  }
  if (c->desc.explicit_unet) {
    helm::set_error("helm_cnn_get_ghat: the explicit U-Net has no implicit layer");
    return HELM_ESTATE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = helm::cnn_derive(c, m, st);
  if (rc) return rc;
  const int nk = c->params[c->pidx.at("s.imp.K")].shape[1];
  HELM_CUDA(cudaMemcpyAsync(out_dev, c->ghat.at(m), static_cast<size_t>(nk) * 4 * m * m * sizeof(float2),
                            cudaMemcpyDeviceToDevice, st));
  return HELM_OK;
}

int helm_cnn_get_ghat_rect(helm_cnn* c, int my, int mx, void* out_dev, void* stream) {
  if (!c || my <= 0 || mx <= 0 || !out_dev) {
    helm::set_error("helm_cnn_get_ghat_rect: invalid argument");
    return HELM_EINVAL;
  }
  if (c->desc.explicit_unet) {
    helm::set_error("helm_cnn_get_ghat_rect: the explicit U-Net has no implicit layer");
    return HELM_ESTATE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = helm::cnn_derive(c, my, mx, st);
  if (rc) return rc;
  const int nk = c->params[c->pidx.at("s.imp.K")].shape[1];
  HELM_CUDA(cudaMemcpyAsync(out_dev, helm::ghat_of(c, my, mx), static_cast<size_t>(nk) * 4 * my * mx * sizeof(float2),
                            cudaMemcpyDeviceToDevice, st));
  return HELM_OK;
}

int helm_cnn_precond_apply(const helm_problem* p, helm_cnn* c, const void* r, void* z, int batch, void* ws,
                           size_t ws_bytes, void* stream) {
  if (!p || !c || !r || !z || batch <= 0 || r == z) {
    helm::set_error("helm_cnn_precond_apply: invalid argument");
    return HELM_EINVAL;
  }
  helm::Carve cv(ws, ws_bytes);
  helm::VcycleScratch vs;
  helm::carve_vcycle(cv, p, batch, &vs);
  if (cv.overflow || !ws) {
    helm::set_error("helm_cnn_precond_apply: workspace too small");
    return HELM_EWORKSPACE;
  }
  return helm::launch_cnn_precond(p, c, static_cast<const float2*>(r), static_cast<float2*>(z), batch, cv, vs,
                                  nullptr, static_cast<cudaStream_t>(stream), nullptr, -1, nullptr);
}

}  // extern "C"
