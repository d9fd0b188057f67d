// Learned warm start and spectral resampling.
//
// Not part of the paper's method. A small 3D encoder-decoder maps (m_T, m_R), spectrally truncated to a coarse
// network grid, to the low-frequency part of the velocity; the prediction, zero-padded in Fourier space to the
// registration grid (and Leray-projected when div v = 0 is imposed), seeds v_0 of the unchanged Gauss-Newton-Krylov
// solve (Alg. 1). The relative stopping test keeps g_0 = g(v = 0) (Sec. 2.3.2), so a warm start changes only how
// many iterations are needed, never what "converged" means.
//
// Network (channels after the slash): four levels, two periodic 3x3x3 convolutions + ReLU per level,
// 2x2x2 average pooling down, nearest-neighbour upsampling up, additive skip connections:
//   e0 16/16 16/16 | pool | e1 16/32 32/32 | pool | e2 32/64 64/64 | pool | b 64/128 128/128 | up |
//   d2 128/64 (+e2) 64/64 | up | d1 64/32 (+e1) 32/32 | up | d0 32/16 (+e0) 16/16 | head 16/16 (no ReLU)
// The inputs are m_T and kDiffScale (m_R - m_T) (the same information as (m_T, m_R), but the small difference is
// formed in FP32 before the BF16 rounding instead of after it), zero-padded to 16 channels; the 3 output
// channels are the first 3 of the head's 16.
// BF16 weights and activations, FP32 accumulation, FP32 master weights, gradients and Adam moments.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "impl.cuh"
#include "nn.cuh"

using namespace claire;
typedef nn::bf16 bf16;

namespace {

constexpr float kDiffScale = 8.f;

struct Layer {
  int cin_true, cin, cout, level, relu;
  int in, out, skip;  // tensor ids; out = -1: the FP32 prediction
  long long woff, boff;
};
struct Op {
  int kind;  // 0 conv, 1 pool, 2 up
  int layer, in, out;
};
struct Tensor {
  int level, C;
  bf16* y = nullptr;
  float* g = nullptr;
};

__global__ void k_resample_modes(const cplx<float>* __restrict__ S, Dims ds, cplx<float>* __restrict__ D, Dims dd,
                                 int kmax) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < dd.Ns;
       i += (long long)gridDim.x * blockDim.x) {
    const int k3 = (int)(i % dd.n3h);
    const long long t = i / dd.n3h;
    const int k2 = (int)(t % dd.n2);
    const int k1 = (int)(t / dd.n2);
    const int w1 = 2 * k1 <= dd.n1 ? k1 : k1 - dd.n1;
    const int w2 = 2 * k2 <= dd.n2 ? k2 : k2 - dd.n2;
    const int a1 = w1 < 0 ? -w1 : w1, a2 = w2 < 0 ? -w2 : w2;
    const bool keep = 2 * a1 < ds.n1 && 2 * a1 < dd.n1 && 2 * a2 < ds.n2 && 2 * a2 < dd.n2 && 2 * k3 < ds.n3 &&
                      2 * k3 < dd.n3 && (kmax <= 0 || (a1 <= kmax && a2 <= kmax && k3 <= kmax));
    cplx<float> v{0.f, 0.f};
    if (keep) {
      const int s1 = w1 >= 0 ? w1 : w1 + ds.n1, s2 = w2 >= 0 ? w2 : w2 + ds.n2;
      v = S[((long long)s1 * ds.n2 + s2) * ds.n3h + k3];
    }
    D[i] = v;
  }
}

claire_status resample(claire_ctx* src, claire_ctx* dst, const float* f, float* g, int ncomp, bool project,
                       int kmax, cudaStream_t st) {
  cplx<float>* S = src->work<float>().spec;
  cplx<float>* D = dst->work<float>().spec + 3 * dst->d.Ns;
  for (int c = 0; c < ncomp; ++c) {
    CL_TRY(fft_r2c<float>(src, f + (long long)c * src->d.N, S, st));
    const long long nb = (dst->d.Ns + 255) / 256;
    dst->prof_begin("resample_modes", st);
    k_resample_modes<<<(unsigned)(nb < 4864 ? nb : 4864), 256, 0, st>>>(S, src->d, D + c * dst->d.Ns, dst->d, kmax);
    CL_LAUNCHED(dst);
  }
  if (project) CL_TRY(spec_leray<float>(dst, D, D + dst->d.Ns, D + 2 * dst->d.Ns, st));
  const float scale = float(1.0 / double(src->d.N));
  for (int c = 0; c < ncomp; ++c) CL_TRY(fft_c2r<float>(dst, D + c * dst->d.Ns, g + (long long)c * dst->d.N, scale, st));
  return CLAIRE_OK;
}

// counter-based normal deviates (splitmix64 + Box-Muller) for a platform-independent initialisation
inline uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ULL;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
  return x ^ (x >> 31);
}
inline double normal_at(uint64_t seed, uint64_t i) {
  const double u1 = (double((splitmix64(seed ^ (2 * i)) >> 11)) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = (double((splitmix64(seed ^ (2 * i + 1)) >> 11)) + 0.5) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

}  // namespace

struct claire_ws {
  int B = 0;
  int n[3] = {0, 0, 0};
  float vscale = 1.f;
  std::vector<Layer> layers;
  std::vector<Op> ops;
  std::vector<Tensor> T;
  long long nparam = 0, nparam_host = 0;
  float *P = nullptr, *G = nullptr, *M1 = nullptr, *M2 = nullptr;
  bf16 *Pb = nullptr, *Wt = nullptr;
  float *pred = nullptr, *dpred = nullptr, *tgt = nullptr, *dz = nullptr, *work = nullptr;
  float* bwork = nullptr;  // per-block bias-gradient partials of the layer being differentiated
  bf16* dzb = nullptr;
  double* part = nullptr;
  double* hpart = nullptr;
  float *img = nullptr, *vnet = nullptr;
  claire_ctx* net = nullptr;
  int t = 0;
  std::string err;
  std::vector<void*> allocs;

  static constexpr int kParts = 256;

  long long N(int level) const {
    return (long long)(n[0] >> level) * (n[1] >> level) * (n[2] >> level);
  }
  nn::Geo geo(int level, int nb) const { return nn::mkgeo(nb, n[0] >> level, n[1] >> level, n[2] >> level); }
  template <class P> bool alloc(P*& p, size_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(P)) != cudaSuccess) return false;
    allocs.push_back(q);
    p = static_cast<P*>(q);
    return true;
  }
  claire_status fail(const std::string& s, claire_status code) {
    err = s;
    return code;
  }
  claire_status cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return CLAIRE_OK;
    err = std::string(what) + ": " + cudaGetErrorString(e);
    // nn::status reports an expired bounded tensor-core wait as cudaErrorLaunchTimeout
    return e == cudaErrorLaunchTimeout ? CLAIRE_ETIMEOUT : CLAIRE_ECUDA;
  }
};

#define WS_CUDA(ws, call)                                   \
  do {                                                      \
    claire_status s_ = (ws)->cuda((call), #call);           \
    if (s_ != CLAIRE_OK) return s_;                         \
  } while (0)

namespace {

void build_graph(claire_ws* w) {
  const int ch[4] = {16, 32, 64, 128};
  auto tensor = [&](int level, int C) {
    Tensor t;
    t.level = level;
    t.C = C;
    w->T.push_back(t);
    return (int)w->T.size() - 1;
  };
  auto conv = [&](int cin_true, int cin, int cout, int level, int relu, int in, int out, int skip) {
    Layer l{cin_true, cin, cout, level, relu, in, out, skip, 0, 0};
    w->layers.push_back(l);
    w->ops.push_back(Op{0, (int)w->layers.size() - 1, in, out});
  };
  int x = tensor(0, 16);
  int skips[3];
  int cur = x, cin = 16, cin_true = 2;
  for (int l = 0; l < 3; ++l) {
    const int a = tensor(l, ch[l]);
    conv(cin_true, cin, ch[l], l, 1, cur, a, -1);
    const int s = tensor(l, ch[l]);
    conv(ch[l], ch[l], ch[l], l, 1, a, s, -1);
    skips[l] = s;
    const int p = tensor(l + 1, ch[l]);
    w->ops.push_back(Op{1, -1, s, p});
    cur = p;
    cin = cin_true = ch[l];
  }
  const int a3 = tensor(3, 128);
  conv(64, 64, 128, 3, 1, cur, a3, -1);
  const int h3 = tensor(3, 128);
  conv(128, 128, 128, 3, 1, a3, h3, -1);
  cur = h3;
  int ccur = 128;
  for (int l = 2; l >= 0; --l) {
    const int u = tensor(l, ccur);
    w->ops.push_back(Op{2, -1, cur, u});
    const int c = tensor(l, ch[l]);
    conv(ccur, ccur, ch[l], l, 1, u, c, skips[l]);
    const int h = tensor(l, ch[l]);
    conv(ch[l], ch[l], ch[l], l, 1, c, h, -1);
    cur = h;
    ccur = ch[l];
  }
  conv(16, 16, 16, 0, 0, cur, -1, -1);
  long long off = 0, host = 0;
  for (Layer& l : w->layers) {
    l.woff = off;
    off += (27LL * l.cin * l.cout + 63) / 64 * 64;
    l.boff = off;
    off += (l.cout + 63) / 64 * 64;
    host += 27LL * l.cin * l.cout + l.cout;
  }
  w->nparam = off;
  w->nparam_host = host;
}

claire_status ws_destroy(claire_ws* w) {
  if (!w) return CLAIRE_OK;
  for (void* p : w->allocs) cudaFree(p);
  if (w->hpart) cudaFreeHost(w->hpart);
  if (w->net) claire_destroy(w->net);
  delete w;
  return CLAIRE_OK;
}

// forward pass for samples img[b] = images + idx[b] * 2 N0 (idx == nullptr: b); prediction left in w->pred
claire_status forward(claire_ws* w, const float* images, const int* idx, int nb, cudaStream_t st) {
  const long long N0 = w->N(0);
  for (int b0 = 0; b0 < nb; b0 += nn::SampleIdx::kMax) {
    const int nc = std::min(nb - b0, nn::SampleIdx::kMax);
    nn::SampleIdx si;
    for (int b = 0; b < nc; ++b) si.v[b] = idx ? idx[b0 + b] : b0 + b;
    WS_CUDA(w, nn::pack_images(images, si, nc, w->T[0].y + b0 * N0 * 16, N0, 16, kDiffScale, st));
  }
  for (const Op& op : w->ops) {
    if (op.kind == 0) {
      const Layer& l = w->layers[op.layer];
      WS_CUDA(w, nn::conv3_fwd(w->T[l.in].y, w->Pb + l.woff, w->P + l.boff, l.skip >= 0 ? w->T[l.skip].y : nullptr,
                               l.out >= 0 ? w->T[l.out].y : nullptr, l.out >= 0 ? nullptr : w->pred, 0,
                               w->geo(l.level, nb), l.cin, l.cout, l.relu, w->work, st));
    } else if (op.kind == 1) {
      const Tensor& ti = w->T[op.in];
      WS_CUDA(w, nn::pool_fwd(ti.y, w->T[op.out].y, w->geo(ti.level, nb), ti.C, st));
    } else {
      const Tensor& ti = w->T[op.in];
      WS_CUDA(w, nn::up_fwd(ti.y, w->T[op.out].y, w->geo(ti.level, nb), ti.C, st));
    }
  }
  return CLAIRE_OK;
}

claire_status read_loss(claire_ws* w, double* loss, cudaStream_t st) {
  WS_CUDA(w, cudaMemcpyAsync(w->hpart, w->part, sizeof(double) * claire_ws::kParts, cudaMemcpyDeviceToHost, st));
  WS_CUDA(w, nn::status(st));
  double s = 0.0;
  for (int i = 0; i < claire_ws::kParts; ++i) s += w->hpart[i];
  *loss = s;
  return CLAIRE_OK;
}

// loss (MSE of the scaled velocity over the 3 output channels) and, with backward, all parameter gradients
claire_status loss_grad(claire_ws* w, const float* images, const float* targets, const int* idx, int nb,
                        bool backward, double* loss, cudaStream_t st) {
  CL_TRY(forward(w, images, idx, nb, st));
  const long long N0 = w->N(0);
  for (int b0 = 0; b0 < nb; b0 += nn::SampleIdx::kMax) {
    const int nc = std::min(nb - b0, nn::SampleIdx::kMax);
    nn::SampleIdx si;
    for (int b = 0; b < nc; ++b) si.v[b] = idx ? idx[b0 + b] : b0 + b;
    WS_CUDA(w, nn::interleave_batch(targets, si, nc, w->tgt + b0 * N0 * 3, N0, 3, w->vscale, st));
  }
  const long long M0 = N0 * nb;
  WS_CUDA(w, nn::mse(w->pred, w->tgt, backward ? w->dpred : nullptr, M0, 16, 3, w->part, claire_ws::kParts, st));
  if (backward) {
    // the adjoint-convolution weights of every layer that passes a gradient to its input, in one launch
    nn::FlipTable ft;
    ft.n = 0;
    for (const Layer& l : w->layers) {
      if (l.in == 0) continue;
      ft.cin[ft.n] = l.cin;
      ft.cout[ft.n] = l.cout;
      ft.woff[ft.n] = l.woff;
      ++ft.n;
    }
    WS_CUDA(w, nn::weight_flip_all(w->Pb, w->Wt, ft, st));
    std::vector<char> written(w->T.size(), 0);
    for (int k = (int)w->ops.size() - 1; k >= 0; --k) {
      const Op& op = w->ops[k];
      if (op.kind == 0) {
        const Layer& l = w->layers[op.layer];
        const nn::Geo g = w->geo(l.level, nb);
        const float* dy = l.out >= 0 ? w->T[l.out].g : w->dpred;
        const bf16* y = (l.out >= 0 && l.relu) ? w->T[l.out].y : nullptr;
        // the bias gradient's partials, summed in the weight gradient's reduction launch
        WS_CUDA(w, nn::relu_bwd_bias(dy, y, l.skip >= 0 ? w->dz : nullptr, w->dzb, g.M, l.cout, nullptr, w->bwork,
                                     st));
        WS_CUDA(w, nn::conv3_wgrad(w->dzb, w->T[l.in].y, w->G + l.woff, w->work, g, l.cin, l.cout, st, w->bwork,
                                   w->G + l.boff));
        if (l.in != 0) {
          WS_CUDA(w, nn::conv3_fwd(w->dzb, w->Wt + l.woff, nullptr, nullptr, nullptr, w->T[l.in].g,
                                   written[l.in], g, l.cout, l.cin, 0, w->work, st));
          written[l.in] = 1;
        }
        if (l.skip >= 0) {
          if (written[l.skip]) {
            WS_CUDA(w, nn::add(w->dz, w->T[l.skip].g, g.M * l.cout, st));
          } else {
            WS_CUDA(w, cudaMemcpyAsync(w->T[l.skip].g, w->dz, sizeof(float) * g.M * l.cout,
                                       cudaMemcpyDeviceToDevice, st));
          }
          written[l.skip] = 1;
        }
      } else {
        const Tensor& ti = w->T[op.in];
        if (op.kind == 1) {
          WS_CUDA(w, nn::pool_bwd(w->T[op.out].g, ti.g, written[op.in], w->geo(ti.level, nb), ti.C, st));
        } else {
          WS_CUDA(w, nn::up_bwd(w->T[op.out].g, ti.g, written[op.in], w->geo(ti.level, nb), ti.C, st));
        }
        written[op.in] = 1;
      }
    }
  }
  if (loss) CL_TRY(read_loss(w, loss, st));
  return CLAIRE_OK;
}

bool batch_ok(const claire_ws* w, int nb) { return nb >= 1 && nb <= w->B; }

}  // namespace

extern "C" {

claire_status claire_ws_create(int batch, int n1, int n2, int n3, float vscale, unsigned long long seed,
                               claire_ws** out) {
  if (!out) return CLAIRE_EINVAL;
  *out = nullptr;
  if (batch < 1 || n1 < 8 || n2 < 8 || n3 < 8 || n1 % 8 || n2 % 8 || n3 % 8 || !(vscale > 0.f)) return CLAIRE_EINVAL;
  if (((long long)(n1 / 8) * (n2 / 8) * (n3 / 8)) % 16 != 0) return CLAIRE_EINVAL;
  if ((long long)batch * n1 * n2 * n3 >= (1LL << 31) / 16) return CLAIRE_EINVAL;
  claire_ws* w = new claire_ws();
  w->B = batch;
  w->n[0] = n1;
  w->n[1] = n2;
  w->n[2] = n3;
  w->vscale = vscale;
  build_graph(w);
  claire_opts o;
  claire_default_opts(&o, n1, n2, n3, CLAIRE_F32);
  if (claire_create(&o, &w->net) != CLAIRE_OK) {
    ws_destroy(w);
    return CLAIRE_ENOMEM;
  }
  bool ok = w->alloc(w->P, w->nparam) && w->alloc(w->G, w->nparam) && w->alloc(w->M1, w->nparam) &&
            w->alloc(w->M2, w->nparam) && w->alloc(w->Pb, w->nparam) && w->alloc(w->Wt, w->nparam);
  size_t work = 0, dmax = 0;
  for (const Layer& l : w->layers) {
    const nn::Geo g = w->geo(l.level, batch);
    work = std::max(work, nn::wgrad_work_elems(g, l.cin, l.cout));
    work = std::max(work, nn::fwd_work_elems(g, l.cout));  // forward split-K partials
    work = std::max(work, nn::fwd_work_elems(g, l.cin));   // input-gradient (adjoint convolution) partials
    dmax = std::max(dmax, size_t(g.M) * l.cout);
  }
  for (Tensor& t : w->T) {
    const size_t cnt = size_t(w->N(t.level)) * batch * t.C;
    ok = ok && w->alloc(t.y, cnt) && w->alloc(t.g, cnt);
  }
  const size_t M0 = size_t(w->N(0)) * batch;
  ok = ok && w->alloc(w->pred, M0 * 16) && w->alloc(w->dpred, M0 * 16) && w->alloc(w->tgt, M0 * 3) &&
       w->alloc(w->dz, dmax) && w->alloc(w->dzb, dmax) && w->alloc(w->work, work) &&
       w->alloc(w->bwork, nn::bias_work_elems(128)) && w->alloc(w->part, claire_ws::kParts) &&
       w->alloc(w->img, 2 * size_t(w->N(0))) && w->alloc(w->vnet, 3 * size_t(w->N(0)));
  ok = ok && cudaMallocHost(&w->hpart, sizeof(double) * claire_ws::kParts) == cudaSuccess;
  if (!ok) {
    ws_destroy(w);
    return CLAIRE_ENOMEM;
  }
  // He-normal initialisation (std sqrt(2 / fan_in)), the head scaled by 0.1 so the first prediction is near 0
  std::vector<float> h(w->nparam, 0.f);
  uint64_t counter = 0;
  for (const Layer& l : w->layers) {
    const double sd = std::sqrt(2.0 / (27.0 * l.cin_true)) * (l.out < 0 ? 0.1 : 1.0);
    for (int co = 0; co < l.cout; ++co)
      for (int off = 0; off < 27; ++off)
        for (int ci = 0; ci < l.cin; ++ci) {
          const double z = normal_at(seed, counter++);
          h[l.woff + ((long long)co * 27 + off) * l.cin + ci] = ci < l.cin_true ? float(sd * z) : 0.f;
        }
  }
  if (cudaMemcpy(w->P, h.data(), sizeof(float) * w->nparam, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(w->G, 0, sizeof(float) * w->nparam) != cudaSuccess ||
      cudaMemset(w->M1, 0, sizeof(float) * w->nparam) != cudaSuccess ||
      cudaMemset(w->M2, 0, sizeof(float) * w->nparam) != cudaSuccess ||
      nn::to_bf16(w->P, w->Pb, w->nparam, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    ws_destroy(w);
    return CLAIRE_ECUDA;
  }
  *out = w;
  return CLAIRE_OK;
}

claire_status claire_ws_destroy(claire_ws* w) { return ws_destroy(w); }

const char* claire_ws_last_error(const claire_ws* w) { return w ? w->err.c_str() : "null network"; }

long long claire_ws_num_params(const claire_ws* w) { return w ? w->nparam_host : 0; }

int claire_ws_num_layers(const claire_ws* w) { return w ? (int)w->layers.size() : 0; }

claire_status claire_ws_layer(const claire_ws* w, int i, int* info) {
  if (!w || !info || i < 0 || i >= (int)w->layers.size()) return CLAIRE_EINVAL;
  const Layer& l = w->layers[i];
  const int v[8] = {l.cin_true, l.cin, l.cout, l.level, l.relu, l.in, l.out, l.skip};
  std::memcpy(info, v, sizeof(v));
  return CLAIRE_OK;
}

int claire_ws_num_ops(const claire_ws* w) { return w ? (int)w->ops.size() : 0; }

claire_status claire_ws_op(const claire_ws* w, int i, int* info) {
  if (!w || !info || i < 0 || i >= (int)w->ops.size()) return CLAIRE_EINVAL;
  const Op& o = w->ops[i];
  const int v[4] = {o.kind, o.layer, o.in, o.out};
  std::memcpy(info, v, sizeof(v));
  return CLAIRE_OK;
}

static claire_status copy_params(claire_ws* w, float* host, const float* dev_base, bool to_host) {
  long long h = 0;
  for (const Layer& l : w->layers) {
    const long long nw = 27LL * l.cin * l.cout;
    float* dw = const_cast<float*>(dev_base) + l.woff;
    float* db = const_cast<float*>(dev_base) + l.boff;
    if (to_host) {
      WS_CUDA(w, cudaMemcpy(host + h, dw, sizeof(float) * nw, cudaMemcpyDeviceToHost));
      WS_CUDA(w, cudaMemcpy(host + h + nw, db, sizeof(float) * l.cout, cudaMemcpyDeviceToHost));
    } else {
      WS_CUDA(w, cudaMemcpy(dw, host + h, sizeof(float) * nw, cudaMemcpyHostToDevice));
      WS_CUDA(w, cudaMemcpy(db, host + h + nw, sizeof(float) * l.cout, cudaMemcpyHostToDevice));
    }
    h += nw + l.cout;
  }
  return CLAIRE_OK;
}

claire_status claire_ws_get_params(claire_ws* w, float* host) {
  if (!w || !host) return CLAIRE_EINVAL;
  WS_CUDA(w, cudaDeviceSynchronize());
  return copy_params(w, host, w->P, true);
}

claire_status claire_ws_get_grads(claire_ws* w, float* host) {
  if (!w || !host) return CLAIRE_EINVAL;
  WS_CUDA(w, cudaDeviceSynchronize());
  return copy_params(w, host, w->G, true);
}

claire_status claire_ws_set_params(claire_ws* w, const float* host) {
  if (!w || !host) return CLAIRE_EINVAL;
  WS_CUDA(w, cudaDeviceSynchronize());
  CL_TRY(copy_params(w, const_cast<float*>(host), w->P, false));
  WS_CUDA(w, cudaMemset(w->M1, 0, sizeof(float) * w->nparam));
  WS_CUDA(w, cudaMemset(w->M2, 0, sizeof(float) * w->nparam));
  WS_CUDA(w, nn::to_bf16(w->P, w->Pb, w->nparam, 0));
  WS_CUDA(w, cudaDeviceSynchronize());
  w->t = 0;
  return CLAIRE_OK;
}

claire_status claire_ws_forward_f32(claire_ws* w, const float* images, const int* idx, int nb, float* v,
                                    void* stream) {
  if (!w || !images || !v) return CLAIRE_EINVAL;
  if (!batch_ok(w, nb)) return w->fail("batch larger than the network was created for", CLAIRE_EINVAL);
  cudaStream_t st = (cudaStream_t)stream;
  CL_TRY(forward(w, images, idx, nb, st));
  const long long N0 = w->N(0);
  for (int b = 0; b < nb; ++b)
    WS_CUDA(w, nn::unpack(w->pred + b * N0 * 16, v + b * 3 * N0, N0, 3, 16, 1.f / w->vscale, st));
  return CLAIRE_OK;
}

claire_status claire_ws_loss_f32(claire_ws* w, const float* images, const float* targets, const int* idx, int nb,
                                 int backward, double* loss, void* stream) {
  if (!w || !images || !targets) return CLAIRE_EINVAL;
  if (!batch_ok(w, nb)) return w->fail("batch larger than the network was created for", CLAIRE_EINVAL);
  return loss_grad(w, images, targets, idx, nb, backward != 0, loss, (cudaStream_t)stream);
}

claire_status claire_ws_adam_step(claire_ws* w, float lr, void* stream) {
  if (!w || !(lr >= 0.f)) return CLAIRE_EINVAL;
  w->t += 1;
  WS_CUDA(w, nn::adam(w->P, w->G, w->M1, w->M2, w->Pb, w->nparam, lr, 0.9f, 0.999f, 1e-8f, w->t,
                      (cudaStream_t)stream));
  return CLAIRE_OK;
}

claire_status claire_ws_train_step_f32(claire_ws* w, const float* images, const float* targets, const int* idx,
                                       int nb, float lr, double* loss, void* stream) {
  CL_TRY(claire_ws_loss_f32(w, images, targets, idx, nb, 1, nullptr, stream));
  CL_TRY(claire_ws_adam_step(w, lr, stream));
  if (loss) CL_TRY(read_loss(w, loss, (cudaStream_t)stream));
  return CLAIRE_OK;
}

claire_status claire_ws_predict_f32(claire_ws* w, claire_ctx* ctx, const float* mT, const float* mR, float* v,
                                    int kmax, void* stream) {
  if (!w || !ctx || !mT || !mR || !v) return CLAIRE_EINVAL;
  if (ctx->o.precision != CLAIRE_F32) {
    ctx->set_error("the warm start needs an FP32 context");
    return CLAIRE_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const long long N0 = w->N(0);
  CL_TRY(resample(ctx, w->net, mT, w->img, 1, false, 0, st));
  CL_TRY(resample(ctx, w->net, mR, w->img + N0, 1, false, 0, st));
  CL_TRY(forward(w, w->img, nullptr, 1, st));
  WS_CUDA(w, nn::unpack(w->pred, w->vnet, N0, 3, 16, 1.f / w->vscale, st));
  WS_CUDA(w, nn::status(st));
  return resample(w->net, ctx, w->vnet, v, 3, ctx->o.divfree != 0, kmax, st);
}

claire_status claire_resample_f32(claire_ctx* src, claire_ctx* dst, const float* f, float* g, int ncomp,
                                  int project, int kmax, void* stream) {
  if (!src || !dst || !f || !g || ncomp < 1 || ncomp > 3 || (project && ncomp != 3)) return CLAIRE_EINVAL;
  if (src->o.precision != CLAIRE_F32 || dst->o.precision != CLAIRE_F32) {
    dst->set_error("claire_resample_f32 needs FP32 contexts");
    return CLAIRE_EINVAL;
  }
  return resample(src, dst, f, g, ncomp, project != 0, kmax, (cudaStream_t)stream);
}

}  // extern "C"
