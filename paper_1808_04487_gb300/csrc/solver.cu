// Operators and the inexact Gauss-Newton-Krylov solver on top of the kernels, and the C-ABI entry points.
//
// Memory-reduced Gauss-Newton (Sec. 3.5): the state history m^j and its spectral gradients are kept per
// linearisation (departure points are computed once per v, Sec. 3.4); the adjoint and incremental adjoint are
// never stored in time, their time integrals are accumulated during the backward sweeps. The host drives the
// outer loop (Alg. 1); every scalar it needs (objective, norms, Armijo test) is reduced in FP64 on the device and
// read back once per use. The inner loop (Alg. 2) runs either on the host the same way or, with the spectral
// preconditioner and per-kernel profiling off, as one CUDA graph launch whose scalars stay on the device.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>
#include <utility>

#include "impl.cuh"

using namespace claire;

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

inline double cellvol(const Dims& d) { return kTwoPi * kTwoPi * kTwoPi / double(d.N); }

template <class T> claire_status alloc_work(claire_ctx* c) {
  Work<T>& W = c->work<T>();
  const long long N = c->d.N, Ns = c->d.Ns;
  const int nt = c->o.nt;
  auto takeT = [&](T*& p, long long count) -> bool {
    p = static_cast<T*>(c->take(sizeof(T) * size_t(count)));
    return p != nullptr;
  };
  auto takeC = [&](cplx<T>*& p, long long count) -> bool {
    p = static_cast<cplx<T>*>(c->take(sizeof(cplx<T>) * size_t(count)));
    return p != nullptr;
  };
  bool ok = true;
  ok &= takeT(W.dX, 3 * N);
  ok &= takeT(W.dY, 3 * N);
  ok &= takeT(W.m, (nt + 1) * N);
  if (c->gm16_on) {
    W.gm16 = c->take(2 * size_t(3 * (nt + 1) * N));
    ok &= W.gm16 != nullptr;
  } else {
    ok &= takeT(W.gm, 3 * (nt + 1) * N);
  }
  if (!c->o.divfree) ok &= takeT(W.rho, N);
  ok &= takeT(W.la, N);
  ok &= takeT(W.lb, N);
  if (!c->o.divfree) {
    ok &= takeT(W.ra, N);
    ok &= takeT(W.rb, N);
  }
  ok &= takeT(W.b, 3 * N);
  ok &= takeC(W.spec, 6 * Ns);
  ok &= takeT(W.s, 3 * N);
  if (c->is_coarse) {
    // the two-level preconditioner's coarse problem keeps its restricted m_T and v here; it runs no line search
    // (no trial velocity) and restricts v through W.Gh (no master copy V^)
    ok &= takeT(W.vdev, 3 * N);
    ok &= takeT(W.mTdev, N);
    for (cplx<T>** p : {&W.Gh, &W.Rh, &W.Sh, &W.VTh}) ok &= takeC(*p, 3 * Ns);
  } else {
    ok &= takeT(W.vtrial, 3 * N);
    for (cplx<T>** p : {&W.Vh, &W.Vtrh, &W.Gh, &W.Rh, &W.Sh, &W.VTh}) ok &= takeC(*p, 3 * Ns);
  }
  // the transform of the time integral and the inverse-transform work array share the six spectra of W.spec:
  // neither is live while a spectral operator works in W.spec
  W.Bh = W.spec;
  W.Sc = W.spec + 3 * Ns;
  const Launch3 L = launch3(c->d);
  W.nbig = (long long)L.grid.x * L.grid.y * L.grid.z;
  W.bigpart = static_cast<double*>(c->take(sizeof(double) * size_t(W.nbig)));
  W.partials = static_cast<double*>(c->take(sizeof(double) * 4 * kReduceBlocks));
  W.scal = static_cast<double*>(c->take(sizeof(double) * kScalSlots));
  ok &= W.partials != nullptr && W.scal != nullptr && W.bigpart != nullptr;
  if (!ok) {
    c->set_error("workspace arena too small");
    return CLAIRE_ENOMEM;
  }
  return CLAIRE_OK;
}

template <class T> size_t work_bytes(const claire_opts& o, const Dims& d, bool coarse) {
  const long long N = d.N, Ns = d.Ns;
  const int nt = o.nt;
  // dX, dY; m history; (rho, rho lambda ping/pong); lambda ping/pong; b; s; vtrial (coarse: v, m_T instead)
  const long long elems = 3 * N * 2 + (nt + 1) * N + (o.divfree ? 0 : 3 * N) + 2 * N + 3 * N + 3 * N +
                          (coarse ? 4 * N : 3 * N);
  // gradient history, FP32/FP64 or BF16
  const size_t gm_bytes = (o.bf16_mask & 1) ? 2 * size_t(3 * (nt + 1) * N) : sizeof(T) * size_t(3 * (nt + 1) * N);
  // spec; the Fourier-domain solver vectors (V^, V^trial, G^, R^, S^, V~^; the coarse problem needs four)
  const long long celems = 6 * Ns + (coarse ? 4 : 6) * 3 * Ns;
  const Launch3 L = launch3(d);
  const long long nbig = (long long)L.grid.x * L.grid.y * L.grid.z;
  // FP32 contexts also hold FP64 twiddle tables (stand-alone operators transform some inputs in FP64)
  const size_t tables = fft_table_bytes<T>(d) + (sizeof(T) == 4 ? fft_table_bytes<double>(d) : 0);
  return sizeof(T) * size_t(elems) + gm_bytes + sizeof(cplx<T>) * size_t(celems) +
         sizeof(double) * size_t(nbig + 4 * kReduceBlocks + kScalSlots) + tables + 64 * 256;
}

// Read scal[slot] to the host (synchronises the stream).
claire_status read_scalar(claire_ctx* c, double* dev, double* out, cudaStream_t st) {
  CL_CUDA(c, cudaMemcpyAsync(c->hscal, dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  CL_CUDA(c, cudaStreamSynchronize(st));
  *out = c->hscal[0];
  return CLAIRE_OK;
}

// <a, b> = h1 h2 h3 sum a b over n values (FP64)
template <class T> claire_status inner(claire_ctx* c, const T* a, const T* b, long long n, double* out, cudaStream_t st) {
  Work<T>& W = c->work<T>();
  CL_TRY(dot_partial<T>(c, a, b, n, W.partials, st));
  CL_TRY(reduce_final(c, W.partials, cellvol(c->d), W.scal, st));
  return read_scalar(c, W.scal, out, st);
}

template <class T> inline T* comp(T* v, const Dims& d, int k) { return v + (long long)k * d.N; }
template <class T> inline const T* comp(const T* v, const Dims& d, int k) { return v + (long long)k * d.N; }

// ---------------------------------------------------------------------------------------------------------------
// spectral building blocks
template <class T> claire_status grad_spectral(claire_ctx* c, const T* f, T* out, cudaStream_t st) {
  Work<T>& W = c->work<T>();
  const Dims& d = c->d;
  cplx<T>* S = W.spec;
  const T inv = T(1.0 / double(d.N));
  CL_TRY(fft_r2c<T>(c, f, S, st));
  CL_TRY(spec_grad<T>(c, S, S + d.Ns, S + 2 * d.Ns, S + 3 * d.Ns, st));
  for (int k = 0; k < 3; ++k) CL_TRY(fft_c2r<T>(c, S + (k + 1) * d.Ns, comp(out, d, k), inv, st));
  return CLAIRE_OK;
}

template <class T> claire_status vec_r2c(claire_ctx* c, const T* v, cplx<T>* S, cudaStream_t st) {
  for (int k = 0; k < 3; ++k) CL_TRY(fft_r2c<T>(c, comp(v, c->d, k), S + k * c->d.Ns, st));
  return CLAIRE_OK;
}
template <class T> claire_status vec_c2r(claire_ctx* c, cplx<T>* S, T* v, cudaStream_t st) {
  const T inv = T(1.0 / double(c->d.N));
  for (int k = 0; k < 3; ++k) CL_TRY(fft_c2r<T>(c, S + k * c->d.Ns, comp(v, c->d, k), inv, st));
  return CLAIRE_OK;
}

template <class T> claire_status div_spectral(claire_ctx* c, const T* v, T* out, cudaStream_t st) {
  Work<T>& W = c->work<T>();
  const Dims& d = c->d;
  cplx<T>* S = W.spec;
  CL_TRY(vec_r2c<T>(c, v, S, st));
  CL_TRY(spec_div<T>(c, S, S + d.Ns, S + 2 * d.Ns, S + 3 * d.Ns, st));
  return fft_c2r<T>(c, S + 3 * d.Ns, out, T(1.0 / double(d.N)), st);
}

template <class T> claire_status leray_inplace(claire_ctx* c, const T* v, T* out, cudaStream_t st) {
  Work<T>& W = c->work<T>();
  cplx<T>* S = W.spec;
  const long long Ns = c->d.Ns;
  CL_TRY(vec_r2c<T>(c, v, S, st));
  CL_TRY(spec_leray<T>(c, S, S + Ns, S + 2 * Ns, st));
  return vec_c2r<T>(c, S, out, st);
}

// z = M^-1 r (Sec. 2.3.3)
template <class T> claire_status precond_apply(claire_ctx* c, const T* r, T* z, cudaStream_t st) {
  Work<T>& W = c->work<T>();
  CL_TRY(vec_r2c<T>(c, r, W.spec, st));
  CL_TRY(spec_scale<T>(c, W.spec, 3, c->d.Ns, 1, c->o.beta, st));
  return vec_c2r<T>(c, W.spec, z, st);
}

// S_k = f(k) F[x_k] for the three components of a physical FP32 field, with the transform in FP64 (f = scale a(k),
// mode 0, or -|k|^2, mode 2). A symbol that grows with |k| multiplies the rounding error of an FP32 transform --
// spread over all modes -- by up to its largest value (beta |k|^4 reaches 1e4 on a 40^3 grid at beta = 1e-2),
// while the field itself may hold little at high k; the FP64 transform keeps that product at FP32 rounding. Uses
// the trial-velocity array (N doubles) and the inverse-transform work array (Ns complex doubles, the upper half of
// W.spec) as scratch, so S must lie in the lower half of W.spec.
claire_status symbol_vec_f64(claire_ctx* c, const float* x, cplx<float>* S, int ncomp, int mode, double scale,
                             cudaStream_t st) {
  Work<float>& W = c->work<float>();
  double* fd = reinterpret_cast<double*>(W.vtrial);
  cplx<double>* Sd = reinterpret_cast<cplx<double>*>(W.Sc);
  for (int k = 0; k < ncomp; ++k)
    CL_TRY(symbol_r2c_f64(c, x + (long long)k * c->d.N, fd, Sd, S + (long long)k * c->d.Ns, mode, scale, st));
  return CLAIRE_OK;
}
template <class T> inline bool precise_symbols(const claire_ctx* c) { return sizeof(T) == 4 && c->f64_plan; }

// out = beta A v + K b (the spectral tail of Eq. (5) and Eq. (7)); b is consumed
template <class T> claire_status spectral_tail(claire_ctx* c, const T* v, const T* b, T* out, double* reg,
                                               cudaStream_t st) {
  Work<T>& W = c->work<T>();
  const long long Ns = c->d.Ns;
  cplx<T>* V = W.spec;
  cplx<T>* B = W.spec + 3 * Ns;
  const bool precise = precise_symbols<T>(c);
  if (!precise || reg) CL_TRY(vec_r2c<T>(c, v, V, st));
  if (reg) {
    // beta/2 sum_c <v_c, A v_c> by Parseval: h^3/N sum_k a(k) |v^(k)|^2
    CL_TRY(spec_reg_partial<T>(c, V, W.partials, st));
    CL_TRY(reduce_final(c, W.partials, 0.5 * c->o.beta * cellvol(c->d) / double(c->d.N), W.scal + 1, st));
  }
  if constexpr (sizeof(T) == 4) {
    if (precise) {
      // (its FP64 scratch lies in the upper half of W.spec: before b is transformed there)
      CL_TRY(symbol_vec_f64(c, v, V, 3, 0, c->o.beta, st));
      CL_TRY(vec_r2c<T>(c, b, B, st));
      CL_TRY(spec_addk<T>(c, V, B, st));
      return vec_c2r<T>(c, B, out, st);
    }
  }
  CL_TRY(vec_r2c<T>(c, b, B, st));
  CL_TRY(spec_combine<T>(c, V, B, st));
  return vec_c2r<T>(c, B, out, st);
}

// slice j of the gradient history (FP32/FP64, or BF16 in the reduced-storage mode)
template <class T> inline const void* gm_at(claire_ctx* c, int j) {
  Work<T>& W = c->work<T>();
  const long long off = 3LL * j * c->d.N;
  if (c->gm16_on) return static_cast<const char*>(W.gm16) + 2 * off;
  return W.gm + off;
}

// Autotuner of the gather schedule: for a grid and brick halo, time the brick-tiled and the plain gathers once (on
// scratch buffers) for two classes of kernels and keep the faster of each; the choice is cached for the process.
// Light: the one-field steps compiled for 8 resident CTAs (incremental state step, store/accumulate adjoint step,
// state interpolation), timed on the incremental state step. Heavy: the steps with more live state and 4 CTAs
// (last incremental step, adjoint step with the fused <s, b~> or the div v source), timed on the adjoint step
// with the fused product -- the shared-memory taps gain most where few warps are resident.
struct Schedule {
  bool light = true, heavy = true;  // tiled
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, Schedule> g_tune;

template <class T> claire_status tune_tiling(claire_ctx* c, int H, Schedule* out, cudaStream_t st) {
  const auto key = std::make_tuple(c->d.n1, c->d.n2, c->d.n3, H, c->gm16_on ? 1 : 0);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      *out = it->second;
      return CLAIRE_OK;
    }
  }
  Work<T>& W = c->work<T>();
  cudaEvent_t e[2];
  for (auto& x : e) CL_CUDA(c, cudaEventCreate(&x));
  float ms[2][2] = {{0.f, 0.f}, {0.f, 0.f}};  // [class][tiled, plain]
  for (int cls = 0; cls < 2; ++cls) {
    for (int variant = 0; variant < 2; ++variant) {
      const int h = variant == 0 ? H : -1;
      auto run = [&]() -> claire_status {
        if (cls == 0)
          return sl_incstate_step<T>(c, W.la, W.dX, W.s, gm_at<T>(c, 0), c->gm16_on, W.lb, false, nullptr, nullptr,
                                     nullptr, T(0), st, h);
        return sl_adjoint_step<T>(c, W.la, nullptr, nullptr, W.dX, nullptr, nullptr, W.b, gm_at<T>(c, 0), c->gm16_on,
                                  T(0), st, W.s, W.bigpart, h);
      };
      CL_TRY(run());  // warm-up
      CL_CUDA(c, cudaEventRecord(e[0], st));
      for (int r = 0; r < 3; ++r) CL_TRY(run());
      CL_CUDA(c, cudaEventRecord(e[1], st));
      CL_CUDA(c, cudaEventSynchronize(e[1]));
      CL_CUDA(c, cudaEventElapsedTime(&ms[cls][variant], e[0], e[1]));
    }
  }
  for (auto& x : e) cudaEventDestroy(x);
  out->light = ms[0][0] <= ms[0][1];
  out->heavy = ms[1][0] <= ms[1][1];
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = *out;
  return CLAIRE_OK;
}

// Brick halo for the tiled gathers: max |displacement| D in voxels over the field -> H = ceil(D) + 1, per kernel
// class (light, heavy), or -1 where the plain gathers run (the autotuner's choice on this grid, or
// CLAIRE_GATHER=plain; CLAIRE_GATHER=tiled forces the bricks wherever a halo exists)
template <class T> claire_status update_halo(claire_ctx* c, const T* disp, int* halo, int* halo_heavy,
                                             cudaStream_t st) {
  if (c->halo_fixed) return CLAIRE_OK;
  Work<T>& W = c->work<T>();
  CL_TRY(absmax_partial<T>(c, disp, 3 * c->d.N, W.partials, st));
  CL_TRY(max_final(c, W.partials, kReduceBlocks, W.scal + 12, st));
  double D;
  CL_TRY(read_scalar(c, W.scal + 12, &D, st));
  const int H = (std::isfinite(D) && D < 64.0) ? (int)std::ceil(D + 1e-3) + 1 : -1;
  *halo = *halo_heavy = H;
  if (H < 0) return CLAIRE_OK;
  const char* force = std::getenv("CLAIRE_GATHER");
  if (force && std::strcmp(force, "plain") == 0) {
    *halo = *halo_heavy = -1;
  } else if (force && std::strcmp(force, "tiled") == 0) {
    // bricks wherever a halo exists
  } else if (sizeof(T) == 4 && c->gm_ready) {
    Schedule sch;
    CL_TRY(tune_tiling<T>(c, H < 2 ? 2 : H, &sch, st));
    if (!sch.light) *halo = -1;
    if (!sch.heavy) *halo_heavy = -1;
  }
  return CLAIRE_OK;
}

// ---------------------------------------------------------------------------------------------------------------
// state solve along X into the history W.m (m^0 = mT)
template <class T> claire_status state_history(claire_ctx* c, const T* mT, cudaStream_t st) {
  Work<T>& W = c->work<T>();
  const long long N = c->d.N;
  if (W.m != mT) CL_TRY(scale_copy<T>(c, N, 1.0, mT, W.m, st));  // (a kernel: also capturable in a loop body)
  for (int j = 0; j < c->o.nt; ++j) CL_TRY(sl_interp<T>(c, W.m + j * N, W.dX, W.m + (j + 1) * N, st, c->haloX));
  return CLAIRE_OK;
}

// the part of the linearisation that the state history does not cover: Y, grad m^j, div v
template <class T> claire_status finish_linearization(claire_ctx* c, const T* v, cudaStream_t st) {
  Work<T>& W = c->work<T>();
  const long long N = c->d.N;
  CL_TRY(sl_departure<T>(c, v, -1, W.dY, st));
  CL_TRY(update_halo<T>(c, W.dY, &c->haloY, &c->haloYh, st));
  for (int j = 0; j <= c->o.nt; ++j) {
    if (c->gm16_on) {
      // FP32 gradient into the b scratch, then stored in BF16
      CL_TRY(grad_spectral<T>(c, W.m + j * N, W.b, st));
      CL_TRY(to_bf16(c, reinterpret_cast<const float*>(W.b), static_cast<char*>(W.gm16) + 2 * 3LL * j * N, 3 * N,
                     st));
    } else {
      CL_TRY(grad_spectral<T>(c, W.m + j * N, W.gm + 3LL * j * N, st));
    }
  }
  if (!c->o.divfree) CL_TRY(div_spectral<T>(c, v, W.rho, st));
  c->lin_valid = true;
  c->gm_ready = true;
  return CLAIRE_OK;
}

template <class T> claire_status linearize(claire_ctx* c, const T* mT, const T* v, cudaStream_t st) {
  Work<T>& W = c->work<T>();
  c->lin_valid = false;
  CL_TRY(sl_departure<T>(c, v, +1, W.dX, st));
  CL_TRY(update_halo<T>(c, W.dX, &c->haloX, &c->haloXh, st));
  CL_TRY(state_history<T>(c, mT, st));
  return finish_linearization<T>(c, v, st);
}

inline double tweight(int j, int nt) { return (j == 0 || j == nt) ? 0.5 / nt : 1.0 / nt; }


// adjoint backward from lam^{nt} = mR - m^{nt}; b = sum_j w_j lam^j grad m^j (Eq. (4), (5))
template <class T> claire_status adjoint_integral(claire_ctx* c, const T* mR, cudaStream_t st) {
  Work<T>& W = c->work<T>();
  const long long N = c->d.N;
  const int nt = c->o.nt;
  T* lam[2] = {W.la, W.lb};
  T* rl[2] = {W.ra, W.rb};
  const T* rho = c->o.divfree ? nullptr : W.rho;
  CL_TRY(sl_adjoint_terminal<T>(c, mR, W.m + nt * N, rho, lam[0], rl[0], W.b, gm_at<T>(c, nt), c->gm16_on,
                                T(tweight(nt, nt)), st));
  int cur = 0;
  for (int j = nt - 1; j >= 0; --j) {
    const bool store = j > 0;
    CL_TRY(sl_adjoint_step<T>(c, lam[cur], rho ? rl[cur] : nullptr, rho, W.dY, store ? lam[1 - cur] : nullptr,
                              (store && rho) ? rl[1 - cur] : nullptr, W.b, gm_at<T>(c, j), c->gm16_on,
                              T(tweight(j, nt)), st,
                              nullptr, nullptr, rho ? c->haloYh : c->haloY));
    cur = 1 - cur;
  }
  return CLAIRE_OK;
}

// g = beta A v + K b; if J != nullptr also the objective (synchronises)
template <class T> claire_status gradient_at_lin(claire_ctx* c, const T* mR, const T* v, T* g, double* J,
                                                 cudaStream_t st) {
  Work<T>& W = c->work<T>();
  const long long N = c->d.N;
  if (J) {
    CL_TRY(diffsq_partial<T>(c, W.m + c->o.nt * N, mR, N, W.partials, st));
    CL_TRY(reduce_final(c, W.partials, 0.5 * cellvol(c->d), W.scal, st));
  }
  CL_TRY(adjoint_integral<T>(c, mR, st));
  CL_TRY(spectral_tail<T>(c, v, W.b, g, J ? W.scal : nullptr, st));
  if (J) {
    // scal[0] mismatch, scal[1] regularisation (written by spectral_tail into scal + 1)
    CL_CUDA(c, cudaMemcpyAsync(c->hscal, W.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CL_CUDA(c, cudaStreamSynchronize(st));
    *J = c->hscal[0] + c->hscal[1];
  }
  return CLAIRE_OK;
}

// out = u + K b with b the time integral of the last backward sweep (u = beta A v carried by the caller)
template <class T> claire_status add_projected_b(claire_ctx* c, const T* u, T* out, cudaStream_t st) {
  Work<T>& W = c->work<T>();
  const long long n3 = 3 * c->d.N;
  if (c->o.divfree) {
    CL_TRY(leray_inplace<T>(c, W.b, W.b, st));
  } else if (c->o.beta_w > 0.0) {
    const long long Ns = c->d.Ns;
    CL_TRY(vec_r2c<T>(c, W.b, W.spec, st));
    CL_TRY(spec_kop<T>(c, W.spec, W.spec + Ns, W.spec + 2 * Ns, st));
    CL_TRY(vec_c2r<T>(c, W.spec, W.b, st));
  }
  return waxpy<T>(c, n3, u, 1.0, W.b, out, st);
}

// data part of the Gauss-Newton matvec at the cached linearisation: W.b = int lambda~ grad m dt (Eq. (8), (9)).
// With dot = true the last backward step also writes the per-block partials of <vt, W.b> to W.bigpart.
template <class T> claire_status hess_data(claire_ctx* c, const T* vt, cudaStream_t st, bool dot = false) {
  Work<T>& W = c->work<T>();
  const int nt = c->o.nt;
  T* buf[2] = {W.la, W.lb};
  T* rl[2] = {W.ra, W.rb};
  const T* rho = c->o.divfree ? nullptr : W.rho;
  int cur = 0;
  CL_TRY(sl_incstate_init<T>(c, vt, gm_at<T>(c, 0), c->gm16_on, buf[cur], st));
  for (int j = 0; j < nt; ++j) {
    const bool last = j == nt - 1;
    CL_TRY(sl_incstate_step<T>(c, buf[cur], W.dX, vt, gm_at<T>(c, j + 1), c->gm16_on, buf[1 - cur], last, rho,
                               rl[1 - cur], W.b, T(tweight(nt, nt)), st, last ? c->haloXh : c->haloX));
    cur = 1 - cur;
  }
  for (int j = nt - 1; j >= 0; --j) {
    const bool store = j > 0;
    CL_TRY(sl_adjoint_step<T>(c, buf[cur], rho ? rl[cur] : nullptr, rho, W.dY, store ? buf[1 - cur] : nullptr,
                              (store && rho) ? rl[1 - cur] : nullptr, W.b, gm_at<T>(c, j), c->gm16_on,
                              T(tweight(j, nt)),
                              st, (dot && j == 0) ? vt : nullptr, (dot && j == 0) ? W.bigpart : nullptr,
                              ((dot && j == 0) || rho) ? c->haloYh : c->haloY));
    cur = 1 - cur;
  }
  return CLAIRE_OK;
}

// Gauss-Newton matvec at the cached linearisation (Eq. (7)-(9), lambda terms dropped), applying beta A to vt
// through its Fourier symbol (the entry point for an arbitrary vt)
template <class T> claire_status hessvec_at_lin(claire_ctx* c, const T* vt, T* Hvt, cudaStream_t st) {
  CL_TRY(hess_data<T>(c, vt, st));
  return spectral_tail<T>(c, vt, c->work<T>().b, Hvt, nullptr, st);
}

// 1/2 ||m^{nt} - mR||^2 of the state at v (departure X + state history; one PDE solve) into scal[slot]
template <class T> claire_status state_mismatch(claire_ctx* c, const T* mT, const T* mR, const T* v, int slot,
                                                cudaStream_t st) {
  Work<T>& W = c->work<T>();
  const long long N = c->d.N;
  c->lin_valid = false;
  CL_TRY(sl_departure<T>(c, v, +1, W.dX, st));
  CL_TRY(update_halo<T>(c, W.dX, &c->haloX, &c->haloXh, st));
  CL_TRY(state_history<T>(c, mT, st));
  CL_TRY(diffsq_partial<T>(c, W.m + c->o.nt * N, mR, N, W.partials, st));
  return reduce_final(c, W.partials, 0.5 * cellvol(c->d), W.scal + slot, st);
}

claire_status read_scalars(claire_ctx* c, const double* dev, int n, double* out, cudaStream_t st) {
  CL_CUDA(c, cudaMemcpyAsync(c->hscal, dev, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  CL_CUDA(c, cudaStreamSynchronize(st));
  for (int i = 0; i < n; ++i) out[i] = c->hscal[i];
  return CLAIRE_OK;
}

// s = F^-1 S (three components; S is left untouched, W.Sc is the work array)
template <class T> claire_status spec_to_phys(claire_ctx* c, const cplx<T>* S, T* s, cudaStream_t st) {
  Work<T>& W = c->work<T>();
  const long long Ns = c->d.Ns;
  const T inv = T(1.0 / double(c->d.N));
  for (int k = 0; k < 3; ++k) CL_TRY(fft_c2r<T>(c, W.Sc + k * Ns, comp(s, c->d, k), inv, st, S + k * Ns));
  return CLAIRE_OK;
}

// gradient at the cached linearisation into W.Gh: G = beta A V + K F[b] (V null: v = 0); scal[slot] = ||g||^2
template <class T> claire_status gradient_spec(claire_ctx* c, const T* mR, const cplx<T>* V, int slot,
                                               cudaStream_t st) {
  Work<T>& W = c->work<T>();
  CL_TRY(adjoint_integral<T>(c, mR, st));
  CL_TRY(vec_r2c<T>(c, W.b, W.Bh, st));
  CL_TRY(sp_grad<T>(c, V, W.Bh, W.Gh, W.partials, st));
  return reduce_final_v(c, W.partials, 1, kReduceBlocks, cellvol(c->d) / double(c->d.N), W.scal + slot, st);
}

// Two-level preconditioner (Sec. 2.3.3): Z = M^-1 R for the fine residual W.Rh into W.Vtrh, with rz = <R, Z>
// (the K^-1-weighted product for the H1-div model). The coarse right-hand side is the restriction of
// R^-1/2 R; CG on the coarse split system I + R^-1/2 H_data R^-1/2 (direct coarse discretisation at the coarse
// linearisation; no further preconditioner) runs to ||r|| < eps_M ||f||; its solution replaces the coarse modes
// of R^-1/2 R, and Z = R^-1/2 of the result. Coarse vectors: X = VTh, residual Rh, direction Sh, H P = Gh.
template <class T> claire_status twolevel_apply(claire_ctx* c, double eps_M, claire_report* rep, double* rz,
                                                cudaStream_t st) {
  Work<T>& W = c->work<T>();
  claire_ctx* cc = c->coarse;
  Work<T>& Wc = cc->work<T>();
  const double scc = cellvol(cc->d) / double(cc->d.N);
  CL_TRY(tl_restrict<T>(c, cc, W.Rh, Wc.Rh, Wc.Sh, Wc.VTh, 3, true, Wc.partials, st));
  CL_TRY(reduce_final_v(cc, Wc.partials, 2, kReduceBlocks, scc, Wc.scal, st));  // ||f||^2, <K^-1 f, f>
  double v2[2];
  CL_TRY(read_scalars(cc, Wc.scal, 2, v2, st));
  const double f0 = std::sqrt(v2[0]);
  double rr = v2[1];
  if (!std::isfinite(f0) || !std::isfinite(rr)) {
    c->set_error("non-finite coarse right-hand side");
    return CLAIRE_ENAN;
  }
  for (int it = 0; f0 > 0.0 && it < cc->o.max_krylov; ++it) {
    CL_TRY(tl_scale<T>(cc, Wc.Sh, Wc.Sc, st));
    CL_TRY(vec_c2r<T>(cc, Wc.Sc, Wc.s, st));
    CL_TRY(hess_data<T>(cc, Wc.s, st));
    CL_TRY(vec_r2c<T>(cc, Wc.b, Wc.Bh, st));
    CL_TRY(tl_apply<T>(cc, Wc.Sh, Wc.Bh, Wc.Gh, Wc.partials, st));
    CL_TRY(reduce_final_v(cc, Wc.partials, 1, kReduceBlocks, scc, Wc.scal + 2, st));
    double pHp;
    CL_TRY(read_scalars(cc, Wc.scal + 2, 1, &pHp, st));
    rep->coarse_matvecs++;
    if (!(pHp > 0.0)) break;
    const double alpha = rr / pHp;
    CL_TRY(tl_update<T>(cc, Wc.VTh, Wc.Rh, Wc.Sh, Wc.Gh, alpha, Wc.partials, st));
    CL_TRY(reduce_final_v(cc, Wc.partials, 2, kReduceBlocks, scc, Wc.scal, st));
    CL_TRY(read_scalars(cc, Wc.scal, 2, v2, st));
    if (std::sqrt(v2[0]) < eps_M * f0) break;
    const double mu = v2[1] / rr;
    rr = v2[1];
    CL_TRY(tl_dir2<T>(cc, Wc.Rh, Wc.Sh, mu, st));
  }
  CL_TRY(tl_prolong<T>(c, cc, W.Rh, Wc.VTh, W.Vtrh, W.partials, st));
  CL_TRY(reduce_final_v(c, W.partials, 1, kReduceBlocks, cellvol(c->d) / double(c->d.N), W.scal, st));
  return read_scalars(c, W.scal, 1, rz, st);
}

// the coarse problem's linearisation at the current iterate: v restricted spectrally from its master copy W.Vh
template <class T> claire_status coarse_linearize(claire_ctx* c, cudaStream_t st) {
  Work<T>& W = c->work<T>();
  claire_ctx* cc = c->coarse;
  Work<T>& Wc = cc->work<T>();
  CL_TRY(tl_restrict<T>(c, cc, W.Vh, Wc.Gh, nullptr, nullptr, 3, false, Wc.partials, st));  // G^ is free here
  CL_TRY(vec_c2r<T>(cc, Wc.Gh, Wc.vdev, st));
  return linearize<T>(cc, Wc.mTdev, Wc.vdev, st);
}

// m_T on the coarse grid (spectral restriction), kept in the coarse context's Wc.mTdev
template <class T> claire_status coarse_template(claire_ctx* c, const T* mT, cudaStream_t st) {
  Work<T>& W = c->work<T>();
  claire_ctx* cc = c->coarse;
  Work<T>& Wc = cc->work<T>();
  CL_TRY(fft_r2c<T>(c, mT, W.spec, st));
  CL_TRY(tl_restrict<T>(c, cc, W.spec, Wc.spec, nullptr, nullptr, 1, false, Wc.partials, st));
  return fft_c2r<T>(cc, Wc.spec, Wc.mTdev, T(1.0 / double(cc->d.N)), st);
}

// Alg. 2 in the Fourier domain: PCG for H vt = -g with M^-1 = (beta A)^-1 and the relative break
// ||r|| < eps_H ||r_0||. r, s, vt and g are half spectra; beta A, M^-1 and K act as exact diagonal multiplies, and
// inner products follow from Parseval, so the iterates are those of Alg. 2 in exact arithmetic. Each iteration
// transforms s back to physical space for the incremental solves (Eq. (8), (9)) and their time integral b~ forward;
// <s, H s> = <s, beta A s> (spectral) + <s, b~> (fused into the last backward gather).
// ---------------------------------------------------------------------------------------------------------------
// Device-driven PCG (Alg. 2 with the spectral preconditioner): one iteration -- Gauss-Newton matvec, the three
// reductions and the scalar updates -- is captured once into the body of a conditional WHILE graph node; the
// scalars (kappa, mu, the stopping test) are computed by one-thread kernels into the state block ps, in the same
// FP64 operations and order as the host loop, so the iterates are bit-identical. The loop ends on convergence,
// breakdown, a non-finite <s, H s>, or after max_krylov iterations (ps[kPcgCount] counts the matvecs): it cannot
// run unbounded. One graph launch replaces three host round trips per iteration.
__global__ void k_pcg_kappa(double* __restrict__ ps, const double* __restrict__ sBt) {
  if (ps[kPcgDone] != 0.0) return;
  ps[kPcgCount] += 1.0;
  const double sHs = ps[kPcgSAs] + sBt[0];
  if (!isfinite(sHs)) {
    ps[kPcgNan] = 1.0;
    ps[kPcgDone] = 1.0;
  } else if (!(sHs > 0.0)) {
    ps[kPcgBreakdown] = 1.0;
    if (ps[kPcgCount] == 1.0) ps[kPcgCopyS] = 1.0;
    ps[kPcgDone] = 1.0;
  } else {
    ps[kPcgKappa] = ps[kPcgRz] / sHs;
  }
}
// rr[0] = ||r||^2, rr[1] = <r, z> after the step
__global__ void k_pcg_check(double* __restrict__ ps, const double* __restrict__ rr) {
  if (ps[kPcgDone] != 0.0) return;
  if (sqrt(rr[0]) < ps[kPcgEps] * ps[kPcgR0]) {
    ps[kPcgDone] = 1.0;
    return;
  }
  ps[kPcgMu] = rr[1] / ps[kPcgRz];
  ps[kPcgRz] = rr[1];
}
__global__ void k_pcg_next(double* __restrict__ ps, const double* __restrict__ sAs, cudaGraphConditionalHandle h) {
  if (ps[kPcgDone] == 0.0) ps[kPcgSAs] = sAs[0];
  const bool more = ps[kPcgDone] == 0.0 && ps[kPcgCount] < ps[kPcgMaxIt];
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

// One PCG iteration (Alg. 2 lines 6-12) with its scalars on the device, for capture into the body of a
// conditional WHILE node whose handle h k_pcg_next sets: Gauss-Newton matvec with the fused <s, b~>, kappa,
// the fused residual/step update with ||r||^2 and <r, z>, the stopping test, the new direction and s in physical
// space. The FP64 operations and their order are those of the host loop.
template <class T> claire_status pcg_body(claire_ctx* c, cudaStream_t st, cudaGraphConditionalHandle h) {
  Work<T>& W = c->work<T>();
  const double sc = cellvol(c->d) / double(c->d.N);
  double* ps = W.scal + kPcgBase;
  CL_TRY(hess_data<T>(c, W.s, st, true));
  CL_TRY(reduce_final_v(c, W.bigpart, 1, (int)c->dot_blocks, cellvol(c->d), W.scal + 4, st));
  CL_TRY(vec_r2c<T>(c, W.b, W.Bh, st));
  c->prof_begin("pcg_kappa", st);
  k_pcg_kappa<<<1, 1, 0, st>>>(ps, W.scal + 4);
  CL_LAUNCHED(c);
  CL_TRY(sp_pcg_step<T>(c, W.Sh, W.Bh, W.Rh, W.VTh, 0.0, W.partials, st, ps));
  CL_TRY(reduce_final_v(c, W.partials, 2, kReduceBlocks, sc, W.scal, st));
  c->prof_begin("pcg_check", st);
  k_pcg_check<<<1, 1, 0, st>>>(ps, W.scal);
  CL_LAUNCHED(c);
  CL_TRY(sp_pcg_dir<T>(c, W.Rh, W.Sh, 0.0, W.partials, st, ps));
  CL_TRY(reduce_final_v(c, W.partials, 1, kReduceBlocks, sc, W.scal + 2, st));
  c->prof_begin("pcg_next", st);
  k_pcg_next<<<1, 1, 0, st>>>(ps, W.scal + 2, h);
  CL_LAUNCHED(c);
  return spec_to_phys<T>(c, W.Sh, W.s, st);
}

void pcg_graph_release(claire_ctx* c) {
  if (c->pcg_exec) cudaGraphExecDestroy(c->pcg_exec);
  if (c->pcg_graph) cudaGraphDestroy(c->pcg_graph);
  c->pcg_exec = nullptr;
  c->pcg_graph = nullptr;
}

// the PCG loop graph for the current gather schedule and beta_v (captured on first use, and again when either
// changed: both are baked into the captured kernels)
template <class T> claire_status pcg_graph_get(claire_ctx* c, bool* ok) {
  *ok = false;
  const bool verbose = [] {
    const char* m = std::getenv("CLAIRE_PCG");
    return m && std::strcmp(m, "verbose") == 0;
  }();
  auto fail = [&](const char* what, cudaError_t e) {
    if (verbose) std::fprintf(stderr, "claire: PCG graph not used (%s: %s)\n", what, cudaGetErrorString(e));
    cudaGetLastError();
    return CLAIRE_OK;
  };
  const int key[4] = {c->haloX, c->haloXh, c->haloY, c->haloYh};
  if (c->pcg_exec && std::equal(key, key + 4, c->pcg_key) && c->pcg_beta == c->o.beta) {
    *ok = true;
    return CLAIRE_OK;
  }
  pcg_graph_release(c);
  Work<T>& W = c->work<T>();
  const double sc = cellvol(c->d) / double(c->d.N);
  double* ps = W.scal + kPcgBase;
  cudaError_t e;
  if (!c->pcg_cap_stream && (e = cudaStreamCreateWithFlags(&c->pcg_cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return fail("capture stream", e);
  // captured launches do not run, so capturing on a stream of its own needs no ordering against the solve's stream
  cudaStream_t st = c->pcg_cap_stream;
  cudaGraph_t g = nullptr;
  if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return fail("graph", e);
  cudaGraphConditionalHandle h;
  cudaGraphNodeParams np = {};
  cudaGraphNode_t node;
  if ((e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail("conditional handle", e);
  }
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  if ((e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np)) != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail("conditional node", e);
  }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess) {
    cudaGraphDestroy(g);
    return fail("begin capture", e);
  }
  const long long launches0 = c->counters.launches;
  const claire_status cs = pcg_body<T>(c, st, h);
  const std::string cap_err = c->err;
  cudaGraph_t captured = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(st, &captured);
  c->pcg_body_launches = c->counters.launches - launches0;
  c->counters.launches = launches0;
  cudaGraphExec_t ex = nullptr;
  // (any failure: the host-driven loop runs instead)
  if (cs != CLAIRE_OK || ce != cudaSuccess) {
    c->err.clear();
    cudaGraphDestroy(g);
    if (verbose) std::fprintf(stderr, "claire: PCG graph capture failed (%s)\n", cap_err.c_str());
    return fail("end capture", ce);
  }
  if ((e = cudaGraphInstantiate(&ex, g, 0)) != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail("instantiate", e);
  }
  c->pcg_graph = g;
  c->pcg_exec = ex;
  std::copy(key, key + 4, c->pcg_key);
  c->pcg_beta = c->o.beta;
  *ok = true;
  return CLAIRE_OK;
}

template <class T> claire_status pcg(claire_ctx* c, double eps_H, claire_report* rep, cudaStream_t st) {
  Work<T>& W = c->work<T>();
  const double sc = cellvol(c->d) / double(c->d.N);  // Parseval scale h1 h2 h3 / N
  const bool two = c->coarse != nullptr;
  const double eps_M = c->o.pc_kappa * eps_H;
  CL_TRY(sp_pcg0<T>(c, W.Gh, W.Rh, W.Sh, W.VTh, W.partials, st));
  CL_TRY(reduce_final_v(c, W.partials, 3, kReduceBlocks, sc, W.scal, st));  // <r,z>, ||r||^2, <s,beta A s>
  double v3[3];
  CL_TRY(read_scalars(c, W.scal, 3, v3, st));
  double rz = v3[0];
  const double r0 = std::sqrt(v3[1]);
  double sAs = v3[2];
  if (two) {
    // z = M^-1 r of the two-level preconditioner replaces the spectral one: s = z
    CL_TRY(twolevel_apply<T>(c, eps_M, rep, &rz, st));
    CL_TRY(tl_dir<T>(c, W.Vtrh, W.Sh, 0.0, W.partials, st));
    CL_TRY(reduce_final_v(c, W.partials, 1, kReduceBlocks, sc, W.scal + 2, st));
    CL_TRY(read_scalars(c, W.scal + 2, 1, &sAs, st));
  }
  if (!std::isfinite(rz) || !std::isfinite(r0)) {
    c->set_error("non-finite PCG scalar");
    return CLAIRE_ENAN;
  }
  CL_TRY(spec_to_phys<T>(c, W.Sh, W.s, st));
  // host-side fake of a non-positive first <s, H s> (tests of the breakdown path; runs the host-driven loop)
  const bool fake_breakdown = fault_injected("pcg_breakdown");
  // device-driven loop: spectral preconditioner, no per-kernel profiling (its events are per launch, not per
  // graph execution), unless CLAIRE_PCG=host
  const char* mode = std::getenv("CLAIRE_PCG");
  if (!two && !c->prof_on && !c->pcg_graph_failed && !fake_breakdown && !(mode && std::strcmp(mode, "host") == 0)) {
    bool ok = false;
    CL_TRY(pcg_graph_get<T>(c, &ok));
    if (!ok) {
      c->pcg_graph_failed = true;
    } else {
      double* hs = c->hscal + 32;
      for (int k = 0; k < kPcgSlots; ++k) hs[k] = 0.0;
      hs[kPcgRz] = rz;
      hs[kPcgR0] = r0;
      hs[kPcgSAs] = sAs;
      hs[kPcgEps] = eps_H;
      hs[kPcgMaxIt] = double(c->o.max_krylov);
      double* ps = W.scal + kPcgBase;
      CL_CUDA(c, cudaMemcpyAsync(ps, hs, sizeof(double) * kPcgSlots, cudaMemcpyHostToDevice, st));
      CL_CUDA(c, cudaGraphLaunch(c->pcg_exec, st));
      c->pcg_graph_runs++;
      CL_CUDA(c, cudaMemcpyAsync(hs, ps, sizeof(double) * kPcgSlots, cudaMemcpyDeviceToHost, st));
      CL_CUDA(c, cudaStreamSynchronize(st));
      const long long n = (long long)hs[kPcgCount];
      rep->matvecs += (int)n;
      rep->pde_solves += 2 * (int)n;
      c->counters.launches += n * c->pcg_body_launches;
      if (hs[kPcgNan] != 0.0) {
        c->set_error("non-finite <s, Hs>");
        return CLAIRE_ENAN;
      }
      if (hs[kPcgBreakdown] != 0.0) {
        rep->pcg_breakdowns++;
        if (hs[kPcgCopyS] != 0.0)
          CL_CUDA(c, cudaMemcpyAsync(W.VTh, W.Sh, sizeof(cplx<T>) * 3 * c->d.Ns, cudaMemcpyDeviceToDevice, st));
      }
      return CLAIRE_OK;
    }
  }
  for (int it = 0; it < c->o.max_krylov; ++it) {
    CL_TRY(hess_data<T>(c, W.s, st, true));
    CL_TRY(reduce_final_v(c, W.bigpart, 1, (int)c->dot_blocks, cellvol(c->d), W.scal + 4, st));
    CL_TRY(vec_r2c<T>(c, W.b, W.Bh, st));
    rep->matvecs++;
    rep->pde_solves += 2;
    double sBt;
    CL_TRY(read_scalars(c, W.scal + 4, 1, &sBt, st));
    const double sHs = (fake_breakdown && it == 0) ? -std::fabs(sAs + sBt) : sAs + sBt;
    if (!std::isfinite(sHs)) {
      c->set_error("non-finite <s, Hs>");
      return CLAIRE_ENAN;
    }
    if (!(sHs > 0.0)) {
      rep->pcg_breakdowns++;
      if (it == 0)
        CL_CUDA(c, cudaMemcpyAsync(W.VTh, W.Sh, sizeof(cplx<T>) * 3 * c->d.Ns, cudaMemcpyDeviceToDevice, st));
      break;
    }
    const double kappa = rz / sHs;
    CL_TRY(sp_pcg_step<T>(c, W.Sh, W.Bh, W.Rh, W.VTh, kappa, W.partials, st));
    CL_TRY(reduce_final_v(c, W.partials, 2, kReduceBlocks, sc, W.scal, st));  // ||r||^2, <r, z>
    double v2[2];
    CL_TRY(read_scalars(c, W.scal, 2, v2, st));
    if (std::sqrt(v2[0]) < eps_H * r0) break;
    if (two) {
      double rz_new;
      CL_TRY(twolevel_apply<T>(c, eps_M, rep, &rz_new, st));
      const double mu = rz_new / rz;
      rz = rz_new;
      CL_TRY(tl_dir<T>(c, W.Vtrh, W.Sh, mu, W.partials, st));
    } else {
      const double mu = v2[1] / rz;
      rz = v2[1];
      CL_TRY(sp_pcg_dir<T>(c, W.Rh, W.Sh, mu, W.partials, st));
    }
    CL_TRY(reduce_final_v(c, W.partials, 1, kReduceBlocks, sc, W.scal + 2, st));
    CL_TRY(read_scalars(c, W.scal + 2, 1, &sAs, st));
    CL_TRY(spec_to_phys<T>(c, W.Sh, W.s, st));
  }
  return CLAIRE_OK;
}

// ---------------------------------------------------------------------------------------------------------------
// Alg. 1 driven from the device. A whole zero-start solve -- the reference gradient at v = 0, the Gauss-Newton
// loop, PCG (Alg. 2), the Armijo search and the stopping tests of Sec. 2.3.2 -- is captured once into a CUDA graph
// of conditional nodes: an outer WHILE over a table of pairs (m_T, m_R, v) copied through the context's own
// buffers, a WHILE over Gauss-Newton iterations, and inside it the PCG WHILE, the Armijo WHILE and an IF for the
// accepted step. Every decision is taken by one-thread kernels on an FP64 state block (GnSlot) in the same FP64
// operations and order as the host-driven loop, so the iterates are bit-identical to it. Every loop is bounded by
// the options (max_gn, max_krylov, max_ls), and the pair loop by the table's length. The gathers keep the halos
// fixed at capture time: the brick-tiled and the global-tap gathers produce the same values, so the halo choice
// changes only speed.
struct PairRef {
  const void* mT;
  const void* mR;
  void* v;
};

__device__ __forceinline__ void gn_decide(double* gs, cudaGraphConditionalHandle h) {
  bool more = false;
  if (gs[kGnStatus] == 0.0) {
    const double g = gs[kGnGnorm];
    if (g <= gs[kGnGtolRel] * gs[kGnGnorm0] || g <= gs[kGnGtolAbs])
      gs[kGnStatus] = 1.0;
    else if (gs[kGnIters] >= gs[kGnMaxGn])
      gs[kGnStatus] = 2.0;
    else
      more = true;
  }
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

__global__ void k_pairs_first(int* __restrict__ k, const int* __restrict__ n, cudaGraphConditionalHandle h) {
  *k = 0;
  cudaGraphSetConditional(h, *n > 0 ? 1u : 0u);
}
__global__ void k_pairs_next(int* __restrict__ k, const int* __restrict__ n, cudaGraphConditionalHandle h) {
  const int j = *k + 1;
  *k = j;
  cudaGraphSetConditional(h, j < *n ? 1u : 0u);
}
// pair k's images into the context's buffers, v = 0, and the state block reset from its template
template <class T>
__global__ void k_pair_in(const PairRef* __restrict__ tab, const int* __restrict__ k, T* __restrict__ mT,
                          T* __restrict__ mR, T* __restrict__ v, long long N, double* __restrict__ gs,
                          const double* __restrict__ tmpl) {
  const PairRef p = tab[*k];
  const T* a = static_cast<const T*>(p.mT);
  const T* b = static_cast<const T*>(p.mR);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    mT[i] = a[i];
    mR[i] = b[i];
    v[i] = T(0);
    v[N + i] = T(0);
    v[2 * N + i] = T(0);
  }
  if (blockIdx.x == 0 && threadIdx.x < kGnSlots) gs[threadIdx.x] = tmpl[threadIdx.x];
}
// v to pair k's array and the state block to its report row
template <class T>
__global__ void k_pair_out(const PairRef* __restrict__ tab, const int* __restrict__ k, const T* __restrict__ v,
                           long long N, const double* __restrict__ gs, double* __restrict__ reports) {
  const PairRef p = tab[*k];
  T* out = static_cast<T*>(p.v);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * N;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = v[i];
  if (blockIdx.x == 0 && threadIdx.x < kGnSlots) reports[(long long)(*k) * kGnSlots + threadIdx.x] = gs[threadIdx.x];
}
// after the reference gradient at v = 0: non-finite inputs, mismatch0 = J0, g_0, then the first stopping test
__global__ void k_gn_start(double* __restrict__ gs, const double* __restrict__ in2, double half_cell,
                           const double* __restrict__ gg, cudaGraphConditionalHandle h) {
  if (in2[0] != 0.0) gs[kGnStatus] = 4.0;
  const double J = half_cell * in2[1];
  gs[kGnJ0] = J;
  gs[kGnJ] = J;
  const double gn = sqrt(gg[0]);
  gs[kGnGnorm0] = gn;
  gs[kGnGnorm] = gn;
  gs[kGnPde] = 2.0;
  if (!isfinite(J) || !isfinite(gn)) gs[kGnStatus] = 4.0;
  gn_decide(gs, h);
}
// forcing term and the PCG state from <r, z>, ||r||^2, <s, beta A s> (Alg. 2 lines 1-4)
__global__ void k_gn_pcg_init(double* __restrict__ gs, double* __restrict__ ps, const double* __restrict__ s3,
                              cudaGraphConditionalHandle h) {
  for (int i = 0; i < kPcgSlots; ++i) ps[i] = 0.0;
  ps[kPcgDone] = 1.0;
  if (gs[kGnStatus] != 0.0) {
    cudaGraphSetConditional(h, 0u);
    return;
  }
  const double rz = s3[0], r0 = sqrt(s3[1]);
  if (!isfinite(rz) || !isfinite(r0)) {
    gs[kGnStatus] = 4.0;
    cudaGraphSetConditional(h, 0u);
    return;
  }
  ps[kPcgRz] = rz;
  ps[kPcgR0] = r0;
  ps[kPcgSAs] = s3[2];
  ps[kPcgEps] = gs[kGnPcgRtol] > 0 ? gs[kGnPcgRtol] : fmin(0.5, sqrt(gs[kGnGnorm] / gs[kGnGnorm0]));
  ps[kPcgMaxIt] = gs[kGnMaxKrylov];
  ps[kPcgDone] = 0.0;
  cudaGraphSetConditional(h, 1u);
}
// after the PCG loop: counts, breakdown, non-finite <s, H s>
__global__ void k_gn_pcg_end(double* __restrict__ gs, const double* __restrict__ ps) {
  if (gs[kGnStatus] != 0.0) return;
  const double n = ps[kPcgCount];
  gs[kGnMatvecs] += n;
  gs[kGnPde] += 2.0 * n;
  if (ps[kPcgNan] != 0.0) gs[kGnStatus] = 4.0;
  if (ps[kPcgBreakdown] != 0.0) gs[kGnBreakdowns] += 1.0;
}
// breakdown in the first PCG iteration: the step is the first direction
template <class T>
__global__ void k_copy_if_first_breakdown(const double* __restrict__ ps, const T* __restrict__ src, T* __restrict__ dst,
                                          long long n) {
  if (ps[kPcgBreakdown] == 0.0 || ps[kPcgCopyS] == 0.0) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}
__global__ void k_ls_init(double* __restrict__ gs, const double* __restrict__ gvt, cudaGraphConditionalHandle h) {
  gs[kGnGvt] = gvt[0];
  gs[kGnAlpha] = 1.0;
  gs[kGnTrial] = 0.0;
  gs[kGnAccepted] = 0.0;
  cudaGraphSetConditional(h, gs[kGnStatus] == 0.0 ? 1u : 0u);
}
// one Armijo test (Alg. 1 line 9): J(v + alpha vt) <= J + c1 alpha <g, vt>, else alpha /= 2
__global__ void k_ls_check(double* __restrict__ gs, const double* __restrict__ r2, cudaGraphConditionalHandle h) {
  const double Jt = r2[0] + r2[1];
  gs[kGnJt] = Jt;
  gs[kGnLsTrials] += 1.0;
  gs[kGnPde] += 1.0;
  gs[kGnTrial] += 1.0;
  if (!isfinite(Jt)) {
    gs[kGnStatus] = 4.0;
    cudaGraphSetConditional(h, 0u);
    return;
  }
  const double alpha = gs[kGnAlpha];
  if (Jt <= gs[kGnJ] + gs[kGnC1] * alpha * gs[kGnGvt]) {
    gs[kGnAccepted] = 1.0;
    cudaGraphSetConditional(h, 0u);
    return;
  }
  gs[kGnAlpha] = alpha * 0.5;
  cudaGraphSetConditional(h, gs[kGnTrial] < gs[kGnMaxLs] ? 1u : 0u);
}
__global__ void k_ls_end(double* __restrict__ gs, cudaGraphConditionalHandle h) {
  const bool ok = gs[kGnStatus] == 0.0;
  if (ok && gs[kGnAccepted] == 0.0) gs[kGnStatus] = 3.0;
  cudaGraphSetConditional(h, (ok && gs[kGnAccepted] != 0.0) ? 1u : 0u);
}
// the accepted step's gradient norm, then the stopping tests for the next iteration
__global__ void k_gn_update(double* __restrict__ gs, const double* __restrict__ gg) {
  gs[kGnJ] = gs[kGnJt];
  gs[kGnPde] += 1.0;
  const double gn = sqrt(gg[0]);
  gs[kGnGnorm] = gn;
  gs[kGnIters] += 1.0;
  if (!isfinite(gn)) gs[kGnStatus] = 4.0;
}
__global__ void k_gn_next(double* __restrict__ gs, cudaGraphConditionalHandle h) { gn_decide(gs, h); }
__global__ void k_gn_after(const double* __restrict__ gs, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, gs[kGnStatus] == 3.0 ? 1u : 0u);
}

// a handle for a conditional node that will be added to the graph stream st is capturing into
cudaError_t cond_handle(cudaStream_t st, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive || !g) return cudaErrorStreamCaptureInvalidated;
  return cudaGraphConditionalHandleCreate(h, g, 0, cudaGraphCondAssignDefault);
}
// appends a conditional node (WHILE or IF, one body) after the capture position of st; *body is its body graph
cudaError_t cond_node(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                      cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive || !g) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np)) != cudaSuccess) return e;
  *body = np.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

#define GN_CE(call)                                                                                  \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) {                                                                         \
      c->set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                              \
      return CLAIRE_ECUDA;                                                                           \
    }                                                                                                \
  } while (0)

// layout of the graph's device block
struct GnBlock {
  int* k;
  int* n;
  PairRef* tab;
  double* tmpl;
  double* reports;
};
inline GnBlock gn_block(claire_ctx* c) {
  char* p = static_cast<char*>(c->gn_dev);
  GnBlock b;
  b.k = reinterpret_cast<int*>(p);
  b.n = b.k + 1;
  b.tmpl = reinterpret_cast<double*>(p + 256);
  b.tab = reinterpret_cast<PairRef*>(p + 256 + 8 * kGnSlots);
  b.reports = reinterpret_cast<double*>(p + 256 + 8 * kGnSlots + sizeof(PairRef) * size_t(c->gn_cap));
  return b;
}
inline size_t gn_block_bytes(int cap) { return 256 + 8 * kGnSlots + (sizeof(PairRef) + 8 * kGnSlots) * size_t(cap); }

inline unsigned copy_blocks(long long n) {
  const long long b = (n + 255) / 256;
  return (unsigned)(b < 4864 ? b : 4864);
}

// capture the whole solve into a new graph (the context's halos are held fixed while it runs)
// Captures the device-driven solve of this context's pair table into a new graph (*out), or, with `into`, appends it
// to that graph as an independent branch (the batch's single graph: one branch per context).
template <class T> claire_status gn_capture(claire_ctx* c, cudaGraph_t* out, cudaGraph_t into = nullptr) {
  Work<T>& W = c->work<T>();
  const Dims& d = c->d;
  const long long N = d.N, n3 = 3 * N, Ns = d.Ns;
  const double sc = cellvol(d) / double(N);
  double* gs = W.scal + kGnBase;
  double* ps = W.scal + kPcgBase;
  const GnBlock B = gn_block(c);
  cudaStream_t s0 = c->pcg_cap_stream, s1 = c->gn_cap_streams[0], s2 = c->gn_cap_streams[1],
               s3 = c->gn_cap_streams[2];
  cudaGraph_t g = into;
  if (!g) {
    GN_CE(cudaGraphCreate(&g, 0));
    *out = g;
  }
  GN_CE(cudaStreamBeginCaptureToGraph(s0, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  auto body = [&](cudaStream_t st, cudaGraph_t bg, long long* count, auto&& fn) -> claire_status {
    GN_CE(cudaStreamBeginCaptureToGraph(st, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const long long l0 = c->counters.launches;
    const claire_status r = fn();
    cudaGraph_t tmp = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &tmp);
    if (count) *count = c->counters.launches - l0;
    if (r != CLAIRE_OK) return r;
    GN_CE(e);
    return CLAIRE_OK;
  };
  long long l_pcg = 0, l_trial = 0, l_acc = 0, l_fail = 0, l_iter_all = 0, l_pair_all = 0;
  auto top = [&]() -> claire_status {
    cudaGraphConditionalHandle hp;
    GN_CE(cond_handle(s0, &hp));
    k_pairs_first<<<1, 1, 0, s0>>>(B.k, B.n, hp);
    GN_CE(cudaGetLastError());
    cudaGraph_t bp;
    GN_CE(cond_node(s0, hp, cudaGraphCondTypeWhile, &bp));
    // ---- one pair: its images in, the reference gradient at v = 0, the Gauss-Newton loop, v and report out
    return body(s1, bp, &l_pair_all, [&]() -> claire_status {
      cudaStream_t st = s1;
      c->prof_begin("pair_in", st);
      k_pair_in<T><<<copy_blocks(N), 256, 0, st>>>(B.tab, B.k, W.mTdev, W.mRdev, W.vdev, N, gs, B.tmpl);
      CL_LAUNCHED(c);
      CL_TRY(nonfinite_partial<T>(c, W.mTdev, N, W.mRdev, N, W.partials, st));
      CL_TRY(diffsq_partial<T>(c, W.mTdev, W.mRdev, N, W.partials + kReduceBlocks, st));
      CL_TRY(reduce_final_v(c, W.partials, 2, kReduceBlocks, 1.0, W.scal + 13, st));
      CL_TRY(zero_fill<T>(c, n3, W.vtrial, st));
      CL_TRY(linearize<T>(c, W.mTdev, W.vtrial, st));
      CL_TRY(gradient_spec<T>(c, W.mRdev, (const cplx<T>*)nullptr, 0, st));
      CL_TRY(zero_fill<T>(c, 2 * 3 * Ns, reinterpret_cast<T*>(W.Vh), st));
      cudaGraphConditionalHandle hg;
      GN_CE(cond_handle(st, &hg));
      c->prof_begin("gn_start", st);
      k_gn_start<<<1, 1, 0, st>>>(gs, W.scal + 13, 0.5 * cellvol(d), W.scal, hg);
      CL_LAUNCHED(c);
      cudaGraph_t bg;
      GN_CE(cond_node(st, hg, cudaGraphCondTypeWhile, &bg));
      // ---- one Gauss-Newton iteration (Alg. 1 lines 4-12)
      CL_TRY(body(s2, bg, &l_iter_all, [&]() -> claire_status {
        cudaStream_t st = s2;
        CL_TRY(sp_pcg0<T>(c, W.Gh, W.Rh, W.Sh, W.VTh, W.partials, st));
        CL_TRY(reduce_final_v(c, W.partials, 3, kReduceBlocks, sc, W.scal, st));
        cudaGraphConditionalHandle hpcg;
        GN_CE(cond_handle(st, &hpcg));
        c->prof_begin("gn_pcg_init", st);
        k_gn_pcg_init<<<1, 1, 0, st>>>(gs, ps, W.scal, hpcg);
        CL_LAUNCHED(c);
        CL_TRY(spec_to_phys<T>(c, W.Sh, W.s, st));
        cudaGraph_t bpcg;
        GN_CE(cond_node(st, hpcg, cudaGraphCondTypeWhile, &bpcg));
        CL_TRY(body(s3, bpcg, &l_pcg, [&]() { return pcg_body<T>(c, s3, hpcg); }));
        c->prof_begin("gn_pcg_end", st);
        k_gn_pcg_end<<<1, 1, 0, st>>>(gs, ps);
        CL_LAUNCHED(c);
        c->prof_begin("copy_if_breakdown", st);
        k_copy_if_first_breakdown<T><<<copy_blocks(2 * 3 * Ns), 256, 0, st>>>(
            ps, reinterpret_cast<const T*>(W.Sh), reinterpret_cast<T*>(W.VTh), 2 * 3 * Ns);
        CL_LAUNCHED(c);
        CL_TRY(sp_project_dot<T>(c, W.Gh, W.VTh, W.partials, st));
        CL_TRY(reduce_final_v(c, W.partials, 1, kReduceBlocks, sc, W.scal + 7, st));
        cudaGraphConditionalHandle hls;
        GN_CE(cond_handle(st, &hls));
        c->prof_begin("ls_init", st);
        k_ls_init<<<1, 1, 0, st>>>(gs, W.scal + 7, hls);
        CL_LAUNCHED(c);
        cudaGraph_t bls;
        GN_CE(cond_node(st, hls, cudaGraphCondTypeWhile, &bls));
        // ---- one Armijo trial
        CL_TRY(body(s3, bls, &l_trial, [&]() -> claire_status {
          cudaStream_t st = s3;
          CL_TRY(sp_trial<T>(c, W.Vh, W.VTh, W.Vtrh, W.Sc, 0.0, W.partials, st, gs + kGnAlpha));
          CL_TRY(reduce_final_v(c, W.partials, 1, kReduceBlocks, 0.5 * c->o.beta * sc, W.scal + 5, st));
          CL_TRY(vec_c2r<T>(c, W.Sc, W.vtrial, st));
          CL_TRY(state_mismatch<T>(c, W.mTdev, W.mRdev, W.vtrial, 6, st));
          c->prof_begin("ls_check", st);
          k_ls_check<<<1, 1, 0, st>>>(gs, W.scal + 5, hls);
          CL_LAUNCHED(c);
          return CLAIRE_OK;
        }));
        cudaGraphConditionalHandle hacc;
        GN_CE(cond_handle(st, &hacc));
        c->prof_begin("ls_end", st);
        k_ls_end<<<1, 1, 0, st>>>(gs, hacc);
        CL_LAUNCHED(c);
        cudaGraph_t bacc;
        GN_CE(cond_node(st, hacc, cudaGraphCondTypeIf, &bacc));
        // ---- the accepted step: new iterate, its linearisation and gradient
        CL_TRY(body(s3, bacc, &l_acc, [&]() -> claire_status {
          cudaStream_t st = s3;
          CL_TRY(scale_copy<T>(c, 2 * 3 * Ns, 1.0, reinterpret_cast<const T*>(W.Vtrh), reinterpret_cast<T*>(W.Vh),
                               st));
          CL_TRY(scale_copy<T>(c, n3, 1.0, W.vtrial, W.vdev, st));
          CL_TRY(finish_linearization<T>(c, W.vdev, st));
          CL_TRY(gradient_spec<T>(c, W.mRdev, W.Vh, 0, st));
          c->prof_begin("gn_update", st);
          k_gn_update<<<1, 1, 0, st>>>(gs, W.scal);
          CL_LAUNCHED(c);
          return CLAIRE_OK;
        }));
        c->prof_begin("gn_next", st);
        k_gn_next<<<1, 1, 0, st>>>(gs, hg);
        CL_LAUNCHED(c);
        return CLAIRE_OK;
      }));
      // ---- after a failed line search the state is recomputed at the last accepted v
      cudaGraphConditionalHandle hf;
      GN_CE(cond_handle(st, &hf));
      c->prof_begin("gn_after", st);
      k_gn_after<<<1, 1, 0, st>>>(gs, hf);
      CL_LAUNCHED(c);
      cudaGraph_t bf;
      GN_CE(cond_node(st, hf, cudaGraphCondTypeIf, &bf));
      CL_TRY(body(s2, bf, &l_fail, [&]() -> claire_status {
        CL_TRY(sl_departure<T>(c, W.vdev, +1, W.dX, s2));
        return state_history<T>(c, W.mTdev, s2);
      }));
      CL_TRY(diffsq_partial<T>(c, W.m + c->o.nt * N, W.mRdev, N, W.partials, st));
      CL_TRY(reduce_final(c, W.partials, 0.5 * cellvol(d), gs + kGnMismatch, st));
      c->prof_begin("pair_out", st);
      k_pair_out<T><<<copy_blocks(n3), 256, 0, st>>>(B.tab, B.k, W.vdev, N, gs, B.reports);
      CL_LAUNCHED(c);
      c->prof_begin("pairs_next", st);
      k_pairs_next<<<1, 1, 0, st>>>(B.k, B.n, hp);
      CL_LAUNCHED(c);
      return CLAIRE_OK;
    });
  };
  const long long launches0 = c->counters.launches;
  const claire_status r = top();
  cudaGraph_t tmp = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s0, &tmp);
  c->counters.launches = launches0;
  if (r != CLAIRE_OK) return r;
  GN_CE(e);
  // launches per part, each body counted without the bodies nested in it
  c->gn_l_pcg = l_pcg;
  c->gn_l_trial = l_trial;
  c->gn_l_accept = l_acc;
  c->gn_l_iter = l_iter_all - l_pcg - l_trial - l_acc;
  c->gn_l_pair = l_pair_all - l_iter_all - l_fail + 2;
  return CLAIRE_OK;
}

// the device copies of m_T, m_R and v that the host-array calls and the device-driven solve work on
template <class T> claire_status ensure_hostbuf(claire_ctx* c) {
  Work<T>& W = c->work<T>();
  if (W.mRdev) return CLAIRE_OK;
  const long long N = c->d.N;
  if (cudaMalloc(&c->hostbuf, sizeof(T) * 5 * size_t(N)) != cudaSuccess) {
    cudaGetLastError();
    c->hostbuf = nullptr;
    c->set_error("cudaMalloc of the context's copies of m_T, m_R and v failed");
    return CLAIRE_ENOMEM;
  }
  W.vdev = static_cast<T*>(c->hostbuf);
  W.mTdev = W.vdev + 3 * N;
  W.mRdev = W.mTdev + N;
  return CLAIRE_OK;
}

// Halos of a solve driven from the device, fixed before capture: 2 (departure points up to 1 voxel per time step
// stay inside the bricks; farther ones fall back to global taps node by node; CLAIRE_GN_HALO=2..5 picks another;
// measured on the 64-pair batch: 1.047 s at halo 2 against 1.076 s at halo 3, whose larger bricks and staged
// operands leave two CTAs per SM instead of three),
// or global taps for a kernel class where the autotuner has preferred them on this grid; CLAIRE_GATHER=plain|tiled
// overrides as elsewhere.
template <class T> claire_status gn_fix_halos(claire_ctx* c, cudaStream_t st) {
  int H = sizeof(T) == 4 ? 2 : -1;
  const char* hv = std::getenv("CLAIRE_GN_HALO");  // another fixed halo (2..5)
  if (hv && sizeof(T) == 4) {
    const int h = std::atoi(hv);
    if (h >= 2 && h <= 5) H = h;
  }
  c->haloX = c->haloXh = c->haloY = c->haloYh = H;
  const char* force = std::getenv("CLAIRE_GATHER");
  if (force && std::strcmp(force, "plain") == 0) {
    c->haloX = c->haloXh = c->haloY = c->haloYh = -1;
  } else if (!(force && std::strcmp(force, "tiled") == 0) && sizeof(T) == 4 && c->gm_ready) {
    Schedule sch;
    CL_TRY(tune_tiling<T>(c, H, &sch, st));
    if (!sch.light) c->haloX = c->haloY = -1;
    if (!sch.heavy) c->haloXh = c->haloYh = -1;
  }
  return CLAIRE_OK;
}

void gn_graph_release(claire_ctx* c) {
  if (c->gn_exec) cudaGraphExecDestroy(c->gn_exec);
  if (c->gn_graph) cudaGraphDestroy(c->gn_graph);
  c->gn_exec = nullptr;
  c->gn_graph = nullptr;
}

// Enqueues the solves of pairs[0..n) (device arrays of this context's grid; every v is overwritten, the solves
// start from v = 0) as one graph launch on st; the per-pair state blocks land in reports (pinned host memory,
// n x kGnSlots doubles) once st has been synchronised.
// Buffers, capture streams, halos and TMA maps of a device-driven solve of n pairs on this context.
template <class T> claire_status gn_setup(claire_ctx* c, int n, cudaStream_t st) {
  CL_TRY(ensure_hostbuf<T>(c));
  if (!c->gn_dev || c->gn_cap < n) {
    gn_graph_release(c);
    if (c->gn_dev) cudaFree(c->gn_dev);
    c->gn_dev = nullptr;
    const int cap = n < 8 ? 8 : n;
    if (cudaMalloc(&c->gn_dev, gn_block_bytes(cap)) != cudaSuccess) {
      cudaGetLastError();
      c->set_error("cudaMalloc of the device-driven solve's pair table failed");
      return CLAIRE_ENOMEM;
    }
    c->gn_cap = cap;
  }
  if (!c->pcg_cap_stream) CL_CUDA(c, cudaStreamCreateWithFlags(&c->pcg_cap_stream, cudaStreamNonBlocking));
  for (cudaStream_t& s : c->gn_cap_streams)
    if (!s) CL_CUDA(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  CL_TRY(gn_fix_halos<T>(c, st));
  if constexpr (sizeof(T) == 4) sl_tma_prepare(c);  // host-side set-up of the staged gathers, before any capture
  return CLAIRE_OK;
}

// The pair table, the solver settings and the pair count of a device-driven solve, copied to the device on st.
template <class T> claire_status gn_upload(claire_ctx* c, const PairRef* pairs, int n, cudaStream_t st) {
  const GnBlock B = gn_block(c);
  double tmpl[kGnSlots] = {};
  const claire_opts& o = c->o;
  tmpl[kGnMaxGn] = o.max_gn;
  tmpl[kGnMaxLs] = o.max_ls;
  tmpl[kGnC1] = o.armijo_c1;
  tmpl[kGnGtolRel] = o.gtol_rel;
  tmpl[kGnGtolAbs] = o.gtol_abs;
  tmpl[kGnPcgRtol] = o.pcg_rtol;
  tmpl[kGnMaxKrylov] = o.max_krylov;
  // (pageable sources: each copy is staged before the call returns)
  CL_CUDA(c, cudaMemcpyAsync(B.tmpl, tmpl, sizeof(tmpl), cudaMemcpyHostToDevice, st));
  CL_CUDA(c, cudaMemcpyAsync(B.tab, pairs, sizeof(PairRef) * size_t(n), cudaMemcpyHostToDevice, st));
  CL_CUDA(c, cudaMemcpyAsync(B.n, &n, sizeof(int), cudaMemcpyHostToDevice, st));
  return CLAIRE_OK;
}

template <class T> claire_status gn_run(claire_ctx* c, const PairRef* pairs, int n, double* reports, cudaStream_t st) {
  CL_TRY(gn_setup<T>(c, n, st));
  const int key[4] = {c->haloX, c->haloXh, c->haloY, c->haloYh};
  if (!c->gn_exec || !std::equal(key, key + 4, c->gn_key_halo) || c->gn_beta != c->o.beta) {
    gn_graph_release(c);
    c->halo_fixed = true;
    cudaGraph_t g = nullptr;
    const claire_status cs = gn_capture<T>(c, &g);
    c->halo_fixed = false;
    if (cs != CLAIRE_OK) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return cs;
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      c->set_error(std::string("cudaGraphInstantiate (device-driven solve): ") + cudaGetErrorString(e));
      return CLAIRE_ECUDA;
    }
    c->gn_graph = g;
    c->gn_exec = ex;
    std::copy(key, key + 4, c->gn_key_halo);
    c->gn_beta = c->o.beta;
  }
  const GnBlock B = gn_block(c);
  CL_TRY(gn_upload<T>(c, pairs, n, st));
  CL_CUDA(c, cudaGraphLaunch(c->gn_exec, st));
  c->gn_graph_runs++;
  CL_CUDA(c, cudaMemcpyAsync(reports, B.reports, sizeof(double) * kGnSlots * size_t(n), cudaMemcpyDeviceToHost, st));
  return CLAIRE_OK;
}

// a pair's report and status from its device state block (after the stream has been synchronised)
claire_status gn_report(claire_ctx* c, const double* gs, claire_report* rep) {
  std::memset(rep, 0, sizeof(*rep));
  rep->gn_iters = (int)gs[kGnIters];
  rep->matvecs = (int)gs[kGnMatvecs];
  rep->pde_solves = (int)gs[kGnPde];
  rep->ls_trials = (int)gs[kGnLsTrials];
  rep->pcg_breakdowns = (int)gs[kGnBreakdowns];
  rep->J0 = gs[kGnJ0];
  rep->mismatch0 = gs[kGnJ0];
  rep->J = gs[kGnJ];
  rep->mismatch = gs[kGnMismatch];
  rep->gnorm0 = gs[kGnGnorm0];
  rep->gnorm = gs[kGnGnorm];
  const int status = (int)gs[kGnStatus];
  rep->converged = status == 1;
  const long long entered = rep->gn_iters + ((status == 3 || status == 4) ? 1 : 0);
  c->counters.launches += c->gn_l_pair + entered * c->gn_l_iter + rep->matvecs * c->gn_l_pcg +
                          rep->ls_trials * c->gn_l_trial + rep->gn_iters * c->gn_l_accept;
  switch (status) {
    case 1: return CLAIRE_OK;
    case 2: return CLAIRE_ENOTCONV;
    case 3: return CLAIRE_ELINESEARCH;
    case 4: c->set_error("non-finite input, objective or gradient"); return CLAIRE_ENAN;
    default: c->set_error("device-driven solve ended without a status"); return CLAIRE_ECUDA;
  }
}

// the device-driven form of register_dev for a zero initial guess (one pair)
template <class T> claire_status register_graph(claire_ctx* c, const T* mT, const T* mR, T* v, claire_report* rep,
                                                cudaStream_t st) {
  cudaEvent_t e0, e1;
  CL_CUDA(c, cudaEventCreate(&e0));
  CL_CUDA(c, cudaEventCreate(&e1));
  CL_CUDA(c, cudaEventRecord(e0, st));
  const PairRef p{mT, mR, v};
  double* hs = c->hscal + 64;
  claire_status s = gn_run<T>(c, &p, 1, hs, st);
  if (s == CLAIRE_OK) {
    CL_CUDA(c, cudaEventRecord(e1, st));
    CL_CUDA(c, cudaEventSynchronize(e1));
    s = gn_report(c, hs, rep);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    rep->ms_total = ms;
    if (sizeof(T) == 4 && c->tma_steps > 0) {
      const claire_status ts = sl_tma_take_error(c);
      if (ts != CLAIRE_OK) s = ts;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}

// Alg. 1 with Armijo backtracking and the stopping rules of Sec. 2.3.2. The iterate is kept as its half spectrum
// (master copy) next to its physical values (needed by the departure points); the gradient, the step and the
// regularisation value live in the Fourier domain (see pcg).
template <class T> claire_status register_dev(claire_ctx* c, const T* mT, const T* mR, T* v, claire_report* rep,
                                              cudaStream_t st) {
  Work<T>& W = c->work<T>();
  const long long N = c->d.N, n3 = 3 * N;
  const claire_opts& o = c->o;
  const double sc = cellvol(c->d) / double(N);
  std::memset(rep, 0, sizeof(*rep));
  {
    // the whole zero-start solve as one graph launch (CLAIRE_GN=device; spectral preconditioner, no profiling)
    const char* gm = std::getenv("CLAIRE_GN");
    if (gm && std::strcmp(gm, "device") == 0 && !c->prof_on && !c->coarse) {
      double vv = 0.0;
      CL_TRY(inner<T>(c, v, v, n3, &vv, st));
      if (vv == 0.0) return register_graph<T>(c, mT, mR, v, rep, st);
    }
  }
  cudaEvent_t e0, e1;
  CL_CUDA(c, cudaEventCreate(&e0));
  CL_CUDA(c, cudaEventCreate(&e1));
  CL_CUDA(c, cudaEventRecord(e0, st));
  claire_status status = CLAIRE_OK;
  do {
    // non-finite inputs are rejected before anything else runs: counts of NaN/Inf in (m_T, m_R) and in v, and
    // the initial mismatch sum, in one read
    CL_TRY(nonfinite_partial<T>(c, mT, N, mR, N, W.partials, st));
    CL_TRY(nonfinite_partial<T>(c, v, n3, (const T*)nullptr, 0, W.partials + kReduceBlocks, st));
    CL_TRY(diffsq_partial<T>(c, mT, mR, N, W.partials + 2 * kReduceBlocks, st));
    CL_TRY(reduce_final_v(c, W.partials, 3, kReduceBlocks, 1.0, W.scal + 13, st));
    double in3[3];
    CL_TRY(read_scalars(c, W.scal + 13, 3, in3, st));
    if (in3[0] != 0.0 || in3[1] != 0.0) {
      c->set_error(in3[0] != 0.0 ? "non-finite values in m_T or m_R" : "non-finite values in the initial v");
      status = CLAIRE_ENAN;
      break;
    }
    rep->mismatch0 = 0.5 * cellvol(c->d) * in3[2];
    // reference gradient at v = 0 (Sec. 2.3.2)
    double vv;
    CL_TRY(inner<T>(c, v, v, n3, &vv, st));
    CL_CUDA(c, cudaMemsetAsync(W.vtrial, 0, sizeof(T) * n3, st));
    CL_TRY(linearize<T>(c, mT, W.vtrial, st));
    CL_TRY(gradient_spec<T>(c, mR, (const cplx<T>*)nullptr, 0, st));
    rep->pde_solves += 2;
    double gg;
    CL_TRY(read_scalars(c, W.scal, 1, &gg, st));
    rep->gnorm0 = std::sqrt(gg);
    double J = rep->mismatch0;
    if (vv > 0.0) {
      CL_TRY(vec_r2c<T>(c, v, W.Vh, st));
      if (o.divfree) {
        // The reduced space is divergence-free (Sec. 2.2): project the initial guess onto it and continue from
        // the projected v. Without this, the curl-free part of v (for a nonzero guess at least its rounding
        // error) stays in beta A v, where no projected Gauss-Newton step can remove it.
        CL_TRY(spec_leray<T>(c, W.Vh, W.Vh + c->d.Ns, W.Vh + 2 * c->d.Ns, st));
        CL_TRY(spec_to_phys<T>(c, W.Vh, v, st));
      }
      CL_TRY(sp_copy_reg<T>(c, W.Vh, nullptr, W.partials, st));
      CL_TRY(reduce_final_v(c, W.partials, 1, kReduceBlocks, 0.5 * o.beta * sc, W.scal + 5, st));
      CL_TRY(linearize<T>(c, mT, v, st));
      CL_TRY(diffsq_partial<T>(c, W.m + o.nt * N, mR, N, W.partials, st));
      CL_TRY(reduce_final(c, W.partials, 0.5 * cellvol(c->d), W.scal + 6, st));
      CL_TRY(gradient_spec<T>(c, mR, W.Vh, 0, st));
      rep->pde_solves += 2;
      double r3[7];
      CL_TRY(read_scalars(c, W.scal, 7, r3, st));
      gg = r3[0];
      J = r3[6] + r3[5];
    } else {
      CL_CUDA(c, cudaMemsetAsync(W.Vh, 0, sizeof(cplx<T>) * 3 * c->d.Ns, st));
    }
    rep->J0 = J;
    double gnorm = std::sqrt(gg);
    if (!std::isfinite(J) || !std::isfinite(gnorm)) {
      c->set_error("non-finite objective or gradient");
      status = CLAIRE_ENAN;
      break;
    }
    while (true) {
      if (gnorm <= o.gtol_rel * rep->gnorm0 || gnorm <= o.gtol_abs) {
        rep->converged = 1;
        break;
      }
      if (rep->gn_iters >= o.max_gn) {
        status = CLAIRE_ENOTCONV;
        break;
      }
      const double eps_H = o.pcg_rtol > 0 ? o.pcg_rtol : std::fmin(0.5, std::sqrt(gnorm / rep->gnorm0));
      if (c->coarse) {
        if (rep->gn_iters == 0) CL_TRY(coarse_template<T>(c, mT, st));
        CL_TRY(coarse_linearize<T>(c, st));
      }
      CL_TRY(pcg<T>(c, eps_H, rep, st));
      // re-project the step under div v = 0 (idempotent in exact arithmetic) and <g, vt> for the Armijo test
      CL_TRY(sp_project_dot<T>(c, W.Gh, W.VTh, W.partials, st));
      CL_TRY(reduce_final_v(c, W.partials, 1, kReduceBlocks, sc, W.scal + 7, st));
      double gvt;
      CL_TRY(read_scalars(c, W.scal + 7, 1, &gvt, st));
      double alpha = 1.0, Jt = 0.0;
      bool accepted = false;
      for (int t = 0; t < o.max_ls; ++t) {
        CL_TRY(sp_trial<T>(c, W.Vh, W.VTh, W.Vtrh, W.Sc, alpha, W.partials, st));
        CL_TRY(reduce_final_v(c, W.partials, 1, kReduceBlocks, 0.5 * o.beta * sc, W.scal + 5, st));
        CL_TRY(vec_c2r<T>(c, W.Sc, W.vtrial, st));
        CL_TRY(state_mismatch<T>(c, mT, mR, W.vtrial, 6, st));
        double r2[2];
        CL_TRY(read_scalars(c, W.scal + 5, 2, r2, st));
        Jt = r2[0] + r2[1];
        rep->ls_trials++;
        rep->pde_solves++;
        if (!std::isfinite(Jt)) {
          c->set_error("non-finite objective in the line search");
          status = CLAIRE_ENAN;
          break;
        }
        if (Jt <= J + o.armijo_c1 * alpha * gvt) {
          accepted = true;
          break;
        }
        alpha *= 0.5;
      }
      if (status != CLAIRE_OK) break;
      if (!accepted) {
        status = CLAIRE_ELINESEARCH;
        CL_TRY(sl_departure<T>(c, v, +1, W.dX, st));
        CL_TRY(update_halo<T>(c, W.dX, &c->haloX, &c->haloXh, st));
        CL_TRY(state_history<T>(c, mT, st));
        break;
      }
      std::swap(W.Vh, W.Vtrh);
      CL_CUDA(c, cudaMemcpyAsync(v, W.vtrial, sizeof(T) * n3, cudaMemcpyDeviceToDevice, st));
      // the accepted trial's state history is the state at the new v; only the adjoint solve is new
      CL_TRY(finish_linearization<T>(c, v, st));
      CL_TRY(gradient_spec<T>(c, mR, W.Vh, 0, st));
      rep->pde_solves += 1;
      J = Jt;
      CL_TRY(read_scalars(c, W.scal, 1, &gg, st));
      gnorm = std::sqrt(gg);
      rep->gn_iters++;
      if (!std::isfinite(gnorm)) {
        c->set_error("non-finite gradient norm");
        status = CLAIRE_ENAN;
        break;
      }
    }
    rep->J = J;
    rep->gnorm = gnorm;
    CL_TRY(diffsq_partial<T>(c, W.m + o.nt * N, mR, N, W.partials, st));
    CL_TRY(reduce_final(c, W.partials, 0.5 * cellvol(c->d), W.scal, st));
    CL_TRY(read_scalar(c, W.scal, &rep->mismatch, st));
  } while (false);
  CL_CUDA(c, cudaEventRecord(e1, st));
  CL_CUDA(c, cudaEventSynchronize(e1));
  float ms = 0.f;
  CL_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
  rep->ms_total = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // a staged gather whose bounded wait ran out left its outputs incomplete
  if (sizeof(T) == 4 && c->tma_steps > 0) {
    const claire_status ts = sl_tma_take_error(c);
    if (ts != CLAIRE_OK) return ts;
  }
  return status;
}

// Batched registration with every solve driven from the device: the pairs are grouped by grid; each group gets up
// to nworkers contexts with a stream each, and each context runs its share of the group as ONE graph launch (the
// pair loop of the captured solve), all launches issued before the first synchronisation. Pairs with a nonzero
// initial guess take the host-driven solve afterwards.
std::atomic<long long> g_last_batch_launches(0);

claire_status register_batch_device(const claire_opts* base, claire_pair_f32* pairs, int npairs, int nworkers) {
  g_last_batch_launches.store(0);
  std::map<std::tuple<int, int, int>, std::vector<int>> groups;
  for (int i = 0; i < npairs; ++i) groups[std::make_tuple(pairs[i].n[0], pairs[i].n[1], pairs[i].n[2])].push_back(i);
  struct Lane {
    claire_ctx* c = nullptr;
    cudaStream_t st = nullptr;
    std::vector<int> idx;
    std::vector<PairRef> tab;
    double* reports = nullptr;  // pinned
  };
  std::vector<Lane> lanes;
  std::vector<std::pair<int, int>> host_pairs;  // (pair, lane of its group) with a nonzero initial guess
  claire_status first = CLAIRE_OK;
  auto note = [&](int i, claire_status s) {
    pairs[i].status = s;
    if (s != CLAIRE_OK && s != CLAIRE_ENOTCONV && s != CLAIRE_ELINESEARCH && first == CLAIRE_OK) first = s;
  };
  for (auto& kv : groups) {
    const std::vector<int>& members = kv.second;
    const int nl = nworkers < (int)members.size() ? nworkers : (int)members.size();
    const size_t l0 = lanes.size();
    for (int w = 0; w < nl; ++w) {
      claire_opts o = *base;
      o.n[0] = std::get<0>(kv.first);
      o.n[1] = std::get<1>(kv.first);
      o.n[2] = std::get<2>(kv.first);
      Lane L;
      const claire_status cs = claire_create(&o, &L.c);
      if (cs != CLAIRE_OK) {
        for (int i : members) note(i, cs);
        break;
      }
      if (cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking) != cudaSuccess) {
        claire_destroy(L.c);
        for (int i : members) note(i, CLAIRE_ECUDA);
        break;
      }
      lanes.push_back(L);
    }
    if (lanes.size() == l0) continue;
    const int nlan = (int)(lanes.size() - l0);
    int r = 0;
    for (int i : members) {
      Lane& L = lanes[l0 + (r++ % nlan)];
      double vv = 0.0;
      const claire_status s = inner<float>(L.c, pairs[i].v, pairs[i].v, 3LL * L.c->d.N, &vv, L.st);
      if (s != CLAIRE_OK) {
        note(i, s);
      } else if (vv != 0.0) {
        host_pairs.emplace_back(i, (int)(l0 + (r - 1) % nlan));
      } else {
        L.idx.push_back(i);
        L.tab.push_back(PairRef{pairs[i].mT, pairs[i].mR, pairs[i].v});
      }
    }
  }
  for (Lane& L : lanes) {
    if (L.idx.empty()) continue;
    if (cudaMallocHost(&L.reports, sizeof(double) * kGnSlots * L.idx.size()) != cudaSuccess) {
      cudaGetLastError();
      L.reports = nullptr;
      for (int i : L.idx) note(i, CLAIRE_ENOMEM);
      L.idx.clear();
    }
  }
  // The whole batch as one graph launch: every lane's device-driven solve captured as an independent branch of one
  // graph (the lanes' branches run concurrently). CLAIRE_BATCH_GRAPH=lanes launches one graph per lane instead; so
  // does any failure to build the single graph.
  std::vector<Lane*> act;
  for (Lane& L : lanes)
    if (!L.idx.empty()) act.push_back(&L);
  const char* bg_env = std::getenv("CLAIRE_BATCH_GRAPH");
  bool one = !act.empty() && !(bg_env && std::strcmp(bg_env, "lanes") == 0);
  cudaGraph_t whole = nullptr;
  cudaGraphExec_t whole_exec = nullptr;
  cudaStream_t st0 = act.empty() ? nullptr : act.front()->st;
  if (one) {
    claire_status s = cudaGraphCreate(&whole, 0) == cudaSuccess ? CLAIRE_OK : CLAIRE_ECUDA;
    for (Lane* L : act) {
      if (s != CLAIRE_OK) break;
      s = gn_setup<float>(L->c, (int)L->idx.size(), L->st);
      if (s == CLAIRE_OK && cudaStreamSynchronize(L->st) != cudaSuccess) s = CLAIRE_ECUDA;
      if (s == CLAIRE_OK) {
        L->c->halo_fixed = true;
        cudaGraph_t unused = nullptr;
        s = gn_capture<float>(L->c, &unused, whole);
        L->c->halo_fixed = false;
      }
    }
    if (s == CLAIRE_OK && cudaGraphInstantiate(&whole_exec, whole, 0) != cudaSuccess) s = CLAIRE_ECUDA;
    for (Lane* L : act)
      if (s == CLAIRE_OK) s = gn_upload<float>(L->c, L->tab.data(), (int)L->idx.size(), st0);
    if (s == CLAIRE_OK && cudaGraphLaunch(whole_exec, st0) != cudaSuccess) s = CLAIRE_ECUDA;
    if (s == CLAIRE_OK) g_last_batch_launches.store(1);
    if (s == CLAIRE_OK) {
      for (Lane* L : act) {
        L->c->gn_graph_runs++;
        const GnBlock B = gn_block(L->c);
        if (s == CLAIRE_OK && cudaMemcpyAsync(L->reports, B.reports, sizeof(double) * kGnSlots * L->idx.size(),
                                               cudaMemcpyDeviceToHost, st0) != cudaSuccess)
          s = CLAIRE_ECUDA;
      }
    }
    if (s != CLAIRE_OK) {
      // nothing of the single graph ran (or its launch failed): per-lane launches instead
      cudaGetLastError();
      if (whole_exec) cudaGraphExecDestroy(whole_exec);
      whole_exec = nullptr;
      if (cudaStreamSynchronize(st0) != cudaSuccess) cudaGetLastError();
      one = false;
    }
  }
  if (!one) {
    g_last_batch_launches.store(0);
    for (Lane* L : act) {
      const claire_status s = gn_run<float>(L->c, L->tab.data(), (int)L->idx.size(), L->reports, L->st);
      if (s == CLAIRE_OK) g_last_batch_launches.fetch_add(1);
      if (s != CLAIRE_OK) {
        for (int i : L->idx) note(i, s);
        L->idx.clear();
      }
    }
  }
  const bool one_ok = !one || cudaStreamSynchronize(st0) == cudaSuccess;
  for (Lane& L : lanes) {
    if (!one_ok || cudaStreamSynchronize(L.st) != cudaSuccess) {
      for (int i : L.idx) note(i, CLAIRE_ECUDA);
      L.idx.clear();
    }
    for (size_t k = 0; k < L.idx.size(); ++k) {
      const int i = L.idx[k];
      note(i, gn_report(L.c, L.reports + k * kGnSlots, &pairs[i].rep));
    }
    if (!L.idx.empty() && L.c->tma_steps > 0 && sl_tma_take_error(L.c) != CLAIRE_OK)
      for (int i : L.idx) note(i, CLAIRE_ETIMEOUT);
  }
  for (auto& hp : host_pairs) {
    Lane& L = lanes[hp.second];
    claire_pair_f32& p = pairs[hp.first];
    note(hp.first, register_dev<float>(L.c, p.mT, p.mR, p.v, &p.rep, L.st));
  }
  if (whole_exec) cudaGraphExecDestroy(whole_exec);
  if (whole) cudaGraphDestroy(whole);
  for (Lane& L : lanes) {
    if (L.reports) cudaFreeHost(L.reports);
    claire_destroy(L.c);
    cudaStreamDestroy(L.st);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return CLAIRE_ECUDA;
  return first;
}

template <class T> claire_status transport_dev(claire_ctx* c, const T* m0, const T* v, int dir, T* m1,
                                               cudaStream_t st) {
  Work<T>& W = c->work<T>();
  const long long N = c->d.N;
  const int nt = c->o.nt;
  c->lin_valid = false;
  c->haloX = c->haloY = c->haloXh = c->haloYh = -1;
  T* buf[2] = {W.la, W.lb};
  if (dir > 0) {
    CL_TRY(sl_departure<T>(c, v, +1, W.dX, st));
    const T* src = m0;
    int cur = 0;
    for (int j = 0; j < nt; ++j) {
      T* dst = buf[cur];
      CL_TRY(sl_interp<T>(c, src, W.dX, dst, st));
      src = dst;
      cur = 1 - cur;
    }
    CL_CUDA(c, cudaMemcpyAsync(m1, src, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
    return CLAIRE_OK;
  }
  CL_TRY(sl_departure<T>(c, v, -1, W.dY, st));
  const T* rho = nullptr;
  T* rl[2] = {W.ra, W.rb};
  if (!c->o.divfree) {
    CL_TRY(div_spectral<T>(c, v, W.rho, st));
    rho = W.rho;
  }
  CL_CUDA(c, cudaMemcpyAsync(buf[0], m0, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
  if (rho) CL_TRY(sl_hadamard<T>(c, rho, buf[0], rl[0], st));
  int cur = 0;
  for (int j = 0; j < nt; ++j) {
    CL_TRY(sl_adjoint_step<T>(c, buf[cur], rho ? rl[cur] : nullptr, rho, W.dY, buf[1 - cur], rho ? rl[1 - cur] : nullptr,
                              nullptr, nullptr, false, T(0), st));
    cur = 1 - cur;
  }
  CL_CUDA(c, cudaMemcpyAsync(m1, buf[cur], sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
  return CLAIRE_OK;
}

template <class T> claire_status objective_dev(claire_ctx* c, const T* m1, const T* mR, const T* v, double* J,
                                               cudaStream_t st) {
  Work<T>& W = c->work<T>();
  const long long N = c->d.N;
  CL_TRY(diffsq_partial<T>(c, m1, mR, N, W.partials, st));
  CL_TRY(reduce_final(c, W.partials, 0.5 * cellvol(c->d), W.scal, st));
  CL_TRY(vec_r2c<T>(c, v, W.spec, st));
  CL_TRY(spec_reg_partial<T>(c, W.spec, W.partials, st));
  CL_TRY(reduce_final(c, W.partials, 0.5 * c->o.beta * cellvol(c->d) / double(N), W.scal + 1, st));
  CL_CUDA(c, cudaMemcpyAsync(c->hscal, W.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CL_CUDA(c, cudaStreamSynchronize(st));
  *J = c->hscal[0] + c->hscal[1];
  return CLAIRE_OK;
}

template <class T> claire_status spectral_dev(claire_ctx* c, int op, const T* in, T* out, cudaStream_t st) {
  Work<T>& W = c->work<T>();
  const Dims& d = c->d;
  cplx<T>* S = W.spec;
  switch (op) {
    case 0: return grad_spectral<T>(c, in, out, st);
    case 1: return div_spectral<T>(c, in, out, st);
    case 2: return leray_inplace<T>(c, in, out, st);
    case 3:
      if constexpr (sizeof(T) == 4) {
        if (precise_symbols<T>(c)) {
          CL_TRY(symbol_vec_f64(c, in, S, 3, 0, 1.0, st));
          return vec_c2r<T>(c, S, out, st);
        }
      }
      CL_TRY(vec_r2c<T>(c, in, S, st));
      CL_TRY(spec_scale<T>(c, S, 3, d.Ns, 0, 1.0, st));
      return vec_c2r<T>(c, S, out, st);
    case 4:
      if constexpr (sizeof(T) == 4) {
        if (precise_symbols<T>(c)) {
          CL_TRY(symbol_vec_f64(c, in, S, 1, 2, 1.0, st));
          return fft_c2r<T>(c, S, out, T(1.0 / double(d.N)), st);
        }
      }
      CL_TRY(fft_r2c<T>(c, in, S, st));
      CL_TRY(spec_scale<T>(c, S, 1, d.Ns, 2, 1.0, st));
      return fft_c2r<T>(c, S, out, T(1.0 / double(d.N)), st);
    default: c->set_error("unknown spectral op"); return CLAIRE_EINVAL;
  }
}

template <class T> bool is_prec(const claire_ctx* c);
template <> bool is_prec<float>(const claire_ctx* c) { return c->o.precision == CLAIRE_F32; }
template <> bool is_prec<double>(const claire_ctx* c) { return c->o.precision == CLAIRE_F64; }

#define CHECK_CTX(ctx, T)                                                                    \
  do {                                                                                       \
    if (!(ctx)) return CLAIRE_EINVAL;                                                        \
    if (!is_prec<T>(ctx)) {                                                                  \
      (ctx)->set_error("context precision does not match the call");                         \
      return CLAIRE_EINVAL;                                                                  \
    }                                                                                        \
  } while (0)
#define CHECK_PTR(ctx, p)                                                                    \
  do {                                                                                       \
    if (!(p)) {                                                                              \
      (ctx)->set_error("null pointer argument: " #p);                                        \
      return CLAIRE_EINVAL;                                                                  \
    }                                                                                        \
  } while (0)

template <class T> claire_status api_transport(claire_ctx* c, const T* m0, const T* v, int dir, T* m1, void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, m0);
  CHECK_PTR(c, v);
  CHECK_PTR(c, m1);
  if (dir != 1 && dir != -1) {
    c->set_error("dir must be +1 or -1");
    return CLAIRE_EINVAL;
  }
  return transport_dev<T>(c, m0, v, dir, m1, (cudaStream_t)s);
}
template <class T> claire_status api_gradient(claire_ctx* c, const T* mT, const T* mR, const T* v, T* g, double* J,
                                              void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, mT);
  CHECK_PTR(c, mR);
  CHECK_PTR(c, v);
  CHECK_PTR(c, g);
  CL_TRY(linearize<T>(c, mT, v, (cudaStream_t)s));
  return gradient_at_lin<T>(c, mR, v, g, J, (cudaStream_t)s);
}
// data term of the reduced gradient, K[int_0^1 lambda grad m dt] (Eq. (5) without beta A v); J optional
template <class T> claire_status api_gradient_data(claire_ctx* c, const T* mT, const T* mR, const T* v, T* out,
                                                   double* J, void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, mT);
  CHECK_PTR(c, mR);
  CHECK_PTR(c, v);
  CHECK_PTR(c, out);
  cudaStream_t st = (cudaStream_t)s;
  Work<T>& W = c->work<T>();
  const long long N = c->d.N;
  CL_TRY(linearize<T>(c, mT, v, st));
  if (J) {
    CL_TRY(diffsq_partial<T>(c, W.m + c->o.nt * N, mR, N, W.partials, st));
    CL_TRY(reduce_final(c, W.partials, 0.5 * cellvol(c->d), W.scal, st));
    CL_TRY(vec_r2c<T>(c, v, W.spec, st));
    CL_TRY(spec_reg_partial<T>(c, W.spec, W.partials, st));
    CL_TRY(reduce_final(c, W.partials, 0.5 * c->o.beta * cellvol(c->d) / double(N), W.scal + 1, st));
  }
  CL_TRY(adjoint_integral<T>(c, mR, st));
  CL_CUDA(c, cudaMemsetAsync(out, 0, sizeof(T) * 3 * N, st));
  CL_TRY(add_projected_b<T>(c, out, out, st));
  if (J) {
    double r2[2];
    CL_TRY(read_scalars(c, W.scal, 2, r2, st));
    *J = r2[0] + r2[1];
  }
  return CLAIRE_OK;
}
// a diagonal Fourier symbol of the method on ncomp half spectra: 0 beta A, 1 M^-1, 2 K (ncomp = 3)
template <class T> claire_status api_symbol(claire_ctx* c, int op, const T* in, T* out, int ncomp, void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, in);
  CHECK_PTR(c, out);
  if (op < 0 || op > 2 || ncomp < 1 || ncomp > 3 || (op == 2 && ncomp != 3)) {
    c->set_error("claire_symbol: op must be 0, 1 or 2, 1 <= ncomp <= 3, and ncomp = 3 for K");
    return CLAIRE_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)s;
  const long long Ns = c->d.Ns;
  cplx<T>* V = reinterpret_cast<cplx<T>*>(out);
  if ((const void*)in != (const void*)out)
    CL_CUDA(c, cudaMemcpyAsync(out, in, sizeof(cplx<T>) * ncomp * Ns, cudaMemcpyDeviceToDevice, st));
  if (op == 2) return spec_kop<T>(c, V, V + Ns, V + 2 * Ns, st);
  return spec_scale<T>(c, V, ncomp, Ns, op == 0 ? 0 : 1, c->o.beta, st);
}
template <class T> claire_status api_linearize(claire_ctx* c, const T* mT, const T* v, void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, mT);
  CHECK_PTR(c, v);
  return linearize<T>(c, mT, v, (cudaStream_t)s);
}
template <class T> claire_status api_hessvec_cached(claire_ctx* c, const T* vt, T* Hvt, void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, vt);
  CHECK_PTR(c, Hvt);
  if (!c->lin_valid) {
    c->set_error("no cached linearisation");
    return CLAIRE_EINVAL;
  }
  if ((const void*)vt == (const void*)Hvt) {
    c->set_error("vt and Hvt must not alias");
    return CLAIRE_EINVAL;
  }
  return hessvec_at_lin<T>(c, vt, Hvt, (cudaStream_t)s);
}
template <class T> claire_status api_hessvec_data(claire_ctx* c, const T* vt, T* out, void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, vt);
  CHECK_PTR(c, out);
  if (!c->lin_valid) {
    c->set_error("no cached linearisation");
    return CLAIRE_EINVAL;
  }
  if ((const void*)vt == (const void*)out) {
    c->set_error("vt and out must not alias");
    return CLAIRE_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)s;
  CL_CUDA(c, cudaMemsetAsync(out, 0, sizeof(T) * 3 * c->d.N, st));
  CL_TRY(hess_data<T>(c, vt, st));
  return add_projected_b<T>(c, out, out, st);
}
template <class T> claire_status api_hessvec(claire_ctx* c, const T* mT, const T* v, const T* vt, T* Hvt, void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, mT);
  CHECK_PTR(c, v);
  CL_TRY(linearize<T>(c, mT, v, (cudaStream_t)s));
  return api_hessvec_cached<T>(c, vt, Hvt, s);
}
template <class T> claire_status api_precond(claire_ctx* c, const T* r, T* z, void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, r);
  CHECK_PTR(c, z);
  return precond_apply<T>(c, r, z, (cudaStream_t)s);
}
template <class T> claire_status api_register(claire_ctx* c, const T* mT, const T* mR, T* v, claire_report* rep,
                                              void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, mT);
  CHECK_PTR(c, mR);
  CHECK_PTR(c, v);
  claire_report local;
  return register_dev<T>(c, mT, mR, v, rep ? rep : &local, (cudaStream_t)s);
}
// Parameter continuation in beta_v (Sec. 3.6): levels beta_start, beta_start f, beta_start f^2, ... while above the
// context's beta_v, then beta_v itself; each level is a full solve warm-started from the previous level's v.
template <class T> claire_status api_register_continuation(claire_ctx* c, const T* mT, const T* mR, T* v,
                                                           double beta_start, double factor, claire_report* reps,
                                                           int max_levels, int* nlevels, void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, mT);
  CHECK_PTR(c, mR);
  CHECK_PTR(c, v);
  if (!(beta_start > 0.0) || !(factor > 0.0 && factor < 1.0) || max_levels < 1) {
    c->set_error("continuation needs beta_start > 0, 0 < factor < 1 and max_levels >= 1");
    return CLAIRE_EINVAL;
  }
  const double target = c->o.beta;
  std::vector<double> betas;
  for (double b = beta_start; b > target * (1.0 + 1e-12) && (int)betas.size() < max_levels - 1; b *= factor)
    betas.push_back(b);
  betas.push_back(target);
  claire_status st = CLAIRE_OK;
  int done = 0;
  for (double b : betas) {
    c->o.beta = b;
    if (c->coarse) c->coarse->o.beta = b;
    claire_report local;
    claire_report* r = reps ? reps + done : &local;
    st = register_dev<T>(c, mT, mR, v, r, (cudaStream_t)s);
    ++done;
    if (st != CLAIRE_OK && st != CLAIRE_ENOTCONV) break;
  }
  c->o.beta = target;
  if (c->coarse) c->coarse->o.beta = target;
  if (nlevels) *nlevels = done;
  return st;
}

template <class T> claire_status api_register_host(claire_ctx* c, const T* mT, const T* mR, T* v, claire_report* rep,
                                                   void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, mT);
  CHECK_PTR(c, mR);
  CHECK_PTR(c, v);
  Work<T>& W = c->work<T>();
  cudaStream_t st = (cudaStream_t)s;
  const long long N = c->d.N;
  CL_TRY(ensure_hostbuf<T>(c));  // device copies of m_T, m_R and v, allocated on first use (kept until destroy)
  CL_CUDA(c, cudaMemcpyAsync(W.mTdev, mT, sizeof(T) * N, cudaMemcpyHostToDevice, st));
  CL_CUDA(c, cudaMemcpyAsync(W.mRdev, mR, sizeof(T) * N, cudaMemcpyHostToDevice, st));
  CL_CUDA(c, cudaMemcpyAsync(W.vdev, v, sizeof(T) * 3 * N, cudaMemcpyHostToDevice, st));
  claire_report local;
  claire_status stat = register_dev<T>(c, W.mTdev, W.mRdev, W.vdev, rep ? rep : &local, st);
  if (stat != CLAIRE_OK && stat != CLAIRE_ENOTCONV && stat != CLAIRE_ELINESEARCH) return stat;
  CL_CUDA(c, cudaMemcpyAsync(v, W.vdev, sizeof(T) * 3 * N, cudaMemcpyDeviceToHost, st));
  CL_CUDA(c, cudaStreamSynchronize(st));
  return stat;
}
template <class T> claire_status api_departure(claire_ctx* c, const T* v, int dir, T* disp, void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, v);
  CHECK_PTR(c, disp);
  if (dir != 1 && dir != -1) {
    c->set_error("dir must be +1 or -1");
    return CLAIRE_EINVAL;
  }
  return sl_departure<T>(c, v, dir, disp, (cudaStream_t)s);
}
template <class T> claire_status api_interp(claire_ctx* c, const T* f, const T* disp, T* out, void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, f);
  CHECK_PTR(c, disp);
  CHECK_PTR(c, out);
  return sl_interp<T>(c, f, disp, out, (cudaStream_t)s);
}
template <class T> claire_status api_spectral(claire_ctx* c, int op, const T* in, T* out, void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, in);
  CHECK_PTR(c, out);
  return spectral_dev<T>(c, op, in, out, (cudaStream_t)s);
}
template <class T> claire_status api_objective(claire_ctx* c, const T* m1, const T* mR, const T* v, double* J,
                                               void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, m1);
  CHECK_PTR(c, mR);
  CHECK_PTR(c, v);
  CHECK_PTR(c, J);
  return objective_dev<T>(c, m1, mR, v, J, (cudaStream_t)s);
}
template <class T> claire_status api_dot(claire_ctx* c, const T* a, const T* b, long long n, double* out, void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, a);
  CHECK_PTR(c, b);
  CHECK_PTR(c, out);
  if (n < 0) {
    c->set_error("negative count");
    return CLAIRE_EINVAL;
  }
  return inner<T>(c, a, b, n, out, (cudaStream_t)s);
}
template <class T> claire_status api_fft(claire_ctx* c, const T* f, T* spec, void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, f);
  CHECK_PTR(c, spec);
  return fft_r2c<T>(c, f, reinterpret_cast<cplx<T>*>(spec), (cudaStream_t)s);
}
template <class T> claire_status api_ifft(claire_ctx* c, const T* spec, T* f, void* s) {
  CHECK_CTX(c, T);
  CHECK_PTR(c, spec);
  CHECK_PTR(c, f);
  Work<T>& W = c->work<T>();
  CL_CUDA(c, cudaMemcpyAsync(W.spec, spec, sizeof(cplx<T>) * c->d.Ns, cudaMemcpyDeviceToDevice, (cudaStream_t)s));
  return fft_c2r<T>(c, W.spec, f, T(1.0 / double(c->d.N)), (cudaStream_t)s);
}

}  // namespace

// =================================================================================================================
extern "C" {

claire_status claire_default_opts(claire_opts* o, int n1, int n2, int n3, int precision) {
  if (!o) return CLAIRE_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->n[0] = n1;
  o->n[1] = n2;
  o->n[2] = n3;
  o->precision = precision;
  o->beta = 1e-2;
  o->nt = 4;
  o->regnorm = 1;
  o->divfree = 0;
  o->gtol_rel = 5e-2;
  o->gtol_abs = 1e-6;
  o->max_gn = 50;
  o->max_krylov = 100;
  o->pcg_rtol = 0.0;
  o->max_ls = 10;
  o->armijo_c1 = 1e-4;
  o->pc_kappa = 0.1;
  return CLAIRE_OK;
}

namespace {
claire_status create_ctx(const claire_opts* opts, bool coarse, claire_ctx** out);
}

claire_status claire_create(const claire_opts* opts, claire_ctx** out) { return create_ctx(opts, false, out); }

namespace {
claire_status create_ctx(const claire_opts* opts, bool coarse, claire_ctx** out) {
  if (!opts || !out) return CLAIRE_EINVAL;
  *out = nullptr;
  const claire_opts& o = *opts;
  for (int a = 0; a < 3; ++a)
    if (o.n[a] < 4 || (o.n[a] & 1)) return CLAIRE_EINVAL;
  if (o.nt < 1 || !(o.beta > 0) || (o.regnorm != 1 && o.regnorm != 2) || (o.divfree != 0 && o.divfree != 1) ||
      (o.precision != CLAIRE_F32 && o.precision != CLAIRE_F64) || o.max_gn < 0 || o.max_krylov < 1 || o.max_ls < 1)
    return CLAIRE_EINVAL;
  const long long N = (long long)o.n[0] * o.n[1] * o.n[2];
  // 32-bit node indices in the kernels and the launch grid's z extent (one i1 slab per grid z index)
  if (N > (1LL << 31) - 1 || o.n[0] > 65535) return CLAIRE_EINVAL;
  if (o.bf16_mask < 0 || o.bf16_mask > 1 || (o.bf16_mask && o.precision != CLAIRE_F32)) return CLAIRE_EINVAL;
  if (!(o.beta_w >= 0.0) || (o.beta_w > 0.0 && (o.divfree || o.regnorm != 1))) return CLAIRE_EINVAL;
  if (o.precond != 0 && o.precond != 1) return CLAIRE_EINVAL;
  if (o.precond == 1) {
    for (int a = 0; a < 3; ++a)
      if (o.n[a] % 4 || o.n[a] < 8) return CLAIRE_EINVAL;
    if (!(o.pc_kappa > 0.0 && o.pc_kappa < 1.0)) return CLAIRE_EINVAL;
  }
  claire_ctx* c = new (std::nothrow) claire_ctx();
  if (!c) return CLAIRE_ENOMEM;
  c->o = o;
  c->is_coarse = coarse;
  c->gm16_on = (o.bf16_mask & 1) != 0;
  c->d.n1 = o.n[0];
  c->d.n2 = o.n[1];
  c->d.n3 = o.n[2];
  c->d.n3h = o.n[2] / 2 + 1;
  c->d.N = N;
  c->d.Ns = (long long)o.n[0] * o.n[1] * c->d.n3h;
  c->d.by_n3h = FastDiv((unsigned)c->d.n3h);
  c->d.by_n2 = FastDiv((unsigned)o.n[1]);
  RadixPlan tmp;
  if (!radix_plan(o.n[0], tmp) || !radix_plan(o.n[1], tmp) || !radix_plan(o.n[2] / 2, tmp)) {
    delete c;
    return CLAIRE_EINVAL;
  }
  const size_t bytes =
      o.precision == CLAIRE_F32 ? work_bytes<float>(o, c->d, coarse) : work_bytes<double>(o, c->d, coarse);
  if (cudaMalloc(&c->arena, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return CLAIRE_ENOMEM;
  }
  c->arena_bytes = bytes;
  if (cudaMallocHost(&c->hscal, 128 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->arena);
    delete c;
    return CLAIRE_ENOMEM;
  }
  claire_status s = o.precision == CLAIRE_F32 ? fft_init<float>(c) : fft_init<double>(c);
  if (s == CLAIRE_OK && o.precision == CLAIRE_F32) {
    // an FP64 plan for the stand-alone operators; where the FP64 passes do not fit (very long axes), those
    // operators transform in FP32 instead
    c->f64_plan = fft_init<double>(c) == CLAIRE_OK;
    if (!c->f64_plan) c->err.clear();
  }
  if (s == CLAIRE_OK) s = o.precision == CLAIRE_F32 ? sl_init<float>(c) : sl_init<double>(c);
  if (s == CLAIRE_OK) s = o.precision == CLAIRE_F32 ? alloc_work<float>(c) : alloc_work<double>(c);
  if (s == CLAIRE_OK && o.precision == CLAIRE_F32) s = fft_tune<float>(c);
  if (s != CLAIRE_OK) {
    cudaFreeHost(c->hscal);
    cudaFree(c->arena);
    delete c;
    return s;
  }
  if (o.precond == 1) {
    // the half-resolution problem of the two-level preconditioner: same model, spectral preconditioner
    claire_opts oc = o;
    for (int a = 0; a < 3; ++a) oc.n[a] = o.n[a] / 2;
    oc.precond = 0;
    s = create_ctx(&oc, true, &c->coarse);
    if (s != CLAIRE_OK) {
      c->coarse = nullptr;
      claire_destroy(c);
      return s;
    }
  }
  *out = c;
  return CLAIRE_OK;
}
}  // namespace

claire_status claire_profile_enable(claire_ctx* c, int on) {
  if (!c) return CLAIRE_EINVAL;
  c->prof_on = on != 0;
  if (c->coarse) c->coarse->prof_on = on != 0;
  return CLAIRE_OK;
}

claire_status claire_profile_report(claire_ctx* c, char* buf, size_t len) {
  if (!c || !buf || len == 0) return CLAIRE_EINVAL;
  CL_CUDA(c, cudaDeviceSynchronize());
  std::map<std::string, std::pair<long long, double>> agg;
  for (claire_ctx* x : {c, c->coarse}) {
    if (!x) continue;
    for (auto& r : x->prof_recs) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) ms = 0.f;
      auto& e = agg[std::string(x == c ? "" : "coarse:") + r.name];
      e.first += 1;
      e.second += ms;
      x->prof_pool.push_back(r.a);
      x->prof_pool.push_back(r.b);
    }
    x->prof_recs.clear();
  }
  std::string out = "{";
  bool first = true;
  for (auto& kv : agg) {
    char tmp[256];
    std::snprintf(tmp, sizeof(tmp), "%s\"%s\": [%lld, %.6f]", first ? "" : ", ", kv.first.c_str(), kv.second.first,
                  kv.second.second);
    out += tmp;
    first = false;
  }
  out += "}";
  std::strncpy(buf, out.c_str(), len - 1);
  buf[len - 1] = 0;
  return CLAIRE_OK;
}

claire_status claire_destroy(claire_ctx* c) {
  if (!c) return CLAIRE_OK;
  cudaDeviceSynchronize();
  if (c->coarse) claire_destroy(c->coarse);
  if (c->pcg_exec) cudaGraphExecDestroy(c->pcg_exec);
  if (c->pcg_graph) cudaGraphDestroy(c->pcg_graph);
  if (c->pcg_cap_stream) cudaStreamDestroy(c->pcg_cap_stream);
  gn_graph_release(c);
  if (c->gn_dev) cudaFree(c->gn_dev);
  for (cudaStream_t s : c->gn_cap_streams)
    if (s) cudaStreamDestroy(s);
  for (auto& r : c->prof_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->prof_pool) cudaEventDestroy(e);
  if (c->arena) cudaFree(c->arena);
  if (c->hostbuf) cudaFree(c->hostbuf);
  if (c->hscal) cudaFreeHost(c->hscal);
  delete c;
  return CLAIRE_OK;
}

const char* claire_last_error(const claire_ctx* c) { return c ? c->err.c_str() : "null context"; }

size_t claire_workspace_bytes(const claire_ctx* c) {
  return c ? c->arena_bytes + (c->coarse ? c->coarse->arena_bytes : 0) : 0;
}

claire_status claire_get_counters(const claire_ctx* c, claire_counters* out) {
  if (!c || !out) return CLAIRE_EINVAL;
  out->launches = c->counters.launches + (c->coarse ? c->coarse->counters.launches : 0);
  out->halo_x = c->haloX;
  out->halo_y = c->haloY;
  out->halo_x_heavy = c->haloXh;
  out->halo_y_heavy = c->haloYh;
  out->pcg_graph_runs = c->pcg_graph_runs;
  out->tma_steps = c->tma_steps + (c->coarse ? c->coarse->tma_steps : 0);
  out->gn_graph_runs = c->gn_graph_runs;
  const auto& fp = c->pf;  // (FP64 passes have no tile variants)
  out->fft_tile[0] = fp.var_z;
  out->fft_tile[1] = fp.var_y;
  out->fft_tile[2] = fp.var_x;
  return CLAIRE_OK;
}

claire_status claire_transport_f32(claire_ctx* c, const float* m0, const float* v, int dir, float* m1, void* s) {
  return api_transport<float>(c, m0, v, dir, m1, s);
}
claire_status claire_transport_f64(claire_ctx* c, const double* m0, const double* v, int dir, double* m1, void* s) {
  return api_transport<double>(c, m0, v, dir, m1, s);
}
claire_status claire_gradient_f32(claire_ctx* c, const float* mT, const float* mR, const float* v, float* g, double* J,
                                  void* s) {
  return api_gradient<float>(c, mT, mR, v, g, J, s);
}
claire_status claire_gradient_f64(claire_ctx* c, const double* mT, const double* mR, const double* v, double* g,
                                  double* J, void* s) {
  return api_gradient<double>(c, mT, mR, v, g, J, s);
}
claire_status claire_hessvec_f32(claire_ctx* c, const float* mT, const float* mR, const float* v, const float* vt,
                                 float* Hvt, void* s) {
  (void)mR;
  return api_hessvec<float>(c, mT, v, vt, Hvt, s);
}
claire_status claire_hessvec_f64(claire_ctx* c, const double* mT, const double* mR, const double* v, const double* vt,
                                 double* Hvt, void* s) {
  (void)mR;
  return api_hessvec<double>(c, mT, v, vt, Hvt, s);
}
claire_status claire_hessvec_cached_f32(claire_ctx* c, const float* vt, float* Hvt, void* s) {
  return api_hessvec_cached<float>(c, vt, Hvt, s);
}
claire_status claire_hessvec_cached_f64(claire_ctx* c, const double* vt, double* Hvt, void* s) {
  return api_hessvec_cached<double>(c, vt, Hvt, s);
}
claire_status claire_hessvec_data_f32(claire_ctx* c, const float* vt, float* out, void* s) {
  return api_hessvec_data<float>(c, vt, out, s);
}
claire_status claire_hessvec_data_f64(claire_ctx* c, const double* vt, double* out, void* s) {
  return api_hessvec_data<double>(c, vt, out, s);
}
claire_status claire_gradient_data_f32(claire_ctx* c, const float* mT, const float* mR, const float* v, float* out,
                                       double* J, void* s) {
  return api_gradient_data<float>(c, mT, mR, v, out, J, s);
}
claire_status claire_gradient_data_f64(claire_ctx* c, const double* mT, const double* mR, const double* v,
                                       double* out, double* J, void* s) {
  return api_gradient_data<double>(c, mT, mR, v, out, J, s);
}
claire_status claire_symbol_f32(claire_ctx* c, int op, const float* in, float* out, int ncomp, void* s) {
  return api_symbol<float>(c, op, in, out, ncomp, s);
}
claire_status claire_symbol_f64(claire_ctx* c, int op, const double* in, double* out, int ncomp, void* s) {
  return api_symbol<double>(c, op, in, out, ncomp, s);
}
claire_status claire_linearize_f32(claire_ctx* c, const float* mT, const float* v, void* s) {
  return api_linearize<float>(c, mT, v, s);
}
claire_status claire_linearize_f64(claire_ctx* c, const double* mT, const double* v, void* s) {
  return api_linearize<double>(c, mT, v, s);
}
claire_status claire_precond_f32(claire_ctx* c, const float* r, float* z, void* s) {
  return api_precond<float>(c, r, z, s);
}
claire_status claire_precond_f64(claire_ctx* c, const double* r, double* z, void* s) {
  return api_precond<double>(c, r, z, s);
}
claire_status claire_register_f32(claire_ctx* c, const float* mT, const float* mR, float* v, claire_report* rep,
                                  void* s) {
  return api_register<float>(c, mT, mR, v, rep, s);
}
claire_status claire_register_f64(claire_ctx* c, const double* mT, const double* mR, double* v, claire_report* rep,
                                  void* s) {
  return api_register<double>(c, mT, mR, v, rep, s);
}
claire_status claire_register_continuation_f32(claire_ctx* c, const float* mT, const float* mR, float* v,
                                               double beta_start, double factor, claire_report* reps,
                                               int max_levels, int* nlevels, void* s) {
  return api_register_continuation<float>(c, mT, mR, v, beta_start, factor, reps, max_levels, nlevels, s);
}
claire_status claire_register_continuation_f64(claire_ctx* c, const double* mT, const double* mR, double* v,
                                               double beta_start, double factor, claire_report* reps,
                                               int max_levels, int* nlevels, void* s) {
  return api_register_continuation<double>(c, mT, mR, v, beta_start, factor, reps, max_levels, nlevels, s);
}
claire_status claire_set_beta(claire_ctx* c, double beta) {
  if (!c || !(beta > 0.0)) return CLAIRE_EINVAL;
  c->o.beta = beta;
  if (c->coarse) c->coarse->o.beta = beta;
  return CLAIRE_OK;
}
claire_status claire_register_host_f32(claire_ctx* c, const float* mT, const float* mR, float* v, claire_report* rep,
                                       void* s) {
  return api_register_host<float>(c, mT, mR, v, rep, s);
}
claire_status claire_register_host_f64(claire_ctx* c, const double* mT, const double* mR, double* v,
                                       claire_report* rep, void* s) {
  return api_register_host<double>(c, mT, mR, v, rep, s);
}
long long claire_last_batch_graph_launches(void) { return g_last_batch_launches.load(); }

claire_status claire_register_batch_f32(const claire_opts* base, claire_pair_f32* pairs, int npairs, int nworkers) {
  if (!base || (!pairs && npairs > 0) || npairs < 0 || nworkers < 1) return CLAIRE_EINVAL;
  g_last_batch_launches.store(0);
  if (base->precision != CLAIRE_F32) return CLAIRE_EINVAL;
  for (int i = 0; i < npairs; ++i)
    if (!pairs[i].mT || !pairs[i].mR || !pairs[i].v) return CLAIRE_EINVAL;
  {
    const char* gm = std::getenv("CLAIRE_GN");
    if (!(gm && std::strcmp(gm, "host") == 0) && base->precond == 0) return register_batch_device(base, pairs, npairs, nworkers);
  }
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return CLAIRE_ECUDA;
  // largest grids first (longest-processing-time order over the workers)
  std::vector<int> order(npairs);
  for (int i = 0; i < npairs; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const long long na = (long long)pairs[a].n[0] * pairs[a].n[1] * pairs[a].n[2];
    const long long nb = (long long)pairs[b].n[0] * pairs[b].n[1] * pairs[b].n[2];
    return na > nb;
  });
  std::atomic<int> next(0);
  std::atomic<int> first_error(0);
  auto worker = [&]() {
    if (cudaSetDevice(device) != cudaSuccess) {
      first_error.store(CLAIRE_ECUDA);
      return;
    }
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      first_error.store(CLAIRE_ECUDA);
      return;
    }
    std::map<std::tuple<int, int, int>, claire_ctx*> ctxs;
    for (int k = next.fetch_add(1); k < npairs; k = next.fetch_add(1)) {
      claire_pair_f32& p = pairs[order[k]];
      const auto key = std::make_tuple(p.n[0], p.n[1], p.n[2]);
      claire_ctx* c = nullptr;
      auto it = ctxs.find(key);
      if (it != ctxs.end()) {
        c = it->second;
      } else {
        claire_opts o = *base;
        o.n[0] = p.n[0];
        o.n[1] = p.n[1];
        o.n[2] = p.n[2];
        const claire_status cs = claire_create(&o, &c);
        if (cs != CLAIRE_OK) {
          p.status = cs;
          int zero = 0;
          first_error.compare_exchange_strong(zero, (int)cs);
          continue;
        }
        ctxs[key] = c;
      }
      const claire_status rs = register_dev<float>(c, p.mT, p.mR, p.v, &p.rep, st);
      p.status = rs;
      if (rs != CLAIRE_OK && rs != CLAIRE_ENOTCONV && rs != CLAIRE_ELINESEARCH) {
        int zero = 0;
        first_error.compare_exchange_strong(zero, (int)rs);
      }
    }
    cudaStreamSynchronize(st);
    for (auto& kv : ctxs) {
      // the context's own destroy synchronises the whole device; free its memory directly instead
      claire_ctx* c = kv.second;
      for (auto& r : c->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
      }
      for (auto e : c->prof_pool) cudaEventDestroy(e);
      cudaFree(c->arena);
      if (c->hostbuf) cudaFree(c->hostbuf);
      cudaFreeHost(c->hscal);
      delete c;
    }
    cudaStreamDestroy(st);
  };
  std::vector<std::thread> threads;
  const int nw = nworkers < npairs ? nworkers : (npairs > 0 ? npairs : 1);
  for (int w = 0; w < nw; ++w) threads.emplace_back(worker);
  for (auto& t : threads) t.join();
  if (cudaDeviceSynchronize() != cudaSuccess) return CLAIRE_ECUDA;
  return (claire_status)first_error.load();
}

claire_status claire_departure_f32(claire_ctx* c, const float* v, int dir, float* disp, void* s) {
  return api_departure<float>(c, v, dir, disp, s);
}
claire_status claire_departure_f64(claire_ctx* c, const double* v, int dir, double* disp, void* s) {
  return api_departure<double>(c, v, dir, disp, s);
}
claire_status claire_interp_f32(claire_ctx* c, const float* f, const float* disp, float* out, void* s) {
  return api_interp<float>(c, f, disp, out, s);
}
claire_status claire_interp_f64(claire_ctx* c, const double* f, const double* disp, double* out, void* s) {
  return api_interp<double>(c, f, disp, out, s);
}
claire_status claire_spectral_f32(claire_ctx* c, int op, const float* in, float* out, void* s) {
  return api_spectral<float>(c, op, in, out, s);
}
claire_status claire_spectral_f64(claire_ctx* c, int op, const double* in, double* out, void* s) {
  return api_spectral<double>(c, op, in, out, s);
}
claire_status claire_objective_f32(claire_ctx* c, const float* m1, const float* mR, const float* v, double* J,
                                   void* s) {
  return api_objective<float>(c, m1, mR, v, J, s);
}
claire_status claire_objective_f64(claire_ctx* c, const double* m1, const double* mR, const double* v, double* J,
                                   void* s) {
  return api_objective<double>(c, m1, mR, v, J, s);
}
claire_status claire_dot_f32(claire_ctx* c, const float* a, const float* b, long long n, double* out, void* s) {
  return api_dot<float>(c, a, b, n, out, s);
}
claire_status claire_dot_f64(claire_ctx* c, const double* a, const double* b, long long n, double* out, void* s) {
  return api_dot<double>(c, a, b, n, out, s);
}
claire_status claire_fft_f32(claire_ctx* c, const float* f, float* spec, void* s) { return api_fft<float>(c, f, spec, s); }
claire_status claire_fft_f64(claire_ctx* c, const double* f, double* spec, void* s) {
  return api_fft<double>(c, f, spec, s);
}
claire_status claire_ifft_f32(claire_ctx* c, const float* spec, float* f, void* s) {
  return api_ifft<float>(c, spec, f, s);
}
claire_status claire_ifft_f64(claire_ctx* c, const double* spec, double* f, void* s) {
  return api_ifft<double>(c, spec, f, s);
}

}  // extern "C"
