// Semi-Lagrangian transport kernels (Sec. 2.3.1, Sec. 3.4): RK2 characteristics and tricubic Lagrange gathers.
//
// One thread per grid node. The departure point of node i is xi = i + disp (grid units); per axis the stencil is
// b - 1 .. b + 2 with b = i + floor(disp) and t = disp - floor(disp) (splitting off the integer node index keeps
// t accurate in FP32 on large grids), the four cubic Lagrange weights on the nodes -1, 0, 1, 2 and periodic wrap.
// The 64-tap sum is evaluated separably (16 four-tap sums along i3, 4 along i2, 1 along i1: 84 FMA). Source
// terms and the time-integral accumulation of the adjoints (Sec. 3.5, memory-reduced Gauss-Newton) are fused
// into the epilogue of the gather so each step streams its fields once.
#include "sl_kernels.cuh"

namespace claire {

// the tiled FP32 launchers live in sl_h<H>.cu (FP32 gradient history) and sl_h<H>_bf16.cu (BF16 history)
CLAIRE_SL_LAUNCHERS(extern, float, 2)
CLAIRE_SL_LAUNCHERS(extern, float, 3)
CLAIRE_SL_LAUNCHERS(extern, float, 4)
CLAIRE_SL_LAUNCHERS(extern, float, 5)
CLAIRE_SL_LAUNCHERS_G(extern, float, 2, __nv_bfloat16)
CLAIRE_SL_LAUNCHERS_G(extern, float, 3, __nv_bfloat16)
CLAIRE_SL_LAUNCHERS_G(extern, float, 4, __nv_bfloat16)
CLAIRE_SL_LAUNCHERS_G(extern, float, 5, __nv_bfloat16)

// Calls f(g) with g a typed pointer to the gradient history: T, or BF16 when g16 (FP32 only).
template <class T, class F> static void with_gm(const void* gm, bool g16, F&& f) {
  if constexpr (sizeof(T) == 4) {
    if (g16) {
      f(static_cast<const __nv_bfloat16*>(gm));
      return;
    }
  }
  f(static_cast<const T*>(gm));
}

static inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// 3D launch shape of the gather kernels: 256 threads, x along i3 (32 wide: one warp per row), y along i2 (8 rows,
// whose stencils share 3 of their 4 tap rows in L1), z = i1. Measured at 256^3 against 64 x 4: 2-3% faster.
Launch3 launch3(const Dims& d) {
  const int bx = d.n3 >= 32 ? 32 : 16;
  const int by = 256 / bx;
  Launch3 L;
  L.block = dim3(bx, by, 1);
  L.grid = dim3((d.n3 + bx - 1) / bx, (d.n2 + by - 1) / by, d.n1);
  return L;
}

template <class T> claire_status sl_departure(claire_ctx* c, const T* v, int dir, T* disp, cudaStream_t st) {
  const Dims& d = c->d;
  const double dt = 1.0 / c->o.nt;
  const double twopi = 6.283185307179586476925286766559;
  const T ih1 = T(d.n1 / twopi), ih2 = T(d.n2 / twopi), ih3 = T(d.n3 / twopi);
  c->prof_begin("sl_departure", st);
  const Launch3 L = launch3(d);
  k_departure<T><<<L.grid, L.block, 0, st>>>(v, disp, T(dir * dt), ih1, ih2, ih3, d);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

// Calls f(std::integral_constant<int, Hc>) with Hc the compile-time halo (-1: plain gathers). Only FP32 has
// tiled instantiations (the FP64 path is bound by the FP64 pipe, not by the gathers' memory traffic).
template <class T, class F> static void with_halo(int H, F&& f) {
  if constexpr (sizeof(T) == 4) {
    switch (H) {
      case 2: f(std::integral_constant<int, 2>()); return;
      case 3: f(std::integral_constant<int, 3>()); return;
      case 4: f(std::integral_constant<int, 4>()); return;
      case 5: f(std::integral_constant<int, 5>()); return;
      default: break;
    }
  }
  f(std::integral_constant<int, -1>());
}

template <class T>
claire_status sl_interp(claire_ctx* c, const T* f, const T* disp, T* out, cudaStream_t st, int H) {
  const int h = tile_halo<T>(H);
  c->prof_begin(h >= 0 ? "sl_interp_tiled" : "sl_interp", st);
  with_halo<T>(h, [&](auto hc) { sl_launch_interp<T, decltype(hc)::value>(f, disp, out, c->d, st); });
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

template <class T>
claire_status sl_adjoint_terminal(claire_ctx* c, const T* mR, const T* m1, const T* rho, T* lam, T* rl, T* b,
                                  const void* gmj, bool g16, T w, cudaStream_t st) {
  c->prof_begin(rho ? "sl_adj_terminal_rho" : "sl_adj_terminal", st);
  with_gm<T>(gmj, g16, [&](auto g) {
    using G = std::remove_const_t<std::remove_pointer_t<decltype(g)>>;
    if (rho)
      k_adj_terminal<T, true, G><<<blocks_for(c->d.N), kThreads, 0, st>>>(mR, m1, rho, lam, rl, b, g, w, c->d);
    else
      k_adj_terminal<T, false, G><<<blocks_for(c->d.N), kThreads, 0, st>>>(mR, m1, rho, lam, rl, b, g, w, c->d);
  });
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

template <class T>
claire_status sl_adjoint_step(claire_ctx* c, const T* lam_next, const T* rl_next, const T* rho, const T* dY, T* lam,
                              T* rl, T* b, const void* gmj, bool g16, T w, cudaStream_t st, const T* sdot, double* part,
                              int H) {
  const T dt = T(1.0 / c->o.nt);
  const bool dot = sdot != nullptr && b != nullptr && lam == nullptr;
  const int key = (rho ? 4 : 0) | (lam ? 2 : 0) | (b ? 1 : 0);
  static const char* names[8] = {"sl_adj_step", "sl_adj_step_acc", "sl_adj_step_store", "sl_adj_step_store_acc",
                                 "sl_adj_step_rho", "sl_adj_step_rho_acc", "sl_adj_step_rho_store",
                                 "sl_adj_step_rho_store_acc"};
  c->prof_begin(dot ? (rho ? "sl_adj_step_rho_acc_dot" : "sl_adj_step_acc_dot") : names[key], st);
  if (!b) {
    // transport without accumulation (claire_transport): plain gathers
    dim3 grid, block;
    tiled_shape<-1>(c->d, grid, block);
#define ADJ_PLAIN(R, S)                                                                                          \
  k_adj_step<T, R, S, false, false, -1, T><<<grid, block, 0, st>>>(lam_next, rl_next, rho, dY, lam, rl, b,       \
                                                                   (const T*)nullptr, w, dt, c->d, sdot, part)
    if (rho) {
      if (lam)
        ADJ_PLAIN(true, true);
      else
        ADJ_PLAIN(true, false);
    } else {
      if (lam)
        ADJ_PLAIN(false, true);
      else
        ADJ_PLAIN(false, false);
    }
#undef ADJ_PLAIN
  } else {
    const int h = tile_halo<T>(H);
    if constexpr (sizeof(T) == 4) {
      // the accumulating step on the context's own arrays with bricks: its streamed operands staged by TMA. The
      // step with the fused <s, b~> keeps per-thread loads: with the staged operands' shared memory it would run
      // three CTAs per SM instead of four (measured at 256^3: 325 us against 310 us)
      Work<float>& W = c->work<float>();
      const void* gbase = g16 ? W.gm16 : (const void*)W.gm;
      const char* tma_env = std::getenv("CLAIRE_TMA");
      const bool own = b == W.b && dY == W.dY && rho == nullptr && !dot && gbase;
      if (h >= 2 && own && !(tma_env && std::strcmp(tma_env, "0") == 0) && sl_tma_prepare(c)) {
        const long long off = (static_cast<const char*>(gmj) - static_cast<const char*>(gbase)) / (g16 ? 2 : 4);
        const int j = (int)(off / (3 * c->d.N));
        CL_TRY(sl_adjoint_step_tma(c, lam_next, lam, j, w, dot ? sdot : nullptr, part, h, st));
        c->tma_steps++;
        CL_LAUNCHED(c);
        return CLAIRE_OK;
      }
    }
    with_halo<T>(h, [&](auto hc) {
      with_gm<T>(gmj, g16, [&](auto g) {
        using G = std::remove_const_t<std::remove_pointer_t<decltype(g)>>;
        const long long nb = sl_launch_adj<T, decltype(hc)::value, G>(rho != nullptr, lam != nullptr, dot, lam_next,
                                                                      rl_next, rho, dY, lam, rl, b, g, w, dt, c->d,
                                                                      sdot, part, st);
        if (dot) c->dot_blocks = nb;
      });
    });
  }
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

template <class T>
claire_status sl_incstate_init(claire_ctx* c, const T* vt, const void* gm0, bool g16, T* q, cudaStream_t st) {
  c->prof_begin("sl_inc_init", st);
  with_gm<T>(gm0, g16, [&](auto g) {
    using G = std::remove_const_t<std::remove_pointer_t<decltype(g)>>;
    k_inc_init<T, G><<<blocks_for(c->d.N), kThreads, 0, st>>>(vt, g, q, T(0.5 / c->o.nt), c->d);
  });
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

template <class T>
claire_status sl_incstate_step(claire_ctx* c, const T* q, const T* dX, const T* vt, const void* gmj1, bool g16,
                               T* qout, bool last, const T* rho, T* rl, T* b, T w, cudaStream_t st, int H) {
  const T hdt = T(0.5 / c->o.nt);
  c->prof_begin(!last ? "sl_inc_step" : (rho ? "sl_inc_step_last_rho" : "sl_inc_step_last"), st);
  const int variant = !last ? 0 : (rho ? 2 : 1);
  const int h = tile_halo<T>(H);
  if constexpr (sizeof(T) == 4) {
    // the step on the context's own arrays with bricks: X, vt and grad m^{j+1} staged by TMA
    Work<float>& W = c->work<float>();
    const void* gbase = g16 ? W.gm16 : (const void*)W.gm;
    const char* tma_env = std::getenv("CLAIRE_TMA");
    const bool own = dX == W.dX && vt == W.s && rho == nullptr && (!last || b == W.b) && gbase;
    if (h >= 2 && own && !(tma_env && std::strcmp(tma_env, "0") == 0) && sl_tma_prepare(c)) {
      const long long off = (static_cast<const char*>(gmj1) - static_cast<const char*>(gbase)) / (g16 ? 2 : 4);
      CL_TRY(sl_incstate_step_tma(c, q, qout, (int)(off / (3 * c->d.N)), last, hdt, w, h, st));
      c->tma_steps++;
      CL_LAUNCHED(c);
      return CLAIRE_OK;
    }
  }
  with_halo<T>(h, [&](auto hc) {
    with_gm<T>(gmj1, g16, [&](auto g) {
      using G = std::remove_const_t<std::remove_pointer_t<decltype(g)>>;
      sl_launch_inc<T, decltype(hc)::value, G>(variant, q, dX, vt, g, qout, rho, rl, b, hdt, w, c->d, st);
    });
  });
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

// Allow the brick-tiled kernels enough dynamic shared memory for two bricks of the largest halo.
template <class T> claire_status sl_init(claire_ctx* c) {
  cudaError_t e = cudaSuccess;
  for (int H = 2; H <= kMaxHalo; ++H) {
    with_halo<T>(H, [&](auto hc) {
      const cudaError_t r = sl_set_attrs<T, decltype(hc)::value>();
      if (r != cudaSuccess) e = r;
    });
  }
  if (e != cudaSuccess) {
    c->set_error(std::string("cudaFuncSetAttribute (tiled gathers): ") + cudaGetErrorString(e));
    return CLAIRE_ECUDA;
  }
  return CLAIRE_OK;
}

template <class T> claire_status sl_hadamard(claire_ctx* c, const T* a, const T* x, T* y, cudaStream_t st) {
  c->prof_begin("hadamard", st);
  k_hadamard<T><<<blocks_for(c->d.N), kThreads, 0, st>>>(a, x, y, c->d.N);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

#define INST(T)                                                                                                  \
  template claire_status sl_hadamard<T>(claire_ctx*, const T*, const T*, T*, cudaStream_t);                      \
  template claire_status sl_departure<T>(claire_ctx*, const T*, int, T*, cudaStream_t);                         \
  template claire_status sl_init<T>(claire_ctx*);                                                                \
  template claire_status sl_interp<T>(claire_ctx*, const T*, const T*, T*, cudaStream_t, int);                  \
  template claire_status sl_adjoint_terminal<T>(claire_ctx*, const T*, const T*, const T*, T*, T*, T*,           \
                                                const void*, bool, T, cudaStream_t);                            \
  template claire_status sl_adjoint_step<T>(claire_ctx*, const T*, const T*, const T*, const T*, T*, T*, T*,     \
                                            const void*, bool, T, cudaStream_t, const T*, double*, int);        \
  template claire_status sl_incstate_init<T>(claire_ctx*, const T*, const void*, bool, T*, cudaStream_t);      \
  template claire_status sl_incstate_step<T>(claire_ctx*, const T*, const T*, const T*, const void*, bool, T*,  \
                                             bool, const T*, T*, T*, T, cudaStream_t, int);
INST(float)
INST(double)
#undef INST

}  // namespace claire
