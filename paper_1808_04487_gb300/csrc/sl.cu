// Semi-Lagrangian transport kernels (Sec. 2.3.1, Sec. 3.4): RK2 characteristics and tricubic Lagrange gathers.
//
// One thread per grid node. The departure point of node i is xi = i + disp (grid units); per axis the stencil is
// b - 1 .. b + 2 with b = i + floor(disp) and t = disp - floor(disp) (splitting off the integer node index keeps
// t accurate in FP32 on large grids), the four cubic Lagrange weights on the nodes -1, 0, 1, 2 and periodic wrap.
// The 64-tap sum is evaluated separably (16 four-tap sums along i3, 4 along i2, 1 along i1: 84 FMA). Source
// terms and the time-integral accumulation of the adjoints (Sec. 3.5, memory-reduced Gauss-Newton) are fused
// into the epilogue of the gather so each step streams its fields once.
#include "impl.cuh"

namespace claire {

template <class T> struct Axis {
  int o[4];
  T w[4];
};

template <class T> __device__ __forceinline__ void axis_setup(int i, T disp, int n, int stride, Axis<T>& ax) {
  const T fd = floor(disp);
  const T t = disp - fd;
  const T tp1 = t + T(1), tm1 = t - T(1), tm2 = t - T(2);
  ax.w[0] = -(t * tm1 * tm2) * T(1.0 / 6.0);
  ax.w[1] = (tp1 * tm1 * tm2) * T(0.5);
  ax.w[2] = -(tp1 * t * tm2) * T(0.5);
  ax.w[3] = (tp1 * t * tm1) * T(1.0 / 6.0);
  int b = (i + (int)fd - 1) % n;
  if (b < 0) b += n;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    int q = b + p;
    if (q >= n) q -= n;
    ax.o[p] = q * stride;
  }
}

template <class T> struct Stencil {
  Axis<T> a1, a2, a3;
};

template <class T> __device__ __forceinline__ T gather(const T* __restrict__ f, const Stencil<T>& s) {
  T acc = T(0);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    T a1 = T(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T* row = f + (s.a1.o[p] + s.a2.o[q]);
      T a2 = s.a3.w[0] * __ldg(row + s.a3.o[0]);
      a2 = fma(s.a3.w[1], __ldg(row + s.a3.o[1]), a2);
      a2 = fma(s.a3.w[2], __ldg(row + s.a3.o[2]), a2);
      a2 = fma(s.a3.w[3], __ldg(row + s.a3.o[3]), a2);
      a1 = fma(s.a2.w[q], a2, a1);
    }
    acc = fma(s.a1.w[p], a1, acc);
  }
  return acc;
}

struct Node {
  int i1, i2, i3;
};

__device__ __forceinline__ Node node_of(long long idx, const Dims& d) {
  Node n;
  n.i3 = (int)(idx % d.n3);
  const long long t = idx / d.n3;
  n.i2 = (int)(t % d.n2);
  n.i1 = (int)(t / d.n2);
  return n;
}

template <class T>
__device__ __forceinline__ void stencil_at(const Node& x, T d1, T d2, T d3, const Dims& d, Stencil<T>& s) {
  axis_setup<T>(x.i1, d1, d.n1, d.n2 * d.n3, s.a1);
  axis_setup<T>(x.i2, d2, d.n2, d.n3, s.a2);
  axis_setup<T>(x.i3, d3, d.n3, 1, s.a3);
}

// ---------------------------------------------------------------------------------------------------------------
// RK2 (Heun) departure points of one step: X* = x - s dt v(x), X = x - s dt/2 (v(x) + v(X*)), s = +1 state, -1
// adjoint; stored as (X - x)/h per axis.
template <class T>
__global__ void __launch_bounds__(256) k_departure(const T* __restrict__ v, T* __restrict__ disp, T sdt, T ih1,
                                                   T ih2, T ih3, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.N) return;
  const long long N = d.N;
  const T v1 = v[idx], v2 = v[N + idx], v3 = v[2 * N + idx];
  const Node x = node_of(idx, d);
  Stencil<T> s;
  stencil_at<T>(x, -sdt * v1 * ih1, -sdt * v2 * ih2, -sdt * v3 * ih3, d, s);
  const T w1 = gather<T>(v, s), w2 = gather<T>(v + N, s), w3 = gather<T>(v + 2 * N, s);
  const T h = T(0.5) * sdt;
  disp[idx] = -h * (v1 + w1) * ih1;
  disp[N + idx] = -h * (v2 + w2) * ih2;
  disp[2 * N + idx] = -h * (v3 + w3) * ih3;
}

template <class T>
__global__ void __launch_bounds__(256) k_interp(const T* __restrict__ f, const T* __restrict__ disp,
                                                T* __restrict__ out, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.N) return;
  const long long N = d.N;
  const Node x = node_of(idx, d);
  Stencil<T> s;
  stencil_at<T>(x, disp[idx], disp[N + idx], disp[2 * N + idx], d, s);
  out[idx] = gather<T>(f, s);
}

// lam = mR - m1 (Eq. (4) final condition), rl = rho lam, b = w lam grad m^{nt}
template <class T, bool RHO>
__global__ void __launch_bounds__(256) k_adj_terminal(const T* __restrict__ mR, const T* __restrict__ m1,
                                                      const T* __restrict__ rho, T* __restrict__ lam,
                                                      T* __restrict__ rl, T* __restrict__ b,
                                                      const T* __restrict__ gm, T w, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.N) return;
  const long long N = d.N;
  const T l = mR[idx] - m1[idx];
  lam[idx] = l;
  if (RHO) rl[idx] = rho[idx] * l;
  const T wl = w * l;
  b[idx] = wl * gm[idx];
  b[N + idx] = wl * gm[N + idx];
  b[2 * N + idx] = wl * gm[2 * N + idx];
}

// One backward step of -d_t lam - div(lam v) = 0 along Y (Eq. (4), (9)):
//   a = lam^{j+1}(Y); with the div source: c = (rho lam^{j+1})(Y), lam^j = a + dt/2 (c + rho(x)(a + dt c)).
// Epilogue: optional store of lam^j and rho lam^j, and b += w_j lam^j grad m^j.
template <class T, bool RHO, bool STORE, bool ACC>
__global__ void __launch_bounds__(256) k_adj_step(const T* __restrict__ lam_next, const T* __restrict__ rl_next,
                                                  const T* __restrict__ rho, const T* __restrict__ dY,
                                                  T* __restrict__ lam, T* __restrict__ rl, T* __restrict__ b,
                                                  const T* __restrict__ gm, T w, T dt, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.N) return;
  const long long N = d.N;
  const Node x = node_of(idx, d);
  Stencil<T> s;
  stencil_at<T>(x, dY[idx], dY[N + idx], dY[2 * N + idx], d, s);
  T l = gather<T>(lam_next, s);
  T r = T(0);
  if (RHO) {
    const T cc = gather<T>(rl_next, s);
    r = rho[idx];
    l = l + T(0.5) * dt * (cc + r * (l + dt * cc));
  }
  if (STORE) {
    lam[idx] = l;
    if (RHO) rl[idx] = r * l;
  }
  if (ACC) {
    const T wl = w * l;
    b[idx] = fma(wl, gm[idx], b[idx]);
    b[N + idx] = fma(wl, gm[N + idx], b[N + idx]);
    b[2 * N + idx] = fma(wl, gm[2 * N + idx], b[2 * N + idx]);
  }
}

// q^0 = m~^0 + dt/2 f^0 with m~^0 = 0, f = -vt . grad m (Eq. (8))
template <class T>
__global__ void __launch_bounds__(256) k_inc_init(const T* __restrict__ vt, const T* __restrict__ gm,
                                                  T* __restrict__ q, T hdt, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.N) return;
  const long long N = d.N;
  const T f = -(vt[idx] * gm[idx] + vt[N + idx] * gm[N + idx] + vt[2 * N + idx] * gm[2 * N + idx]);
  q[idx] = hdt * f;
}

// m~^{j+1}(x) = q^j(X) + dt/2 f^{j+1}(x); not last: q^{j+1} = m~^{j+1} + dt/2 f^{j+1}.
// last: lam~ = -m~(1) (Eq. (9) final condition), rl = rho lam~, b = w lam~ grad m^{nt}.
template <class T, bool LAST, bool RHO>
__global__ void __launch_bounds__(256) k_inc_step(const T* __restrict__ q, const T* __restrict__ dX,
                                                  const T* __restrict__ vt, const T* __restrict__ gm,
                                                  T* __restrict__ qout, const T* __restrict__ rho,
                                                  T* __restrict__ rl, T* __restrict__ b, T hdt, T w, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.N) return;
  const long long N = d.N;
  const Node x = node_of(idx, d);
  Stencil<T> s;
  stencil_at<T>(x, dX[idx], dX[N + idx], dX[2 * N + idx], d, s);
  const T g1 = gm[idx], g2 = gm[N + idx], g3 = gm[2 * N + idx];
  const T f = -(vt[idx] * g1 + vt[N + idx] * g2 + vt[2 * N + idx] * g3);
  const T mt = gather<T>(q, s) + hdt * f;
  if (!LAST) {
    qout[idx] = mt + hdt * f;
  } else {
    const T l = -mt;
    qout[idx] = l;
    if (RHO) rl[idx] = rho[idx] * l;
    const T wl = w * l;
    b[idx] = wl * g1;
    b[N + idx] = wl * g2;
    b[2 * N + idx] = wl * g3;
  }
}

// y = a .* x
template <class T>
__global__ void __launch_bounds__(256) k_hadamard(const T* __restrict__ a, const T* __restrict__ x,
                                                  T* __restrict__ y, long long n) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n) y[idx] = a[idx] * x[idx];
}

// ---------------------------------------------------------------------------------------------------------------
static inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

template <class T> claire_status sl_departure(claire_ctx* c, const T* v, int dir, T* disp, cudaStream_t st) {
  const Dims& d = c->d;
  const double dt = 1.0 / c->o.nt;
  const double twopi = 6.283185307179586476925286766559;
  const T ih1 = T(d.n1 / twopi), ih2 = T(d.n2 / twopi), ih3 = T(d.n3 / twopi);
  c->prof_begin("sl_departure", st);
  k_departure<T><<<blocks_for(d.N), kThreads, 0, st>>>(v, disp, T(dir * dt), ih1, ih2, ih3, d);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

template <class T> claire_status sl_interp(claire_ctx* c, const T* f, const T* disp, T* out, cudaStream_t st) {
  c->prof_begin("sl_interp", st);
  k_interp<T><<<blocks_for(c->d.N), kThreads, 0, st>>>(f, disp, out, c->d);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

template <class T>
claire_status sl_adjoint_terminal(claire_ctx* c, const T* mR, const T* m1, const T* rho, T* lam, T* rl, T* b,
                                  const T* gmj, T w, cudaStream_t st) {
  c->prof_begin(rho ? "sl_adj_terminal_rho" : "sl_adj_terminal", st);
  if (rho)
    k_adj_terminal<T, true><<<blocks_for(c->d.N), kThreads, 0, st>>>(mR, m1, rho, lam, rl, b, gmj, w, c->d);
  else
    k_adj_terminal<T, false><<<blocks_for(c->d.N), kThreads, 0, st>>>(mR, m1, rho, lam, rl, b, gmj, w, c->d);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

template <class T>
claire_status sl_adjoint_step(claire_ctx* c, const T* lam_next, const T* rl_next, const T* rho, const T* dY, T* lam,
                              T* rl, T* b, const T* gmj, T w, cudaStream_t st) {
  const T dt = T(1.0 / c->o.nt);
  const unsigned g = blocks_for(c->d.N);
  const int key = (rho ? 4 : 0) | (lam ? 2 : 0) | (b ? 1 : 0);
  static const char* names[8] = {"sl_adj_step", "sl_adj_step_acc", "sl_adj_step_store", "sl_adj_step_store_acc",
                                 "sl_adj_step_rho", "sl_adj_step_rho_acc", "sl_adj_step_rho_store",
                                 "sl_adj_step_rho_store_acc"};
  c->prof_begin(names[key], st);
#define ADJ(R, S, A) \
  k_adj_step<T, R, S, A><<<g, kThreads, 0, st>>>(lam_next, rl_next, rho, dY, lam, rl, b, gmj, w, dt, c->d)
  switch (key) {
    case 0: ADJ(false, false, false); break;
    case 1: ADJ(false, false, true); break;
    case 2: ADJ(false, true, false); break;
    case 3: ADJ(false, true, true); break;
    case 4: ADJ(true, false, false); break;
    case 5: ADJ(true, false, true); break;
    case 6: ADJ(true, true, false); break;
    default: ADJ(true, true, true); break;
  }
#undef ADJ
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

template <class T> claire_status sl_incstate_init(claire_ctx* c, const T* vt, const T* gm0, T* q, cudaStream_t st) {
  c->prof_begin("sl_inc_init", st);
  k_inc_init<T><<<blocks_for(c->d.N), kThreads, 0, st>>>(vt, gm0, q, T(0.5 / c->o.nt), c->d);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

template <class T>
claire_status sl_incstate_step(claire_ctx* c, const T* q, const T* dX, const T* vt, const T* gmj1, T* qout, bool last,
                               const T* rho, T* rl, T* b, T w, cudaStream_t st) {
  const T hdt = T(0.5 / c->o.nt);
  const unsigned g = blocks_for(c->d.N);
  c->prof_begin(!last ? "sl_inc_step" : (rho ? "sl_inc_step_last_rho" : "sl_inc_step_last"), st);
  if (!last)
    k_inc_step<T, false, false><<<g, kThreads, 0, st>>>(q, dX, vt, gmj1, qout, rho, rl, b, hdt, w, c->d);
  else if (rho)
    k_inc_step<T, true, true><<<g, kThreads, 0, st>>>(q, dX, vt, gmj1, qout, rho, rl, b, hdt, w, c->d);
  else
    k_inc_step<T, true, false><<<g, kThreads, 0, st>>>(q, dX, vt, gmj1, qout, rho, rl, b, hdt, w, c->d);
  CL_LAUNCHED(c);
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
  template claire_status sl_interp<T>(claire_ctx*, const T*, const T*, T*, cudaStream_t);                       \
  template claire_status sl_adjoint_terminal<T>(claire_ctx*, const T*, const T*, const T*, T*, T*, T*, const T*, \
                                                T, cudaStream_t);                                               \
  template claire_status sl_adjoint_step<T>(claire_ctx*, const T*, const T*, const T*, const T*, T*, T*, T*,     \
                                            const T*, T, cudaStream_t);                                         \
  template claire_status sl_incstate_init<T>(claire_ctx*, const T*, const T*, T*, cudaStream_t);                \
  template claire_status sl_incstate_step<T>(claire_ctx*, const T*, const T*, const T*, const T*, T*, bool,     \
                                             const T*, T*, T*, T, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace claire
