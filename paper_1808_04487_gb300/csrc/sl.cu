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

// Per-axis part of a stencil: the four cubic Lagrange weights and the first stencil node b - 1, reduced into
// [0, n) by a periodic shift when it lies outside [-n, n) (only for displacements beyond one period).
template <class T> __device__ __forceinline__ int axis_setup(int i, T disp, int n, T* w) {
  const T fd = floor(disp);
  const T t = disp - fd;
  const T tp1 = t + T(1), tm1 = t - T(1), tm2 = t - T(2);
  w[0] = -(t * tm1 * tm2) * T(1.0 / 6.0);
  w[1] = (tp1 * tm1 * tm2) * T(0.5);
  w[2] = -(tp1 * t * tm2) * T(0.5);
  w[3] = (tp1 * t * tm1) * T(1.0 / 6.0);
  int b = i + (int)fd - 1;
  if (b < -n || b >= n) {
    b %= n;
    if (b < 0) b += n;
  }
  return b;
}

// q in [-n, 2n) -> [0, n)
__device__ __forceinline__ int wrapc(int q, int n) {
  q = q < 0 ? q + n : q;
  return q >= n ? q - n : q;
}

template <class T> struct Stencil {
  T w1[4], w2[4], w3[4];
  int b1, b2, b3;  // first stencil node per axis, in [-n, n)
  bool inside;     // the whole warp's stencils lie inside the box: no periodic wrap needed
};

template <class T>
__device__ __forceinline__ void stencil_at(int i1, int i2, int i3, T d1, T d2, T d3, const Dims& d, Stencil<T>& s) {
  s.b1 = axis_setup<T>(i1, d1, d.n1, s.w1);
  s.b2 = axis_setup<T>(i2, d2, d.n2, s.w2);
  s.b3 = axis_setup<T>(i3, d3, d.n3, s.w3);
  const bool in = (unsigned)s.b1 <= (unsigned)(d.n1 - 4) && (unsigned)s.b2 <= (unsigned)(d.n2 - 4) &&
                  (unsigned)s.b3 <= (unsigned)(d.n3 - 4);
  // one path per warp: a warp with any wrapping lane takes the wrapping path for all its lanes
  s.inside = __all_sync(__activemask(), in);
}

// sum_{p,q,r} w1[p] w2[q] w3[r] f[row(p,q) + col(r)], evaluated as 16 four-tap sums along i3, then i2, then i1.
// Both branches use the same order of operations, so the result does not depend on which one runs.
template <class T> __device__ __forceinline__ T gather(const T* __restrict__ f, const Stencil<T>& s, const Dims& d) {
  const int s2 = d.n3, s1 = d.n2 * d.n3;
  T acc = T(0);
  if (s.inside) {
    const T* corner = f + (s.b1 * s1 + s.b2 * s2 + s.b3);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      T a1 = T(0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T* row = corner + (p * s1 + q * s2);
        T a2 = s.w3[0] * __ldg(row);
        a2 = fma(s.w3[1], __ldg(row + 1), a2);
        a2 = fma(s.w3[2], __ldg(row + 2), a2);
        a2 = fma(s.w3[3], __ldg(row + 3), a2);
        a1 = fma(s.w2[q], a2, a1);
      }
      acc = fma(s.w1[p], a1, acc);
    }
  } else {
    int o1[4], o2[4], o3[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      o1[p] = wrapc(s.b1 + p, d.n1) * s1;
      o2[p] = wrapc(s.b2 + p, d.n2) * s2;
      o3[p] = wrapc(s.b3 + p, d.n3);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      T a1 = T(0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T* row = f + (o1[p] + o2[q]);
        T a2 = s.w3[0] * __ldg(row + o3[0]);
        a2 = fma(s.w3[1], __ldg(row + o3[1]), a2);
        a2 = fma(s.w3[2], __ldg(row + o3[2]), a2);
        a2 = fma(s.w3[3], __ldg(row + o3[3]), a2);
        a1 = fma(s.w2[q], a2, a1);
      }
      acc = fma(s.w1[p], a1, acc);
    }
  }
  return acc;
}

// Node of the calling thread: 3D launch grid, x along i3 (coalesced), y along i2, z over i1; no division.
struct Node {
  int i1, i2, i3, idx;
  bool valid;
};

__device__ __forceinline__ Node node3d(const Dims& d) {
  Node n;
  n.i3 = blockIdx.x * blockDim.x + threadIdx.x;
  n.i2 = blockIdx.y * blockDim.y + threadIdx.y;
  n.i1 = blockIdx.z;
  n.valid = n.i3 < d.n3 && n.i2 < d.n2;
  n.idx = (n.i1 * d.n2 + n.i2) * d.n3 + n.i3;
  return n;
}

// ---------------------------------------------------------------------------------------------------------------
// RK2 (Heun) departure points of one step: X* = x - s dt v(x), X = x - s dt/2 (v(x) + v(X*)), s = +1 state, -1
// adjoint; stored as (X - x)/h per axis.
template <class T>
__global__ void __launch_bounds__(256) k_departure(const T* __restrict__ v, T* __restrict__ disp, T sdt, T ih1,
                                                   T ih2, T ih3, Dims d) {
  const Node x = node3d(d);
  if (!x.valid) return;
  const int idx = x.idx;
  const long long N = d.N;
  const T v1 = v[idx], v2 = v[N + idx], v3 = v[2 * N + idx];
  Stencil<T> s;
  stencil_at<T>(x.i1, x.i2, x.i3, -sdt * v1 * ih1, -sdt * v2 * ih2, -sdt * v3 * ih3, d, s);
  const T w1 = gather<T>(v, s, d), w2 = gather<T>(v + N, s, d), w3 = gather<T>(v + 2 * N, s, d);
  const T h = T(0.5) * sdt;
  disp[idx] = -h * (v1 + w1) * ih1;
  disp[N + idx] = -h * (v2 + w2) * ih2;
  disp[2 * N + idx] = -h * (v3 + w3) * ih3;
}

template <class T>
__global__ void __launch_bounds__(256) k_interp(const T* __restrict__ f, const T* __restrict__ disp,
                                                T* __restrict__ out, Dims d) {
  const Node x = node3d(d);
  if (!x.valid) return;
  const int idx = x.idx;
  const long long N = d.N;
  Stencil<T> s;
  stencil_at<T>(x.i1, x.i2, x.i3, disp[idx], disp[N + idx], disp[2 * N + idx], d, s);
  out[idx] = gather<T>(f, s, d);
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
template <class T, bool RHO, bool STORE, bool ACC, bool DOT>
__global__ void __launch_bounds__(256) k_adj_step(const T* __restrict__ lam_next, const T* __restrict__ rl_next,
                                                  const T* __restrict__ rho, const T* __restrict__ dY,
                                                  T* __restrict__ lam, T* __restrict__ rl, T* __restrict__ b,
                                                  const T* __restrict__ gm, T w, T dt, Dims d,
                                                  const T* __restrict__ sv, double* __restrict__ part) {
  const Node x = node3d(d);
  Acc<T> contrib;
  if (x.valid) {
    const int idx = x.idx;
    const long long N = d.N;
    Stencil<T> s;
    stencil_at<T>(x.i1, x.i2, x.i3, dY[idx], dY[N + idx], dY[2 * N + idx], d, s);
    T l = gather<T>(lam_next, s, d);
    T r = T(0);
    if (RHO) {
      const T cc = gather<T>(rl_next, s, d);
      r = rho[idx];
      l = l + T(0.5) * dt * (cc + r * (l + dt * cc));
    }
    if (STORE) {
      lam[idx] = l;
      if (RHO) rl[idx] = r * l;
    }
    if (ACC) {
      const T wl = w * l;
      const T b0 = fma(wl, gm[idx], b[idx]);
      const T b1 = fma(wl, gm[N + idx], b[N + idx]);
      const T b2 = fma(wl, gm[2 * N + idx], b[2 * N + idx]);
      b[idx] = b0;
      b[N + idx] = b1;
      b[2 * N + idx] = b2;
      // <s, b>: the final time integral against a vector s, for PCG's <s, H s> (Alg. 2)
      if (DOT) {
        contrib.add_prod(sv[idx], b0);
        contrib.add_prod(sv[N + idx], b1);
        contrib.add_prod(sv[2 * N + idx], b2);
      }
    }
  }
  if (DOT) {
    __shared__ double red[32];
    double cs = contrib.value();
    for (int o = 16; o > 0; o >>= 1) cs += __shfl_down_sync(0xffffffffu, cs, o);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if ((tid & 31) == 0) red[tid >> 5] = cs;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < (int)((blockDim.x * blockDim.y) >> 5); ++i) t += red[i];
      part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = t;
    }
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
  const Node x = node3d(d);
  if (!x.valid) return;
  const int idx = x.idx;
  const long long N = d.N;
  Stencil<T> s;
  stencil_at<T>(x.i1, x.i2, x.i3, dX[idx], dX[N + idx], dX[2 * N + idx], d, s);
  const T g1 = gm[idx], g2 = gm[N + idx], g3 = gm[2 * N + idx];
  const T f = -(vt[idx] * g1 + vt[N + idx] * g2 + vt[2 * N + idx] * g3);
  const T mt = gather<T>(q, s, d) + hdt * f;
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

// 3D launch shape of the gather kernels: 256 threads, x along i3 (up to 64 wide), y along i2, z = i1
Launch3 launch3(const Dims& d) {
  const int bx = d.n3 >= 64 ? 64 : (d.n3 >= 32 ? 32 : 16);
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

template <class T> claire_status sl_interp(claire_ctx* c, const T* f, const T* disp, T* out, cudaStream_t st) {
  c->prof_begin("sl_interp", st);
  const Launch3 L = launch3(c->d);
  k_interp<T><<<L.grid, L.block, 0, st>>>(f, disp, out, c->d);
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
                              T* rl, T* b, const T* gmj, T w, cudaStream_t st, const T* sdot, double* part) {
  const T dt = T(1.0 / c->o.nt);
  const bool dot = sdot != nullptr && b != nullptr && lam == nullptr;
  const int key = (rho ? 4 : 0) | (lam ? 2 : 0) | (b ? 1 : 0);
  static const char* names[8] = {"sl_adj_step", "sl_adj_step_acc", "sl_adj_step_store", "sl_adj_step_store_acc",
                                 "sl_adj_step_rho", "sl_adj_step_rho_acc", "sl_adj_step_rho_store",
                                 "sl_adj_step_rho_store_acc"};
  c->prof_begin(dot ? (rho ? "sl_adj_step_rho_acc_dot" : "sl_adj_step_acc_dot") : names[key], st);
  const Launch3 L3 = launch3(c->d);
#define ADJ(R, S, A, D)                                                                                         \
  k_adj_step<T, R, S, A, D><<<L3.grid, L3.block, 0, st>>>(lam_next, rl_next, rho, dY, lam, rl, b, gmj, w, dt, c->d, \
                                                          sdot, part)
  if (dot) {
    if (rho)
      ADJ(true, false, true, true);
    else
      ADJ(false, false, true, true);
  } else {
    switch (key) {
      case 0: ADJ(false, false, false, false); break;
      case 1: ADJ(false, false, true, false); break;
      case 2: ADJ(false, true, false, false); break;
      case 3: ADJ(false, true, true, false); break;
      case 4: ADJ(true, false, false, false); break;
      case 5: ADJ(true, false, true, false); break;
      case 6: ADJ(true, true, false, false); break;
      default: ADJ(true, true, true, false); break;
    }
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
  c->prof_begin(!last ? "sl_inc_step" : (rho ? "sl_inc_step_last_rho" : "sl_inc_step_last"), st);
  const Launch3 L = launch3(c->d);
  if (!last)
    k_inc_step<T, false, false><<<L.grid, L.block, 0, st>>>(q, dX, vt, gmj1, qout, rho, rl, b, hdt, w, c->d);
  else if (rho)
    k_inc_step<T, true, true><<<L.grid, L.block, 0, st>>>(q, dX, vt, gmj1, qout, rho, rl, b, hdt, w, c->d);
  else
    k_inc_step<T, true, false><<<L.grid, L.block, 0, st>>>(q, dX, vt, gmj1, qout, rho, rl, b, hdt, w, c->d);
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
                                            const T*, T, cudaStream_t, const T*, double*);                      \
  template claire_status sl_incstate_init<T>(claire_ctx*, const T*, const T*, T*, cudaStream_t);                \
  template claire_status sl_incstate_step<T>(claire_ctx*, const T*, const T*, const T*, const T*, T*, bool,     \
                                             const T*, T*, T*, T, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace claire
