// Fourier-domain symbols of the pseudo-spectral operators (Sec. 2.3.1) on the half spectrum [n1][n2][n3/2+1]:
// gradient i k', divergence i k'., Leray projection I - k'k'^T/|k'|^2 (Sec. 2.2), regularisation A with symbol
// |k|^2 (H1) or |k|^4 (H2) (Sec. 2.1), its inverse as the spectral preconditioner with the zero eigenvalue set to
// 1 (Sec. 2.3.3, Remark), and the Parseval form of sum_c <v_c, A v_c>. Integer wavenumbers; first-order symbols
// use k' with the Nyquist entry zeroed, even-order symbols the full k. All kernels stream float2/double2 values.
#include "impl.cuh"

namespace claire {

struct Wave {
  int k1, k2, k3;     // full wavenumbers (Nyquist as +n/2)
  int p1, p2, p3;     // first-order wavenumbers (Nyquist zeroed)
};

__device__ __forceinline__ Wave wavenumbers(long long idx, const Dims& d) {
  Wave w;
  const int i3 = (int)(idx % d.n3h);
  const long long t = idx / d.n3h;
  const int i2 = (int)(t % d.n2);
  const int i1 = (int)(t / d.n2);
  w.k1 = i1 <= d.n1 / 2 ? i1 : i1 - d.n1;
  w.k2 = i2 <= d.n2 / 2 ? i2 : i2 - d.n2;
  w.k3 = i3;
  w.p1 = (2 * w.k1 == d.n1) ? 0 : w.k1;
  w.p2 = (2 * w.k2 == d.n2) ? 0 : w.k2;
  w.p3 = (2 * w.k3 == d.n3) ? 0 : w.k3;
  return w;
}

template <class T> __device__ __forceinline__ T reg_symbol(const Wave& w, int regnorm) {
  const T ksq = T(w.k1) * T(w.k1) + T(w.k2) * T(w.k2) + T(w.k3) * T(w.k3);
  return regnorm == 2 ? ksq * ksq : ksq;
}

// i*k*F
template <class T> __device__ __forceinline__ cplx<T> ik(T k, cplx<T> f) { return mk<T>(-k * f.y, k * f.x); }

template <class T>
__global__ void k_spec_grad(const cplx<T>* __restrict__ F, cplx<T>* __restrict__ G0, cplx<T>* __restrict__ G1,
                            cplx<T>* __restrict__ G2, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.Ns) return;
  const Wave w = wavenumbers(idx, d);
  const cplx<T> f = F[idx];
  G0[idx] = ik<T>(T(w.p1), f);
  G1[idx] = ik<T>(T(w.p2), f);
  G2[idx] = ik<T>(T(w.p3), f);
}

template <class T>
__global__ void k_spec_div(const cplx<T>* __restrict__ V0, const cplx<T>* __restrict__ V1,
                           const cplx<T>* __restrict__ V2, cplx<T>* __restrict__ D, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.Ns) return;
  const Wave w = wavenumbers(idx, d);
  const cplx<T> a = ik<T>(T(w.p1), V0[idx]), b = ik<T>(T(w.p2), V1[idx]), c = ik<T>(T(w.p3), V2[idx]);
  D[idx] = mk<T>(a.x + b.x + c.x, a.y + b.y + c.y);
}

template <class T> __device__ __forceinline__ void leray_apply(const Wave& w, cplx<T>& a, cplx<T>& b, cplx<T>& c) {
  const T q1 = T(w.p1), q2 = T(w.p2), q3 = T(w.p3);
  const T qq = q1 * q1 + q2 * q2 + q3 * q3;
  if (qq > T(0)) {
    const T inv = T(1) / qq;
    const T sr = (q1 * a.x + q2 * b.x + q3 * c.x) * inv;
    const T si = (q1 * a.y + q2 * b.y + q3 * c.y) * inv;
    a = mk<T>(a.x - q1 * sr, a.y - q1 * si);
    b = mk<T>(b.x - q2 * sr, b.y - q2 * si);
    c = mk<T>(c.x - q3 * sr, c.y - q3 * si);
  }
}

template <class T>
__global__ void k_spec_leray(cplx<T>* __restrict__ V0, cplx<T>* __restrict__ V1, cplx<T>* __restrict__ V2, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.Ns) return;
  const Wave w = wavenumbers(idx, d);
  cplx<T> a = V0[idx], b = V1[idx], c = V2[idx];
  leray_apply<T>(w, a, b, c);
  V0[idx] = a;
  V1[idx] = b;
  V2[idx] = c;
}

template <class T>
__global__ void k_spec_scale(cplx<T>* __restrict__ V, int ncomp, long long cstride, int mode, int regnorm, T beta,
                             Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.Ns) return;
  const Wave w = wavenumbers(idx, d);
  T f;
  if (mode == 0) {
    f = beta * reg_symbol<T>(w, regnorm);
  } else if (mode == 1) {
    const T a = reg_symbol<T>(w, regnorm);
    f = a > T(0) ? T(1) / (beta * a) : T(1);
  } else {
    f = -(T(w.k1) * T(w.k1) + T(w.k2) * T(w.k2) + T(w.k3) * T(w.k3));
  }
  for (int c = 0; c < ncomp; ++c) {
    cplx<T> x = V[c * cstride + idx];
    V[c * cstride + idx] = mk<T>(x.x * f, x.y * f);
  }
}

template <class T>
__global__ void k_spec_combine(const cplx<T>* __restrict__ V, cplx<T>* __restrict__ B, int regnorm, int divfree,
                               T beta, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.Ns) return;
  const Wave w = wavenumbers(idx, d);
  const long long s = d.Ns;
  cplx<T> b0 = B[idx], b1 = B[s + idx], b2 = B[2 * s + idx];
  if (divfree) leray_apply<T>(w, b0, b1, b2);
  const T f = beta * reg_symbol<T>(w, regnorm);
  const cplx<T> v0 = V[idx], v1 = V[s + idx], v2 = V[2 * s + idx];
  B[idx] = mk<T>(f * v0.x + b0.x, f * v0.y + b0.y);
  B[s + idx] = mk<T>(f * v1.x + b1.x, f * v1.y + b1.y);
  B[2 * s + idx] = mk<T>(f * v2.x + b2.x, f * v2.y + b2.y);
}

// sum over the half spectrum with weight 1 on the k3 = 0 and k3 = n3/2 planes and 2 elsewhere (Parseval)
template <class T>
__global__ void __launch_bounds__(256) k_spec_reg_partial(const cplx<T>* __restrict__ V, int regnorm, Dims d,
                                                          double* __restrict__ partials) {
  double acc = 0.0;
  const long long s = d.Ns;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < s;
       idx += (long long)gridDim.x * blockDim.x) {
    const Wave w = wavenumbers(idx, d);
    const double a = reg_symbol<double>(w, regnorm);
    const double wt = (w.k3 == 0 || 2 * w.k3 == d.n3) ? 1.0 : 2.0;
    double e = 0.0;
    for (int c = 0; c < 3; ++c) {
      const cplx<T> x = V[c * s + idx];
      e += double(x.x) * double(x.x) + double(x.y) * double(x.y);
    }
    acc += wt * a * e;
  }
  __shared__ double red[256 / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    partials[blockIdx.x] = t;
  }
}

static inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

template <class T>
claire_status spec_grad(claire_ctx* c, const cplx<T>* F, cplx<T>* G0, cplx<T>* G1, cplx<T>* G2, cudaStream_t st) {
  c->prof_begin("spec_grad", st);
  k_spec_grad<T><<<blocks_for(c->d.Ns), kThreads, 0, st>>>(F, G0, G1, G2, c->d);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T>
claire_status spec_div(claire_ctx* c, const cplx<T>* V0, const cplx<T>* V1, const cplx<T>* V2, cplx<T>* D,
                       cudaStream_t st) {
  c->prof_begin("spec_div", st);
  k_spec_div<T><<<blocks_for(c->d.Ns), kThreads, 0, st>>>(V0, V1, V2, D, c->d);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T> claire_status spec_leray(claire_ctx* c, cplx<T>* V0, cplx<T>* V1, cplx<T>* V2, cudaStream_t st) {
  c->prof_begin("spec_leray", st);
  k_spec_leray<T><<<blocks_for(c->d.Ns), kThreads, 0, st>>>(V0, V1, V2, c->d);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T>
claire_status spec_scale(claire_ctx* c, cplx<T>* V, int ncomp, long long cstride, int mode, double beta,
                         cudaStream_t st) {
  c->prof_begin("spec_scale", st);
  k_spec_scale<T><<<blocks_for(c->d.Ns), kThreads, 0, st>>>(V, ncomp, cstride, mode, c->o.regnorm, T(beta), c->d);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T> claire_status spec_combine(claire_ctx* c, const cplx<T>* V, cplx<T>* B, cudaStream_t st) {
  c->prof_begin("spec_combine", st);
  k_spec_combine<T><<<blocks_for(c->d.Ns), kThreads, 0, st>>>(V, B, c->o.regnorm, c->o.divfree, T(c->o.beta), c->d);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T> claire_status spec_reg_partial(claire_ctx* c, const cplx<T>* V, double* partials, cudaStream_t st) {
  c->prof_begin("spec_reg_partial", st);
  k_spec_reg_partial<T><<<kReduceBlocks, 256, 0, st>>>(V, c->o.regnorm, c->d, partials);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

#define INST(T)                                                                                                   \
  template claire_status spec_grad<T>(claire_ctx*, const cplx<T>*, cplx<T>*, cplx<T>*, cplx<T>*, cudaStream_t);  \
  template claire_status spec_div<T>(claire_ctx*, const cplx<T>*, const cplx<T>*, const cplx<T>*, cplx<T>*,      \
                                     cudaStream_t);                                                              \
  template claire_status spec_leray<T>(claire_ctx*, cplx<T>*, cplx<T>*, cplx<T>*, cudaStream_t);                 \
  template claire_status spec_scale<T>(claire_ctx*, cplx<T>*, int, long long, int, double, cudaStream_t);        \
  template claire_status spec_combine<T>(claire_ctx*, const cplx<T>*, cplx<T>*, cudaStream_t);                   \
  template claire_status spec_reg_partial<T>(claire_ctx*, const cplx<T>*, double*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace claire
