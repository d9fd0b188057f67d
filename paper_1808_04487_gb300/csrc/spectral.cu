// Fourier-domain symbols of the pseudo-spectral operators (Sec. 2.3.1) on the half spectrum [n1][n2][n3/2+1]:
// gradient i k', divergence i k'., Leray projection I - k'k'^T/|k'|^2 (Sec. 2.2), regularisation A with symbol
// |k|^2 (H1) or |k|^4 (H2) (Sec. 2.1), its inverse as the spectral preconditioner with the zero eigenvalue set to
// 1 (Sec. 2.3.3, Remark), and the Parseval form of sum_c <v_c, A v_c>. Integer wavenumbers; first-order symbols
// use k' with the Nyquist entry zeroed, even-order symbols the full k. All kernels stream float2/double2 values.
//
// K of Eq. (5) comes in three forms (kmode): 0 identity, 1 Leray (div v = 0), 2 the H1-div model (H1 seminorm for
// v plus the penalty beta_w/2 ||div v||^2_H1, Sec. 2.1-2.2): K^ = I - q k'k'^T with
// q = rw (|k|^2 + 1) / (|k|^2 + rw (|k|^2 + 1) |k'|^2), rw = beta_w / beta_v, which is the paper's
// I - grad (beta_v (beta_w (-Lap + I))^-1 + I)^-1 Lap^-1 div off the Nyquist planes. beta_v A + K H_data (Eq. (7))
// is then self-adjoint in <K^-1 a, b>, K^-1 = I + s k'k'^T with s = rw (|k|^2 + 1) / |k|^2; the PCG products and
// the Armijo slope of the solver use that form, and the regularisation value gains rw (|k|^2 + 1) |k'.v|^2.
#include "impl.cuh"

namespace claire {

struct Wave {
  int k1, k2, k3;     // full wavenumbers (Nyquist as +n/2)
  int p1, p2, p3;     // first-order wavenumbers (Nyquist zeroed)
};

__device__ __forceinline__ Wave wavenumbers(long long idx, const Dims& d) {
  Wave w;
  const unsigned j = (unsigned)idx;
  const unsigned t = d.by_n3h.div(j);
  const unsigned i3 = j - t * (unsigned)d.n3h;
  const unsigned i1 = d.by_n2.div(t);
  const unsigned i2 = t - i1 * (unsigned)d.n2;
  w.k1 = (int)i1 <= d.n1 / 2 ? (int)i1 : (int)i1 - d.n1;
  w.k2 = (int)i2 <= d.n2 / 2 ? (int)i2 : (int)i2 - d.n2;
  w.k3 = (int)i3;
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

template <class T, class WV>
__device__ __forceinline__ void leray_apply(const WV& w, cplx<T>& a, cplx<T>& b, cplx<T>& c) {
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

// k'.x for the three components (complex)
template <class T, class WV> __device__ __forceinline__ cplx<T> kdot(const WV& w, cplx<T> a, cplx<T> b, cplx<T> c) {
  const T q1 = T(w.p1), q2 = T(w.p2), q3 = T(w.p3);
  return mk<T>(q1 * a.x + q2 * b.x + q3 * c.x, q1 * a.y + q2 * b.y + q3 * c.y);
}
template <class T, class WV> __device__ __forceinline__ T ksq_of(const WV& w) {
  return T(w.k1) * T(w.k1) + T(w.k2) * T(w.k2) + T(w.k3) * T(w.k3);
}

// x = K x for kmode 0 / 1 / 2
template <class T, class WV>
__device__ __forceinline__ void kop_apply(int kmode, T rw, const WV& w, cplx<T>& a, cplx<T>& b, cplx<T>& c) {
  if (kmode == 1) {
    leray_apply<T>(w, a, b, c);
  } else if (kmode == 2) {
    const T ksq = ksq_of<T>(w);
    const T kpsq = T(w.p1) * T(w.p1) + T(w.p2) * T(w.p2) + T(w.p3) * T(w.p3);
    const T num = rw * (ksq + T(1));
    const T den = ksq + num * kpsq;
    if (den > T(0)) {
      const T q = num / den;
      const cplx<T> d = kdot<T>(w, a, b, c);
      const T q1 = q * T(w.p1), q2 = q * T(w.p2), q3 = q * T(w.p3);
      a = mk<T>(a.x - q1 * d.x, a.y - q1 * d.y);
      b = mk<T>(b.x - q2 * d.x, b.y - q2 * d.y);
      c = mk<T>(c.x - q3 * d.x, c.y - q3 * d.y);
    }
  }
}

// the weight s of K^-1 = I + s k'k'^T (kmode 2; 0 otherwise and at k = 0)
template <class T, class WV> __device__ __forceinline__ T kinv_s(int kmode, T rw, const WV& w) {
  if (kmode != 2) return T(0);
  const T ksq = ksq_of<T>(w);
  return ksq > T(0) ? rw * (ksq + T(1)) / ksq : T(0);
}
// Re(x . conj y) + s Re((k'.x) conj(k'.y)): <K^-1 x, y> per mode (s = 0: the plain product)
template <class T, class WV>
__device__ __forceinline__ T kinv_dot(T s, const WV& w, const cplx<T> (&x)[3], const cplx<T> (&y)[3]) {
  T e = x[0].x * y[0].x + x[0].y * y[0].y + x[1].x * y[1].x + x[1].y * y[1].y + x[2].x * y[2].x + x[2].y * y[2].y;
  if (s != T(0)) {
    const cplx<T> dx = kdot<T>(w, x[0], x[1], x[2]), dy = kdot<T>(w, y[0], y[1], y[2]);
    e += s * (dx.x * dy.x + dx.y * dy.y);
  }
  return e;
}
// a(k) |x|^2, plus rw (|k|^2 + 1) |k'.x|^2 for kmode 2: the regularisation density divided by beta_v
template <class T, class WV>
__device__ __forceinline__ T reg_density(int regnorm, int kmode, T rw, const WV& w, const cplx<T> (&x)[3]) {
  const T ksq = ksq_of<T>(w);
  const T a = regnorm == 2 ? ksq * ksq : ksq;
  T e = a * (x[0].x * x[0].x + x[0].y * x[0].y + x[1].x * x[1].x + x[1].y * x[1].y + x[2].x * x[2].x +
             x[2].y * x[2].y);
  if (kmode == 2) {
    const cplx<T> d = kdot<T>(w, x[0], x[1], x[2]);
    e += rw * (ksq + T(1)) * (d.x * d.x + d.y * d.y);
  }
  return e;
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

// V = K V (kmode 1: Leray, 2: H1-div)
template <class T>
__global__ void k_spec_kop(cplx<T>* __restrict__ V0, cplx<T>* __restrict__ V1, cplx<T>* __restrict__ V2, int kmode,
                           T rw, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.Ns) return;
  const Wave w = wavenumbers(idx, d);
  cplx<T> a = V0[idx], b = V1[idx], c = V2[idx];
  kop_apply<T>(kmode, rw, w, a, b, c);
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
__global__ void k_spec_combine(const cplx<T>* __restrict__ V, cplx<T>* __restrict__ B, int regnorm, int kmode,
                               T rw, T beta, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.Ns) return;
  const Wave w = wavenumbers(idx, d);
  const long long s = d.Ns;
  cplx<T> b0 = B[idx], b1 = B[s + idx], b2 = B[2 * s + idx];
  kop_apply<T>(kmode, rw, w, b0, b1, b2);
  const T f = beta * reg_symbol<T>(w, regnorm);
  const cplx<T> v0 = V[idx], v1 = V[s + idx], v2 = V[2 * s + idx];
  B[idx] = mk<T>(f * v0.x + b0.x, f * v0.y + b0.y);
  B[s + idx] = mk<T>(f * v1.x + b1.x, f * v1.y + b1.y);
  B[2 * s + idx] = mk<T>(f * v2.x + b2.x, f * v2.y + b2.y);
}

// B = V + K^ B (V already multiplied by its symbol)
template <class T>
__global__ void k_spec_addk(const cplx<T>* __restrict__ V, cplx<T>* __restrict__ B, int kmode, T rw, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.Ns) return;
  const Wave w = wavenumbers(idx, d);
  const long long s = d.Ns;
  cplx<T> b0 = B[idx], b1 = B[s + idx], b2 = B[2 * s + idx];
  kop_apply<T>(kmode, rw, w, b0, b1, b2);
  const cplx<T> v0 = V[idx], v1 = V[s + idx], v2 = V[2 * s + idx];
  B[idx] = mk<T>(v0.x + b0.x, v0.y + b0.y);
  B[s + idx] = mk<T>(v1.x + b1.x, v1.y + b1.y);
  B[2 * s + idx] = mk<T>(v2.x + b2.x, v2.y + b2.y);
}

// V = f(k) S in FP64, rounded once to FP32: f = scale a(k) (mode 0) or -|k|^2 (mode 2)
__global__ void k_symbol_f64_to_f32(const cplx<double>* __restrict__ S, cplx<float>* __restrict__ V, int mode,
                                    int regnorm, double scale, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.Ns) return;
  const Wave w = wavenumbers(idx, d);
  const double f = mode == 0 ? scale * reg_symbol<double>(w, regnorm)
                             : -(double(w.k1) * w.k1 + double(w.k2) * w.k2 + double(w.k3) * w.k3);
  const cplx<double> x = S[idx];
  V[idx] = mk<float>(float(x.x * f), float(x.y * f));
}

__global__ void k_f32_to_f64(const float* __restrict__ x, double* __restrict__ y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = double(x[i]);
}

// sum over the half spectrum with weight 1 on the k3 = 0 and k3 = n3/2 planes and 2 elsewhere (Parseval)
template <class T>
__global__ void __launch_bounds__(256) k_spec_reg_partial(const cplx<T>* __restrict__ V, int regnorm, int kmode,
                                                          T rw, Dims d, double* __restrict__ partials) {
  Acc<T> acc;
  const long long s = d.Ns;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < s;
       idx += (long long)gridDim.x * blockDim.x) {
    const Wave w = wavenumbers(idx, d);
    const T wt = (w.k3 == 0 || 2 * w.k3 == d.n3) ? T(1) : T(2);
    const cplx<T> x[3] = {V[idx], V[s + idx], V[2 * s + idx]};
    acc.add(wt * reg_density<T>(regnorm, kmode, rw, w, x));
  }
  __shared__ double red[256 / 32];
  double t0 = acc.value();
  for (int o = 16; o > 0; o >>= 1) t0 += __shfl_down_sync(0xffffffffu, t0, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t0;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    partials[blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------------------------------------------------------
// Fourier-domain PCG / Gauss-Newton vector kernels. The solver keeps v, g, r, s, vt as half spectra (3 components,
// component stride Ns); beta A, M^-1 and K are then exact diagonal multiplies on these master copies, and inner
// products follow from Parseval: <a, b> = h1 h2 h3 / N sum_k w(k3) Re(a^ conj b^), w = 1 on the k3 = 0 and
// k3 = n3/2 planes and 2 elsewhere. Grid-stride over the half spectrum with 32-bit indices; FP64 partial sums,
// one slot per block and value (partials[v * kReduceBlocks + block]).
struct HWave {
  int k1, k2, k3, p1, p2, p3;
  double w;  // Parseval weight
};

__device__ __forceinline__ HWave hwave(unsigned j, const Dims& d) {
  HWave h;
  const unsigned t = d.by_n3h.div(j);
  const unsigned i3 = j - t * (unsigned)d.n3h;
  const unsigned i1 = d.by_n2.div(t);
  const unsigned i2 = t - i1 * (unsigned)d.n2;
  h.k1 = (int)i1 <= d.n1 / 2 ? (int)i1 : (int)i1 - d.n1;
  h.k2 = (int)i2 <= d.n2 / 2 ? (int)i2 : (int)i2 - d.n2;
  h.k3 = (int)i3;
  h.p1 = (2 * h.k1 == d.n1) ? 0 : h.k1;
  h.p2 = (2 * h.k2 == d.n2) ? 0 : h.k2;
  h.p3 = (2 * h.k3 == d.n3) ? 0 : h.k3;
  h.w = (h.k3 == 0 || 2 * h.k3 == d.n3) ? 1.0 : 2.0;
  return h;
}

template <class T> __device__ __forceinline__ T hsym(const HWave& h, int regnorm) {
  const T ksq = T(h.k1) * T(h.k1) + T(h.k2) * T(h.k2) + T(h.k3) * T(h.k3);
  return regnorm == 2 ? ksq * ksq : ksq;
}


template <class T> __device__ __forceinline__ T csq(cplx<T> a) { return a.x * a.x + a.y * a.y; }
template <class T> __device__ __forceinline__ T cre(cplx<T> a, cplx<T> b) { return a.x * b.x + a.y * b.y; }

// M^-1 symbol 1/(beta a) (1 where a = 0); FP32 uses the correctly rounded reciprocal intrinsic
__device__ __forceinline__ float precond_sym(float ba, float a) { return a > 0.f ? __frcp_rn(ba) : 1.f; }
__device__ __forceinline__ double precond_sym(double ba, double a) { return a > 0.0 ? 1.0 / ba : 1.0; }

template <class T, int V>
__device__ __forceinline__ void block_reduce_v(const Acc<T> (&accs)[V], double* __restrict__ partials) {
  __shared__ double red[V][32];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    double a = accs[v].value();
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) red[v][threadIdx.x >> 5] = a;
  }
  __syncthreads();
  if (threadIdx.x < V) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[threadIdx.x][i];
    partials[threadIdx.x * kReduceBlocks + blockIdx.x] = t;
  }
}

#define HLOOP for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < (unsigned)d.Ns; j += gridDim.x * blockDim.x)

// G = beta a V + K B (V may be null: v = 0); partial ||G||^2
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 4) k_sp_grad(const cplx<T>* __restrict__ V, const cplx<T>* __restrict__ B,
                                                 cplx<T>* __restrict__ G, int regnorm, int kmode, T rw, T beta,
                                                 Dims d, double* __restrict__ partials) {
  const long long s = d.Ns;
  Acc<T> acc[1];
  HLOOP {
    const HWave h = hwave(j, d);
    cplx<T> b0 = B[j], b1 = B[s + j], b2 = B[2 * s + j];
    kop_apply<T>(kmode, rw, h, b0, b1, b2);
    if (V) {
      const T f = beta * hsym<T>(h, regnorm);
      const cplx<T> v0 = V[j], v1 = V[s + j], v2 = V[2 * s + j];
      b0 = mk<T>(fma(f, v0.x, b0.x), fma(f, v0.y, b0.y));
      b1 = mk<T>(fma(f, v1.x, b1.x), fma(f, v1.y, b1.y));
      b2 = mk<T>(fma(f, v2.x, b2.x), fma(f, v2.y, b2.y));
    }
    G[j] = b0;
    G[s + j] = b1;
    G[2 * s + j] = b2;
    acc[0].add(T(h.w) * (csq<T>(b0) + csq<T>(b1) + csq<T>(b2)));
  }
  block_reduce_v<T, 1>(acc, partials);
}

// PCG start (Alg. 2): R = -G, S = Z = M^-1 R, Vt = 0; partials <K^-1 R, Z>, ||R||^2, <K^-1 S, beta A S>
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 4) k_sp_pcg0(const cplx<T>* __restrict__ G, cplx<T>* __restrict__ R,
                                                 cplx<T>* __restrict__ S, cplx<T>* __restrict__ Vt, int regnorm,
                                                 int kmode, T rw, T beta, Dims d, double* __restrict__ partials) {
  const long long s = d.Ns;
  Acc<T> acc[3];
  HLOOP {
    const HWave h = hwave(j, d);
    const T a = hsym<T>(h, regnorm);
    const T ba = beta * a;
    const T m = precond_sym(ba, a);
    const T sk = kinv_s<T>(kmode, rw, h);
    cplx<T> rv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cplx<T> g = G[c * s + j];
      const cplx<T> r = mk<T>(-g.x, -g.y);
      rv[c] = r;
      R[c * s + j] = r;
      S[c * s + j] = mk<T>(m * r.x, m * r.y);
      Vt[c * s + j] = mk<T>(T(0), T(0));
    }
    const T rr = T(h.w) * (csq<T>(rv[0]) + csq<T>(rv[1]) + csq<T>(rv[2]));
    const T rkr = T(h.w) * kinv_dot<T>(sk, h, rv, rv);
    acc[0].add(m * rkr);
    acc[1].add(rr);
    acc[2].add(ba * m * m * rkr);
  }
  block_reduce_v<T, 3>(acc, partials);
}

// PCG update: H S = beta a S + K Bt; R -= kappa H S; Vt += kappa S; partials ||R||^2, <K^-1 R, M^-1 R>
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 4) k_sp_pcg_step(const cplx<T>* __restrict__ S, const cplx<T>* __restrict__ Bt,
                                                     cplx<T>* __restrict__ R, cplx<T>* __restrict__ Vt, T kappa,
                                                     int regnorm, int kmode, T rw, T beta, Dims d,
                                                     double* __restrict__ partials, const double* __restrict__ ps) {
  if (ps) {  // device-driven PCG: kappa from the state block; nothing to do once the iteration has ended
    if (ps[kPcgDone] != 0.0) return;
    kappa = T(ps[kPcgKappa]);
  }
  const long long s = d.Ns;
  Acc<T> acc[2];
  HLOOP {
    const HWave h = hwave(j, d);
    const T a = hsym<T>(h, regnorm);
    const T ba = beta * a;
    const T m = precond_sym(ba, a);
    cplx<T> b0 = Bt[j], b1 = Bt[s + j], b2 = Bt[2 * s + j];
    kop_apply<T>(kmode, rw, h, b0, b1, b2);
    const cplx<T> bb[3] = {b0, b1, b2};
    cplx<T> rv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cplx<T> sv = S[c * s + j];
      const cplx<T> hs = mk<T>(fma(ba, sv.x, bb[c].x), fma(ba, sv.y, bb[c].y));
      cplx<T> r = R[c * s + j];
      r = mk<T>(fma(-kappa, hs.x, r.x), fma(-kappa, hs.y, r.y));
      R[c * s + j] = r;
      rv[c] = r;
      cplx<T> vt = Vt[c * s + j];
      Vt[c * s + j] = mk<T>(fma(kappa, sv.x, vt.x), fma(kappa, sv.y, vt.y));
    }
    acc[0].add(T(h.w) * (csq<T>(rv[0]) + csq<T>(rv[1]) + csq<T>(rv[2])));
    acc[1].add(m * T(h.w) * kinv_dot<T>(kinv_s<T>(kmode, rw, h), h, rv, rv));
  }
  block_reduce_v<T, 2>(acc, partials);
}

// PCG direction: S = M^-1 R + mu S; partial <K^-1 S, beta A S>
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 4) k_sp_pcg_dir(const cplx<T>* __restrict__ R, cplx<T>* __restrict__ S, T mu,
                                                    int regnorm, int kmode, T rw, T beta, Dims d,
                                                    double* __restrict__ partials, const double* __restrict__ ps) {
  if (ps) {
    if (ps[kPcgDone] != 0.0) return;
    mu = T(ps[kPcgMu]);
  }
  const long long s = d.Ns;
  Acc<T> acc[1];
  HLOOP {
    const HWave h = hwave(j, d);
    const T a = hsym<T>(h, regnorm);
    const T ba = beta * a;
    const T m = precond_sym(ba, a);
    cplx<T> sw[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cplx<T> r = R[c * s + j];
      cplx<T> sv = S[c * s + j];
      sv = mk<T>(fma(mu, sv.x, m * r.x), fma(mu, sv.y, m * r.y));
      S[c * s + j] = sv;
      sw[c] = sv;
    }
    acc[0].add(T(h.w) * ba * kinv_dot<T>(kinv_s<T>(kmode, rw, h), h, sw, sw));
  }
  block_reduce_v<T, 1>(acc, partials);
}

// projection Vt = K Vt under div v = 0 (kmode 1), then partial <K^-1 G, Vt> (the slope of J along Vt)
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 4) k_sp_project_dot(const cplx<T>* __restrict__ G, cplx<T>* __restrict__ Vt,
                                                        int kmode, T rw, Dims d, double* __restrict__ partials) {
  const long long s = d.Ns;
  Acc<T> acc[1];
  HLOOP {
    const HWave h = hwave(j, d);
    cplx<T> v0 = Vt[j], v1 = Vt[s + j], v2 = Vt[2 * s + j];
    if (kmode == 1) {
      leray_apply<T>(h, v0, v1, v2);
      Vt[j] = v0;
      Vt[s + j] = v1;
      Vt[2 * s + j] = v2;
    }
    const cplx<T> gv[3] = {G[j], G[s + j], G[2 * s + j]};
    const cplx<T> vv[3] = {v0, v1, v2};
    acc[0].add(T(h.w) * kinv_dot<T>(kinv_s<T>(kmode, rw, h), h, gv, vv));
  }
  block_reduce_v<T, 1>(acc, partials);
}

// line-search trial: Vtr = V + alpha Vt (also copied to Sc, the work array of the inverse transform);
// partial sum_k w a(k) |Vtr|^2 (the regularisation value)
template <class T>
__global__ void __launch_bounds__(256) k_sp_trial(const cplx<T>* __restrict__ V, const cplx<T>* __restrict__ Vt,
                                                  cplx<T>* __restrict__ Vtr, cplx<T>* __restrict__ Sc, T alpha_h,
                                                  const double* __restrict__ alpha_dev, int regnorm, int kmode, T rw,
                                                  Dims d, double* __restrict__ partials) {
  const long long s = d.Ns;
  const T alpha = alpha_dev ? T(*alpha_dev) : alpha_h;
  Acc<T> acc[1];
  HLOOP {
    const HWave h = hwave(j, d);
    cplx<T> xs[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cplx<T> v = V[c * s + j], t = Vt[c * s + j];
      const cplx<T> x = mk<T>(fma(alpha, t.x, v.x), fma(alpha, t.y, v.y));
      Vtr[c * s + j] = x;
      Sc[c * s + j] = x;
      xs[c] = x;
    }
    acc[0].add(T(h.w) * reg_density<T>(regnorm, kmode, rw, h, xs));
  }
  block_reduce_v<T, 1>(acc, partials);
}

// partial sum_k w a(k) |V|^2 and a copy of V into Sc (used for a nonzero initial guess)
template <class T>
__global__ void __launch_bounds__(256) k_sp_copy_reg(const cplx<T>* __restrict__ V, cplx<T>* __restrict__ Sc,
                                                     int regnorm, int kmode, T rw, Dims d,
                                                     double* __restrict__ partials) {
  const long long s = d.Ns;
  Acc<T> acc[1];
  HLOOP {
    const HWave h = hwave(j, d);
    cplx<T> xs[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cplx<T> x = V[c * s + j];
      if (Sc) Sc[c * s + j] = x;
      xs[c] = x;
    }
    acc[0].add(T(h.w) * reg_density<T>(regnorm, kmode, rw, h, xs));
  }
  block_reduce_v<T, 1>(acc, partials);
}
// ---------------------------------------------------------------------------------------------------------------
// Two-level preconditioner (Sec. 2.3.3) on the split system I + R^-1/2 H_data R^-1/2, R = beta A (zero mode 1):
// spectral transfer between the fine half spectrum and the half-resolution one (a mode moves iff 2|k_a| < n_a of
// the coarse grid, i.e. the coarse Nyquist modes are dropped), the scaled operator pieces of the nested CG on the
// coarse grid, and the assembly z = R^-1/2 (y_H + P x) of the preconditioned residual.
__device__ __forceinline__ bool on_coarse(const HWave& h, const Dims& dc) {
  return 2 * abs(h.k1) < dc.n1 && 2 * abs(h.k2) < dc.n2 && 2 * h.k3 < dc.n3;
}
__device__ __forceinline__ unsigned index_of(const HWave& h, const Dims& d) {
  const unsigned i1 = (unsigned)(h.k1 < 0 ? h.k1 + d.n1 : h.k1);
  const unsigned i2 = (unsigned)(h.k2 < 0 ? h.k2 + d.n2 : h.k2);
  return (i1 * (unsigned)d.n2 + i2) * (unsigned)d.n3h + (unsigned)h.k3;
}
// (beta a(k))^-1/2, 1 at a = 0
template <class T> __device__ __forceinline__ T split_sym(const HWave& h, int regnorm, T beta) {
  const T a = hsym<T>(h, regnorm);
  return a > T(0) ? T(1) / sqrt(beta * a) : T(1);
}

#define CLOOP for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < (unsigned)dc.Ns; j += gridDim.x * blockDim.x)
#define FLOOP for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < (unsigned)df.Ns; j += gridDim.x * blockDim.x)

// coarse F = scale * (split ? R^-1/2 : 1) * (fine R restricted); optional copies P = F, X = 0;
// partials ||F||^2 and <K^-1 F, F> (coarse Parseval weights)
template <class T>
__global__ void __launch_bounds__(256) k_tl_restrict(const cplx<T>* __restrict__ R, cplx<T>* __restrict__ F,
                                                     cplx<T>* __restrict__ P, cplx<T>* __restrict__ X, int ncomp,
                                                     Dims df, Dims dc, int split, int regnorm, T beta, int kmode,
                                                     T rw, T scale, double* __restrict__ partials) {
  Acc<T> acc[2];
  CLOOP {
    const HWave h = hwave(j, dc);
    const bool keep = on_coarse(h, dc);
    const unsigned jf = keep ? index_of(h, df) : 0u;
    const T f = scale * (split ? split_sym<T>(h, regnorm, beta) : T(1));
    cplx<T> x[3] = {mk<T>(T(0), T(0)), mk<T>(T(0), T(0)), mk<T>(T(0), T(0))};
    for (int c = 0; c < ncomp; ++c) {
      if (keep) {
        const cplx<T> r = R[(long long)c * df.Ns + jf];
        x[c] = mk<T>(f * r.x, f * r.y);
      }
      F[(long long)c * dc.Ns + j] = x[c];
      if (P) P[(long long)c * dc.Ns + j] = x[c];
      if (X) X[(long long)c * dc.Ns + j] = mk<T>(T(0), T(0));
    }
    if (ncomp == 3) {
      acc[0].add(T(h.w) * (csq<T>(x[0]) + csq<T>(x[1]) + csq<T>(x[2])));
      acc[1].add(T(h.w) * kinv_dot<T>(kinv_s<T>(kmode, rw, h), h, x, x));
    }
  }
  block_reduce_v<T, 2>(acc, partials);
}

// U = R^-1/2 P (coarse; U is the input of the inverse transforms)
template <class T>
__global__ void __launch_bounds__(256) k_tl_scale(const cplx<T>* __restrict__ P, cplx<T>* __restrict__ U, Dims dc,
                                                  int regnorm, T beta) {
  CLOOP {
    const HWave h = hwave(j, dc);
    const T f = split_sym<T>(h, regnorm, beta);
    for (int c = 0; c < 3; ++c) {
      const cplx<T> p = P[(long long)c * dc.Ns + j];
      U[(long long)c * dc.Ns + j] = mk<T>(f * p.x, f * p.y);
    }
  }
}

// HP = P + R^-1/2 K Bt (Bt: transform of the data term at U = R^-1/2 P); partial <K^-1 HP, P>
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 4) k_tl_apply(const cplx<T>* __restrict__ P, const cplx<T>* __restrict__ Bt,
                                                  cplx<T>* __restrict__ HP, Dims dc, int regnorm, T beta, int kmode,
                                                  T rw, double* __restrict__ partials) {
  Acc<T> acc[1];
  CLOOP {
    const HWave h = hwave(j, dc);
    const T f = split_sym<T>(h, regnorm, beta);
    cplx<T> b0 = Bt[j], b1 = Bt[dc.Ns + j], b2 = Bt[2 * dc.Ns + j];
    kop_apply<T>(kmode, rw, h, b0, b1, b2);
    const cplx<T> bb[3] = {b0, b1, b2};
    cplx<T> hp[3], pv[3];
    for (int c = 0; c < 3; ++c) {
      pv[c] = P[(long long)c * dc.Ns + j];
      hp[c] = mk<T>(fma(f, bb[c].x, pv[c].x), fma(f, bb[c].y, pv[c].y));
      HP[(long long)c * dc.Ns + j] = hp[c];
    }
    acc[0].add(T(h.w) * kinv_dot<T>(kinv_s<T>(kmode, rw, h), h, hp, pv));
  }
  block_reduce_v<T, 1>(acc, partials);
}

// X += alpha P, Rr -= alpha HP; partials ||Rr||^2 and <K^-1 Rr, Rr>
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 4) k_tl_update(cplx<T>* __restrict__ X, cplx<T>* __restrict__ Rr,
                                                   const cplx<T>* __restrict__ P, const cplx<T>* __restrict__ HP,
                                                   T alpha, Dims dc, int kmode, T rw, double* __restrict__ partials) {
  Acc<T> acc[2];
  CLOOP {
    const HWave h = hwave(j, dc);
    cplx<T> rv[3];
    for (int c = 0; c < 3; ++c) {
      const long long o = (long long)c * dc.Ns + j;
      const cplx<T> p = P[o], hp = HP[o];
      cplx<T> x = X[o], r = Rr[o];
      X[o] = mk<T>(fma(alpha, p.x, x.x), fma(alpha, p.y, x.y));
      r = mk<T>(fma(-alpha, hp.x, r.x), fma(-alpha, hp.y, r.y));
      Rr[o] = r;
      rv[c] = r;
    }
    acc[0].add(T(h.w) * (csq<T>(rv[0]) + csq<T>(rv[1]) + csq<T>(rv[2])));
    acc[1].add(T(h.w) * kinv_dot<T>(kinv_s<T>(kmode, rw, h), h, rv, rv));
  }
  block_reduce_v<T, 2>(acc, partials);
}

// P = Rr + mu P
template <class T>
__global__ void __launch_bounds__(256) k_tl_dir2(const cplx<T>* __restrict__ Rr, cplx<T>* __restrict__ P, T mu,
                                                 Dims dc) {
  CLOOP {
    for (int c = 0; c < 3; ++c) {
      const long long o = (long long)c * dc.Ns + j;
      const cplx<T> r = Rr[o], p = P[o];
      P[o] = mk<T>(fma(mu, p.x, r.x), fma(mu, p.y, r.y));
    }
  }
}

// fine Z = R^-1/2 (y with its coarse modes replaced by scale * X), y = R^-1/2 R; partial <K^-1 R, Z>
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 4) k_tl_prolong(const cplx<T>* __restrict__ R, const cplx<T>* __restrict__ X,
                                                    cplx<T>* __restrict__ Z, Dims df, Dims dc, int regnorm, T beta,
                                                    int kmode, T rw, T scale, double* __restrict__ partials) {
  Acc<T> acc[1];
  FLOOP {
    const HWave h = hwave(j, df);
    const T f = split_sym<T>(h, regnorm, beta);
    const bool low = on_coarse(h, dc);
    const unsigned jc = low ? index_of(h, dc) : 0u;
    cplx<T> rv[3], zv[3];
    for (int c = 0; c < 3; ++c) {
      rv[c] = R[(long long)c * df.Ns + j];
      cplx<T> y = low ? X[(long long)c * dc.Ns + jc] : rv[c];
      const T g = low ? scale * f : f * f;
      zv[c] = mk<T>(g * y.x, g * y.y);
      Z[(long long)c * df.Ns + j] = zv[c];
    }
    acc[0].add(T(h.w) * kinv_dot<T>(kinv_s<T>(kmode, rw, h), h, rv, zv));
  }
  block_reduce_v<T, 1>(acc, partials);
}

// outer direction with an explicit preconditioned residual: S = Z + mu S; partial <K^-1 S, beta A S>
template <class T>
__global__ void __launch_bounds__(256) k_tl_dir(const cplx<T>* __restrict__ Z, cplx<T>* __restrict__ S, T mu,
                                                Dims df, int regnorm, T beta, int kmode, T rw,
                                                double* __restrict__ partials) {
  Acc<T> acc[1];
  FLOOP {
    const HWave h = hwave(j, df);
    const T ba = beta * hsym<T>(h, regnorm);
    cplx<T> sw[3];
    for (int c = 0; c < 3; ++c) {
      const long long o = (long long)c * df.Ns + j;
      const cplx<T> z = Z[o], sv = S[o];
      sw[c] = mk<T>(fma(mu, sv.x, z.x), fma(mu, sv.y, z.y));
      S[o] = sw[c];
    }
    acc[0].add(T(h.w) * ba * kinv_dot<T>(kinv_s<T>(kmode, rw, h), h, sw, sw));
  }
  block_reduce_v<T, 1>(acc, partials);
}
#undef CLOOP
#undef FLOOP
#undef HLOOP

static inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }
// form of K (0 identity, 1 Leray, 2 H1-div) and rw = beta_w / beta_v
static inline int kmode_of(const claire_ctx* c) { return c->o.divfree ? 1 : (c->o.beta_w > 0.0 ? 2 : 0); }
static inline double rw_of(const claire_ctx* c) { return c->o.beta_w > 0.0 ? c->o.beta_w / c->o.beta : 0.0; }

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
template <class T> claire_status spec_kop(claire_ctx* c, cplx<T>* V0, cplx<T>* V1, cplx<T>* V2, cudaStream_t st) {
  c->prof_begin("spec_kop", st);
  k_spec_kop<T><<<blocks_for(c->d.Ns), kThreads, 0, st>>>(V0, V1, V2, kmode_of(c), T(rw_of(c)), c->d);
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
template <class T> claire_status spec_addk(claire_ctx* c, const cplx<T>* V, cplx<T>* B, cudaStream_t st) {
  c->prof_begin("spec_addk", st);
  k_spec_addk<T><<<blocks_for(c->d.Ns), kThreads, 0, st>>>(V, B, kmode_of(c), T(rw_of(c)), c->d);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
claire_status symbol_r2c_f64(claire_ctx* c, const float* f, double* fd, cplx<double>* Sd, cplx<float>* V, int mode,
                             double scale, cudaStream_t st) {
  const long long n = c->d.N;
  c->prof_begin("f32_to_f64", st);
  const long long nb = (n + kThreads - 1) / kThreads;
  k_f32_to_f64<<<(unsigned)(nb < 4864 ? nb : 4864), kThreads, 0, st>>>(f, fd, n);
  CL_LAUNCHED(c);
  CL_TRY(fft_r2c<double>(c, fd, Sd, st));
  c->prof_begin("symbol_f64_to_f32", st);
  k_symbol_f64_to_f32<<<blocks_for(c->d.Ns), kThreads, 0, st>>>(Sd, V, mode, c->o.regnorm, scale, c->d);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T> claire_status spec_combine(claire_ctx* c, const cplx<T>* V, cplx<T>* B, cudaStream_t st) {
  c->prof_begin("spec_combine", st);
  k_spec_combine<T><<<blocks_for(c->d.Ns), kThreads, 0, st>>>(V, B, c->o.regnorm, kmode_of(c), T(rw_of(c)),
                                                               T(c->o.beta), c->d);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T> claire_status spec_reg_partial(claire_ctx* c, const cplx<T>* V, double* partials, cudaStream_t st) {
  c->prof_begin("spec_reg_partial", st);
  k_spec_reg_partial<T><<<kReduceBlocks, 256, 0, st>>>(V, c->o.regnorm, kmode_of(c), T(rw_of(c)), c->d, partials);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

template <class T>
claire_status sp_grad(claire_ctx* c, const cplx<T>* V, const cplx<T>* B, cplx<T>* G, double* partials,
                      cudaStream_t st) {
  c->prof_begin("sp_grad", st);
  k_sp_grad<T><<<kReduceBlocks, 256, 0, st>>>(V, B, G, c->o.regnorm, kmode_of(c), T(rw_of(c)), T(c->o.beta), c->d,
                                              partials);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T>
claire_status sp_pcg0(claire_ctx* c, const cplx<T>* G, cplx<T>* R, cplx<T>* S, cplx<T>* Vt, double* partials,
                      cudaStream_t st) {
  c->prof_begin("sp_pcg0", st);
  k_sp_pcg0<T><<<kReduceBlocks, 256, 0, st>>>(G, R, S, Vt, c->o.regnorm, kmode_of(c), T(rw_of(c)), T(c->o.beta), c->d,
                                              partials);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T>
claire_status sp_pcg_step(claire_ctx* c, const cplx<T>* S, const cplx<T>* Bt, cplx<T>* R, cplx<T>* Vt, double kappa,
                          double* partials, cudaStream_t st, const double* ps) {
  c->prof_begin("sp_pcg_step", st);
  k_sp_pcg_step<T><<<kReduceBlocks, 256, 0, st>>>(S, Bt, R, Vt, T(kappa), c->o.regnorm, kmode_of(c), T(rw_of(c)),
                                                  T(c->o.beta), c->d, partials, ps);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T>
claire_status sp_pcg_dir(claire_ctx* c, const cplx<T>* R, cplx<T>* S, double mu, double* partials, cudaStream_t st,
                         const double* ps) {
  c->prof_begin("sp_pcg_dir", st);
  k_sp_pcg_dir<T><<<kReduceBlocks, 256, 0, st>>>(R, S, T(mu), c->o.regnorm, kmode_of(c), T(rw_of(c)), T(c->o.beta),
                                                 c->d, partials, ps);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T>
claire_status sp_project_dot(claire_ctx* c, const cplx<T>* G, cplx<T>* Vt, double* partials, cudaStream_t st) {
  c->prof_begin("sp_project_dot", st);
  k_sp_project_dot<T><<<kReduceBlocks, 256, 0, st>>>(G, Vt, kmode_of(c), T(rw_of(c)), c->d, partials);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T>
claire_status sp_trial(claire_ctx* c, const cplx<T>* V, const cplx<T>* Vt, cplx<T>* Vtr, cplx<T>* Sc, double alpha,
                       double* partials, cudaStream_t st, const double* alpha_dev) {
  c->prof_begin("sp_trial", st);
  k_sp_trial<T><<<kReduceBlocks, 256, 0, st>>>(V, Vt, Vtr, Sc, T(alpha), alpha_dev, c->o.regnorm, kmode_of(c),
                                               T(rw_of(c)), c->d, partials);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T>
claire_status sp_copy_reg(claire_ctx* c, const cplx<T>* V, cplx<T>* Sc, double* partials, cudaStream_t st) {
  c->prof_begin("sp_copy_reg", st);
  k_sp_copy_reg<T><<<kReduceBlocks, 256, 0, st>>>(V, Sc, c->o.regnorm, kmode_of(c), T(rw_of(c)), c->d, partials);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

template <class T>
claire_status tl_restrict(claire_ctx* c, claire_ctx* cc, const cplx<T>* R, cplx<T>* F, cplx<T>* P, cplx<T>* X,
                          int ncomp, bool split, double* partials, cudaStream_t st) {
  cc->prof_begin("tl_restrict", st);
  k_tl_restrict<T><<<kReduceBlocks, 256, 0, st>>>(R, F, P, X, ncomp, c->d, cc->d, split ? 1 : 0, c->o.regnorm,
                                                  T(c->o.beta), kmode_of(c), T(rw_of(c)),
                                                  T(double(cc->d.N) / double(c->d.N)), partials);
  CL_LAUNCHED(cc);
  return CLAIRE_OK;
}
template <class T> claire_status tl_scale(claire_ctx* cc, const cplx<T>* P, cplx<T>* U, cudaStream_t st) {
  cc->prof_begin("tl_scale", st);
  k_tl_scale<T><<<kReduceBlocks, 256, 0, st>>>(P, U, cc->d, cc->o.regnorm, T(cc->o.beta));
  CL_LAUNCHED(cc);
  return CLAIRE_OK;
}
template <class T>
claire_status tl_apply(claire_ctx* cc, const cplx<T>* P, const cplx<T>* Bt, cplx<T>* HP, double* partials,
                       cudaStream_t st) {
  cc->prof_begin("tl_apply", st);
  k_tl_apply<T><<<kReduceBlocks, 256, 0, st>>>(P, Bt, HP, cc->d, cc->o.regnorm, T(cc->o.beta), kmode_of(cc),
                                               T(rw_of(cc)), partials);
  CL_LAUNCHED(cc);
  return CLAIRE_OK;
}
template <class T>
claire_status tl_update(claire_ctx* cc, cplx<T>* X, cplx<T>* Rr, const cplx<T>* P, const cplx<T>* HP, double alpha,
                        double* partials, cudaStream_t st) {
  cc->prof_begin("tl_update", st);
  k_tl_update<T><<<kReduceBlocks, 256, 0, st>>>(X, Rr, P, HP, T(alpha), cc->d, kmode_of(cc), T(rw_of(cc)), partials);
  CL_LAUNCHED(cc);
  return CLAIRE_OK;
}
template <class T> claire_status tl_dir2(claire_ctx* cc, const cplx<T>* Rr, cplx<T>* P, double mu, cudaStream_t st) {
  cc->prof_begin("tl_dir2", st);
  k_tl_dir2<T><<<kReduceBlocks, 256, 0, st>>>(Rr, P, T(mu), cc->d);
  CL_LAUNCHED(cc);
  return CLAIRE_OK;
}
template <class T>
claire_status tl_prolong(claire_ctx* c, claire_ctx* cc, const cplx<T>* R, const cplx<T>* X, cplx<T>* Z,
                         double* partials, cudaStream_t st) {
  c->prof_begin("tl_prolong", st);
  k_tl_prolong<T><<<kReduceBlocks, 256, 0, st>>>(R, X, Z, c->d, cc->d, c->o.regnorm, T(c->o.beta), kmode_of(c),
                                                 T(rw_of(c)), T(double(c->d.N) / double(cc->d.N)), partials);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T>
claire_status tl_dir(claire_ctx* c, const cplx<T>* Z, cplx<T>* S, double mu, double* partials, cudaStream_t st) {
  c->prof_begin("tl_dir", st);
  k_tl_dir<T><<<kReduceBlocks, 256, 0, st>>>(Z, S, T(mu), c->d, c->o.regnorm, T(c->o.beta), kmode_of(c),
                                             T(rw_of(c)), partials);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

#define INST(T)                                                                                                   \
  template claire_status sp_grad<T>(claire_ctx*, const cplx<T>*, const cplx<T>*, cplx<T>*, double*, cudaStream_t); \
  template claire_status sp_pcg0<T>(claire_ctx*, const cplx<T>*, cplx<T>*, cplx<T>*, cplx<T>*, double*,           \
                                    cudaStream_t);                                                               \
  template claire_status sp_pcg_step<T>(claire_ctx*, const cplx<T>*, const cplx<T>*, cplx<T>*, cplx<T>*, double,  \
                                        double*, cudaStream_t, const double*);                                   \
  template claire_status sp_pcg_dir<T>(claire_ctx*, const cplx<T>*, cplx<T>*, double, double*, cudaStream_t,      \
                                       const double*);                                                           \
  template claire_status sp_project_dot<T>(claire_ctx*, const cplx<T>*, cplx<T>*, double*, cudaStream_t);        \
  template claire_status sp_trial<T>(claire_ctx*, const cplx<T>*, const cplx<T>*, cplx<T>*, cplx<T>*, double,      \
                                     double*, cudaStream_t, const double*);                                      \
  template claire_status sp_copy_reg<T>(claire_ctx*, const cplx<T>*, cplx<T>*, double*, cudaStream_t);          \
  template claire_status spec_grad<T>(claire_ctx*, const cplx<T>*, cplx<T>*, cplx<T>*, cplx<T>*, cudaStream_t);  \
  template claire_status spec_div<T>(claire_ctx*, const cplx<T>*, const cplx<T>*, const cplx<T>*, cplx<T>*,      \
                                     cudaStream_t);                                                              \
  template claire_status spec_leray<T>(claire_ctx*, cplx<T>*, cplx<T>*, cplx<T>*, cudaStream_t);                 \
  template claire_status spec_kop<T>(claire_ctx*, cplx<T>*, cplx<T>*, cplx<T>*, cudaStream_t);                   \
  template claire_status spec_scale<T>(claire_ctx*, cplx<T>*, int, long long, int, double, cudaStream_t);        \
  template claire_status spec_combine<T>(claire_ctx*, const cplx<T>*, cplx<T>*, cudaStream_t);                   \
  template claire_status spec_addk<T>(claire_ctx*, const cplx<T>*, cplx<T>*, cudaStream_t);                      \
  template claire_status spec_reg_partial<T>(claire_ctx*, const cplx<T>*, double*, cudaStream_t);                \
  template claire_status tl_restrict<T>(claire_ctx*, claire_ctx*, const cplx<T>*, cplx<T>*, cplx<T>*, cplx<T>*,  \
                                        int, bool, double*, cudaStream_t);                                       \
  template claire_status tl_scale<T>(claire_ctx*, const cplx<T>*, cplx<T>*, cudaStream_t);                       \
  template claire_status tl_apply<T>(claire_ctx*, const cplx<T>*, const cplx<T>*, cplx<T>*, double*,            \
                                     cudaStream_t);                                                              \
  template claire_status tl_update<T>(claire_ctx*, cplx<T>*, cplx<T>*, const cplx<T>*, const cplx<T>*, double,  \
                                      double*, cudaStream_t);                                                    \
  template claire_status tl_dir2<T>(claire_ctx*, const cplx<T>*, cplx<T>*, double, cudaStream_t);                \
  template claire_status tl_prolong<T>(claire_ctx*, claire_ctx*, const cplx<T>*, const cplx<T>*, cplx<T>*,      \
                                       double*, cudaStream_t);                                                   \
  template claire_status tl_dir<T>(claire_ctx*, const cplx<T>*, cplx<T>*, double, double*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace claire
