// Length-specialised FFT passes for the pseudo-spectral operators (Sec. 2.3.1). For a line of length L = R1 * R2
// (both known at compile time) each pass is two radix stages with one shared-memory exchange between them:
//
//   stage 1 (butterfly j < R2): x[j + r R2], r < R1  --DFT_R1 (registers)-->  y[j R1 + q]        (shared memory)
//   stage 2 (butterfly j < R1): y[j + r R1] w_L^{r j}, r < R2  --DFT_R2-->    z[j + q R1] = X     (global memory)
//
// (a two-stage Stockham/Cooley-Tukey split; stage 1 reads global memory directly and stage 2 writes it directly,
// so every element crosses HBM once each way per pass). The register DFTs of composite size R = P Q use the
// index maps n = i + Q m, k = k1 + P k2 with internal twiddles w_R^{i k1}, recursively down to hard-coded radix
// 2, 4, 8 butterflies and table-driven radix 3, 5, 7. All twiddles come from host FP64 tables staged in shared
// memory. Strided passes put TI consecutive columns on threadIdx.x (coalesced rows); the contiguous-axis R2C/C2R
// passes put the line on threadIdx.x and pad shared memory by one slot per R1 entries to avoid bank conflicts.
#include "impl.cuh"

namespace claire {
namespace {

template <class T, int SIGN>
__device__ __forceinline__ cplx<T> twid(cplx<T> x, cplx<T> w) {
  return SIGN < 0 ? cmul<T>(x, w) : cmulc<T>(x, w);
}

template <int R> __host__ __device__ constexpr int first_factor() {
  return (R % 8 == 0 && R > 8) ? 8 : (R % 4 == 0 && R > 4) ? 4 : (R % 2 == 0 && R > 2) ? 2 : (R % 3 == 0 && R > 3) ? 3
         : (R % 5 == 0 && R > 5) ? 5 : (R % 7 == 0 && R > 7) ? 7 : R;
}

// DFT of R values in registers; W = exp(-2 pi i t / L), t < L, with R | L.
template <class T, int SIGN, int R, int L>
__device__ __forceinline__ void rdft(cplx<T>* v, const cplx<T>* W) {
  if constexpr (R == 1) {
    return;
  } else if constexpr (R == 2) {
    const cplx<T> a = v[0], b = v[1];
    v[0] = cadd<T>(a, b);
    v[1] = csub<T>(a, b);
  } else if constexpr (R == 4) {
    const cplx<T> a0 = cadd<T>(v[0], v[2]), a1 = csub<T>(v[0], v[2]);
    const cplx<T> a2 = cadd<T>(v[1], v[3]), a3 = mul_i<SIGN, T>(csub<T>(v[1], v[3]));
    v[0] = cadd<T>(a0, a2);
    v[2] = csub<T>(a0, a2);
    v[1] = cadd<T>(a1, a3);
    v[3] = csub<T>(a1, a3);
  } else if constexpr (R == 8) {
    cplx<T> e[4] = {v[0], v[2], v[4], v[6]};
    cplx<T> o[4] = {v[1], v[3], v[5], v[7]};
    rdft<T, SIGN, 4, L>(e, W);
    rdft<T, SIGN, 4, L>(o, W);
    const T s = T(0.70710678118654752440084436210484903928);
    const cplx<T> o1 = SIGN < 0 ? mk<T>((o[1].x + o[1].y) * s, (o[1].y - o[1].x) * s)
                                : mk<T>((o[1].x - o[1].y) * s, (o[1].y + o[1].x) * s);
    const cplx<T> o2 = mul_i<SIGN, T>(o[2]);
    const cplx<T> o3 = SIGN < 0 ? mk<T>((-o[3].x + o[3].y) * s, (-o[3].y - o[3].x) * s)
                                : mk<T>((-o[3].x - o[3].y) * s, (-o[3].y + o[3].x) * s);
    v[0] = cadd<T>(e[0], o[0]);
    v[4] = csub<T>(e[0], o[0]);
    v[1] = cadd<T>(e[1], o1);
    v[5] = csub<T>(e[1], o1);
    v[2] = cadd<T>(e[2], o2);
    v[6] = csub<T>(e[2], o2);
    v[3] = cadd<T>(e[3], o3);
    v[7] = csub<T>(e[3], o3);
  } else if constexpr (R == 3 || R == 5 || R == 7) {
    cplx<T> out[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      cplx<T> acc = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) acc = cadd<T>(acc, twid<T, SIGN>(v[r], W[((r * q) % R) * (L / R)]));
      out[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = out[q];
  } else {
    constexpr int P = first_factor<R>();
    constexpr int Q = R / P;
    static_assert(P * Q == R && P < R, "unsupported radix");
    cplx<T> u[R];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      cplx<T> t[P];
#pragma unroll
      for (int m = 0; m < P; ++m) t[m] = v[i + Q * m];
      rdft<T, SIGN, P, L>(t, W);
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) u[i * P + k1] = (i * k1 == 0) ? t[k1] : twid<T, SIGN>(t[k1], W[(i * k1) * (L / R)]);
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      cplx<T> t[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) t[i] = u[i * P + k1];
      rdft<T, SIGN, Q, L>(t, W);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) v[k1 + P * k2] = t[k2];
    }
  }
}

template <int A, int B> __host__ __device__ constexpr int cmax() { return A > B ? A : B; }

// ---------------------------------------------------------------------------------------------------------------
// Strided axis (in place or src -> dst): line length L = R1 R2 with element stride `inner`; TI columns per CTA.
template <class T, int SIGN, int R1, int R2, int TI>
__global__ void __launch_bounds__(TI * cmax<R1, R2>()) k_fft2_strided(const cplx<T>* src, cplx<T>* dst,
                                                                       long long inner,
                                                                       const cplx<T>* __restrict__ Wg) {
  constexpr int L = R1 * R2;
  constexpr int TT = cmax<R1, R2>();
  __shared__ cplx<T> W[L];
  __shared__ cplx<T> Y[L * TI];
  const int c = threadIdx.x, t = threadIdx.y;
  const long long i0 = (long long)blockIdx.x * TI;
  const bool col_ok = i0 + c < inner;
  const long long off = (long long)blockIdx.y * L * inner + i0 + c;
  for (int k = t * TI + c; k < L; k += TI * TT) W[k] = Wg[k];
  __syncthreads();
  // every global load of the CTA is consumed before the barrier below, so the in-place stores after it are safe
  if (t < R2) {
    cplx<T> v[R1];
#pragma unroll
    for (int r = 0; r < R1; ++r) v[r] = col_ok ? src[off + (long long)(t + r * R2) * inner] : mk<T>(T(0), T(0));
    rdft<T, SIGN, R1, L>(v, W);
#pragma unroll
    for (int q = 0; q < R1; ++q) Y[(t * R1 + q) * TI + c] = v[q];
  }
  __syncthreads();
  if (t < R1 && col_ok) {
    cplx<T> u[R2];
#pragma unroll
    for (int r = 0; r < R2; ++r) {
      const cplx<T> x = Y[(t + r * R1) * TI + c];
      u[r] = (r == 0) ? x : twid<T, SIGN>(x, W[r * t]);
    }
    rdft<T, SIGN, R2, L>(u, W);
#pragma unroll
    for (int q = 0; q < R2; ++q) dst[off + (long long)(t + q * R1) * inner] = u[q];
  }
}

// shared-memory index of entry a of a line with one pad slot per R1 entries
template <int R1> __device__ __forceinline__ int padi(int a) { return a + a / R1; }

// Contiguous axis, forward: real lines of n3 = 2L -> half spectra of L + 1 (see fft.cu for the split formulas).
template <class T, int R1, int R2, int LPC>
__global__ void __launch_bounds__(LPC * cmax<R1, R2>()) k_fft2_z_r2c(const T* __restrict__ in,
                                                                      cplx<T>* __restrict__ out, long long nlines,
                                                                      const cplx<T>* __restrict__ Wn3) {
  constexpr int L = R1 * R2;
  constexpr int TT = cmax<R1, R2>();
  constexpr int S = L + L / R1 + 1;
  __shared__ cplx<T> W[L];
  __shared__ cplx<T> W2[L + 1];
  __shared__ cplx<T> Y[LPC * S];
  const int t = threadIdx.x, l = threadIdx.y;
  const int tid = l * TT + t;
  for (int k = tid; k < L; k += LPC * TT) W[k] = Wn3[2 * k];
  for (int k = tid; k <= L; k += LPC * TT) W2[k] = Wn3[k];
  const long long line = (long long)blockIdx.x * LPC + l;
  const bool ok = line < nlines;
  const cplx<T>* src = reinterpret_cast<const cplx<T>*>(in + line * 2 * L);
  cplx<T>* Yl = Y + l * S;
  __syncthreads();
  if (t < R2) {
    cplx<T> v[R1];
#pragma unroll
    for (int r = 0; r < R1; ++r) v[r] = ok ? src[t + r * R2] : mk<T>(T(0), T(0));
    rdft<T, -1, R1, L>(v, W);
#pragma unroll
    for (int q = 0; q < R1; ++q) Yl[padi<R1>(t * R1 + q)] = v[q];
  }
  __syncthreads();
  cplx<T> u[R2];
  if (t < R1) {
#pragma unroll
    for (int r = 0; r < R2; ++r) {
      const cplx<T> x = Yl[padi<R1>(t + r * R1)];
      u[r] = (r == 0) ? x : twid<T, -1>(x, W[r * t]);
    }
    rdft<T, -1, R2, L>(u, W);
  }
  if constexpr (R1 == TT && 32 % TT == 0) {
    // Thread t holds Z[k], k = t + q R1; the mirrored Z[L - k] is Z[(R1 - t) + (R2 - 1 - q) R1] of thread R1 - t
    // (for t = 0: its own Z[(R2 - q) R1], and Z[0] for k = 0 and k = L), fetched by warp shuffle -- a line's R1
    // threads are consecutive lanes of one warp -- instead of a shared-memory round trip.
    const int lane = tid & 31;
    const int partner = (lane - t) + (R1 - t) % R1;
    cplx<T> zm[R2];
#pragma unroll
    for (int q = 0; q < R2; ++q) {
      const cplx<T> sent = u[R2 - 1 - q];
      const cplx<T> got = mk<T>(__shfl_sync(0xffffffffu, sent.x, partner), __shfl_sync(0xffffffffu, sent.y, partner));
      zm[q] = t == 0 ? u[(R2 - q) % R2] : got;
    }
    if (ok) {
      cplx<T>* dst = out + line * (L + 1);
#pragma unroll
      for (int q = 0; q < R2; ++q) {
        const int k = t + q * R1;
        const cplx<T> zk = u[q], zc = cconj<T>(zm[q]);
        const cplx<T> sum = cadd<T>(zk, zc), dif = csub<T>(zk, zc);
        const cplx<T> wd = cmul<T>(W2[k], dif);
        dst[k] = mk<T>(T(0.5) * (sum.x + wd.y), T(0.5) * (sum.y - wd.x));
      }
      if (t == 0) {
        const cplx<T> zk = u[0], zc = cconj<T>(u[0]);
        const cplx<T> sum = cadd<T>(zk, zc), dif = csub<T>(zk, zc);
        const cplx<T> wd = cmul<T>(W2[L], dif);
        dst[L] = mk<T>(T(0.5) * (sum.x + wd.y), T(0.5) * (sum.y - wd.x));
      }
    }
    return;
  }
  __syncthreads();
  if (t < R1) {
#pragma unroll
    for (int q = 0; q < R2; ++q) Yl[padi<R1>(t + q * R1)] = u[q];
  }
  __syncthreads();
  if (ok) {
    cplx<T>* dst = out + line * (L + 1);
    for (int k = t; k <= L; k += TT) {
      const cplx<T> zk = Yl[padi<R1>(k == L ? 0 : k)];
      const cplx<T> zc = cconj<T>(Yl[padi<R1>(k == 0 ? 0 : L - k)]);
      const cplx<T> sum = cadd<T>(zk, zc), dif = csub<T>(zk, zc);
      const cplx<T> wd = cmul<T>(W2[k], dif);
      dst[k] = mk<T>(T(0.5) * (sum.x + wd.y), T(0.5) * (sum.y - wd.x));
    }
  }
}

// Contiguous axis, inverse: half spectra of L + 1 -> real lines of 2L, times scale.
template <class T, int R1, int R2, int LPC>
__global__ void __launch_bounds__(LPC * cmax<R1, R2>(), 4) k_fft2_z_c2r(const cplx<T>* __restrict__ in,
                                                                      T* __restrict__ out, long long nlines,
                                                                      const cplx<T>* __restrict__ Wn3, T scale) {
  constexpr int L = R1 * R2;
  constexpr int TT = cmax<R1, R2>();
  constexpr int S = L + L / R1 + 1;
  __shared__ cplx<T> W[L];
  __shared__ cplx<T> W2[L + 1];
  __shared__ cplx<T> Y[LPC * S];
  const int t = threadIdx.x, l = threadIdx.y;
  const int tid = l * TT + t;
  for (int k = tid; k < L; k += LPC * TT) W[k] = Wn3[2 * k];
  for (int k = tid; k <= L; k += LPC * TT) W2[k] = Wn3[k];
  const long long line = (long long)blockIdx.x * LPC + l;
  const bool ok = line < nlines;
  cplx<T>* Yl = Y + l * S;
  __syncthreads();
  // Z'[k] = (X[k] + conj X[L-k]) + i exp(+2 pi i k / n3) (X[k] - conj X[L-k]) for the stage-1 inputs k = t + r R2,
  // read straight from global memory. When a line's threads are consecutive lanes of one warp, the mirrored
  // X[L - k] = X[(R2 - t) + (R1 - 1 - r) R2] comes from thread R2 - t by warp shuffle (for t = 0: its own
  // X[(R1 - r) R2], and X[L] for r = 0); otherwise it is read again (another thread's X[k]: an L1 hit).
  cplx<T> v[R1];
  const cplx<T>* src = in + line * (L + 1);
  if constexpr (32 % TT == 0) {
    cplx<T> xs[R1];
#pragma unroll
    for (int r = 0; r < R1; ++r) xs[r] = (ok && t < R2) ? src[t + r * R2] : mk<T>(T(0), T(0));
    const cplx<T> xL = (ok && t == 0) ? src[L] : mk<T>(T(0), T(0));
    const int lane = tid & 31;
    const int partner = (lane - t) + (t < R2 ? (R2 - t) % R2 : t);
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const cplx<T> sent = xs[R1 - 1 - r];
      const cplx<T> got = mk<T>(__shfl_sync(0xffffffffu, sent.x, partner), __shfl_sync(0xffffffffu, sent.y, partner));
      const cplx<T> xk = xs[r];
      const cplx<T> xc = cconj<T>(t == 0 ? (r == 0 ? xL : xs[R1 - r]) : got);
      const cplx<T> sum = cadd<T>(xk, xc), dif = csub<T>(xk, xc);
      const cplx<T> wd = cmulc<T>(dif, W2[t < R2 ? t + r * R2 : 0]);
      v[r] = mk<T>(sum.x - wd.y, sum.y + wd.x);
    }
    if (t < R2) {
      rdft<T, +1, R1, L>(v, W);
#pragma unroll
      for (int q = 0; q < R1; ++q) Yl[padi<R1>(t * R1 + q)] = v[q];
    }
  } else if (t < R2) {
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int k = t + r * R2;
      const cplx<T> xk = ok ? src[k] : mk<T>(T(0), T(0));
      const cplx<T> xc = ok ? cconj<T>(src[L - k]) : mk<T>(T(0), T(0));
      const cplx<T> sum = cadd<T>(xk, xc), dif = csub<T>(xk, xc);
      const cplx<T> wd = cmulc<T>(dif, W2[k]);
      v[r] = mk<T>(sum.x - wd.y, sum.y + wd.x);
    }
    rdft<T, +1, R1, L>(v, W);
#pragma unroll
    for (int q = 0; q < R1; ++q) Yl[padi<R1>(t * R1 + q)] = v[q];
  }
  __syncthreads();
  if (t < R1 && ok) {
    cplx<T> u[R2];
#pragma unroll
    for (int r = 0; r < R2; ++r) {
      const cplx<T> x = Yl[padi<R1>(t + r * R1)];
      u[r] = (r == 0) ? x : twid<T, +1>(x, W[r * t]);
    }
    rdft<T, +1, R2, L>(u, W);
    cplx<T>* dst = reinterpret_cast<cplx<T>*>(out + line * 2 * L);
#pragma unroll
    for (int q = 0; q < R2; ++q) dst[t + q * R1] = mk<T>(u[q].x * scale, u[q].y * scale);
  }
}

template <class T> __host__ __device__ constexpr int strided_ti() { return sizeof(T) == 4 ? 16 : 8; }
template <class T, int TT> __host__ __device__ constexpr int z_lpc() { return (256 / TT) / (sizeof(T) == 4 ? 1 : 2) > 0 ? (256 / TT) / (sizeof(T) == 4 ? 1 : 2) : 1; }

// Tile variants of the specialised FP32 passes, chosen per grid by the autotuner in fft.cu: 0 the default
// columns (strided) or lines (contiguous) per CTA, 1 half as many, 2 twice as many -- where the static shared
// memory (48 KB) and the block size allow, else the default. FP64 passes keep the default.
template <class T, int V> __host__ __device__ constexpr int ti_of() {
  return V == 0 ? strided_ti<T>() : (V == 1 ? strided_ti<T>() / 2 : strided_ti<T>() * 2);
}
template <class T, int R1, int R2, int TI> __host__ __device__ constexpr bool strided_fits() {
  return TI >= 1 && (size_t(R1 * R2) * TI + R1 * R2) * sizeof(cplx<T>) <= 48 * 1024 && TI * cmax<R1, R2>() <= 1024;
}

template <class T, int R1, int R2, int TI>
void launch_strided_ti(int sign, const cplx<T>* src, cplx<T>* dst, long long inner, int outer, const cplx<T>* W,
                       cudaStream_t st) {
  constexpr int TT = cmax<R1, R2>();
  dim3 grid((unsigned)((inner + TI - 1) / TI), (unsigned)outer);
  dim3 block(TI, TT);
  if (sign < 0)
    k_fft2_strided<T, -1, R1, R2, TI><<<grid, block, 0, st>>>(src, dst, inner, W);
  else
    k_fft2_strided<T, +1, R1, R2, TI><<<grid, block, 0, st>>>(src, dst, inner, W);
}

template <class T, int R1, int R2>
void launch_strided(int sign, const cplx<T>* src, cplx<T>* dst, long long inner, int outer, const cplx<T>* W,
                    cudaStream_t st, int var) {
  if constexpr (sizeof(T) == 4) {
    if (var == 1 && strided_fits<T, R1, R2, ti_of<T, 1>()>()) {
      if constexpr (strided_fits<T, R1, R2, ti_of<T, 1>()>())
        launch_strided_ti<T, R1, R2, ti_of<T, 1>()>(sign, src, dst, inner, outer, W, st);
      return;
    }
    if (var == 2 && strided_fits<T, R1, R2, ti_of<T, 2>()>()) {
      if constexpr (strided_fits<T, R1, R2, ti_of<T, 2>()>())
        launch_strided_ti<T, R1, R2, ti_of<T, 2>()>(sign, src, dst, inner, outer, W, st);
      return;
    }
  }
  launch_strided_ti<T, R1, R2, strided_ti<T>()>(sign, src, dst, inner, outer, W, st);
}

template <class T, int R1, int R2, int LPC> __host__ __device__ constexpr bool z_fits() {
  return LPC >= 1 && (size_t(LPC) * (R1 * R2 + R1 * R2 / R1 + 1) + 2 * R1 * R2 + 1) * sizeof(cplx<T>) <= 48 * 1024 &&
         LPC * cmax<R1, R2>() <= 1024;
}
template <class T, int R1, int R2, int V> __host__ __device__ constexpr int lpc_of() {
  return V == 0 ? z_lpc<T, cmax<R1, R2>()>() : (V == 1 ? z_lpc<T, cmax<R1, R2>()>() / 2 : z_lpc<T, cmax<R1, R2>()>() * 2);
}

template <class T, int R1, int R2, int C1, int C2, int V>
bool launch_z_v(int sign, const void* in, void* out, long long nlines, const cplx<T>* Wn3, T scale, cudaStream_t st) {
  if (sign < 0) {
    constexpr int TT = cmax<R1, R2>();
    constexpr int LPC = lpc_of<T, R1, R2, V>();
    if constexpr (z_fits<T, R1, R2, LPC>()) {
      k_fft2_z_r2c<T, R1, R2, LPC><<<dim3((unsigned)((nlines + LPC - 1) / LPC)), dim3(TT, LPC), 0, st>>>(
          static_cast<const T*>(in), static_cast<cplx<T>*>(out), nlines, Wn3);
      return true;
    }
  } else {
    constexpr int TT = cmax<C1, C2>();
    constexpr int LPC = lpc_of<T, C1, C2, V>();
    if constexpr (z_fits<T, C1, C2, LPC>()) {
      k_fft2_z_c2r<T, C1, C2, LPC><<<dim3((unsigned)((nlines + LPC - 1) / LPC)), dim3(TT, LPC), 0, st>>>(
          static_cast<const cplx<T>*>(in), static_cast<T*>(out), nlines, Wn3, scale);
      return true;
    }
  }
  return false;
}

// (R1, R2) of the forward pass; the inverse pass may use another split (C1, C2) of the same length
template <class T, int R1, int R2, int C1 = R1, int C2 = R2>
void launch_z(int sign, const void* in, void* out, long long nlines, const cplx<T>* Wn3, T scale, cudaStream_t st,
              int var) {
  static_assert(R1 * R2 == C1 * C2, "one line length");
  if constexpr (sizeof(T) == 4) {
    if (var == 1 && launch_z_v<T, R1, R2, C1, C2, 1>(sign, in, out, nlines, Wn3, scale, st)) return;
    if (var == 2 && launch_z_v<T, R1, R2, C1, C2, 2>(sign, in, out, nlines, Wn3, scale, st)) return;
  }
  launch_z_v<T, R1, R2, C1, C2, 0>(sign, in, out, nlines, Wn3, scale, st);
}

}  // namespace

// Specialised strided pass for line length L; returns false when L has no specialisation.
template <class T>
bool fft2_strided(int L, int sign, const cplx<T>* src, cplx<T>* dst, long long inner, int outer, const cplx<T>* W,
                  cudaStream_t st, int var) {
  switch (L) {
    case 16: launch_strided<T, 4, 4>(sign, src, dst, inner, outer, W, st, var); return true;
    case 32: launch_strided<T, 8, 4>(sign, src, dst, inner, outer, W, st, var); return true;
    case 48: launch_strided<T, 8, 6>(sign, src, dst, inner, outer, W, st, var); return true;
    case 64: launch_strided<T, 8, 8>(sign, src, dst, inner, outer, W, st, var); return true;
    case 96: launch_strided<T, 8, 12>(sign, src, dst, inner, outer, W, st, var); return true;
    case 112: launch_strided<T, 16, 7>(sign, src, dst, inner, outer, W, st, var); return true;
    case 128: launch_strided<T, 16, 8>(sign, src, dst, inner, outer, W, st, var); return true;
    case 144: launch_strided<T, 12, 12>(sign, src, dst, inner, outer, W, st, var); return true;
    case 160: launch_strided<T, 16, 10>(sign, src, dst, inner, outer, W, st, var); return true;
    case 192: launch_strided<T, 16, 12>(sign, src, dst, inner, outer, W, st, var); return true;
    case 256: launch_strided<T, 16, 16>(sign, src, dst, inner, outer, W, st, var); return true;
    default: return false;
  }
}

// Specialised contiguous-axis pass for complex length L = n3/2 (sign -1: R2C from real `in`; +1: C2R to `out`).
template <class T>
bool fft2_z(int L, int sign, const void* in, void* out, long long nlines, const cplx<T>* Wn3, T scale,
            cudaStream_t st, int var) {
  switch (L) {
    case 16: launch_z<T, 4, 4>(sign, in, out, nlines, Wn3, scale, st, var); return true;
    case 24: launch_z<T, 8, 3>(sign, in, out, nlines, Wn3, scale, st, var); return true;
    case 32: launch_z<T, 8, 4>(sign, in, out, nlines, Wn3, scale, st, var); return true;
    case 48: launch_z<T, 8, 6>(sign, in, out, nlines, Wn3, scale, st, var); return true;
    case 56: launch_z<T, 8, 7>(sign, in, out, nlines, Wn3, scale, st, var); return true;
    case 64: launch_z<T, 8, 8>(sign, in, out, nlines, Wn3, scale, st, var); return true;
    case 72: launch_z<T, 8, 9>(sign, in, out, nlines, Wn3, scale, st, var); return true;
    case 80: launch_z<T, 8, 10>(sign, in, out, nlines, Wn3, scale, st, var); return true;
    case 96: launch_z<T, 8, 12>(sign, in, out, nlines, Wn3, scale, st, var); return true;
    // inverse 8 x 16: its first stage, which also applies the Hermitian split, runs on all 16 threads of a line
    case 128: launch_z<T, 16, 8, 8, 16>(sign, in, out, nlines, Wn3, scale, st, var); return true;
    default: return false;
  }
}

template bool fft2_strided<float>(int, int, const cplx<float>*, cplx<float>*, long long, int, const cplx<float>*,
                                  cudaStream_t, int);
template bool fft2_strided<double>(int, int, const cplx<double>*, cplx<double>*, long long, int,
                                   const cplx<double>*, cudaStream_t, int);
template bool fft2_z<float>(int, int, const void*, void*, long long, const cplx<float>*, float, cudaStream_t, int);
template bool fft2_z<double>(int, int, const void*, void*, long long, const cplx<double>*, double, cudaStream_t, int);

}  // namespace claire
