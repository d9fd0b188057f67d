// Shared device/host helpers of the sm_103a registration library (internal; not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <string>

#include "claire.h"

namespace claire {

template <class T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };
template <class T> using cplx = typename C2<T>::type;

template <class T> __host__ __device__ __forceinline__ cplx<T> mk(T re, T im) {
  cplx<T> r;
  r.x = re;
  r.y = im;
  return r;
}
template <class T> __device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <class T> __device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <class T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <class T> __device__ __forceinline__ cplx<T> cmulc(cplx<T> a, cplx<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <class T> __device__ __forceinline__ cplx<T> cconj(cplx<T> a) { return mk<T>(a.x, -a.y); }
template <class T> __device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// multiply by -i (SIGN = -1) or +i (SIGN = +1)
template <int SIGN, class T> __device__ __forceinline__ cplx<T> mul_i(cplx<T> a) {
  return SIGN < 0 ? mk<T>(a.y, -a.x) : mk<T>(-a.y, a.x);
}

// Division of 32-bit unsigned integers by an invariant divisor through a multiply-high and a shift
// (Granlund & Montgomery, "Division by invariant integers using multiplication", PLDI 1994, round-up variant):
// q = (umulhi(x, m) + x) >> s with s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1, exact for all x < 2^32.
struct FastDiv {
  unsigned d = 1, m = 1, s = 0;
  FastDiv() = default;
  explicit FastDiv(unsigned div) : d(div) {
    s = 0;
    while ((1ull << s) < div) ++s;
    m = (unsigned)(((1ull << 32) * ((1ull << s) - div)) / div + 1);
  }
  __device__ __forceinline__ unsigned div(unsigned x) const {
    return (unsigned)(((unsigned long long)__umulhi(x, m) + x) >> s);
  }
};

// Grid geometry handed to every kernel by value.
struct Dims {
  int n1, n2, n3;  // real grid
  int n3h;         // n3/2 + 1 (half spectrum along the contiguous axis)
  long long N;     // n1*n2*n3
  long long Ns;    // n1*n2*n3h (complex values of one half spectrum)
  FastDiv by_n3h, by_n2;
};

// Accumulator of FP64-class accuracy for reductions. For FP32 data it keeps an unevaluated float pair (hi, lo)
// updated with error-free transformations -- Knuth's two-sum and the FMA two-product -- as in the "Sum2"/"Dot2"
// algorithms of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005), so a
// thread's partial sum is as accurate as if accumulated in twice the working precision while running on the FP32
// pipes (the FP64 pipe of this GPU is a small fraction of its FP32 rate). The _rn intrinsics keep the compiler
// from contracting the transformations into FMAs. For FP64 data it is a plain double.
template <class T> struct Acc;
template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = __fadd_rn(hi, x);
    const float z = __fsub_rn(t, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(x, z));
    hi = t;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);
    add(p);
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

// Radix schedule of one complex 1D transform of length L (product of the radices).
struct RadixPlan {
  int L;
  int nst;
  int r[16];
};

struct Counters {
  long long launches = 0;
};

// Host-side fault injection for tests of the failure paths: the environment variable CLAIRE_FAULT holds a
// comma-separated list of fault names, and the host code that reads a device result consults it where a named
// fault can be faked (the device work itself is unchanged; nothing faults, traps or hangs on the GPU).
inline bool fault_injected(const char* name) {
  const char* f = std::getenv("CLAIRE_FAULT");
  if (!f || !*f) return false;
  const size_t n = std::strlen(name);
  for (const char* p = f; *p;) {
    const char* e = std::strchr(p, ',');
    const size_t len = e ? size_t(e - p) : std::strlen(p);
    if (len == n && std::strncmp(p, name, n) == 0) return true;
    if (!e) break;
    p = e + 1;
  }
  return false;
}

}  // namespace claire

// Error plumbing: every internal host function returns claire_status and records a message on failure.
#define CL_CUDA(ctxp, call)                                                                              \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess) {                                                                             \
      (ctxp)->set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                             \
      return CLAIRE_ECUDA;                                                                               \
    }                                                                                                    \
  } while (0)

#define CL_LAUNCHED(ctxp)                                                                                \
  do {                                                                                                   \
    (ctxp)->prof_end(st);                                                                                \
    (ctxp)->counters.launches++;                                                                         \
    cudaError_t e_ = cudaGetLastError();                                                                 \
    if (e_ != cudaSuccess) {                                                                             \
      (ctxp)->set_error(std::string("kernel launch (") + (ctxp)->last_launch + "): " + cudaGetErrorString(e_)); \
      return CLAIRE_ECUDA;                                                                               \
    }                                                                                                    \
  } while (0)

#define CL_TRY(expr)                                                                                     \
  do {                                                                                                   \
    claire_status s_ = (expr);                                                                           \
    if (s_ != CLAIRE_OK) return s_;                                                                      \
  } while (0)
