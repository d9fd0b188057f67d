// Shared device/host helpers of the sm_103a registration library (internal; not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
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

// Grid geometry handed to every kernel by value.
struct Dims {
  int n1, n2, n3;  // real grid
  int n3h;         // n3/2 + 1 (half spectrum along the contiguous axis)
  long long N;     // n1*n2*n3
  long long Ns;    // n1*n2*n3h (complex values of one half spectrum)
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
      (ctxp)->set_error(std::string("kernel launch: ") + cudaGetErrorString(e_));                        \
      return CLAIRE_ECUDA;                                                                               \
    }                                                                                                    \
  } while (0)

#define CL_TRY(expr)                                                                                     \
  do {                                                                                                   \
    claire_status s_ = (expr);                                                                           \
    if (s_ != CLAIRE_OK) return s_;                                                                      \
  } while (0)
