// Streaming vector kernels of the Krylov and Gauss-Newton loops (Alg. 1, Alg. 2): FP64-accumulated inner products
// (warp-shuffle + shared-memory block reduction into a fixed number of partials, then a one-block deterministic
// finish, so results are reproducible run to run) and the fused PCG updates.
#include <cuda_bf16.h>

#include <mutex>

#include "impl.cuh"

namespace claire {

__device__ __forceinline__ void block_partial(double acc, double* __restrict__ partials) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    partials[blockIdx.x] = t;
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_dot(const T* __restrict__ a, const T* __restrict__ b, long long n,
                                             double* __restrict__ partials) {
  Acc<T> acc;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc.add_prod(a[i], b[i]);
  block_partial(acc.value(), partials);
}

template <class T>
__global__ void __launch_bounds__(256) k_diffsq(const T* __restrict__ a, const T* __restrict__ b, long long n,
                                                double* __restrict__ partials) {
  Acc<T> acc;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T e = a[i] - b[i];
    acc.add_prod(e, e);
  }
  block_partial(acc.value(), partials);
}

// number of non-finite values (NaN or +-Inf) in a[0..na) and b[0..nb), one partial per block
template <class T>
__global__ void __launch_bounds__(256) k_nonfinite(const T* __restrict__ a, long long na, const T* __restrict__ b,
                                                   long long nb, double* __restrict__ partials) {
  double cnt = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += stride) {
    const T x = i < na ? a[i] : b[i - na];
    if (!isfinite(x)) cnt += 1.0;
  }
  block_partial(cnt, partials);
}

__global__ void __launch_bounds__(1024) k_reduce_final(const double* __restrict__ partials, int np, double scale,
                                                       double* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partials[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) *out = scale * t;
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_absmax(const T* __restrict__ a, long long n, double* __restrict__ partials) {
  T m = T(0);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(a[i]));
  __shared__ double red[32];
  double v = double(m);
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, red[i]);
    partials[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_max_final(const double* __restrict__ partials, int np,
                                                    double* __restrict__ out) {
  __shared__ double red[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) v = fmax(v, partials[i]);
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, red[i]);
    *out = t;
  }
}

__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

template <class T>
__global__ void k_axpy(long long n, T a, const T* __restrict__ x, T* __restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}
template <class T>
__global__ void k_xpay(long long n, const T* __restrict__ x, T a, T* __restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(a, y[i], x[i]);
}
template <class T>
__global__ void k_waxpy(long long n, const T* __restrict__ x, T a, const T* __restrict__ y, T* __restrict__ z) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = fma(a, y[i], x[i]);
}
template <class T>
__global__ void k_scale_copy(long long n, T a, const T* __restrict__ x, T* __restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}
// y = 0 over n words of 4 or 8 bytes (T = float or double; complex arrays pass twice their length)
template <class T> __global__ void k_zero(long long n, T* __restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = T(0);
}
static inline unsigned stream_blocks(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  return (unsigned)(b < 8 * 152 * 4 ? b : 8 * 152 * 4);
}

template <class T>
claire_status dot_partial(claire_ctx* c, const T* a, const T* b, long long n, double* partials, cudaStream_t st) {
  c->prof_begin("dot", st);
  k_dot<T><<<kReduceBlocks, 256, 0, st>>>(a, b, n, partials);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T>
claire_status diffsq_partial(claire_ctx* c, const T* a, const T* b, long long n, double* partials, cudaStream_t st) {
  c->prof_begin("diffsq", st);
  k_diffsq<T><<<kReduceBlocks, 256, 0, st>>>(a, b, n, partials);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
__global__ void __launch_bounds__(1024) k_reduce_final_v(const double* __restrict__ partials, int np, double scale,
                                                         double* __restrict__ out) {
  __shared__ double red[32];
  const double* p = partials + (long long)blockIdx.x * np;
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += p[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) out[blockIdx.x] = scale * t;
  }
}

claire_status reduce_final_v(claire_ctx* c, const double* partials, int nv, int np, double scale, double* out,
                             cudaStream_t st) {
  c->prof_begin("reduce_final_v", st);
  k_reduce_final_v<<<nv, 1024, 0, st>>>(partials, np, scale, out);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

claire_status reduce_final(claire_ctx* c, const double* partials, double scale, double* out, cudaStream_t st) {
  c->prof_begin("reduce_final", st);
  k_reduce_final<<<1, 1024, 0, st>>>(partials, kReduceBlocks, scale, out);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T>
claire_status nonfinite_partial(claire_ctx* c, const T* a, long long na, const T* b, long long nb, double* partials,
                                cudaStream_t st) {
  c->prof_begin("nonfinite", st);
  k_nonfinite<T><<<kReduceBlocks, 256, 0, st>>>(a, na, b, nb, partials);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T>
claire_status absmax_partial(claire_ctx* c, const T* a, long long n, double* partials, cudaStream_t st) {
  c->prof_begin("absmax", st);
  k_absmax<T><<<kReduceBlocks, 256, 0, st>>>(a, n, partials);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
claire_status max_final(claire_ctx* c, const double* partials, int np, double* out, cudaStream_t st) {
  c->prof_begin("max_final", st);
  k_max_final<<<1, 1024, 0, st>>>(partials, np, out);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

claire_status to_bf16(claire_ctx* c, const float* x, void* y, long long n, cudaStream_t st) {
  c->prof_begin("to_bf16", st);
  k_to_bf16<<<stream_blocks(n), kThreads, 0, st>>>(x, static_cast<__nv_bfloat16*>(y), n);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

template <class T> claire_status axpy(claire_ctx* c, long long n, double a, const T* x, T* y, cudaStream_t st) {
  c->prof_begin("axpy", st);
  k_axpy<T><<<stream_blocks(n), kThreads, 0, st>>>(n, T(a), x, y);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T> claire_status xpay(claire_ctx* c, long long n, const T* x, double a, T* y, cudaStream_t st) {
  c->prof_begin("xpay", st);
  k_xpay<T><<<stream_blocks(n), kThreads, 0, st>>>(n, x, T(a), y);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T>
claire_status waxpy(claire_ctx* c, long long n, const T* x, double a, const T* y, T* z, cudaStream_t st) {
  c->prof_begin("waxpy", st);
  k_waxpy<T><<<stream_blocks(n), kThreads, 0, st>>>(n, x, T(a), y, z);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T> claire_status zero_fill(claire_ctx* c, long long n, T* y, cudaStream_t st) {
  c->prof_begin("zero", st);
  k_zero<T><<<stream_blocks(n), kThreads, 0, st>>>(n, y);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}
template <class T> claire_status scale_copy(claire_ctx* c, long long n, double a, const T* x, T* y, cudaStream_t st) {
  c->prof_begin("scale_copy", st);
  k_scale_copy<T><<<stream_blocks(n), kThreads, 0, st>>>(n, T(a), x, y);
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}


// ---- inner product without any allocation ------------------------------------------------------------------
// The partial sums of k_dot go to this file-scope array instead of a context workspace. Each block writes its own
// slot before the finishing kernel reads it, so nothing has to be cleared between calls.
constexpr int kNoAllocBlocks = 1 << 16;           // partial-sum slots (512 KiB of FP64 on every device)
constexpr long long kNoAllocChunk = 256LL * 8;    // values reduced per block
static __device__ __align__(256) double g_noalloc_partials[kNoAllocBlocks];

// Host-side address of g_noalloc_partials on each device, looked up once per device (the host symbol itself is
// only a stand-in and must never be passed to a kernel). The cached address belongs to the device's primary context:
// after a reset of that context (cudaDeviceReset) it is stale, so the call must not be used across a device reset.
static double* noalloc_scratch_on_current_device(claire_status* st) {
  static std::mutex mu;
  static double* addr[256] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    *st = CLAIRE_ECUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) {
      *st = CLAIRE_ECUDA;
      return nullptr;
    }
    addr[dev] = static_cast<double*>(p);
  }
  *st = CLAIRE_OK;
  return addr[dev];
}

#define INST(T)                                                                                                   \
  template claire_status absmax_partial<T>(claire_ctx*, const T*, long long, double*, cudaStream_t);              \
  template claire_status nonfinite_partial<T>(claire_ctx*, const T*, long long, const T*, long long, double*,    \
                                              cudaStream_t);                                                     \
  template claire_status dot_partial<T>(claire_ctx*, const T*, const T*, long long, double*, cudaStream_t);       \
  template claire_status diffsq_partial<T>(claire_ctx*, const T*, const T*, long long, double*, cudaStream_t);    \
  template claire_status axpy<T>(claire_ctx*, long long, double, const T*, T*, cudaStream_t);                     \
  template claire_status xpay<T>(claire_ctx*, long long, const T*, double, T*, cudaStream_t);                     \
  template claire_status waxpy<T>(claire_ctx*, long long, const T*, double, const T*, T*, cudaStream_t);          \
  template claire_status scale_copy<T>(claire_ctx*, long long, double, const T*, T*, cudaStream_t);              \
  template claire_status zero_fill<T>(claire_ctx*, long long, T*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace claire

extern "C" claire_status claire_dot_noalloc_f32(const float* a, const float* b, long long count, double scale,
                                                double* out, void* stream) {
  using namespace claire;
  if (!a || !b || !out || count < 0) return CLAIRE_EINVAL;
  // the size check comes before any arithmetic on count, so that no count can overflow the block computation
  if (count > (long long)kNoAllocBlocks * kNoAllocChunk) return CLAIRE_EINVAL;
  const long long blocks = (count + kNoAllocChunk - 1) / kNoAllocChunk;
  claire_status st = CLAIRE_OK;
  double* partials = noalloc_scratch_on_current_device(&st);
  if (st != CLAIRE_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = blocks > 0 ? (int)blocks : 1;
  k_dot<float><<<nb, 256, 0, s>>>(a, b, count, partials);
  if (cudaGetLastError() != cudaSuccess) return CLAIRE_ECUDA;
  k_reduce_final<<<1, 1024, 0, s>>>(partials, nb, scale, out);
  if (cudaGetLastError() != cudaSuccess) return CLAIRE_ECUDA;
  return CLAIRE_OK;
}
