// Layer kernels of the learned warm start: a 3D convolutional encoder-decoder that predicts the low-frequency part
// of the velocity from (m_T, m_R). Not part of the paper's method; the network only seeds v_0 of the unchanged
// Gauss-Newton-Krylov solve (Alg. 1), whose relative stopping test keeps g_0 = g(v = 0).
//
// Activations are channels-last BF16, gradients FP32 (rounded to BF16 where they feed a tensor-core product),
// weights [Cout][27][Cin]. Convolutions are 3x3x3, stride 1, periodic (the registration domain is periodic), and
// run as implicit GEMMs on the tensor cores through the warp-level WMMA interface (16x16x16 BF16 tiles, FP32
// accumulators):
//   forward  y[m, co] = sum_{off, ci} x[nb(m, off), ci] w[co, off, ci]      (M = voxels, N = Cout, K = 27 Cin)
//   dgrad    the forward kernel applied to dz with w^T[ci, 26 - off, co] = w[co, off, ci]
//   wgrad    dw[co, off, ci] = sum_m dz[m, co] x[nb(m, off), ci]           (K = voxels, split into chunks that
//            are reduced in a fixed order, so the result does not depend on scheduling)
// A 16-voxel tile is 16 consecutive voxels of the flattened batch; each row of a staged tile carries its own
// periodic neighbour index, so no grid extent needs to be a multiple of 16.
#include <cuda_bf16.h>
#include <mma.h>

#include <cmath>

#include "impl.cuh"
#include "nn.cuh"

namespace claire {
namespace nn {
namespace {

using namespace nvcuda;

constexpr int kMaxC = 128;

__device__ __forceinline__ int pw(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// coordinates of voxel m of the flattened batch
struct Vox {
  int b, i1, i2, i3;
};
__device__ __forceinline__ Vox vox_of(const Geo& g, int m) {
  Vox v;
  v.i3 = m % g.n3;
  int t = m / g.n3;
  v.i2 = t % g.n2;
  t /= g.n2;
  v.i1 = t % g.n1;
  v.b = t / g.n1;
  return v;
}
// flattened index of the periodic neighbour of v at offset off = 9 (o1 + 1) + 3 (o2 + 1) + (o3 + 1)
__device__ __forceinline__ int nb_of(const Geo& g, const Vox& v, int off) {
  const int o1 = off / 9 - 1, o2 = (off / 3) % 3 - 1, o3 = off % 3 - 1;
  return ((v.b * g.n1 + pw(v.i1 + o1, g.n1)) * g.n2 + pw(v.i2 + o2, g.n2)) * g.n3 + pw(v.i3 + o3, g.n3);
}

// 4 warps per CTA, one 16-voxel tile per warp, NT tiles of 16 output channels per warp. For each of the 27
// offsets the warp stages its 16 neighbour rows (all Cin channels, 16-byte vectors) in shared memory and runs
// Cin/16 x NT tensor-core products; B fragments come from the weights through L1/L2.
template <int NT>
__global__ void __launch_bounds__(128) k_conv3_fwd(const bf16* __restrict__ x, const bf16* __restrict__ w,
                                                   const float* __restrict__ bias, const bf16* __restrict__ skip,
                                                   bf16* __restrict__ y, float* __restrict__ yf, int accum, Geo g,
                                                   int Cin, int Cout, int relu) {
  __shared__ __align__(128) bf16 As[4][16 * kMaxC];
  __shared__ __align__(128) float Cs[4][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = (blockIdx.x * 4 + warp) * 16;
  if (m0 >= g.M) return;
  const int j = lane >> 1, h = lane & 1;
  const Vox me = vox_of(g, m0 + j);
  bf16* A = As[warp];
  wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) wmma::fill_fragment(acc[t], 0.0f);
  const int kcb = Cin / 16, nvec = Cin / 8;
  const long long ldb = 27LL * Cin;
  for (int off = 0; off < 27; ++off) {
    const uint4* src = reinterpret_cast<const uint4*>(x + (long long)nb_of(g, me, off) * Cin);
    uint4* dst = reinterpret_cast<uint4*>(A + j * Cin);
    for (int q = h; q < nvec; q += 2) dst[q] = src[q];
    __syncwarp();
    for (int cb = 0; cb < kcb; ++cb) {
      wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> a;
      wmma::load_matrix_sync(a, A + cb * 16, (unsigned)Cin);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::col_major> bm;
        wmma::load_matrix_sync(bm, w + (long long)t * 16 * ldb + off * Cin + cb * 16, (unsigned)ldb);
        wmma::mma_sync(acc[t], a, bm, acc[t]);
      }
    }
    __syncwarp();
  }
  float* C = Cs[warp];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    wmma::store_matrix_sync(C, acc[t], 16, wmma::mem_row_major);
    __syncwarp();
    for (int e = lane; e < 256; e += 32) {
      const int r = e >> 4, co = t * 16 + (e & 15);
      const long long o = (long long)(m0 + r) * Cout + co;
      float val = C[e];
      if (bias) val += bias[co];
      if (skip) val += __bfloat162float(skip[o]);
      if (relu) val = fmaxf(val, 0.f);
      if (y) y[o] = __float2bfloat16_rn(val);
      if (yf) yf[o] = accum ? yf[o] + val : val;
    }
    __syncwarp();
  }
}

// Partial weight gradients of one voxel chunk (grid.y): warp task (ct, off, it) accumulates the 16 x 16 block
// dw[ct*16.., off, it*16..] over the chunk's 16-voxel tiles.
__global__ void __launch_bounds__(128) k_conv3_wgrad(const bf16* __restrict__ dz, const bf16* __restrict__ x,
                                                     float* __restrict__ part, Geo g, int Cin, int Cout,
                                                     int chunk) {
  __shared__ __align__(128) bf16 Bs[4][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncit = Cin / 16;
  const int ntask = (Cout / 16) * 27 * ncit;
  const int task = blockIdx.x * 4 + warp;
  if (task >= ntask) return;
  const int ct = task / (27 * ncit);
  const int rem = task - ct * 27 * ncit;
  const int off = rem / ncit, it = rem - off * ncit;
  const int j = lane >> 1, h = lane & 1;
  bf16* Bt = Bs[warp];
  wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
  wmma::fill_fragment(acc, 0.0f);
  const int c0 = blockIdx.y * chunk;
  const int c1 = (long long)c0 + chunk < g.M ? c0 + chunk : (int)g.M;
  for (int m0 = c0; m0 < c1; m0 += 16) {
    const Vox me = vox_of(g, m0 + j);
    *reinterpret_cast<uint4*>(Bt + j * 16 + h * 8) =
        *reinterpret_cast<const uint4*>(x + (long long)nb_of(g, me, off) * Cin + it * 16 + h * 8);
    __syncwarp();
    wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::col_major> a;  // (co, m) = dz[m][co]
    wmma::load_matrix_sync(a, dz + (long long)m0 * Cout + ct * 16, (unsigned)Cout);
    wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> bm;  // (m, ci)
    wmma::load_matrix_sync(bm, Bt, 16);
    wmma::mma_sync(acc, a, bm, acc);
    __syncwarp();
  }
  const long long ldo = 27LL * Cin;
  float* dst = part + (long long)blockIdx.y * Cout * ldo + (long long)(ct * 16) * ldo + off * Cin + it * 16;
  wmma::store_matrix_sync(dst, acc, (unsigned)ldo, wmma::mem_row_major);
}

// dst[i] = sum_c part[c][i], c in order
__global__ void k_sum_chunks(const float* __restrict__ part, int nchunks, long long count, float* __restrict__ dst) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < nchunks; ++c) s += part[(long long)c * count + i];
    dst[i] = s;
  }
}

__global__ void k_wt_flip(const bf16* __restrict__ w, bf16* __restrict__ wt, int Cin, int Cout) {
  const long long total = 27LL * Cin * Cout;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int ci = (int)(i % Cin);
    const long long t = i / Cin;
    const int off = (int)(t % 27);
    const int co = (int)(t / 27);
    wt[((long long)ci * 27 + (26 - off)) * Cout + co] = w[i];
  }
}

__global__ void k_relu_bwd(const float* __restrict__ dy, const bf16* __restrict__ y, float* __restrict__ dz,
                           bf16* __restrict__ dzb, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = (y == nullptr || __bfloat162float(y[i]) > 0.f) ? dy[i] : 0.f;
    dz[i] = v;
    dzb[i] = __float2bfloat16_rn(v);
  }
}

// per-block channel sums: blockDim = (256 / C) C threads, thread t owns channel t % C and rows t / C + k rpb
constexpr int kBiasBlocks = 304;
__global__ void k_chan_sum(const float* __restrict__ dz, long long M, int C, float* __restrict__ part) {
  __shared__ float sh[256];
  const int c = threadIdx.x % C, r = threadIdx.x / C, rpb = blockDim.x / C;
  float s = 0.f;
  for (long long m = (long long)blockIdx.x * rpb + r; m < M; m += (long long)gridDim.x * rpb) s += dz[m * C + c];
  sh[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < C) {
    float t = 0.f;
    for (int k = 0; k < rpb; ++k) t += sh[k * C + threadIdx.x];
    part[(long long)blockIdx.x * C + threadIdx.x] = t;
  }
}

// fine voxel of the 2x2x2 block (d = 4 d1 + 2 d2 + d3) under coarse voxel (b, k1, k2, k3)
__device__ __forceinline__ long long fine_of(const Geo& gc, int b, int k1, int k2, int k3, int d) {
  return (((long long)b * (2 * gc.n1) + 2 * k1 + (d >> 2)) * (2 * gc.n2) + 2 * k2 + ((d >> 1) & 1)) * (2 * gc.n3) +
         2 * k3 + (d & 1);
}
__device__ __forceinline__ long long coarse_of(const Geo& gc, long long f) {
  const int N3 = 2 * gc.n3, N2 = 2 * gc.n2, N1 = 2 * gc.n1;
  const int j3 = (int)(f % N3);
  long long t = f / N3;
  const int j2 = (int)(t % N2);
  t /= N2;
  const int j1 = (int)(t % N1);
  const int b = (int)(t / N1);
  return (((long long)b * gc.n1 + j1 / 2) * gc.n2 + j2 / 2) * gc.n3 + j3 / 2;
}
__device__ __forceinline__ void coarse_coords(const Geo& gc, long long p, int& b, int& k1, int& k2, int& k3) {
  k3 = (int)(p % gc.n3);
  long long t = p / gc.n3;
  k2 = (int)(t % gc.n2);
  t /= gc.n2;
  k1 = (int)(t % gc.n1);
  b = (int)(t / gc.n1);
}

__global__ void k_pool_fwd(const bf16* __restrict__ x, bf16* __restrict__ y, Geo gc, int C) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < gc.M * C;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    int b, k1, k2, k3;
    coarse_coords(gc, i / C, b, k1, k2, k3);
    float s = 0.f;
    for (int d = 0; d < 8; ++d) s += __bfloat162float(x[fine_of(gc, b, k1, k2, k3, d) * C + c]);
    y[i] = __float2bfloat16_rn(0.125f * s);
  }
}
__global__ void k_pool_bwd(const float* __restrict__ dy, float* __restrict__ dx, int accum, Geo gc, int C) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < gc.M * 8 * C;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = 0.125f * dy[coarse_of(gc, i / C) * C + i % C];
    dx[i] = accum ? dx[i] + v : v;
  }
}
__global__ void k_up_fwd(const bf16* __restrict__ x, bf16* __restrict__ y, Geo gc, int C) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < gc.M * 8 * C;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[coarse_of(gc, i / C) * C + i % C];
}
__global__ void k_up_bwd(const float* __restrict__ dy, float* __restrict__ dx, int accum, Geo gc, int C) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < gc.M * C;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    int b, k1, k2, k3;
    coarse_coords(gc, i / C, b, k1, k2, k3);
    float s = 0.f;
    for (int d = 0; d < 8; ++d) s += dy[fine_of(gc, b, k1, k2, k3, d) * C + c];
    dx[i] = accum ? dx[i] + s : s;
  }
}

__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ pred, const float* __restrict__ target,
                                             float* __restrict__ grad, long long M, int C, int cu, double inv_count,
                                             double* __restrict__ partials) {
  double acc = 0.0;
  const float gscale = float(2.0 * inv_count);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M * C;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    float gval = 0.f;
    if (c < cu) {
      const float e = pred[i] - target[(i / C) * cu + c];
      acc += double(e) * double(e);
      gval = gscale * e;
    }
    if (grad) grad[i] = gval;
  }
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    partials[blockIdx.x] = t * inv_count;
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m1,
                       float* __restrict__ m2, bf16* __restrict__ pb, long long count, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const float g = gr[i];
    const float a = b1 * m1[i] + (1.f - b1) * g;
    const float v = b2 * m2[i] + (1.f - b2) * g * g;
    m1[i] = a;
    m2[i] = v;
    const float np = p[i] - lr * (a * c1) / (sqrtf(v * c2) + eps);
    p[i] = np;
    if (pb) pb[i] = __float2bfloat16_rn(np);
  }
}

// network input: channel 0 = m_T, channel 1 = sdiff (m_R - m_T) (formed in FP32 before rounding), others 0
__global__ void k_pack_images(const float* __restrict__ src, bf16* __restrict__ dst, long long M, int C,
                              float sdiff) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M * C;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long m = i / C;
    float v = 0.f;
    if (c == 0) v = src[m];
    if (c == 1) v = sdiff * (src[M + m] - src[m]);
    dst[i] = __float2bfloat16_rn(v);
  }
}
__global__ void k_unpack(const float* __restrict__ src, float* __restrict__ dst, long long M, int ncomp, int C,
                         float s) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M * ncomp;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / M);
    dst[i] = s * src[(i - (long long)c * M) * C + c];
  }
}
__global__ void k_interleave(const float* __restrict__ src, float* __restrict__ dst, long long M, int ncomp,
                             float s) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M * ncomp;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = s * src[(long long)(i % ncomp) * M + i / ncomp];
}
__global__ void k_add_f32(const float* __restrict__ a, float* __restrict__ b, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    b[i] += a[i];
}
__global__ void k_f32_to_bf16(const float* __restrict__ a, bf16* __restrict__ b, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

inline unsigned nblocks(long long n) {
  const long long b = (n + 255) / 256;
  return (unsigned)(b < 4864 ? (b > 0 ? b : 1) : 4864);
}

// chunk of the weight-gradient split: about 8 resident CTAs per SM over all chunks, whole 16-voxel tiles
inline int wgrad_chunk(const Geo& g, int Cin, int Cout) {
  const long long ctas = ((long long)(Cout / 16) * 27 * (Cin / 16) + 3) / 4;
  long long nchunks = (1216 + ctas - 1) / ctas;
  const long long tiles = g.M / 16;
  if (nchunks > tiles) nchunks = tiles;
  if (nchunks < 1) nchunks = 1;
  const long long per = (tiles + nchunks - 1) / nchunks;
  return (int)(per * 16);
}

}  // namespace

cudaError_t conv3_fwd(const bf16* x, const bf16* w, const float* bias, const bf16* skip, bf16* y, float* yf,
                      int accum, const Geo& g, int Cin, int Cout, int relu, cudaStream_t st) {
  const unsigned grid = (unsigned)((g.M / 16 + 3) / 4);
#define CL_CONV_CASE(NT)                                                                                         \
  case NT:                                                                                                       \
    k_conv3_fwd<NT><<<grid, 128, 0, st>>>(x, w, bias, skip, y, yf, accum, g, Cin, Cout, relu);                   \
    break;
  switch (Cout / 16) {
    CL_CONV_CASE(1)
    CL_CONV_CASE(2)
    CL_CONV_CASE(3)
    CL_CONV_CASE(4)
    CL_CONV_CASE(5)
    CL_CONV_CASE(6)
    CL_CONV_CASE(7)
    CL_CONV_CASE(8)
    default: return cudaErrorInvalidValue;
  }
#undef CL_CONV_CASE
  return cudaGetLastError();
}

size_t wgrad_work_elems(const Geo& g, int Cin, int Cout) {
  const long long chunk = wgrad_chunk(g, Cin, Cout);
  const long long nchunks = (g.M + chunk - 1) / chunk;
  return size_t(nchunks) * size_t(Cout) * 27 * size_t(Cin);
}

cudaError_t conv3_wgrad(const bf16* dz, const bf16* x, float* dw, float* work, const Geo& g, int Cin, int Cout,
                        cudaStream_t st) {
  const int chunk = wgrad_chunk(g, Cin, Cout);
  const int nchunks = (int)((g.M + chunk - 1) / chunk);
  const int ntask = (Cout / 16) * 27 * (Cin / 16);
  k_conv3_wgrad<<<dim3((unsigned)((ntask + 3) / 4), (unsigned)nchunks), 128, 0, st>>>(dz, x, work, g, Cin, Cout,
                                                                                        chunk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long count = 27LL * Cin * Cout;
  k_sum_chunks<<<nblocks(count), 256, 0, st>>>(work, nchunks, count, dw);
  return cudaGetLastError();
}

cudaError_t weight_flip(const bf16* w, bf16* wt, int Cin, int Cout, cudaStream_t st) {
  k_wt_flip<<<nblocks(27LL * Cin * Cout), 256, 0, st>>>(w, wt, Cin, Cout);
  return cudaGetLastError();
}

cudaError_t relu_bwd(const float* dy, const bf16* y, float* dz, bf16* dzb, long long count, cudaStream_t st) {
  k_relu_bwd<<<nblocks(count), 256, 0, st>>>(dy, y, dz, dzb, count);
  return cudaGetLastError();
}

size_t bias_work_elems(int C) { return size_t(kBiasBlocks) * size_t(C); }

cudaError_t bias_grad(const float* dz, long long M, int C, float* db, float* work, cudaStream_t st) {
  const int threads = (256 / C) * C;
  k_chan_sum<<<kBiasBlocks, threads, 0, st>>>(dz, M, C, work);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_chunks<<<nblocks(C), 256, 0, st>>>(work, kBiasBlocks, C, db);
  return cudaGetLastError();
}

cudaError_t pool_fwd(const bf16* x, bf16* y, const Geo& gf, int C, cudaStream_t st) {
  const Geo gc = mkgeo(gf.B, gf.n1 / 2, gf.n2 / 2, gf.n3 / 2);
  k_pool_fwd<<<nblocks(gc.M * C), 256, 0, st>>>(x, y, gc, C);
  return cudaGetLastError();
}
cudaError_t pool_bwd(const float* dy, float* dx, int accum, const Geo& gf, int C, cudaStream_t st) {
  const Geo gc = mkgeo(gf.B, gf.n1 / 2, gf.n2 / 2, gf.n3 / 2);
  k_pool_bwd<<<nblocks(gf.M * C), 256, 0, st>>>(dy, dx, accum, gc, C);
  return cudaGetLastError();
}
cudaError_t up_fwd(const bf16* x, bf16* y, const Geo& gc, int C, cudaStream_t st) {
  k_up_fwd<<<nblocks(gc.M * 8 * C), 256, 0, st>>>(x, y, gc, C);
  return cudaGetLastError();
}
cudaError_t up_bwd(const float* dy, float* dx, int accum, const Geo& gc, int C, cudaStream_t st) {
  k_up_bwd<<<nblocks(gc.M * C), 256, 0, st>>>(dy, dx, accum, gc, C);
  return cudaGetLastError();
}

cudaError_t mse(const float* pred, const float* target, float* grad, long long M, int C, int cu, double* partials,
                int nb, cudaStream_t st) {
  k_mse<<<nb, 256, 0, st>>>(pred, target, grad, M, C, cu, 1.0 / double(M * cu), partials);
  return cudaGetLastError();
}

cudaError_t adam(float* p, const float* g, float* m1, float* m2, bf16* pb, long long count, float lr, float b1,
                 float b2, float eps, int t, cudaStream_t st) {
  const float c1 = float(1.0 / (1.0 - std::pow(double(b1), t)));
  const float c2 = float(1.0 / (1.0 - std::pow(double(b2), t)));
  k_adam<<<nblocks(count), 256, 0, st>>>(p, g, m1, m2, pb, count, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t pack_images(const float* src, bf16* dst, long long M, int C, float sdiff, cudaStream_t st) {
  k_pack_images<<<nblocks(M * C), 256, 0, st>>>(src, dst, M, C, sdiff);
  return cudaGetLastError();
}
cudaError_t unpack(const float* src, float* dst, long long M, int ncomp, int C, float s, cudaStream_t st) {
  k_unpack<<<nblocks(M * ncomp), 256, 0, st>>>(src, dst, M, ncomp, C, s);
  return cudaGetLastError();
}
cudaError_t interleave(const float* src, float* dst, long long M, int ncomp, float s, cudaStream_t st) {
  k_interleave<<<nblocks(M * ncomp), 256, 0, st>>>(src, dst, M, ncomp, s);
  return cudaGetLastError();
}
cudaError_t add(const float* a, float* b, long long count, cudaStream_t st) {
  k_add_f32<<<nblocks(count), 256, 0, st>>>(a, b, count);
  return cudaGetLastError();
}
cudaError_t to_bf16(const float* a, bf16* b, long long count, cudaStream_t st) {
  k_f32_to_bf16<<<nblocks(count), 256, 0, st>>>(a, b, count);
  return cudaGetLastError();
}

}  // namespace nn
}  // namespace claire

// ---------------------------------------------------------------------------------------------------------------
// C-ABI of the individual layers (argument checks, then the launchers above)
using namespace claire::nn;

namespace {
inline claire_status st_of(cudaError_t e) { return e == cudaSuccess ? CLAIRE_OK : CLAIRE_ECUDA; }
inline bool geo_args(int B, int n1, int n2, int n3) { return B > 0 && n1 > 0 && n2 > 0 && n3 > 0; }
inline bool pool_args(int B, int n1, int n2, int n3) {
  return geo_args(B, n1, n2, n3) && n1 % 2 == 0 && n2 % 2 == 0 && n3 % 2 == 0;
}
}  // namespace

extern "C" {

claire_status claire_nn_conv3_fwd(const void* x, const void* w, const float* bias, const void* skip, void* y,
                                  float* yf, int accum, int B, int n1, int n2, int n3, int Cin, int Cout, int relu,
                                  void* stream) {
  if (!x || !w || (!y && !yf) || !geo_args(B, n1, n2, n3)) return CLAIRE_EINVAL;
  const Geo g = mkgeo(B, n1, n2, n3);
  if (!conv_geo_ok(g) || !conv_chan_ok(Cin) || !conv_chan_ok(Cout)) return CLAIRE_EINVAL;
  return st_of(conv3_fwd(static_cast<const bf16*>(x), static_cast<const bf16*>(w), bias,
                         static_cast<const bf16*>(skip), static_cast<bf16*>(y), yf, accum ? 1 : 0, g, Cin, Cout,
                         relu ? 1 : 0, (cudaStream_t)stream));
}

size_t claire_nn_wgrad_workspace_bytes(int B, int n1, int n2, int n3, int Cin, int Cout) {
  if (!geo_args(B, n1, n2, n3) || !conv_chan_ok(Cin) || !conv_chan_ok(Cout)) return 0;
  const Geo g = mkgeo(B, n1, n2, n3);
  if (!conv_geo_ok(g)) return 0;
  return wgrad_work_elems(g, Cin, Cout) * sizeof(float);
}

claire_status claire_nn_conv3_wgrad(const void* dz, const void* x, float* dw, float* work, int B, int n1, int n2,
                                    int n3, int Cin, int Cout, void* stream) {
  if (!dz || !x || !dw || !work || !geo_args(B, n1, n2, n3)) return CLAIRE_EINVAL;
  const Geo g = mkgeo(B, n1, n2, n3);
  if (!conv_geo_ok(g) || !conv_chan_ok(Cin) || !conv_chan_ok(Cout)) return CLAIRE_EINVAL;
  return st_of(conv3_wgrad(static_cast<const bf16*>(dz), static_cast<const bf16*>(x), dw, work, g, Cin, Cout,
                           (cudaStream_t)stream));
}

claire_status claire_nn_weight_flip(const void* w, void* wt, int Cin, int Cout, void* stream) {
  if (!w || !wt || Cin <= 0 || Cout <= 0) return CLAIRE_EINVAL;
  return st_of(weight_flip(static_cast<const bf16*>(w), static_cast<bf16*>(wt), Cin, Cout, (cudaStream_t)stream));
}

claire_status claire_nn_relu_bwd(const float* dy, const void* y, float* dz, void* dzb, long long count,
                                 void* stream) {
  if (!dy || !dz || !dzb || count < 0) return CLAIRE_EINVAL;
  return st_of(relu_bwd(dy, static_cast<const bf16*>(y), dz, static_cast<bf16*>(dzb), count, (cudaStream_t)stream));
}

size_t claire_nn_bias_workspace_bytes(int C) { return C > 0 && C <= 256 ? bias_work_elems(C) * sizeof(float) : 0; }

claire_status claire_nn_bias_grad(const float* dz, long long M, int C, float* db, float* work, void* stream) {
  if (!dz || !db || !work || M <= 0 || C <= 0 || C > 256) return CLAIRE_EINVAL;
  return st_of(bias_grad(dz, M, C, db, work, (cudaStream_t)stream));
}

claire_status claire_nn_pool_fwd(const void* x, void* y, int B, int n1, int n2, int n3, int C, void* stream) {
  if (!x || !y || !pool_args(B, n1, n2, n3) || C <= 0) return CLAIRE_EINVAL;
  return st_of(pool_fwd(static_cast<const bf16*>(x), static_cast<bf16*>(y), mkgeo(B, n1, n2, n3), C,
                        (cudaStream_t)stream));
}
claire_status claire_nn_pool_bwd(const float* dy, float* dx, int accum, int B, int n1, int n2, int n3, int C,
                                 void* stream) {
  if (!dy || !dx || !pool_args(B, n1, n2, n3) || C <= 0) return CLAIRE_EINVAL;
  return st_of(pool_bwd(dy, dx, accum ? 1 : 0, mkgeo(B, n1, n2, n3), C, (cudaStream_t)stream));
}
claire_status claire_nn_up_fwd(const void* x, void* y, int B, int n1, int n2, int n3, int C, void* stream) {
  if (!x || !y || !geo_args(B, n1, n2, n3) || C <= 0) return CLAIRE_EINVAL;
  return st_of(
      up_fwd(static_cast<const bf16*>(x), static_cast<bf16*>(y), mkgeo(B, n1, n2, n3), C, (cudaStream_t)stream));
}
claire_status claire_nn_up_bwd(const float* dy, float* dx, int accum, int B, int n1, int n2, int n3, int C,
                               void* stream) {
  if (!dy || !dx || !geo_args(B, n1, n2, n3) || C <= 0) return CLAIRE_EINVAL;
  return st_of(up_bwd(dy, dx, accum ? 1 : 0, mkgeo(B, n1, n2, n3), C, (cudaStream_t)stream));
}

claire_status claire_nn_mse(const float* pred, const float* target, float* grad, long long M, int C, int cu,
                            double* partials, int npartials, void* stream) {
  if (!pred || !target || !partials || M <= 0 || C <= 0 || cu <= 0 || cu > C || npartials < 1) return CLAIRE_EINVAL;
  return st_of(mse(pred, target, grad, M, C, cu, partials, npartials, (cudaStream_t)stream));
}

claire_status claire_nn_adam(float* p, const float* g, float* m1, float* m2, void* pb, long long count, float lr,
                             float b1, float b2, float eps, int step, void* stream) {
  if (!p || !g || !m1 || !m2 || count < 0 || step < 1) return CLAIRE_EINVAL;
  return st_of(adam(p, g, m1, m2, static_cast<bf16*>(pb), count, lr, b1, b2, eps, step, (cudaStream_t)stream));
}

}  // extern "C"
