// Adjoint / incremental-adjoint step of the memory-reduced Gauss-Newton sweeps (Eq. (4), (9), Sec. 3.5) with its
// streamed operands staged by the Tensor Memory Accelerator.
//
// The brick-tiled step (sl_kernels.cuh, k_adj_step) loads the departure displacement Y (3 words per node), the
// gradient history slice grad m^j (3) and the time-integral accumulator b (3) with per-thread global loads and
// writes b back the same way. A CTA covers 16 (i3) x 16 (i2) x 4 (i1) nodes, so each warp-wide access touches two
// 64-byte row segments: those accesses cost about twice the L1 data-pipe wavefronts of their bytes, and the data
// pipe is the kernel's limit (it also carries the 64 shared-memory taps per node). Here one thread issues three
// tiled TMA loads per CTA -- boxes of 16 x 16 x 4 nodes x 3 components of Y, grad m^j (FP32 or BF16) and b --
// which land in shared memory without passing through the load/store units, and one TMA store writes the updated
// b back. The gathered field still fills its brick with cp.async (its periodic wrap has no tiled-TMA form), and
// lambda^j is stored per thread. Same arithmetic in the same order as k_adj_step: the results are bit-identical.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "sl_kernels.cuh"
#include "tc.cuh"
#include "tma.cuh"

namespace claire {

namespace {

__device__ int g_sl_tma_error = 0;  // set by a CTA whose bounded wait for its staged operands ran out

constexpr int kTileNodes = kTX * kTY * kTZ;  // 1024
constexpr long long kWaitCycles = 2000000000LL;  // about a second at 2 GHz

__host__ __device__ constexpr size_t align128(size_t b) { return (b + 127) / 128 * 128; }

// shared-memory layout: [brick][Y: 3 x 1024 FP32][grad m: 3 x 1024 G][b: 3 x 1024 FP32] (73 KB at halo 2: three
// CTAs per SM; the direction s of the fused <s, b~> is read per thread, staging it too left two)
template <int H, class G> struct StageLayout {
  static constexpr size_t brick = align128(size_t(TileGeom<H>::vol) * 4);
  static constexpr size_t y = brick;
  static constexpr size_t g = y + 3 * kTileNodes * 4;
  static constexpr size_t b = g + align128(3 * kTileNodes * sizeof(G));
  __host__ __device__ static constexpr size_t bytes() { return b + 3 * kTileNodes * 4; }
  __host__ __device__ static constexpr uint32_t tx_bytes() { return uint32_t(3 * kTileNodes * (4 + sizeof(G) + 4)); }
};

template <class G> __device__ __forceinline__ float as_f32(G x) {
  if constexpr (std::is_same<G, __nv_bfloat16>::value) {
    return __bfloat162float(x);
  } else {
    return x;
  }
}

template <int H, bool STORE, bool DOT, class G>
__global__ void __launch_bounds__(256, 3)
    k_adj_step_tma(const float* __restrict__ lam_next, float* __restrict__ lam, const __grid_constant__ CUtensorMap mY,
                   const __grid_constant__ CUtensorMap mG, const __grid_constant__ CUtensorMap mB,
                   const float* __restrict__ sv, int j, float w, Dims d, double* __restrict__ part) {
  using L = StageLayout<H, G>;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  __shared__ __align__(8) uint64_t bar;
  float* brick = reinterpret_cast<float*>(sm_raw);
  const float* sY = reinterpret_cast<const float*>(sm_raw + L::y);
  const G* sG = reinterpret_cast<const G*>(sm_raw + L::g);
  float* sB = reinterpret_cast<float*>(sm_raw + L::b);
  const int tid = threadIdx.y * kTX + threadIdx.x;
  const Tile tl = tile_of<H>(d);
  const uint32_t b = tma::smem_addr(&bar);
  if (tid == 0) tc::mbar_init(b, 1);
  __syncthreads();
  if (tid == 0) {
    tma::expect_tx(b, L::tx_bytes());
    tma::load4(tma::smem_addr(sm_raw + L::y), &mY, tl.x0, tl.y0, tl.z0, 0, b);
    tma::load5(tma::smem_addr(sm_raw + L::g), &mG, tl.x0, tl.y0, tl.z0, 0, j, b);
    tma::load4(tma::smem_addr(sm_raw + L::b), &mB, tl.x0, tl.y0, tl.z0, 0, b);
  }
  load_bricks<float, H>(brick, lam_next, (const float*)nullptr, tl, d);
  __syncthreads();
  // bounded wait for the staged operands; every thread takes the same decision
  const bool ok = tc::mbar_wait(b, 0, kWaitCycles);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicExch(&g_sl_tma_error, 1);
    tc::mbar_wait(b, 0, kWaitCycles);  // the copies may still land: wait (bounded) before the CTA leaves
    return;
  }
  double contrib = 0.0;
#pragma unroll 1
  for (int tz = 0; tz < kTZ; ++tz) {
    const int i1 = tl.z0 + tz, i2 = tl.y0 + threadIdx.y, i3 = tl.x0 + threadIdx.x;
    if (i1 < d.n1 && i2 < d.n2 && i3 < d.n3) {
      const int s = (tz * kTY + threadIdx.y) * kTX + threadIdx.x;
      const int idx = (i1 * d.n2 + i2) * d.n3 + i3;
      Stencil<float> st;
      stencil_at<float>(i1, i2, i3, sY[s], sY[kTileNodes + s], sY[2 * kTileNodes + s], d, st);
      const float l = sample<float, H>(lam_next, brick, 0, tl, st, d);
      if (STORE) lam[idx] = l;
      const float wl = w * l;
      const float b0 = fmaf(wl, as_f32<G>(sG[s]), sB[s]);
      const float b1 = fmaf(wl, as_f32<G>(sG[kTileNodes + s]), sB[kTileNodes + s]);
      const float b2 = fmaf(wl, as_f32<G>(sG[2 * kTileNodes + s]), sB[2 * kTileNodes + s]);
      sB[s] = b0;
      sB[kTileNodes + s] = b1;
      sB[2 * kTileNodes + s] = b2;
      if (DOT) contrib += double(fmaf(sv[2 * d.N + idx], b2, fmaf(sv[d.N + idx], b1, sv[idx] * b0)));
    }
  }
  tma::fence_to_async();
  __syncthreads();
  if (tid == 0) {
    tma::store4(&mB, tma::smem_addr(sB), tl.x0, tl.y0, tl.z0, 0);
    tma::store_commit();
  }
  if (DOT) {
    __shared__ double red[8];
    double cs = contrib;
    for (int o = 16; o > 0; o >>= 1) cs += __shfl_down_sync(0xffffffffu, cs, o);
    if ((tid & 31) == 0) red[tid >> 5] = cs;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < 8; ++i) t += red[i];
      part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = t;
    }
  }
  if (tid == 0) tma::store_wait_read();
}

// Incremental state step (Eq. (8), Sec. 2.3.1) with X, vt and grad m^{j+1} staged by TMA:
// m~^{j+1}(x) = q^j(X) + dt/2 f^{j+1}(x), f = -vt . grad m; not last: q^{j+1} = m~^{j+1} + dt/2 f^{j+1};
// last: lambda~ = -m~(1), b = w lambda~ grad m^{nt} (written into the staging slots of X, then one TMA store).
// Same arithmetic in the same order as k_inc_step.
template <int H, bool LAST, class G>
__global__ void __launch_bounds__(256, 3)
    k_inc_step_tma(const float* __restrict__ q, float* __restrict__ qout, const __grid_constant__ CUtensorMap mX,
                   const __grid_constant__ CUtensorMap mV, const __grid_constant__ CUtensorMap mG,
                   const __grid_constant__ CUtensorMap mB, int j, float hdt, float w, Dims d) {
  using L = StageLayout<H, G>;  // [brick][X][grad m][vt] (the b slot of the adjoint layout holds vt)
  extern __shared__ __align__(128) unsigned char sm_raw[];
  __shared__ __align__(8) uint64_t bar;
  float* brick = reinterpret_cast<float*>(sm_raw);
  float* sX = reinterpret_cast<float*>(sm_raw + L::y);
  const G* sG = reinterpret_cast<const G*>(sm_raw + L::g);
  const float* sV = reinterpret_cast<const float*>(sm_raw + L::b);
  const int tid = threadIdx.y * kTX + threadIdx.x;
  const Tile tl = tile_of<H>(d);
  const uint32_t b = tma::smem_addr(&bar);
  if (tid == 0) tc::mbar_init(b, 1);
  __syncthreads();
  if (tid == 0) {
    tma::expect_tx(b, L::tx_bytes());
    tma::load4(tma::smem_addr(sm_raw + L::y), &mX, tl.x0, tl.y0, tl.z0, 0, b);
    tma::load5(tma::smem_addr(sm_raw + L::g), &mG, tl.x0, tl.y0, tl.z0, 0, j, b);
    tma::load4(tma::smem_addr(sm_raw + L::b), &mV, tl.x0, tl.y0, tl.z0, 0, b);
  }
  load_bricks<float, H>(brick, q, (const float*)nullptr, tl, d);
  __syncthreads();
  const bool ok = tc::mbar_wait(b, 0, kWaitCycles);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicExch(&g_sl_tma_error, 1);
    tc::mbar_wait(b, 0, kWaitCycles);
    return;
  }
#pragma unroll 1
  for (int tz = 0; tz < kTZ; ++tz) {
    const int i1 = tl.z0 + tz, i2 = tl.y0 + threadIdx.y, i3 = tl.x0 + threadIdx.x;
    if (i1 < d.n1 && i2 < d.n2 && i3 < d.n3) {
      const int s = (tz * kTY + threadIdx.y) * kTX + threadIdx.x;
      const int idx = (i1 * d.n2 + i2) * d.n3 + i3;
      Stencil<float> st;
      stencil_at<float>(i1, i2, i3, sX[s], sX[kTileNodes + s], sX[2 * kTileNodes + s], d, st);
      const float g1 = as_f32<G>(sG[s]), g2 = as_f32<G>(sG[kTileNodes + s]), g3 = as_f32<G>(sG[2 * kTileNodes + s]);
      const float f = -(sV[s] * g1 + sV[kTileNodes + s] * g2 + sV[2 * kTileNodes + s] * g3);
      const float mt = sample<float, H>(q, brick, 0, tl, st, d) + hdt * f;
      if (!LAST) {
        qout[idx] = mt + hdt * f;
      } else {
        const float l = -mt;
        qout[idx] = l;
        const float wl = w * l;
        // this thread's X slots are read; they now take b
        sX[s] = wl * g1;
        sX[kTileNodes + s] = wl * g2;
        sX[2 * kTileNodes + s] = wl * g3;
      }
    }
  }
  if (LAST) {
    tma::fence_to_async();
    __syncthreads();
    if (tid == 0) {
      tma::store4(&mB, tma::smem_addr(sX), tl.x0, tl.y0, tl.z0, 0);
      tma::store_commit();
      tma::store_wait_read();
    }
  }
}

// ---- tensor maps ---------------------------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// a map over [extra][3][n1][n2][n3] (rank 4 without `extra`, 5 with it) and a box of 16 x 16 x 4 nodes x 3
// components x 1
bool encode(CUtensorMap* m, const void* base, const Dims& d, size_t esize, int extra) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[5] = {(cuuint64_t)d.n3, (cuuint64_t)d.n2, (cuuint64_t)d.n1, 3, (cuuint64_t)(extra > 0 ? extra : 1)};
  const cuuint64_t strides[4] = {(cuuint64_t)d.n3 * esize, (cuuint64_t)d.n2 * d.n3 * esize, (cuuint64_t)d.N * esize,
                                 (cuuint64_t)3 * d.N * esize};
  const cuuint32_t box[5] = {(cuuint32_t)kTX, (cuuint32_t)kTY, (cuuint32_t)kTZ, 3, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = fn(m, esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                        extra > 0 ? 5 : 4, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int H, bool STORE, bool DOT, class G> cudaError_t set_smem() {
  return cudaFuncSetAttribute((const void*)k_adj_step_tma<H, STORE, DOT, G>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)StageLayout<H, G>::bytes());
}

template <int H, class G> cudaError_t set_all_smem() {
  cudaError_t e = set_smem<H, true, false, G>();
  if (e == cudaSuccess) e = set_smem<H, false, false, G>();
  if (e == cudaSuccess) e = set_smem<H, false, true, G>();
  for (const void* fn : {(const void*)k_inc_step_tma<H, false, G>, (const void*)k_inc_step_tma<H, true, G>})
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)StageLayout<H, G>::bytes());
  return e;
}

template <int H, class G>
void launch(bool store, bool dot, const float* lam_next, float* lam, const float* sv, const TmaMaps& M, int j,
            float w, const Dims& d, double* part, cudaStream_t st) {
  dim3 grid, block;
  tiled_shape<H>(d, grid, block);
  const CUtensorMap& mG = std::is_same<G, float>::value ? M.gm : M.gm16;
  const size_t smem = StageLayout<H, G>::bytes();
  if (dot)
    k_adj_step_tma<H, false, true, G><<<grid, block, smem, st>>>(lam_next, lam, M.dY, mG, M.b, sv, j, w, d, part);
  else if (store)
    k_adj_step_tma<H, true, false, G><<<grid, block, smem, st>>>(lam_next, lam, M.dY, mG, M.b, sv, j, w, d, part);
  else
    k_adj_step_tma<H, false, false, G><<<grid, block, smem, st>>>(lam_next, lam, M.dY, mG, M.b, sv, j, w, d, part);
}

template <int H, class G>
void launch_inc(bool last, const float* q, float* qout, const TmaMaps& M, int j, float hdt, float w, const Dims& d,
                cudaStream_t st) {
  dim3 grid, block;
  tiled_shape<H>(d, grid, block);
  const CUtensorMap& mG = std::is_same<G, float>::value ? M.gm : M.gm16;
  const size_t smem = StageLayout<H, G>::bytes();
  if (last)
    k_inc_step_tma<H, true, G><<<grid, block, smem, st>>>(q, qout, M.dX, M.s, mG, M.b, j, hdt, w, d);
  else
    k_inc_step_tma<H, false, G><<<grid, block, smem, st>>>(q, qout, M.dX, M.s, mG, M.b, j, hdt, w, d);
}

}  // namespace

claire_status sl_incstate_step_tma(claire_ctx* c, const float* q, float* qout, int j, bool last, float hdt, float w,
                                   int H, cudaStream_t st) {
  auto go = [&](auto hc) {
    constexpr int HC = decltype(hc)::value;
    if (c->gm16_on)
      launch_inc<HC, __nv_bfloat16>(last, q, qout, c->tma, j, hdt, w, c->d, st);
    else
      launch_inc<HC, float>(last, q, qout, c->tma, j, hdt, w, c->d, st);
  };
  switch (H) {
    case 2: go(std::integral_constant<int, 2>()); break;
    case 3: go(std::integral_constant<int, 3>()); break;
    case 4: go(std::integral_constant<int, 4>()); break;
    case 5: go(std::integral_constant<int, 5>()); break;
    default: c->set_error("sl_incstate_step_tma: unsupported halo"); return CLAIRE_EINVAL;
  }
  return CLAIRE_OK;
}

bool sl_tma_prepare(claire_ctx* c) {
  Work<float>& W = c->work<float>();
  TmaMaps& M = c->tma;
  const Dims& d = c->d;
  const void* key[4] = {W.dY, c->gm16_on ? W.gm16 : (const void*)W.gm, W.b, W.dX};
  if (M.tried && std::memcmp(key, M.key, sizeof(key)) == 0) return M.ok;
  M.tried = true;
  std::memcpy(M.key, key, sizeof(key));
  M.ok = false;
  // 16-byte aligned rows and component strides, whole tiles along i3
  if (d.n3 % kTX != 0 || !encode_fn()) return false;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    for (cudaError_t e : {set_all_smem<2, float>(), set_all_smem<3, float>(), set_all_smem<4, float>(),
                          set_all_smem<5, float>(), set_all_smem<2, __nv_bfloat16>(),
                          set_all_smem<3, __nv_bfloat16>(), set_all_smem<4, __nv_bfloat16>(),
                          set_all_smem<5, __nv_bfloat16>()})
      if (e != cudaSuccess) attr = e;
  });
  if (attr != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  bool ok = encode(&M.dY, W.dY, d, 4, 0) && encode(&M.b, W.b, d, 4, 0) && encode(&M.dX, W.dX, d, 4, 0) &&
            encode(&M.s, W.s, d, 4, 0);
  if (c->gm16_on)
    ok = ok && encode(&M.gm16, W.gm16, d, 2, c->o.nt + 1);
  else
    ok = ok && encode(&M.gm, W.gm, d, 4, c->o.nt + 1);
  M.ok = ok;
  return ok;
}

claire_status sl_adjoint_step_tma(claire_ctx* c, const float* lam_next, float* lam, int j, float w,
                                  const float* sv, double* part, int H, cudaStream_t st) {
  const bool dot = sv != nullptr;
  const Dims& d = c->d;
  auto go = [&](auto hc) {
    constexpr int HC = decltype(hc)::value;
    if (c->gm16_on)
      launch<HC, __nv_bfloat16>(lam != nullptr, dot, lam_next, lam, sv, c->tma, j, w, d, part, st);
    else
      launch<HC, float>(lam != nullptr, dot, lam_next, lam, sv, c->tma, j, w, d, part, st);
  };
  switch (H) {
    case 2: go(std::integral_constant<int, 2>()); break;
    case 3: go(std::integral_constant<int, 3>()); break;
    case 4: go(std::integral_constant<int, 4>()); break;
    case 5: go(std::integral_constant<int, 5>()); break;
    default: c->set_error("sl_adjoint_step_tma: unsupported halo"); return CLAIRE_EINVAL;
  }
  if (dot) {
    dim3 grid, block;
    tiled_shape<2>(d, grid, block);
    c->dot_blocks = (long long)grid.x * grid.y * grid.z;
  }
  return CLAIRE_OK;
}

claire_status sl_tma_take_error(claire_ctx* c) {
  int flag = 0, zero = 0;
  CL_CUDA(c, cudaMemcpyFromSymbol(&flag, g_sl_tma_error, sizeof(int)));
  if (flag) {
    CL_CUDA(c, cudaMemcpyToSymbol(g_sl_tma_error, &zero, sizeof(int)));
    c->set_error("a gather's bounded wait for its staged operands ran out");
    return CLAIRE_ETIMEOUT;
  }
  return CLAIRE_OK;
}

}  // namespace claire
