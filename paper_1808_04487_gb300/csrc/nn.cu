// Layer kernels of the learned warm start: a 3D convolutional encoder-decoder that predicts the low-frequency part
// of the velocity from (m_T, m_R). Not part of the paper's method; the network only seeds v_0 of the unchanged
// Gauss-Newton-Krylov solve (Alg. 1), whose relative stopping test keeps g_0 = g(v = 0).
//
// Activations are channels-last BF16, gradients FP32 (rounded to BF16 where they feed a tensor-core product),
// weights [Cout][27][Cin]. Convolutions are 3x3x3, stride 1, periodic (the registration domain is periodic), and
// run as implicit GEMMs on the fifth-generation tensor cores (tcgen05.mma, BF16 operands staged in shared memory,
// FP32 accumulators in tensor memory; tc.cuh):
//   forward  y[m, co] = sum_{off, ci} x[nb(m, off), ci] w[co, off, ci]      (M = voxels, N = Cout, K = 27 Cin):
//            a CTA owns 128 voxels; per K step it stages the 128 neighbour rows of a group of offsets and the
//            matching Cout x (G Cin) weight slice, and one thread issues the MMAs into the 128 x Cout accumulator
//   dgrad    the forward kernel applied to dz with w^T[ci, 26 - off, co] = w[co, off, ci]
//   wgrad    dw[co, off, ci] = sum_m x[nb(m, off), ci] dz[m, co]           (M = G Cin rows for a group of G
//            offsets, N = Cout, K = voxels): a CTA owns one offset group and one chunk of voxels; chunks are
//            summed in a fixed order, so results do not depend on scheduling
// Every wait on the tensor core is bounded (about a second); a timeout sets an error flag that
// claire_nn_status reports, and the CTA still waits (bounded) for its MMAs and frees its tensor memory.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <mutex>

#include "impl.cuh"
#include "nn.cuh"
#include "tc.cuh"

namespace claire {
namespace nn {
namespace {

constexpr int kMaxC = 128;
constexpr int kTileM = 128;                        // voxels (forward) or output channels (wgrad) per CTA
constexpr int kTileK = 64;                         // voxels per K step of the weight gradient
constexpr long long kWaitCycles = 2000000000LL;    // bound of every tensor-core wait (~1 s at 2 GHz)

__device__ int g_nn_error = 0;                     // set by a CTA whose tensor-core wait timed out

// true when every given pointer (null ones ignored) is a multiple of `bytes`
inline bool aligned_to(unsigned bytes, std::initializer_list<const void*> ptrs) {
  for (const void* p : ptrs)
    if (reinterpret_cast<uintptr_t>(p) % bytes) return false;
  return true;
}

__device__ __forceinline__ int pw(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// coordinates of voxel m of the flattened batch
struct Vox {
  int b, i1, i2, i3;
};
__device__ __forceinline__ Vox vox_of(const Geo& g, int m) {
  Vox v;
  const unsigned t = g.by_n3.div((unsigned)m);
  v.i3 = m - (int)t * g.n3;
  const unsigned t2 = g.by_n2.div(t);
  v.i2 = (int)t - (int)t2 * g.n2;
  v.b = (int)g.by_n1.div(t2);
  v.i1 = (int)t2 - v.b * g.n1;
  return v;
}
// The periodic neighbours of one voxel: per axis the three wrapped coordinates (axis 1 already scaled to its slab
// of n2 rows), so the flattened index of the neighbour at offset off = 9 (o1 + 1) + 3 (o2 + 1) + (o3 + 1) is two
// selects per axis and one multiply-add.
struct Nbr {
  int r1[3], r2[3], r3[3];
};
__device__ __forceinline__ Nbr nbr_of(const Geo& g, const Vox& v) {
  Nbr n;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    n.r1[k] = (v.b * g.n1 + pw(v.i1 + k - 1, g.n1)) * g.n2;
    n.r2[k] = pw(v.i2 + k - 1, g.n2);
    n.r3[k] = pw(v.i3 + k - 1, g.n3);
  }
  return n;
}
__device__ __forceinline__ int sel3(const int* a, int k) { return k == 0 ? a[0] : (k == 1 ? a[1] : a[2]); }
__device__ __forceinline__ int nb_of(const Geo& g, const Nbr& n, int off) {
  return (sel3(n.r1, off / 9) + sel3(n.r2, (off / 3) % 3)) * g.n3 + sel3(n.r3, off % 3);
}

// Epilogue of the forward kernels for 16 consecutive output channels c0 .. c0+15 of voxel row m (v: the FP32
// accumulators): val = v + bias + skip, ReLU, then y (BF16) and/or yf (FP32, overwritten or accumulated), with
// 16-byte accesses (the per-channel arithmetic and its order are those of a scalar loop over the channels)
__device__ __forceinline__ void conv_epilogue16(float* v, long long m, int c0, int Cout, const float* __restrict__ bias,
                                                const bf16* __restrict__ skip, bf16* __restrict__ y,
                                                float* __restrict__ yf, int accum, int relu) {
  const long long o = m * Cout + c0;
  if (bias) {
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] += bias[c0 + j];
  }
  if (skip) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint4 u = *reinterpret_cast<const uint4*>(skip + o + 8 * h);
      const __nv_bfloat162* b2 = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 f = __bfloat1622float2(b2[k]);
        v[8 * h + 2 * k] += f.x;
        v[8 * h + 2 * k + 1] += f.y;
      }
    }
  }
  if (relu) {
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.f);
  }
  if (y) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint4 u;
      __nv_bfloat162* b2 = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
      for (int k = 0; k < 4; ++k) b2[k] = __floats2bfloat162_rn(v[8 * h + 2 * k], v[8 * h + 2 * k + 1]);
      *reinterpret_cast<uint4*>(y + o + 8 * h) = u;
    }
  }
  if (yf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float4* d = reinterpret_cast<float4*>(yf + o + 4 * q);
      float4 r = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      if (accum) {
        const float4 a = *d;
        r = make_float4(a.x + r.x, a.y + r.y, a.z + r.z, a.w + r.w);
      }
      *d = r;
    }
  }
}

// Forward convolution on tcgen05: 128 threads; thread r stages row r (voxel m0 + r). Offsets [off0, off1) of the
// 27 (split-K when the grid has few voxel tiles: blockIdx.y picks the range), taken G = group at a time so that
// a K step spans G Cin = min(64, Cin) or more channels: the A tile row r holds x[nb(m0 + r, off), ci] for the G
// offsets side by side (K index j Cin + ci), the B tile row co the matching contiguous run of w[co][off][ci]. Two
// shared-memory stages {A [128 x KS], B [Cout x KS]}, KS = G Cin, as K-major core-matrix tiles, with one
// mbarrier each: the staging of step i + 1 overlaps the MMAs of step i, and a stage is rewritten only after the
// MMAs that read it have completed. Epilogue: with part == nullptr the full result (bias, skip, ReLU) goes to
// y / yf; otherwise the raw FP32 partial sums go to part[blockIdx.y][m][co] for k_conv3_reduce.
// CIN > 0: the input channel count as a compile-time constant (see k_conv3_wgrad_tc), else Cin_rt.
template <int CIN>
__global__ void __launch_bounds__(128, 1) k_conv3_fwd_tc(const bf16* __restrict__ x, const bf16* __restrict__ w,
                                                         const float* __restrict__ bias,
                                                         const bf16* __restrict__ skip, bf16* __restrict__ y,
                                                         float* __restrict__ yf, int accum, Geo g, int Cin_rt,
                                                         int Cout, int relu, int offs_per_split, int group_rt,
                                                         float* __restrict__ part) {
  const int Cin = CIN > 0 ? CIN : Cin_rt;
  const int group = CIN > 0 ? (CIN < 64 ? 64 / CIN : 1) : group_rt;
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  unsigned char* sm = sm_raw + ((1024u - (tc::smem_addr(sm_raw) & 1023u)) & 1023u);
  const int KS = group * Cin;  // K extent of a full step
  const uint32_t a_bytes = (uint32_t)kTileM * KS * 2, b_bytes = (uint32_t)Cout * KS * 2;
  const uint32_t stage_bytes = a_bytes + b_bytes;  // a multiple of 512 (unswizzled tiles need 16-byte alignment)
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm + 2 * stage_bytes);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t ncols = tc::tmem_cols(Cout);
  const uint32_t bar_a[2] = {tc::smem_addr(bar), tc::smem_addr(bar + 1)};
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(slot), ncols);
  if (tid == 0) {
    tc::mbar_init(bar_a[0], 1);
    tc::mbar_init(bar_a[1], 1);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *slot;
  const int m0 = blockIdx.x * kTileM;
  const int m = m0 + tid;
  const bool valid = m < g.M;
  const Nbr nb = nbr_of(g, vox_of(g, valid ? m : 0));
  const int nvec = Cin / 8;
  const uint32_t kbytes = 16u * (uint32_t)KS;  // row-group stride of both tiles
  const uint32_t idesc = tc::idesc_bf16(kTileM, Cout);
  const uint32_t base = tc::smem_addr(sm);
  const int off0 = blockIdx.y * offs_per_split;
  const int off1 = off0 + offs_per_split < 27 ? off0 + offs_per_split : 27;
  const int nsteps = (off1 - off0 + group - 1) / group;
  uint32_t phase[2] = {0u, 0u};
  bool ok = true;
  for (int i = 0; i < nsteps && ok; ++i) {
    const int sidx = i & 1;
    const int oa = off0 + i * group;
    const int ob = oa + group < off1 ? oa + group : off1;
    const int nk = (ob - oa) * Cin;  // K extent of this step
    if (i >= 2) {
      // the MMAs of step i - 2 read this stage
      const bool mine = tc::mbar_wait(bar_a[sidx], phase[sidx], kWaitCycles);
      phase[sidx] ^= 1u;
      ok = __syncthreads_and(mine) != 0;
      if (!ok) break;
    }
    // neighbour rows (zero-filled past the last voxel) and the weight slice by cp.async: all of the thread's
    // copies in flight at once
    const uint32_t As = base + sidx * stage_bytes;
    const uint32_t Bs = As + a_bytes;
    for (int off = oa; off < ob; ++off) {
      const bf16* src = valid ? x + (long long)nb_of(g, nb, off) * Cin : x;
      const int kb = (off - oa) * Cin;
      for (int c = 0; c < nvec; ++c)
        tc::cp_async_16_zfill(As + tc::kmajor_offset(tid, kb + 8 * c, KS), src + 8 * c, valid);
    }
    const int nv = nk / 8;
    auto stage_w = [&](int nvc) {
      for (int q = tid; q < Cout * nvc; q += kTileM) {
        const int co = q / nvc, c = q - co * nvc;
        tc::cp_async_16(Bs + tc::kmajor_offset(co, 8 * c, KS), w + ((long long)co * 27 + oa) * Cin + 8 * c);
      }
    };
    if (CIN > 0 && nk == KS)
      stage_w(CIN > 0 ? (CIN < 64 ? 64 / CIN : 1) * CIN / 8 : 1);  // a full step: a constant divisor
    else
      stage_w(nv);
    tc::cp_async_wait_all();
    tc::fence_smem_to_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t a_s = base + sidx * stage_bytes, b_s = a_s + a_bytes;
      for (int kk = 0; kk < nk / 16; ++kk)
        tc::mma_bf16(tmem, tc::smem_desc(a_s + 256u * kk, 128u, kbytes), tc::smem_desc(b_s + 256u * kk, 128u, kbytes),
                     idesc, (i > 0 || kk > 0) ? 1u : 0u);
      tc::commit(bar_a[sidx]);
    }
  }
  // the last one or two stages in flight (their completion also covers every earlier MMA of the CTA)
  if (ok) {
    for (int sidx = 0; sidx < 2; ++sidx) {
      const int issued = (nsteps + 1 - sidx) / 2;  // commits made on this stage's barrier
      if (issued > 0) {
        const bool mine = tc::mbar_wait(bar_a[sidx], phase[sidx], kWaitCycles);
        phase[sidx] ^= 1u;
        ok = ok && mine;
      }
    }
    ok = __syncthreads_and(ok) != 0;
  }
  tc::fence_after();
  if (!ok) {
    if (tid == 0) atomicExch(&g_nn_error, 1);
    tc::mbar_wait(bar_a[0], phase[0], kWaitCycles);  // whatever is still in flight, bounded
    tc::mbar_wait(bar_a[1], phase[1], kWaitCycles);
  } else {
    const int r = m0 + 32 * warp + lane;  // this lane's accumulator row
    for (int c0 = 0; c0 < Cout; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
      if (r < g.M) {
        if (part) {
          float4* dst = reinterpret_cast<float4*>(part + ((long long)blockIdx.y * g.M + r) * Cout + c0);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
          conv_epilogue16(v, r, c0, Cout, bias, skip, y, yf, accum, relu);
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// split-K epilogue: out[m][co] = act(sum_s part[s][m][co] (s in order) + bias + skip)
__global__ void k_conv3_reduce(const float* __restrict__ part, int nsplit, const float* __restrict__ bias,
                               const bf16* __restrict__ skip, bf16* __restrict__ y, float* __restrict__ yf, int accum,
                               long long count, int Cout, int relu) {
  const long long step = (long long)gridDim.x * blockDim.x;
  const int co_step = (int)(step % Cout);
  long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int co = (int)(o % Cout);
  for (; o < count; o += step, co = co + co_step >= Cout ? co + co_step - Cout : co + co_step) {
    float val = 0.f;
    int sp = 0;
    for (; sp + 8 <= nsplit; sp += 8) {  // eight loads in flight, added in split order
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = part[(long long)(sp + u) * count + o];
#pragma unroll
      for (int u = 0; u < 8; ++u) val += v[u];
    }
    for (; sp < nsplit; ++sp) val += part[(long long)sp * count + o];
    if (bias) val += bias[co];
    if (skip) val += __bfloat162float(skip[o]);
    if (relu) val = fmaxf(val, 0.f);
    if (y) y[o] = __float2bfloat16_rn(val);
    if (yf) yf[o] = accum ? yf[o] + val : val;
  }
}

// Partial weight gradients on tcgen05. CTA (offset group og = blockIdx.x, voxel chunk blockIdx.y) handles the
// G = group offsets off = og G + j (those below 27) at once: the 128 x Cout accumulator row j Cin + ci holds
//   D[j Cin + ci, co] = sum over the chunk's voxels m of x[nb(m, off), ci] dz[m, co]
// (rows past the group's last offset stay zero), built in K steps of 64 voxels, then written to
// part[chunk][co][off][ci]. Both operands are staged as they lie in memory, channel index contiguous, i.e.
// MN-major: tile A holds 8-channel x 8-voxel core matrices at (row / 8) * 128 + (k / 8) * 2048 bytes, tile B
// likewise with the Cout channels of dz; thread t copies the 16-byte channel groups of voxel t % 64 (half t / 64
// of them). In the unswizzled MN-major layout the descriptor's leading offset steps along K (8-voxel groups) and
// its stride offset along M / N. Two stages with one mbarrier each: the loads of step s + 1 overlap the MMAs of s.
// CIN > 0: the input channel count as a compile-time constant (the network's 16, 32, 64, 128: the staging index
// arithmetic then divides by constants), else Cin_rt at run time.
template <int CIN>
__global__ void __launch_bounds__(128, 5) k_conv3_wgrad_tc(const bf16* __restrict__ dz, const bf16* __restrict__ x,
                                                           float* __restrict__ part, Geo g, int Cin_rt, int Cout,
                                                           int group, int chunk) {
  const int Cin = CIN > 0 ? CIN : Cin_rt;
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  unsigned char* sm = sm_raw + ((1024u - (tc::smem_addr(sm_raw) & 1023u)) & 1023u);
  constexpr uint32_t a_bytes = kTileM * kTileK * 2;  // 16 KB
  const uint32_t b_bytes = (uint32_t)Cout * kTileK * 2;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm + 2 * stage_bytes);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int off_first = blockIdx.x * group;
  const int ng = 27 - off_first < group ? 27 - off_first : group;  // offsets of this group
  const uint32_t ncols = tc::tmem_cols(Cout);
  const uint32_t bar_a[2] = {tc::smem_addr(bar), tc::smem_addr(bar + 1)};
  // rows past ng Cin of A are zero for every step: clear both A tiles once
  for (int s = 0; s < 2; ++s)
    for (int q = tid; q < (int)(a_bytes / 16); q += kTileM)
      reinterpret_cast<uint4*>(sm + s * stage_bytes)[q] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(slot), ncols);
  if (tid == 0) {
    tc::mbar_init(bar_a[0], 1);
    tc::mbar_init(bar_a[1], 1);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *slot;
  // MN-major operands: bit 15 (A) and bit 16 (B) of the instruction descriptor
  const uint32_t idesc = tc::idesc_bf16(kTileM, Cout) | (1u << 15) | (1u << 16);
  const uint32_t base = tc::smem_addr(sm);
  const uint32_t a_kgroup = 16u * kTileM, b_kgroup = 16u * (uint32_t)Cout;  // bytes between 8-voxel groups
  const int k = tid & (kTileK - 1), half = tid >> 6;
  const int c0 = blockIdx.y * chunk;
  const int c1 = (long long)c0 + chunk < g.M ? c0 + chunk : (int)g.M;
  const int nsteps = (c1 - c0 + kTileK - 1) / kTileK;
  const uint32_t kpos = (uint32_t)(k & 7) * 16u;  // K row of the voxel inside its core matrix
  const int cvec = Cin / 8, nva = ng * cvec, nvb = Cout / 8;  // 16-byte vectors of one voxel
  uint32_t phase[2] = {0u, 0u};
  bool ok = true;
  for (int s = 0; s < nsteps && ok; ++s) {
    const int sidx = s & 1;
    const int mv = c0 + s * kTileK + k;
    const bool valid = mv < c1;
    const Nbr nb = nbr_of(g, vox_of(g, valid ? mv : c0));
    // issue this step's loads before waiting for the stage
    uint4 va[8], vb[8];
    if constexpr (CIN > 0) {
      // half h stages the A vectors v = 8 h .. 8 h + 7 of its voxel (v = j CV + cv: offset j, channel vector cv),
      // so one neighbour index serves the CV vectors of an offset
      constexpr int CV = CIN / 8;
      if constexpr (CV <= 8) {
        const bf16* row = x;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = half * (8 / CV) + q / CV;
          if (q % CV == 0) row = x + (long long)nb_of(g, nb, off_first + (j < ng ? j : 0)) * CIN;
          va[q] = (valid && j < ng) ? *reinterpret_cast<const uint4*>(row + 8 * (q % CV)) : make_uint4(0u, 0u, 0u, 0u);
        }
      } else {
        // one offset of 16 channel vectors: half h takes vectors 8 h .. 8 h + 7
        const bf16* row = x + (long long)nb_of(g, nb, off_first) * CIN + 64 * half;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          va[q] = valid ? *reinterpret_cast<const uint4*>(row + 8 * q) : make_uint4(0u, 0u, 0u, 0u);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int v = half + 2 * q;
        va[q] = make_uint4(0u, 0u, 0u, 0u);
        if (valid && v < nva) {
          const int j = v / cvec, cv = v - j * cvec;
          va[q] = *reinterpret_cast<const uint4*>(x + (long long)nb_of(g, nb, off_first + j) * Cin + 8 * cv);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int v = half + 2 * q;
      vb[q] = make_uint4(0u, 0u, 0u, 0u);
      if (valid && v < nvb) vb[q] = *reinterpret_cast<const uint4*>(dz + (long long)mv * Cout + 8 * v);
    }
    if (s >= 2) {
      // the MMAs of step s - 2 read this stage
      const bool mine = tc::mbar_wait(bar_a[sidx], phase[sidx], kWaitCycles);
      phase[sidx] ^= 1u;
      ok = __syncthreads_and(mine) != 0;
      if (!ok) break;
    }
    unsigned char* As = sm + sidx * stage_bytes;
    unsigned char* Bs = As + a_bytes;
    const uint32_t koff_a = (uint32_t)(k >> 3) * a_kgroup + kpos, koff_b = (uint32_t)(k >> 3) * b_kgroup + kpos;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      // A vector v (offset j, channel vector cv) is core-matrix row group (j Cin + 8 cv) / 8 = v
      const int v = CIN > 0 ? 8 * half + q : half + 2 * q;
      if (v < nva) *reinterpret_cast<uint4*>(As + v * 128 + koff_a) = va[q];
      const int vbv = half + 2 * q;
      if (vbv < nvb) *reinterpret_cast<uint4*>(Bs + vbv * 128 + koff_b) = vb[q];
    }
    tc::fence_smem_to_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t a_s = base + sidx * stage_bytes, b_s = a_s + a_bytes;
      for (int kk = 0; kk < kTileK / 16; ++kk)
        tc::mma_bf16(tmem, tc::smem_desc(a_s + 2u * a_kgroup * kk, a_kgroup, 128u),
                     tc::smem_desc(b_s + 2u * b_kgroup * kk, b_kgroup, 128u), idesc, (s > 0 || kk > 0) ? 1u : 0u);
      tc::commit(bar_a[sidx]);
    }
  }
  if (ok) {
    for (int sidx = 0; sidx < 2; ++sidx) {
      if ((nsteps + 1 - sidx) / 2 > 0) {  // one commit on this stage's barrier is still unwaited
        const bool mine = tc::mbar_wait(bar_a[sidx], phase[sidx], kWaitCycles);
        phase[sidx] ^= 1u;
        ok = ok && mine;
      }
    }
    ok = __syncthreads_and(ok) != 0;
  }
  tc::fence_after();
  if (!ok) {
    if (tid == 0) atomicExch(&g_nn_error, 1);
    tc::mbar_wait(bar_a[0], phase[0], kWaitCycles);  // whatever is still in flight, bounded
    tc::mbar_wait(bar_a[1], phase[1], kWaitCycles);
  } else if (nsteps > 0) {
    const int r = 32 * warp + lane;  // accumulator row j Cin + ci
    const int j = r / Cin, ci = r - j * Cin;
    float* dst = part + (long long)blockIdx.y * Cout * 27 * Cin + (long long)(off_first + j) * Cin + ci;
    for (int n0 = 0; n0 < Cout; n0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)n0, v);
      if (j < ng) {
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) dst[(long long)(n0 + jj) * 27 * Cin] = v[jj];
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// Fixed-order sums over chunks: dst[i] = sum_c part[c][i]. A 256-thread CTA takes opb consecutive outputs i;
// thread t sums range r = t / opb, one contiguous R-th of the chunks (R = 256 / opb: about eight chunks per range,
// from R = 1 for a few chunks of many outputs to R = 64 for the 1216 per-block bias partials of a few channels), in
// chunk order with eight loads in flight, and the R range sums are added in range order. Two independent jobs
// share one launch (CTAs [0, a.blocks) take job a, the rest job b), so the bias gradient of a layer is summed in
// the launch that sums its weight gradient. (One thread per i summing all chunks
// in order left a few dozen CTAs on the GPU, each thread a chain of ~190 strided loads.)
struct SumJob {
  const float* part;
  float* dst;
  long long count;
  int nchunks, opb, blocks;
};
inline SumJob sum_job(const float* part, int nchunks, long long count, float* dst) {
  SumJob j;
  j.part = part;
  j.dst = dst;
  j.count = count;
  j.nchunks = nchunks;
  int R = 1;
  while (R < 64 && 8 * 2 * R <= nchunks) R *= 2;
  j.opb = 256 / R;
  const long long b = (count + j.opb - 1) / j.opb;
  j.blocks = (int)(b < 4864 ? (b > 0 ? b : 1) : 4864);
  return j;
}
__global__ void __launch_bounds__(256) k_sum_chunks(SumJob a, SumJob b) {
  __shared__ float red[256];
  const bool first = (int)blockIdx.x < a.blocks;
  const SumJob& j = first ? a : b;
  const int blk = first ? (int)blockIdx.x : (int)blockIdx.x - a.blocks;
  const int oi = threadIdx.x % j.opb, r = threadIdx.x / j.opb, R = 256 / j.opb;
  const int per = (j.nchunks + R - 1) / R;
  const int c0 = r * per, c1 = min(j.nchunks, c0 + per);
  for (long long base = (long long)blk * j.opb; base < j.count; base += (long long)j.blocks * j.opb) {
    const long long i = base + oi;
    float s = 0.f;
    if (i < j.count) {
      for (int c = c0; c < c1; c += 8) {  // the last batch's loads past c1 are skipped
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = c + u < c1 ? j.part[(long long)(c + u) * j.count + i] : 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (c + u < c1) s += v[u];
      }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    if ((int)threadIdx.x < j.opb && base + threadIdx.x < j.count) {
      float t = red[threadIdx.x];
      for (int k = 1; k < R; ++k) t += red[k * j.opb + threadIdx.x];
      j.dst[base + threadIdx.x] = t;
    }
    __syncthreads();
  }
}
inline cudaError_t sum_chunks(const SumJob& a, const SumJob* b, cudaStream_t st) {
  SumJob none = a;
  none.blocks = 0;
  k_sum_chunks<<<a.blocks + (b ? b->blocks : 0), 256, 0, st>>>(a, b ? *b : none);
  return cudaGetLastError();
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

// k_wt_flip for a table of layers in one launch: CTA (layer t, offset off) transposes the Cout x Cin slice
// w[co][off][ci] into wt[ci][26 - off][co] through shared memory (coalesced reads along ci, writes along co)
__global__ void __launch_bounds__(256) k_wt_flip_all(const bf16* __restrict__ w, bf16* __restrict__ wt,
                                                     FlipTable tab) {
  __shared__ bf16 tile[kMaxC][kMaxC + 2];
  const int t = blockIdx.x / 27, off = blockIdx.x - 27 * (blockIdx.x / 27);
  const int Cin = tab.cin[t], Cout = tab.cout[t];
  const bf16* src = w + tab.woff[t];
  bf16* dst = wt + tab.woff[t];
  for (int q = threadIdx.x; q < Cout * Cin; q += 256) {
    const int co = q / Cin, ci = q - co * Cin;
    tile[co][ci] = src[(co * 27 + off) * Cin + ci];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < Cout * Cin; q += 256) {
    const int ci = q / Cout, co = q - ci * Cout;
    dst[(ci * 27 + 26 - off) * Cout + co] = tile[co][ci];
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

constexpr int kBiasBlocks = 1216;  // 8 per SM: enough rows in flight for the fused ReLU backward

// Per-block channel sums of v = dy (y > 0) (y null: v = dy), fused with dzb = bf16(v) and dz = v (each written only
// when given): thread t owns the V channels V g .. V g + V - 1, g = t % G (G = C / V; V = 4, one 16-byte load of
// dy, where C allows) and the rows t / G + k rpb (rpb = blockDim / G), four rows' loads in flight, summed in row
// order; the rpb row sums of a channel are then added in order. The bias gradient (bias_grad, relu_bwd_bias) is the
// fixed-order sum of these partials over the blocks; the FP32 dz is written only for a layer whose gradient also
// feeds a skip connection (the weight and input gradients read dzb).
template <int V> __device__ __forceinline__ void relu_row(const float* __restrict__ dy, const bf16* __restrict__ y,
                                                          long long i, float* v) {
  if constexpr (V == 4) {
    const float4 d = *reinterpret_cast<const float4*>(dy + i);
    v[0] = d.x;
    v[1] = d.y;
    v[2] = d.z;
    v[3] = d.w;
    if (y) {
      const uint2 u = *reinterpret_cast<const uint2*>(y + i);
      const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
      const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
      v[0] = a.x > 0.f ? v[0] : 0.f;
      v[1] = a.y > 0.f ? v[1] : 0.f;
      v[2] = b.x > 0.f ? v[2] : 0.f;
      v[3] = b.y > 0.f ? v[3] : 0.f;
    }
  } else {
    v[0] = (y == nullptr || __bfloat162float(y[i]) > 0.f) ? dy[i] : 0.f;
  }
}
template <int V> __device__ __forceinline__ void relu_store(float* __restrict__ dz, bf16* __restrict__ dzb, long long i,
                                                            const float* v) {
  if constexpr (V == 4) {
    if (dz) *reinterpret_cast<float4*>(dz + i) = make_float4(v[0], v[1], v[2], v[3]);
    if (dzb) {
      uint2 u;
      *reinterpret_cast<__nv_bfloat162*>(&u.x) = __floats2bfloat162_rn(v[0], v[1]);
      *reinterpret_cast<__nv_bfloat162*>(&u.y) = __floats2bfloat162_rn(v[2], v[3]);
      *reinterpret_cast<uint2*>(dzb + i) = u;
    }
  } else {
    if (dz) dz[i] = v[0];
    if (dzb) dzb[i] = __float2bfloat16_rn(v[0]);
  }
}
template <int V>
__global__ void __launch_bounds__(256) k_relu_bwd_bias(const float* __restrict__ dy, const bf16* __restrict__ y,
                                                       float* __restrict__ dz, bf16* __restrict__ dzb, long long M,
                                                       int C, float* __restrict__ part) {
  __shared__ float sh[256 * V];
  const int G = C / V;
  const int g = threadIdx.x % G, r = threadIdx.x / G, rpb = blockDim.x / G;
  const int c0 = V * g;
  const long long step = (long long)gridDim.x * rpb;
  float s[V];
#pragma unroll
  for (int j = 0; j < V; ++j) s[j] = 0.f;
  long long m = (long long)blockIdx.x * rpb + r;
  for (; m + 3 * step < M; m += 4 * step) {
    float v[4][V];
#pragma unroll
    for (int u = 0; u < 4; ++u) relu_row<V>(dy, y, (m + u * step) * C + c0, v[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      relu_store<V>(dz, dzb, (m + u * step) * C + c0, v[u]);
#pragma unroll
      for (int j = 0; j < V; ++j) s[j] += v[u][j];
    }
  }
  for (; m < M; m += step) {
    float v[V];
    relu_row<V>(dy, y, m * C + c0, v);
    relu_store<V>(dz, dzb, m * C + c0, v);
#pragma unroll
    for (int j = 0; j < V; ++j) s[j] += v[j];
  }
#pragma unroll
  for (int j = 0; j < V; ++j) sh[threadIdx.x * V + j] = s[j];
  __syncthreads();
  if ((int)threadIdx.x < C) {
    const int gx = threadIdx.x / V, j = threadIdx.x - gx * V;
    float t = 0.f;
    for (int k = 0; k < rpb; ++k) t += sh[(k * G + gx) * V + j];
    part[(long long)blockIdx.x * C + threadIdx.x] = t;
  }
}
// per-block channel sums of (dy, y, dz, dzb) as above, 16-byte rows where C allows
inline void launch_relu_bwd_bias(const float* dy, const bf16* y, float* dz, bf16* dzb, long long M, int C,
                                 float* part, cudaStream_t st) {
  if (C % 4 == 0 && aligned_to(16, {dy, dz}) && aligned_to(8, {y, dzb})) {
    const int G = C / 4;
    k_relu_bwd_bias<4><<<kBiasBlocks, (256 / G) * G, 0, st>>>(dy, y, dz, dzb, M, C, part);
  } else {
    k_relu_bwd_bias<1><<<kBiasBlocks, (256 / C) * C, 0, st>>>(dy, y, dz, dzb, M, C, part);
  }
}

// Pooling and upsampling: thread (coarse voxel p, channel vector cv) moves V channels (V = 8 BF16 or 4 FP32 in
// one 16-byte access when C allows, else 1) between p and the 2 x 2 x 2 fine voxels under it, fine voxel
// d = 4 d1 + 2 d2 + d3 at f0 + d1 P + d2 R + d3 (R = fine row, P = fine plane); sums run over d in ascending order.
struct Block8 {
  long long f0;
  long long R, P;
  __device__ __forceinline__ long long at(int d) const { return f0 + (d >> 2) * P + ((d >> 1) & 1) * R + (d & 1); }
};
__device__ __forceinline__ Block8 block_of(const Geo& gc, int p) {
  const Vox v = vox_of(gc, p);
  Block8 k;
  k.R = 2LL * gc.n3;
  k.P = 4LL * gc.n2 * gc.n3;
  k.f0 = ((long long)(v.b * gc.n1 + v.i1) * 2 * (2 * gc.n2) + 2 * v.i2) * (2 * gc.n3) + 2 * v.i3;
  return k;
}
template <int V> __device__ __forceinline__ void ld_vec(const bf16* p, float* f) {
  if constexpr (V == 8) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 t = __bfloat1622float2(h[k]);
      f[2 * k] = t.x;
      f[2 * k + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) f[k] = __bfloat162float(p[k]);
  }
}
template <int V> __device__ __forceinline__ void ld_vec(const float* p, float* f) {
  if constexpr (V == 4) {
    const float4 u = *reinterpret_cast<const float4*>(p);
    f[0] = u.x;
    f[1] = u.y;
    f[2] = u.z;
    f[3] = u.w;
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) f[k] = p[k];
  }
}
template <int V> __device__ __forceinline__ void st_vec(float* p, const float* f) {
  if constexpr (V == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(f[0], f[1], f[2], f[3]);
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) p[k] = f[k];
  }
}

template <int V>
__global__ void k_pool_fwd(const bf16* __restrict__ x, bf16* __restrict__ y, Geo gc, int C, FastDiv by_g) {
  const long long total = gc.M * (C / V);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)by_g.div((unsigned)i), c = (int)(i - (long long)p * (C / V)) * V;
    const Block8 k = block_of(gc, p);
    float s[V];
#pragma unroll
    for (int j = 0; j < V; ++j) s[j] = 0.f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      float f[V];
      ld_vec<V>(x + k.at(d) * C + c, f);
#pragma unroll
      for (int j = 0; j < V; ++j) s[j] += f[j];
    }
    bf16* dst = y + (long long)p * C + c;
    if constexpr (V == 8) {
      uint4 u;
      __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
      for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(0.125f * s[2 * j], 0.125f * s[2 * j + 1]);
      *reinterpret_cast<uint4*>(dst) = u;
    } else {
#pragma unroll
      for (int j = 0; j < V; ++j) dst[j] = __float2bfloat16_rn(0.125f * s[j]);
    }
  }
}
template <int V>
__global__ void k_pool_bwd(const float* __restrict__ dy, float* __restrict__ dx, int accum, Geo gc, int C,
                           FastDiv by_g) {
  const long long total = gc.M * (C / V);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)by_g.div((unsigned)i), c = (int)(i - (long long)p * (C / V)) * V;
    const Block8 k = block_of(gc, p);
    float v[V];
    ld_vec<V>(dy + (long long)p * C + c, v);
#pragma unroll
    for (int j = 0; j < V; ++j) v[j] *= 0.125f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      float* dst = dx + k.at(d) * C + c;
      float o[V];
      if (accum) {
        ld_vec<V>(dst, o);
#pragma unroll
        for (int j = 0; j < V; ++j) o[j] += v[j];
      } else {
#pragma unroll
        for (int j = 0; j < V; ++j) o[j] = v[j];
      }
      st_vec<V>(dst, o);
    }
  }
}
template <int V>
__global__ void k_up_fwd(const bf16* __restrict__ x, bf16* __restrict__ y, Geo gc, int C, FastDiv by_g) {
  const long long total = gc.M * (C / V);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)by_g.div((unsigned)i), c = (int)(i - (long long)p * (C / V)) * V;
    const Block8 k = block_of(gc, p);
    if constexpr (V == 8) {
      const uint4 u = *reinterpret_cast<const uint4*>(x + (long long)p * C + c);
#pragma unroll
      for (int d = 0; d < 8; ++d) *reinterpret_cast<uint4*>(y + k.at(d) * C + c) = u;
    } else {
      bf16 u[V];
#pragma unroll
      for (int j = 0; j < V; ++j) u[j] = x[(long long)p * C + c + j];
#pragma unroll
      for (int d = 0; d < 8; ++d)
#pragma unroll
        for (int j = 0; j < V; ++j) y[k.at(d) * C + c + j] = u[j];
    }
  }
}
template <int V>
__global__ void k_up_bwd(const float* __restrict__ dy, float* __restrict__ dx, int accum, Geo gc, int C,
                         FastDiv by_g) {
  const long long total = gc.M * (C / V);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)by_g.div((unsigned)i), c = (int)(i - (long long)p * (C / V)) * V;
    const Block8 k = block_of(gc, p);
    float s[V];
#pragma unroll
    for (int j = 0; j < V; ++j) s[j] = 0.f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      float f[V];
      ld_vec<V>(dy + k.at(d) * C + c, f);
#pragma unroll
      for (int j = 0; j < V; ++j) s[j] += f[j];
    }
    float* dst = dx + (long long)p * C + c;
    if (accum) {
      float o[V];
      ld_vec<V>(dst, o);
#pragma unroll
      for (int j = 0; j < V; ++j) s[j] += o[j];
    }
    st_vec<V>(dst, s);
  }
}

// loss partials (FP64) and gradient of the mean squared error over the first cu of C channels: thread per voxel,
// C gradient values written (zero past cu), 16-byte stores when C allows
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ pred, const float* __restrict__ target,
                                             float* __restrict__ grad, long long M, int C, int cu, double inv_count,
                                             double* __restrict__ partials, int vec) {
  double acc = 0.0;
  const float gscale = float(2.0 * inv_count);
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < M;
       m += (long long)gridDim.x * blockDim.x) {
    float e[4] = {0.f, 0.f, 0.f, 0.f};  // the first min(cu, 4) errors
    for (int c = 0; c < cu; ++c) {
      const float ec = pred[m * C + c] - target[m * cu + c];
      acc += double(ec) * double(ec);
      if (c < 4) e[c] = ec;
    }
    if (!grad) continue;
    float* g = grad + m * C;
    if (vec) {
      *reinterpret_cast<float4*>(g) = make_float4(gscale * e[0], 1 < cu ? gscale * e[1] : 0.f,
                                                  2 < cu ? gscale * e[2] : 0.f, 3 < cu ? gscale * e[3] : 0.f);
      for (int c = 4; c < C; c += 4) *reinterpret_cast<float4*>(g + c) = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      for (int c = 0; c < C; ++c) g[c] = c < cu ? gscale * (pred[m * C + c] - target[m * cu + c]) : 0.f;
    }
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

__device__ __forceinline__ float adam_one(float& p, float g, float& m1, float& m2, float lr, float b1, float b2,
                                          float eps, float c1, float c2) {
  const float a = b1 * m1 + (1.f - b1) * g;
  const float v = b2 * m2 + (1.f - b2) * g * g;
  m1 = a;
  m2 = v;
  p = p - lr * (a * c1) / (sqrtf(v * c2) + eps);
  return p;
}
// one Adam step per element; four elements per thread with 16-byte accesses where count and the pointers allow
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m1,
                       float* __restrict__ m2, bf16* __restrict__ pb, long long count, float lr, float b1, float b2,
                       float eps, float c1, float c2, int vec) {
  if (vec) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; 4 * i < count;
         i += (long long)gridDim.x * blockDim.x) {
      float4 P = reinterpret_cast<float4*>(p)[i], A = reinterpret_cast<float4*>(m1)[i],
             B = reinterpret_cast<float4*>(m2)[i];
      const float4 G = reinterpret_cast<const float4*>(gr)[i];
      adam_one(P.x, G.x, A.x, B.x, lr, b1, b2, eps, c1, c2);
      adam_one(P.y, G.y, A.y, B.y, lr, b1, b2, eps, c1, c2);
      adam_one(P.z, G.z, A.z, B.z, lr, b1, b2, eps, c1, c2);
      adam_one(P.w, G.w, A.w, B.w, lr, b1, b2, eps, c1, c2);
      reinterpret_cast<float4*>(p)[i] = P;
      reinterpret_cast<float4*>(m1)[i] = A;
      reinterpret_cast<float4*>(m2)[i] = B;
      if (pb) {
        uint2 u;
        *reinterpret_cast<__nv_bfloat162*>(&u.x) = __floats2bfloat162_rn(P.x, P.y);
        *reinterpret_cast<__nv_bfloat162*>(&u.y) = __floats2bfloat162_rn(P.z, P.w);
        reinterpret_cast<uint2*>(pb)[i] = u;
      }
    }
    return;
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    float P = p[i], A = m1[i], B = m2[i];
    adam_one(P, gr[i], A, B, lr, b1, b2, eps, c1, c2);
    p[i] = P;
    m1[i] = A;
    m2[i] = B;
    if (pb) pb[i] = __float2bfloat16_rn(P);
  }
}

// network input of a minibatch: sample b (of nb) is images[idx[b]] = (m_T, m_R), [2][N0]; channel 0 = m_T,
// channel 1 = sdiff (m_R - m_T) (formed in FP32 before rounding), channels 2 .. C-1 zero; thread per voxel
__global__ void k_pack_images(const float* __restrict__ images, SampleIdx idx, int nb, bf16* __restrict__ dst,
                              long long N0, int C, float sdiff) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nb * N0;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / N0);
    const long long m = i - b * N0;
    const float* src = images + idx.v[b] * 2 * N0;
    const float v0 = src[m], v1 = sdiff * (src[N0 + m] - src[m]);
    bf16* d = dst + i * C;
    if (C % 8 == 0) {
      uint4 u = make_uint4(0u, 0u, 0u, 0u);
      __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
      u.x = *reinterpret_cast<unsigned*>(&h);
      *reinterpret_cast<uint4*>(d) = u;
      for (int c = 8; c < C; c += 8) *reinterpret_cast<uint4*>(d + c) = make_uint4(0u, 0u, 0u, 0u);
    } else {
      for (int c = 0; c < C; ++c) d[c] = __float2bfloat16_rn(c == 0 ? v0 : (c == 1 ? v1 : 0.f));
    }
  }
}
// targets of a minibatch: dst[b][m][c] = s * targets[idx[b]][c][m] (ncomp components); thread per voxel
__global__ void k_interleave_batch(const float* __restrict__ targets, SampleIdx idx, int nb, float* __restrict__ dst,
                                   long long N0, int ncomp, float s) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nb * N0;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / N0);
    const long long m = i - b * N0;
    const float* src = targets + idx.v[b] * ncomp * N0 + m;
    for (int c = 0; c < ncomp; ++c) dst[i * ncomp + c] = s * src[c * N0];
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

// offsets per CTA of the weight gradient: as many as fill the 128 accumulator rows (G Cin <= 128), at most 27
inline int wgrad_group(int Cin) {
  const int G = kTileM / Cin;
  return G > 27 ? 27 : (G < 1 ? 1 : G);
}
// voxels per CTA of the weight gradient: about five CTAs per SM (its occupancy limit) over the offset groups x
// chunks, whole K steps
inline int wgrad_chunk(const Geo& g, int Cin) {
  const long long ngroups = (27 + wgrad_group(Cin) - 1) / wgrad_group(Cin);
  const long long target = (5 * 152 + ngroups - 1) / ngroups;
  long long per = (g.M + target - 1) / target;
  per = (per + kTileK - 1) / kTileK * kTileK;
  return (int)(per < kTileK ? kTileK : per);
}
// neighbour offsets per K step of the forward convolution: a step spans at least 64 channels when Cin allows
inline int fwd_group(int Cin) { return Cin < 64 ? (64 / Cin > 0 ? 64 / Cin : 1) : 1; }

inline size_t fwd_smem(int Cin, int Cout) {
  const size_t KS = size_t(fwd_group(Cin)) * Cin;
  return 1024 + 2 * (size_t(kTileM) * KS * 2 + size_t(Cout) * KS * 2) + 32;
}
// neighbour offsets per CTA of the forward convolution: all 27, or a split over blockIdx.y (partial sums reduced by
// k_conv3_reduce) when a batch of 8 of these grids has fewer voxel tiles than about two CTAs per SM. The choice
// depends on the grid, not on the batch size, so a sample's result does not depend on the batch it is in.
inline int fwd_offsets_per_split(const Geo& g) {
  const long long per_sample = g.M / g.B;
  const long long tiles = (8 * per_sample + kTileM - 1) / kTileM;
  if (tiles >= 2 * 152) return 27;
  long long split = (2 * 152 + tiles - 1) / tiles;
  if (split > 27) split = 27;
  return (int)((27 + split - 1) / split);
}
inline size_t wgrad_smem(int Cout) { return 1024 + 2 * (size_t(kTileM) * kTileK * 2 + size_t(Cout) * kTileK * 2) + 32; }

// ---- forward convolution from a shared-memory halo -----------------------------------------------------------
// A CTA covers tz (1, 2 or 4) planes of a tile of 8 (i3) x 16 (i2) voxels of one sample (128 rows of the implicit
// GEMM per plane, each plane its own TMEM accumulator). Its input halo -- the 10 x 18 x (tz + 2) voxels around the
// tile, periodic -- is loaded once, as Cin/8 planes of 16-byte voxel rows (8 channels each):
// [plane][hz][hy][hx] x 16 B. In that layout the A operand of every neighbour offset is a shifted view of the halo
// that a matrix descriptor expresses directly -- core matrix (row group g, channel group j) at plane j, rows
// (p + o1, g + o2, o3 .. o3 + 7) for tile plane p: leading (K) byte offset = one plane, stride (M) byte offset = one
// halo row of 10 voxels = 160 B -- so no per-offset staging is needed: one thread issues the 27 Cin / 16 MMAs per
// tile plane back to back against the resident weights (K-major [Cout][27 Cin]). The MMAs of a voxel run in the K
// order of k_conv3_fwd_tc (offsets ascending, 16 channels at a time), so its accumulator and result are the same;
// the tz planes share one weight load and read (tz + 2) / tz halo rows per voxel row instead of 3.
constexpr int kHaloRowsPerZ = 18 * 10;
inline int halo_rows(int tz) { return (tz + 2) * kHaloRowsPerZ; }

inline size_t halo_smem(int Cin, int Cout, int tz) {
  const size_t halo = (size_t(Cin / 8) * halo_rows(tz) * 16 + 1023) / 1024 * 1024;
  return 1024 + halo + size_t(Cout) * 27 * Cin * 2 + 64;
}
inline bool halo_fits(const Geo& g, int Cin, int Cout) {
  return Cin % 16 == 0 && Cin <= 64 && g.n3 % 8 == 0 && g.n2 % 16 == 0 && 27LL * Cout * Cin * 2 <= 110592 &&
         halo_smem(Cin, Cout, 1) <= 227 * 1024;
}
// tile planes per CTA: four or two where the grid has enough tiles for about three or four CTAs per SM of that
// size and the halo stays small (C_in <= 32), else one
// the CTAs that fit an SM by shared memory also fit its 512 tensor-memory columns (tz Cout accumulator columns each)
inline bool halo_planes_fit(int Cin, int Cout, int tz) {
  const size_t sm = halo_smem(Cin, Cout, tz);
  if (sm > 227 * 1024) return false;
  const size_t ctas = (228 * 1024) / (sm + 1024);
  return ctas * tc::tmem_cols(tz * Cout) <= 512;
}
inline int halo_tz(const Geo& g, int Cin, int Cout) {
  const long long tiles = (long long)(g.n3 / 8) * (g.n2 / 16) * g.n1 * g.B;
  if (Cin > 32) return 1;
  if (g.n1 % 4 == 0 && tiles / 4 >= 3 * 152 && halo_planes_fit(Cin, Cout, 4)) return 4;
  return (g.n1 % 2 == 0 && tiles / 2 >= 4 * 152 && halo_planes_fit(Cin, Cout, 2)) ? 2 : 1;
}

template <int CIN>  // CIN > 0: the input channel count at compile time (constant divisors), else Cin_rt
__global__ void __launch_bounds__(128, 1) k_conv3_fwd_halo(const bf16* __restrict__ x, const bf16* __restrict__ w,
                                                           const float* __restrict__ bias,
                                                           const bf16* __restrict__ skip, bf16* __restrict__ y,
                                                           float* __restrict__ yf, int accum, Geo g, int Cin_rt,
                                                           int Cout, int relu, int tz) {
  const int Cin = CIN > 0 ? CIN : Cin_rt;
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  unsigned char* sm = sm_raw + ((1024u - (tc::smem_addr(sm_raw) & 1023u)) & 1023u);
  const int nplanes = Cin / 8;
  const int K = 27 * Cin;
  const int hrows = (tz + 2) * kHaloRowsPerZ;
  const uint32_t hplane = (uint32_t)hrows * 16u;  // bytes of one channel-group plane of the halo
  unsigned char* halo = sm;
  unsigned char* Bs = sm + (size_t(nplanes) * hplane + 1023) / 1024 * 1024;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(Bs + size_t(Cout) * K * 2);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t ncols = tc::tmem_cols(tz * Cout);
  const uint32_t b0 = tc::smem_addr(bar);
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(slot), ncols);
  if (tid == 0) tc::mbar_init(b0, 1);
  // the tile: blockIdx.x = ((b (n1 / tz) + zt) ty + iy) tx + ix
  const int tx = g.n3 / 8, ty = g.n2 / 16, nzt = g.n1 / tz;
  int t = blockIdx.x;
  const int ix = t % tx;
  t /= tx;
  const int iy = t % ty;
  t /= ty;
  const int z = (t % nzt) * tz, b = t / nzt;
  const int x0 = 8 * ix, y0 = 16 * iy;
  // halo rows and weights by cp.async: every copy of the thread in flight at once, none through registers
  const uint32_t hsm = tc::smem_addr(halo), bsm = tc::smem_addr(Bs);
  for (int q = tid; q < nplanes * hrows; q += 128) {
    const int cc = q / hrows, r = q - cc * hrows;
    const int hz = r / kHaloRowsPerZ, rr = r - hz * kHaloRowsPerZ;
    const int hy = rr / 10, hx = rr - hy * 10;
    const int gz = pw(z + hz - 1, g.n1), gy = pw(y0 + hy - 1, g.n2), gx = pw(x0 + hx - 1, g.n3);
    const long long vox = ((long long)(b * g.n1 + gz) * g.n2 + gy) * g.n3 + gx;
    tc::cp_async_16(hsm + (uint32_t)(cc * hrows + r) * 16u, x + vox * Cin + 8 * cc);
  }
  const int nv = K / 8;
  for (int q = tid; q < Cout * nv; q += 128) {
    const int co = q / nv, c = q - co * nv;
    tc::cp_async_16(bsm + (uint32_t)tc::kmajor_offset(co, 8 * c, K), w + (long long)co * K + 8 * c);
  }
  tc::cp_async_wait_all();
  tc::fence_smem_to_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *slot;
  if (tid == 0) {
    const uint32_t idesc = tc::idesc_bf16(kTileM, Cout);
    const int kpo = Cin / 16;  // MMAs per offset
    for (int p = 0; p < tz; ++p) {
      for (int off = 0; off < 27; ++off) {
        const int o1 = off / 9, o2 = (off / 3) % 3, o3 = off % 3;
        const uint32_t row0 = (uint32_t)(((p + o1) * 18 + o2) * 10 + o3);
        for (int kk = 0; kk < kpo; ++kk) {
          const uint64_t ad = tc::smem_desc(hsm + 2u * kk * hplane + 16u * row0, hplane, 160u);
          const uint64_t bd = tc::smem_desc(bsm + 256u * (off * kpo + kk), 128u, 16u * K);
          tc::mma_bf16(tmem + (uint32_t)(p * Cout), ad, bd, idesc, (off > 0 || kk > 0) ? 1u : 0u);
        }
      }
    }
    tc::commit(b0);
  }
  bool ok = tc::mbar_wait(b0, 0, kWaitCycles);
  ok = __syncthreads_and(ok) != 0;
  tc::fence_after();
  if (!ok) {
    if (tid == 0) atomicExch(&g_nn_error, 1);
    tc::mbar_wait(b0, 0, kWaitCycles);  // whatever is still in flight, bounded
  } else {
    const int r = 32 * warp + lane;  // this lane's accumulator row: voxel (x0 + r % 8, y0 + r / 8) of each plane
    for (int p = 0; p < tz; ++p) {
      const long long m = ((long long)(b * g.n1 + z + p) * g.n2 + y0 + (r >> 3)) * g.n3 + x0 + (r & 7);
      for (int c0 = 0; c0 < Cout; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(p * Cout + c0), v);
        conv_epilogue16(v, m, c0, Cout, bias, skip, y, yf, accum, relu);
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}


// f(std::integral_constant<int, C>) with C = Cin for the channel counts that have their own instantiation, else 0
template <class F> void with_cin(int Cin, F&& f) {
  switch (Cin) {
    case 16: f(std::integral_constant<int, 16>()); break;
    case 32: f(std::integral_constant<int, 32>()); break;
    case 64: f(std::integral_constant<int, 64>()); break;
    case 128: f(std::integral_constant<int, 128>()); break;
    default: f(std::integral_constant<int, 0>()); break;
  }
}
template <int C> cudaError_t conv_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_conv3_fwd_tc<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fwd_smem(kMaxC, kMaxC));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_conv3_wgrad_tc<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)wgrad_smem(kMaxC));
  return e;
}
cudaError_t conv_attrs_once() {
  static std::once_flag once;
  static cudaError_t e = cudaSuccess;
  std::call_once(once, [] {
    for (cudaError_t r : {conv_attrs<0>(), conv_attrs<16>(), conv_attrs<32>(), conv_attrs<64>(), conv_attrs<128>()})
      if (r != cudaSuccess) e = r;
  });
  return e;
}

}  // namespace

size_t fwd_work_elems(const Geo& g, int Cout) {
  const int per = fwd_offsets_per_split(g);
  const int nsplit = (27 + per - 1) / per;
  return nsplit > 1 ? size_t(nsplit) * size_t(g.M) * size_t(Cout) : 0;
}

cudaError_t conv3_fwd(const bf16* x, const bf16* w, const float* bias, const bf16* skip, bf16* y, float* yf,
                      int accum, const Geo& g, int Cin, int Cout, int relu, float* work, cudaStream_t st) {
  const cudaError_t attr = conv_attrs_once();
  if (attr != cudaSuccess) return attr;
  const unsigned tiles = (unsigned)((g.M + kTileM - 1) / kTileM);
  const int per = work ? fwd_offsets_per_split(g) : 27;
  const int nsplit = (27 + per - 1) / per;
  const char* conv_env = std::getenv("CLAIRE_CONV");
  if (halo_fits(g, Cin, Cout) && !(conv_env && std::strcmp(conv_env, "gather") == 0)) {
    // the same MMAs from a shared-memory halo (k_conv3_fwd_halo): no per-offset gather, and no offset split even
    // on grids with few voxel tiles (a halo tile's 27 offsets cost one staging; the choice depends on the
    // per-sample grid and the channels only, so a sample's output does not depend on its batch)
    static std::once_flag once;
    static cudaError_t hattr = cudaSuccess;
    std::call_once(once, [] {
      for (const void* fn : {(const void*)k_conv3_fwd_halo<0>, (const void*)k_conv3_fwd_halo<16>,
                             (const void*)k_conv3_fwd_halo<32>, (const void*)k_conv3_fwd_halo<64>})
        if (hattr == cudaSuccess)
          hattr = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    if (hattr != cudaSuccess) return hattr;
    const int tz = halo_tz(g, Cin, Cout);
    const unsigned htiles = (unsigned)((g.n3 / 8) * (g.n2 / 16) * (g.n1 / tz) * g.B);
    auto go = [&](auto cc) {
      k_conv3_fwd_halo<decltype(cc)::value><<<htiles, kTileM, halo_smem(Cin, Cout, tz), st>>>(
          x, w, bias, skip, y, yf, accum, g, Cin, Cout, relu, tz);
    };
    switch (Cin) {
      case 16: go(std::integral_constant<int, 16>()); break;
      case 32: go(std::integral_constant<int, 32>()); break;
      case 64: go(std::integral_constant<int, 64>()); break;
      default: go(std::integral_constant<int, 0>()); break;
    }
    return cudaGetLastError();
  }
  if (nsplit == 1) {
    with_cin(Cin, [&](auto cc) {
      k_conv3_fwd_tc<decltype(cc)::value><<<dim3(tiles, 1u), kTileM, fwd_smem(Cin, Cout), st>>>(
          x, w, bias, skip, y, yf, accum, g, Cin, Cout, relu, 27, fwd_group(Cin), nullptr);
    });
    return cudaGetLastError();
  }
  with_cin(Cin, [&](auto cc) {
    k_conv3_fwd_tc<decltype(cc)::value><<<dim3(tiles, (unsigned)nsplit), kTileM, fwd_smem(Cin, Cout), st>>>(
        x, w, nullptr, nullptr, nullptr, nullptr, 0, g, Cin, Cout, 0, per, fwd_group(Cin), work);
  });
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long count = g.M * Cout;
  k_conv3_reduce<<<nblocks(count), 256, 0, st>>>(work, nsplit, bias, skip, y, yf, accum, count, Cout, relu);
  return cudaGetLastError();
}

size_t wgrad_work_elems(const Geo& g, int Cin, int Cout) {
  const long long chunk = wgrad_chunk(g, Cin);
  const long long nchunks = (g.M + chunk - 1) / chunk;
  return size_t(nchunks) * size_t(Cout) * 27 * size_t(Cin);
}

cudaError_t conv3_wgrad(const bf16* dz, const bf16* x, float* dw, float* work, const Geo& g, int Cin, int Cout,
                        cudaStream_t st, const float* bias_part, float* db) {
  const cudaError_t attr = conv_attrs_once();
  if (attr != cudaSuccess) return attr;
  const int group = wgrad_group(Cin);
  const int chunk = wgrad_chunk(g, Cin);
  const int nchunks = (int)((g.M + chunk - 1) / chunk);
  const unsigned ngroups = (unsigned)((27 + group - 1) / group);
  with_cin(Cin, [&](auto cc) {
    k_conv3_wgrad_tc<decltype(cc)::value><<<dim3(ngroups, (unsigned)nchunks), kTileM, wgrad_smem(Cout), st>>>(
        dz, x, work, g, Cin, Cout, group, chunk);
  });
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const SumJob jw = sum_job(work, nchunks, 27LL * Cin * Cout, dw);
  if (!bias_part) return sum_chunks(jw, nullptr, st);
  const SumJob jb = sum_job(bias_part, kBiasBlocks, Cout, db);
  return sum_chunks(jw, &jb, st);
}

cudaError_t status(cudaStream_t st) {
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  int flag = 0, zero = 0;
  e = cudaMemcpyFromSymbol(&flag, g_nn_error, sizeof(int));
  if (e != cudaSuccess) return e;
  if (flag) {
    cudaMemcpyToSymbol(g_nn_error, &zero, sizeof(int));
    return cudaErrorLaunchTimeout;
  }
  // host-side fake of an expired wait (CLAIRE_FAULT=nn_timeout), for tests of the status path
  if (fault_injected("nn_timeout")) return cudaErrorLaunchTimeout;
  return cudaSuccess;
}

cudaError_t weight_flip_all(const bf16* w, bf16* wt, const FlipTable& tab, cudaStream_t st) {
  if (tab.n < 1 || tab.n > FlipTable::kMax) return cudaErrorInvalidValue;
  for (int t = 0; t < tab.n; ++t)
    if (tab.cin[t] < 1 || tab.cout[t] < 1 || tab.cin[t] > kMaxC || tab.cout[t] > kMaxC) return cudaErrorInvalidValue;
  k_wt_flip_all<<<27 * tab.n, 256, 0, st>>>(w, wt, tab);
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

cudaError_t relu_bwd_bias(const float* dy, const bf16* y, float* dz, bf16* dzb, long long M, int C, float* db,
                          float* work, cudaStream_t st) {
  launch_relu_bwd_bias(dy, y, dz, dzb, M, C, work, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !db) return e;
  return sum_chunks(sum_job(work, kBiasBlocks, C, db), nullptr, st);
}

cudaError_t bias_grad(const float* dz, long long M, int C, float* db, float* work, cudaStream_t st) {
  launch_relu_bwd_bias(dz, nullptr, nullptr, nullptr, M, C, work, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return sum_chunks(sum_job(work, kBiasBlocks, C, db), nullptr, st);
}

cudaError_t pool_fwd(const bf16* x, bf16* y, const Geo& gf, int C, cudaStream_t st) {
  const Geo gc = mkgeo(gf.B, gf.n1 / 2, gf.n2 / 2, gf.n3 / 2);
  if (C % 8 == 0 && aligned_to(16, {x, y}))
    k_pool_fwd<8><<<nblocks(gc.M * C / 8), 256, 0, st>>>(x, y, gc, C, FastDiv((unsigned)(C / 8)));
  else
    k_pool_fwd<1><<<nblocks(gc.M * C), 256, 0, st>>>(x, y, gc, C, FastDiv((unsigned)C));
  return cudaGetLastError();
}
cudaError_t pool_bwd(const float* dy, float* dx, int accum, const Geo& gf, int C, cudaStream_t st) {
  const Geo gc = mkgeo(gf.B, gf.n1 / 2, gf.n2 / 2, gf.n3 / 2);
  if (C % 4 == 0 && aligned_to(16, {dy, dx}))
    k_pool_bwd<4><<<nblocks(gc.M * C / 4), 256, 0, st>>>(dy, dx, accum, gc, C, FastDiv((unsigned)(C / 4)));
  else
    k_pool_bwd<1><<<nblocks(gc.M * C), 256, 0, st>>>(dy, dx, accum, gc, C, FastDiv((unsigned)C));
  return cudaGetLastError();
}
cudaError_t up_fwd(const bf16* x, bf16* y, const Geo& gc, int C, cudaStream_t st) {
  if (C % 8 == 0 && aligned_to(16, {x, y}))
    k_up_fwd<8><<<nblocks(gc.M * C / 8), 256, 0, st>>>(x, y, gc, C, FastDiv((unsigned)(C / 8)));
  else
    k_up_fwd<1><<<nblocks(gc.M * C), 256, 0, st>>>(x, y, gc, C, FastDiv((unsigned)C));
  return cudaGetLastError();
}
cudaError_t up_bwd(const float* dy, float* dx, int accum, const Geo& gc, int C, cudaStream_t st) {
  if (C % 4 == 0 && aligned_to(16, {dy, dx}))
    k_up_bwd<4><<<nblocks(gc.M * C / 4), 256, 0, st>>>(dy, dx, accum, gc, C, FastDiv((unsigned)(C / 4)));
  else
    k_up_bwd<1><<<nblocks(gc.M * C), 256, 0, st>>>(dy, dx, accum, gc, C, FastDiv((unsigned)C));
  return cudaGetLastError();
}

cudaError_t mse(const float* pred, const float* target, float* grad, long long M, int C, int cu, double* partials,
                int nb, cudaStream_t st) {
  const int vec = C % 4 == 0 && cu <= 4 && aligned_to(16, {grad});
  k_mse<<<nb, 256, 0, st>>>(pred, target, grad, M, C, cu, 1.0 / double(M * cu), partials, vec);
  return cudaGetLastError();
}

cudaError_t adam(float* p, const float* g, float* m1, float* m2, bf16* pb, long long count, float lr, float b1,
                 float b2, float eps, int t, cudaStream_t st) {
  const float c1 = float(1.0 / (1.0 - std::pow(double(b1), t)));
  const float c2 = float(1.0 / (1.0 - std::pow(double(b2), t)));
  const uintptr_t al = reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(g) |
                       reinterpret_cast<uintptr_t>(m1) | reinterpret_cast<uintptr_t>(m2);
  const int vec = count % 4 == 0 && (al & 15) == 0 && (reinterpret_cast<uintptr_t>(pb) & 7) == 0;
  k_adam<<<nblocks(vec ? count / 4 : count), 256, 0, st>>>(p, g, m1, m2, pb, count, lr, b1, b2, eps, c1, c2, vec);
  return cudaGetLastError();
}

cudaError_t pack_images(const float* images, const SampleIdx& idx, int nb, bf16* dst, long long N0, int C,
                        float sdiff, cudaStream_t st) {
  if (nb < 1 || nb > SampleIdx::kMax) return cudaErrorInvalidValue;
  k_pack_images<<<nblocks(nb * N0), 256, 0, st>>>(images, idx, nb, dst, N0, C, sdiff);
  return cudaGetLastError();
}
cudaError_t interleave_batch(const float* targets, const SampleIdx& idx, int nb, float* dst, long long N0, int ncomp,
                             float s, cudaStream_t st) {
  if (nb < 1 || nb > SampleIdx::kMax) return cudaErrorInvalidValue;
  k_interleave_batch<<<nblocks(nb * N0), 256, 0, st>>>(targets, idx, nb, dst, N0, ncomp, s);
  return cudaGetLastError();
}
cudaError_t unpack(const float* src, float* dst, long long M, int ncomp, int C, float s, cudaStream_t st) {
  k_unpack<<<nblocks(M * ncomp), 256, 0, st>>>(src, dst, M, ncomp, C, s);
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
// an expired bounded tensor-core wait (reported by nn::status as cudaErrorLaunchTimeout) is CLAIRE_ETIMEOUT
inline claire_status st_of(cudaError_t e) {
  return e == cudaSuccess ? CLAIRE_OK : (e == cudaErrorLaunchTimeout ? CLAIRE_ETIMEOUT : CLAIRE_ECUDA);
}
inline bool geo_args(int B, int n1, int n2, int n3) { return B > 0 && n1 > 0 && n2 > 0 && n3 > 0; }
inline bool pool_args(int B, int n1, int n2, int n3) {
  return geo_args(B, n1, n2, n3) && n1 % 2 == 0 && n2 % 2 == 0 && n3 % 2 == 0;
}
// pooling and upsampling index fine voxels and channels in 32 bits: the fine grid's values below 2^31
inline bool fine_fits(int B, int n1, int n2, int n3, int C, int scale) {
  return C > 0 && (long long)B * n1 * n2 * n3 * scale * C < (1LL << 31);
}
}  // namespace

extern "C" {

claire_status claire_nn_status(void* stream) { return st_of(status((cudaStream_t)stream)); }

size_t claire_nn_fwd_workspace_bytes(int B, int n1, int n2, int n3, int Cout) {
  if (!geo_args(B, n1, n2, n3) || !conv_chan_ok(Cout)) return 0;
  const Geo g = mkgeo(B, n1, n2, n3);
  if (!conv_geo_ok(g)) return 0;
  return fwd_work_elems(g, Cout) * sizeof(float);
}

claire_status claire_nn_conv3_fwd(const void* x, const void* w, const float* bias, const void* skip, void* y,
                                  float* yf, int accum, int B, int n1, int n2, int n3, int Cin, int Cout, int relu,
                                  float* work, void* stream) {
  if (!x || !w || (!y && !yf) || !geo_args(B, n1, n2, n3)) return CLAIRE_EINVAL;
  if (!aligned_to(16, {x, w, skip, y, yf, work}) || !aligned_to(4, {bias})) return CLAIRE_EINVAL;
  const Geo g = mkgeo(B, n1, n2, n3);
  if (!conv_geo_ok(g) || !conv_chan_ok(Cin) || !conv_chan_ok(Cout)) return CLAIRE_EINVAL;
  return st_of(conv3_fwd(static_cast<const bf16*>(x), static_cast<const bf16*>(w), bias,
                         static_cast<const bf16*>(skip), static_cast<bf16*>(y), yf, accum ? 1 : 0, g, Cin, Cout,
                         relu ? 1 : 0, work, (cudaStream_t)stream));
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
  if (!aligned_to(16, {dz, x}) || !aligned_to(4, {dw, work})) return CLAIRE_EINVAL;
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
  if (!x || !y || !pool_args(B, n1, n2, n3) || !fine_fits(B, n1, n2, n3, C, 1)) return CLAIRE_EINVAL;
  return st_of(pool_fwd(static_cast<const bf16*>(x), static_cast<bf16*>(y), mkgeo(B, n1, n2, n3), C,
                        (cudaStream_t)stream));
}
claire_status claire_nn_pool_bwd(const float* dy, float* dx, int accum, int B, int n1, int n2, int n3, int C,
                                 void* stream) {
  if (!dy || !dx || !pool_args(B, n1, n2, n3) || !fine_fits(B, n1, n2, n3, C, 1)) return CLAIRE_EINVAL;
  return st_of(pool_bwd(dy, dx, accum ? 1 : 0, mkgeo(B, n1, n2, n3), C, (cudaStream_t)stream));
}
claire_status claire_nn_up_fwd(const void* x, void* y, int B, int n1, int n2, int n3, int C, void* stream) {
  if (!x || !y || !geo_args(B, n1, n2, n3) || !fine_fits(B, n1, n2, n3, C, 8)) return CLAIRE_EINVAL;
  return st_of(
      up_fwd(static_cast<const bf16*>(x), static_cast<bf16*>(y), mkgeo(B, n1, n2, n3), C, (cudaStream_t)stream));
}
claire_status claire_nn_up_bwd(const float* dy, float* dx, int accum, int B, int n1, int n2, int n3, int C,
                               void* stream) {
  if (!dy || !dx || !geo_args(B, n1, n2, n3) || !fine_fits(B, n1, n2, n3, C, 8)) return CLAIRE_EINVAL;
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
