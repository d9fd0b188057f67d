// Semi-Lagrangian device code shared by sl.cu and the per-halo units sl_h<H>.cu (internal).
#pragma once

#include <cuda_bf16.h>

#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

#include "impl.cuh"

namespace claire {

// Element of a gradient history stored as G (the compute type T, or BF16 for the reduced-storage mode)
template <class T, class G> __device__ __forceinline__ T ldg_as(const G* p) {
  if constexpr (std::is_same<G, __nv_bfloat16>::value) {
    return T(__bfloat162float(p[0]));
  } else {
    return __ldg(p);
  }
}

// Per-axis part of a stencil: the four cubic Lagrange weights and the unwrapped first stencil node b - 1.
template <class T> __device__ __forceinline__ int axis_setup(int i, T disp, T* w) {
  const T fd = floor(disp);
  const T t = disp - fd;
  const T tp1 = t + T(1), tm1 = t - T(1), tm2 = t - T(2);
  w[0] = -(t * tm1 * tm2) * T(1.0 / 6.0);
  w[1] = (tp1 * tm1 * tm2) * T(0.5);
  w[2] = -(tp1 * t * tm2) * T(0.5);
  w[3] = (tp1 * t * tm1) * T(1.0 / 6.0);
  return i + (int)fd - 1;
}

// periodic index of q: two conditional shifts for q in [-n, 2n), a modulo beyond (displacements over a period)
__device__ __forceinline__ int wrapc(int q, int n) {
  if (q >= -n && q < 2 * n) {
    q = q < 0 ? q + n : q;
    return q >= n ? q - n : q;
  }
  q %= n;
  return q < 0 ? q + n : q;
}

template <class T> struct Stencil {
  T w1[4], w2[4], w3[4];
  int b1, b2, b3;  // unwrapped first stencil node per axis
  bool inside;     // the whole warp's stencils lie inside the box: no periodic wrap needed
};

template <class T>
__device__ __forceinline__ void stencil_at(int i1, int i2, int i3, T d1, T d2, T d3, const Dims& d, Stencil<T>& s) {
  s.b1 = axis_setup<T>(i1, d1, s.w1);
  s.b2 = axis_setup<T>(i2, d2, s.w2);
  s.b3 = axis_setup<T>(i3, d3, s.w3);
  const bool in = (unsigned)s.b1 <= (unsigned)(d.n1 - 4) && (unsigned)s.b2 <= (unsigned)(d.n2 - 4) &&
                  (unsigned)s.b3 <= (unsigned)(d.n3 - 4);
  // one path per warp: a warp with any wrapping lane takes the wrapping path for all its lanes
  s.inside = __all_sync(__activemask(), in);
}

// FP32 rows for even n3 and an 8-byte aligned field (a row then starts on an 8-byte boundary): the taps [b3, b3 + 3]
// of each row come from two aligned float2 loads at b3 - (b3 & 1) and, for odd b3, one scalar load at b3 + 3;
// the row weights are shifted by b3 & 1 and padded with exact zeros. A zero weight adds an exact zero, so each row
// sum makes the same roundings as the four scalar taps (up to the sign of a zero result). Measured on an adjoint-
// step-shaped kernel at 256^3: 2-5% faster than four scalar loads per row; aligned float4 pairs were slower, and so
// were pairs in the three-field departure gather with all planes' loads in flight (PB = 4), which keeps the
// scalar taps. Wrapping stencils keep the scalar path (pairs with wrapped offsets measured no faster).
template <int PB>
__device__ __forceinline__ float gather_pairs(const float* __restrict__ f, const Stencil<float>& s, const Dims& d) {
  const int s2 = d.n3, s1 = d.n2 * d.n3;
  const int sh = s.b3 & 1;
  const float* corner = f + (s.b1 * s1 + s.b2 * s2 + (s.b3 - sh));
  const float W0 = sh ? 0.f : s.w3[0], W1 = sh ? s.w3[0] : s.w3[1], W2 = sh ? s.w3[1] : s.w3[2],
              W3 = sh ? s.w3[2] : s.w3[3], W4 = sh ? s.w3[3] : 0.f;
  float acc = 0.f;
#pragma unroll
  for (int p0 = 0; p0 < 4; p0 += PB) {
    float2 P0[PB][4], P1[PB][4];
    float P2[PB][4];
#pragma unroll
    for (int pp = 0; pp < PB; ++pp)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float* row = corner + ((p0 + pp) * s1 + q * s2);
        P0[pp][q] = __ldg(reinterpret_cast<const float2*>(row));
        P1[pp][q] = __ldg(reinterpret_cast<const float2*>(row) + 1);
        P2[pp][q] = sh ? __ldg(row + 4) : 0.f;
      }
#pragma unroll
    for (int pp = 0; pp < PB; ++pp) {
      float a1 = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float a2 = W0 * P0[pp][q].x;
        a2 = fmaf(W1, P0[pp][q].y, a2);
        a2 = fmaf(W2, P1[pp][q].x, a2);
        a2 = fmaf(W3, P1[pp][q].y, a2);
        a2 = fmaf(W4, P2[pp][q], a2);
        a1 = fmaf(s.w2[q], a2, a1);
      }
      acc = fmaf(s.w1[p0 + pp], a1, acc);
    }
  }
  return acc;
}

// sum_{p,q,r} w1[p] w2[q] w3[r] f[row(p,q) + col(r)], evaluated as 16 four-tap sums along i3, then i2, then i1.
// Both branches use the same order of operations, so the result does not depend on which one runs.
// PB i1 planes (16 taps each) are loaded before their first use: PB = 4 issues all 64 loads at once (measured:
// 10% faster for the three-field departure-point gather, but slower for the gathers of kernels with more live
// state, which keep PB = 1).
template <class T, int PB = 1>
__device__ __forceinline__ T gather(const T* __restrict__ f, const Stencil<T>& s, const Dims& d) {
  static_assert(PB == 1 || PB == 2 || PB == 4, "planes per batch");
  const int s2 = d.n3, s1 = d.n2 * d.n3;
  T acc = T(0);
  if constexpr (std::is_same<T, float>::value && PB == 1) {
    // (a caller's field may start at any 4-byte boundary: the pair loads need an 8-byte aligned f)
    if (s.inside && (d.n3 & 1) == 0 && (reinterpret_cast<uintptr_t>(f) & 7) == 0) return gather_pairs<PB>(f, s, d);
  }
  if (s.inside) {
    const T* corner = f + (s.b1 * s1 + s.b2 * s2 + s.b3);
#pragma unroll
    for (int p0 = 0; p0 < 4; p0 += PB) {
      T val[PB][16];
#pragma unroll
      for (int pp = 0; pp < PB; ++pp)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const T* row = corner + ((p0 + pp) * s1 + q * s2);
#pragma unroll
          for (int r = 0; r < 4; ++r) val[pp][4 * q + r] = __ldg(row + r);
        }
#pragma unroll
      for (int pp = 0; pp < PB; ++pp) {
        T a1 = T(0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          T a2 = s.w3[0] * val[pp][4 * q];
          a2 = fma(s.w3[1], val[pp][4 * q + 1], a2);
          a2 = fma(s.w3[2], val[pp][4 * q + 2], a2);
          a2 = fma(s.w3[3], val[pp][4 * q + 3], a2);
          a1 = fma(s.w2[q], a2, a1);
        }
        acc = fma(s.w1[p0 + pp], a1, acc);
      }
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

// ---------------------------------------------------------------------------------------------------------------
// Shared-memory bricks. A CTA of 16 x 16 threads handles a tile of 16 (i3) x 16 (i2) x 4 (i1) nodes. With every
// displacement bounded by D voxels (measured after the departure points are computed), all stencils of the tile
// lie in the brick of nodes [tile - H, tile + H] per axis, H = ceil(D) + 1 below and one more above (along i3 widened
// to 16-byte boundaries). The brick is loaded once with coalesced periodic-wrapped reads (whole 16-byte copies away
// from the box's faces); each of the 64 taps then is a shared-memory read instead of
// L1 lines. A warp holds 16 (i3) x 2 (i2) nodes, and the brick's row pitch px is 16 modulo 32 words (as is its
// plane pitch), so the two half-warps -- and lanes whose stencils sit one row or plane apart -- read disjoint
// bank ranges: with 32 nodes along one row, stencil spans over 32 words made two-way bank conflicts (measured:
// 56% extra wavefronts). A stencil outside the brick (never, when D is exact) falls back to the global gather.
constexpr int kTX = 16, kTY = 16, kTZ = 4;

template <int H> struct TileGeom {
  // along i3 the brick starts xa nodes left of the tile, on a 16-byte boundary, and its width ex (a multiple of 4)
  // covers [x0 - H, x0 + kTX + H]: rows load as whole 16-byte copies
  static constexpr int xa = (H + 3) / 4 * 4;
  static constexpr int ex = kTX + xa + (H + 4) / 4 * 4, ey = kTY + 2 * H + 1, ez = kTZ + 2 * H + 1;
  static constexpr int px = ex + (16 - ex % 32 + 32) % 32;  // row pitch: >= ex, 16 mod 32
  static constexpr int vol = px * ey * ez;
  static_assert(px % 32 == 16 && (px * ey) % 32 == 16, "row and plane pitch 16 mod 32 words");
};

struct Tile {
  int x0, y0, z0;
  bool interior;  // the whole brick lies inside the box (no periodic wrap while loading)
};

template <int H> __device__ __forceinline__ Tile tile_of(const Dims& d) {
  using G = TileGeom<H>;
  Tile t;
  t.x0 = blockIdx.x * kTX;
  t.y0 = blockIdx.y * kTY;
  t.z0 = blockIdx.z * kTZ;
  t.interior = t.x0 - G::xa >= 0 && t.x0 - G::xa + G::ex <= d.n3 && t.y0 - H >= 0 && t.y0 - H + G::ey <= d.n2 &&
               t.z0 - H >= 0 && t.z0 - H + G::ez <= d.n1;
  return t;
}

// asynchronous 4- or 8-byte global -> shared copy (no register staging; completion via wait_all below)
template <class T> __device__ __forceinline__ void cp_async_elem(T* sdst, const T* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_16(void* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// cooperative load of f0 (and f1 when not null) into the bricks sm[0..vol) and sm[vol..2 vol); every copy is
// issued before any is waited for, so the brick fill is bandwidth- rather than latency-bound
template <class T, int H>
__device__ __forceinline__ void load_bricks(T* sm, const T* __restrict__ f0, const T* __restrict__ f1, const Tile& tl,
                                            const Dims& d) {
  using G = TileGeom<H>;
  constexpr int rows = G::ey * G::ez;
  const T* g0 = f0 + ((tl.z0 - H) * d.n2 + (tl.y0 - H)) * d.n3 + (tl.x0 - G::xa);
  const T* g1 = f1 ? f1 + ((tl.z0 - H) * d.n2 + (tl.y0 - H)) * d.n3 + (tl.x0 - G::xa) : nullptr;
  // 16-byte copies: FP32, rows of a multiple of 4 words, fields on 16-byte boundaries
  const bool vec = sizeof(T) == 4 && (d.n3 & 3) == 0 && ((reinterpret_cast<uintptr_t>(f0) | reinterpret_cast<uintptr_t>(f1)) & 15) == 0;
  // the brick's rows lie inside the box along i3 (only their i1, i2 indices may wrap)
  const bool x_in = tl.x0 - G::xa >= 0 && tl.x0 - G::xa + G::ex <= d.n3;
  if (tl.interior && vec) {
    constexpr int nv = G::ex * (int)sizeof(T) / 16;  // 16-byte vectors per row
    const int tid = threadIdx.y * kTX + threadIdx.x;
    for (int q = tid; q < rows * nv; q += kTX * kTY) {
      const int row = q / nv, v = q - row * nv;
      const int z = row / G::ey, y = row - z * G::ey;
      const int goff = z * d.n2 * d.n3 + y * d.n3 + 4 * v;
      cp_async_16(sm + row * G::px + 4 * v, g0 + goff);
      if (f1) cp_async_16(sm + G::vol + row * G::px + 4 * v, g1 + goff);
    }
  } else if (x_in && vec) {
    // a tile on an i1 or i2 face: whole 16-byte copies of rows whose row index wraps
    constexpr int nv = G::ex * (int)sizeof(T) / 16;
    const int tid = threadIdx.y * kTX + threadIdx.x;
    for (int q = tid; q < rows * nv; q += kTX * kTY) {
      const int row = q / nv, v = q - row * nv;
      const int z = row / G::ey, y = row - z * G::ey;
      const int gz = wrapc(tl.z0 - H + z, d.n1), gy = wrapc(tl.y0 - H + y, d.n2);
      const int goff = (gz * d.n2 + gy) * d.n3 + (tl.x0 - G::xa) + 4 * v;
      cp_async_16(sm + row * G::px + 4 * v, f0 + goff);
      if (f1) cp_async_16(sm + G::vol + row * G::px + 4 * v, f1 + goff);
    }
  } else if (tl.interior) {
#pragma unroll 2
    for (int row = threadIdx.y; row < rows; row += kTY) {
      const int z = row / G::ey, y = row - z * G::ey;
      const int goff = z * d.n2 * d.n3 + y * d.n3;
#pragma unroll
      for (int x = threadIdx.x; x < G::ex; x += kTX) {
        cp_async_elem<T>(sm + row * G::px + x, g0 + goff + x);
        if (f1) cp_async_elem<T>(sm + G::vol + row * G::px + x, g1 + goff + x);
      }
    }
  } else {
    for (int row = threadIdx.y; row < rows; row += kTY) {
      const int z = row / G::ey, y = row - z * G::ey;
      const int gz = wrapc(tl.z0 - H + z, d.n1), gy = wrapc(tl.y0 - H + y, d.n2);
      const int base = (gz * d.n2 + gy) * d.n3;
      for (int x = threadIdx.x; x < G::ex; x += kTX) {
        const int gx = wrapc(tl.x0 - G::xa + x, d.n3);
        cp_async_elem<T>(sm + row * G::px + x, f0 + base + gx);
        if (f1) cp_async_elem<T>(sm + G::vol + row * G::px + x, f1 + base + gx);
      }
    }
  }
  cp_async_wait_all();
}

template <class T, int H>
__device__ __forceinline__ bool in_brick(const Stencil<T>& s, const Tile& tl, int& lz, int& ly, int& lx) {
  using G = TileGeom<H>;
  lz = s.b1 - (tl.z0 - H);
  ly = s.b2 - (tl.y0 - H);
  lx = s.b3 - (tl.x0 - G::xa);
  return (unsigned)lz <= (unsigned)(G::ez - 4) && (unsigned)ly <= (unsigned)(G::ey - 4) &&
         (unsigned)lx <= (unsigned)(G::ex - 4);
}

// same tap order and arithmetic as gather()
template <class T, int H>
__device__ __forceinline__ T gather_brick(const T* sb, int lz, int ly, int lx, const Stencil<T>& s) {
  using G = TileGeom<H>;
  const T* corner = sb + (lz * G::ey + ly) * G::px + lx;
  T acc = T(0);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    T a1 = T(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T* row = corner + (p * G::ey * G::px + q * G::px);
      T a2 = s.w3[0] * row[0];
      a2 = fma(s.w3[1], row[1], a2);
      a2 = fma(s.w3[2], row[2], a2);
      a2 = fma(s.w3[3], row[3], a2);
      a1 = fma(s.w2[q], a2, a1);
    }
    acc = fma(s.w1[p], a1, acc);
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
  const T w1 = gather<T, 4>(v, s, d), w2 = gather<T, 4>(v + N, s, d), w3 = gather<T, 4>(v + 2 * N, s, d);
  const T h = T(0.5) * sdt;
  disp[idx] = -h * (v1 + w1) * ih1;
  disp[N + idx] = -h * (v2 + w2) * ih2;
  disp[2 * N + idx] = -h * (v3 + w3) * ih3;
}

// node loop shared by the global (H < 0) and the brick-tiled (H >= 0) launch shapes: body(i1, i2, i3, idx)
template <int H, class Body>
__device__ __forceinline__ void for_nodes(const Dims& d, const Tile& tl, Body&& body) {
  if constexpr (H >= 0) {
#pragma unroll 1
    for (int tz = 0; tz < kTZ; ++tz) {
      const int i1 = tl.z0 + tz, i2 = tl.y0 + threadIdx.y, i3 = tl.x0 + threadIdx.x;
      if (i1 < d.n1 && i2 < d.n2 && i3 < d.n3) body(i1, i2, i3, (i1 * d.n2 + i2) * d.n3 + i3);
    }
  } else {
    const Node x = node3d(d);
    if (x.valid) body(x.i1, x.i2, x.i3, x.idx);
  }
}

// value of f (brick slot k when tiled) at the stencil s
template <class T, int H>
__device__ __forceinline__ T sample(const T* __restrict__ f, const T* sm, int k, const Tile& tl, const Stencil<T>& s,
                                    const Dims& d) {
  if constexpr (H >= 0) {
    int lz, ly, lx;
    if (in_brick<T, H>(s, tl, lz, ly, lx)) return gather_brick<T, H>(sm + k * TileGeom<H>::vol, lz, ly, lx, s);
  }
  return gather<T>(f, s, d);
}

template <int H> __device__ __forceinline__ Tile tile_or_empty(const Dims& d) {
  if constexpr (H >= 0) {
    return tile_of<H>(d);
  } else {
    return Tile{0, 0, 0, false};
  }
}

// Launch bounds of the gather kernels: 8 resident CTAs (32 registers) for the FP32 one-field global gathers --
// measured 4-10% faster at 256^3 than the compiler's own 40-48 registers, since their long-scoreboard stalls want
// more warps; 4 CTAs (64 registers) for FP64 and for the variants with more live state (RHO, last step), which
// spill at 32. The brick-tiled gathers are bound by the L1 data pipe, not by latency: 5 CTAs (48 registers), since
// spills cost L1 wavefronts (measured at 32 registers: 15% of them; 40 registers still spill).
template <class T, int H, bool HEAVY> constexpr int gather_min_ctas() {
  return sizeof(T) != 4 || HEAVY ? 4 : (H >= 0 ? 5 : 8);
}
template <class T, int H>
__global__ void __launch_bounds__(256, gather_min_ctas<T, H, false>())
    k_interp(const T* __restrict__ f, const T* __restrict__ disp, T* __restrict__ out, Dims d) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  const Tile tl = tile_or_empty<H>(d);
  if constexpr (H >= 0) {
    load_bricks<T, H>(sm, f, (const T*)nullptr, tl, d);
    __syncthreads();
  }
  const long long N = d.N;
  for_nodes<H>(d, tl, [&](int i1, int i2, int i3, int idx) {
    Stencil<T> s;
    stencil_at<T>(i1, i2, i3, disp[idx], disp[N + idx], disp[2 * N + idx], d, s);
    out[idx] = sample<T, H>(f, sm, 0, tl, s, d);
  });
}

// lam = mR - m1 (Eq. (4) final condition), rl = rho lam, b = w lam grad m^{nt}
template <class T, bool RHO, class G>
__global__ void __launch_bounds__(256) k_adj_terminal(const T* __restrict__ mR, const T* __restrict__ m1,
                                                      const T* __restrict__ rho, T* __restrict__ lam,
                                                      T* __restrict__ rl, T* __restrict__ b,
                                                      const G* __restrict__ gm, T w, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.N) return;
  const long long N = d.N;
  const T l = mR[idx] - m1[idx];
  lam[idx] = l;
  if (RHO) rl[idx] = rho[idx] * l;
  const T wl = w * l;
  b[idx] = wl * ldg_as<T, G>(gm + idx);
  b[N + idx] = wl * ldg_as<T, G>(gm + N + idx);
  b[2 * N + idx] = wl * ldg_as<T, G>(gm + 2 * N + idx);
}

// One backward step of -d_t lam - div(lam v) = 0 along Y (Eq. (4), (9)):
//   a = lam^{j+1}(Y); with the div source: c = (rho lam^{j+1})(Y), lam^j = a + dt/2 (c + rho(x)(a + dt c)).
// Epilogue: optional store of lam^j and rho lam^j, and b += w_j lam^j grad m^j.
template <class T, bool RHO, bool STORE, bool ACC, bool DOT, int H, class G>
__global__ void __launch_bounds__(256, gather_min_ctas<T, H, RHO>())
    k_adj_step(const T* __restrict__ lam_next, const T* __restrict__ rl_next,
                                                  const T* __restrict__ rho, const T* __restrict__ dY,
                                                  T* __restrict__ lam, T* __restrict__ rl, T* __restrict__ b,
                                                  const G* __restrict__ gm, T w, T dt, Dims d,
                                                  const T* __restrict__ sv, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  const Tile tl = tile_or_empty<H>(d);
  if constexpr (H >= 0) {
    load_bricks<T, H>(sm, lam_next, RHO ? rl_next : (const T*)nullptr, tl, d);
    __syncthreads();
  }
  double contrib = 0.0;  // this thread's <s, b> terms: three products per node in T, the sum over nodes in FP64
  const long long N = d.N;
  for_nodes<H>(d, tl, [&](int i1, int i2, int i3, int idx) {
    Stencil<T> s;
    stencil_at<T>(i1, i2, i3, dY[idx], dY[N + idx], dY[2 * N + idx], d, s);
    T l = sample<T, H>(lam_next, sm, 0, tl, s, d);
    T r = T(0);
    if (RHO) {
      const T cc = sample<T, H>(rl_next, sm, 1, tl, s, d);
      r = rho[idx];
      l = l + T(0.5) * dt * (cc + r * (l + dt * cc));
    }
    if (STORE) {
      lam[idx] = l;
      if (RHO) rl[idx] = r * l;
    }
    if (ACC) {
      const T wl = w * l;
      const T b0 = fma(wl, ldg_as<T, G>(gm + idx), b[idx]);
      const T b1 = fma(wl, ldg_as<T, G>(gm + N + idx), b[N + idx]);
      const T b2 = fma(wl, ldg_as<T, G>(gm + 2 * N + idx), b[2 * N + idx]);
      b[idx] = b0;
      b[N + idx] = b1;
      b[2 * N + idx] = b2;
      // <s, b>: the final time integral against a vector s, for PCG's <s, H s> (Alg. 2)
      if (DOT) contrib += double(fma(sv[2 * N + idx], b2, fma(sv[N + idx], b1, sv[idx] * b0)));
    }
  });
  if (DOT) {
    __shared__ double red[32];
    double cs = contrib;
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
template <class T, class G>
__global__ void __launch_bounds__(256) k_inc_init(const T* __restrict__ vt, const G* __restrict__ gm,
                                                  T* __restrict__ q, T hdt, Dims d) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.N) return;
  const long long N = d.N;
  const T f = -(vt[idx] * ldg_as<T, G>(gm + idx) + vt[N + idx] * ldg_as<T, G>(gm + N + idx) +
                vt[2 * N + idx] * ldg_as<T, G>(gm + 2 * N + idx));
  q[idx] = hdt * f;
}

// m~^{j+1}(x) = q^j(X) + dt/2 f^{j+1}(x); not last: q^{j+1} = m~^{j+1} + dt/2 f^{j+1}.
// last: lam~ = -m~(1) (Eq. (9) final condition), rl = rho lam~, b = w lam~ grad m^{nt}.
template <class T, bool LAST, bool RHO, int H, class G>
__global__ void __launch_bounds__(256, gather_min_ctas<T, H, LAST>())
    k_inc_step(const T* __restrict__ q, const T* __restrict__ dX,
                                                  const T* __restrict__ vt, const G* __restrict__ gm,
                                                  T* __restrict__ qout, const T* __restrict__ rho,
                                                  T* __restrict__ rl, T* __restrict__ b, T hdt, T w, Dims d) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  const Tile tl = tile_or_empty<H>(d);
  if constexpr (H >= 0) {
    load_bricks<T, H>(sm, q, (const T*)nullptr, tl, d);
    __syncthreads();
  }
  const long long N = d.N;
  for_nodes<H>(d, tl, [&](int i1, int i2, int i3, int idx) {
    Stencil<T> s;
    stencil_at<T>(i1, i2, i3, dX[idx], dX[N + idx], dX[2 * N + idx], d, s);
    const T g1 = ldg_as<T, G>(gm + idx), g2 = ldg_as<T, G>(gm + N + idx), g3 = ldg_as<T, G>(gm + 2 * N + idx);
    const T f = -(vt[idx] * g1 + vt[N + idx] * g2 + vt[2 * N + idx] * g3);
    const T mt = sample<T, H>(q, sm, 0, tl, s, d) + hdt * f;
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
  });
}

// y = a .* x
template <class T>
__global__ void __launch_bounds__(256) k_hadamard(const T* __restrict__ a, const T* __restrict__ x,
                                                  T* __restrict__ y, long long n) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n) y[idx] = a[idx] * x[idx];
}

// ---------------------------------------------------------------------------------------------------------------
// Launch shape: brick-tiled for FP32 with a supported halo (2 <= H <= kMaxHalo), else the plain global gather.
constexpr int kMaxHalo = 5;
template <class T> static int tile_halo(int H) {
  return (sizeof(T) == 4 && H >= 0 && H <= kMaxHalo) ? (H < 2 ? 2 : H) : -1;
}
template <int H> static void tiled_shape(const Dims& d, dim3& grid, dim3& block) {
  if constexpr (H >= 0) {
    block = dim3(kTX, kTY, 1);
    grid = dim3((d.n3 + kTX - 1) / kTX, (d.n2 + kTY - 1) / kTY, (d.n1 + kTZ - 1) / kTZ);
  } else {
    const Launch3 L = launch3(d);
    block = L.block;
    grid = L.grid;
  }
}
template <class T, int H> static size_t tiled_smem(int nf) {
  if constexpr (H >= 0) {
    return size_t(TileGeom<H>::vol) * nf * sizeof(T);
  } else {
    return 0;
  }
}


// The dynamic shared-memory limit of a kernel, raised where the kernel is launched (once per kernel): the tiled
// launchers live in several translation units, and each sets the attribute on the instance it launches.
inline cudaError_t smem_limit_once(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::vector<std::pair<const void*, size_t>> done;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& e : done)
    if (e.first == fn && e.second >= bytes) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done.emplace_back(fn, bytes);
  return e;
}

// ---------------------------------------------------------------------------------------------------------------
// Host-side launchers, one instantiation per (precision, halo). The tiled FP32 ones (halo 2..kMaxHalo) are compiled
// in sl_h<H>.cu so that the build compiles them in parallel; sl.cu instantiates the plain (-1) ones.
template <class T, int HC>
void sl_launch_interp(const T* f, const T* disp, T* out, const Dims& d, cudaStream_t st) {
  dim3 grid, block;
  tiled_shape<HC>(d, grid, block);
  smem_limit_once((const void*)k_interp<T, HC>, tiled_smem<T, HC>(1));
  k_interp<T, HC><<<grid, block, tiled_smem<T, HC>(1), st>>>(f, disp, out, d);
}

// variant: 0 inner step, 1 last step, 2 last step with the div source
template <class T, int HC, class G>
void sl_launch_inc(int variant, const T* q, const T* dX, const T* vt, const G* gm, T* qout, const T* rho, T* rl, T* b,
                   T hdt, T w, const Dims& d, cudaStream_t st) {
  dim3 grid, block;
  tiled_shape<HC>(d, grid, block);
  const size_t sm = tiled_smem<T, HC>(1);
  if (variant == 0) {
    smem_limit_once((const void*)k_inc_step<T, false, false, HC, G>, sm);
    k_inc_step<T, false, false, HC, G><<<grid, block, sm, st>>>(q, dX, vt, gm, qout, rho, rl, b, hdt, w, d);
  } else if (variant == 2) {
    smem_limit_once((const void*)k_inc_step<T, true, true, HC, G>, sm);
    k_inc_step<T, true, true, HC, G><<<grid, block, sm, st>>>(q, dX, vt, gm, qout, rho, rl, b, hdt, w, d);
  } else {
    smem_limit_once((const void*)k_inc_step<T, true, false, HC, G>, sm);
    k_inc_step<T, true, false, HC, G><<<grid, block, sm, st>>>(q, dX, vt, gm, qout, rho, rl, b, hdt, w, d);
  }
}

// accumulating adjoint steps (rho: div source; store: keep lambda; dot: fused <sv, b>); returns the block count
template <class T, int HC, class G>
long long sl_launch_adj(bool rho_on, bool store, bool dot, const T* lam_next, const T* rl_next, const T* rho,
                        const T* dY, T* lam, T* rl, T* b, const G* gm, T w, T dt, const Dims& d, const T* sv,
                        double* part, cudaStream_t st) {
  dim3 grid, block;
  tiled_shape<HC>(d, grid, block);
  const size_t sm = tiled_smem<T, HC>(rho_on ? 2 : 1);
#define ADJ(R, S, D)                                                                                           \
  do {                                                                                                         \
    smem_limit_once((const void*)k_adj_step<T, R, S, true, D, HC, G>, sm);                                     \
    k_adj_step<T, R, S, true, D, HC, G><<<grid, block, sm, st>>>(lam_next, rl_next, rho, dY, lam, rl, b, gm, w, \
                                                                 dt, d, sv, part);                             \
  } while (0)
  if (dot) {
    if (rho_on)
      ADJ(true, false, true);
    else
      ADJ(false, false, true);
  } else if (rho_on) {
    if (store)
      ADJ(true, true, false);
    else
      ADJ(true, false, false);
  } else {
    if (store)
      ADJ(false, true, false);
    else
      ADJ(false, false, false);
  }
#undef ADJ
  return (long long)grid.x * grid.y * grid.z;
}

// allow the tiled kernels of halo HC the shared memory of two bricks
template <class T, int HC, class G> cudaError_t sl_set_attrs_g() {
  if constexpr (HC >= 0) {
    const int two = (int)tiled_smem<T, HC>(2);
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* fn) {
      cudaError_t r = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, two);
      if (r != cudaSuccess) e = r;
    };
    set((const void*)k_inc_step<T, false, false, HC, G>);
    set((const void*)k_inc_step<T, true, true, HC, G>);
    set((const void*)k_inc_step<T, true, false, HC, G>);
    set((const void*)k_adj_step<T, true, false, true, true, HC, G>);
    set((const void*)k_adj_step<T, false, false, true, true, HC, G>);
    set((const void*)k_adj_step<T, false, false, true, false, HC, G>);
    set((const void*)k_adj_step<T, false, true, true, false, HC, G>);
    set((const void*)k_adj_step<T, true, false, true, false, HC, G>);
    set((const void*)k_adj_step<T, true, true, true, false, HC, G>);
    return e;
  } else {
    return cudaSuccess;
  }
}

// allow the tiled kernels of halo HC the shared memory of two bricks
template <class T, int HC> cudaError_t sl_set_attrs() {
  if constexpr (HC >= 0) {
    cudaError_t e = cudaFuncSetAttribute((const void*)k_interp<T, HC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tiled_smem<T, HC>(2));
    const cudaError_t e1 = sl_set_attrs_g<T, HC, T>();
    if (e == cudaSuccess) e = e1;
    if constexpr (sizeof(T) == 4) {
      const cudaError_t e2 = sl_set_attrs_g<T, HC, __nv_bfloat16>();
      if (e == cudaSuccess) e = e2;
    }
    return e;
  } else {
    return cudaSuccess;
  }
}

#define CLAIRE_SL_LAUNCHERS_G(EXT, T, HC, G)                                                                      \
  EXT template void sl_launch_inc<T, HC, G>(int, const T*, const T*, const T*, const G*, T*, const T*, T*, T*, T, T, \
                                            const Dims&, cudaStream_t);                                           \
  EXT template long long sl_launch_adj<T, HC, G>(bool, bool, bool, const T*, const T*, const T*, const T*, T*, T*,  \
                                                 T*, const G*, T, T, const Dims&, const T*, double*, cudaStream_t);
#define CLAIRE_SL_LAUNCHERS(EXT, T, HC)                                                                           \
  EXT template void sl_launch_interp<T, HC>(const T*, const T*, T*, const Dims&, cudaStream_t);                   \
  CLAIRE_SL_LAUNCHERS_G(EXT, T, HC, T)                                                                            \
  EXT template cudaError_t sl_set_attrs<T, HC>();

}  // namespace claire
