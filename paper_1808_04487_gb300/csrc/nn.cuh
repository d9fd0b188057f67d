// Layer kernels of the learned warm start (nn.cu) and the shapes they share with the network runtime
// (warmstart.cu). Not part of the paper's method: the network only proposes the initial velocity of Alg. 1.
// The convolutions run on the tcgen05 tensor cores (tc.cuh).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

#include "common.cuh"

namespace claire {
namespace nn {

typedef __nv_bfloat16 bf16;

// A batch of channels-last fields [B][n1][n2][n3][C]; M = B n1 n2 n3 voxels.
struct Geo {
  int B, n1, n2, n3;
  long long M;
  FastDiv by_n3, by_n2, by_n1;  // voxel-index decoding without hardware division
};
inline Geo mkgeo(int B, int n1, int n2, int n3) {
  return Geo{B, n1, n2, n3, (long long)B * n1 * n2 * n3, FastDiv((unsigned)n3), FastDiv((unsigned)n2),
             FastDiv((unsigned)n1)};
}
// shape rules of the tensor-core convolution: whole 16-voxel tiles, 32-bit voxel indices
inline bool conv_geo_ok(const Geo& g) {
  return g.B > 0 && g.n1 > 0 && g.n2 > 0 && g.n3 > 0 && g.M % 16 == 0 && g.M < (1LL << 31);
}
inline bool conv_chan_ok(int C) { return C >= 16 && C <= 128 && C % 16 == 0; }

// y = act(conv3x3x3_periodic(x, w) + bias + skip). x, skip, y BF16 [M][Cin|Cout]; w BF16 [Cout][27][Cin];
// yf (optional) FP32 [M][Cout], overwritten (accum = 0) or added to (accum = 1). relu applies to y and yf.
// work (fwd_work_elems floats, may be null: no split) holds the split-K partial sums of grids with few voxel tiles.
size_t fwd_work_elems(const Geo& g, int Cout);
cudaError_t conv3_fwd(const bf16* x, const bf16* w, const float* bias, const bf16* skip, bf16* y, float* yf,
                      int accum, const Geo& g, int Cin, int Cout, int relu, float* work, cudaStream_t st);
// dw[Cout][27][Cin] = sum_m dz[m][co] x[nb(m, off)][ci] (FP32), computed in fixed-size voxel chunks reduced in a
// fixed order; work holds wgrad_work_elems() floats. With bias_part (the per-block partials that relu_bwd_bias
// leaves when its db is null), db[Cout] = their sum is formed in the same reduction launch.
size_t wgrad_work_elems(const Geo& g, int Cin, int Cout);
cudaError_t conv3_wgrad(const bf16* dz, const bf16* x, float* dw, float* work, const Geo& g, int Cin, int Cout,
                        cudaStream_t st, const float* bias_part = nullptr, float* db = nullptr);
// wt[Cin][27][Cout] with wt[ci][26 - off][co] = w[co][off][ci]: the weights of the adjoint convolution
cudaError_t weight_flip(const bf16* w, bf16* wt, int Cin, int Cout, cudaStream_t st);
// weight_flip for every layer of a table in one launch: layer t's weights lie at w + woff[t] (27 cin cout values,
// cin and cout at most 128) and go to wt + woff[t]
struct FlipTable {
  static constexpr int kMax = 32;
  int n;
  int cin[kMax], cout[kMax];
  long long woff[kMax];
};
cudaError_t weight_flip_all(const bf16* w, bf16* wt, const FlipTable& tab, cudaStream_t st);
// dz = dy (y > 0) (y == nullptr: dz = dy), FP32 and BF16 copies
cudaError_t relu_bwd(const float* dy, const bf16* y, float* dz, bf16* dzb, long long count, cudaStream_t st);
// db[c] = sum_m dz[m][c]; work holds bias_work_elems(C) floats
size_t bias_work_elems(int C);
cudaError_t bias_grad(const float* dz, long long M, int C, float* db, float* work, cudaStream_t st);
// dzb = bf16(dy (y > 0)), dz = dy (y > 0) when dz != nullptr, and db = bias_grad of dy (y > 0), bit for bit, in
// one pass; with db == nullptr the per-block partials stay in work (bias_work_elems(C) floats) for conv3_wgrad
cudaError_t relu_bwd_bias(const float* dy, const bf16* y, float* dz, bf16* dzb, long long M, int C, float* db,
                          float* work, cudaStream_t st);
// 2x2x2 average pooling (fine geometry gf) and its adjoint (dx overwritten or accumulated)
cudaError_t pool_fwd(const bf16* x, bf16* y, const Geo& gf, int C, cudaStream_t st);
cudaError_t pool_bwd(const float* dy, float* dx, int accum, const Geo& gf, int C, cudaStream_t st);
// nearest-neighbour x2 upsampling (coarse geometry gc) and its adjoint
cudaError_t up_fwd(const bf16* x, bf16* y, const Geo& gc, int C, cudaStream_t st);
cudaError_t up_bwd(const float* dy, float* dx, int accum, const Geo& gc, int C, cudaStream_t st);
// mean squared error over the first cu of C channels of pred [M][C] against target [M][cu]; grad [M][C]
// (optional) = d loss / d pred; partials[nblocks] (device, FP64) sum to the loss.
cudaError_t mse(const float* pred, const float* target, float* grad, long long M, int C, int cu, double* partials,
                int nblocks, cudaStream_t st);
// one Adam step (Kingma and Ba, 2015) with bias correction for step t >= 1; pb (optional) gets a BF16 copy
cudaError_t adam(float* p, const float* g, float* m1, float* m2, bf16* pb, long long count, float lr, float b1,
                 float b2, float eps, int t, cudaStream_t st);
// sample indices of a minibatch, passed by value to the batched input kernels
struct SampleIdx {
  static constexpr int kMax = 64;
  long long v[kMax];
};
// planar FP32 images [2][N0] (m_T, m_R) of samples idx[0 .. nb-1] of images -> channels-last BF16 [nb][N0][C]:
// channel 0 = m_T, channel 1 = sdiff (m_R - m_T) formed in FP32, channels >= 2 zero
cudaError_t pack_images(const float* images, const SampleIdx& idx, int nb, bf16* dst, long long N0, int C,
                        float sdiff, cudaStream_t st);
// planar FP32 [ncomp][N0] of samples idx[0 .. nb-1] of targets -> channels-last FP32 [nb][N0][ncomp], scaled by s
cudaError_t interleave_batch(const float* targets, const SampleIdx& idx, int nb, float* dst, long long N0, int ncomp,
                             float s, cudaStream_t st);
// channels-last FP32 [M][C] -> planar [ncomp][M], scaled by s
cudaError_t unpack(const float* src, float* dst, long long M, int ncomp, int C, float s, cudaStream_t st);
cudaError_t add(const float* a, float* b, long long count, cudaStream_t st);
// synchronises st, then reports (and clears) a timed-out tensor-core wait of the convolution kernels
// (cudaErrorLaunchTimeout)
cudaError_t status(cudaStream_t st);
cudaError_t to_bf16(const float* a, bf16* b, long long count, cudaStream_t st);

}  // namespace nn
}  // namespace claire
