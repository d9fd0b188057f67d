// Batched mixed-radix 3D real FFT for the pseudo-spectral operators (Sec. 2.3.1: forward FFT, multiply by the
// symbol, inverse FFT). One kernel per axis pass; every pass reads and writes the array once.
//
//  * contiguous axis (i3): a real line of n3 values is read as n3/2 complex pairs (even + i*odd), transformed
//    with a complex FFT of length n3/2 and split into the n3/2+1 half-spectrum values (and the reverse for C2R);
//  * strided axes (i2, i1): a CTA stages TI consecutive columns of the half spectrum (rows of TI contiguous
//    complex values, coalesced) for the whole line length in shared memory and transforms them in place.
//
// Inside shared memory each transform is a Stockham autosort FFT: stage s with radix R reads x[j + r L/R],
// multiplies by exp(-+2 pi i r (j mod Ns) / (Ns R)), applies the R-point DFT in registers and writes
// y[(j / Ns) Ns R + (j mod Ns) + q Ns]. Radices 8, 4, 2 are hard-coded; 3, 5 and 7 use the twiddle table.
// Twiddle tables are computed on the host in FP64 (std::cos / std::sin) and staged in shared memory.
#include <cmath>
#include <vector>

#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>

#include "impl.cuh"

namespace claire {

bool radix_plan(int L, RadixPlan& p) {
  p.L = L;
  p.nst = 0;
  int n = L;
  const int order[6] = {8, 4, 2, 3, 5, 7};
  for (int r : order) {
    while (n % r == 0) {
      if (p.nst >= 16) return false;
      p.r[p.nst++] = r;
      n /= r;
    }
  }
  return n == 1;
}

// ------------------------------------------------------------------------------------------ register DFTs
template <class T, int SIGN, int R>
__device__ __forceinline__ void dft(cplx<T>* v, const cplx<T>* W, int L, int tws) {
  if constexpr (R == 2) {
    cplx<T> a = v[0], b = v[1];
    v[0] = cadd<T>(a, b);
    v[1] = csub<T>(a, b);
  } else if constexpr (R == 4) {
    cplx<T> a0 = cadd<T>(v[0], v[2]), a1 = csub<T>(v[0], v[2]);
    cplx<T> a2 = cadd<T>(v[1], v[3]), a3 = mul_i<SIGN, T>(csub<T>(v[1], v[3]));
    v[0] = cadd<T>(a0, a2);
    v[2] = csub<T>(a0, a2);
    v[1] = cadd<T>(a1, a3);
    v[3] = csub<T>(a1, a3);
  } else if constexpr (R == 8) {
    // X[k] = E[k] + W8^k O[k], X[k+4] = E[k] - W8^k O[k], E/O the 4-point DFTs of the even/odd inputs
    cplx<T> e[4] = {v[0], v[2], v[4], v[6]};
    cplx<T> o[4] = {v[1], v[3], v[5], v[7]};
    dft<T, SIGN, 4>(e, W, L, tws);
    dft<T, SIGN, 4>(o, W, L, tws);
    const T s = T(0.70710678118654752440084436210484903928);
    // W8^1 = (1 -+ i)/sqrt2, W8^2 = -+i, W8^3 = (-1 -+ i)/sqrt2 (upper sign forward)
    cplx<T> o1 = SIGN < 0 ? mk<T>((o[1].x + o[1].y) * s, (o[1].y - o[1].x) * s)
                          : mk<T>((o[1].x - o[1].y) * s, (o[1].y + o[1].x) * s);
    cplx<T> o2 = mul_i<SIGN, T>(o[2]);
    cplx<T> o3 = SIGN < 0 ? mk<T>((-o[3].x + o[3].y) * s, (-o[3].y - o[3].x) * s)
                          : mk<T>((-o[3].x - o[3].y) * s, (-o[3].y + o[3].x) * s);
    v[0] = cadd<T>(e[0], o[0]);
    v[4] = csub<T>(e[0], o[0]);
    v[1] = cadd<T>(e[1], o1);
    v[5] = csub<T>(e[1], o1);
    v[2] = cadd<T>(e[2], o2);
    v[6] = csub<T>(e[2], o2);
    v[3] = cadd<T>(e[3], o3);
    v[7] = csub<T>(e[3], o3);
  } else {
    // generic odd radix: X[q] = sum_r x[r] W_R^{+-rq}, W_R^t = table[t L / R]
    cplx<T> out[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      cplx<T> acc = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const cplx<T> w = W[(((r * q) % R) * (L / R)) * tws];
        acc = cadd<T>(acc, SIGN < 0 ? cmul<T>(v[r], w) : cmulc<T>(v[r], w));
      }
      out[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = out[q];
  }
}

template <class T, int SIGN, int R>
__device__ __forceinline__ void stage_body(const cplx<T>* __restrict__ a, cplx<T>* __restrict__ b, int j, int col,
                                           int Ns, int L, int cs, int es, const cplx<T>* W, int tws) {
  const int nb = L / R;
  const int k = j % Ns;
  const int tstep = k * (L / (Ns * R));
  cplx<T> v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    cplx<T> x = a[col * cs + (j + r * nb) * es];
    if (r > 0) {
      const cplx<T> w = W[(r * tstep) * tws];
      x = SIGN < 0 ? cmul<T>(x, w) : cmulc<T>(x, w);
    }
    v[r] = x;
  }
  dft<T, SIGN, R>(v, W, L, tws);
  const int idxD = (j / Ns) * Ns * R + k;
#pragma unroll
  for (int q = 0; q < R; ++q) b[col * cs + (idxD + q * Ns) * es] = v[q];
}

// Stockham FFT of `ncols` independent lines held in shared memory at a[col*cs + i*es]; returns the buffer that
// holds the result (a or b). colfast selects which index consecutive threads walk (column or butterfly).
template <class T, int SIGN>
__device__ cplx<T>* stockham(cplx<T>* a, cplx<T>* b, const RadixPlan& rp, int ncols, int cs, int es, bool colfast,
                             const cplx<T>* W, int tws) {
  int Ns = 1;
  const int L = rp.L;
  for (int s = 0; s < rp.nst; ++s) {
    const int R = rp.r[s];
    const int nb = L / R;
    const int total = nb * ncols;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      int col, j;
      if (colfast) {
        col = idx % ncols;
        j = idx / ncols;
      } else {
        j = idx % nb;
        col = idx / nb;
      }
      switch (R) {
        case 8: stage_body<T, SIGN, 8>(a, b, j, col, Ns, L, cs, es, W, tws); break;
        case 4: stage_body<T, SIGN, 4>(a, b, j, col, Ns, L, cs, es, W, tws); break;
        case 2: stage_body<T, SIGN, 2>(a, b, j, col, Ns, L, cs, es, W, tws); break;
        case 3: stage_body<T, SIGN, 3>(a, b, j, col, Ns, L, cs, es, W, tws); break;
        case 5: stage_body<T, SIGN, 5>(a, b, j, col, Ns, L, cs, es, W, tws); break;
        default: stage_body<T, SIGN, 7>(a, b, j, col, Ns, L, cs, es, W, tws); break;
      }
    }
    __syncthreads();
    cplx<T>* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// ------------------------------------------------------------------------------------------ pass kernels
// Contiguous axis, forward: real lines of n3 -> half spectra of n3/2+1.
template <class T>
__global__ void __launch_bounds__(256) k_fft_z_r2c(const T* __restrict__ in, cplx<T>* __restrict__ out,
                                                   long long nlines, int n3, RadixPlan rp,
                                                   const cplx<T>* __restrict__ Wg, int lpc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* W = reinterpret_cast<cplx<T>*>(smem_raw);
  const int L = rp.L;
  const int S = L + 1;
  cplx<T>* A = W + n3;
  cplx<T>* B = A + lpc * S;
  const long long line0 = (long long)blockIdx.x * lpc;
  const int nl = (int)min((long long)lpc, nlines - line0);
  for (int t = threadIdx.x; t < n3; t += blockDim.x) W[t] = Wg[t];
  const cplx<T>* src = reinterpret_cast<const cplx<T>*>(in + line0 * n3);
  for (int t = threadIdx.x; t < nl * L; t += blockDim.x) {
    const int l = t / L, i = t - l * L;
    A[l * S + i] = src[t];
  }
  __syncthreads();
  const cplx<T>* Z = stockham<T, -1>(A, B, rp, nl, S, 1, false, W, 2);
  cplx<T>* dst = out + line0 * (long long)S;
  for (int t = threadIdx.x; t < nl * S; t += blockDim.x) {
    const int l = t / S, k = t - l * S;
    const cplx<T> zk = Z[l * S + (k == L ? 0 : k)];
    const cplx<T> zc = cconj<T>(Z[l * S + (k == 0 ? 0 : L - k)]);
    const cplx<T> sum = cadd<T>(zk, zc), dif = csub<T>(zk, zc);
    const cplx<T> wd = cmul<T>(W[k], dif);
    // X[k] = (Z[k] + conj Z[L-k]) / 2 - i/2 exp(-2 pi i k/n3) (Z[k] - conj Z[L-k])
    dst[t] = mk<T>(T(0.5) * (sum.x + wd.y), T(0.5) * (sum.y - wd.x));
  }
}

// Contiguous axis, inverse: half spectra of n3/2+1 -> real lines of n3, times `scale`.
template <class T>
__global__ void __launch_bounds__(256) k_fft_z_c2r(const cplx<T>* __restrict__ in, T* __restrict__ out,
                                                   long long nlines, int n3, RadixPlan rp,
                                                   const cplx<T>* __restrict__ Wg, int lpc, T scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* W = reinterpret_cast<cplx<T>*>(smem_raw);
  const int L = rp.L;
  const int S = L + 1;
  cplx<T>* A = W + n3;
  cplx<T>* B = A + lpc * S;
  const long long line0 = (long long)blockIdx.x * lpc;
  const int nl = (int)min((long long)lpc, nlines - line0);
  for (int t = threadIdx.x; t < n3; t += blockDim.x) W[t] = Wg[t];
  const cplx<T>* src = in + line0 * (long long)S;
  for (int t = threadIdx.x; t < nl * S; t += blockDim.x) B[t] = src[t];
  __syncthreads();
  for (int t = threadIdx.x; t < nl * L; t += blockDim.x) {
    const int l = t / L, k = t - l * L;
    const cplx<T> xk = B[l * S + k];
    const cplx<T> xc = cconj<T>(B[l * S + L - k]);
    const cplx<T> sum = cadd<T>(xk, xc), dif = csub<T>(xk, xc);
    const cplx<T> wd = cmulc<T>(dif, W[k]);  // (X[k] - conj X[L-k]) exp(+2 pi i k/n3)
    A[l * S + k] = mk<T>(sum.x - wd.y, sum.y + wd.x);
  }
  __syncthreads();
  const cplx<T>* Z = stockham<T, +1>(A, B, rp, nl, S, 1, false, W, 2);
  cplx<T>* dst = reinterpret_cast<cplx<T>*>(out + line0 * n3);
  for (int t = threadIdx.x; t < nl * L; t += blockDim.x) {
    const int l = t / L, i = t - l * L;
    const cplx<T> z = Z[l * S + i];
    dst[t] = mk<T>(z.x * scale, z.y * scale);
  }
}

// Strided axis (length L, element stride `inner`): reads src, writes data (src == data: in place); grid.x over
// column tiles, grid.y over outer slabs.
template <class T, int SIGN>
__global__ void __launch_bounds__(256) k_fft_strided(const cplx<T>* src, cplx<T>* data, long long inner,
                                                     RadixPlan rp, const cplx<T>* __restrict__ Wg, int TI) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* W = reinterpret_cast<cplx<T>*>(smem_raw);
  const int L = rp.L;
  cplx<T>* A = W + L;
  cplx<T>* B = A + L * TI;
  for (int t = threadIdx.x; t < L; t += blockDim.x) W[t] = Wg[t];
  const long long i0 = (long long)blockIdx.x * TI;
  const int nc = (int)min((long long)TI, inner - i0);
  const long long off = (long long)blockIdx.y * L * inner + i0;
  cplx<T>* base = data + off;
  const cplx<T>* sbase = src + off;
  for (int t = threadIdx.x; t < L * TI; t += blockDim.x) {
    const int a = t / TI, c = t - a * TI;
    if (c < nc) A[t] = sbase[(long long)a * inner + c];
  }
  __syncthreads();
  const cplx<T>* Y = stockham<T, SIGN>(A, B, rp, nc, 1, TI, true, W, 1);
  for (int t = threadIdx.x; t < L * TI; t += blockDim.x) {
    const int a = t / TI, c = t - a * TI;
    if (c < nc) base[(long long)a * inner + c] = Y[t];
  }
}

// ------------------------------------------------------------------------------------------ host side
template <class T> static std::vector<cplx<T>> make_table(int n) {
  std::vector<cplx<T>> w(n);
  const double twopi = 6.283185307179586476925286766559;
  for (int t = 0; t < n; ++t) {
    const double ang = -twopi * double(t) / double(n);
    w[t] = mk<T>(T(std::cos(ang)), T(std::sin(ang)));
  }
  return w;
}

template <class T> size_t fft_table_bytes(const Dims& d) {
  return size_t(d.n1 + d.n2 + d.n3) * sizeof(cplx<T>) + 3 * 256;
}

static constexpr int kMaxSmem = 200 * 1024;

template <class T> static size_t smem_z(int n3, int lpc) {
  return (size_t(n3) + 2 * size_t(lpc) * size_t(n3 / 2 + 1)) * sizeof(cplx<T>);
}
template <class T> static size_t smem_s(int L, int ti) { return (size_t(L) + 2 * size_t(L) * ti) * sizeof(cplx<T>); }

template <class T> claire_status fft_init(claire_ctx* c) {
  FFTPlan<T>& p = c->plan<T>();
  const Dims& d = c->d;
  if (!radix_plan(d.n1, p.ax1) || !radix_plan(d.n2, p.ax2) || !radix_plan(d.n3 / 2, p.ax3)) {
    c->set_error("grid sizes must factor into 2, 3, 5 and 7");
    return CLAIRE_EINVAL;
  }
  // columns per CTA of the strided passes: rows of 128 bytes when the two buffers fit in ~100 KB
  const int maxL = d.n1 > d.n2 ? d.n1 : d.n2;
  int ti = 128 / int(sizeof(cplx<T>));
  while (ti > 1 && smem_s<T>(maxL, ti) > 100 * 1024) ti /= 2;
  p.ti12 = ti;
  int lpc = 2048 / (d.n3 / 2);
  if (lpc < 1) lpc = 1;
  while (lpc > 1 && smem_z<T>(d.n3, lpc) > 100 * 1024) lpc /= 2;
  p.lpc3 = lpc;
  if (smem_s<T>(maxL, ti) > size_t(kMaxSmem) || smem_z<T>(d.n3, lpc) > size_t(kMaxSmem)) {
    c->set_error("grid too large for the shared-memory FFT passes");
    return CLAIRE_EINVAL;
  }
  p.tw1 = static_cast<cplx<T>*>(c->take(sizeof(cplx<T>) * d.n1));
  p.tw2 = static_cast<cplx<T>*>(c->take(sizeof(cplx<T>) * d.n2));
  p.tw3 = static_cast<cplx<T>*>(c->take(sizeof(cplx<T>) * d.n3));
  if (!p.tw1 || !p.tw2 || !p.tw3) {
    c->set_error("workspace arena too small for twiddle tables");
    return CLAIRE_ENOMEM;
  }
  auto w1 = make_table<T>(d.n1), w2 = make_table<T>(d.n2), w3 = make_table<T>(d.n3);
  CL_CUDA(c, cudaMemcpy(p.tw1, w1.data(), sizeof(cplx<T>) * d.n1, cudaMemcpyHostToDevice));
  CL_CUDA(c, cudaMemcpy(p.tw2, w2.data(), sizeof(cplx<T>) * d.n2, cudaMemcpyHostToDevice));
  CL_CUDA(c, cudaMemcpy(p.tw3, w3.data(), sizeof(cplx<T>) * d.n3, cudaMemcpyHostToDevice));
  CL_CUDA(c, cudaFuncSetAttribute(k_fft_z_r2c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
  CL_CUDA(c, cudaFuncSetAttribute(k_fft_z_c2r<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
  CL_CUDA(c, cudaFuncSetAttribute(k_fft_strided<T, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
  CL_CUDA(c, cudaFuncSetAttribute(k_fft_strided<T, +1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
  return CLAIRE_OK;
}

template <class T> claire_status fft_r2c(claire_ctx* c, const T* in, cplx<T>* out, cudaStream_t st) {
  const FFTPlan<T>& p = c->plan<T>();
  const Dims& d = c->d;
  const long long nlines = (long long)d.n1 * d.n2;
  const long long inner1 = (long long)d.n2 * d.n3h;
  c->prof_begin("fft_z_r2c", st);
  if (!fft2_z<T>(d.n3 / 2, -1, in, out, nlines, p.tw3, T(1), st, p.var_z)) {
    const unsigned grid = (unsigned)((nlines + p.lpc3 - 1) / p.lpc3);
    k_fft_z_r2c<T><<<grid, 256, smem_z<T>(d.n3, p.lpc3), st>>>(in, out, nlines, d.n3, p.ax3, p.tw3, p.lpc3);
  }
  CL_LAUNCHED(c);
  c->prof_begin("fft_y_fwd", st);
  if (!fft2_strided<T>(d.n2, -1, out, out, d.n3h, d.n1, p.tw2, st, p.var_y)) {
    dim3 grid((unsigned)((d.n3h + p.ti12 - 1) / p.ti12), (unsigned)d.n1);
    k_fft_strided<T, -1><<<grid, 256, smem_s<T>(d.n2, p.ti12), st>>>(out, out, d.n3h, p.ax2, p.tw2, p.ti12);
  }
  CL_LAUNCHED(c);
  c->prof_begin("fft_x_fwd", st);
  if (!fft2_strided<T>(d.n1, -1, out, out, inner1, 1, p.tw1, st, p.var_x)) {
    dim3 grid((unsigned)((inner1 + p.ti12 - 1) / p.ti12), 1u);
    k_fft_strided<T, -1><<<grid, 256, smem_s<T>(d.n1, p.ti12), st>>>(out, out, inner1, p.ax1, p.tw1, p.ti12);
  }
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

template <class T>
claire_status fft_c2r(claire_ctx* c, cplx<T>* spec, T* out, T scale, cudaStream_t st, const cplx<T>* src) {
  const FFTPlan<T>& p = c->plan<T>();
  const Dims& d = c->d;
  const long long nlines = (long long)d.n1 * d.n2;
  const long long inner1 = (long long)d.n2 * d.n3h;
  const cplx<T>* first = src ? src : spec;
  c->prof_begin("fft_x_inv", st);
  if (!fft2_strided<T>(d.n1, +1, first, spec, inner1, 1, p.tw1, st, p.var_x)) {
    dim3 grid((unsigned)((inner1 + p.ti12 - 1) / p.ti12), 1u);
    k_fft_strided<T, +1><<<grid, 256, smem_s<T>(d.n1, p.ti12), st>>>(first, spec, inner1, p.ax1, p.tw1, p.ti12);
  }
  CL_LAUNCHED(c);
  c->prof_begin("fft_y_inv", st);
  if (!fft2_strided<T>(d.n2, +1, spec, spec, d.n3h, d.n1, p.tw2, st, p.var_y)) {
    dim3 grid((unsigned)((d.n3h + p.ti12 - 1) / p.ti12), (unsigned)d.n1);
    k_fft_strided<T, +1><<<grid, 256, smem_s<T>(d.n2, p.ti12), st>>>(spec, spec, d.n3h, p.ax2, p.tw2, p.ti12);
  }
  CL_LAUNCHED(c);
  c->prof_begin("fft_z_c2r", st);
  if (!fft2_z<T>(d.n3 / 2, +1, spec, out, nlines, p.tw3, scale, st, p.var_z)) {
    const unsigned grid = (unsigned)((nlines + p.lpc3 - 1) / p.lpc3);
    k_fft_z_c2r<T><<<grid, 256, smem_z<T>(d.n3, p.lpc3), st>>>(spec, out, nlines, d.n3, p.ax3, p.tw3, p.lpc3,
                                                                scale);
  }
  CL_LAUNCHED(c);
  return CLAIRE_OK;
}

// Autotuner of the FFT tile shapes: for each axis whose length has a specialised pass, time a forward and an
// inverse pass of each tile variant (columns per CTA of the strided y and x passes, lines per CTA of the contiguous
// z passes) on this context's work arrays, three times after a warm-up, and keep the fastest; the choice is cached
// per grid for the process. Only FP32 passes have variants. CLAIRE_FFT_TILES=default keeps the defaults;
// CLAIRE_FFT_TILES=z,y,x (three variants 0..2) forces a choice. A variant changes only how many lines one CTA
// transforms: every line takes the same arithmetic in the same order, so the results are bit-identical.
template <class T> claire_status fft_tune(claire_ctx* c) {
  if (sizeof(T) != 4) return CLAIRE_OK;
  FFTPlan<T>& p = c->plan<T>();
  const char* env = std::getenv("CLAIRE_FFT_TILES");
  if (env && std::strcmp(env, "default") == 0) return CLAIRE_OK;
  int fz = 0, fy = 0, fx = 0;
  if (env && std::sscanf(env, "%d,%d,%d", &fz, &fy, &fx) == 3) {  // forced variants (z, y, x), each 0..2
    if (fz < 0 || fz > 2 || fy < 0 || fy > 2 || fx < 0 || fx > 2) return CLAIRE_EINVAL;
    p.var_z = fz;
    p.var_y = fy;
    p.var_x = fx;
    return CLAIRE_OK;
  }
  static std::mutex mu;
  static std::map<std::tuple<int, int, int>, std::tuple<int, int, int>> cache;
  const Dims& d = c->d;
  const auto key = std::make_tuple(d.n1, d.n2, d.n3);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      std::tie(p.var_y, p.var_x, p.var_z) = it->second;
      return CLAIRE_OK;
    }
  }
  Work<T>& W = c->work<T>();
  cplx<T>* S = W.spec;
  T* f = W.b;  // 3N values, at least N
  cudaStream_t st;
  CL_CUDA(c, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e[2];
  CL_CUDA(c, cudaEventCreate(&e[0]));
  CL_CUDA(c, cudaEventCreate(&e[1]));
  claire_status status = CLAIRE_OK;
  auto best_of = [&](auto&& run, int* out) -> claire_status {
    float best = 0.f;
    int bv = 0;
    for (int v = 0; v < 3; ++v) {
      if (!run(v)) return CLAIRE_OK;  // no specialised pass for this length
      CL_CUDA(c, cudaEventRecord(e[0], st));
      for (int r = 0; r < 3; ++r) run(v);
      CL_CUDA(c, cudaEventRecord(e[1], st));
      CL_CUDA(c, cudaEventSynchronize(e[1]));
      float ms = 0.f;
      CL_CUDA(c, cudaEventElapsedTime(&ms, e[0], e[1]));
      CL_CUDA(c, cudaGetLastError());
      if (v == 0 || ms < best) {
        best = ms;
        bv = v;
      }
    }
    *out = bv;
    return CLAIRE_OK;
  };
  const long long nlines = (long long)d.n1 * d.n2;
  const long long inner1 = (long long)d.n2 * d.n3h;
  status = zero_fill<T>(c, d.N, f, st);
  if (status == CLAIRE_OK) status = zero_fill<T>(c, 2 * d.Ns, reinterpret_cast<T*>(S), st);
  int vy = 0, vx = 0, vz = 0;
  if (status == CLAIRE_OK)
    status = best_of([&](int v) { return fft2_strided<T>(d.n2, -1, S, S, d.n3h, d.n1, p.tw2, st, v) &&
                                         fft2_strided<T>(d.n2, +1, S, S, d.n3h, d.n1, p.tw2, st, v); }, &vy);
  if (status == CLAIRE_OK)
    status = best_of([&](int v) { return fft2_strided<T>(d.n1, -1, S, S, inner1, 1, p.tw1, st, v) &&
                                         fft2_strided<T>(d.n1, +1, S, S, inner1, 1, p.tw1, st, v); }, &vx);
  if (status == CLAIRE_OK)
    status = best_of([&](int v) { return fft2_z<T>(d.n3 / 2, -1, f, S, nlines, p.tw3, T(1), st, v) &&
                                         fft2_z<T>(d.n3 / 2, +1, S, f, nlines, p.tw3, T(1), st, v); }, &vz);
  cudaEventDestroy(e[0]);
  cudaEventDestroy(e[1]);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (status != CLAIRE_OK) return status;
  p.var_y = vy;
  p.var_x = vx;
  p.var_z = vz;
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = std::make_tuple(vy, vx, vz);
  return CLAIRE_OK;
}

template size_t fft_table_bytes<float>(const Dims&);
template claire_status fft_tune<float>(claire_ctx*);
template claire_status fft_tune<double>(claire_ctx*);
template size_t fft_table_bytes<double>(const Dims&);
template claire_status fft_init<float>(claire_ctx*);
template claire_status fft_init<double>(claire_ctx*);
template claire_status fft_r2c<float>(claire_ctx*, const float*, cplx<float>*, cudaStream_t);
template claire_status fft_r2c<double>(claire_ctx*, const double*, cplx<double>*, cudaStream_t);
template claire_status fft_c2r<float>(claire_ctx*, cplx<float>*, float*, float, cudaStream_t, const cplx<float>*);
template claire_status fft_c2r<double>(claire_ctx*, cplx<double>*, double*, double, cudaStream_t,
                                        const cplx<double>*);

}  // namespace claire
