// Internal interfaces between the translation units of the library (not part of the C-ABI).
#pragma once

#include <cuda.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace claire {

// TMA tensor maps of the operands the staged adjoint and incremental-state steps load (sl_tma.cu): boxes of
// 16 x 16 x 4 nodes x 3 components of Y, X, the PCG direction s, the gradient history (FP32 or BF16, with the time
// index as a fifth dimension) and b; built once per context for the workspace arrays they describe
struct TmaMaps {
  CUtensorMap dY, dX, s, gm, gm16, b;
  const void* key[4] = {nullptr, nullptr, nullptr, nullptr};
  bool tried = false, ok = false;
};

// Twiddle tables and radix schedules of the three 1D passes of a 3D real FFT (Sec. 2.3.1 spectral operators).
template <class T> struct FFTPlan {
  RadixPlan ax1{}, ax2{}, ax3{};  // complex lengths n1, n2 and n3/2
  cplx<T>* tw1 = nullptr;          // exp(-2 pi i t / n1), t < n1
  cplx<T>* tw2 = nullptr;          // exp(-2 pi i t / n2), t < n2
  cplx<T>* tw3 = nullptr;          // exp(-2 pi i t / n3), t < n3 (the z pass uses every other entry)
  int ti12 = 16;                   // columns per CTA of the strided passes
  int lpc3 = 16;                   // lines per CTA of the contiguous pass
  int var_y = 0, var_x = 0, var_z = 0;  // tile variants of the specialised passes (chosen by fft_tune)
};

// Device workspace of one context (all owned by the context arena).
template <class T> struct Work {
  T* dX = nullptr;      // [3][N] state departure displacement (grid units)
  T* dY = nullptr;      // [3][N] adjoint departure displacement
  T* m = nullptr;       // [nt+1][N] state history
  T* gm = nullptr;      // [nt+1][3][N] spectral gradients of the state history
  void* gm16 = nullptr; // [nt+1][3][N] the same history in BF16 (reduced-storage mode, FP32 only)
  T* rho = nullptr;     // [N] div v (only without the div v = 0 constraint)
  T* la = nullptr;      // [N] adjoint ping
  T* lb = nullptr;      // [N] adjoint pong
  T* ra = nullptr;      // [N] rho * adjoint ping (only without the div v = 0 constraint)
  T* rb = nullptr;      // [N] rho * adjoint pong (only without the div v = 0 constraint)
  T* b = nullptr;       // [3][N] time integral accumulator
  cplx<T>* spec = nullptr;  // 6 half spectra of Ns values
  T* s = nullptr;       // [3][N] PCG search direction in physical space (input of the matvec's SL solves)
  T* vtrial = nullptr;  // [3][N] line-search trial velocity
  T* vdev = nullptr;    // [3][N] device copy of v for the host-array API (allocated on first use; in the arena of
                        // a two-level coarse context, which keeps its restricted v here)
  T* mTdev = nullptr;   // [N] (the same; the coarse context's restricted m_T)
  T* mRdev = nullptr;   // [N] (host-array API only)
  // Fourier-domain solver vectors, 3 half spectra (component stride Ns) each
  cplx<T>* Vh = nullptr;   // v (master copy)
  cplx<T>* Vtrh = nullptr; // line-search trial v
  cplx<T>* Gh = nullptr;   // reduced gradient
  cplx<T>* Rh = nullptr;   // PCG residual
  cplx<T>* Sh = nullptr;   // PCG direction
  cplx<T>* VTh = nullptr;  // Newton step vt
  cplx<T>* Bh = nullptr;   // transform of the time integral b (= spec, the lower three spectra)
  cplx<T>* Sc = nullptr;   // work array of inverse transforms (= spec + 3 Ns, the upper three)
  double* bigpart = nullptr;   // one FP64 partial per block of the gather launch shape
  long long nbig = 0;
  double* partials = nullptr;  // reduction partials, [4][kReduceBlocks]
  double* scal = nullptr;      // device scalars (kScalSlots doubles)
};

constexpr int kScalSlots = 64;

constexpr int kReduceBlocks = 1216;  // 8 per SM on 152 SMs: the FP32 kernels on this grid are compiled for 8 resident
                                     // CTAs (32 registers), so the grid is one wave (two waves cost up to 1.5x)

// Device-side PCG state (Alg. 2 driven from the device inside a CUDA graph): FP64 slots of Work::scal from kPcgBase.
enum PcgSlot {
  kPcgRz = 0,      // <r, z>
  kPcgR0,          // ||r_0||
  kPcgSAs,         // <s, beta A s>
  kPcgEps,         // forcing term eps_H
  kPcgKappa,       // step length of the current iteration
  kPcgMu,          // direction update
  kPcgDone,        // 1 once converged, broken down or non-finite
  kPcgBreakdown,   // <s, H s> <= 0
  kPcgNan,         // non-finite <s, H s>
  kPcgCopyS,       // breakdown in the first iteration: the step is the first direction
  kPcgCount,       // matvecs done
  kPcgMaxIt,       // Krylov iteration cap
  kPcgSlots
};
constexpr int kPcgBase = 16;

// Device-side state of Alg. 1 driven from the device (FP64 slots of Work::scal from kGnBase): the iterate's
// objective and gradient norm, the Armijo search, the counts of the report and the outcome.
enum GnSlot {
  kGnJ = 0,        // objective at the current iterate
  kGnJt,           // objective at the last trial
  kGnGnorm,        // ||g_k||
  kGnGnorm0,       // ||g(v = 0)||
  kGnGvt,          // <g, vt> (the Armijo slope)
  kGnAlpha,        // step length of the current trial
  kGnTrial,        // trials of the current search
  kGnAccepted,     // the current search accepted a step
  kGnIters,        // Gauss-Newton iterations
  kGnMatvecs,      // Hessian matvecs
  kGnPde,          // PDE solves
  kGnLsTrials,     // objective evaluations of the Armijo searches
  kGnBreakdowns,   // PCG iterations stopped by <s, H s> <= 0
  kGnStatus,       // 0 running, 1 converged, 2 max_gn, 3 line search failed, 4 non-finite
  kGnMaxGn,        // the options the loop reads
  kGnMaxLs,
  kGnC1,
  kGnGtolRel,
  kGnGtolAbs,
  kGnPcgRtol,
  kGnMaxKrylov,
  kGnMismatch,     // 1/2 ||m_1 - m_R||^2 at the returned v
  kGnJ0,           // objective (= mismatch) at v = 0
  kGnSlots
};
constexpr int kGnBase = 32;
static_assert(kGnBase + kGnSlots <= kScalSlots, "device state block");
constexpr int kThreads = 256;

}  // namespace claire

struct claire_ctx {
  claire_opts o{};
  claire_ctx* coarse = nullptr;  // half-resolution context of the two-level preconditioner (opts.precond = 1)
  claire::Dims d{};
  claire::Counters counters{};
  std::string err;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  void* hostbuf = nullptr;     // device copies for the host-array calls, allocated on first use
  bool is_coarse = false;      // the half-resolution context of a two-level preconditioner
  size_t arena_used = 0;
  claire::FFTPlan<float> pf{};
  claire::FFTPlan<double> pd{};
  claire::Work<float> wf{};
  claire::Work<double> wd{};
  bool lin_valid = false;
  bool f64_plan = false;       // FP32 context with an FP64 FFT plan (stand-alone operators that apply a growing
                               // symbol to a physical field transform it in FP64)
  bool gm16_on = false;        // gradient history stored in BF16 (claire_opts.bf16_mask bit 0)
  bool gm_ready = false;       // the gradient history holds finite values (used as autotuning input)
  int haloX = -1, haloY = -1;    // brick halo of the cached departure points (-1: plain gathers), light kernels
  int haloXh = -1, haloYh = -1;  // the same for the heavy kernels (last incremental step, fused-product/div steps)
  bool halo_fixed = false;       // keep the halos above (a solve driven from the device cannot read max |Y|)
  // CUDA graph of a whole zero-start solve driven from the device (Alg. 1 and Alg. 2 as conditional nodes), kept
  // for the pointers, halos and beta_v it was captured with
  cudaGraph_t gn_graph = nullptr;
  cudaGraphExec_t gn_exec = nullptr;
  const void* gn_key_ptr[3] = {nullptr, nullptr, nullptr};
  int gn_key_halo[4] = {0, 0, 0, 0};
  double gn_beta = 0.0;
  // launches per part of the captured solve (for the launch counter): per pair outside the loops, per GN
  // iteration outside its inner loops, per PCG iteration, per Armijo trial, per accepted step
  long long gn_l_pair = 0, gn_l_iter = 0, gn_l_pcg = 0, gn_l_trial = 0, gn_l_accept = 0;
  // device block of the graph: current pair index, pair count, pair table, per-pair reports, state template
  void* gn_dev = nullptr;
  int gn_cap = 0;
  cudaStream_t gn_cap_streams[3] = {nullptr, nullptr, nullptr};  // capture streams of the nested loop bodies
  long long dot_blocks = 0;    // partials written by the last dot-fused adjoint step
  claire::TmaMaps tma;         // tensor maps of the TMA-staged adjoint steps (FP32 contexts)
  long long tma_steps = 0;     // adjoint steps run with TMA-staged operands
  // CUDA graph of the device-driven PCG loop (one conditional WHILE node around one iteration), kept for the
  // gather schedule it was captured with
  cudaGraph_t pcg_graph = nullptr;
  cudaGraphExec_t pcg_exec = nullptr;
  int pcg_key[4] = {0, 0, 0, 0};
  double pcg_beta = 0.0;  // beta_v baked into the captured kernels' arguments (continuation changes it)
  long long pcg_body_launches = 0;
  long long pcg_graph_runs = 0;  // PCG solves run as one graph launch
  long long gn_graph_runs = 0;   // launches of the device-driven solve graph
  bool pcg_graph_failed = false;
  cudaStream_t pcg_cap_stream = nullptr;  // capture needs a stream other than the legacy default stream
  double* hscal = nullptr;  // pinned host mirror of Work::scal
  // optional per-launch CUDA-event timing (off by default): one event pair per kernel launch, summed per name
  struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  ProfRec prof_pending{};
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  cudaEvent_t prof_event() {
    cudaEvent_t e = nullptr;
    if (!prof_pool.empty()) {
      e = prof_pool.back();
      prof_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
      e = nullptr;
    }
    return e;
  }
  const char* last_launch = "";  // name of the last kernel launched (for error messages)
  void prof_begin(const char* name, cudaStream_t st) {
    last_launch = name;
    if (!prof_on) return;
    prof_pending.name = name;
    prof_pending.a = prof_event();
    prof_pending.b = prof_event();
    if (prof_pending.a) cudaEventRecord(prof_pending.a, st);
  }
  void prof_end(cudaStream_t st) {
    if (!prof_on || !prof_pending.a || !prof_pending.b) return;
    cudaEventRecord(prof_pending.b, st);
    prof_recs.push_back(prof_pending);
    prof_pending = ProfRec{};
  }
  void set_error(const std::string& s) { err = s; }
  template <class T> claire::Work<T>& work();
  template <class T> claire::FFTPlan<T>& plan();
  void* take(size_t bytes) {
    size_t off = (arena_used + 255) & ~size_t(255);
    if (off + bytes > arena_bytes) return nullptr;
    arena_used = off + bytes;
    return arena + off;
  }
};
template <> inline claire::Work<float>& claire_ctx::work<float>() { return wf; }
template <> inline claire::Work<double>& claire_ctx::work<double>() { return wd; }
template <> inline claire::FFTPlan<float>& claire_ctx::plan<float>() { return pf; }
template <> inline claire::FFTPlan<double>& claire_ctx::plan<double>() { return pd; }

namespace claire {

// ---- fft.cu ---------------------------------------------------------------------------------------------------
bool radix_plan(int L, RadixPlan& p);
template <class T> size_t fft_table_bytes(const Dims& d);
template <class T> claire_status fft_init(claire_ctx* c);
// forward R2C of a scalar: in [N] real -> out [Ns] half spectrum (unnormalised)
template <class T> claire_status fft_r2c(claire_ctx* c, const T* in, cplx<T>* out, cudaStream_t st);
// inverse C2R: spec [Ns] (overwritten) -> out [N], multiplied by `scale` (1/N for the true inverse). With src
// given, the first pass reads src instead of spec (src is left untouched; spec is used as the work array).
template <class T> claire_status fft_c2r(claire_ctx* c, cplx<T>* spec, T* out, T scale, cudaStream_t st,
                                         const cplx<T>* src = nullptr);

// ---- fft2.cu: length-specialised passes (false: no specialisation for L) ----
// var: tile variant of the FP32 passes (0 default, 1 half, 2 double the columns or lines per CTA; see fft2.cu)
template <class T> bool fft2_strided(int L, int sign, const cplx<T>* src, cplx<T>* dst, long long inner, int outer,
                                     const cplx<T>* W, cudaStream_t st, int var = 0);
template <class T> bool fft2_z(int L, int sign, const void* in, void* out, long long nlines, const cplx<T>* Wn3,
                               T scale, cudaStream_t st, int var = 0);
// time the tile variants of the specialised passes on this grid once (FP32; cached per grid) and keep the fastest
template <class T> claire_status fft_tune(claire_ctx* c);

// ---- spectral.cu ----------------------------------------------------------------------------------------------
template <class T> claire_status spec_grad(claire_ctx* c, const cplx<T>* F, cplx<T>* G0, cplx<T>* G1, cplx<T>* G2,
                                           cudaStream_t st);
template <class T> claire_status spec_div(claire_ctx* c, const cplx<T>* V0, const cplx<T>* V1, const cplx<T>* V2,
                                          cplx<T>* D, cudaStream_t st);
template <class T> claire_status spec_leray(claire_ctx* c, cplx<T>* V0, cplx<T>* V1, cplx<T>* V2, cudaStream_t st);
// V = K V with the context's K of Eq. (5) (identity, Leray, or the H1-div operator)
template <class T> claire_status spec_kop(claire_ctx* c, cplx<T>* V0, cplx<T>* V1, cplx<T>* V2, cudaStream_t st);
// mode 0: V *= scale * a(k); mode 1: V *= 1/(beta a(k)) (1 where a = 0); mode 2: V *= -|k|^2 (Laplacian)
template <class T> claire_status spec_scale(claire_ctx* c, cplx<T>* V, int ncomp, long long comp_stride, int mode,
                                            double beta, cudaStream_t st);
// B = beta a(k) V + K^ B (K^ = I or Leray)
template <class T> claire_status spec_combine(claire_ctx* c, const cplx<T>* V, cplx<T>* B, cudaStream_t st);
// B = V + K^ B (V already multiplied by its symbol)
template <class T> claire_status spec_addk(claire_ctx* c, const cplx<T>* V, cplx<T>* B, cudaStream_t st);
// FP32 context, FP64 transform: fd = f as FP64, Sd = its half spectrum (FP64 plan), V = f(k) Sd rounded once to
// FP32 with f = scale a(k) (mode 0) or -|k|^2 (mode 2). fd needs N doubles, Sd Ns complex doubles.
claire_status symbol_r2c_f64(claire_ctx* c, const float* f, double* fd, cplx<double>* Sd, cplx<float>* V, int mode,
                             double scale, cudaStream_t st);
// partial sums of sum_c sum_{half k} w(k3) a(k) |V_c(k)|^2 into partials[kReduceBlocks]
template <class T> claire_status spec_reg_partial(claire_ctx* c, const cplx<T>* V, double* partials, cudaStream_t st);

// Fourier-domain solver vectors (3 components of Ns each); partials laid out [value][kReduceBlocks]
template <class T> claire_status sp_grad(claire_ctx* c, const cplx<T>* V, const cplx<T>* B, cplx<T>* G,
                                         double* partials, cudaStream_t st);
template <class T> claire_status sp_pcg0(claire_ctx* c, const cplx<T>* G, cplx<T>* R, cplx<T>* S, cplx<T>* Vt,
                                         double* partials, cudaStream_t st);
// ps (optional): the device-side PCG state block; the step then reads kappa (mu) from it and does nothing once its
// done flag is set
template <class T> claire_status sp_pcg_step(claire_ctx* c, const cplx<T>* S, const cplx<T>* Bt, cplx<T>* R,
                                             cplx<T>* Vt, double kappa, double* partials, cudaStream_t st,
                                             const double* ps = nullptr);
template <class T> claire_status sp_pcg_dir(claire_ctx* c, const cplx<T>* R, cplx<T>* S, double mu, double* partials,
                                            cudaStream_t st, const double* ps = nullptr);
template <class T> claire_status sp_project_dot(claire_ctx* c, const cplx<T>* G, cplx<T>* Vt, double* partials,
                                                cudaStream_t st);
// alpha_dev (optional): the step length read from device memory instead of alpha
template <class T> claire_status sp_trial(claire_ctx* c, const cplx<T>* V, const cplx<T>* Vt, cplx<T>* Vtr,
                                          cplx<T>* Sc, double alpha, double* partials, cudaStream_t st,
                                          const double* alpha_dev = nullptr);
// two-level preconditioner (Sec. 2.3.3): c the fine context, cc its half-resolution context
template <class T>
claire_status tl_restrict(claire_ctx* c, claire_ctx* cc, const cplx<T>* R, cplx<T>* F, cplx<T>* P, cplx<T>* X,
                          int ncomp, bool split, double* partials, cudaStream_t st);
template <class T> claire_status tl_scale(claire_ctx* cc, const cplx<T>* P, cplx<T>* U, cudaStream_t st);
template <class T>
claire_status tl_apply(claire_ctx* cc, const cplx<T>* P, const cplx<T>* Bt, cplx<T>* HP, double* partials,
                       cudaStream_t st);
template <class T>
claire_status tl_update(claire_ctx* cc, cplx<T>* X, cplx<T>* Rr, const cplx<T>* P, const cplx<T>* HP, double alpha,
                        double* partials, cudaStream_t st);
template <class T> claire_status tl_dir2(claire_ctx* cc, const cplx<T>* Rr, cplx<T>* P, double mu, cudaStream_t st);
template <class T>
claire_status tl_prolong(claire_ctx* c, claire_ctx* cc, const cplx<T>* R, const cplx<T>* X, cplx<T>* Z,
                         double* partials, cudaStream_t st);
template <class T>
claire_status tl_dir(claire_ctx* c, const cplx<T>* Z, cplx<T>* S, double mu, double* partials, cudaStream_t st);
template <class T> claire_status sp_copy_reg(claire_ctx* c, const cplx<T>* V, cplx<T>* Sc, double* partials,
                                             cudaStream_t st);

// ---- sl.cu ----------------------------------------------------------------------------------------------------
template <class T> claire_status sl_hadamard(claire_ctx* c, const T* a, const T* x, T* y, cudaStream_t st);
template <class T> claire_status sl_departure(claire_ctx* c, const T* v, int dir, T* disp, cudaStream_t st);
// H >= 0: brick-tiled gathers for displacements bounded by H - 1 voxels; H < 0: plain global gathers
template <class T> claire_status sl_init(claire_ctx* c);
template <class T> claire_status sl_interp(claire_ctx* c, const T* f, const T* disp, T* out, cudaStream_t st,
                                           int H = -1);
// lam = mR - m1; optionally rl = rho*lam; b = w * lam * gm  (terminal condition of the adjoint, Eq. (4))
// gm arguments point to a gradient history slice of type T, or BF16 when g16 (FP32 only)
template <class T> claire_status sl_adjoint_terminal(claire_ctx* c, const T* mR, const T* m1, const T* rho, T* lam,
                                                     T* rl, T* b, const void* gmj, bool g16, T w, cudaStream_t st);
// one backward continuity step along Y; rho/rl_next: div source (or null); lam/rl: stores (or null);
// b: accumulation b += w lam grad m (or null)
// with sdot (and lam == null, b != null): also part[block] = partial <sdot, b_final>, one slot per block of launch3
template <class T> claire_status sl_adjoint_step(claire_ctx* c, const T* lam_next, const T* rl_next, const T* rho,
                                                 const T* dY, T* lam, T* rl, T* b, const void* gmj, bool g16, T w,
                                                 cudaStream_t st, const T* sdot = nullptr, double* part = nullptr,
                                                 int H = -1);
// ---- sl_tma.cu: the accumulating adjoint step with TMA-staged operands (FP32, brick halo 2..5, no div source;
// its operands must be the context's own Y, gradient history, b and s) ----
bool sl_tma_prepare(claire_ctx* c);
// sv (optional): also part[block] = partial <sv, b_final> (the fused product of PCG's <s, H s>)
claire_status sl_adjoint_step_tma(claire_ctx* c, const float* lam_next, float* lam, int j, float w,
                                  const float* sv, double* part, int H, cudaStream_t st);
// the incremental state step with TMA-staged operands (FP32, brick halo 2..5, no div source; X, vt = s, the
// gradient history and b must be the context's own arrays)
claire_status sl_incstate_step_tma(claire_ctx* c, const float* q, float* qout, int j, bool last, float hdt, float w,
                                   int H, cudaStream_t st);
// CLAIRE_ETIMEOUT (and clears the flag) if a staged step's bounded wait ran out since the last call
claire_status sl_tma_take_error(claire_ctx* c);
// launch shape of the gather kernels: 256 threads, x along i3 (up to 64 wide), y along i2, z = i1
struct Launch3 {
  dim3 grid, block;
};
Launch3 launch3(const Dims& d);
// q^0 = -(dt/2) vt . grad m^0
template <class T> claire_status sl_incstate_init(claire_ctx* c, const T* vt, const void* gm0, bool g16, T* q,
                                                  cudaStream_t st);
// m~^{j+1} = q^j(X) + dt/2 f^{j+1}; writes q^{j+1}, or on the last step lam~ = -m~, rho*lam~, b = w lam~ grad m
template <class T> claire_status sl_incstate_step(claire_ctx* c, const T* q, const T* dX, const T* vt,
                                                  const void* gmj1, bool g16, T* qout, bool last, const T* rho, T* rl,
                                                  T* b, T w, cudaStream_t st, int H = -1);

// ---- blas.cu --------------------------------------------------------------------------------------------------
// partials[kReduceBlocks] of sum a*b (FP64 accumulation); a == b allowed
template <class T> claire_status dot_partial(claire_ctx* c, const T* a, const T* b, long long n, double* partials,
                                             cudaStream_t st);
// partials[kReduceBlocks] of max |a_i| (as double)
template <class T> claire_status absmax_partial(claire_ctx* c, const T* a, long long n, double* partials,
                                                cudaStream_t st);
// partials[kReduceBlocks] of the number of non-finite values in a[0..na) and b[0..nb)
template <class T> claire_status nonfinite_partial(claire_ctx* c, const T* a, long long na, const T* b, long long nb,
                                                   double* partials, cudaStream_t st);
// out = max(partials[0..np))
claire_status max_final(claire_ctx* c, const double* partials, int np, double* out, cudaStream_t st);
// partials of sum (a - b)^2
template <class T> claire_status diffsq_partial(claire_ctx* c, const T* a, const T* b, long long n, double* partials,
                                                cudaStream_t st);
// out[slot] = scale * sum(partials[0..kReduceBlocks))
claire_status reduce_final(claire_ctx* c, const double* partials, double scale, double* out, cudaStream_t st);
// y = x rounded to BF16 (round to nearest even)
claire_status to_bf16(claire_ctx* c, const float* x, void* y, long long n, cudaStream_t st);
// y = a*x + y
template <class T> claire_status axpy(claire_ctx* c, long long n, double a, const T* x, T* y, cudaStream_t st);
// y = x + a*y
template <class T> claire_status xpay(claire_ctx* c, long long n, const T* x, double a, T* y, cudaStream_t st);
// z = x + a*y
template <class T> claire_status waxpy(claire_ctx* c, long long n, const T* x, double a, const T* y, T* z,
                                       cudaStream_t st);
template <class T> claire_status scale_copy(claire_ctx* c, long long n, double a, const T* x, T* y, cudaStream_t st);
// y = 0 (n values of T)
template <class T> claire_status zero_fill(claire_ctx* c, long long n, T* y, cudaStream_t st);
// out[v] = scale * sum(partials[v * np .. v * np + np)) for v < nv
claire_status reduce_final_v(claire_ctx* c, const double* partials, int nv, int np, double scale, double* out,
                             cudaStream_t st);
}  // namespace claire
