/*
 * claire.h -- C-ABI of the GB300 (sm_103a) hot path of the reduced-space Gauss--Newton--Krylov solver for
 * stationary-velocity diffeomorphic image registration (Mang, Gholami, Davatzikos, Biros, "CLAIRE",
 * arXiv 1808.04487).
 *
 * Problem (Sec. 2.1, Eq. (2)): find a stationary velocity v on the periodic box [0, 2*pi)^3 minimising
 *     J(v) = 1/2 <m_1 - m_R, m_1 - m_R> + beta/2 sum_c <v_c, A v_c>,
 * where m_1 = m(t = 1) and m solves the transport equation d_t m + grad m . v = 0, m(0) = m_T, optionally with
 * div v = 0 (Leray projection K, Sec. 2.2). The calls below evaluate the transport solves (Eq. (2), (4)), the
 * reduced gradient (Eq. (5)), the Gauss--Newton Hessian matvec (Eq. (7)-(9), Sec. 2.3.2), the spectral
 * preconditioner (Sec. 2.3.3) and the full inexact GN--Krylov solve (Alg. 1, Alg. 2).
 *
 * Conventions shared by every call
 * --------------------------------
 * Grid        n = (n1, n2, n3), every n_a even and >= 4; node x = (2 pi i1/n1, 2 pi i2/n2, 2 pi i3/n3).
 * Scalars     C-ordered [n1][n2][n3] arrays, i3 fastest (N = n1*n2*n3 values).
 * Vectors     planar [3][n1][n2][n3] arrays; component c points along axis c (3N values).
 * Precision   the _f32 calls take float arrays and the _f64 calls double arrays; a context is created for one
 *             precision (claire_opts.precision) and rejects calls of the other with CLAIRE_EINVAL.
 *             Reductions (objective, inner products, norms, PCG scalars, Armijo test) accumulate in FP64.
 * Memory      unless a call says otherwise, every array argument is a DEVICE pointer (cudaMalloc'd or from a
 *             framework allocator) on the current device, owned by the caller; the library never frees or keeps
 *             caller memory beyond the call. The context owns its own workspace (allocated by claire_create).
 * Streams     calls enqueue work on the caller's cudaStream_t (passed as void*; NULL = legacy default stream)
 *             and return without synchronising, except where a host scalar or report is returned: those calls
 *             synchronise that stream before returning.
 * Errors      no exception crosses the ABI; every call returns a claire_status. On failure the context keeps a
 *             message readable with claire_last_error(). claire_register_* scans m_T, m_R and the initial v on the
 *             device and returns CLAIRE_ENAN if any value is NaN or infinite (nothing else runs, v is unchanged);
 *             a non-finite objective, gradient norm or PCG scalar during the solve also returns CLAIRE_ENAN. The
 *             operator calls (transport, gradient, matvec, ...) do not scan their inputs.
 * Faults      for tests of the failure paths only, the environment variable CLAIRE_FAULT (a comma-separated list)
 *             fakes a failure on the host where the library reads a device result: "pcg_breakdown" makes the
 *             first <s, H s> of every PCG solve read as non-positive (the host-driven loop then runs),
 *             "nn_timeout" makes claire_nn_status report an expired tensor-core wait. Unset in normal use.
 * Threads     a context is not thread safe; use one context per host thread (or serialise calls).
 * Discrete    inner product <a, b> = h1 h2 h3 sum a*b; forward FFT unnormalised, inverse scaled by 1/N;
 * readings    first-order spectral symbols use k' (Nyquist set to 0), even-order symbols the full k; RK2 (Heun)
 *             characteristics; tricubic Lagrange interpolation on the 4^3 stencil b-1..b+2 around b = floor(xi)
 *             with periodic wrap; trapezoidal time quadrature on n_t + 1 nodes.
 */
#ifndef CLAIRE_GB300_H
#define CLAIRE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CLAIRE_OK = 0,
    CLAIRE_EINVAL = 1,       /* bad argument: null pointer, odd or < 4 grid size, nt < 1, beta <= 0, wrong dtype */
    CLAIRE_ENOMEM = 2,       /* device or host allocation failed in claire_create */
    CLAIRE_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed; see claire_last_error */
    CLAIRE_ENAN = 4,         /* a non-finite objective, gradient norm or PCG scalar was produced */
    CLAIRE_ENOTCONV = 5,     /* register: max_gn Gauss-Newton iterations reached; v holds the last iterate */
    CLAIRE_ELINESEARCH = 6,  /* register: Armijo failed after max_ls trials; v holds the last accepted iterate */
    CLAIRE_EBREAKDOWN = 7,   /* PCG: <s, H s> <= 0 (counted in claire_report.pcg_breakdowns; the solve continues,
                                no call returns this status) */
    CLAIRE_ETIMEOUT = 8      /* a bounded device wait expired (the warm-start network's tensor-core waits, about
                                a second each); the kernel released its resources and the context stays usable */
} claire_status;

typedef enum { CLAIRE_F32 = 0, CLAIRE_F64 = 1 } claire_precision;

/* Solver parameters (Sec. 2.3.2, Table 2). claire_default_opts fills the paper's defaults. */
typedef struct {
    int n[3];            /* grid size n1, n2, n3 (even, >= 4) */
    int precision;       /* claire_precision */
    double beta;         /* regularisation weight beta_v > 0 */
    int nt;              /* number of semi-Lagrangian time steps (default 4, Sec. 2.3.1) */
    int regnorm;         /* 1: H1 seminorm, A = -Laplacian; 2: H2 seminorm, A = Laplacian^2 (Sec. 2.1) */
    int divfree;         /* 0: K = I (or the H1-div K, see beta_w); 1: div v = 0 via the Leray projection
                            K = I - grad Lap^-1 div (Sec. 2.2) */
    double gtol_rel;     /* eps_g: stop when ||g_k|| <= eps_g ||g(v=0)|| (default 5e-2, Sec. 2.3.2) */
    double gtol_abs;     /* stop when ||g_k|| <= gtol_abs (default 1e-6, Sec. 2.3.2) */
    int max_gn;          /* Gauss-Newton iteration cap (default 50, Sec. 4.4) */
    int max_krylov;      /* PCG iteration cap per GN step (default 100, Sec. 4.4) */
    double pcg_rtol;     /* > 0: fixed relative PCG tolerance; <= 0: eps_H = min(0.5, sqrt(||g_k||/||g_0||)) (Alg. 2) */
    int max_ls;          /* Armijo trials (default 10); alpha starts at 1 and is halved */
    double armijo_c1;    /* sufficient-decrease constant (default 1e-4) */
    int bf16_mask;       /* reduced-precision storage (FP32 contexts only; default 0): bit 0 stores the spectral
                            gradients of the state history, grad m^j, in BF16 (read by every incremental state and
                            adjoint step; arithmetic stays FP32, reductions FP64). The error this adds is measured,
                            not bounded by the FP32 tolerance. */
    double beta_w;       /* > 0: the H1-div model (Sec. 2.1-2.2): regnorm 1 plus the penalty beta_w/2 ||div v||^2_H1
                            (w = div v in Eq. (2)), K = I - grad (beta_v (beta_w (-Lap + I))^-1 + I)^-1 Lap^-1 div in
                            Eq. (5) and (7); requires regnorm = 1 and divfree = 0. 0 (default): off. PCG and the
                            Armijo slope use the <K^-1 a, b> products in which beta_v A + K H_data is self-adjoint;
                            the stopping test uses ||g|| of Eq. (5). */
    int precond;         /* 0 (default): spectral preconditioner (beta A)^-1; 1: two-level preconditioner (Sec. 2.3.3)
                            on the half-resolution grid (n_a divisible by 4, n_a >= 8): the low modes of
                            R^-1/2 r, R = beta A, are replaced by a nested CG solution of the coarse split system
                            I + R^-1/2 H_data R^-1/2 (direct coarse discretisation, spectral transfer), the high
                            modes are kept */
    double pc_kappa;     /* nested tolerance eps_M = pc_kappa eps_H of the two-level preconditioner (default 0.1) */
} claire_opts;

/* What claire_register reports (the quantities of Table 3 plus timing). Host struct, filled on return. */
typedef struct {
    int gn_iters;        /* Gauss-Newton iterations taken */
    int matvecs;         /* Hessian matvecs (each = one incremental state + one incremental adjoint solve) */
    int pde_solves;      /* transport solves: gradient 2 (+1 per accepted step), matvec 2, line-search trial 1 */
    int ls_trials;       /* objective evaluations in the Armijo search */
    int pcg_breakdowns;  /* PCG iterations stopped by <s, H s> <= 0 */
    int converged;       /* 1 if a gradient tolerance was met */
    double J0, J;        /* objective at the initial guess and at the returned v */
    double mismatch0;    /* 1/2 ||m_T - m_R||^2 (v = 0) */
    double mismatch;     /* 1/2 ||m_1 - m_R||^2 at the returned v */
    double gnorm0;       /* ||g(v = 0)||, the reference of the relative stopping test */
    double gnorm;        /* ||g|| at the returned v */
    double ms_total;     /* wall time of the call on the stream, milliseconds (CUDA events) */
    int coarse_matvecs;  /* matvecs of the nested solver on the half-resolution grid (two-level preconditioner) */
} claire_report;

typedef struct claire_ctx claire_ctx;

/* Fill *opts with the paper's defaults for grid n (beta = 1e-2, nt = 4, H1, no constraint, eps_g = 5e-2, ...). */
claire_status claire_default_opts(claire_opts* opts, int n1, int n2, int n3, int precision);

/* Validate *opts, build FFT plans (twiddle tables computed on the host in FP64) and allocate the context's
 * device workspace for grid opts->n. The context keeps a copy of *opts. Returns CLAIRE_EINVAL for bad options,
 * CLAIRE_ENOMEM / CLAIRE_ECUDA on allocation failure (then *out is NULL). Uses the current CUDA device. */
claire_status claire_create(const claire_opts* opts, claire_ctx** out);
/* (FP32 contexts also time the tile variants of the FFT passes on their grid once per process; see
 * claire_counters.fft_tile.) */

/* Free the context and its workspace (synchronises the device first). NULL is accepted. */
claire_status claire_destroy(claire_ctx* ctx);

/* Message of the last failure on ctx ("" if none). The pointer stays valid until the next call on ctx. */
const char* claire_last_error(const claire_ctx* ctx);

/* Bytes of device workspace the context holds (with the two-level preconditioner: including its coarse context). */
size_t claire_workspace_bytes(const claire_ctx* ctx);

/* ---- transport (Eq. (2) state, Eq. (4) continuity-form adjoint; Sec. 2.3.1 semi-Lagrangian RK2) ----------------
 * dir = +1: m1 = m(t=1) of d_t m + grad m . v = 0 with m(0) = m0 (state equation, n_t steps forward).
 * dir = -1: m1 = lambda(t=0) of -d_t lambda - div(lambda v) = 0 with lambda(1) = m0 (adjoint, n_t steps backward;
 *           the div v source is dropped when opts.divfree = 1). m0, m1: scalars; v: vector. m0 and m1 may alias. */
claire_status claire_transport_f32(claire_ctx* ctx, const float* m0, const float* v, int dir, float* m1, void* stream);
claire_status claire_transport_f64(claire_ctx* ctx, const double* m0, const double* v, int dir, double* m1, void* stream);

/* ---- reduced gradient (Eq. (5); Alg. 1 lines 2-5) ----------------------------------------------------------
 * Solves the state forward and the adjoint backward at v and writes g = beta A v + K[int_0^1 lambda grad m dt]
 * (vector). If J is not NULL the objective J(v) is written to *J (host double; the call then synchronises).
 * The linearisation at v (departure points, state history and its gradients) stays cached in the context for
 * claire_hessvec_cached_*. */
claire_status claire_gradient_f32(claire_ctx* ctx, const float* mT, const float* mR, const float* v, float* g,
                                  double* J, void* stream);
claire_status claire_gradient_f64(claire_ctx* ctx, const double* mT, const double* mR, const double* v, double* g,
                                  double* J, void* stream);

/* ---- Gauss-Newton Hessian matvec (Eq. (7) with Eq. (8), (9); lambda terms dropped, Sec. 2.3.2) --------------
 * Hvt = beta A vt + K[int_0^1 lambda~ grad m dt] at the linearisation point v. claire_hessvec_* re-linearises at
 * (mT, v) first (departure points, state solve, spectral gradients of the state history); mR is not used by the
 * Gauss-Newton approximation and may be NULL. vt and Hvt are vectors and must not alias. */
claire_status claire_hessvec_f32(claire_ctx* ctx, const float* mT, const float* mR, const float* v, const float* vt,
                                 float* Hvt, void* stream);
claire_status claire_hessvec_f64(claire_ctx* ctx, const double* mT, const double* mR, const double* v,
                                 const double* vt, double* Hvt, void* stream);
/* Same matvec at the linearisation cached by the last claire_gradient_* / claire_linearize_* / claire_hessvec_*
 * call on ctx (CLAIRE_EINVAL if there is none). This is the operator PCG applies (Alg. 2 lines 6-8). */
claire_status claire_hessvec_cached_f32(claire_ctx* ctx, const float* vt, float* Hvt, void* stream);
claire_status claire_hessvec_cached_f64(claire_ctx* ctx, const double* vt, double* Hvt, void* stream);
/* Data term of the matvec alone, out = K[int_0^1 lambda~ grad m dt] (H_data of Eq. (7)), at the cached
 * linearisation. With H_reg = beta A known in closed form this is what a caller composing its own Krylov solver or
 * a split-preconditioned system (Sec. 2.3.3) needs; claire_register's PCG uses it with beta A s carried by
 * recurrence. vt and out must not alias. */
claire_status claire_hessvec_data_f32(claire_ctx* ctx, const float* vt, float* out, void* stream);
claire_status claire_hessvec_data_f64(claire_ctx* ctx, const double* vt, double* out, void* stream);
/* Data term of the reduced gradient alone, out = K[int_0^1 lambda grad m dt] (Eq. (5) without beta A v), at
 * (mT, mR, v); the linearisation at v stays cached as after claire_gradient_*. If J is not NULL the objective J(v)
 * is written to *J (host double; the call then synchronises). With beta A v known in closed form (it is a Fourier
 * multiplier, see claire_symbol_*), this is the part of the gradient that the transport solves produce. */
claire_status claire_gradient_data_f32(claire_ctx* ctx, const float* mT, const float* mR, const float* v, float* out,
                                       double* J, void* stream);
claire_status claire_gradient_data_f64(claire_ctx* ctx, const double* mT, const double* mR, const double* v,
                                       double* out, double* J, void* stream);
/* Cache the linearisation at (mT, v) without computing anything else. */
claire_status claire_linearize_f32(claire_ctx* ctx, const float* mT, const float* v, void* stream);
claire_status claire_linearize_f64(claire_ctx* ctx, const double* mT, const double* v, void* stream);

/* ---- spectral preconditioner (Sec. 2.3.3 and its Remark) -----------------------------------------------------
 * z = (beta A)^-1 r in the Fourier domain, the zero eigenvalue of beta A (k = 0) replaced by 1. r, z: vectors;
 * they may alias. */
claire_status claire_precond_f32(claire_ctx* ctx, const float* r, float* z, void* stream);
claire_status claire_precond_f64(claire_ctx* ctx, const double* r, double* z, void* stream);

/* ---- full inexact Gauss-Newton-Krylov solve (Alg. 1 with Alg. 2, Armijo line search, Sec. 2.3.2) -------------
 * v is in/out: on entry the initial guess (zeros = the plain method), on return the solution. With div v = 0 a
 * nonzero guess is first Leray-projected (Sec. 2.2). The relative stopping test always uses ||g(v = 0)||
 * (Sec. 2.3.2), also for a nonzero initial guess. rep (host) may be NULL.
 * Returns CLAIRE_OK on convergence, CLAIRE_ENOTCONV when max_gn is reached (v = the last iterate, a valid
 * solution of lower accuracy), CLAIRE_ELINESEARCH when Armijo fails (v = the last accepted iterate), CLAIRE_ENAN
 * when m_T, m_R or the initial v hold a NaN or an infinity (checked on the device before anything else runs; v is
 * left unchanged) or the objective or gradient becomes non-finite. Synchronises stream. */
claire_status claire_register_f32(claire_ctx* ctx, const float* mT, const float* mR, float* v, claire_report* rep,
                                  void* stream);
claire_status claire_register_f64(claire_ctx* ctx, const double* mT, const double* mR, double* v,
                                  claire_report* rep, void* stream);
/* Same solve with HOST arrays (pageable or pinned): mT, mR and v are copied to the context's device buffers on
 * stream, the solve runs, and v is copied back before the call returns. The first host-array call on a context
 * allocates those device buffers (5 N values, kept until claire_destroy; CLAIRE_ENOMEM if that fails), so the
 * workspace of a context that only takes device arrays stays smaller. */
claire_status claire_register_host_f32(claire_ctx* ctx, const float* mT, const float* mR, float* v,
                                       claire_report* rep, void* stream);
claire_status claire_register_host_f64(claire_ctx* ctx, const double* mT, const double* mR, double* v,
                                       claire_report* rep, void* stream);

/* Parameter continuation in beta_v (Sec. 3.6: start at beta_v = 1 and reduce it until the target is reached).
 * Levels beta_start, beta_start*factor, beta_start*factor^2, ... while above the context's beta (the target), then
 * the target itself, at most max_levels in all; every level is a claire_register solve warm-started from the
 * previous level's v (with its own ||g(v = 0)|| in the relative test). v is in/out as for claire_register. reps
 * (host, max_levels entries, may be NULL) receives one report per level, *nlevels (host, may be NULL) the number
 * of levels run. Stops early on a status other than OK / ENOTCONV and returns the last level's status. The
 * context's beta is restored before returning. 0 < factor < 1, beta_start > 0, else CLAIRE_EINVAL. */
claire_status claire_register_continuation_f32(claire_ctx* ctx, const float* mT, const float* mR, float* v,
                                               double beta_start, double factor, claire_report* reps,
                                               int max_levels, int* nlevels, void* stream);
claire_status claire_register_continuation_f64(claire_ctx* ctx, const double* mT, const double* mR, double* v,
                                               double beta_start, double factor, claire_report* reps,
                                               int max_levels, int* nlevels, void* stream);
/* Changes the regularisation weight beta_v of a context (beta > 0); nothing else is invalidated. */
claire_status claire_set_beta(claire_ctx* ctx, double beta);

/* ---- batched registration of many independent pairs (population-to-atlas) ------------------------------------
 * Solves every pair with claire_register_f32's algorithm (Alg. 1 with Alg. 2); pairs may have different grids. mT,
 * mR, v are DEVICE arrays of the pair's grid on the current device; v is in/out (zeros = the plain method). By
 * default every zero-start solve is driven from the device: the pairs are grouped by grid, each group is split over
 * up to nworkers (>= 1) contexts (created from *base with n replaced by the group's grid, freed before the call
 * returns), each context's share becomes one branch of a single CUDA graph -- a WHILE over its pairs around the
 * Gauss-Newton WHILE, the PCG WHILE and the Armijo WHILE as conditional nodes, every decision taken on the device --
 * and the whole batch runs as ONE graph launch whose branches overlap on the GPU. Results are bit-identical to the
 * single-pair solves. A pair with a nonzero v, and every pair when base->precond != 0 or CLAIRE_GN=host, is solved by
 * the host-driven loop (CLAIRE_GN=host: nworkers host threads, one stream and one context per grid each, pairs taken
 * largest grid first). CLAIRE_BATCH_GRAPH=lanes launches one graph per context instead of one for the batch; so does
 * the call if the single graph cannot be built. Per-pair results land in rep and status; the call returns CLAIRE_OK
 * when every pair ran (statuses CLAIRE_OK / ENOTCONV / ELINESEARCH), else the first failing status. Synchronises the
 * device. */
typedef struct {
    int n[3];
    const float* mT;
    const float* mR;
    float* v;
    claire_report rep;
    int status;
} claire_pair_f32;
claire_status claire_register_batch_f32(const claire_opts* base, claire_pair_f32* pairs, int npairs, int nworkers);
/* Graph launches made by the most recent claire_register_batch_f32 call of this process: 1 when the batch ran as one
 * graph, one per context on the per-context path, 0 when every pair took the host-driven loop. */
long long claire_last_batch_graph_launches(void);

/* ---- building blocks exposed for testing and for callers composing their own solver --------------------------
 * claire_departure_*: RK2 departure points of one time step (dt = 1/nt) in grid units, disp = (X - x) / h per
 *   axis (dir = +1: state characteristics X of v; dir = -1: adjoint characteristics Y of -v). v, disp: vectors.
 * claire_interp_*: out(x) = tricubic Lagrange interpolant of f at x + disp(x) (grid units, periodic).
 * claire_spectral_*: op = 0 gradient (scalar in, vector out), 1 divergence (vector in, scalar out),
 *   2 Leray projection K (vector -> vector), 3 A = regnorm operator (vector -> vector), 4 Laplacian
 *   (scalar -> scalar). in and out must not alias.
 * claire_objective_*: *J = 1/2 <m1 - mR, m1 - mR> + beta/2 sum_c <v_c, A v_c> (host double; synchronises).
 * claire_dot_*: *out = <a, b> = h1 h2 h3 sum a*b over count values, accumulated in FP64 (host double;
 *   synchronises). */
claire_status claire_departure_f32(claire_ctx* ctx, const float* v, int dir, float* disp, void* stream);
claire_status claire_departure_f64(claire_ctx* ctx, const double* v, int dir, double* disp, void* stream);
claire_status claire_interp_f32(claire_ctx* ctx, const float* f, const float* disp, float* out, void* stream);
claire_status claire_interp_f64(claire_ctx* ctx, const double* f, const double* disp, double* out, void* stream);
claire_status claire_spectral_f32(claire_ctx* ctx, int op, const float* in, float* out, void* stream);
claire_status claire_spectral_f64(claire_ctx* ctx, int op, const double* in, double* out, void* stream);
claire_status claire_objective_f32(claire_ctx* ctx, const float* m1, const float* mR, const float* v, double* J,
                                   void* stream);
claire_status claire_objective_f64(claire_ctx* ctx, const double* m1, const double* mR, const double* v, double* J,
                                   void* stream);
claire_status claire_dot_f32(claire_ctx* ctx, const float* a, const float* b, long long count, double* out,
                             void* stream);
claire_status claire_dot_f64(claire_ctx* ctx, const double* a, const double* b, long long count, double* out,
                             void* stream);

/* A diagonal Fourier symbol of the method applied to ncomp (1..3) half spectra (layout of claire_fft_*, component
 * stride n1*n2*(n3/2+1) complex values; in and out may alias): op 0: out = beta a(k) in, the regularisation
 * operator beta A of Eq. (2) (a = |k|^2 for H1, |k|^4 for H2, full k); op 1: out = M^-1 in, the spectral
 * preconditioner (beta A)^-1 with the zero eigenvalue replaced by 1 (Sec. 2.3.3); op 2 (ncomp = 3): out = K in,
 * the context's K of Eq. (5) (identity, the Leray projection of Sec. 2.2, or the H1-div operator). These are the
 * exact diagonal multiplies the solver applies to its Fourier-domain vectors. Bad op/ncomp: CLAIRE_EINVAL. */
claire_status claire_symbol_f32(claire_ctx* ctx, int op, const float* in, float* out, int ncomp, void* stream);
claire_status claire_symbol_f64(claire_ctx* ctx, int op, const double* in, double* out, int ncomp, void* stream);

/* Unnormalised forward 3D real FFT of a scalar (Sec. 2.3.1): spec is the half spectrum [n1][n2][n3/2+1] of
 * interleaved (re, im) pairs, i.e. 2*n1*n2*(n3/2+1) values. claire_ifft_* is the inverse, scaled by 1/N; it
 * reads spec as a Hermitian half spectrum and does not modify it. */
claire_status claire_fft_f32(claire_ctx* ctx, const float* f, float* spec, void* stream);
claire_status claire_fft_f64(claire_ctx* ctx, const double* f, double* spec, void* stream);
claire_status claire_ifft_f32(claire_ctx* ctx, const float* spec, float* f, void* stream);
claire_status claire_ifft_f64(claire_ctx* ctx, const double* spec, double* f, void* stream);

/* Kernel launches the library has made on this context (and its coarse context) since claire_create, and the
 * gather schedule of the cached linearisation: the brick halo (voxels) of the shared-memory tiled gathers along X
 * (state, incremental state) and Y (adjoints), or -1 where the plain gathers run. Chosen per grid by timing both
 * once, separately for the light kernels (halo_x, halo_y: incremental state steps, store/accumulate adjoint steps,
 * state interpolation) and the heavy ones (halo_x_heavy, halo_y_heavy: last incremental step, adjoint steps with
 * the fused inner product or the div v source); the environment variable CLAIRE_GATHER=plain or =tiled overrides
 * the choice. With the spectral preconditioner and per-kernel profiling off, each PCG solve runs as one CUDA graph
 * whose conditional WHILE node repeats one iteration with its scalars computed on the device (bit-identical to the
 * host-driven loop, which CLAIRE_PCG=host forces). */
typedef struct {
    long long launches;
    int halo_x, halo_y;
    int halo_x_heavy, halo_y_heavy;
    long long pcg_graph_runs; /* PCG solves (Alg. 2) run as one CUDA-graph launch, the loop driven on the device */
    long long gn_graph_runs;  /* launches of the graph of the whole solve driven from the device (batched calls, or
                                 CLAIRE_GN=device for single zero-start solves) */
    long long tma_steps;      /* accumulating adjoint steps whose streamed operands (Y, grad m^j, b) were staged
                                 in shared memory by TMA (FP32, brick-tiled schedule, n3 a multiple of 16; the
                                 environment variable CLAIRE_TMA=0 turns this off) */
    int fft_tile[3];          /* tile variant of the length-specialised FFT passes chosen by the autotuner at
                                 claire_create (FP32) for the contiguous (z), y and x passes: 0 the default lines or
                                 columns per CTA, 1 half as many, 2 twice as many (CLAIRE_FFT_TILES=default keeps 0; CLAIRE_FFT_TILES=z,y,x forces
                                 the three; a variant that does not fit a length runs as 0); a variant changes
                                 no result bit */
} claire_counters;
claire_status claire_get_counters(const claire_ctx* ctx, claire_counters* out);

/* Inner product that allocates nothing (the paper has no counterpart; this is a service for callers).
 * *out (a DEVICE pointer to one double, written on `stream`) = scale * sum_i a[i] * b[i] over `count` floats. It
 * runs the reduction kernels of claire_dot_f32 -- per-thread float-float (FP64-class) accumulation, FP64 block
 * and final sums -- but on a grid of ceil(count / 2048) blocks instead of that call's fixed grid, so the summation
 * order differs and the result equals claire_dot_f32's up to rounding, not bitwise (pass scale = h1 h2 h3 to get
 * that call's <a, b>). No context is needed, and the call makes no cudaMalloc/cudaFree and calls no allocating
 * library: it is meant for callers that must not allocate device memory, e.g. code running inside a fixed
 * memory budget or a framework allocator that owns the device, or a loop that cannot afford cudaMalloc's implicit
 * device synchronisation. Its partial sums live in a file-scope device array of 65536 doubles (512 KiB) that every
 * GPU which loads this library keeps until the process exits, so count is limited to 65536 * 2048 = 134217728
 * values (larger counts return CLAIRE_EINVAL, as do null pointers and count < 0; a CUDA launch error returns
 * CLAIRE_ECUDA). The array is shared by every call in the process: calls whose kernels overlap on the GPU (two
 * streams, or two host threads) race on it and must be serialised by the caller; nothing in it needs clearing
 * between calls. The first call on each device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current and keeps it; make that first call before any stream capture, and do not use the call
 * across a reset of the device (cudaDeviceReset), which invalidates the kept address. */
claire_status claire_dot_noalloc_f32(const float* a, const float* b, long long count, double scale, double* out,
                                     void* stream);

/* Per-kernel timing (not part of the method; for measurement). While enabled, every kernel launch on ctx is
 * bracketed by a pair of CUDA events on its stream. claire_profile_report synchronises the device, writes a JSON
 * object {"kernel name": [launches, total_ms], ...} of everything recorded since the last report into buf
 * (truncated to len bytes, NUL-terminated), and clears the records. Enabling adds two event records per launch. */
claire_status claire_profile_enable(claire_ctx* ctx, int on);
claire_status claire_profile_report(claire_ctx* ctx, char* buf, size_t len);

/* ============================================================================================================
 * Spectral resampling and the learned warm start. Neither is part of the paper's method: the network only
 * proposes the initial guess v_0 of Alg. 1, and the solve that follows is the unchanged Gauss-Newton-Krylov
 * method with ||g(v = 0)|| in its relative stopping test (Sec. 2.3.2). All pointers below are device pointers
 * unless marked (host); calls are asynchronous on `stream` unless they return a host value.
 * ============================================================================================================ */

/* g = f resampled from src's grid to dst's grid by truncating or zero-padding its Fourier series: a mode with
 * signed wavenumber w is kept iff 2|w_i| < n_i on both grids for every axis (Nyquist modes are dropped), so a
 * trigonometric polynomial of degree below half of both grids is reproduced exactly. f is [ncomp][N_src], g is
 * [ncomp][N_dst] (planar). kmax > 0 also drops every mode with some |w_i| > kmax (a spectral low-pass; 0: none).
 * project = 1 (ncomp = 3 only) applies the Leray projection of Sec. 2.2 on dst's grid.
 * Both contexts must be FP32; their internal work arrays are used (no other call on either context meanwhile;
 * src == dst is allowed). */
claire_status claire_resample_f32(claire_ctx* src, claire_ctx* dst, const float* f, float* g, int ncomp, int project,
                                  int kmax, void* stream);

/* Warm-start network: a 3D encoder-decoder with four levels (16, 32, 64, 128 channels; two periodic 3x3x3
 * convolutions + ReLU per level, 2x2x2 average pooling, nearest-neighbour upsampling, additive skips; a linear
 * 16-channel head of which channels 0..2 are the velocity, scaled by vscale). It runs on a coarse network grid
 * n (each n_i a multiple of 8, (n1/8)(n2/8)(n3/8) a multiple of 16) for up to `batch` samples at a time. BF16
 * weights and activations, FP32 accumulation on the tensor cores, FP32 master weights, gradients and Adam state.
 * The handle owns its device memory and an FP32 claire_ctx on the network grid; it is not thread-safe. */
typedef struct claire_ws claire_ws;
claire_status claire_ws_create(int batch, int n1, int n2, int n3, float vscale, unsigned long long seed,
                               claire_ws** out);
claire_status claire_ws_destroy(claire_ws* ws);
const char* claire_ws_last_error(const claire_ws* ws);
/* Parameters in host order: for each layer, weights [Cout][27][Cin] (offset 9(o1+1)+3(o2+1)+(o3+1) for the
 * neighbour at (i1+o1, i2+o2, i3+o3)) then bias [Cout]. */
long long claire_ws_num_params(const claire_ws* ws);
int claire_ws_num_layers(const claire_ws* ws);
/* info[8] (host) = {Cin used, Cin stored, Cout, level, relu, input tensor, output tensor (-1: prediction),
 * skip tensor (-1: none)} */
claire_status claire_ws_layer(const claire_ws* ws, int i, int* info);
int claire_ws_num_ops(const claire_ws* ws);
/* info[4] (host) = {kind (0 conv, 1 pool, 2 upsample), layer (conv only), input tensor, output tensor} */
claire_status claire_ws_op(const claire_ws* ws, int i, int* info);
/* host copies (synchronise the device); set_params also resets the Adam state */
claire_status claire_ws_get_params(claire_ws* ws, float* host_params);
claire_status claire_ws_set_params(claire_ws* ws, const float* host_params);
claire_status claire_ws_get_grads(claire_ws* ws, float* host_grads);
/* Samples are rows of images [S][2][N] (m_T, m_R; planar on the network grid) and targets [S][3][N] (v); idx
 * (host, nb entries) selects rows, NULL means rows 0..nb-1; nb <= batch. v_out is [nb][3][N] (planar, physical
 * units). The loss is the mean squared error of vscale v over all voxels and 3 components; with backward = 1
 * the parameter gradients are formed (claire_ws_get_grads). loss (host, optional) synchronises the stream. */
claire_status claire_ws_forward_f32(claire_ws* ws, const float* images, const int* idx, int nb, float* v_out,
                                    void* stream);
claire_status claire_ws_loss_f32(claire_ws* ws, const float* images, const float* targets, const int* idx, int nb,
                                 int backward, double* loss, void* stream);
/* one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the current gradients */
claire_status claire_ws_adam_step(claire_ws* ws, float lr, void* stream);
/* loss + gradients + Adam step; loss (host, optional) is the loss before the step */
claire_status claire_ws_train_step_f32(claire_ws* ws, const float* images, const float* targets, const int* idx,
                                       int nb, float lr, double* loss, void* stream);
/* v = the network's velocity for (mT, mR) on ctx's grid: both images resampled to the network grid, one forward
 * pass, the prediction resampled back with modes |w_i| <= kmax (kmax <= 0: all the network grid holds), and
 * Leray-projected when ctx imposes div v = 0. ctx must be FP32. v can be passed as the initial guess of
 * claire_register_f32. */
claire_status claire_ws_predict_f32(claire_ws* ws, claire_ctx* ctx, const float* mT, const float* mR, float* v,
                                    int kmax, void* stream);

/* The network's layers one by one (used to check each against a reference). BF16 tensors are passed as void*,
 * channels-last [B][n1][n2][n3][C]; C, Cin, Cout multiples of 16 in [16, 128]; B n1 n2 n3 a multiple of 16. The
 * convolutions read and write 16-byte vectors: x, w, skip, y, yf, work of conv3_fwd and dz, x of conv3_wgrad must be
 * 16-byte aligned (CLAIRE_EINVAL otherwise); the other layers take any alignment of their element type.
 * conv3_fwd: y (BF16) and/or yf (FP32; overwritten, or added to with accum = 1) = act(conv(x, w) + bias + skip),
 * w [Cout][27][Cin]; bias, skip, y, yf optional (y or yf required); work optional (see below). conv3_wgrad: dw[Cout][27][Cin] =
 * sum over voxels of dz[m][co] x[nb(m, off)][ci] (work: claire_nn_wgrad_workspace_bytes). weight_flip: wt =
 * the weights of the adjoint convolution, [Cin][27][Cout]. relu_bwd: dz = dy where y > 0 (y NULL: everywhere),
 * FP32 dz and BF16 dzb. bias_grad: db[c] = sum_m dz[m][c] (work: claire_nn_bias_workspace_bytes). pool: 2x2x2
 * average over the fine grid (n1, n2, n3 even) and its adjoint; up: nearest-neighbour x2 from the coarse grid
 * (n1, n2, n3) and its adjoint (accum = 1 adds to dx); for both, the fine grid's B n1 n2 n3 C values must stay below
 * 2^31 (CLAIRE_EINVAL otherwise). mse: loss partials (FP64, npartials blocks) of the mean
 * squared error over the first cu of C channels, grad (optional) = d loss / d pred. adam: one bias-corrected Adam
 * step number `step` >= 1; pb (optional) receives a BF16 copy of p. */
claire_status claire_nn_conv3_fwd(const void* x, const void* w, const float* bias, const void* skip, void* y,
                                  float* yf, int accum, int B, int n1, int n2, int n3, int Cin, int Cout, int relu,
                                  float* work, void* stream);
/* work of claire_nn_conv3_fwd (device, may be NULL): grids with fewer 128-voxel tiles than about two per SM split
 * the 27 neighbour offsets over CTAs and reduce the FP32 partial sums in a fixed order; 0 bytes when not needed */
size_t claire_nn_fwd_workspace_bytes(int B, int n1, int n2, int n3, int Cout);
size_t claire_nn_wgrad_workspace_bytes(int B, int n1, int n2, int n3, int Cin, int Cout);
claire_status claire_nn_conv3_wgrad(const void* dz, const void* x, float* dw, float* work, int B, int n1, int n2,
                                    int n3, int Cin, int Cout, void* stream);
claire_status claire_nn_weight_flip(const void* w, void* wt, int Cin, int Cout, void* stream);
claire_status claire_nn_relu_bwd(const float* dy, const void* y, float* dz, void* dzb, long long count,
                                 void* stream);
size_t claire_nn_bias_workspace_bytes(int C);
claire_status claire_nn_bias_grad(const float* dz, long long M, int C, float* db, float* work, void* stream);
claire_status claire_nn_pool_fwd(const void* x, void* y, int B, int n1, int n2, int n3, int C, void* stream);
claire_status claire_nn_pool_bwd(const float* dy, float* dx, int accum, int B, int n1, int n2, int n3, int C,
                                 void* stream);
claire_status claire_nn_up_fwd(const void* x, void* y, int B, int n1, int n2, int n3, int C, void* stream);
claire_status claire_nn_up_bwd(const float* dy, float* dx, int accum, int B, int n1, int n2, int n3, int C,
                               void* stream);
claire_status claire_nn_mse(const float* pred, const float* target, float* grad, long long M, int C, int cu,
                            double* partials, int npartials, void* stream);
claire_status claire_nn_adam(float* p, const float* g, float* m1, float* m2, void* pb, long long count, float lr,
                             float b1, float b2, float eps, int step, void* stream);
/* Synchronises the stream, then reports whether a convolution's bounded tensor-core wait timed out since the last
 * call (CLAIRE_ETIMEOUT; the flag is cleared), a CUDA error (CLAIRE_ECUDA) or CLAIRE_OK. claire_ws_loss_f32 /
 * _train_step_f32 (with a loss) and claire_ws_predict_f32 check it themselves and return the same statuses. */
claire_status claire_nn_status(void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CLAIRE_GB300_H */
