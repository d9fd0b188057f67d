"""Plain FP64 CPU oracle of the reduced-space Gauss--Newton--Krylov registration hot path.

TEST INFRASTRUCTURE, NOT PRODUCT CODE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may import or run this module. It shares no code with the CUDA path: it has its own
interpolation, its own spectral operators (``numpy.fft`` as the library FFT step) and its own solver loops, written
in the order of the paper (Sec. 2.2-2.3, Alg. 1, Alg. 2) for a reader to check by eye. Everything is float64.

Discrete conventions (the readings of the paper that both this oracle and the CUDA path follow):

* Grid: n = (n1, n2, n3), each n_a even and >= 4, nodes x = h * i with h_a = 2*pi/n_a (Sec. 2.3.1). Scalars are
  [n1][n2][n3] arrays, vectors are [3][n1][n2][n3]; component c points along axis c.
* Spectral operators (Sec. 2.3.1): forward FFT unnormalised, inverse scaled by 1/N. Integer wavenumbers
  k_a in {0..n_a/2-1, n_a/2, -n_a/2+1..-1}. First-order symbols (gradient, divergence, Leray) use k'_a with the
  Nyquist entry k_a = n_a/2 set to 0; even-order symbols (A, preconditioner) use the full k.
* Inner product <a, b> = h1 h2 h3 sum(a * b) (trapezoidal rule on a periodic grid, Sec. 2.3.1); ||g|| = sqrt(<g, g>).
* Regularisation (Sec. 2.1, Eq. (5)): A = -Laplacian (H1 seminorm, symbol |k|^2) or A = Laplacian^2 (H2 seminorm,
  symbol |k|^4); the penalty is (beta/2) sum_c <v_c, A v_c>.
* Projection K (Sec. 2.2, after Eq. (5)): identity without the constraint; the Leray projector
  I - k' k'^T / |k'|^2 (identity where k' = 0) with div v = 0.
* H1-div model (Sec. 2.1-2.2: H1 seminorm for v plus beta_w/2 ||div v||^2_H1 with w = div v in the objective):
  K^ = I - q(k) k' k'^T, q = beta_w (|k|^2 + 1) / (beta_v |k|^2 + beta_w (|k|^2 + 1) |k'|^2) (the paper's K off
  the Nyquist planes). Eq. (5) and (7) keep their form with this K; beta_v A + K H_data is self-adjoint in
  <K^-1 a, b>, which PCG's kappa, mu and the Armijo slope <K^-1 g, dv> use; the stopping test uses ||g||.
* Semi-Lagrangian transport (Sec. 2.3.1, Sec. 3.4): nodal time grid t_j = j dt, dt = 1/n_t; RK2 (Heun)
  characteristics X* = x - dt v(x), X = x - dt/2 (v(x) + v(X*)) for the state, and Y with -v for the adjoints;
  tricubic Lagrange interpolation on the 4^3 stencil b-1..b+2 around b = floor(xi), indices taken periodically.
* Source terms: the incremental state integrates dm~/dt = -v~ . grad m along the characteristic with the
  trapezoidal (Heun) rule; the continuity-form adjoints integrate d lambda/ds = (div v) lambda along -v with Heun.
  Under the div v = 0 constraint div v is taken as 0 and the adjoints are pure transport.
* Time quadrature: trapezoidal weights w_0 = w_{n_t} = dt/2, w_j = dt otherwise (Sec. 2.3.1).
* Gauss-Newton (Sec. 2.3.2): the terms with lambda in Eq. (7) and Eq. (9) are dropped.
* Stopping (Sec. 2.3.2): ||g_k|| <= eps_g ||g_0|| with g_0 the gradient at v = 0, or ||g_k|| <= gtol_abs.
  PCG forcing eps_H = min(0.5, sqrt(||g_k|| / ||g_0||)) relative to ||r_0|| = ||g_k|| (Alg. 2), or a fixed
  relative tolerance when given. Armijo backtracking: alpha = 1, halved, sufficient decrease c1 = 1e-4, at most
  10 trials.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------------------------------------------
# Grid, inner product, spectral operators (Sec. 2.3.1)
# ----------------------------------------------------------------------------------------------------------------
class Grid:
    """Periodic grid on [0, 2*pi)^3 with its wavenumber tables."""

    def __init__(self, n):
        n = tuple(int(a) for a in n)
        if len(n) != 3 or any(a < 4 or a % 2 for a in n):
            raise ValueError("grid sizes must be three even integers >= 4")
        self.n = n
        self.N = n[0] * n[1] * n[2]
        self.h = tuple(2.0 * math.pi / a for a in n)
        self.cell = self.h[0] * self.h[1] * self.h[2]
        k1 = np.fft.fftfreq(n[0], 1.0 / n[0])
        k2 = np.fft.fftfreq(n[1], 1.0 / n[1])
        k3 = np.arange(n[2] // 2 + 1, dtype=np.float64)
        # full wavenumbers, the Nyquist entry taken as +n_a/2 (only its even powers are used)
        self.k = [np.where(ka == -na / 2, na / 2, ka) for ka, na in zip((k1, k2, k3), n)]
        # first-order wavenumbers: Nyquist zeroed
        self.kp = [np.where(np.abs(ka) == na / 2, 0.0, ka) for ka, na in zip(self.k, n)]
        shp = (n[0], n[1], n[2] // 2 + 1)
        self.K = [np.broadcast_to(self.k[0][:, None, None], shp),
                  np.broadcast_to(self.k[1][None, :, None], shp),
                  np.broadcast_to(self.k[2][None, None, :], shp)]
        self.KP = [np.broadcast_to(self.kp[0][:, None, None], shp),
                   np.broadcast_to(self.kp[1][None, :, None], shp),
                   np.broadcast_to(self.kp[2][None, None, :], shp)]
        self.ksq = self.K[0] ** 2 + self.K[1] ** 2 + self.K[2] ** 2
        self.kpsq = self.KP[0] ** 2 + self.KP[1] ** 2 + self.KP[2] ** 2

    def fft(self, f):
        return np.fft.rfftn(f)

    def ifft(self, F):
        return np.fft.irfftn(F, s=self.n, axes=(0, 1, 2))


def inner(grid, a, b):
    """<a, b> = h1 h2 h3 sum a*b over all entries (trapezoidal rule on the periodic grid, Sec. 2.3.1)."""
    return grid.cell * float(np.sum(np.asarray(a, dtype=np.float64) * np.asarray(b, dtype=np.float64)))


def norm(grid, a):
    return math.sqrt(inner(grid, a, a))


def gradient_spectral(grid, f):
    """grad f = F^-1[i k'_a F f], a = 1, 2, 3 (Sec. 2.3.1)."""
    F = grid.fft(f)
    return np.stack([grid.ifft(1j * grid.KP[a] * F) for a in range(3)])


def divergence_spectral(grid, v):
    """div v = F^-1[sum_a i k'_a F v_a] (Sec. 2.3.1)."""
    S = sum(1j * grid.KP[a] * grid.fft(v[a]) for a in range(3))
    return grid.ifft(S)


def laplacian_spectral(grid, f):
    """Laplacian f = F^-1[-|k|^2 F f]."""
    return grid.ifft(-grid.ksq * grid.fft(f))


def reg_symbol(grid, regnorm):
    """Symbol a(k) of A = B*B: |k|^2 for the H1 seminorm, |k|^4 for the H2 seminorm (Sec. 2.1, Eq. (5))."""
    if regnorm == 1:
        return grid.ksq
    if regnorm == 2:
        return grid.ksq ** 2
    raise ValueError("regnorm must be 1 (H1) or 2 (H2)")


def apply_A(grid, v, regnorm):
    """A v componentwise."""
    a = reg_symbol(grid, regnorm)
    return np.stack([grid.ifft(a * grid.fft(v[c])) for c in range(3)])


def leray(grid, v):
    """K v = v - grad Lap^-1 div v, i.e. K^ = I - k' k'^T / |k'|^2 with K^ = I where k' = 0 (Sec. 2.2)."""
    V = [grid.fft(v[c]) for c in range(3)]
    kv = grid.KP[0] * V[0] + grid.KP[1] * V[1] + grid.KP[2] * V[2]
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(grid.kpsq > 0, kv / np.where(grid.kpsq > 0, grid.kpsq, 1.0), 0.0)
    return np.stack([grid.ifft(V[c] - grid.KP[c] * s) for c in range(3)])


def apply_K(grid, v, divfree):
    return leray(grid, v) if divfree else v


def _h1div_coeff(grid, beta, beta_w):
    """q(k) with K^ = I - q k' k'^T for the H1-div model (Sec. 2.2, the K following Eq. (5), A = -Lap).

    The paper's K = I - grad (beta_v (beta_w (-Lap + I))^-1 + I)^-1 Lap^-1 div has, with first-order symbols k'
    and even-order symbols k, the symbol I - c(k) k' k'^T / |k'|^2, c = beta_w (|k|^2 + 1) / (beta_v + beta_w
    (|k|^2 + 1)). Written with |k'|^2 in the denominator's divergence term (equal off the Nyquist planes),
    q = beta_w (|k|^2 + 1) / (beta_v |k|^2 + beta_w (|k|^2 + 1) |k'|^2), which makes K beta_v^-1 A^-1 the exact
    inverse of the regularisation operator of the objective (see regularization_h1div)."""
    ksq, kpsq = grid.ksq, grid.kpsq
    den = beta * ksq + beta_w * (ksq + 1.0) * kpsq
    return np.where(den > 0, beta_w * (ksq + 1.0) / np.where(den > 0, den, 1.0), 0.0)


def _apply_rank1(grid, v, coeff, sign):
    """v + sign F^-1[coeff k' (k' . F v)]."""
    V = [grid.fft(v[c]) for c in range(3)]
    kv = grid.KP[0] * V[0] + grid.KP[1] * V[1] + grid.KP[2] * V[2]
    return np.stack([grid.ifft(V[c] + sign * coeff * grid.KP[c] * kv) for c in range(3)])


def h1div_K(grid, v, beta, beta_w):
    """K v of the H1-div model (near-incompressible, Sec. 2.1-2.2)."""
    return _apply_rank1(grid, v, _h1div_coeff(grid, beta, beta_w), -1.0)


def h1div_Kinv(grid, v, beta, beta_w):
    """K^-1 v = v + F^-1[beta_w (|k|^2 + 1) / (beta_v |k|^2) k' (k' . F v)] (identity at k = 0)."""
    ksq = grid.ksq
    s = np.where(ksq > 0, beta_w * (ksq + 1.0) / (beta * np.where(ksq > 0, ksq, 1.0)), 0.0)
    return _apply_rank1(grid, v, s, +1.0)


def regularization_h1div(grid, v, beta_w):
    """beta_w <w, (-Lap + I) w> with w = div v: twice the divergence penalty of the objective (Eq. (1))."""
    w = divergence_spectral(grid, v)
    return beta_w * inner(grid, w, w - laplacian_spectral(grid, w))


def apply_Kp(prob, v):
    """The K of Eq. (5) for the problem's model: identity, Leray, or the H1-div operator."""
    if prob.beta_w > 0:
        return h1div_K(prob.grid, v, prob.beta, prob.beta_w)
    return apply_K(prob.grid, v, prob.divfree)


def control_inner(prob, a, b):
    """Inner product of the Newton system: <a, b>, or <K^-1 a, b> for the H1-div model. With it the operator
    beta_v A + K H_data of Eq. (7) is self-adjoint, and <K^-1 g, dv> is the derivative of J along dv."""
    if prob.beta_w > 0:
        return inner(prob.grid, h1div_Kinv(prob.grid, a, prob.beta, prob.beta_w), b)
    return inner(prob.grid, a, b)


def precond(grid, r, beta, regnorm):
    """Spectral preconditioner M^-1 = (beta A)^-1 with the zero eigenvalue replaced by 1 (Sec. 2.3.3, Remark)."""
    a = reg_symbol(grid, regnorm)
    inv = np.where(a > 0, 1.0 / np.where(a > 0, beta * a, 1.0), 1.0)
    return np.stack([grid.ifft(inv * grid.fft(r[c])) for c in range(3)])


def regularization_value(grid, v, regnorm):
    """R(v) = sum_c <v_c, A v_c>."""
    return inner(grid, v, apply_A(grid, v, regnorm))


# ----------------------------------------------------------------------------------------------------------------
# Tricubic Lagrange interpolation and RK2 characteristics (Sec. 2.3.1, Sec. 3.4)
# ----------------------------------------------------------------------------------------------------------------
def lagrange_weights(t):
    """Cubic Lagrange basis on the nodes -1, 0, 1, 2 evaluated at t (returns 4 arrays)."""
    return ((-t * (t - 1.0) * (t - 2.0)) / 6.0,
            ((t + 1.0) * (t - 1.0) * (t - 2.0)) / 2.0,
            (-(t + 1.0) * t * (t - 2.0)) / 2.0,
            ((t + 1.0) * t * (t - 1.0)) / 6.0)


def interp(f, disp, chunk=1 << 20):
    """Evaluate the periodic tricubic Lagrange interpolant of f at xi = i + disp (grid units).

    f: [n1][n2][n3]; disp: [3][n1][n2][n3] displacement of every node in grid units.
    For each axis: b = floor(xi), t = xi - b, stencil nodes b-1, b, b+1, b+2 taken modulo n_a; the value is the
    tensor-product sum of the 4 x 4 x 4 taps.
    """
    n = f.shape
    N = f.size
    ff = f.ravel()
    out = np.empty(N, dtype=np.float64)
    ii = np.indices(n).reshape(3, -1)
    dd = disp.reshape(3, -1)
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        idx, wts = [], []
        for a in range(3):
            xi = ii[a, s:e] + dd[a, s:e]
            b = np.floor(xi)
            t = xi - b
            b = b.astype(np.int64)
            idx.append([np.mod(b + p, n[a]) for p in (-1, 0, 1, 2)])
            wts.append(lagrange_weights(t))
        acc = np.zeros(e - s, dtype=np.float64)
        for p in range(4):
            for q in range(4):
                w12 = wts[0][p] * wts[1][q]
                base = (idx[0][p] * n[1] + idx[1][q]) * n[2]
                for r in range(4):
                    acc += w12 * wts[2][r] * ff[base + idx[2][r]]
        out[s:e] = acc
    return out.reshape(n)


def departure(grid, v, nt, sign):
    """RK2 departure points in grid units for one time step of length dt = 1/nt.

    sign = +1: state characteristics (backtrace along v):  X* = x - dt v(x), X = x - dt/2 (v(x) + v(X*)).
    sign = -1: adjoint characteristics (backtrace along -v): Y* = x + dt v(x), Y = x + dt/2 (v(x) + v(Y*)).
    Returns [3][n1][n2][n3] displacements (X - x) / h per axis.
    """
    dt = 1.0 / nt
    h = grid.h
    dstar = np.stack([-sign * dt * v[a] / h[a] for a in range(3)])
    vstar = np.stack([interp(v[a], dstar) for a in range(3)])
    return np.stack([-sign * 0.5 * dt * (v[a] + vstar[a]) / h[a] for a in range(3)])


# ----------------------------------------------------------------------------------------------------------------
# PDE solves (Eq. (2), (4), (8), (9)) and the reduced gradient / GN Hessian matvec (Eq. (5), (7))
# ----------------------------------------------------------------------------------------------------------------
@dataclass
class Problem:
    n: tuple
    beta: float
    nt: int = 4
    regnorm: int = 1          # 1: H1 seminorm (A = -Lap), 2: H2 seminorm (A = Lap^2)
    divfree: bool = False     # div v = 0 via the Leray projection
    beta_w: float = 0.0       # > 0: H1-div model, penalty beta_w/2 ||div v||_H1^2 (needs regnorm 1, no divfree)
    precond: int = 0          # 0: spectral preconditioner; 1: two-level preconditioner (Sec. 2.3.3)
    pc_kappa: float = 0.1     # nested PCG tolerance eps_M = pc_kappa eps_H (two-level)
    gtol_rel: float = 5e-2
    gtol_abs: float = 1e-6
    max_gn: int = 50
    max_krylov: int = 100
    pcg_rtol: float = 0.0     # <= 0: superlinear forcing of Alg. 2
    max_ls: int = 10
    armijo_c1: float = 1e-4

    def __post_init__(self):
        self.grid = Grid(self.n)
        if self.nt < 1 or not (self.beta > 0):
            raise ValueError("nt >= 1 and beta > 0 required")
        if self.beta_w < 0 or (self.beta_w > 0 and (self.divfree or self.regnorm != 1)):
            raise ValueError("beta_w > 0 (H1-div) needs regnorm 1 and no div v = 0 constraint")
        if self.precond == 1 and any(a % 4 for a in self.n):
            raise ValueError("the two-level preconditioner needs grid sizes divisible by 4")

    def time_weights(self):
        dt = 1.0 / self.nt
        w = np.full(self.nt + 1, dt)
        w[0] = w[-1] = 0.5 * dt
        return w


@dataclass
class Linearization:
    """Everything that depends only on v: departure points, state history and its spectral gradients."""
    v: np.ndarray
    dX: np.ndarray
    dY: np.ndarray
    m: list
    gradm: list
    rho: np.ndarray | None


def state_solve(prob, mT, dX):
    """State equation (2) forward in time: m^{j+1}(x) = m^j(X(x)), m^0 = m_T."""
    m = [np.array(mT, dtype=np.float64)]
    for _ in range(prob.nt):
        m.append(interp(m[-1], dX))
    return m


def linearize(prob, mT, v):
    g = prob.grid
    v = np.asarray(v, dtype=np.float64)
    dX = departure(g, v, prob.nt, +1)
    dY = departure(g, v, prob.nt, -1)
    m = state_solve(prob, mT, dX)
    gradm = [gradient_spectral(g, mj) for mj in m]
    rho = None if prob.divfree else divergence_spectral(g, v)
    return Linearization(v=v, dX=dX, dY=dY, m=m, gradm=gradm, rho=rho)


def continuity_step(prob, lam_next, dY, rho):
    """One backward step of -d_t lam - div(lam v) = 0 (Eq. (4), (9)) along the -v characteristics.

    Pure transport a = lam^{j+1}(Y) when div v is taken as 0; otherwise Heun on d lam/ds = rho lam:
    c = (rho lam^{j+1})(Y), lam^j = a + dt/2 (c + rho(x) (a + dt c)).
    """
    a = interp(lam_next, dY)
    if rho is None:
        return a
    dt = 1.0 / prob.nt
    c = interp(rho * lam_next, dY)
    return a + 0.5 * dt * (c + rho * (a + dt * c))


def adjoint_integral(prob, lin, lam_final):
    """Solve the (incremental) adjoint backward and return b = sum_j w_j lam^j grad m^j (trapezoid in time)."""
    w = prob.time_weights()
    lam = lam_final
    b = w[prob.nt] * lam * lin.gradm[prob.nt]
    for j in range(prob.nt - 1, -1, -1):
        lam = continuity_step(prob, lam, lin.dY, lin.rho)
        b = b + w[j] * lam * lin.gradm[j]
    return b


def objective(prob, mR, m1, v):
    """J = 1/2 <m_1 - m_R, m_1 - m_R> + beta/2 sum_c <v_c, A v_c> (Eq. (2), objective), plus
    beta_w/2 (<grad w, grad w> + <w, w>) with w = div v for the H1-div model."""
    g = prob.grid
    res = m1 - mR
    J = 0.5 * inner(g, res, res) + 0.5 * prob.beta * regularization_value(g, v, prob.regnorm)
    if prob.beta_w > 0:
        J += 0.5 * regularization_h1div(g, v, prob.beta_w)
    return J


def reduced_gradient(prob, lin, mR):
    """g = beta A v + K[ int_0^1 lam grad m dt ] with lam(1) = m_R - m_1 (Eq. (4), (5))."""
    g = prob.grid
    lam1 = mR - lin.m[prob.nt]
    b = adjoint_integral(prob, lin, lam1)
    return prob.beta * apply_A(g, lin.v, prob.regnorm) + apply_Kp(prob, b)


def incremental_state(prob, lin, vt):
    """Eq. (8): d_t m~ + grad m~ . v + grad m . v~ = 0, m~(0) = 0; returns m~(1).

    With f^j = -v~ . grad m^j, the Heun step along the state characteristic is
    m~^{j+1}(x) = [m~^j + dt/2 f^j](X) + dt/2 f^{j+1}(x).
    """
    dt = 1.0 / prob.nt
    f = [-(vt[0] * gm[0] + vt[1] * gm[1] + vt[2] * gm[2]) for gm in lin.gradm]
    mt = np.zeros(prob.grid.n)
    for j in range(prob.nt):
        mt = interp(mt + 0.5 * dt * f[j], lin.dX) + 0.5 * dt * f[j + 1]
    return mt


def hessvec(prob, lin, vt):
    """Gauss-Newton Hessian matvec (Eq. (7) without the lambda terms, Sec. 2.3.2).

    m~ from Eq. (8); lam~ from Eq. (9) (lam v~ term dropped) with lam~(1) = -m~(1);
    H v~ = beta A v~ + K[ int_0^1 lam~ grad m dt ].
    """
    g = prob.grid
    mt1 = incremental_state(prob, lin, vt)
    bt = adjoint_integral(prob, lin, -mt1)
    return prob.beta * apply_A(g, vt, prob.regnorm) + apply_Kp(prob, bt)


def transport(prob, m0, v, direction=+1):
    """Transport m0 over the unit time interval: direction=+1 state equation (2); -1 continuity-form adjoint (4)
    run backward from t = 1 (final condition m0) to t = 0."""
    g = prob.grid
    if direction == +1:
        dX = departure(g, v, prob.nt, +1)
        return state_solve(prob, m0, dX)[-1]
    dY = departure(g, v, prob.nt, -1)
    rho = None if prob.divfree else divergence_spectral(g, v)
    lam = np.array(m0, dtype=np.float64)
    for _ in range(prob.nt):
        lam = continuity_step(prob, lam, dY, rho)
    return lam


# ----------------------------------------------------------------------------------------------------------------
# Inexact Gauss-Newton-Krylov solver (Alg. 1, Alg. 2, Sec. 2.3.2)
# ----------------------------------------------------------------------------------------------------------------
@dataclass
class Report:
    gn_iters: int = 0
    matvecs: int = 0
    pde_solves: int = 0
    ls_trials: int = 0
    pcg_iters: list = field(default_factory=list)
    J0: float = 0.0
    J: float = 0.0
    mismatch0: float = 0.0
    mismatch: float = 0.0
    gnorm0: float = 0.0
    gnorm: float = 0.0
    coarse_matvecs: int = 0
    converged: bool = False
    status: str = "ok"

    @property
    def gnorm_rel(self):
        return self.gnorm / self.gnorm0 if self.gnorm0 > 0 else 0.0

    @property
    def mismatch_rel(self):
        return self.mismatch / self.mismatch0 if self.mismatch0 > 0 else 0.0


def pcg(prob, lin, g_k, eps_H, report, coarse=None):
    """Alg. 2: PCG on H v~ = -g with the spectral preconditioner; break when ||r|| < eps_H ||r_0||.

    The inner products of kappa and mu are control_inner (the K^-1-weighted one for the H1-div model, where
    H = beta_v A + K H_data is self-adjoint in it); the break test uses the plain norm of r."""
    grid = prob.grid

    def M(r):
        if prob.precond == 1:
            return twolevel_apply(prob, coarse, r, prob.pc_kappa * eps_H, report)
        return precond(grid, r, prob.beta, prob.regnorm)

    vt = np.zeros_like(g_k)
    r = -g_k
    z = M(r)
    s = z.copy()
    rz = control_inner(prob, r, z)
    r0 = norm(grid, r)
    it = 0
    while it < prob.max_krylov:
        Hs = hessvec(prob, lin, s)
        report.matvecs += 1
        report.pde_solves += 2
        sHs = control_inner(prob, Hs, s)
        if not (sHs > 0):
            if it == 0:
                vt = s.copy()
            break
        kappa = rz / sHs
        vt = vt + kappa * s
        r = r - kappa * Hs
        it += 1
        if norm(grid, r) < eps_H * r0:
            break
        z = M(r)
        rz_new = control_inner(prob, r, z)
        mu = rz_new / rz
        rz = rz_new
        s = z + mu * s
    report.pcg_iters.append(it)
    return vt


def evaluate(prob, mT, mR, v):
    """State solve + objective for a trial v (one PDE solve)."""
    g = prob.grid
    dX = departure(g, v, prob.nt, +1)
    m = state_solve(prob, mT, dX)
    return objective(prob, mR, m[-1], v), m[-1]


def register(prob, mT, mR, v0=None):
    """Alg. 1 with the stopping rules of Sec. 2.3.2 and an Armijo line search; returns (v, Report)."""
    grid = prob.grid
    mT = np.asarray(mT, dtype=np.float64)
    mR = np.asarray(mR, dtype=np.float64)
    v = np.zeros((3,) + grid.n) if v0 is None else np.array(v0, dtype=np.float64)
    rep = Report()
    res0 = mR - mT
    rep.mismatch0 = 0.5 * inner(grid, res0, res0)
    # reference gradient g_0 at v = 0
    lin = linearize(prob, mT, np.zeros((3,) + grid.n))
    g0 = reduced_gradient(prob, lin, mR)
    rep.gnorm0 = norm(grid, g0)
    rep.pde_solves += 2
    if v0 is not None and np.any(v != 0):
        if prob.divfree:
            # the control space is divergence-free (Sec. 2.2): a nonzero initial guess is projected onto it
            v = leray(grid, v)
        lin = linearize(prob, mT, v)
        g = reduced_gradient(prob, lin, mR)
        rep.pde_solves += 2
    else:
        g = g0
    J = objective(prob, mR, lin.m[-1], v)
    rep.J0 = J
    gnorm = norm(grid, g)
    cprob = coarse_problem(prob) if prob.precond == 1 else None
    mT_c = restrict_field(grid, cprob.grid, mT) if cprob is not None else None
    while True:
        if gnorm <= prob.gtol_rel * rep.gnorm0 or gnorm <= prob.gtol_abs:
            rep.converged = True
            break
        if rep.gn_iters >= prob.max_gn:
            rep.status = "max_gn"
            break
        if prob.pcg_rtol > 0:
            eps_H = prob.pcg_rtol
        else:
            eps_H = min(0.5, math.sqrt(gnorm / rep.gnorm0))
        coarse = None
        if cprob is not None:
            coarse = (cprob, linearize(cprob, mT_c, np.stack([restrict_field(grid, cprob.grid, v[c])
                                                              for c in range(3)])))
        vt = pcg(prob, lin, g, eps_H, rep, coarse)
        if prob.divfree:
            vt = leray(grid, vt)
        gvt = control_inner(prob, g, vt)
        alpha = 1.0
        accepted = False
        for _ in range(prob.max_ls):
            vtrial = v + alpha * vt
            Jt, _ = evaluate(prob, mT, mR, vtrial)
            rep.ls_trials += 1
            rep.pde_solves += 1
            if Jt <= J + prob.armijo_c1 * alpha * gvt:
                accepted = True
                break
            alpha *= 0.5
        if not accepted:
            rep.status = "linesearch"
            break
        v = vtrial
        lin = linearize(prob, mT, v)
        g = reduced_gradient(prob, lin, mR)
        rep.pde_solves += 1     # the state of the accepted trial is reused; only the adjoint solve is new
        J = objective(prob, mR, lin.m[-1], v)
        gnorm = norm(grid, g)
        rep.gn_iters += 1
    rep.J = J
    res = mR - lin.m[-1]
    rep.mismatch = 0.5 * inner(grid, res, res)
    rep.gnorm = gnorm
    return v, rep


def continuation_levels(beta_target, beta_start=1.0, factor=0.1, max_levels=16):
    """beta_v of each level of the parameter continuation (Sec. 3.6): beta_start, beta_start*factor, ... while
    above the target, then the target."""
    betas = []
    b = beta_start
    while b > beta_target * (1.0 + 1e-12) and len(betas) < max_levels - 1:
        betas.append(b)
        b *= factor
    betas.append(beta_target)
    return betas


def register_continuation(prob, mT, mR, v0=None, beta_start=1.0, factor=0.1, max_levels=16):
    """Parameter continuation in beta_v (Sec. 3.6): one full solve per level, each warm-started from the previous
    level's solution; returns (v, [Report per level])."""
    from dataclasses import replace
    v = v0
    reports = []
    for b in continuation_levels(prob.beta, beta_start, factor, max_levels):
        v, rep = register(replace(prob, beta=b), mT, mR, v)
        reports.append(rep)
        if not rep.converged and rep.status != "max_gn":
            break
    return v, reports



# ----------------------------------------------------------------------------------------------------------------
# Two-level preconditioner (Sec. 2.3.3)
# ----------------------------------------------------------------------------------------------------------------
# It acts on the regularisation split-preconditioned system (I + R^-1/2 H_data R^-1/2) w = -R^-1/2 g with
# R = beta A (its zero eigenvalue set to 1) and w = R^1/2 v~. For s = R^-1/2 r, the low-frequency part (the modes
# the half-resolution grid holds, Nyquist excluded) is replaced by the nested-PCG solution of the same system
# discretised directly on the coarse grid; the high-frequency part is kept (H_H replaced by I). Restriction and
# prolongation are spectral. In the original variables the preconditioner is M^-1 r = R^-1/2 P(R^-1/2 r).
def coarse_problem(prob):
    """The same problem on the grid n/2 (spectral preconditioner; the nested solver iterates on it)."""
    from dataclasses import replace
    return replace(prob, n=tuple(a // 2 for a in prob.n), precond=0)


def split_symbol(grid, beta, regnorm):
    """(beta a(k))^-1/2, 1 where a(k) = 0."""
    a = reg_symbol(grid, regnorm)
    return np.where(a > 0, 1.0 / np.sqrt(np.where(a > 0, beta * a, 1.0)), 1.0)


def _kept_pairs(n_f, n_c, half):
    """Index pairs (fine, coarse) of the wavenumbers kept along one axis: 2|k| < n_c (coarse Nyquist dropped)."""
    top = (n_c - 1) // 2
    ks = np.arange(0, top + 1) if half else np.arange(-top, top + 1)
    return ks % n_f, ks % n_c


def low_mask(grid_f, grid_c):
    """Fine half-spectrum mask of the modes the coarse grid holds."""
    mask = np.zeros((grid_f.n[0], grid_f.n[1], grid_f.n[2] // 2 + 1), dtype=bool)
    f1, _ = _kept_pairs(grid_f.n[0], grid_c.n[0], False)
    f2, _ = _kept_pairs(grid_f.n[1], grid_c.n[1], False)
    f3, _ = _kept_pairs(grid_f.n[2], grid_c.n[2], True)
    mask[np.ix_(f1, f2, f3)] = True
    return mask


def restrict_spectrum(grid_f, grid_c, F):
    """Fine half spectrum -> coarse half spectrum of the same function (scaled by N_c / N_f)."""
    f1, c1 = _kept_pairs(grid_f.n[0], grid_c.n[0], False)
    f2, c2 = _kept_pairs(grid_f.n[1], grid_c.n[1], False)
    f3, c3 = _kept_pairs(grid_f.n[2], grid_c.n[2], True)
    G = np.zeros((grid_c.n[0], grid_c.n[1], grid_c.n[2] // 2 + 1), dtype=complex)
    G[np.ix_(c1, c2, c3)] = F[np.ix_(f1, f2, f3)] * (grid_c.N / grid_f.N)
    return G


def prolong_spectrum(grid_f, grid_c, G):
    """Coarse half spectrum -> fine half spectrum (zero outside the coarse modes; scaled by N_f / N_c)."""
    f1, c1 = _kept_pairs(grid_f.n[0], grid_c.n[0], False)
    f2, c2 = _kept_pairs(grid_f.n[1], grid_c.n[1], False)
    f3, c3 = _kept_pairs(grid_f.n[2], grid_c.n[2], True)
    F = np.zeros((grid_f.n[0], grid_f.n[1], grid_f.n[2] // 2 + 1), dtype=complex)
    F[np.ix_(f1, f2, f3)] = G[np.ix_(c1, c2, c3)] * (grid_f.N / grid_c.N)
    return F


def restrict_field(grid_f, grid_c, f):
    return grid_c.ifft(restrict_spectrum(grid_f, grid_c, grid_f.fft(f)))


def hess_data(prob, lin, vt):
    """Data part K[int lam~ grad m dt] of the Gauss-Newton matvec (Eq. (7)-(9))."""
    mt1 = incremental_state(prob, lin, vt)
    return apply_Kp(prob, adjoint_integral(prob, lin, -mt1))


def _scale(grid, x, sym):
    return np.stack([grid.ifft(sym * grid.fft(x[c])) for c in range(3)])


def coarse_operator(cprob, clin, x):
    """(I + R^-1/2 H_data R^-1/2) x on the coarse grid."""
    s = split_symbol(cprob.grid, cprob.beta, cprob.regnorm)
    return x + _scale(cprob.grid, hess_data(cprob, clin, _scale(cprob.grid, x, s)), s)


def nested_pcg(cprob, clin, f, eps_M, report):
    """CG on the coarse split system (already regularisation-preconditioned, so no further preconditioner);
    u = 0 at the start, break when ||r|| < eps_M ||f||, at most max_krylov iterations."""
    grid = cprob.grid
    u = np.zeros_like(f)
    r = f.copy()
    p = r.copy()
    rr = control_inner(cprob, r, r)
    f0 = norm(grid, f)
    if f0 == 0.0:
        return u
    for _ in range(cprob.max_krylov):
        Hp = coarse_operator(cprob, clin, p)
        report.coarse_matvecs += 1
        pHp = control_inner(cprob, Hp, p)
        if not (pHp > 0):
            break
        alpha = rr / pHp
        u = u + alpha * p
        r = r - alpha * Hp
        if norm(grid, r) < eps_M * f0:
            break
        rr_new = control_inner(cprob, r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return u


def twolevel_apply(prob, coarse, r, eps_M, report):
    """z = M^-1 r of the two-level preconditioner; coarse = (coarse problem, its linearization at v)."""
    cprob, clin = coarse
    gf, gc = prob.grid, cprob.grid
    sf = split_symbol(gf, prob.beta, prob.regnorm)
    Y = [gf.fft(r[c]) * sf for c in range(3)]
    f = np.stack([gc.ifft(restrict_spectrum(gf, gc, Y[c])) for c in range(3)])
    u = nested_pcg(cprob, clin, f, eps_M, report)
    low = low_mask(gf, gc)
    Z = [np.where(low, prolong_spectrum(gf, gc, gc.fft(u[c])), Y[c]) * sf for c in range(3)]
    return np.stack([gf.ifft(Z[c]) for c in range(3)])
