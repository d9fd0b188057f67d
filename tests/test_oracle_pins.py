"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU, no CUDA code involved).

Every oracle function is tied here to something other than itself: closed forms of trigonometric polynomials,
exact identities of the discrete scheme (identity / constant-velocity transport, Parseval), brute force on tiny
grids, the convergence order of the RK2 characteristics, finite differences of the objective and the paper's
printed solver bookkeeping.
"""
import math
import os

import numpy as np
import pytest

import claire_inputs as I
from oracle import claire_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def coords(n):
    x = I.grid_coords(n)
    return np.meshgrid(*x, indexing="ij")


# ---------------------------------------------------------------------------------------------- spectral (P1-P3)
NONCUBIC = (12, 16, 20)


def trig_poly(n, seed=3):
    """Random trigonometric polynomial with |k_a| < n_a/2 and its exact gradient and Laplacian."""
    rng = np.random.default_rng(seed)
    X = coords(n)
    f = np.zeros(n)
    gf = np.zeros((3,) + n)
    lap = np.zeros(n)
    for _ in range(6):
        k = [int(rng.integers(-(na // 2) + 1, na // 2)) for na in n]
        a, b = rng.normal(size=2)
        ph = k[0] * X[0] + k[1] * X[1] + k[2] * X[2]
        f += a * np.cos(ph) + b * np.sin(ph)
        for c in range(3):
            gf[c] += k[c] * (-a * np.sin(ph) + b * np.cos(ph))
        lap += -(k[0] ** 2 + k[1] ** 2 + k[2] ** 2) * (a * np.cos(ph) + b * np.sin(ph))
    return f, gf, lap


@pytest.mark.parametrize("n", [(16, 16, 16), NONCUBIC])
def test_P1_spectral_derivatives_exact(n):
    g = O.Grid(n)
    f, gf, lap = trig_poly(n)
    assert rel(O.gradient_spectral(g, f), gf) < 1e-13
    assert rel(O.laplacian_spectral(g, f), lap) < 1e-13
    # divergence of a gradient is the Laplacian
    assert rel(O.divergence_spectral(g, gf), lap) < 1e-13


def test_P1_nyquist_mode_has_zero_first_derivative_and_full_second():
    n = (8, 8, 8)
    g = O.Grid(n)
    X = coords(n)
    f = np.cos(4 * X[2])  # Nyquist along axis 3: samples (+1,-1,...)
    assert np.abs(O.gradient_spectral(g, f)).max() < 1e-13
    assert rel(O.laplacian_spectral(g, f), -16 * f) < 1e-13


@pytest.mark.parametrize("regnorm,power", [(1, 1), (2, 2)])
def test_regularization_symbol_on_trig(regnorm, power):
    n = NONCUBIC
    g = O.Grid(n)
    X = coords(n)
    v = np.stack([np.cos(2 * X[0] + X[1]), np.sin(3 * X[2]), np.cos(X[0] - 2 * X[1] + 4 * X[2])])
    ksq = [5, 9, 21]
    Av = O.apply_A(g, v, regnorm)
    for c in range(3):
        assert rel(Av[c], ksq[c] ** power * v[c]) < 1e-13
    # R(v) = sum_c <v_c, A v_c>; each cos^2/sin^2 averages to 1/2 over the box of volume (2 pi)^3
    expect = sum(k ** power for k in ksq) * 0.5 * (2 * math.pi) ** 3
    assert abs(O.regularization_value(g, v, regnorm) - expect) < 1e-10 * expect


def test_P2_fft_step_matches_naive_dft_and_parseval():
    n = (4, 6, 8)
    g = O.Grid(n)
    rng = np.random.default_rng(0)
    f = rng.normal(size=n)
    F = g.fft(f)
    i = np.indices(n).reshape(3, -1)
    for k in [(0, 0, 0), (1, 2, 3), (3, 5, 4), (2, 0, 1)]:
        ph = sum(-2j * math.pi * k[a] * i[a] / n[a] for a in range(3))
        assert abs(F[k] - np.sum(f.ravel() * np.exp(ph))) < 1e-12
    assert rel(g.ifft(F), f) < 1e-14
    # Parseval on the half spectrum: interior planes count twice
    w = np.full(F.shape[2], 2.0)
    w[0] = 1.0
    w[-1] = 1.0
    assert abs(np.sum(w * np.abs(F) ** 2) / g.N - np.sum(f ** 2)) < 1e-10 * np.sum(f ** 2)


def test_P3_leray_projection():
    n = NONCUBIC
    g = O.Grid(n)
    rng = np.random.default_rng(1)
    v = rng.normal(size=(3,) + n)
    w = rng.normal(size=(3,) + n)
    Kv = O.leray(g, v)
    assert rel(O.leray(g, Kv), Kv) < 1e-13                       # K^2 = K
    assert abs(O.inner(g, Kv, w) - O.inner(g, v, O.leray(g, w))) < 1e-11 * O.norm(g, v) * O.norm(g, w)  # K^T = K
    assert np.abs(O.divergence_spectral(g, Kv)).max() < 1e-11 * np.abs(v).max()
    phi, gphi, _ = trig_poly(n, seed=5)
    assert np.abs(O.leray(g, gphi)).max() < 1e-12 * np.abs(gphi).max()  # K grad phi = 0
    # Helmholtz split: curl part is kept exactly
    X = coords(n)
    curl = np.stack([np.sin(X[2]) * np.cos(2 * X[1]), np.cos(X[0] + X[2]) * 0 + np.sin(3 * X[0]), np.cos(X[1])])
    assert np.abs(O.divergence_spectral(g, curl)).max() < 1e-12
    assert rel(O.leray(g, curl + gphi), curl) < 1e-12
    # the paper's synthetic velocity is divergence free
    _, vstar = I.paper_synthetic((16, 16, 16))
    g16 = O.Grid((16, 16, 16))
    assert rel(O.leray(g16, vstar), vstar) < 1e-13


def test_P10_preconditioner_identity_and_trig():
    n = NONCUBIC
    g = O.Grid(n)
    rng = np.random.default_rng(2)
    v = rng.normal(size=(3,) + n)
    v -= v.mean(axis=(1, 2, 3), keepdims=True)
    for regnorm in (1, 2):
        beta = 3e-3
        assert rel(O.precond(g, beta * O.apply_A(g, v, regnorm), beta, regnorm), v) < 1e-11
    c = np.ones((3,) + n) * np.array([1.0, -2.0, 0.5])[:, None, None, None]
    assert rel(O.precond(g, c, 1e-3, 1), c) < 1e-14              # the mean is left unchanged
    X = coords(n)
    f = np.cos(X[0] + 2 * X[1] - 3 * X[2])
    z = O.precond(g, np.stack([f, f, f]), 0.5, 2)
    assert rel(z[0], f / (0.5 * 14 ** 2)) < 1e-13


def test_inner_product_is_the_box_integral():
    g = O.Grid((8, 10, 12))
    assert abs(O.inner(g, np.ones(g.n), np.ones(g.n)) - (2 * math.pi) ** 3) < 1e-12


# ---------------------------------------------------------------------------------------------- interpolation
def test_lagrange_weights_closed_forms():
    w = O.lagrange_weights(np.array([0.0, 0.5, 1.0]))
    assert np.allclose([x[0] for x in w], [0, 1, 0, 0], atol=0)
    assert np.allclose([x[1] for x in w], [-1 / 16, 9 / 16, 9 / 16, -1 / 16], rtol=0, atol=1e-16)
    assert np.allclose([x[2] for x in w], [0, 0, 1, 0], atol=0)
    t = np.linspace(0, 1, 17)
    ws = O.lagrange_weights(t)
    assert np.abs(sum(ws) - 1).max() < 1e-15                      # partition of unity
    for p in range(4):                                            # reproduces monomials up to degree 3
        mono = sum(wj * (node ** p) for wj, node in zip(ws, (-1.0, 0.0, 1.0, 2.0)))
        assert np.abs(mono - t ** p).max() < 1e-14


def test_interp_reproduces_cubics_away_from_the_wrap():
    n = (16, 16, 16)
    i = np.indices(n).astype(float)
    f = 0.3 + 0.1 * i[0] - 0.02 * i[1] ** 2 + 0.001 * i[2] ** 3 + 0.003 * i[0] * i[1] * i[2]
    rng = np.random.default_rng(0)
    d = rng.uniform(-1.0, 1.0, size=(3,) + n)
    out = O.interp(f, d)
    xi = i + d
    exact = 0.3 + 0.1 * xi[0] - 0.02 * xi[1] ** 2 + 0.001 * xi[2] ** 3 + 0.003 * xi[0] * xi[1] * xi[2]
    inner_sl = (slice(3, 12),) * 3
    assert np.abs(out[inner_sl] - exact[inner_sl]).max() < 1e-12


def const_shift_closed_form(f, c_vox, steps):
    """steps applications of the tricubic shift by c_vox voxels, as a Fourier multiplier (exact for any image)."""
    n = f.shape
    F = np.fft.fftn(f)
    S = np.ones(n, dtype=complex)
    for a in range(3):
        b = math.floor(c_vox[a])
        t = c_vox[a] - b
        w = O.lagrange_weights(np.array(t))
        k = np.fft.fftfreq(n[a], 1.0 / n[a])
        Sa = sum(float(w[p]) * np.exp(2j * math.pi * k * (b + p - 1) / n[a]) for p in range(4))
        shp = [1, 1, 1]
        shp[a] = n[a]
        S = S * Sa.reshape(shp)
    return np.real(np.fft.ifftn(F * S ** steps))


def test_P4_identity_transport_is_bit_exact():
    n = (12, 16, 8)
    p = O.Problem(n, beta=1e-2, nt=4)
    m = I.trig_image(n, 0)
    assert np.array_equal(O.transport(p, m, np.zeros((3,) + n), +1), m)
    assert np.array_equal(O.transport(p, m, np.zeros((3,) + n), -1), m)


@pytest.mark.parametrize("c", [(0.37, -0.91, 0.12), (-1.3, 2.25, 0.6)])
def test_P5_constant_velocity_is_an_exact_fourier_multiplier(c):
    n = (12, 16, 20)
    nt = 4
    g = O.Grid(n)
    p = O.Problem(n, beta=1e-2, nt=nt)
    rng = np.random.default_rng(4)
    m = rng.uniform(size=n)  # any image, not band-limited
    v = np.ones((3,) + n) * np.array(c)[:, None, None, None]
    dX = O.departure(g, v, nt, +1)
    dt = 1.0 / nt
    for a in range(3):
        assert np.abs(dX[a] + c[a] * dt / g.h[a]).max() < 1e-13   # X = x - c dt exactly
    shift = [-c[a] * dt / g.h[a] for a in range(3)]
    assert rel(O.transport(p, m, v, +1), const_shift_closed_form(m, shift, nt)) < 1e-12
    # continuity-form adjoint with constant v: pure transport along -v, mass conserved exactly
    lam = O.transport(p, m, v, -1)
    assert rel(lam, const_shift_closed_form(m, [-s for s in shift], nt)) < 1e-12
    assert abs(lam.sum() - m.sum()) < 1e-11 * m.sum()


def test_P5_integer_shift_is_a_roll():
    n = (8, 12, 16)
    g = O.Grid(n)
    p = O.Problem(n, beta=1e-2, nt=2)
    m = np.random.default_rng(5).uniform(size=n)
    sh = (1, -2, 3)  # voxels per step
    v = np.stack([np.full(n, sh[a] * g.h[a] * p.nt) for a in range(3)])
    out = O.transport(p, m, v, +1)
    assert np.allclose(out, np.roll(m, shift=tuple(s * p.nt for s in sh), axis=(0, 1, 2)), rtol=0, atol=1e-13)


def test_P5_band_limited_shift_converges_fourth_order():
    errs = []
    c = np.array([0.41, -0.23, 0.17])
    for nn in (16, 32):
        n = (nn, nn, nn)
        X = coords(n)
        f = lambda x0, x1, x2: np.sin(x0) * np.cos(2 * x1) + 0.5 * np.cos(x2 + x0)
        p = O.Problem(n, beta=1e-2, nt=1)
        v = np.ones((3,) + n) * c[:, None, None, None]
        out = O.transport(p, f(*X), v, +1)
        exact = f(X[0] - c[0], X[1] - c[1], X[2] - c[2])
        errs.append(np.abs(out - exact).max())
    assert errs[1] < errs[0] / 12  # ~16x for fourth order
    assert errs[1] < 1e-3


def test_rk2_characteristics_are_second_order_and_use_the_midpoint_average():
    """Departure points of a smooth non-constant v against the exact backward flow (dense ODE solve)."""
    from scipy.integrate import solve_ivp

    n = (32, 32, 32)
    g = O.Grid(n)
    X = coords(n)
    vf = lambda x: np.stack([np.sin(x[2]) * np.cos(x[1]) * np.sin(x[1]),
                             np.sin(x[0]) * np.cos(x[2]) * np.sin(x[2]),
                             np.sin(x[1]) * np.cos(x[0]) * np.sin(x[0])])
    v = vf(np.stack(X))
    pts = [(3, 7, 11), (20, 5, 30), (12, 25, 2), (31, 0, 16)]
    errs = {}
    for nt in (2, 4, 8):
        d = O.departure(g, v, nt, +1)
        e = 0.0
        for (i, j, k) in pts:
            x0 = np.array([X[0][i, j, k], X[1][i, j, k], X[2][i, j, k]])
            sol = solve_ivp(lambda s, y: -vf(y.reshape(3, 1)).ravel(), (0, 1.0 / nt), x0, rtol=1e-12, atol=1e-13)
            xe = sol.y[:, -1]
            xd = x0 + d[:, i, j, k] * np.array(g.h)
            e = max(e, np.abs(xd - xe).max())
        errs[nt] = e
    # local error of Heun is O(dt^3); interpolation of v adds O(h^4 dt), far smaller at 32^3
    assert errs[4] < errs[2] / 5 and errs[8] < errs[4] / 5
    # a forward-Euler backtrace (dropping v(X*)) has O(dt^2) local error, i.e. visibly larger
    d_euler = np.stack([-(1.0 / 4) * v[a] / g.h[a] for a in range(3)])
    d_rk2 = O.departure(g, v, 4, +1)
    assert np.abs(d_euler - d_rk2).max() * g.h[0] > 10 * errs[4]
    # adjoint characteristics are the state ones for -v
    assert np.array_equal(O.departure(g, v, 4, -1), O.departure(g, -v, 4, +1))


def test_P6_continuity_adjoint_conserves_mass_to_discretisation_level():
    n = (32, 32, 32)
    g = O.Grid(n)
    lam0 = I.trig_image(n, 2) + 0.5
    v = I.random_velocity(n, seed=3, kmax=2, amplitude=0.4)   # compressible: div v != 0
    assert np.abs(O.divergence_spectral(g, v)).max() > 0.1
    drift = {}
    for nt in (4, 8):
        p = O.Problem(n, beta=1e-2, nt=nt, divfree=False)
        lam = O.transport(p, lam0, v, -1)
        drift[nt] = abs(lam.sum() - lam0.sum()) / lam0.sum()
    assert drift[4] < 2e-3 and drift[8] < drift[4]
    # planting a dropped source term in a copy of the step shows the pin is sensitive to it
    p = O.Problem(n, beta=1e-2, nt=4, divfree=False)
    dY = O.departure(g, v, 4, -1)
    lam = lam0.copy()
    for _ in range(4):
        lam = O.interp(lam, dY)
    assert abs(lam.sum() - lam0.sum()) / lam0.sum() > 10 * drift[4]


# ---------------------------------------------------------------------------------------------- gradient / Hessian
def small_problem(n=(16, 16, 16), divfree=False, regnorm=1, beta=1e-2, nt=4, seed=0):
    p = O.Problem(n, beta=beta, nt=nt, regnorm=regnorm, divfree=divfree)
    mT = I.trig_image(n, seed)
    mR = I.trig_image(n, seed + 100)
    return p, mT, mR


@pytest.mark.parametrize("divfree,regnorm", [(False, 1), (True, 2)])
def test_P7_closed_forms_at_zero_velocity(divfree, regnorm):
    p, mT, mR = small_problem(n=(12, 16, 20), divfree=divfree, regnorm=regnorm)
    g = p.grid
    lin = O.linearize(p, mT, np.zeros((3,) + g.n))
    gm = O.gradient_spectral(g, mT)
    g0 = O.reduced_gradient(p, lin, mR)
    assert rel(g0, O.apply_K(g, (mR - mT) * gm, divfree)) < 1e-13
    vt = I.random_velocity(g.n, seed=7, kmax=3, amplitude=1.0)
    if divfree:
        vt = O.leray(g, vt)
    Hv = O.hessvec(p, lin, vt)
    expect = p.beta * O.apply_A(g, vt, regnorm) + O.apply_K(g, (vt[0] * gm[0] + vt[1] * gm[1] + vt[2] * gm[2]) * gm,
                                                             divfree)
    assert rel(Hv, expect) < 1e-13


def test_P8_gradient_at_the_truth_is_the_regularisation_term():
    n = (16, 16, 16)
    p = O.Problem(n, beta=1e-2, nt=4, regnorm=1, divfree=False)
    mT = I.trig_image(n, 0)
    vs = I.random_velocity(n, seed=1, kmax=3, amplitude=0.3)
    mR = O.transport(p, mT, vs, +1)
    lin = O.linearize(p, mT, vs)
    gv = O.reduced_gradient(p, lin, mR)
    assert rel(gv, p.beta * O.apply_A(p.grid, vs, 1)) < 1e-13


def test_hessian_symmetric_to_rounding_at_constant_velocity():
    n = (12, 16, 20)
    p, mT, _ = small_problem(n=n)
    g = p.grid
    v = np.ones((3,) + n) * np.array([0.31, -0.17, 0.52])[:, None, None, None]
    lin = O.linearize(p, mT, v)
    x = I.random_velocity(n, seed=11, kmax=4, amplitude=1.0)
    y = I.random_velocity(n, seed=12, kmax=4, amplitude=1.0)
    a = O.inner(g, O.hessvec(p, lin, x), y)
    b = O.inner(g, x, O.hessvec(p, lin, y))
    assert abs(a - b) < 1e-12 * abs(a)


def test_hessian_symmetry_defect_shrinks_with_resolution():
    """Optimize-then-discretize: <Hx,y> - <x,Hy> is only zero up to discretisation error at a generic v."""
    defects = []
    for nn in (16, 32):
        n = (nn, nn, nn)
        p = O.Problem(n, beta=1e-2, nt=4)
        mT = I.trig_image(n, 0)
        v = I.random_velocity(n, seed=1, kmax=2, amplitude=0.3)
        lin = O.linearize(p, mT, v)
        x = I.random_velocity(n, seed=11, kmax=2, amplitude=1.0)
        y = I.random_velocity(n, seed=12, kmax=2, amplitude=1.0)
        a = O.inner(p.grid, O.hessvec(p, lin, x), y)
        b = O.inner(p.grid, x, O.hessvec(p, lin, y))
        defects.append(abs(a - b) / abs(a))
    assert defects[1] < defects[0] and defects[1] < 2e-2


def test_P11_gradient_matches_central_differences_of_the_objective():
    out = []
    for nn in (16, 32):
        n = (nn, nn, nn)
        p = O.Problem(n, beta=1e-2, nt=4, regnorm=1)
        mT = I.trig_image(n, 0)
        mR = I.trig_image(n, 100)
        v = I.random_velocity(n, seed=1, kmax=2, amplitude=0.3)
        vt = I.random_velocity(n, seed=2, kmax=2, amplitude=1.0)
        lin = O.linearize(p, mT, v)
        gv = O.reduced_gradient(p, lin, mR)
        eps = 1e-4
        Jp, _ = O.evaluate(p, mT, mR, v + eps * vt)
        Jm, _ = O.evaluate(p, mT, mR, v - eps * vt)
        fd = (Jp - Jm) / (2 * eps)
        out.append(abs(fd - O.inner(p.grid, gv, vt)) / abs(fd))
    assert out[1] < out[0] and out[1] < 2e-2
    # a sign error in the adjoint final condition would give a relative defect near 2
    assert out[0] < 0.2


def test_P8_gauss_newton_is_newton_at_the_truth():
    """At v = v* with m_R from the same discrete solve, lambda = 0, so H~ v~ is the derivative of g along v~ up to
    the discretisation error of optimize-then-discretize, which must fall quickly with resolution."""
    defect = []
    for nn in (16, 32):
        n = (nn, nn, nn)
        p = O.Problem(n, beta=1e-3, nt=4)
        mT = I.trig_image(n, 0, kmax=2)
        vs = I.random_velocity(n, seed=1, kmax=2, amplitude=0.3)
        mR = O.transport(p, mT, vs, +1)
        vt = I.random_velocity(n, seed=2, kmax=2, amplitude=1.0)
        eps = 1e-4
        gp = O.reduced_gradient(p, O.linearize(p, mT, vs + eps * vt), mR)
        gm = O.reduced_gradient(p, O.linearize(p, mT, vs - eps * vt), mR)
        Hv = O.hessvec(p, O.linearize(p, mT, vs), vt)
        defect.append(rel((gp - gm) / (2 * eps), Hv))
    assert defect[0] < 5e-2 and defect[1] < defect[0] / 4 and defect[1] < 1e-2


# ---------------------------------------------------------------------------------------------- brute force (P9)
def dense_hessian(p, lin):
    g = p.grid
    nn = 3 * g.N
    H = np.empty((nn, nn))
    e = np.zeros(nn)
    for j in range(nn):
        e[:] = 0
        e[j] = 1.0
        H[:, j] = O.hessvec(p, lin, e.reshape((3,) + g.n)).ravel()
    return H


@pytest.fixture(scope="module")
def dense8():
    n = (8, 8, 8)
    p = O.Problem(n, beta=5e-2, nt=2, regnorm=1, max_krylov=400)
    mT = I.trig_image(n, 0)
    mR = I.trig_image(n, 9)
    lin0 = O.linearize(p, mT, np.zeros((3,) + n))
    H0 = dense_hessian(p, lin0)
    return p, mT, mR, lin0, H0


def test_P9_dense_hessian_at_zero_is_symmetric_psd(dense8):
    p, mT, mR, lin0, H0 = dense8
    assert np.abs(H0 - H0.T).max() < 1e-12 * np.abs(H0).max()
    ev = np.linalg.eigvalsh(0.5 * (H0 + H0.T))
    assert ev.min() > -1e-12 * ev.max()
    # H = h^3-weighted operator: <x, H y> = cell * x^T H y must match the quadratic form of the data term
    x = np.random.default_rng(0).normal(size=H0.shape[0])
    xs = x.reshape((3,) + p.grid.n)
    gm = lin0.gradm[0]
    q = O.inner(p.grid, xs, H0.dot(x).reshape(xs.shape))
    q_expect = p.beta * O.regularization_value(p.grid, xs, 1) + O.inner(
        p.grid, (xs * gm).sum(0), (xs * gm).sum(0))
    assert abs(q - q_expect) < 1e-10 * abs(q_expect)


def test_P9_pcg_converges_to_the_dense_solve(dense8):
    p, mT, mR, lin0, H0 = dense8
    g0 = O.reduced_gradient(p, lin0, mR)
    rep = O.Report()
    vt = O.pcg(p, lin0, g0, 1e-10, rep)
    exact = np.linalg.solve(H0, -g0.ravel())
    assert rel(vt.ravel(), exact) < 1e-8
    assert rep.matvecs < 400


# ---------------------------------------------------------------------------------------------- solver (P12)
def test_P12_bookkeeping_matches_the_papers_table():
    rows = np.loadtxt(os.path.join(GOLDEN, "table3_spectral_bookkeeping.txt"))
    for _, it, mv, pde in rows:
        assert pde == 2 * mv + 2 * it + 3
    # our solver shares the initial state solve between the objective and the gradient: one solve fewer
    n = (16, 16, 16)
    p = O.Problem(n, beta=1e-2, nt=4, regnorm=1, max_gn=3)
    mT = I.trig_image(n, 0)
    mR = O.transport(p, mT, I.random_velocity(n, seed=0, kmax=3, amplitude=0.3), +1)
    v, rep = O.register(p, mT, mR)
    assert rep.pde_solves == 2 * rep.matvecs + rep.gn_iters + rep.ls_trials + 2
    assert rep.J < rep.J0 and rep.gnorm < rep.gnorm0


def test_P13_divfree_initial_guess_is_projected():
    """Under div v = 0 the control space is divergence-free (Sec. 2.2): a guess v* + grad(phi) must behave exactly
    like v*, because the Leray projection annihilates gradient fields. Restarting from the solution plus a
    gradient field therefore needs no Gauss-Newton step and returns the solution."""
    n = (12, 12, 12)
    p = O.Problem(n, beta=1e-2, nt=4, regnorm=2, divfree=True, gtol_rel=1e-3)
    mT = I.trig_image(n, 0)
    mR = O.transport(p, mT, I.random_velocity(n, seed=1, kmax=2, amplitude=0.3, divfree=True), +1)
    v, rep = O.register(p, mT, mR)
    assert rep.converged
    x1, x2, x3 = I.grid_coords(n)
    X1, X2 = x1[:, None, None] + 0 * x3, x2[None, :, None] + 0 * x3
    # phi = sin(x1) cos(2 x2): grad phi = (cos x1 cos 2x2, -2 sin x1 sin 2x2, 0)
    grad_phi = np.stack([np.cos(X1) * np.cos(2 * X2), -2 * np.sin(X1) * np.sin(2 * X2), np.zeros(n)])
    v2, rep2 = O.register(p, mT, mR, v + 0.05 * grad_phi)
    assert rep2.converged and rep2.gn_iters == 0
    assert np.abs(v2 - v).max() < 1e-12
    assert abs(rep2.gnorm0 - rep.gnorm0) < 1e-12 * rep.gnorm0


# ---------------------------------------------------------------------------------------------- H1-div model (P14)
def _h1div_problem(n=(12, 12, 12), beta=1e-2, beta_w=1e-3):
    return O.Problem(n, beta=beta, nt=4, regnorm=1, beta_w=beta_w)


def test_P14_h1div_K_inverts_the_regularisation_of_the_objective():
    """<v, K^-1 beta_v A v> must equal twice the regularisation of Eq. (2): beta_v <v, A v> + beta_w <w, (I - Lap) w>
    with w = div v, computed from the spectral divergence and Laplacian (independent of K's formula)."""
    p = _h1div_problem()
    g = p.grid
    v = I.random_velocity(g.n, seed=4, kmax=4, amplitude=1.0)
    lhs = O.inner(g, v, O.h1div_Kinv(g, p.beta * O.apply_A(g, v, 1), p.beta, p.beta_w))
    rhs = p.beta * O.regularization_value(g, v, 1) + O.regularization_h1div(g, v, p.beta_w)
    assert abs(lhs - rhs) < 1e-12 * rhs
    assert rel(O.h1div_K(g, O.h1div_Kinv(g, v, p.beta, p.beta_w), p.beta, p.beta_w), v) < 1e-13
    # K is symmetric and positive definite with eigenvalues in (0, 1]
    w = I.random_velocity(g.n, seed=5, kmax=4, amplitude=1.0)
    Kv = O.h1div_K(g, v, p.beta, p.beta_w)
    assert abs(O.inner(g, Kv, w) - O.inner(g, v, O.h1div_K(g, w, p.beta, p.beta_w))) < 1e-12 * O.norm(g, v) * O.norm(g, w)
    assert 0 < O.inner(g, Kv, v) <= O.inner(g, v, v)


def test_P14_h1div_limits_are_leray_and_identity():
    g = O.Grid((12, 10, 8))
    v = I.random_velocity(g.n, seed=6, kmax=3, amplitude=1.0)
    assert rel(O.h1div_K(g, v, 1e-2, 1e6), O.leray(g, v)) < 1e-6
    assert rel(O.h1div_K(g, v, 1e-2, 1e-12), v) < 1e-9
    # a divergence-free field is unchanged for any beta_w
    assert rel(O.h1div_K(g, O.leray(g, v), 1e-2, 3e-3), O.leray(g, v)) < 1e-13


def test_P14_h1div_closed_form_at_zero_and_gradient_fd():
    p = _h1div_problem((16, 16, 16))
    g = p.grid
    mT = I.trig_image(g.n, 0)
    mR = I.trig_image(g.n, 100)
    lin0 = O.linearize(p, mT, np.zeros((3,) + g.n))
    g0 = O.reduced_gradient(p, lin0, mR)
    gm = lin0.gradm[0]
    assert rel(g0, O.h1div_K(g, (mR - mT) * gm, p.beta, p.beta_w)) < 1e-13
    # <K^-1 g, dv> is the derivative of J (with the divergence penalty) along dv, to discretization level
    out = []
    for nn in (16, 32):
        p = _h1div_problem((nn, nn, nn))
        mT = I.trig_image(p.n, 0)
        mR = I.trig_image(p.n, 100)
        v = I.random_velocity(p.n, seed=1, kmax=2, amplitude=0.3)
        vt = I.random_velocity(p.n, seed=2, kmax=2, amplitude=1.0)
        gv = O.reduced_gradient(p, O.linearize(p, mT, v), mR)
        eps = 1e-4
        fd = (O.evaluate(p, mT, mR, v + eps * vt)[0] - O.evaluate(p, mT, mR, v - eps * vt)[0]) / (2 * eps)
        out.append(abs(fd - O.control_inner(p, gv, vt)) / abs(fd))
        plain = abs(fd - O.inner(p.grid, gv, vt)) / abs(fd)
    assert out[1] < out[0] and out[1] < 2e-2
    # the plain <g, dv> is not the derivative: without the K^-1 weighting it misses the divergence penalty
    assert plain > 5 * out[1]


def test_P14_h1div_dense_system_at_zero():
    """At v = 0 the data Hessian is symmetric, so K^-1 H (H = beta_v A + K H_data, Eq. (7)) is a symmetric PSD
    matrix, and PCG with the K^-1-weighted products reaches the dense solution of H dv = -g."""
    p = _h1div_problem((8, 8, 8), beta=1e-2, beta_w=1e-2)
    g = p.grid
    mT = I.trig_image(g.n, 0, kmax=2)
    mR = I.trig_image(g.n, 1, kmax=2)
    lin0 = O.linearize(p, mT, np.zeros((3,) + g.n))
    n = 3 * g.N
    H = np.empty((n, n))
    KH = np.empty((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        col = O.hessvec(p, lin0, e.reshape((3,) + g.n))
        H[:, i] = col.ravel()
        KH[:, i] = O.h1div_Kinv(g, col, p.beta, p.beta_w).ravel()
    assert np.abs(KH - KH.T).max() < 1e-11 * np.abs(KH).max()
    assert np.abs(H - H.T).max() > 1e-3 * np.abs(H).max()   # H itself is not symmetric
    assert np.linalg.eigvalsh(0.5 * (KH + KH.T)).min() > -1e-12 * np.abs(KH).max()
    g0 = O.reduced_gradient(p, lin0, mR)
    rep = O.Report()
    p.max_krylov = 500
    vt = O.pcg(p, lin0, g0, 1e-10, rep)
    assert rel(vt.ravel(), np.linalg.solve(H, -g0.ravel())) < 1e-7


def test_P14_h1div_register_converges():
    p = O.Problem((16, 16, 16), beta=1e-2, nt=4, regnorm=1, beta_w=1e-4, gtol_rel=1e-2)
    mT = I.trig_image(p.n, 0)
    mR = O.transport(p, mT, I.random_velocity(p.n, seed=3, kmax=2, amplitude=0.3), +1)
    v, rep = O.register(p, mT, mR)
    assert rep.converged and rep.gnorm <= 1e-2 * rep.gnorm0 and rep.J < rep.J0


# ---------------------------------------------------------------------------------------- continuation in beta (P15)
def test_P15_continuation_levels_follow_the_paper():
    """Starting at beta_v = 1 and dividing by 10: three levels for a target of 1e-2, four for 1e-3 (the level
    counts of the continuation runs of Tab. 3)."""
    assert O.continuation_levels(1e-2) == pytest.approx([1.0, 1e-1, 1e-2])
    assert O.continuation_levels(1e-3) == pytest.approx([1.0, 1e-1, 1e-2, 1e-3])
    assert O.continuation_levels(2.0) == [2.0]
    assert len(O.continuation_levels(1e-9, max_levels=4)) == 4


def test_P15_continuation_solves_each_level_and_ends_at_the_target():
    n = (16, 16, 16)
    p = O.Problem(n, beta=1e-3, nt=4, regnorm=1, beta_w=1e-4, gtol_rel=1e-2)
    mT = I.trig_image(n, 0)
    mR = O.transport(p, mT, I.random_velocity(n, seed=3, kmax=2, amplitude=0.3), +1)
    v, reps = O.register_continuation(p, mT, mR)
    assert len(reps) == 4 and all(r.converged for r in reps)
    # the last level is a solve of the target problem: its stopping test holds at v
    lin = O.linearize(p, mT, v)
    g = O.reduced_gradient(p, lin, mR)
    assert O.norm(p.grid, g) <= 1e-2 * reps[-1].gnorm0 * (1 + 1e-9)
    # a single level (start at the target) is exactly the plain solve
    v1, reps1 = O.register_continuation(p, mT, mR, beta_start=1e-3)
    v2, rep2 = O.register(p, mT, mR)
    assert len(reps1) == 1 and np.array_equal(v1, v2) and reps1[0].gn_iters == rep2.gn_iters


# ------------------------------------------------------------------------------- two-level preconditioner (P16)
def test_P16_spectral_transfer_operators():
    gf, gc = O.Grid((16, 12, 20)), O.Grid((8, 6, 10))
    rng = np.random.default_rng(0)
    # a trigonometric polynomial the coarse grid holds (|k_a| < n_c/2) restricts to its coarse samples
    x = [2 * np.pi * np.arange(m) / m for m in gf.n]
    xc = [2 * np.pi * np.arange(m) / m for m in gc.n]
    f = lambda X: 0.3 + np.cos(X[0] + 2 * X[1]) - 0.5 * np.sin(3 * X[0] - X[1] + 4 * X[2])
    F = f(np.meshgrid(*x, indexing="ij"))
    assert np.abs(O.restrict_field(gf, gc, F) - f(np.meshgrid(*xc, indexing="ij"))).max() < 1e-12
    # restriction after prolongation is the identity on coarse spectra without the coarse Nyquist modes
    G = gc.fft(rng.normal(size=gc.n))
    G2 = O.restrict_spectrum(gf, gc, O.prolong_spectrum(gf, gc, G))
    keep = O.restrict_spectrum(gf, gc, O.low_mask(gf, gc).astype(complex) * (gf.N / gc.N)) != 0
    assert np.abs(G2[keep] - G[keep]).max() < 1e-12 * np.abs(G).max() and np.all(G2[~keep] == 0)
    # prolongation after restriction is the cut-off filter F_L
    Ff = gf.fft(rng.normal(size=gf.n))
    low = O.low_mask(gf, gc)
    assert np.allclose(O.prolong_spectrum(gf, gc, O.restrict_spectrum(gf, gc, Ff)), np.where(low, Ff, 0), atol=1e-12)


def _tl_problem(n=(16, 16, 16), beta=1e-3, **kw):
    p = O.Problem(n, beta=beta, nt=4, regnorm=1, precond=1, **kw)
    mT = I.trig_image(n, 0, kmax=3)
    mR = I.trig_image(n, 1, kmax=3)
    v = I.random_velocity(n, seed=4, kmax=2, amplitude=0.2)
    cp = O.coarse_problem(p)
    lin = O.linearize(p, mT, v)
    clin = O.linearize(cp, O.restrict_field(p.grid, cp.grid, mT),
                       np.stack([O.restrict_field(p.grid, cp.grid, v[c]) for c in range(3)]))
    return p, mT, mR, v, lin, (cp, clin)


def test_P16_high_frequencies_and_zero_data_reduce_to_the_spectral_preconditioner():
    p, mT, mR, v, lin, coarse = _tl_problem()
    g = p.grid
    rep = O.Report()
    # a residual without coarse modes is only scaled: M^-1 r = (beta A)^-1 r
    r = np.random.default_rng(1).normal(size=(3,) + g.n)
    low = O.low_mask(g, coarse[0].grid)
    r = np.stack([g.ifft(np.where(low, 0, g.fft(r[c]))) for c in range(3)])
    z = O.twolevel_apply(p, coarse, r, 1e-8, rep)
    assert rel(z, O.precond(g, r, p.beta, p.regnorm)) < 1e-12
    # with a constant template the data Hessian vanishes, the coarse system is the identity, and M^-1 = (beta A)^-1
    cp = coarse[0]
    flat = O.linearize(cp, np.full(cp.grid.n, 0.4), np.zeros((3,) + cp.grid.n))
    r = np.random.default_rng(2).normal(size=(3,) + g.n)
    z = O.twolevel_apply(p, (cp, flat), r, 1e-8, rep)
    assert rel(z, O.precond(g, r, p.beta, p.regnorm)) < 1e-12


def test_P16_twolevel_pcg_reaches_the_dense_solution():
    """8^3 fine / 4^3 coarse at v = 0: PCG with the two-level preconditioner (tight outer and nested tolerances)
    solves the dense Gauss-Newton system."""
    p = O.Problem((8, 8, 8), beta=1e-3, nt=4, regnorm=1, precond=1, pc_kappa=1e-6, max_krylov=400)
    mT = I.trig_image(p.n, 0, kmax=2)
    mR = I.trig_image(p.n, 1, kmax=2)
    lin = O.linearize(p, mT, np.zeros((3,) + p.n))
    cp = O.coarse_problem(p)
    clin = O.linearize(cp, O.restrict_field(p.grid, cp.grid, mT), np.zeros((3,) + cp.grid.n))
    n = 3 * p.grid.N
    H = np.empty((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        H[:, i] = O.hessvec(p, lin, e.reshape((3,) + p.n)).ravel()
    g0 = O.reduced_gradient(p, lin, mR)
    rep = O.Report()
    vt = O.pcg(p, lin, g0, 1e-9, rep, (cp, clin))
    assert rel(vt.ravel(), np.linalg.solve(H, -g0.ravel())) < 1e-6


def test_P16_twolevel_needs_fewer_fine_matvecs_at_small_beta():
    """H2, beta 1e-4 on the phantom at 16^3: the Newton system at v = 0 solved to 1e-3 takes well under half the
    fine-grid matvecs with the two-level preconditioner, and both reach the same step within the tolerance."""
    n = (16, 16, 16)
    mT = I.brain_phantom(n, 0)
    p0 = O.Problem(n, beta=1e-4, nt=4, regnorm=2, max_krylov=500)
    mR = O.transport(p0, mT, I.random_velocity(n, seed=1, kmax=6, max_disp_voxels=0.5), +1)
    lin = O.linearize(p0, mT, np.zeros((3,) + n))
    g0 = O.reduced_gradient(p0, lin, mR)
    r1 = O.Report()
    vt1 = O.pcg(p0, lin, g0, 1e-3, r1)
    p1 = O.Problem(n, beta=1e-4, nt=4, regnorm=2, max_krylov=500, precond=1)
    cp = O.coarse_problem(p1)
    clin = O.linearize(cp, O.restrict_field(p1.grid, cp.grid, mT), np.zeros((3,) + cp.grid.n))
    r2 = O.Report()
    vt2 = O.pcg(p1, lin, g0, 1e-3, r2, (cp, clin))
    assert 2 * r2.matvecs < r1.matvecs and r2.coarse_matvecs > 0
    assert rel(vt2, vt1) < 1e-2


def test_P16_twolevel_register_converges():
    n = (16, 16, 16)
    kw = dict(beta=1e-3, nt=4, regnorm=2, divfree=True, gtol_rel=1e-2)
    mT = I.brain_phantom(n, 0)
    mR = O.transport(O.Problem(n, **kw), mT,
                     I.random_velocity(n, seed=1, kmax=4, max_disp_voxels=0.5, divfree=True), +1)
    v, rep = O.register(O.Problem(n, precond=1, **kw), mT, mR)
    assert rep.converged and rep.coarse_matvecs > 0
    assert np.abs(O.divergence_spectral(O.Grid(n), v)).max() < 1e-10 * np.abs(v).max()
