"""GPU (sm_103a kernels through the C-ABI) against the FP64 oracle, element by element on the same seeded inputs.

Tolerances: relative L2 <= 1e-5 for FP32 and <= 1e-12 for FP64 per operator; final velocity of a full solve
relative L2 <= 1e-3 and Gauss-Newton iteration count within +-1. Bit-exact where the method is exact (identity
transport at v = 0).

One documented exception: the FP64 stand-alone gradient (claire_gradient_f64) with the H2 symbol beta |k|^4 applied
to a physical, band-limited v carries the FP64 transform's rounding, spread over all modes and multiplied by up to
beta max|k|^4 = 1.4e4 on the 40 x 36 x 42 grid: measured 1.05e-12 there (the matvec on the same grid: 5.3e-13), so
that one assertion is capped at 10x its measured error (FP64_H2_PHYS). Its data term (8.4e-15), the symbols on half
spectra (what the solver applies to its Fourier-domain vectors) and every FP32 operator meet the stated tolerance;
FP32 contexts form a growing symbol's product from an FP64 transform of the physical input (which took the FP32
gradient on that grid from 3.2e-4 to 1.2e-6).
"""
import math

import numpy as np
import pytest

import claire_inputs as I
from oracle import claire_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-12}
GRIDS = [(16, 16, 16), (12, 16, 20), (40, 36, 42), (4, 4, 4), (24, 20, 14)]


def rel(a, b):
    a = a.detach().cpu().double().numpy() if hasattr(a, "detach") else np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def dev(x, prec):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", torch.float32 if prec == "f32" else torch.float64)


def rounded(x, prec):
    """The input exactly as the GPU sees it (FP32 rounding), so both sides start from the same values."""
    return np.asarray(x, dtype=np.float32).astype(np.float64) if prec == "f32" else np.asarray(x, dtype=np.float64)


# Measured relative error of the FP64 stand-alone gradient with the H2 symbol on the 40 x 36 x 42 grid (see the
# module docstring); its assertion cap is 10x this.
FP64_H2_PHYS = {"gradient": 1.05e-12}


def phys_tol(prec, n, regnorm, what):
    """Tolerance of a stand-alone operator with a physical-space input and output."""
    if prec == "f64" and regnorm == 2 and max(n) >= 40 and what in FP64_H2_PHYS:
        return 10.0 * FP64_H2_PHYS[what]
    return TOL[prec]


def check(name, err, tol):
    print("%s: relative error %.3e (tolerance %.1e)" % (name, err, tol))
    assert err <= tol, name


def half_spectra(x, prec):
    """rfftn of each component of x as a (ncomp, n1, n2, n3//2+1, 2) device tensor (the claire_fft layout)."""
    S = np.stack([np.fft.rfftn(c) for c in x])
    return dev(np.stack([S.real, S.imag], -1), prec)


def as_complex(t):
    a = t.cpu().double().numpy()
    return a[..., 0] + 1j * a[..., 1]


def ctx(n, prec, **kw):
    import paper_1808_04487_gb300 as pkg
    return pkg.Context(n, precision=prec, **kw)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_04487_gb300 import build as b
    b.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


# ------------------------------------------------------------------------------------------------------ FFT (a3)
@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n", GRIDS)
def test_fft_forward_and_inverse(n, prec):
    f = np.random.default_rng(1).normal(size=n)
    with ctx(n, prec) as c:
        spec = c.fft(dev(f, prec))
        ref = np.fft.rfftn(f)
        got = spec[..., 0].cpu().double().numpy() + 1j * spec[..., 1].cpu().double().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL[prec]
        back = c.ifft(spec)
        assert rel(back, f) < TOL[prec]
        # the inverse of an arbitrary (Hermitian-consistent) spectrum
        g = np.random.default_rng(2).normal(size=n)
        G = np.fft.rfftn(g)
        st = torch.from_numpy(np.stack([G.real, G.imag], -1).copy()).to(spec)
        assert rel(c.ifft(st), g) < TOL[prec]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n", [(64, 96, 128), (112, 48, 160), (144, 160, 112), (192, 256, 144), (256, 32, 256),
                               (96, 112, 96), (160, 192, 144)])
def test_fft_length_specialised_passes(n, prec):
    """Every length with a compile-time specialised pass (the population grids 64..256) against numpy."""
    f = np.random.default_rng(11).normal(size=n)
    with ctx(n, prec) as c:
        spec = c.fft(dev(f, prec))
        ref = np.fft.rfftn(f)
        got = spec[..., 0].cpu().double().numpy() + 1j * spec[..., 1].cpu().double().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL[prec]
        assert rel(c.ifft(spec), f) < TOL[prec]


@pytest.mark.parametrize("n", [(64, 96, 128), (112, 48, 160), (192, 256, 144), (256, 32, 256), (96, 112, 96)])
def test_fft_tile_variants_are_bit_identical(n, monkeypatch):
    """The FFT tile autotuner only changes how many lines one CTA transforms: every forced variant (z, y, x) and
    the tuned choice give bit-identical transforms; a variant outside 0..2 is refused at context creation."""
    f = dev(np.random.default_rng(12).normal(size=n), "f32")
    g = np.random.default_rng(13).normal(size=(3,) + n)
    runs = {}
    for tiles in ("default", "1,1,1", "2,2,2", "1,2,0", "2,0,1", None):
        if tiles is None:
            monkeypatch.delenv("CLAIRE_FFT_TILES", raising=False)
        else:
            monkeypatch.setenv("CLAIRE_FFT_TILES", tiles)
        with ctx(n, "f32", regnorm=2) as c:
            spec = c.fft(f)
            runs[tiles] = (spec.clone(), c.ifft(spec.clone()), c.spectral("A", dev(g, "f32")), c.fft_tiles())
    base = runs["default"]
    assert base[3] == {"z": 0, "y": 0, "x": 0}
    assert runs["2,0,1"][3] == {"z": 2, "y": 0, "x": 1}
    assert all(v in (0, 1, 2) for v in runs[None][3].values())
    for tiles, r in runs.items():
        for a, b in zip(r[:3], base[:3]):
            assert torch.equal(a, b), tiles
    monkeypatch.setenv("CLAIRE_FFT_TILES", "3,0,0")
    with pytest.raises(RuntimeError, match="EINVAL"):
        ctx(n, "f32")


# ------------------------------------------------------------------------------------------------------ spectral ops
@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n", [(16, 16, 16), (12, 16, 20), (40, 36, 42)])
def test_spectral_operators(n, prec):
    g = O.Grid(n)
    rng = np.random.default_rng(3)
    f = rng.normal(size=n)
    v = rng.normal(size=(3,) + n)
    for regnorm in (1, 2):
        with ctx(n, prec, regnorm=regnorm) as c:
            assert rel(c.spectral("grad", dev(f, prec)), O.gradient_spectral(g, f)) < TOL[prec]
            assert rel(c.spectral("div", dev(v, prec)), O.divergence_spectral(g, v)) < TOL[prec]
            assert rel(c.spectral("leray", dev(v, prec)), O.leray(g, v)) < TOL[prec]
            check("A %s H%d %s" % (n, regnorm, prec), rel(c.spectral("A", dev(v, prec)), O.apply_A(g, v, regnorm)),
                  phys_tol(prec, n, regnorm, "A"))
            assert rel(c.spectral("lap", dev(f, prec)), O.laplacian_spectral(g, f)) < TOL[prec]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("case", [dict(regnorm=1), dict(regnorm=2, divfree=True), dict(regnorm=1, beta_w=1e-3)])
@pytest.mark.parametrize("n", [(16, 16, 16), (40, 36, 42)])
def test_symbols_on_half_spectra(n, prec, case):
    """beta A, M^-1 and K as the solver applies them to its Fourier-domain vectors (claire_symbol_*): on the half
    spectra of random fields (every mode populated) against the oracle's operators, which act on the physical
    fields; each GPU value is one or two roundings of an exact product."""
    g = O.Grid(n)
    beta = 3e-3
    p = O.Problem(n, beta=beta, **case)
    v = np.random.default_rng(15).normal(size=(3,) + n)
    V = half_spectra(v, prec)
    vr = np.fft.irfftn(as_complex(V), s=n, axes=(1, 2, 3))  # the field whose spectra the GPU received
    with ctx(n, prec, beta=beta, **case) as c:
        ref = {"betaA": beta * O.apply_A(g, vr, case["regnorm"]), "precond": O.precond(g, vr, beta, case["regnorm"]),
               "K": O.apply_Kp(p, vr)}
        for op, r in ref.items():
            R = np.stack([np.fft.rfftn(x) for x in r])
            got = as_complex(c.symbol(op, V))
            check("symbol %s %s %s %s" % (op, n, case, prec), float(np.linalg.norm(got - R) / np.linalg.norm(R)),
                  TOL[prec])
        # in place
        W = V.clone()
        c.symbol("betaA", W, out=W)
        assert torch.equal(W, c.symbol("betaA", V))


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("regnorm", [1, 2])
def test_preconditioner(prec, regnorm):
    n = (24, 20, 14)
    g = O.Grid(n)
    r = np.random.default_rng(4).normal(size=(3,) + n)
    with ctx(n, prec, beta=3e-3, regnorm=regnorm) as c:
        assert rel(c.precond(dev(r, prec)), O.precond(g, r, 3e-3, regnorm)) < TOL[prec]


# ------------------------------------------------------------------------------------------------------ SL kernels
@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n", GRIDS)
def test_interpolation_with_wrapping_displacements(n, prec):
    rng = np.random.default_rng(5)
    f = rng.normal(size=n)
    d = rng.uniform(-6.0, 6.0, size=(3,) + n)  # crosses the periodic wrap, negative and positive
    with ctx(n, prec) as c:
        assert rel(c.interp(dev(f, prec), dev(d, prec)), O.interp(f, d)) < TOL[prec]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n", [(16, 16, 16), (12, 16, 20), (40, 36, 42)])
def test_departure_points(n, prec):
    g = O.Grid(n)
    v = I.random_velocity(n, seed=6, kmax=3, amplitude=2.0)  # several voxels per step
    with ctx(n, prec, nt=4) as c:
        for sign in (+1, -1):
            assert rel(c.departure(dev(v, prec), sign), O.departure(g, v, 4, sign)) < TOL[prec]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("divfree", [False, True])
@pytest.mark.parametrize("n", [(16, 16, 16), (12, 16, 20), (40, 36, 42)])
def test_transport_state_and_adjoint(n, prec, divfree):
    p = O.Problem(n, beta=1e-2, nt=4, divfree=divfree)
    m0 = I.trig_image(n, 7)
    v = I.random_velocity(n, seed=8, kmax=3, amplitude=0.5, divfree=divfree)
    with ctx(n, prec, nt=4, divfree=divfree) as c:
        for direction in (+1, -1):
            got = c.transport(dev(m0, prec), dev(v, prec), direction)
            assert rel(got, O.transport(p, m0, v, direction)) < TOL[prec]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_identity_transport_is_bit_exact(prec):
    n = (12, 16, 20)
    m0 = I.trig_image(n, 9)
    with ctx(n, prec) as c:
        x = dev(m0, prec)
        z = torch.zeros((3,) + n, dtype=x.dtype, device="cuda")
        assert torch.equal(c.transport(x, z, +1), x)
        assert torch.equal(c.transport(x, z, -1), x)


# ------------------------------------------------------------------------------------------------------ gradient / Hessian
CASES = [dict(regnorm=1, divfree=False, nt=4), dict(regnorm=2, divfree=True, nt=4), dict(regnorm=1, divfree=False,
                                                                                          nt=2),
         dict(regnorm=1, divfree=False, nt=4, beta_w=1e-3)]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("n", [(16, 16, 16), (12, 16, 20), (40, 36, 42)])
def test_objective_gradient_hessvec(n, prec, case):
    """The reduced gradient (Eq. (5)) and the Gauss-Newton matvec (Eq. (7)-(9)) at a generic linearisation: their
    data terms (claire_gradient_data, claire_hessvec_data) and the objective at TOL, and the full physical-space
    operators (beta A applied to the physical input) at TOL, or at 10x the measured error for the FP64 H2 cases
    named in the module docstring. Every error is printed."""
    p = O.Problem(n, beta=1e-2, **case)
    mT = rounded(I.trig_image(n, 10), prec)
    mR = rounded(I.trig_image(n, 11), prec)
    v = rounded(I.random_velocity(n, seed=12, kmax=3, amplitude=0.4, divfree=case["divfree"]), prec)
    vt = rounded(I.random_velocity(n, seed=13, kmax=4, amplitude=1.0, divfree=case["divfree"]), prec)
    lin = O.linearize(p, mT, v)
    g_ref = O.reduced_gradient(p, lin, mR)
    h_ref = O.hessvec(p, lin, vt)
    gd_ref = g_ref - p.beta * O.apply_A(p.grid, v, case["regnorm"])
    hd_ref = h_ref - p.beta * O.apply_A(p.grid, vt, case["regnorm"])
    J_ref = O.objective(p, mR, lin.m[-1], v)
    tag = "%s %s %s" % (n, case, prec)
    with ctx(n, prec, beta=1e-2, **case) as c:
        gd, Jd = c.gradient_data(dev(mT, prec), dev(mR, prec), dev(v, prec), objective=True)
        check("gradient data term " + tag, rel(gd, gd_ref), TOL[prec])
        check("objective (data call) " + tag, abs(Jd - J_ref) / abs(J_ref), TOL[prec])
        g, J = c.gradient(dev(mT, prec), dev(mR, prec), dev(v, prec), objective=True)
        check("gradient " + tag, rel(g, g_ref), phys_tol(prec, n, case["regnorm"], "gradient"))
        check("objective " + tag, abs(J - J_ref) / abs(J_ref), TOL[prec])
        h = c.hessvec_cached(dev(vt, prec))
        check("matvec " + tag, rel(h, h_ref), phys_tol(prec, n, case["regnorm"], "hessvec"))
        check("matvec data term " + tag, rel(c.hessvec_data(dev(vt, prec)), hd_ref), TOL[prec])
        h2 = c.hessvec(dev(mT, prec), dev(v, prec), dev(vt, prec))
        check("matvec (relinearised) " + tag, rel(h2, h_ref), phys_tol(prec, n, case["regnorm"], "hessvec"))
        Jo = c.objective(dev(lin.m[-1], prec), dev(mR, prec), dev(v, prec))
        check("objective (stand-alone) " + tag, abs(Jo - J_ref) / J_ref, TOL[prec])


@pytest.mark.parametrize("schedule", ["plain", "tiled"])
@pytest.mark.parametrize("n", [(40, 36, 42), (24, 40, 64)])
def test_gather_schedules_match_the_oracle(schedule, n, monkeypatch):
    """Both FP32 gather schedules -- taps read from global memory, and taps read from shared-memory bricks of
    16 x 16 x 4-node tiles -- with displacements that need a brick halo of 2 or more: on 40 x 36 x 42, whose i2 and
    i3 extents end in partial tiles (bricks loaded word by word), and on 24 x 40 x 64, whose interior tiles load
    their bricks as 16-byte copies; the schedule is forced with CLAIRE_GATHER and read back from the context."""
    monkeypatch.setenv("CLAIRE_GATHER", schedule)
    case = dict(regnorm=2, divfree=True, nt=4)
    p = O.Problem(n, beta=1e-2, **case)
    mT = rounded(I.trig_image(n, 20), "f32")
    mR = rounded(I.trig_image(n, 21), "f32")
    v = rounded(I.random_velocity(n, seed=22, kmax=4, max_disp_voxels=6.0, divfree=True), "f32")
    vt = rounded(I.random_velocity(n, seed=23, kmax=4, amplitude=1.0, divfree=True), "f32")
    lin = O.linearize(p, mT, v)
    g_ref = O.reduced_gradient(p, lin, mR)
    h_ref = O.hessvec(p, lin, vt)
    gd_ref = g_ref - p.beta * O.apply_A(p.grid, v, 2)
    hd_ref = h_ref - p.beta * O.apply_A(p.grid, vt, 2)
    with ctx(n, "f32", beta=1e-2, **case) as c:
        g = c.gradient(dev(mT, "f32"), dev(mR, "f32"), dev(v, "f32"))
        sched = c.gather_schedule()
        if schedule == "tiled":
            assert min(sched.values()) >= 2
        else:
            assert set(sched.values()) == {-1}
        check("gradient %s %s" % (schedule, n), rel(g, g_ref), TOL["f32"])
        check("gradient data term %s %s" % (schedule, n),
              rel(c.gradient_data(dev(mT, "f32"), dev(mR, "f32"), dev(v, "f32")), gd_ref), TOL["f32"])
        assert c.gather_schedule() == sched
        h = c.hessvec_cached(dev(vt, "f32"))
        check("matvec %s %s" % (schedule, n), rel(h, h_ref), TOL["f32"])
        check("matvec data term %s %s" % (schedule, n), rel(c.hessvec_data(dev(vt, "f32")), hd_ref), TOL["f32"])
        m1 = c.transport(dev(mT, "f32"), dev(v, "f32"), +1)
        assert rel(m1, lin.m[-1]) < TOL["f32"]


@pytest.mark.parametrize("case", [dict(regnorm=2, divfree=True), dict(regnorm=2, divfree=True, bf16_mask=1)])
@pytest.mark.parametrize("n", [(48, 40, 64), (36, 20, 32)])
def test_tma_staged_adjoint_steps_are_bit_identical(n, case, monkeypatch):
    """The accumulating adjoint steps with their operands staged by TMA (the default wherever the bricks run and
    n3 is a multiple of 16) against the same steps with per-thread loads (CLAIRE_TMA=0): the same solve, bit for
    bit, with the bricks forced; on 36 x 20 x 32 the tiles along i2 and i1 are partial (TMA fills and clips)."""
    monkeypatch.setenv("CLAIRE_GATHER", "tiled")
    kw = dict(beta=1e-3, nt=4, gtol_rel=1e-2, max_gn=3, **case)
    mT = I.brain_phantom(n, 0)
    vs = I.random_velocity(n, seed=1, kmax=6, max_disp_voxels=3.0, divfree=True)
    runs = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("CLAIRE_TMA", mode)
        with ctx(n, "f32", **kw) as c:
            mR = c.transport(dev(mT, "f32"), dev(vs, "f32"), +1)
            v, rep, st = c.register(dev(mT, "f32"), mR)
            vt = dev(I.random_velocity(n, seed=5, kmax=4, amplitude=1.0, divfree=True), "f32")
            hd = c.hessvec_data(vt)
            g = c.gradient(dev(mT, "f32"), mR, v)
            runs[mode] = (v.cpu(), rep, hd.cpu(), g.cpu())
            assert (c.tma_steps() > 0) == (mode == "1")
    (v0, r0, h0, g0), (v1, r1, h1, g1) = runs["0"], runs["1"]
    assert r0["gn_iters"] == r1["gn_iters"] and r0["matvecs"] == r1["matvecs"]
    assert torch.equal(v0, v1) and torch.equal(h0, h1) and torch.equal(g0, g1)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_inner_product_fp64_accumulation(prec):
    n = (40, 36, 42)
    rng = np.random.default_rng(14)
    a = rng.normal(size=(3,) + n)
    b = rng.normal(size=(3,) + n)
    g = O.Grid(n)
    with ctx(n, prec) as c:
        A, B = dev(a, prec), dev(b, prec)
        ref = O.inner(g, A.cpu().double().numpy(), B.cpu().double().numpy())  # same rounded inputs
        assert abs(c.dot(A, B) - ref) <= 1e-12 * O.norm(g, a) * O.norm(g, b)


# ------------------------------------------------------------------------------------------------------ full solve
def cfg0(n=(32, 32, 32)):
    """32^3 plain method: trig image, v* |k| <= 3 amplitude 0.3, H1, beta 1e-2, nt 4, 2 GN iterations, PCG 0.1."""
    kw = dict(beta=1e-2, nt=4, regnorm=1, divfree=False, max_gn=2, pcg_rtol=0.1)
    p = O.Problem(n, **kw)
    mT = I.trig_image(n, 0)
    vstar = I.random_velocity(n, seed=0, kmax=3, amplitude=0.3)
    mR = O.transport(p, mT, vstar, +1)
    return p, kw, mT, mR


@pytest.fixture(scope="module")
def cfg0_oracle():
    p, kw, mT, mR = cfg0()
    v, rep = O.register(p, mT, mR)
    return p, kw, mT, mR, v, rep


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_register_matches_oracle(cfg0_oracle, prec):
    p, kw, mT, mR, v_ref, rep_ref = cfg0_oracle
    with ctx(p.n, prec, **kw) as c:
        v, rep, status = c.register(dev(mT, prec), dev(mR, prec))
    assert rel(v, v_ref) <= (1e-10 if prec == "f64" else 1e-3)
    assert abs(rep["gn_iters"] - rep_ref.gn_iters) <= 1
    assert abs(rep["gnorm0"] - rep_ref.gnorm0) <= 1e-5 * rep_ref.gnorm0
    if prec == "f64":
        assert rep["matvecs"] == rep_ref.matvecs and rep["pde_solves"] == rep_ref.pde_solves
    assert rep["pde_solves"] == 2 * rep["matvecs"] + rep["gn_iters"] + rep["ls_trials"] + 2


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_register_host_arrays_match_device_arrays(prec):
    p, kw, mT, mR = cfg0(n=(16, 16, 16))
    with ctx(p.n, prec, **kw) as c:
        vd, _, _ = c.register(dev(mT, prec), dev(mR, prec))
        dt = torch.float32 if prec == "f32" else torch.float64
        vh = torch.zeros((3,) + p.n, dtype=dt).pin_memory()
        vh, rep, _ = c.register_host(torch.from_numpy(mT).to(dt).pin_memory(),
                                     torch.from_numpy(mR).to(dt).pin_memory(), vh)
    assert torch.equal(vh, vd.cpu())


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("problem", ["cfg0", "h2_divfree"])
def test_device_driven_pcg_graph_is_bit_identical_to_the_host_loop(prec, problem, monkeypatch):
    """Alg. 2 run as one CUDA graph per solve (conditional WHILE node, scalars on the device) against the
    host-driven loop (CLAIRE_PCG=host): same iterates bit for bit, same counts."""
    if problem == "cfg0":
        p, kw, mT, mR = cfg0(n=(24, 20, 16))
    else:
        n = (32, 32, 32)
        kw = dict(beta=1e-3, nt=4, regnorm=2, divfree=True, max_gn=4, gtol_rel=1e-2)
        mT = I.brain_phantom(n, 0)
        vs = I.random_velocity(n, seed=1, kmax=6, max_disp_voxels=2.0, divfree=True)
        p = O.Problem(n, **kw)
        mR = O.transport(p, mT, vs, +1)
    runs = {}
    for mode in ("host", "graph"):
        if mode == "host":
            monkeypatch.setenv("CLAIRE_PCG", "host")
        else:
            monkeypatch.delenv("CLAIRE_PCG", raising=False)
        with ctx(p.n, prec, **kw) as c:
            v, rep, status = c.register(dev(mT, prec), dev(mR, prec))
            runs[mode] = (v.cpu(), rep, status, c.pcg_graph_runs())
    (vh, rh, sh, gh), (vg, rg, sg, gg) = runs["host"], runs["graph"]
    assert gh == 0 and gg >= max(1, rg["gn_iters"])  # one graph launch per PCG solve
    assert sh == sg
    for k in ("gn_iters", "matvecs", "pde_solves", "ls_trials", "pcg_breakdowns", "converged"):
        assert rh[k] == rg[k], k
    assert torch.equal(vh, vg)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("problem", ["cfg0", "h2_divfree", "h1div", "max_gn", "armijo_fails"])
def test_device_driven_solve_is_bit_identical_to_the_host_loop(prec, problem, monkeypatch):
    """The whole zero-start solve as one CUDA graph launch (Alg. 1 and Alg. 2 as conditional nodes, every scalar
    decision on the device; CLAIRE_GN=device) against the host-driven loop: same iterates bit for bit, same counts
    and the same status, also when the solve stops at max_gn (ENOTCONV) or in a failed Armijo search
    (ELINESEARCH, v = the last accepted iterate, here 0)."""
    if problem in ("cfg0", "max_gn", "armijo_fails"):
        p, kw, mT, mR = cfg0(n=(24, 20, 16))
        if problem == "max_gn":
            kw = dict(kw, max_gn=1, pcg_rtol=0.0, gtol_rel=1e-3)
        elif problem == "armijo_fails":
            kw = dict(kw, armijo_c1=0.9, max_ls=2)
    elif problem == "h2_divfree":
        n = (32, 32, 32)
        kw = dict(beta=1e-3, nt=4, regnorm=2, divfree=True, max_gn=4, gtol_rel=1e-2)
        mT = I.brain_phantom(n, 0)
        mR = O.transport(O.Problem(n, **kw), mT, I.random_velocity(n, seed=1, kmax=6, max_disp_voxels=2.0,
                                                                   divfree=True), +1)
    else:
        n = (32, 32, 32)
        kw = dict(beta=1e-3, nt=4, regnorm=1, beta_w=1e-4, gtol_rel=1e-2)
        mT, vs = I.paper_synthetic(n)
        mR = O.transport(O.Problem(n, **kw), mT, vs, +1)
    n = tuple(mT.shape)
    runs = {}
    for mode in ("host", "device"):
        monkeypatch.setenv("CLAIRE_GN", mode)
        with ctx(n, prec, **kw) as c:
            v, rep, status = c.register(dev(mT, prec), dev(mR, prec))
            runs[mode] = (v.cpu(), rep, status, c.gn_graph_runs())
    (vh, rh, sh, gh), (vd, rd, sd, gd) = runs["host"], runs["device"]
    print(problem, prec, sh, {k: rh[k] for k in ("gn_iters", "matvecs", "ls_trials")})
    assert gh == 0 and gd == 1
    assert sh == sd
    for k in ("gn_iters", "matvecs", "pde_solves", "ls_trials", "pcg_breakdowns", "converged"):
        assert rh[k] == rd[k], k
    for k in ("J", "J0", "gnorm", "gnorm0", "mismatch", "mismatch0"):
        assert rh[k] == rd[k], k
    assert torch.equal(vh, vd)
    if problem == "max_gn":
        assert sh == "ENOTCONV"
    if problem == "armijo_fails":
        assert sh == "ELINESEARCH" and float(vd.abs().max()) == 0.0


def test_device_driven_solve_does_not_depend_on_the_fixed_halo(monkeypatch):
    """The device-driven solve fixes its brick halo at capture (a fresh context has no measured displacement; halo
    2 by default). With 1.5-voxel steps a halo-2 brick misses some stencils, which then take the global taps: the
    solve is bit-identical for fixed halos 2, 3 and 5 and to the host-driven loop, whose halos follow the measured
    displacement (bricks forced, operands TMA-staged: n3 = 64)."""
    n = (48, 40, 64)
    kw = dict(beta=1e-3, nt=4, regnorm=2, divfree=True, max_gn=3, gtol_rel=1e-2)
    mT = I.brain_phantom(n, 0)
    vs = I.random_velocity(n, seed=1, kmax=6, max_disp_voxels=6.0, divfree=True)
    monkeypatch.setenv("CLAIRE_GATHER", "tiled")
    runs = {}
    for mode, halo in (("host", None), ("device", "2"), ("device", "3"), ("device", "5")):
        monkeypatch.setenv("CLAIRE_GN", mode)
        if halo is None:
            monkeypatch.delenv("CLAIRE_GN_HALO", raising=False)
        else:
            monkeypatch.setenv("CLAIRE_GN_HALO", halo)
        with ctx(n, "f32", **kw) as c:
            mR = c.transport(dev(mT, "f32"), dev(vs, "f32"), +1)
            v, rep, status = c.register(dev(mT, "f32"), mR)
            runs[(mode, halo)] = (v.cpu(), rep, status, c.gn_graph_runs(), c.tma_steps())
    vh, rh, sh, gh, th = runs[("host", None)]
    assert gh == 0 and th > 0
    for key, (v, r, st, g, t) in runs.items():
        if key[0] == "device":
            assert g == 1 and t > 0, key
        assert st == sh, key
        for k in ("gn_iters", "matvecs", "pde_solves", "ls_trials", "J", "gnorm"):
            assert r[k] == rh[k], (key, k)
        assert torch.equal(v, vh), key


def test_degenerate_identical_images_converge_immediately():
    n = (16, 16, 16)
    mT = I.trig_image(n, 0)
    with ctx(n, "f64", beta=1e-2) as c:
        v, rep, status = c.register(dev(mT, "f64"), dev(mT, "f64"))
    assert status == "OK" and rep["gn_iters"] == 0 and rep["gnorm0"] == 0.0
    assert float(v.abs().max()) == 0.0


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_register_h2_divfree_phantom_48(prec):
    """The bench's problem family (phantom, H2, div v = 0, beta 1e-3) on a 48^3 grid: FP32 and FP64 against the
    FP64 oracle (final v relative L2 <= 1e-3, GN count within 1)."""
    n = (48, 48, 48)
    kw = dict(beta=1e-3, nt=4, regnorm=2, divfree=True, max_gn=4, gtol_rel=1e-2)
    p = O.Problem(n, **kw)
    mT = I.brain_phantom(n, 0)
    vs = I.random_velocity(n, seed=1, kmax=6, max_disp_voxels=3.0, divfree=True)
    mR = O.transport(p, mT, vs, +1)
    v_ref, rep_ref = O.register(p, rounded(mT, prec), rounded(mR, prec))
    with ctx(n, prec, **kw) as c:
        v, rep, status = c.register(dev(mT, prec), dev(mR, prec))
    assert rel(v, v_ref) <= (1e-9 if prec == "f64" else 1e-3)
    assert abs(rep["gn_iters"] - rep_ref.gn_iters) <= 1
    assert abs(rep["gnorm"] / rep["gnorm0"] - rep_ref.gnorm_rel) <= 1e-3


@pytest.fixture(scope="module")
def phantom64_disp8():
    """The bench's problem family (phantom, H2, div v = 0, beta 1e-3, to 1e-2) on 64^3 with 8 voxels of maximum
    displacement (up to 2 voxels per time step of v*; the iterates reach brick halos of 2 and more). The images
    are rounded to FP32 once, so one oracle solve serves the FP32 and the FP64 comparisons."""
    n = (64, 64, 64)
    kw = dict(beta=1e-3, nt=4, regnorm=2, divfree=True, gtol_rel=1e-2)
    p = O.Problem(n, **kw)
    mT = rounded(I.brain_phantom(n, 0), "f32")
    vs = I.random_velocity(n, seed=1, kmax=6, max_disp_voxels=8.0, divfree=True)
    mR = rounded(O.transport(p, mT, vs, +1), "f32")
    v_ref, rep_ref = O.register(p, mT, mR)
    return n, kw, mT, mR, v_ref, rep_ref


@pytest.mark.parametrize("prec,schedule", [("f32", "tiled"), ("f32", "plain"), ("f64", None)])
def test_register_bench_displacement_regime_64(phantom64_disp8, prec, schedule, monkeypatch):
    """Full solve at the bench's displacement per time step against the FP64 oracle: final v within 1e-3 (FP32,
    with the brick-tiled and with the global-tap gathers forced) and 1e-9 (FP64), GN count within 1, and in FP64
    the same matvec and PDE-solve counts."""
    n, kw, mT, mR, v_ref, rep_ref = phantom64_disp8
    if schedule:
        monkeypatch.setenv("CLAIRE_GATHER", schedule)
    with ctx(n, prec, **kw) as c:
        v, rep, status = c.register(dev(mT, prec), dev(mR, prec))
        sched = c.gather_schedule()
    err = rel(v, v_ref)
    print("64^3, 8 voxels, %s %s: rel v err %.3e, GN %d vs %d, matvecs %d vs %d, schedule %s"
          % (prec, schedule, err, rep["gn_iters"], rep_ref.gn_iters, rep["matvecs"], rep_ref.matvecs, sched))
    assert status == "OK" and rep_ref.converged
    if schedule == "tiled":
        assert min(sched.values()) >= 2
    elif schedule == "plain":
        assert set(sched.values()) == {-1}
    assert abs(rep["gn_iters"] - rep_ref.gn_iters) <= 1
    assert abs(rep["gnorm0"] - rep_ref.gnorm0) <= 1e-5 * rep_ref.gnorm0
    assert err <= (1e-9 if prec == "f64" else 1e-3)
    if prec == "f64":
        assert rep["matvecs"] == rep_ref.matvecs and rep["pde_solves"] == rep_ref.pde_solves


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_register_h1div_paper_synthetic_32(prec):
    """The H1-div model (beta_v 1e-3, beta_w 1e-4, H1, to 1e-2) on the closed-form synthetic problem of Sec. 4.2:
    FP32 and FP64 against the FP64 oracle (final v relative L2 <= 1e-3, GN count within 1). This solve is very
    sensitive to rounding: perturbing m_T by 1e-15 (relative) moves the oracle's own v by 2e-7 with identical
    iteration counts, so FP64 is held to 2e-6 rather than the 1e-9 of the better-conditioned cases."""
    n = (32, 32, 32)
    kw = dict(beta=1e-3, nt=4, regnorm=1, beta_w=1e-4, gtol_rel=1e-2)
    p = O.Problem(n, **kw)
    mT, vs = I.paper_synthetic(n)
    mR = O.transport(p, mT, vs, +1)
    v_ref, rep_ref = O.register(p, rounded(mT, prec), rounded(mR, prec))
    with ctx(n, prec, **kw) as c:
        v, rep, status = c.register(dev(mT, prec), dev(mR, prec))
    assert status == "OK"
    assert abs(rep["gn_iters"] - rep_ref.gn_iters) <= 1
    assert abs(rep["gnorm0"] - rep_ref.gnorm0) <= 1e-5 * rep_ref.gnorm0
    if prec == "f64":
        assert rep["matvecs"] == rep_ref.matvecs
    assert rel(v, v_ref) <= (2e-6 if prec == "f64" else 1e-3)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_register_continuation_matches_oracle(prec):
    """Continuation in beta_v (Sec. 3.6) from 1 down to 1e-3 (four levels) on the H1-div synthetic problem. Four
    chained solves of the rounding-sensitive problem of the test above: FP64 within 2e-6, FP32 within 3e-3 (the
    1e-3 single-solve bound, grown over the levels), GN counts per level within 1."""
    n = (24, 24, 24)
    kw = dict(beta=1e-3, nt=4, regnorm=1, beta_w=1e-4, gtol_rel=1e-2)
    p = O.Problem(n, **kw)
    mT, vs = I.paper_synthetic(n)
    mR = O.transport(p, mT, vs, +1)
    v_ref, reps_ref = O.register_continuation(p, rounded(mT, prec), rounded(mR, prec))
    with ctx(n, prec, **kw) as c:
        v, reps, status = c.register_continuation(dev(mT, prec), dev(mR, prec))
        # the context's beta is the target again: a plain solve from the result needs no step
        v2, rep2, _ = c.register(dev(mT, prec), dev(mR, prec), v.clone())
    assert status == "OK" and len(reps) == len(reps_ref) == 4
    for r, rr in zip(reps, reps_ref):
        assert abs(r["gn_iters"] - rr.gn_iters) <= 1
        assert abs(r["gnorm0"] - rr.gnorm0) <= 1e-5 * rr.gnorm0
    assert rel(v, v_ref) <= (2e-6 if prec == "f64" else 3e-3)
    assert rep2["gn_iters"] <= (0 if prec == "f64" else 1)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("model", ["h2_divfree", "h1div"])
def test_register_twolevel_preconditioner_matches_oracle(prec, model):
    """The two-level preconditioner (Sec. 2.3.3; 32^3 fine, 16^3 coarse, nested CG at 0.1 eps_H) against the
    oracle's: final v within 1e-3, GN count within 1, fine matvecs equal in FP64, and a nonzero coarse matvec
    count. FP64 is held to 1e-4: the nested CG stops at a relative tolerance, so the preconditioner is a nonlinear
    map of the residual and rounding differences in the coarse iterations carry into v (measured 7e-6 and 4e-5
    for these two problems with identical fine matvec counts)."""
    n = (32, 32, 32)
    if model == "h2_divfree":
        kw = dict(beta=1e-4, nt=4, regnorm=2, divfree=True, gtol_rel=1e-2, max_gn=4)
        mT = I.brain_phantom(n, 0)
        vs = I.random_velocity(n, seed=1, kmax=6, max_disp_voxels=1.0, divfree=True)
    else:
        kw = dict(beta=1e-3, nt=4, regnorm=1, beta_w=1e-4, gtol_rel=1e-2)
        mT, vs = I.paper_synthetic(n)
    p = O.Problem(n, precond=1, **kw)
    mR = O.transport(p, mT, vs, +1)
    v_ref, rep_ref = O.register(p, rounded(mT, prec), rounded(mR, prec))
    with ctx(n, prec, precond=1, **kw) as c:
        v, rep, status = c.register(dev(mT, prec), dev(mR, prec))
    assert rep["coarse_matvecs"] > 0 and rep_ref.coarse_matvecs > 0
    assert abs(rep["gn_iters"] - rep_ref.gn_iters) <= 1
    if prec == "f64":
        assert rep["matvecs"] == rep_ref.matvecs
    assert rel(v, v_ref) <= (1e-4 if prec == "f64" else 1e-3)


def test_divfree_register_keeps_v_divergence_free():
    n = (24, 24, 24)
    kw = dict(beta=1e-3, nt=4, regnorm=2, divfree=True, max_gn=3, gtol_rel=1e-2)
    p = O.Problem(n, **kw)
    mT = I.brain_phantom(n, 0)
    vs = I.random_velocity(n, seed=1, kmax=3, max_disp_voxels=2.0, divfree=True)
    mR = O.transport(p, mT, vs, +1)
    v_ref, rep_ref = O.register(p, mT, mR)
    with ctx(n, "f64", **kw) as c:
        v, rep, status = c.register(dev(mT, "f64"), dev(mR, "f64"))
        div = c.spectral("div", v)
    assert rel(v, v_ref) < 1e-10
    assert rep["gn_iters"] == rep_ref.gn_iters
    assert float(div.abs().max()) < 1e-10 * float(v.abs().max())


# ------------------------------------------------------------------------------------------------------ full size
BIG = (256, 256, 256)


@pytest.fixture(scope="module")
def big_inputs():
    mT = I.brain_phantom(BIG, 0)
    mR = I.brain_phantom(BIG, 1)
    return mT, mR


def test_fullsize_identity_and_constant_velocity_transport(big_inputs):
    mT, _ = big_inputs
    c_phys = np.array([0.011, -0.017, 0.023])  # sub-voxel shifts on the 256^3 grid
    with ctx(BIG, "f32", nt=4) as c:
        x = dev(mT, "f32")
        z = torch.zeros((3,) + BIG, dtype=torch.float32, device="cuda")
        assert torch.equal(c.transport(x, z, +1), x)
        v = (torch.ones((3,) + BIG, dtype=torch.float64) * torch.tensor(c_phys)[:, None, None, None]).float().cuda()
        got = c.transport(x, v, +1).cpu().double().numpy()
    # closed form: nt applications of the fixed 4-tap periodic shift per axis, as a Fourier multiplier
    h = 2 * math.pi / 256
    F = np.fft.rfftn(x.cpu().double().numpy())
    for a in range(3):
        s = -np.float32(c_phys[a]).astype(np.float64) * 0.25 / h
        b = math.floor(s)
        t = s - b
        w = O.lagrange_weights(np.array(t))
        k = np.fft.fftfreq(256, 1 / 256) if a < 2 else np.arange(129)
        S = sum(float(w[p]) * np.exp(2j * math.pi * k * (b + p - 1) / 256) for p in range(4)) ** 4
        shp = [1, 1, 1]
        shp[a] = len(k)
        F = F * S.reshape(shp)
    ref = np.fft.irfftn(F, s=BIG, axes=(0, 1, 2))
    assert rel(got, ref) < 1e-5


def test_fullsize_gradient_and_hessvec_closed_forms_at_zero(big_inputs):
    """At v = 0: g = K[(mR - mT) grad mT] and H_data v~ = K[(v~ . grad mT) grad mT] (H2, div v = 0)."""
    mT, mR = big_inputs
    g = O.Grid(BIG)
    beta = 1e-3
    with ctx(BIG, "f32", beta=beta, nt=4, regnorm=2, divfree=True) as c:
        x, y = dev(mT, "f32"), dev(mR, "f32")
        zero = torch.zeros((3,) + BIG, dtype=torch.float32, device="cuda")
        gg = c.gradient(x, y, zero).cpu().double().numpy()
        vt = I.random_velocity(BIG, seed=3, kmax=6, amplitude=1.0, divfree=True)
        hv = c.hessvec_data(dev(vt, "f32")).cpu().double().numpy()
    mT32 = x.cpu().double().numpy()
    mR32 = y.cpu().double().numpy()
    gm = O.gradient_spectral(g, mT32)
    ref_g = O.leray(g, (mR32 - mT32) * gm)
    assert rel(gg, ref_g) < 1e-5
    vt32 = torch.from_numpy(vt).float().double().numpy()
    ref_h = O.leray(g, (vt32 * gm).sum(0) * gm)
    assert rel(hv, ref_h) < 1e-5


def test_fullsize_departure_points_against_the_oracle():
    """The bench's grid and displacement regime (div-free v*, |k| <= 6, 8 voxels over the unit time: 2 per step):
    the RK2 departure points of both directions on the 256^3 grid against the FP64 oracle, every node."""
    vs = I.random_velocity(BIG, seed=1, kmax=6, max_disp_voxels=8.0, divfree=True)
    g = O.Grid(BIG)
    with ctx(BIG, "f32", nt=4) as c:
        v = dev(vs, "f32")
        v64 = v.cpu().double().numpy()
        for sign in (+1, -1):
            got = c.departure(v, sign).cpu().double().numpy()
            ref = O.departure(g, v64, 4, sign)
            assert rel(got, ref) < 1e-5, sign
            assert float(np.abs(ref).max()) > 1.5  # the regime of halo-3 bricks, not a trivial shift


def test_fullsize_solve_is_bit_identical_across_gather_schedules(monkeypatch):
    """The bench's workload at 256^3 (phantom, div-free v* of 8 voxels, H2, beta 1e-3, div v = 0, n_t 4; two GN
    iterations) solved with the schedule the bench runs -- brick-tiled gathers with TMA-staged operands -- and with
    per-thread operand loads (CLAIRE_TMA=0): the same iterates bit for bit; with global taps (CLAIRE_GATHER=plain,
    float2 pair loads whose roundings are those of the scalar taps) the same counts and v within 1e-6. The brick
    and TMA paths are held to the oracle on the small grids; at full size they are held to the global taps."""
    mT = I.brain_phantom(BIG, 0)
    vs = I.random_velocity(BIG, seed=1, kmax=6, max_disp_voxels=8.0, divfree=True)
    kw = dict(beta=1e-3, nt=4, regnorm=2, divfree=True, gtol_rel=1e-2, max_gn=2)
    runs = {}
    for mode, env in (("tma", {"CLAIRE_GATHER": "tiled"}), ("bricks", {"CLAIRE_TMA": "0", "CLAIRE_GATHER": "tiled"}),
                      ("plain", {"CLAIRE_GATHER": "plain"})):
        for k in ("CLAIRE_TMA", "CLAIRE_GATHER"):
            monkeypatch.delenv(k, raising=False)
        for k, val in env.items():
            monkeypatch.setenv(k, val)
        with ctx(BIG, "f32", **kw) as c:
            mR = c.transport(dev(mT, "f32"), dev(vs, "f32"), +1)
            v, rep, status = c.register(dev(mT, "f32"), mR)
            runs[mode] = (v.cpu(), rep, status, c.tma_steps(), c.gather_schedule())
    vt, rt, st, tt, gt = runs["tma"]
    vb, rb, sb, tb, gb = runs["bricks"]
    vp, rp, sp, tp, gp = runs["plain"]
    print(gt, gb, gp, {k: rt[k] for k in ("gn_iters", "matvecs")})
    assert tt > 0 and tb == 0 and tp == 0
    assert gp["halo_x"] == -1 and gb["halo_x"] >= 2
    assert st == sb == sp
    for k in ("gn_iters", "matvecs", "pde_solves", "ls_trials", "J", "gnorm"):
        assert rt[k] == rb[k], k
    assert torch.equal(vt, vb)
    for k in ("gn_iters", "matvecs", "pde_solves", "ls_trials"):
        assert rt[k] == rp[k], k
    assert rel(vp.double(), vt.double()) < 1e-6


# ------------------------------------------------------------------------------------------------------ precision form
@pytest.fixture(scope="module")
def h2_phantom48():
    n = (48, 48, 48)
    kw = dict(beta=1e-3, nt=4, regnorm=2, divfree=True, max_gn=4, gtol_rel=1e-2)
    p = O.Problem(n, **kw)
    mT = I.brain_phantom(n, 0)
    vs = I.random_velocity(n, seed=1, kmax=6, max_disp_voxels=3.0, divfree=True)
    mR = O.transport(p, mT, vs, +1)
    return n, kw, p, rounded(mT, "f32"), rounded(mR, "f32")


def test_bf16_gradient_history_errors_against_the_oracle(h2_phantom48):
    """BF16 storage of grad m^j (claire_opts.bf16_mask bit 0): FP32 arithmetic, FP64 reductions. The stated error of
    the data terms follows from BF16 rounding (relative 2^-9 per stored value); the solve must keep GN +-1 and the
    final mismatch."""
    n, kw, p, mT, mR = h2_phantom48
    v = rounded(I.random_velocity(n, seed=12, kmax=3, max_disp_voxels=2.0, divfree=True), "f32")
    vt = rounded(I.random_velocity(n, seed=13, kmax=4, amplitude=1.0, divfree=True), "f32")
    lin = O.linearize(p, mT, v)
    hd_ref = O.hessvec(p, lin, vt) - p.beta * O.apply_A(p.grid, vt, 2)
    g_ref = O.reduced_gradient(p, lin, mR)
    gd_ref = g_ref - p.beta * O.apply_A(p.grid, v, 2)
    errs = {}
    for mask in (0, 1):
        with ctx(n, "f32", bf16_mask=mask, **kw) as c:
            c.linearize(dev(mT, "f32"), dev(v, "f32"))
            errs[("hdata", mask)] = rel(c.hessvec_data(dev(vt, "f32")), hd_ref)
            errs[("gdata", mask)] = rel(c.gradient_data(dev(mT, "f32"), dev(mR, "f32"), dev(v, "f32")), gd_ref)
            errs[("grad", mask)] = rel(c.gradient(dev(mT, "f32"), dev(mR, "f32"), dev(v, "f32")), g_ref)
    print("per-operator errors vs the FP64 oracle:", errs)
    assert errs[("hdata", 0)] < 1e-5 and errs[("gdata", 0)] < 1e-5 and errs[("grad", 0)] < 1e-5
    assert errs[("hdata", 1)] < 8 * 2.0 ** -9 and errs[("gdata", 1)] < 8 * 2.0 ** -9
    assert errs[("grad", 1)] < 8 * 2.0 ** -9
    v_ref, rep_ref = O.register(p, mT, mR)
    with ctx(n, "f32", bf16_mask=1, **kw) as c:
        v16, rep16, st = c.register(dev(mT, "f32"), dev(mR, "f32"))
    print("register bf16: rel v err %.3e, GN %d vs %d, mismatch %.6e vs %.6e" % (
        rel(v16, v_ref), rep16["gn_iters"], rep_ref.gn_iters, rep16["mismatch"], rep_ref.mismatch))
    assert abs(rep16["gn_iters"] - rep_ref.gn_iters) <= 1
    assert abs(rep16["mismatch"] - rep_ref.mismatch) <= 2e-2 * rep_ref.mismatch
    assert rel(v16, v_ref) < 2e-2


# ------------------------------------------------------------------------------------------------------ batched form
@pytest.mark.parametrize("graph", ["one", "lanes"])
def test_register_batch_matches_single_solves_on_uneven_grids(graph, monkeypatch):
    """claire_register_batch_f32 (several workers, pairs of different grids) reproduces the single-pair solves
    exactly -- same kernels and summation order on every branch -- whether the batch runs as one graph launch
    (every context's device-driven solve a branch of it; the default) or as one graph launch per context."""
    import paper_1808_04487_gb300 as pkg
    if graph == "lanes":
        monkeypatch.setenv("CLAIRE_BATCH_GRAPH", "lanes")
    else:
        monkeypatch.delenv("CLAIRE_BATCH_GRAPH", raising=False)
    kw = dict(beta=5e-3, nt=4, regnorm=1, divfree=False, gtol_rel=5e-2)
    grids = [(32, 32, 32), (24, 28, 20), (32, 32, 32), (16, 24, 32), (24, 28, 20)]
    pairs, singles = [], []
    for i, n in enumerate(grids):
        atlas = dev(I.brain_phantom(n, seed=100), "f32")
        vs = dev(I.random_velocity(n, seed=i, kmax=5, max_disp_voxels=1.5), "f32")
        with ctx(n, "f32", **kw) as c:
            mT = c.transport(atlas, vs, +1)
            v1, rep1, st1 = c.register(mT, atlas)
        singles.append((v1.clone(), rep1, st1))
        pairs.append((mT, atlas, torch.zeros((3,) + n, dtype=torch.float32, device="cuda")))
    out = pkg.register_batch(pairs, nworkers=3, **kw)
    # contexts: 3 grids, (32^3 x2, 24x28x20 x2, 16x24x32 x1) -> 2 + 2 + 1 lanes with nworkers = 3
    assert pkg.last_batch_graph_launches() == (1 if graph == "one" else 5)
    for (mT, mR, v), (rep, st), (v1, rep1, st1) in zip(pairs, out, singles):
        assert st == st1 and rep["gn_iters"] == rep1["gn_iters"] and rep["matvecs"] == rep1["matvecs"]
        assert torch.equal(v, v1)
