"""Failure paths of the solve (Sec. 2.3.2 stopping rules, Sec. 4.4 iteration caps) through the C-ABI.

Each failure is made on the host: non-finite inputs, iteration caps and Armijo constants set by the caller, or a
host-side fake of a device result (CLAIRE_FAULT). Nothing here faults, traps or hangs the GPU.
"""
import numpy as np
import pytest

import claire_inputs as I
from oracle import claire_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_04487_gb300 import build as b
    b.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


def ctx(n, prec, **kw):
    import paper_1808_04487_gb300 as pkg
    return pkg.Context(n, precision=prec, **kw)


def dev(x, prec):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", torch.float32 if prec == "f32" else torch.float64)


def rel(a, b):
    a = a.detach().cpu().double().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def problem(n=(16, 16, 16), **extra):
    kw = dict(beta=1e-2, nt=4, regnorm=1, divfree=False, pcg_rtol=0.1)
    kw.update(extra)
    p = O.Problem(n, **kw)
    mT = I.trig_image(n, 0)
    mR = O.transport(p, mT, I.random_velocity(n, seed=0, kmax=3, amplitude=0.3), +1)
    return p, kw, mT, mR


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("where", ["mT", "mR", "v"])
@pytest.mark.parametrize("value", [float("nan"), float("inf"), -float("inf")])
def test_non_finite_inputs_return_enan_and_leave_v_unchanged(prec, where, value):
    import paper_1808_04487_gb300 as pkg
    p, kw, mT, mR = problem()
    x = {"mT": dev(mT, prec), "mR": dev(mR, prec)}
    v = torch.full((3,) + p.n, 0.25, dtype=x["mT"].dtype, device="cuda")
    target = v if where == "v" else x[where]
    target.view(-1)[1234] = value
    v0 = v.clone()
    with ctx(p.n, prec, **kw) as c:
        with pytest.raises(pkg.ClaireError) as e:
            c.register(x["mT"], x["mR"], v)
        assert e.value.status == pkg.ENAN
        assert "non-finite" in str(e.value)
        # the context stays usable: a clean solve afterwards succeeds
        target.view(-1)[1234] = 0.25 if where == "v" else 0.5
        assert torch.equal(v.view(-1)[:1234], v0.view(-1)[:1234])
        _, rep, st = c.register(x["mT"], x["mR"], torch.zeros_like(v))
        assert st in ("OK", "ENOTCONV")


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_gauss_newton_cap_returns_enotconv_with_the_oracle_iterate(prec):
    """max_gn = 1: CLAIRE_ENOTCONV after one Gauss-Newton step, and v is that step's iterate (the oracle's, to
    1e-10 in FP64 and 1e-3 in FP32)."""
    p, kw, mT, mR = problem(max_gn=1, gtol_rel=1e-3)
    v_ref, rep_ref = O.register(p, mT, mR)
    assert rep_ref.status == "max_gn" and rep_ref.gn_iters == 1
    with ctx(p.n, prec, **kw) as c:
        v, rep, st = c.register(dev(mT, prec), dev(mR, prec))
    assert st == "ENOTCONV" and rep["gn_iters"] == 1 and not rep["converged"]
    assert bool(torch.isfinite(v).all())
    assert rel(v, v_ref) <= (1e-10 if prec == "f64" else 1e-3)
    assert rep["gnorm"] < rep["gnorm0"]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_armijo_failure_returns_elinesearch_with_the_last_accepted_iterate(prec):
    """Armijo with c1 = 0.9 and two trials cannot accept a Gauss-Newton step of a nearly quadratic problem (the
    model decrease at alpha = 1 and 1/2 is 0.5 and 0.375 of <g, vt>, below 0.9 alpha): CLAIRE_ELINESEARCH, and v is
    the last accepted iterate -- here the initial guess, bit for bit. The oracle stops the same way."""
    p1, kw1, mT, mR = problem(max_gn=1)
    v1, _ = O.register(p1, mT, mR)  # a nonzero starting point: one accepted step
    p, kw, _, _ = problem(armijo_c1=0.9, max_ls=2)
    _, rep_ref = O.register(p, mT, mR, v0=v1)
    assert rep_ref.status == "linesearch" and rep_ref.gn_iters == 0
    with ctx(p.n, prec, **kw) as c:
        v0 = dev(v1, prec)
        v = v0.clone()
        v, rep, st = c.register(dev(mT, prec), dev(mR, prec), v)
    assert st == "ELINESEARCH" and rep["gn_iters"] == 0 and rep["ls_trials"] == 2
    assert torch.equal(v, v0)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_pcg_breakdown_is_counted_and_the_solve_continues(prec, monkeypatch):
    """A non-positive <s, H s> (faked on the host for the first PCG iteration of every solve, CLAIRE_FAULT=
    pcg_breakdown) stops PCG with the preconditioned steepest-descent direction as the step (Alg. 2 cannot
    continue): every Gauss-Newton step then costs one matvec and counts one breakdown, and the solve still
    decreases the gradient."""
    p, kw, mT, mR = problem(max_gn=4, gtol_rel=1e-3)
    monkeypatch.setenv("CLAIRE_FAULT", "pcg_breakdown")
    with ctx(p.n, prec, **kw) as c:
        v, rep, st = c.register(dev(mT, prec), dev(mR, prec))
        assert c.pcg_graph_runs() == 0
    pcg_solves = rep["gn_iters"] + (1 if st == "ELINESEARCH" else 0)
    assert st in ("OK", "ENOTCONV", "ELINESEARCH")
    assert rep["pcg_breakdowns"] == pcg_solves == rep["matvecs"] and pcg_solves >= 1
    assert bool(torch.isfinite(v).all()) and rep["gnorm"] < rep["gnorm0"]
    monkeypatch.delenv("CLAIRE_FAULT")
    with ctx(p.n, prec, **kw) as c:
        _, rep2, _ = c.register(dev(mT, prec), dev(mR, prec))
    assert rep2["pcg_breakdowns"] == 0


def test_expired_tensor_core_wait_reports_etimeout(monkeypatch):
    """The warm-start network's bounded waits report an expiry as CLAIRE_ETIMEOUT (faked on the host with
    CLAIRE_FAULT=nn_timeout; no kernel is made to wait)."""
    import paper_1808_04487_gb300 as pkg
    L = pkg.lib()
    stream = torch.cuda.current_stream().cuda_stream
    assert L.claire_nn_status(stream) == pkg.OK
    monkeypatch.setenv("CLAIRE_FAULT", "nn_timeout")
    assert L.claire_nn_status(stream) == pkg.ETIMEOUT
    monkeypatch.delenv("CLAIRE_FAULT")
    assert L.claire_nn_status(stream) == pkg.OK
