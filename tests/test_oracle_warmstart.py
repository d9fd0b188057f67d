"""Pins of the warm-start / resampling oracle against facts that do not come from the oracle itself.

W1 conv3 equals a brute-force sum written with explicit index loops (tiny case).
W2 single-channel conv3 equals scipy.ndimage.correlate with periodic ('wrap') boundaries.
W3 conv3_input_adjoint is the adjoint of conv3: <conv3(x, w), z> = <x, adjoint(z)>.
W4 conv3_weight_grad is the derivative in w: <dw, W> = <conv3(x, W), z> for any W (conv3 is linear in w).
W5 pool / up: adjoint pairs, pool(up(x)) = x, pool of a constant is that constant.
W6 the whole network's gradient matches central finite differences along random directions.
W7 Adam: first step moves every coordinate by lr sign(g) (bias correction), zero gradient leaves p unchanged.
W8 resampling reproduces a trigonometric polynomial sampled directly on the other grid; Nyquist modes dropped.
W9 the Leray projection of a gradient field is zero and of a curl field is the field itself.
"""
import itertools

import numpy as np
import pytest

from oracle import warmstart_oracle as W


def rng(seed=0):
    return np.random.default_rng(seed)


def test_W1_conv3_brute_force():
    r = rng(1)
    B, n, cin, cout = 2, (3, 4, 5), 2, 3
    x = r.standard_normal((B,) + n + (cin,))
    w = r.standard_normal((cout, 27, cin))
    b = r.standard_normal(cout)
    y = W.conv3(x, w, b)
    ref = np.zeros_like(y)
    for bb, i1, i2, i3, co in itertools.product(range(B), range(n[0]), range(n[1]), range(n[2]), range(cout)):
        s = b[co]
        for o1, o2, o3 in itertools.product((-1, 0, 1), repeat=3):
            off = 9 * (o1 + 1) + 3 * (o2 + 1) + (o3 + 1)
            j1, j2, j3 = (i1 + o1) % n[0], (i2 + o2) % n[1], (i3 + o3) % n[2]
            for ci in range(cin):
                s += x[bb, j1, j2, j3, ci] * w[co, off, ci]
        ref[bb, i1, i2, i3, co] = s
    assert np.max(np.abs(y - ref)) < 1e-12


def test_W2_conv3_matches_scipy_correlate():
    ndimage = pytest.importorskip("scipy.ndimage")
    r = rng(2)
    f = r.standard_normal((6, 7, 8))
    k = r.standard_normal((3, 3, 3))
    w = k.reshape(1, 27, 1)
    y = W.conv3(f[None, ..., None], w)[0, ..., 0]
    ref = ndimage.correlate(f, k, mode="wrap")
    assert np.max(np.abs(y - ref)) < 1e-12


def test_W3_input_adjoint():
    r = rng(3)
    x = r.standard_normal((2, 4, 6, 5, 3))
    z = r.standard_normal((2, 4, 6, 5, 4))
    w = r.standard_normal((4, 27, 3))
    lhs = np.sum(W.conv3(x, w) * z)
    rhs = np.sum(x * W.conv3_input_adjoint(z, w))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_W4_weight_grad_is_derivative():
    r = rng(4)
    x = r.standard_normal((1, 5, 4, 6, 3))
    z = r.standard_normal((1, 5, 4, 6, 2))
    dw = W.conv3_weight_grad(z, x)
    for s in range(3):
        Wd = rng(40 + s).standard_normal((2, 27, 3))
        assert abs(np.sum(dw * Wd) - np.sum(W.conv3(x, Wd) * z)) < 1e-10 * np.sum(np.abs(dw * Wd))


def test_W5_pool_up():
    r = rng(5)
    x = r.standard_normal((2, 4, 6, 8, 3))
    y = r.standard_normal((2, 2, 3, 4, 3))
    assert abs(np.sum(W.pool(x) * y) - np.sum(x * W.pool_adjoint(y))) < 1e-12
    assert abs(np.sum(W.up(y) * x) - np.sum(y * W.up_adjoint(x))) < 1e-12
    assert np.max(np.abs(W.pool(W.up(y)) - y)) < 1e-15
    assert np.max(np.abs(W.pool(np.full_like(x, 0.7)) - 0.7)) < 1e-15
    # pool of a field that varies along axis 3 only: the mean of each pair
    f = np.zeros((1, 2, 2, 4, 1))
    f[..., :, 0] = np.array([1.0, 3.0, 5.0, 9.0])
    assert np.allclose(W.pool(f)[0, 0, 0, :, 0], [2.0, 7.0])


def _small_problem(seed=6):
    r = rng(seed)
    n = (8, 8, 8)
    images = r.uniform(0, 1, size=(2, 2) + n)
    targets = 0.1 * r.standard_normal((2, 3) + n)
    params = []
    for (cin_used, cin, cout, _, _, _) in W.layer_table():
        w = r.standard_normal((cout, 27, cin)) * np.sqrt(2.0 / (27 * cin_used))
        w[:, :, cin_used:] = 0.0
        params.append((w, 0.1 * r.standard_normal(cout)))
    return params, images, targets


def test_W6_network_gradient_finite_differences():
    params, images, targets = _small_problem()
    vscale = 5.0
    loss, grads = W.loss_and_grad(params, images, targets, vscale)
    assert loss > 0
    theta = W.flatten(params)
    g = W.flatten(grads)
    assert theta.size == W.num_params()
    for s in range(3):
        d = rng(60 + s).standard_normal(theta.size)
        d /= np.linalg.norm(d)
        eps = 1e-5
        lp, _ = W.loss_and_grad(W.unflatten(theta + eps * d), images, targets, vscale)
        lm, _ = W.loss_and_grad(W.unflatten(theta - eps * d), images, targets, vscale)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-5 * max(abs(fd), 1e-3 * np.linalg.norm(g))
    # single coordinates of the first and last layers (the input packing and the head's channel selection)
    for k in (5, theta.size - 3, theta.size - 20):
        e = np.zeros_like(theta)
        e[k] = 1.0
        lp, _ = W.loss_and_grad(W.unflatten(theta + 1e-5 * e), images, targets, vscale)
        lm, _ = W.loss_and_grad(W.unflatten(theta - 1e-5 * e), images, targets, vscale)
        assert abs((lp - lm) / 2e-5 - g[k]) <= 1e-6 + 1e-4 * abs(g[k])


def test_W6b_unused_head_channels_have_zero_gradient():
    params, images, targets = _small_problem(7)
    _, grads = W.loss_and_grad(params, images, targets, 3.0)
    dw, db = grads[14]
    assert np.all(dw[3:] == 0.0) and np.all(db[3:] == 0.0)
    assert np.linalg.norm(dw[:3]) > 0
    # zero input channels 2..15 of the first layer receive gradient only through zero inputs
    assert np.all(grads[0][0][:, :, 2:] == 0.0)


def test_W7_adam_first_step():
    r = rng(8)
    p = r.standard_normal(50)
    g = r.standard_normal(50)
    g[::7] = 0.0
    q, m1, m2 = W.adam_step(p, g, np.zeros(50), np.zeros(50), t=1, lr=1e-2)
    step = p - q
    nz = g != 0
    assert np.allclose(step[nz], 1e-2 * np.sign(g[nz]), rtol=1e-6)
    assert np.all(step[~nz] == 0.0)


def _trig(n, coeffs):
    """sum over (k, a, b) of a cos(k.x) + b sin(k.x) on the grid n of [0, 2 pi)^3."""
    x = [2 * np.pi * np.arange(m) / m for m in n]
    X = np.meshgrid(*x, indexing="ij")
    f = np.zeros(n)
    for (k1, k2, k3), a, b in coeffs:
        ph = k1 * X[0] + k2 * X[1] + k3 * X[2]
        f += a * np.cos(ph) + b * np.sin(ph)
    return f


def test_W8_resample_trig_polynomial():
    coeffs = [((0, 0, 0), 0.3, 0.0), ((1, -2, 3), 0.5, -0.2), ((4, 0, -1), -0.7, 0.4), ((-3, 5, 2), 0.1, 0.9)]
    for n_src, n_dst in (((12, 16, 10), (20, 18, 24)), ((24, 20, 14), (12, 12, 12)), ((16, 16, 16), (16, 16, 16))):
        f = _trig(n_src, coeffs)
        g = W.resample(f, n_dst)
        assert np.max(np.abs(g - _trig(n_dst, coeffs))) < 1e-12
    # a Nyquist mode of the smaller grid is dropped
    f = _trig((16, 16, 16), [((8, 0, 0), 1.0, 0.0), ((1, 1, 1), 0.5, 0.0)])
    g = W.resample(f, (16, 16, 16))
    assert np.max(np.abs(g - _trig((16, 16, 16), [((1, 1, 1), 0.5, 0.0)]))) < 1e-12
    g = W.resample(_trig((32, 32, 32), [((8, 2, 0), 1.0, 0.0)]), (16, 16, 16))
    assert np.max(np.abs(g)) < 1e-12
    # a low-pass cutoff keeps exactly the modes with every |k_a| <= kmax
    f = _trig((24, 20, 16), coeffs)
    g = W.resample(f, (24, 20, 16), kmax=3)
    low = [c for c in coeffs if max(abs(k) for k in c[0]) <= 3]
    assert np.max(np.abs(g - _trig((24, 20, 16), low))) < 1e-12


def test_W9_leray():
    n = (12, 10, 8)
    phi = _trig(n, [((1, 2, -1), 0.7, 0.3), ((3, 0, 2), -0.4, 0.5)])
    # gradient field of phi (analytic): d/dx_a of cos(k.x) = -k_a sin(k.x)
    grad = np.stack([_trig(n, [((1, 2, -1), 0.3 * ka, -0.7 * ka) for ka in [(1, 2, -1)[a]]] +
                              [((3, 0, 2), 0.5 * kb, 0.4 * kb) for kb in [(3, 0, 2)[a]]]) for a in range(3)])
    assert np.max(np.abs(W.leray(grad))) < 1e-12
    # a divergence-free field (v1 depends on x2 only, etc.) is unchanged
    v = np.stack([_trig(n, [((0, 1, 0), 0.5, 0.2)]), _trig(n, [((0, 0, 2), 0.3, 0.0)]),
                  _trig(n, [((1, 0, 0), 0.0, 0.8)])])
    assert np.max(np.abs(W.leray(v) - v)) < 1e-12
