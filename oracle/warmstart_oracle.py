"""Plain FP64 CPU oracle of the learned warm start and of spectral resampling.

TEST INFRASTRUCTURE, NOT PRODUCT CODE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may import or run this module. It shares no code with the CUDA path.

The warm start is not part of the paper's method: a network proposes the initial velocity v_0 of the Gauss-Newton
loop (Alg. 1), which then runs unchanged with ||g(v = 0)|| in its relative stopping test (Sec. 2.3.2). What this
module computes is therefore fixed by the network's specification, restated here:

* Fields are channels-last float64 arrays [B][n1][n2][n3][C] on a periodic grid.
* conv3(x, w, b): periodic 3x3x3 cross-correlation, y[i, co] = b[co] + sum_{o in {-1,0,1}^3} sum_ci
  x[i + o, ci] w[co, off(o), ci], with off(o) = 9 (o1 + 1) + 3 (o2 + 1) + (o3 + 1) and i + o taken modulo n.
* pool: mean over each 2x2x2 block; up: each coarse voxel copied to its 2x2x2 block.
* Network (channel counts in/out): e0 16/16, 16/16 | pool | e1 16/32, 32/32 | pool | e2 32/64, 64/64 | pool |
  b 64/128, 128/128 | up | d2 128/64 (+ e2's output), 64/64 | up | d1 64/32 (+ e1's), 32/32 | up |
  d0 32/16 (+ e0's), 16/16 | head 16/16. ReLU after every convolution except the head; a skip is added before
  the ReLU. Input channels: (m_T, 8 (m_R - m_T), 0, ..., 0); the velocity is channels 0..2 of the head divided
  by vscale.
* Loss: mean over voxels and the 3 velocity channels of (head - vscale v)^2.
* Adam: Kingma and Ba (2015), Algorithm 1, with bias-corrected first and second moments.
* Resampling: Fourier truncation / zero padding. A mode of signed wavenumber w is kept iff 2 |w_a| < n_a on both
  grids for every axis (so Nyquist modes are dropped); the result is the trigonometric interpolant of the kept
  modes evaluated on the destination grid. With the div v = 0 constraint the Leray projection (Sec. 2.2) follows.

Backpropagation here is written out by hand from the chain rule: the adjoint of a periodic shift is the opposite
shift, the adjoint of pool spreads 1/8 of each coarse value over its block, the adjoint of up sums the block.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (16, 32, 64, 128)


def offsets():
    """The 27 neighbour offsets (o1, o2, o3) in order off = 9 (o1 + 1) + 3 (o2 + 1) + (o3 + 1)."""
    return [(o1, o2, o3) for o1 in (-1, 0, 1) for o2 in (-1, 0, 1) for o3 in (-1, 0, 1)]


def shifted(x, o):
    """s[i] = x[i + o] (periodic) over the spatial axes 1..3 of a [B][n1][n2][n3][C] array."""
    return np.roll(x, shift=(-o[0], -o[1], -o[2]), axis=(1, 2, 3))


def conv3(x, w, b=None):
    """Periodic 3x3x3 cross-correlation; x [B, n1, n2, n3, Cin], w [Cout, 27, Cin] -> [B, n1, n2, n3, Cout]."""
    y = np.zeros(x.shape[:4] + (w.shape[0],))
    for off, o in enumerate(offsets()):
        y += shifted(x, o) @ w[:, off, :].T
    if b is not None:
        y += b
    return y


def conv3_input_adjoint(dz, w):
    """Adjoint of x -> conv3(x, w): sum over offsets of the opposite shift of dz w[:, off, :]."""
    dx = np.zeros(dz.shape[:4] + (w.shape[2],))
    for off, o in enumerate(offsets()):
        dx += shifted(dz @ w[:, off, :], (-o[0], -o[1], -o[2]))
    return dx


def conv3_weight_grad(dz, x):
    """d/dw of sum(dz * conv3(x, w)): dw[co, off, ci] = sum_i dz[i, co] x[i + o, ci]."""
    cout, cin = dz.shape[-1], x.shape[-1]
    dw = np.zeros((cout, 27, cin))
    dz2 = dz.reshape(-1, cout)
    for off, o in enumerate(offsets()):
        dw[:, off, :] = dz2.T @ shifted(x, o).reshape(-1, cin)
    return dw


def pool(x):
    B, n1, n2, n3, C = x.shape
    return x.reshape(B, n1 // 2, 2, n2 // 2, 2, n3 // 2, 2, C).mean(axis=(2, 4, 6))


def pool_adjoint(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up_adjoint(dy):
    B, n1, n2, n3, C = dy.shape
    return dy.reshape(B, n1 // 2, 2, n2 // 2, 2, n3 // 2, 2, C).sum(axis=(2, 4, 6))


def relu(z):
    return np.maximum(z, 0.0)


def layer_table():
    """(Cin used, Cin stored, Cout, level, ReLU, has skip) of the 15 convolutions in execution order."""
    c0, c1, c2, c3 = CHANNELS
    return [(2, 16, c0, 0, 1, 0), (c0, c0, c0, 0, 1, 0),
            (c0, c0, c1, 1, 1, 0), (c1, c1, c1, 1, 1, 0),
            (c1, c1, c2, 2, 1, 0), (c2, c2, c2, 2, 1, 0),
            (c2, c2, c3, 3, 1, 0), (c3, c3, c3, 3, 1, 0),
            (c3, c3, c2, 2, 1, 1), (c2, c2, c2, 2, 1, 0),
            (c2, c2, c1, 1, 1, 1), (c1, c1, c1, 1, 1, 0),
            (c1, c1, c0, 0, 1, 1), (c0, c0, c0, 0, 1, 0),
            (c0, c0, 16, 0, 0, 0)]


def op_kinds():
    """Operation sequence: 'c' convolution, 'p' pool, 'u' upsample."""
    return "ccpccpccpccucc" + "ucc" + "ucc" + "c"


def unflatten(theta):
    """Host parameter vector -> [(w [Cout, 27, Cin], b [Cout])] in layer order."""
    out, k = [], 0
    for (_, cin, cout, _, _, _) in layer_table():
        nw = 27 * cin * cout
        out.append((theta[k:k + nw].reshape(cout, 27, cin).astype(np.float64),
                    theta[k + nw:k + nw + cout].astype(np.float64)))
        k += nw + cout
    assert k == theta.size
    return out


def flatten(params):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])


def num_params():
    return sum(27 * cin * cout + cout for (_, cin, cout, _, _, _) in layer_table())


DIFF_SCALE = 8.0


def pack_input(images):
    """images [B][2][n1][n2][n3] (m_T, m_R) -> x [B][n1][n2][n3][16]: m_T, 8 (m_R - m_T), then zeros."""
    B = images.shape[0]
    x = np.zeros((B,) + images.shape[2:] + (16,))
    x[..., 0] = images[:, 0]
    x[..., 1] = DIFF_SCALE * (images[:, 1] - images[:, 0])
    return x


def forward(params, images):
    """Head output [B][n1][n2][n3][16] and the saved activations (name -> array) of the network."""
    P = params
    s = {}
    s["x"] = pack_input(images)
    s["a0"] = relu(conv3(s["x"], *P[0]))
    s["s0"] = relu(conv3(s["a0"], *P[1]))
    s["p0"] = pool(s["s0"])
    s["a1"] = relu(conv3(s["p0"], *P[2]))
    s["s1"] = relu(conv3(s["a1"], *P[3]))
    s["p1"] = pool(s["s1"])
    s["a2"] = relu(conv3(s["p1"], *P[4]))
    s["s2"] = relu(conv3(s["a2"], *P[5]))
    s["p2"] = pool(s["s2"])
    s["a3"] = relu(conv3(s["p2"], *P[6]))
    s["h3"] = relu(conv3(s["a3"], *P[7]))
    s["u2"] = up(s["h3"])
    s["c2"] = relu(conv3(s["u2"], *P[8]) + s["s2"])
    s["h2"] = relu(conv3(s["c2"], *P[9]))
    s["u1"] = up(s["h2"])
    s["c1"] = relu(conv3(s["u1"], *P[10]) + s["s1"])
    s["h1"] = relu(conv3(s["c1"], *P[11]))
    s["u0"] = up(s["h1"])
    s["c0"] = relu(conv3(s["u0"], *P[12]) + s["s0"])
    s["h0"] = relu(conv3(s["c0"], *P[13]))
    out = conv3(s["h0"], *P[14])
    return out, s


def predict(params, images, vscale):
    """Velocity [B][3][n1][n2][n3] in physical units."""
    out, _ = forward(params, images)
    return np.moveaxis(out[..., :3], -1, 1) / vscale


def loss_and_grad(params, images, targets, vscale):
    """Loss (mean squared error of the scaled velocity) and its gradient, a list like params."""
    out, s = forward(params, images)
    t = vscale * np.moveaxis(targets, 1, -1)  # [B][n1][n2][n3][3]
    e = out[..., :3] - t
    loss = float(np.mean(e * e))
    d_out = np.zeros_like(out)
    d_out[..., :3] = 2.0 * e / e.size
    grads = [None] * len(params)

    def conv_back(k, dz, inp):
        """dz is d loss / d (pre-activation) of layer k; returns d loss / d inp and stores dw, db."""
        w, _ = params[k]
        grads[k] = (conv3_weight_grad(dz, inp), dz.reshape(-1, dz.shape[-1]).sum(axis=0))
        return conv3_input_adjoint(dz, w)

    def mask(d, y):
        return d * (y > 0.0)

    d_h0 = conv_back(14, d_out, s["h0"])
    d_c0 = conv_back(13, mask(d_h0, s["h0"]), s["c0"])
    dz = mask(d_c0, s["c0"])
    d_s0 = dz.copy()
    d_u0 = conv_back(12, dz, s["u0"])
    d_h1 = up_adjoint(d_u0)
    d_c1 = conv_back(11, mask(d_h1, s["h1"]), s["c1"])
    dz = mask(d_c1, s["c1"])
    d_s1 = dz.copy()
    d_u1 = conv_back(10, dz, s["u1"])
    d_h2 = up_adjoint(d_u1)
    d_c2 = conv_back(9, mask(d_h2, s["h2"]), s["c2"])
    dz = mask(d_c2, s["c2"])
    d_s2 = dz.copy()
    d_u2 = conv_back(8, dz, s["u2"])
    d_h3 = up_adjoint(d_u2)
    d_a3 = conv_back(7, mask(d_h3, s["h3"]), s["a3"])
    d_p2 = conv_back(6, mask(d_a3, s["a3"]), s["p2"])
    d_s2 = d_s2 + pool_adjoint(d_p2)
    d_a2 = conv_back(5, mask(d_s2, s["s2"]), s["a2"])
    d_p1 = conv_back(4, mask(d_a2, s["a2"]), s["p1"])
    d_s1 = d_s1 + pool_adjoint(d_p1)
    d_a1 = conv_back(3, mask(d_s1, s["s1"]), s["a1"])
    d_p0 = conv_back(2, mask(d_a1, s["a1"]), s["p0"])
    d_s0 = d_s0 + pool_adjoint(d_p0)
    d_a0 = conv_back(1, mask(d_s0, s["s0"]), s["a0"])
    conv_back(0, mask(d_a0, s["a0"]), s["x"])
    return loss, grads


def adam_step(p, g, m1, m2, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1); returns new (p, m1, m2)."""
    m1 = b1 * m1 + (1.0 - b1) * g
    m2 = b2 * m2 + (1.0 - b2) * g * g
    mhat = m1 / (1.0 - b1 ** t)
    vhat = m2 / (1.0 - b2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m1, m2


def _kept(n_src, n_dst, kmax=0):
    """Signed wavenumbers kept along a full (non-halved) axis."""
    top = (min(n_src, n_dst) - 1) // 2
    if kmax > 0:
        top = min(top, kmax)
    return np.arange(-top, top + 1)


def resample(f, n_dst, kmax=0):
    """Scalar field f on grid f.shape -> grid n_dst by Fourier truncation / zero padding; kmax > 0 also drops
    every mode with some |k_a| > kmax."""
    n_src = f.shape
    F = np.fft.fftn(f)
    G = np.zeros(tuple(n_dst), dtype=complex)
    k1, k2, k3 = (_kept(n_src[a], n_dst[a], kmax) for a in range(3))
    G[np.ix_(k1 % n_dst[0], k2 % n_dst[1], k3 % n_dst[2])] = F[np.ix_(k1 % n_src[0], k2 % n_src[1], k3 % n_src[2])]
    scale = np.prod(n_dst) / np.prod(n_src)
    return np.real(np.fft.ifftn(G)) * scale


def resample_vector(v, n_dst, project=False, kmax=0):
    out = np.stack([resample(v[c], n_dst, kmax) for c in range(v.shape[0])])
    if project:
        out = leray(out)
    return out


def leray(v):
    """Leray projection I - k' k'^T / |k'|^2 (Nyquist entries of k' set to 0; identity where k' = 0)."""
    n = v.shape[1:]
    ks = []
    for a in range(3):
        k = np.fft.fftfreq(n[a]) * n[a]
        k[n[a] // 2] = 0.0 if n[a] % 2 == 0 else k[n[a] // 2]
        ks.append(k)
    K = np.meshgrid(*ks, indexing="ij")
    V = [np.fft.fftn(v[c]) for c in range(3)]
    ksq = K[0] ** 2 + K[1] ** 2 + K[2] ** 2
    safe = np.where(ksq > 0, ksq, 1.0)
    d = (K[0] * V[0] + K[1] * V[1] + K[2] * V[2]) / safe
    return np.stack([np.real(np.fft.ifftn(V[c] - K[c] * d)) for c in range(3)])
