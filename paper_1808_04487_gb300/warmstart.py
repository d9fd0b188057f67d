"""Learned warm start: binding of the network calls of ``include/claire.h`` plus the training driver.

The network and its layers run in the library's CUDA kernels; this module marshals arguments, draws minibatch
indices and loops. The warm start is not part of the paper's method: its prediction is only the initial guess of
``Context.register``, whose relative stopping test keeps ||g(v = 0)|| (Sec. 2.3.2).

Training data are made by the plain solver: seeded phantoms m_T, band-limited divergence-free v* (|k| <= kmax),
m_R = m_T transported along v*, v = the Gauss-Newton-Krylov solution for (m_T, m_R). Images and solutions are
resampled (Fourier truncation) to the network grid.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import (ClaireError, Context, OK, ENOTCONV, ELINESEARCH, STATUS, lib, register_batch, _torch, _VP)

__all__ = ["WarmStart", "conv3_fwd", "conv3_wgrad", "weight_flip", "relu_bwd", "bias_grad", "pool_fwd", "pool_bwd",
           "up_fwd", "up_bwd", "mse", "adam", "make_training_set", "train"]


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


def _ok(st, what):
    if st != OK:
        raise ClaireError(st, what)


def _idx(idx):
    if idx is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# ---------------------------------------------------------------------------------------------------------------
# single layers (channels-last CUDA tensors; BF16 activations and weights, FP32 gradients)
def conv3_fwd(x, w, bias=None, skip=None, relu=False, y=None, yf=None, accum=False, split=True):
    """y / yf = act(conv3(x, w) + bias + skip); x [B, n1, n2, n3, Cin] bf16, w [Cout, 27, Cin] bf16. split=False
    passes no workspace, so a gathering forward runs its 27 offsets in one CTA per voxel tile (no split-K)."""
    B, n1, n2, n3, cin = x.shape
    cout = w.shape[0]
    nbytes = lib().claire_nn_fwd_workspace_bytes(B, n1, n2, n3, cout) if split else 0
    work = _torch().empty(nbytes // 4, dtype=_torch().float32, device="cuda") if nbytes else None
    _ok(lib().claire_nn_conv3_fwd(_ptr(x), _ptr(w), _ptr(bias), _ptr(skip), _ptr(y), _ptr(yf), int(bool(accum)), B,
                                  n1, n2, n3, cin, cout, int(bool(relu)), _ptr(work), _stream()), "claire_nn_conv3_fwd")
    _ok(lib().claire_nn_status(_stream()), "claire_nn_conv3_fwd: tensor-core wait timed out")
    return y, yf


def conv3_wgrad(dz, x):
    torch = _torch()
    B, n1, n2, n3, cin = x.shape
    cout = dz.shape[-1]
    nbytes = lib().claire_nn_wgrad_workspace_bytes(B, n1, n2, n3, cin, cout)
    work = torch.empty(max(nbytes // 4, 1), dtype=torch.float32, device="cuda")
    dw = torch.empty((cout, 27, cin), dtype=torch.float32, device="cuda")
    _ok(lib().claire_nn_conv3_wgrad(_ptr(dz), _ptr(x), _ptr(dw), _ptr(work), B, n1, n2, n3, cin, cout, _stream()),
        "claire_nn_conv3_wgrad")
    _ok(lib().claire_nn_status(_stream()), "claire_nn_conv3_wgrad: tensor-core wait timed out")
    return dw


def weight_flip(w):
    cout, _, cin = w.shape
    wt = _torch().empty((cin, 27, cout), dtype=w.dtype, device="cuda")
    _ok(lib().claire_nn_weight_flip(_ptr(w), _ptr(wt), cin, cout, _stream()), "claire_nn_weight_flip")
    return wt


def relu_bwd(dy, y=None):
    torch = _torch()
    dz = torch.empty_like(dy)
    dzb = torch.empty(dy.shape, dtype=torch.bfloat16, device="cuda")
    _ok(lib().claire_nn_relu_bwd(_ptr(dy), _ptr(y), _ptr(dz), _ptr(dzb), dy.numel(), _stream()),
        "claire_nn_relu_bwd")
    return dz, dzb


def bias_grad(dz):
    torch = _torch()
    C = dz.shape[-1]
    work = torch.empty(lib().claire_nn_bias_workspace_bytes(C) // 4, dtype=torch.float32, device="cuda")
    db = torch.empty(C, dtype=torch.float32, device="cuda")
    _ok(lib().claire_nn_bias_grad(_ptr(dz), dz.numel() // C, C, _ptr(db), _ptr(work), _stream()),
        "claire_nn_bias_grad")
    return db


def pool_fwd(x):
    B, n1, n2, n3, C = x.shape
    y = _torch().empty((B, n1 // 2, n2 // 2, n3 // 2, C), dtype=x.dtype, device="cuda")
    _ok(lib().claire_nn_pool_fwd(_ptr(x), _ptr(y), B, n1, n2, n3, C, _stream()), "claire_nn_pool_fwd")
    return y


def pool_bwd(dy, dx=None, accum=False):
    B, m1, m2, m3, C = dy.shape
    dx = _torch().empty((B, 2 * m1, 2 * m2, 2 * m3, C), dtype=dy.dtype, device="cuda") if dx is None else dx
    _ok(lib().claire_nn_pool_bwd(_ptr(dy), _ptr(dx), int(bool(accum)), B, 2 * m1, 2 * m2, 2 * m3, C, _stream()),
        "claire_nn_pool_bwd")
    return dx


def up_fwd(x):
    B, n1, n2, n3, C = x.shape
    y = _torch().empty((B, 2 * n1, 2 * n2, 2 * n3, C), dtype=x.dtype, device="cuda")
    _ok(lib().claire_nn_up_fwd(_ptr(x), _ptr(y), B, n1, n2, n3, C, _stream()), "claire_nn_up_fwd")
    return y


def up_bwd(dy, dx=None, accum=False):
    B, m1, m2, m3, C = dy.shape
    dx = _torch().empty((B, m1 // 2, m2 // 2, m3 // 2, C), dtype=dy.dtype, device="cuda") if dx is None else dx
    _ok(lib().claire_nn_up_bwd(_ptr(dy), _ptr(dx), int(bool(accum)), B, m1 // 2, m2 // 2, m3 // 2, C, _stream()),
        "claire_nn_up_bwd")
    return dx


def mse(pred, target, nparts=64):
    """(loss, grad) of the mean squared error over the first cu channels; pred [M, C], target [M, cu] FP32."""
    torch = _torch()
    M, C = pred.shape
    cu = target.shape[1]
    grad = torch.empty_like(pred)
    parts = torch.empty(nparts, dtype=torch.float64, device="cuda")
    _ok(lib().claire_nn_mse(_ptr(pred), _ptr(target), _ptr(grad), M, C, cu, _ptr(parts), nparts, _stream()),
        "claire_nn_mse")
    return float(parts.sum().item()), grad


def adam(p, g, m1, m2, lr, step, pb=None, b1=0.9, b2=0.999, eps=1e-8):
    _ok(lib().claire_nn_adam(_ptr(p), _ptr(g), _ptr(m1), _ptr(m2), _ptr(pb), p.numel(), float(lr), float(b1),
                             float(b2), float(eps), int(step), _stream()), "claire_nn_adam")


# ---------------------------------------------------------------------------------------------------------------
class WarmStart:
    """The warm-start network on grid n for up to `batch` samples (see claire_ws_create)."""

    def __init__(self, n=(32, 32, 32), batch=8, vscale=10.0, seed=0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        torch.cuda.init()
        self.n = tuple(int(a) for a in n)
        self.batch = int(batch)
        self.vscale = float(vscale)
        h = _VP()
        st = lib().claire_ws_create(self.batch, self.n[0], self.n[1], self.n[2], self.vscale, int(seed),
                                    ctypes.byref(h))
        _ok(st, "claire_ws_create failed for n=%s batch=%d" % (self.n, self.batch))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().claire_ws_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st, what):
        if st != OK:
            raise ClaireError(st, "%s: %s" % (what, lib().claire_ws_last_error(self._h).decode()))

    @property
    def num_params(self):
        return int(lib().claire_ws_num_params(self._h))

    def layers(self):
        out = []
        info = (ctypes.c_int * 8)()
        for i in range(lib().claire_ws_num_layers(self._h)):
            self._chk(lib().claire_ws_layer(self._h, i, info), "claire_ws_layer")
            out.append(tuple(info))
        return out

    def ops(self):
        out = []
        info = (ctypes.c_int * 4)()
        for i in range(lib().claire_ws_num_ops(self._h)):
            self._chk(lib().claire_ws_op(self._h, i, info), "claire_ws_op")
            out.append(tuple(info))
        return out

    def get_params(self):
        a = np.empty(self.num_params, dtype=np.float32)
        self._chk(lib().claire_ws_get_params(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "get_params")
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
        if a.size != self.num_params:
            raise ValueError("expected %d parameters" % self.num_params)
        self._chk(lib().claire_ws_set_params(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "set_params")

    def get_grads(self):
        a = np.empty(self.num_params, dtype=np.float32)
        self._chk(lib().claire_ws_get_grads(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "get_grads")
        return a

    def _data(self, t, ncomp, name):
        torch = _torch()
        if t.device.type != "cuda" or t.dtype != torch.float32 or tuple(t.shape[1:]) != (ncomp,) + self.n \
                or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CUDA float32 tensor [S, %d, %s]" % (name, ncomp, self.n))
        return _ptr(t)

    def forward(self, images, idx=None):
        torch = _torch()
        keep, pidx = _idx(idx)
        nb = len(keep) if keep is not None else images.shape[0]
        v = torch.empty((nb, 3) + self.n, dtype=torch.float32, device="cuda")
        self._chk(lib().claire_ws_forward_f32(self._h, self._data(images, 2, "images"), pidx, nb, _ptr(v), _stream()),
                  "claire_ws_forward_f32")
        return v

    def loss(self, images, targets, idx=None, backward=False):
        keep, pidx = _idx(idx)
        nb = len(keep) if keep is not None else images.shape[0]
        out = ctypes.c_double()
        self._chk(lib().claire_ws_loss_f32(self._h, self._data(images, 2, "images"), self._data(targets, 3, "targets"),
                                           pidx, nb, int(bool(backward)), ctypes.byref(out), _stream()),
                  "claire_ws_loss_f32")
        return out.value

    def adam_step(self, lr):
        self._chk(lib().claire_ws_adam_step(self._h, float(lr), _stream()), "claire_ws_adam_step")

    def train_step(self, images, targets, idx, lr, want_loss=True):
        keep, pidx = _idx(idx)
        out = ctypes.c_double()
        self._chk(lib().claire_ws_train_step_f32(self._h, self._data(images, 2, "images"),
                                                 self._data(targets, 3, "targets"), pidx, len(keep), float(lr),
                                                 ctypes.byref(out) if want_loss else None, _stream()),
                  "claire_ws_train_step_f32")
        return out.value if want_loss else None

    def predict(self, ctx, mT, mR, out=None, kmax=0):
        """Velocity on ctx's grid for (mT, mR), usable as the initial guess of ctx.register; kmax > 0 keeps only
        modes with every |k_i| <= kmax."""
        out = ctx.empty_vector() if out is None else out
        self._chk(lib().claire_ws_predict_f32(self._h, ctx.handle, ctx._s(mT, "mT"), ctx._s(mR, "mR"),
                                              ctx._v(out, "v"), int(kmax), _stream()), "claire_ws_predict_f32")
        return out


# ---------------------------------------------------------------------------------------------------------------
def make_training_set(count, n_solve=(128, 128, 128), n_net=(32, 32, 32), seed=0, phantoms=64, kmax=6,
                      max_disp_voxels=None, beta=1e-3, regnorm=2, divfree=True, nt=4, gtol_rel=1e-2, chunk=64,
                      nworkers=4, log=None):
    """(images [count, 2, *n_net], targets [count, 3, *n_net], stats) made by the plain solver on n_solve.

    Sample s: m_T = phantom(seed + s % phantoms); v* = random divergence-free field (|k| <= kmax, largest
    displacement max_disp_voxels voxels of n_solve, default 8 n_solve / 256) drawn on n_net and resampled exactly;
    m_R = m_T transported along v*; the target is the solver's v for (m_T, m_R).
    """
    import claire_inputs as I
    torch = _torch()
    n_solve, n_net = tuple(n_solve), tuple(n_net)
    if max_disp_voxels is None:
        max_disp_voxels = 8.0 * max(n_solve) / 256.0
    disp_net = max_disp_voxels * max(n_net) / max(n_solve)
    ctx_s = Context(n_solve, "f32", beta=beta, nt=nt, regnorm=regnorm, divfree=divfree, gtol_rel=gtol_rel)
    ctx_n = Context(n_net, "f32")
    images = torch.empty((count, 2) + n_net, dtype=torch.float32, device="cuda")
    targets = torch.empty((count, 3) + n_net, dtype=torch.float32, device="cuda")
    atlas = {}
    stats = {"gn_iters": [], "matvecs": [], "converged": 0, "seconds": 0.0}
    t0 = time.time()
    for c0 in range(0, count, chunk):
        pairs = []
        for s in range(c0, min(count, c0 + chunk)):
            ph = s % phantoms
            if ph not in atlas:
                atlas[ph] = torch.from_numpy(I.brain_phantom(n_solve, seed=seed + 10007 * ph)).float().cuda()
            mT = atlas[ph]
            vs = I.random_velocity(n_net, seed=seed + 7919 * s + 1, kmax=kmax, max_disp_voxels=disp_net, divfree=True)
            vs = ctx_n.resample_to(ctx_s, torch.from_numpy(vs).float().cuda().contiguous())
            mR = ctx_s.transport(mT, vs, +1)
            pairs.append((mT, mR, torch.zeros((3,) + n_solve, dtype=torch.float32, device="cuda")))
        reps = register_batch(pairs, nworkers=nworkers, beta=beta, nt=nt, regnorm=regnorm, divfree=divfree,
                              gtol_rel=gtol_rel)
        for k, ((mT, mR, v), (rep, status)) in enumerate(zip(pairs, reps)):
            s = c0 + k
            ctx_s.resample_to(ctx_n, mT, out=images[s, 0])
            ctx_s.resample_to(ctx_n, mR, out=images[s, 1])
            ctx_s.resample_to(ctx_n, v, out=targets[s])
            stats["gn_iters"].append(rep["gn_iters"])
            stats["matvecs"].append(rep["matvecs"])
            stats["converged"] += int(status == "OK")
        if log:
            log("training set: %d / %d solved (%.1f s)" % (min(count, c0 + chunk), count, time.time() - t0))
    torch.cuda.synchronize()
    stats["seconds"] = time.time() - t0
    ctx_s.close()
    ctx_n.close()
    return images, targets, stats


def cube_symmetry(images, targets, flips, perm):
    """One symmetry of the periodic cube applied to a minibatch (a data transform, no arithmetic of the method): the
    reflection x_a -> -x_a (index i -> (n - i) mod n) for each axis a with flips[a], then the axis permutation
    (new axis c = old axis perm[c]). Images [B, C, n, n, n] transform as scalars; a velocity [B, 3, n, n, n] as a
    vector: a reflected axis negates its component, a permutation reorders the components. The registration
    problem (periodic domain, isotropic regularisation, Leray projection) is equivariant under these maps, so the
    transformed pair's solution is the transformed solution."""
    torch = _torch()
    for a in range(3):
        if flips[a]:
            d = 2 + a
            images = torch.roll(torch.flip(images, [d]), 1, d)
            targets = torch.roll(torch.flip(targets, [d]), 1, d)
            targets[:, a] = -targets[:, a]
    order = (0, 1) + tuple(2 + p for p in perm)
    images = images.permute(order).contiguous()
    targets = targets.permute(order)[:, list(perm)].contiguous()
    return images, targets


def train(ws, images, targets, steps, lr=1e-3, lr_final=3e-5, seed=0, val=None, log=None, log_every=200,
          augment=False):
    """Adam with a cosine learning-rate schedule over random minibatches of ws.batch rows.

    augment: each minibatch goes through a random symmetry of the periodic cube (cube_symmetry; permutations only
    on cubic grids). val = (images, targets) is evaluated every log_every steps. Returns the per-step training
    losses."""
    rng = np.random.default_rng(seed)
    S = images.shape[0]
    cubic = len(set(images.shape[2:])) == 1
    losses = []
    t0 = time.time()
    for it in range(steps):
        idx = rng.choice(S, size=min(ws.batch, S), replace=False)
        a = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * it / max(1, steps)))
        want = (it % 20 == 0) or it == steps - 1
        if augment:
            flips = rng.integers(0, 2, size=3)
            perm = tuple(rng.permutation(3)) if cubic else (0, 1, 2)
            ti = _torch().as_tensor(idx, device=images.device)
            bi, bt = cube_symmetry(images.index_select(0, ti), targets.index_select(0, ti), flips, perm)
            l = ws.train_step(bi, bt, np.arange(len(idx)), a, want_loss=want)
        else:
            l = ws.train_step(images, targets, idx, a, want_loss=want)
        if want:
            losses.append((it, l))
        if log and (it % log_every == 0 or it == steps - 1):
            msg = "step %d loss %.4e lr %.2e (%.1f s)" % (it, l if l is not None else float("nan"), a,
                                                         time.time() - t0)
            if val is not None:
                msg += " val %.4e" % evaluate(ws, *val)
            log(msg)
    return losses


def evaluate(ws, images, targets):
    """Mean loss over all rows (batches of ws.batch)."""
    S = images.shape[0]
    tot = 0.0
    for b0 in range(0, S, ws.batch):
        idx = np.arange(b0, min(S, b0 + ws.batch))
        tot += ws.loss(images, targets, idx) * len(idx)
    return tot / S
