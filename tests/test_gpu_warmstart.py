"""GPU parity of the warm-start layers, network, resampling and warm-started solve against the FP64 oracle.

Tolerances. Inputs and weights are BF16-representable, so products are exact and the only error of a convolution
is FP32 accumulation: at most one rounding of the accumulator per 16-term tensor-core step, i.e. below
(27 Cin / 16) 2^-23 sum|terms| ~ 3e-5 sum|terms| for Cin = 128 even if every rounding truncates; the test allows
4e-5 sum|terms| per element. A BF16 output adds half an ulp, 2^-9 |y|. The whole network stores every activation
in BF16 and feeds BF16 gradients to the tensor cores: each of its 15 layers adds a relative perturbation of about
2^-9, so loss and gradients are compared normwise at 2e-2 (roughly 15 x 2^-9 with margin; measured values are
printed by the test on failure).
"""
import numpy as np
import pytest

from oracle import warmstart_oracle as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def ws_mod():
    _need_gpu()
    from paper_1808_04487_gb300 import warmstart as WS
    return WS


def bf16(a):
    """numpy float64 -> (CUDA bf16 tensor, the same values as float64)."""
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.cuda(), t.float().numpy().astype(np.float64)


def f32(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    return t.cuda(), t.numpy().astype(np.float64)


def host(t):
    return t.float().cpu().numpy().astype(np.float64)


CONV_CASES = [((2, 6, 5, 8), 16, 16), ((1, 3, 4, 4), 32, 48), ((2, 6, 5, 8), 64, 128), ((1, 8, 6, 10), 128, 64),
              ((3, 4, 4, 4), 48, 80), ((1, 4, 8, 6), 16, 112), ((2, 4, 2, 6), 96, 32)]
# grids whose forward convolution runs from a shared-memory halo (n3 a multiple of 8, n2 of 16, Cin <= 64, the
# weights within 108 KB)
HALO_CASES = [((2, 4, 16, 8), 16, 16), ((1, 3, 16, 16), 32, 64), ((2, 2, 32, 8), 64, 32), ((1, 4, 16, 8), 16, 128),
              ((1, 2, 16, 24), 48, 16)]
# grids with enough tiles (Cin <= 32; n1 even and at least 4 x 152 two-plane CTAs, or n1 a multiple of 4 and at
# least 3 x 152 four-plane CTAs, as the last case) for two or four tile planes per CTA
HALO_TZ2_CASES = [((4, 38, 16, 64), 16, 16), ((2, 38, 16, 128), 32, 16), ((4, 32, 16, 128), 16, 16)]


@pytest.mark.parametrize("shape,cin,cout", CONV_CASES + HALO_CASES + HALO_TZ2_CASES)
def test_conv3_forward(ws_mod, shape, cin, cout):
    r = np.random.default_rng(cin * 1000 + cout)
    xg, x = bf16(r.standard_normal(shape + (cin,)))
    wg, w = bf16(r.standard_normal((cout, 27, cin)) / np.sqrt(27 * cin))
    bg, b = f32(r.standard_normal(cout) * 0.1)
    sg, s = bf16(r.standard_normal(shape + (cout,)) * 0.5)
    yf = torch.empty(shape + (cout,), dtype=torch.float32, device="cuda")
    y = torch.empty(shape + (cout,), dtype=torch.bfloat16, device="cuda")
    ws_mod.conv3_fwd(xg, wg, bias=bg, skip=sg, relu=False, y=y, yf=yf)
    ref = W.conv3(x, w, b) + s
    mag = W.conv3(np.abs(x), np.abs(w)) + np.abs(b) + np.abs(s)
    err = np.abs(host(yf) - ref)
    assert np.all(err <= 4e-5 * mag), err.max()
    assert np.all(np.abs(host(y) - ref) <= 2.0 ** -8 * np.abs(ref) + 4e-5 * mag)
    # ReLU and accumulation into an existing FP32 output
    base = torch.from_numpy(r.standard_normal(shape + (cout,)).astype(np.float32)).cuda()
    acc = base.clone()
    ws_mod.conv3_fwd(xg, wg, bias=bg, relu=True, yf=acc, accum=True)
    ref2 = host(base) + W.relu(W.conv3(x, w, b))
    assert np.all(np.abs(host(acc) - ref2) <= 4e-5 * (mag + np.abs(host(base))))


@pytest.mark.parametrize("shape,cin,cout", HALO_CASES + HALO_TZ2_CASES)
def test_conv3_forward_from_halo_is_bit_identical_to_the_gather_kernel(ws_mod, shape, cin, cout, monkeypatch):
    """The forward convolution from a shared-memory halo (A operands as descriptors into the halo) against the
    kernel that gathers each offset's neighbour rows (CLAIRE_CONV=gather, all 27 offsets in one CTA per tile): the
    same MMAs in the same K order, so the same bits, with bias, skip, ReLU and FP32 accumulation. (The halo form
    also serves the grids whose gathering forward would split the offsets over CTAs; those agree to rounding, and
    both are held to the oracle by test_conv3_forward.)"""
    r = np.random.default_rng(7 + cin + cout)
    xg, _ = bf16(r.standard_normal(shape + (cin,)))
    wg, _ = bf16(r.standard_normal((cout, 27, cin)) / np.sqrt(27 * cin))
    bg, _ = f32(r.standard_normal(cout) * 0.1)
    sg, _ = bf16(r.standard_normal(shape + (cout,)) * 0.5)
    base = torch.from_numpy(r.standard_normal(shape + (cout,)).astype(np.float32)).cuda()
    outs = []
    for mode in ("gather", "halo"):
        if mode == "gather":
            monkeypatch.setenv("CLAIRE_CONV", "gather")
        else:
            monkeypatch.delenv("CLAIRE_CONV", raising=False)
        y = torch.empty(shape + (cout,), dtype=torch.bfloat16, device="cuda")
        acc = base.clone()
        ws_mod.conv3_fwd(xg, wg, bias=bg, skip=sg, relu=True, y=y, yf=acc, accum=True, split=False)
        outs.append((y.cpu(), acc.cpu()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("shape,cin,cout", CONV_CASES[:5] + HALO_CASES[:3])
def test_conv3_weight_and_input_gradients(ws_mod, shape, cin, cout):
    r = np.random.default_rng(7 + cin + cout)
    xg, x = bf16(r.standard_normal(shape + (cin,)))
    dzg, dz = bf16(r.standard_normal(shape + (cout,)))
    wg, w = bf16(r.standard_normal((cout, 27, cin)) / np.sqrt(27 * cin))
    dw = ws_mod.conv3_wgrad(dzg, xg)
    ref = W.conv3_weight_grad(dz, x)
    mag = W.conv3_weight_grad(np.abs(dz), np.abs(x))
    # the voxel sum is split into chunks (FP32) and the chunks summed in FP32: one more rounding per chunk
    assert np.all(np.abs(host(dw) - ref) <= 4e-5 * mag + 1e-6 * np.abs(ref).max())
    wt = ws_mod.weight_flip(wg)
    dx = torch.empty(shape + (cin,), dtype=torch.float32, device="cuda")
    ws_mod.conv3_fwd(dzg, wt, yf=dx)
    ref = W.conv3_input_adjoint(dz, w)
    mag = W.conv3_input_adjoint(np.abs(dz), np.abs(w))
    assert np.all(np.abs(host(dx) - ref) <= 4e-5 * mag)


def test_conv3_wgrad_large_voxel_count(ws_mod):
    """Many chunks: 2 x 32^3 voxels, the split used by training."""
    r = np.random.default_rng(11)
    shape = (2, 32, 32, 32)
    xg, x = bf16(r.standard_normal(shape + (16,)))
    dzg, dz = bf16(r.standard_normal(shape + (16,)))
    dw = host(ws_mod.conv3_wgrad(dzg, xg))
    ref = W.conv3_weight_grad(dz, x)
    mag = W.conv3_weight_grad(np.abs(dz), np.abs(x))
    assert np.all(np.abs(dw - ref) <= 4e-5 * mag + 1e-6 * np.abs(ref).max())


def test_relu_bias_pool_up(ws_mod):
    r = np.random.default_rng(12)
    shape = (2, 4, 6, 8, 32)
    dyg, dy = f32(r.standard_normal(shape))
    yg, y = bf16(r.standard_normal(shape))
    dz, dzb = ws_mod.relu_bwd(dyg, yg)
    assert np.array_equal(host(dz), dy * (y > 0))
    assert torch.equal(dzb.cpu(), dz.cpu().to(torch.bfloat16))
    dz0, _ = ws_mod.relu_bwd(dyg, None)
    assert np.array_equal(host(dz0), dy)
    db = host(ws_mod.bias_grad(dyg.reshape(-1, 32)))
    ref = dy.reshape(-1, 32).sum(axis=0)
    assert np.all(np.abs(db - ref) <= 1e-5 * np.abs(dy).reshape(-1, 32).sum(axis=0))
    p = host(ws_mod.pool_fwd(yg))
    ref = W.pool(y)
    assert np.all(np.abs(p - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-7)
    u = host(ws_mod.up_fwd(yg))
    assert np.array_equal(u, W.up(y))
    cg, c = f32(r.standard_normal((2, 2, 3, 4, 32)))
    assert np.allclose(host(ws_mod.pool_bwd(cg)), W.pool_adjoint(c), rtol=1e-6, atol=1e-7)
    assert np.allclose(host(ws_mod.up_bwd(dyg)), W.up_adjoint(dy), rtol=1e-5, atol=1e-6)
    acc = dyg.clone()
    ws_mod.pool_bwd(cg, dx=acc, accum=True)
    assert np.allclose(host(acc), dy + W.pool_adjoint(c), rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("C", [128, 12, 3])
def test_pool_up_channel_widths(ws_mod, C):
    # 16-byte channel vectors (C % 8 == 0 BF16, C % 4 == 0 FP32) and single channels
    r = np.random.default_rng(40 + C)
    yg, y = bf16(r.standard_normal((2, 4, 6, 8, C)))
    assert np.all(np.abs(host(ws_mod.pool_fwd(yg)) - W.pool(y)) <= 2.0 ** -8 * np.abs(W.pool(y)) + 1e-7)
    assert np.array_equal(host(ws_mod.up_fwd(yg)), W.up(y))
    cg, c = f32(r.standard_normal((2, 2, 3, 4, C)))
    dyg, dy = f32(r.standard_normal((2, 4, 6, 8, C)))
    assert np.allclose(host(ws_mod.pool_bwd(cg)), W.pool_adjoint(c), rtol=1e-6, atol=1e-7)
    assert np.allclose(host(ws_mod.up_bwd(dyg)), W.up_adjoint(dy), rtol=1e-5, atol=1e-6)
    acc = cg.clone()
    ws_mod.up_bwd(dyg, dx=acc, accum=True)
    assert np.allclose(host(acc), c + W.up_adjoint(dy), rtol=1e-5, atol=1e-6)
    # storage off the 16-byte grid takes the single-channel kernels: the same values
    buf = torch.empty(yg.numel() + 1, dtype=yg.dtype, device="cuda")
    ym = buf[1:].view(yg.shape)
    ym.copy_(yg)
    assert torch.equal(ws_mod.pool_fwd(ym), ws_mod.pool_fwd(yg))
    assert torch.equal(ws_mod.up_fwd(ym), ws_mod.up_fwd(yg))


def test_mse_and_adam(ws_mod):
    r = np.random.default_rng(13)
    pg, p = f32(r.standard_normal((4096, 16)))
    tg, t = f32(r.standard_normal((4096, 3)))
    loss, grad = ws_mod.mse(pg, tg)
    e = p[:, :3] - t
    assert abs(loss - np.mean(e * e)) <= 1e-6 * np.mean(e * e)
    g_ref = np.zeros_like(p)
    g_ref[:, :3] = 2 * e / e.size
    assert np.allclose(host(grad), g_ref, rtol=1e-5, atol=1e-12)
    n = 10000
    P, G = r.standard_normal(n), r.standard_normal(n)
    Pg, Gg = f32(P)[0], f32(G)[0]
    P, G = host(Pg), host(Gg)
    m1, m2 = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    M1, M2 = np.zeros(n), np.zeros(n)
    pb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    for step in range(1, 4):
        ws_mod.adam(Pg, Gg, m1, m2, 1e-2, step, pb=pb)
        P, M1, M2 = W.adam_step(P, G, M1, M2, step, 1e-2)
    assert np.allclose(host(Pg), P, rtol=1e-5, atol=1e-6)
    assert torch.equal(pb.cpu(), Pg.cpu().to(torch.bfloat16))


@pytest.fixture(scope="module")
def small_net(ws_mod):
    ws = ws_mod.WarmStart(n=(16, 16, 32), batch=2, vscale=4.0, seed=3)
    yield ws
    ws.close()


def test_network_structure(small_net):
    layers = small_net.layers()
    spec = W.layer_table()
    assert [(l[0], l[1], l[2], l[3], l[4], int(l[7] >= 0)) for l in layers] == spec
    assert "".join("cpu"[o[0]] for o in small_net.ops()) == W.op_kinds()
    assert small_net.num_params == W.num_params()
    assert 1.2e6 < W.num_params() < 1.6e6


def _bf16_params(seed):
    r = np.random.default_rng(seed)
    params = []
    for (cin_used, cin, cout, _, relu, _) in W.layer_table():
        w = r.standard_normal((cout, 27, cin)) * np.sqrt(2.0 / (27 * cin_used)) * (1.0 if relu else 0.3)
        w[:, :, cin_used:] = 0.0
        params.append((w, 0.05 * r.standard_normal(cout)))
    theta = W.flatten(params).astype(np.float32)
    return torch.from_numpy(theta).to(torch.bfloat16).float().numpy()


def test_network_loss_and_gradient(small_net):
    theta = _bf16_params(21)
    small_net.set_params(theta)
    assert np.array_equal(small_net.get_params(), theta)
    r = np.random.default_rng(22)
    n = small_net.n
    img_g, img = bf16(r.uniform(0, 1, size=(2, 2) + n))
    img_g = img_g.float().contiguous()
    tgt_g, tgt = f32(0.2 * r.standard_normal((2, 3) + n))
    loss = small_net.loss(img_g, tgt_g, backward=True)
    grads = small_net.get_grads()
    params = W.unflatten(theta.astype(np.float64))
    loss_ref, g_ref = W.loss_and_grad(params, img, tgt, small_net.vscale)
    assert abs(loss - loss_ref) <= 2e-2 * loss_ref, (loss, loss_ref)
    g = W.unflatten(grads.astype(np.float64))
    for k, ((dw, db), (rw, rb)) in enumerate(zip(g, g_ref)):
        ew = np.linalg.norm(dw - rw) / np.linalg.norm(rw)
        eb = np.linalg.norm(db - rb) / max(np.linalg.norm(rb), 1e-30)
        assert ew <= 2e-2 and eb <= 2e-2, (k, ew, eb)
    # forward agrees with the oracle's prediction
    v = small_net.forward(img_g).cpu().numpy()
    v_ref = W.predict(params, img, small_net.vscale)
    assert np.linalg.norm(v - v_ref) <= 2e-2 * np.linalg.norm(v_ref)
    # selecting rows by index is the same as passing them
    v1 = small_net.forward(img_g, idx=[1]).cpu().numpy()
    assert np.array_equal(v1[0], v[1])
    # the minibatch gathered by index (images and targets) gives the loss and gradients of the same rows passed
    # in that order, bit for bit
    loss_i = small_net.loss(img_g, tgt_g, idx=[1, 0], backward=True)
    grads_i = small_net.get_grads()
    loss_p = small_net.loss(img_g[[1, 0]].contiguous(), tgt_g[[1, 0]].contiguous(), backward=True)
    assert loss_i == loss_p
    assert np.array_equal(grads_i, small_net.get_grads())


def test_training_step_decreases_loss(small_net):
    small_net.set_params(_bf16_params(23))
    r = np.random.default_rng(24)
    n = small_net.n
    img = torch.from_numpy(r.uniform(0, 1, size=(4, 2) + n).astype(np.float32)).cuda()
    # a target the network can fit: a smooth function of the images
    tgt = torch.stack([0.1 * (img[:, 0] - img[:, 1]), 0.05 * img[:, 0], -0.05 * img[:, 1]], dim=1).contiguous()
    from paper_1808_04487_gb300.warmstart import evaluate
    l0 = evaluate(small_net, img, tgt)
    for it in range(40):
        small_net.train_step(img, tgt, [it % 4, (it + 1) % 4], 1e-3, want_loss=False)
    l1 = evaluate(small_net, img, tgt)
    assert l1 < 0.5 * l0, (l0, l1)


RESAMPLE_CASES = [((12, 16, 10), (20, 18, 24)), ((24, 20, 14), (12, 12, 12)), ((32, 32, 32), (64, 64, 64)),
                  ((16, 16, 16), (16, 16, 16))]


@pytest.mark.parametrize("n_src,n_dst", RESAMPLE_CASES)
def test_resample(n_src, n_dst):
    _need_gpu()
    from paper_1808_04487_gb300 import Context
    r = np.random.default_rng(sum(n_src) + sum(n_dst))
    a, b = Context(n_src), Context(n_dst)
    f = r.standard_normal((3,) + n_src)
    out = a.resample_to(b, torch.from_numpy(f.astype(np.float32)).cuda()).cpu().numpy()
    ref = W.resample_vector(f.astype(np.float32).astype(np.float64), n_dst)
    assert np.linalg.norm(out - ref) <= 1e-5 * np.linalg.norm(ref)
    outp = a.resample_to(b, torch.from_numpy(f.astype(np.float32)).cuda(), project=True).cpu().numpy()
    refp = W.resample_vector(f.astype(np.float32).astype(np.float64), n_dst, project=True)
    assert np.linalg.norm(outp - refp) <= 1e-5 * np.linalg.norm(refp)
    s = a.resample_to(b, torch.from_numpy(f[0].astype(np.float32)).cuda()).cpu().numpy()
    assert np.linalg.norm(s - ref[0]) <= 1e-5 * np.linalg.norm(ref[0])


def test_predict_and_warm_started_solve(ws_mod):
    """The prediction is divergence-free on the solve grid; a warm start keeps g_0 = g(v = 0) (Sec. 2.3.2)."""
    import claire_inputs as I
    from paper_1808_04487_gb300 import Context
    n = (48, 48, 48)
    ctx = Context(n, "f32", beta=1e-3, regnorm=2, divfree=True, nt=4, gtol_rel=1e-2)
    mT = torch.from_numpy(I.brain_phantom(n, seed=5)).float().cuda()
    vs = torch.from_numpy(I.random_velocity(n, seed=6, kmax=6, max_disp_voxels=1.5, divfree=True)).float().cuda()
    mR = ctx.transport(mT, vs, +1)
    ws = ws_mod.WarmStart(n=(32, 32, 32), batch=1, vscale=10.0, seed=1)
    v0 = ws.predict(ctx, mT, mR)
    assert torch.isfinite(v0).all()
    div = ctx.spectral("div", v0)
    assert float(div.norm()) <= 1e-4 * float(v0.norm()) + 1e-12
    # the pipeline agrees with the oracle (resample down, network, resample up + Leray)
    params = W.unflatten(ws.get_params().astype(np.float64))
    img = np.stack([W.resample(mT.cpu().numpy().astype(np.float64), ws.n),
                    W.resample(mR.cpu().numpy().astype(np.float64), ws.n)])[None]
    v_net = W.predict(params, img, ws.vscale)[0]
    v_ref = W.resample_vector(v_net, n, project=True)
    assert np.linalg.norm(v0.cpu().numpy() - v_ref) <= 3e-2 * np.linalg.norm(v_ref)
    # zero start, then restart from the solution: no Gauss-Newton step is needed and g_0 is unchanged
    v, rep0, st0 = ctx.register(mT, mR)
    assert st0 == "OK"
    v2, rep1, st1 = ctx.register(mT, mR, v.clone())
    assert st1 == "OK" and rep1["gn_iters"] == 0
    assert abs(rep1["gnorm0"] - rep0["gnorm0"]) <= 1e-6 * rep0["gnorm0"]
    # a gradient field added to the guess is removed by the projection onto div v = 0 (Sec. 2.2)
    x = [2 * np.pi * np.arange(m) / m for m in n]
    X1, X2 = np.meshgrid(x[0], x[1], indexing="ij")
    gp = np.zeros((3,) + n)
    gp[0] = (np.cos(X1) * np.cos(2 * X2))[..., None]
    gp[1] = (-2 * np.sin(X1) * np.sin(2 * X2))[..., None]
    v4 = v + 0.05 * torch.from_numpy(gp).float().cuda()
    v4, rep4, st4 = ctx.register(mT, mR, v4)
    assert st4 == "OK" and rep4["gn_iters"] == 0
    assert float((v4 - v).norm()) <= 1e-5 * float(v.norm())
    # a warm start from the (untrained) prediction still converges to the same relative tolerance
    v3, rep2, st2 = ctx.register(mT, mR, v0.clone())
    assert st2 == "OK"
    assert rep2["gnorm"] <= 1e-2 * rep0["gnorm0"]
    assert abs(rep2["gnorm0"] - rep0["gnorm0"]) <= 1e-6 * rep0["gnorm0"]
    ws.close()


def test_training_set_and_short_training(ws_mod):
    S = 12
    images, targets, stats = ws_mod.make_training_set(S, n_solve=(64, 64, 64), n_net=(32, 32, 32), seed=3,
                                                      phantoms=3, chunk=12, nworkers=4)
    assert stats["converged"] == S
    assert images.shape == (S, 2, 32, 32, 32) and targets.shape == (S, 3, 32, 32, 32)
    assert torch.isfinite(images).all() and torch.isfinite(targets).all()
    rms = float(targets.pow(2).mean().sqrt())
    ws = ws_mod.WarmStart(n=(32, 32, 32), batch=4, vscale=1.0 / rms, seed=2)
    l0 = ws_mod.evaluate(ws, images, targets)
    ws_mod.train(ws, images, targets, steps=300, lr=2e-3, lr_final=1e-4, seed=0)
    l1 = ws_mod.evaluate(ws, images, targets)
    assert l1 < 0.8 * l0, (l0, l1)
    ws.close()


def test_trained_network_saves_gauss_newton_work_on_held_out_pairs(ws_mod):
    """What the learned warm start gains over the method without it. The network is trained on (m_T, m_R, v)
    triples that the plain solver makes (384 seeded phantom pairs on 64^3, H2, beta 1e-3, div v = 0, to
    ||g|| <= 1e-2 ||g(v = 0)||; network grid 32^3, 2000 Adam steps with cube-symmetry augmentation). On 16
    held-out pairs (unseen phantoms and velocities) the unchanged solver then runs from v = 0 and from the
    prediction (low-passed to |k_i| <= 4). Both stop by the same rule of Sec. 2.3.2 with the same reference
    ||g(v = 0)||; the warm start must need fewer Gauss-Newton matvecs on average, no more GN steps, and reach the
    same final mismatch (mean relative difference within 0.5%)."""
    import claire_inputs as I
    from paper_1808_04487_gb300 import Context
    n, n_net = (64, 64, 64), (32, 32, 32)
    images, targets, stats = ws_mod.make_training_set(384, n_solve=n, n_net=n_net, seed=0, phantoms=32, chunk=64)
    assert stats["converged"] == 384
    rms = float(targets.pow(2).mean().sqrt())
    ws = ws_mod.WarmStart(n=n_net, batch=8, vscale=1.0 / rms, seed=0)
    ws_mod.train(ws, images, targets, 2000, lr=2e-3, lr_final=1e-4, seed=0, augment=True)
    del images, targets
    ctx = Context(n, "f32", beta=1e-3, regnorm=2, divfree=True, nt=4, gtol_rel=1e-2)
    ctx_n = Context(n_net, "f32")
    disp_net = 8.0 * max(n) / 256.0 * max(n_net) / max(n)
    zero, warm = [], []
    for j in range(16):
        mT = torch.from_numpy(I.brain_phantom(n, seed=500009 + 7 * j)).float().cuda()
        vs = I.random_velocity(n_net, seed=900001 + 13 * j, kmax=6, max_disp_voxels=disp_net, divfree=True)
        vs = ctx_n.resample_to(ctx, torch.from_numpy(vs).float().cuda().contiguous())
        mR = ctx.transport(mT, vs, +1)
        _, rz, sz = ctx.register(mT, mR)
        v0 = ws.predict(ctx, mT, mR, kmax=4)
        _, rw, sw = ctx.register(mT, mR, v0.clone())
        assert sz == "OK" and sw == "OK"
        assert abs(rw["gnorm0"] - rz["gnorm0"]) <= 1e-6 * rz["gnorm0"]  # the same reference gradient
        assert rw["gnorm"] <= 1e-2 * rw["gnorm0"] and rz["gnorm"] <= 1e-2 * rz["gnorm0"]
        zero.append(rz)
        warm.append(rw)
    mean = lambda rows, k: float(np.mean([r[k] for r in rows]))
    dmis = float(np.mean([w["mismatch"] / z["mismatch"] - 1.0 for w, z in zip(warm, zero)]))
    print("held-out 64^3: zero start %.2f GN / %.2f matvecs, warm start %.2f GN / %.2f matvecs, mismatch %+.4f"
          % (mean(zero, "gn_iters"), mean(zero, "matvecs"), mean(warm, "gn_iters"), mean(warm, "matvecs"), dmis))
    assert mean(warm, "matvecs") < mean(zero, "matvecs")
    assert mean(warm, "gn_iters") <= mean(zero, "gn_iters")
    assert abs(dmis) <= 5e-3
    ws.close()
    ctx.close()
    ctx_n.close()


def test_restart_from_truncated_solution_256():
    """At 256^3 with H2 and div v = 0, a restart from the zero-start solution truncated to 32^3 converges in a
    few Gauss-Newton steps (it needs the projection of the guess: its rounding error has a curl-free part that
    beta A would otherwise keep in the gradient)."""
    _need_gpu()
    import claire_inputs as I
    from paper_1808_04487_gb300 import Context
    n = (256, 256, 256)
    ctx = Context(n, "f32", beta=1e-3, regnorm=2, divfree=True, nt=4, gtol_rel=1e-2)
    net = Context((32, 32, 32), "f32")
    mT = torch.from_numpy(I.brain_phantom(n, seed=11)).float().cuda()
    vs = I.random_velocity((32, 32, 32), seed=12, kmax=6, max_disp_voxels=1.0, divfree=True)
    mR = ctx.transport(mT, net.resample_to(ctx, torch.from_numpy(vs).float().cuda()), +1)
    v, rep, st = ctx.register(mT, mR)
    assert st == "OK"
    vt = net.resample_to(ctx, ctx.resample_to(net, v), project=True)
    assert float((vt - v).norm()) <= 1e-2 * float(v.norm())
    v2, rep2, st2 = ctx.register(mT, mR, vt)
    assert st2 == "OK", rep2
    assert rep2["gn_iters"] <= 4 and rep2["matvecs"] < rep["matvecs"], (rep, rep2)
