"""The allocation-free inner product against the context-based one.

claire_dot_noalloc_f32 serves callers that must not allocate device memory (a fixed memory budget owned by
another allocator, or a loop that cannot pay for cudaMalloc's implicit synchronisation): its partial sums live in
a static device array instead of a context workspace. This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes on its own in a fresh process.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1808_04487_gb300 import build as b
    b.build()
    import paper_1808_04487_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return pkg.lib()


def noalloc_dot(L, a, b, scale):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    st = L.claire_dot_noalloc_f32(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), a.numel(),
                                  float(scale), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    return float(out.item())


def test_noalloc_dot_matches_the_context_dot_twice_in_a_row(L):
    import paper_1808_04487_gb300 as pkg
    n = (64, 48, 40)
    cell = (2 * math.pi) ** 3 / np.prod(n)
    g = torch.Generator(device="cuda").manual_seed(7)
    with pkg.Context(n, precision="f32") as ctx:
        for trial in range(2):  # two calls in a row: stale partials of the first call must not leak
            a = torch.randn((3,) + n, device="cuda", generator=g)
            b = torch.randn((3,) + n, device="cuda", generator=g) + (1.0 if trial else -0.5)
            ref = ctx.dot(a, b)
            got = noalloc_dot(L, a, b, cell)
            assert abs(got - ref) <= 1e-12 * max(abs(ref), 1e-300) + 1e-12 * cell * a.numel()
    # a count that is not a multiple of the block chunk, and the empty input
    a = torch.randn(12345, device="cuda", generator=g)
    assert abs(noalloc_dot(L, a, a, 1.0) - float((a.double() ** 2).sum())) <= 1e-12 * float((a.double() ** 2).sum())
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    assert L.claire_dot_noalloc_f32(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()), 0, 1.0,
                                    ctypes.c_void_p(out.data_ptr()), None) == 0
    assert float(out.item()) == 0.0


def test_noalloc_dot_rejects_sizes_beyond_its_static_scratch(L):
    a = torch.zeros(4, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    too_many = 65536 * 2048 + 1
    st = L.claire_dot_noalloc_f32(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()), too_many, 1.0,
                                  ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1  # CLAIRE_EINVAL, nothing launched
    # the largest count: rejected before any arithmetic on it (no overflow into a small block count)
    st = L.claire_dot_noalloc_f32(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()), 2 ** 63 - 1, 1.0,
                                  ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1
    assert L.claire_dot_noalloc_f32(None, None, 4, 1.0, None, None) == 1
