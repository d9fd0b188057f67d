"""C-ABI checks that need no GPU: the library loads, exports every symbol the header declares, and its host-side
argument validation rejects bad input before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "claire.h")


@pytest.fixture(scope="module")
def L():
    from paper_1808_04487_gb300 import build as b
    b.build()
    import paper_1808_04487_gb300 as pkg
    return pkg.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(claire_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_five_paper_calls():
    names = declared_functions()
    for base in ("claire_transport", "claire_gradient", "claire_hessvec", "claire_precond", "claire_register"):
        assert base + "_f32" in names and base + "_f64" in names


def test_every_declared_symbol_is_exported(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_default_opts_are_the_papers(L):
    import paper_1808_04487_gb300 as pkg
    o = pkg.Opts()
    assert L.claire_default_opts(ctypes.byref(o), 32, 32, 32, 0) == 0
    assert (o.nt, o.regnorm, o.divfree, o.max_gn, o.max_krylov, o.max_ls) == (4, 1, 0, 50, 100, 10)
    assert (o.gtol_rel, o.gtol_abs, o.armijo_c1) == (5e-2, 1e-6, 1e-4)
    assert (o.beta_w, o.precond, o.pc_kappa) == (0.0, 0, 0.1)


@pytest.mark.parametrize("bad", [
    dict(n=(31, 32, 32)), dict(n=(2, 32, 32)), dict(n=(22, 32, 32)), dict(nt=0), dict(beta=0.0), dict(beta=-1.0),
    dict(regnorm=3), dict(divfree=2), dict(precision=5), dict(max_krylov=0), dict(max_ls=0), dict(bf16_mask=2),
    dict(bf16_mask=1, precision=1), dict(beta_w=-1e-4), dict(beta_w=1e-4, divfree=1),
    dict(beta_w=1e-4, regnorm=2), dict(precond=2), dict(precond=1, n=(18, 16, 16)), dict(precond=1, n=(4, 16, 16)), dict(precond=1, pc_kappa=1.5)])
def test_create_rejects_bad_options_before_any_device_call(L, bad):
    import paper_1808_04487_gb300 as pkg
    o = pkg.Opts()
    L.claire_default_opts(ctypes.byref(o), 32, 32, 32, 0)
    for k, val in bad.items():
        if k == "n":
            for a in range(3):
                o.n[a] = val[a]
        else:
            setattr(o, k, val)
    h = ctypes.c_void_p()
    assert L.claire_create(ctypes.byref(o), ctypes.byref(h)) == 1  # CLAIRE_EINVAL
    assert not h.value


def test_null_context_is_rejected(L):
    assert L.claire_transport_f32(None, None, None, 1, None, None) == 1
    assert L.claire_register_f64(None, None, None, None, None, None) == 1
    assert L.claire_destroy(None) == 0
    assert L.claire_last_error(None) == b"null context"


def test_radix_support_matches_the_batched_grids():
    # every grid of the population-to-atlas set factors into the supported radices 2, 3, 5, 7
    for n in (64, 96, 112, 128, 144, 160, 192, 256):
        m = n
        for r in (2, 3, 5, 7):
            while m % r == 0:
                m //= r
        assert m == 1 and (n // 2) * 2 == n


def test_convolutions_reject_pointers_off_the_16_byte_grid(L):
    """Host-only: the convolutions move 16-byte vectors, so a tensor pointer that is not 16-byte aligned is refused
    before any device work (the pointers below are never dereferenced)."""
    f = L.claire_nn_conv3_fwd
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p] * 6 + [ctypes.c_int] * 8 + [ctypes.c_void_p, ctypes.c_void_p]
    assert f(0x10002, 0x20000, None, None, 0x30000, None, 0, 1, 16, 16, 16, 16, 16, 0, None, None) == 1
    assert f(0x10000, 0x20000, None, None, 0x30008, None, 0, 1, 16, 16, 16, 16, 16, 0, None, None) == 1
    g = L.claire_nn_conv3_wgrad
    g.restype = ctypes.c_int
    g.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int] * 6 + [ctypes.c_void_p]
    assert g(0x10004, 0x20000, 0x30000, 0x40000, 1, 16, 16, 16, 16, 16, None) == 1


def test_convolution_workspaces_follow_the_batch_invariant_split_rule(L):
    """Host-only sizing of the convolution workspaces (no device call). The forward split-K over the 27 neighbour
    offsets is chosen from the per-sample grid alone, so a sample's result does not depend on its batch: the
    partial-sum workspace is zero for grids with enough 128-voxel tiles and otherwise scales exactly with the batch.
    Invalid shapes (channels not a multiple of 16, more than 128) size to 0."""
    f = L.claire_nn_fwd_workspace_bytes
    f.restype = ctypes.c_size_t
    f.argtypes = [ctypes.c_int] * 5
    assert f(1, 64, 64, 64, 16) == 0          # 8 x 64^3 / 128 tiles: no split
    assert f(1, 32, 32, 32, 16) == 0          # 8 x 32^3 / 128 = 2048 tiles: no split
    small = f(1, 8, 8, 8, 64)
    assert small > 0                           # 8 x 8^3 / 128 = 32 tiles: split
    for B in (2, 3, 8):
        assert f(B, 8, 8, 8, 64) == B * small
    assert f(1, 8, 8, 8, 24) == 0 and f(1, 8, 8, 8, 144) == 0 and f(0, 8, 8, 8, 64) == 0
    w = L.claire_nn_wgrad_workspace_bytes
    w.restype = ctypes.c_size_t
    w.argtypes = [ctypes.c_int] * 6
    assert w(8, 32, 32, 32, 16, 16) > 0 and w(8, 32, 32, 32, 16, 24) == 0
