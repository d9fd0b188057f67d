"""The cube symmetries used to augment warm-start training batches map a (scalar image, velocity) pair to a pair of
the same problem: checked on a gradient field, v = grad phi, where the transformed velocity must equal the gradient
of the transformed potential (spectral derivatives on a periodic grid). CPU only."""
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def spectral_grad(phi):
    n = phi.shape
    k = [np.fft.fftfreq(na, 1.0 / na) for na in n]
    F = np.fft.fftn(phi)
    out = []
    for a in range(3):
        shape = [1, 1, 1]
        shape[a] = n[a]
        ka = k[a].reshape(shape).copy()
        ka[np.abs(ka) == n[a] // 2] = 0.0
        out.append(np.real(np.fft.ifftn(1j * ka * F)))
    return np.stack(out)


@pytest.mark.parametrize("flips,perm", [((1, 0, 0), (0, 1, 2)), ((0, 1, 1), (0, 1, 2)), ((0, 0, 0), (2, 0, 1)),
                                        ((1, 1, 0), (1, 0, 2)), ((1, 0, 1), (2, 1, 0))])
def test_cube_symmetry_maps_a_gradient_field_to_the_gradient_of_the_mapped_potential(flips, perm):
    from paper_1808_04487_gb300.warmstart import cube_symmetry
    n = (8, 8, 8)
    rng = np.random.default_rng(3)
    x = [2 * np.pi * np.arange(na) / na for na in n]
    X = np.meshgrid(*x, indexing="ij")
    phi = sum(rng.normal() * np.sin(kx * X[0] + ky * X[1] + kz * X[2] + rng.uniform(0, 6))
              for kx, ky, kz in itertools.product(range(-2, 3), repeat=3))
    v = spectral_grad(phi)
    img = torch.from_numpy(phi[None, None].copy())
    tgt = torch.from_numpy(v[None].copy())
    img2, tgt2 = cube_symmetry(img, tgt, flips, perm)
    v_expected = spectral_grad(img2[0, 0].numpy())
    np.testing.assert_allclose(tgt2[0].numpy(), v_expected, atol=1e-9 * np.abs(v).max())


def test_cube_symmetry_reflection_is_an_involution():
    from paper_1808_04487_gb300.warmstart import cube_symmetry
    rng = np.random.default_rng(4)
    img = torch.from_numpy(rng.normal(size=(2, 2, 6, 6, 6)))
    tgt = torch.from_numpy(rng.normal(size=(2, 3, 6, 6, 6)))
    i1, t1 = cube_symmetry(img, tgt, (1, 1, 1), (0, 1, 2))
    i2, t2 = cube_symmetry(i1, t1, (1, 1, 1), (0, 1, 2))
    assert torch.equal(i2, img) and torch.equal(t2, tgt)
