"""Seeded synthetic inputs for the registration hot path.

This module only *makes inputs*: images and velocity fields with the shapes, value ranges and spectral content of
the paper's workloads. It holds none of the method's arithmetic (no transport, no interpolation, no gradient,
Hessian, projection or preconditioner); both the FP64 oracle and the CUDA path consume its arrays.

Conventions shared by every generator:

* grid ``n = (n1, n2, n3)`` on the periodic box [0, 2*pi)^3, node ``x = (2*pi*i1/n1, 2*pi*i2/n2, 2*pi*i3/n3)``
  (Sec. 2.3.1; only the periodic equivalence of the index range matters);
* scalar fields are C-ordered ``[n1][n2][n3]`` float64 arrays (``i3`` fastest);
* vector fields are planar ``[3][n1][n2][n3]`` float64 arrays, component ``c`` along axis ``c``.

Recipes (all seeded with ``numpy.random.default_rng(seed)``):

* ``trig_image``: sum of R=8 products of sin/cos with integer wavenumbers in [0, 4] and U(0,1) amplitudes, then
  min-max normalised to [0, 1] (the smooth 32^3 test image).
* ``brain_phantom``: three nested ellipsoids with random centres and semi-axes and intensities 0.2 / 0.5 / 0.9,
  plus N(0, 0.01^2) noise, Gaussian-smoothed in the spectral domain with sigma = 1 voxel and rescaled to [0, 1]
  (stands in for the NIREP brain volumes of Sec. 4.2, which are not available here; smoothing and rescaling follow
  the pre-processing of Sec. 2.3.1).
* ``random_velocity``: band-limited random field made of Fourier modes 1 <= |k| <= kmax with N(0, 1)
  coefficients. With ``divfree=True`` it is built as the curl of a random band-limited vector potential, so its
  spectral divergence vanishes to rounding. Scaled so that max_x max_c |v_c| equals ``amplitude`` (physical units),
  or ``max_disp_voxels`` grid spacings of the finest axis when that is given (displacement over the unit time
  interval).
* ``paper_synthetic``: the closed-form template and velocity of the scalability problem of Sec. 4.2.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "grid_coords",
    "trig_image",
    "brain_phantom",
    "random_velocity",
    "paper_synthetic",
    "random_field",
]


def grid_coords(n):
    """Return the three 1D coordinate arrays x_a = 2*pi*i/n_a (float64)."""
    return [2.0 * np.pi * np.arange(na, dtype=np.float64) / na for na in n]


def trig_image(n, seed=0, R=8, kmax=4):
    """Smooth image: sum_r a_r prod_a phi_{r,a}(k_{r,a} x_a), phi in {sin, cos}, then min-max to [0, 1]."""
    rng = np.random.default_rng(seed)
    x1, x2, x3 = grid_coords(n)
    m = np.zeros(tuple(n), dtype=np.float64)
    for _ in range(R):
        amp = rng.uniform(0.0, 1.0)
        fac = []
        for xa in (x1, x2, x3):
            k = int(rng.integers(0, kmax + 1))
            phi = np.sin if rng.integers(0, 2) == 0 else np.cos
            fac.append(phi(k * xa))
        m += amp * fac[0][:, None, None] * fac[1][None, :, None] * fac[2][None, None, :]
    lo, hi = m.min(), m.max()
    if hi - lo < 1e-300:
        return np.zeros_like(m)
    return (m - lo) / (hi - lo)


def _spectral_gauss(f, n, sigma_vox):
    """Gaussian smoothing exp(-0.5 * sum_a (sigma * h_a * k_a)^2) applied in the Fourier domain."""
    h = [2.0 * np.pi / na for na in n]
    k1 = np.fft.fftfreq(n[0], 1.0 / n[0])
    k2 = np.fft.fftfreq(n[1], 1.0 / n[1])
    k3 = np.arange(n[2] // 2 + 1, dtype=np.float64)
    g = (np.exp(-0.5 * (sigma_vox * h[0] * k1) ** 2)[:, None, None]
         * np.exp(-0.5 * (sigma_vox * h[1] * k2) ** 2)[None, :, None]
         * np.exp(-0.5 * (sigma_vox * h[2] * k3) ** 2)[None, None, :])
    return np.fft.irfftn(np.fft.rfftn(f) * g, s=tuple(n), axes=(0, 1, 2))


def brain_phantom(n, seed=0, sigma_vox=1.0, noise=0.01):
    """Nested-ellipsoid brain stand-in: intensities 0.2 (head), 0.5 (middle), 0.9 (core); noise; smoothing; [0,1]."""
    rng = np.random.default_rng(seed)
    n = tuple(int(a) for a in n)
    x1, x2, x3 = grid_coords(n)
    X1, X2, X3 = x1[:, None, None], x2[None, :, None], x3[None, None, :]
    m = np.zeros(n, dtype=np.float64)
    # Outer shell radius ~ 0.7*pi, inner shells shrink; centres jitter around the box centre.
    base = np.array([np.pi, np.pi, np.pi])
    scales = [(0.62, 0.78), (0.42, 0.55), (0.20, 0.32)]
    levels = [0.2, 0.5, 0.9]
    c_prev = base.copy()
    for (lo, hi), val in zip(scales, levels):
        c = c_prev + rng.uniform(-0.08, 0.08, size=3) * np.pi
        ax = rng.uniform(lo, hi, size=3) * np.pi
        inside = (((X1 - c[0]) / ax[0]) ** 2 + ((X2 - c[1]) / ax[1]) ** 2 + ((X3 - c[2]) / ax[2]) ** 2) <= 1.0
        m = np.where(inside, val, m)
        c_prev = c
    m = m + rng.normal(0.0, noise, size=n)
    m = _spectral_gauss(m, n, sigma_vox)
    lo, hi = m.min(), m.max()
    return (m - lo) / (hi - lo)


def _random_band_limited(n, kmax, rng, ncomp):
    """ncomp real fields with N(0,1) Fourier coefficients on 1 <= |k| <= kmax (half spectrum, irfftn)."""
    n = tuple(int(a) for a in n)
    k1 = np.fft.fftfreq(n[0], 1.0 / n[0])
    k2 = np.fft.fftfreq(n[1], 1.0 / n[1])
    k3 = np.arange(n[2] // 2 + 1, dtype=np.float64)
    K1, K2, K3 = np.meshgrid(k1, k2, k3, indexing="ij")
    kk = np.sqrt(K1 ** 2 + K2 ** 2 + K3 ** 2)
    mask = (kk >= 1.0) & (kk <= kmax)
    # only modes well below Nyquist are used, so the spectrum is exactly representable on every grid used here
    out = []
    spec = []
    for _ in range(ncomp):
        c = np.zeros(K1.shape, dtype=np.complex128)
        nz = int(mask.sum())
        c[mask] = rng.normal(size=nz) + 1j * rng.normal(size=nz)
        spec.append(c)
    return spec, (K1, K2, K3)


def random_velocity(n, seed=0, kmax=3, amplitude=None, max_disp_voxels=None, divfree=False):
    """Band-limited random velocity [3][n1][n2][n3] (see module docstring for the scaling rule)."""
    rng = np.random.default_rng(seed)
    n = tuple(int(a) for a in n)
    spec, (K1, K2, K3) = _random_band_limited(n, kmax, rng, 3)
    if divfree:
        # v = curl(psi): v^ = i k x psi^, which has zero spectral divergence for every mode.
        p1, p2, p3 = spec
        spec = [1j * (K2 * p3 - K3 * p2), 1j * (K3 * p1 - K1 * p3), 1j * (K1 * p2 - K2 * p1)]
    v = np.stack([np.fft.irfftn(s, s=n, axes=(0, 1, 2)) for s in spec])
    vmax = np.abs(v).max()
    if vmax == 0.0:
        return v
    if max_disp_voxels is not None:
        target = max_disp_voxels * 2.0 * np.pi / max(n)
    elif amplitude is not None:
        target = amplitude
    else:
        target = 1.0
    return v * (target / vmax)


def random_field(n, seed=0, kmax=6, ncomp=1):
    """Unscaled band-limited random real field(s) (test vectors); shape [ncomp][n1][n2][n3] or [n1][n2][n3]."""
    rng = np.random.default_rng(seed)
    spec, _ = _random_band_limited(n, kmax, rng, ncomp)
    f = np.stack([np.fft.irfftn(s, s=tuple(n), axes=(0, 1, 2)) for s in spec])
    f /= np.abs(f).max()
    return f if ncomp > 1 else f[0]


def paper_synthetic(n):
    """Closed-form template and velocity of the scalability test problem (Sec. 4.2).

    m_T = (sin^2 x1 + sin^2 x2 + sin^2 x3) / 3,
    v*_1 = sin x3 cos x2 sin x2,  v*_2 = sin x1 cos x3 sin x3,  v*_3 = sin x2 cos x1 sin x1.
    Each v*_i does not depend on x_i, so div v* = 0 exactly.
    """
    x1, x2, x3 = grid_coords(n)
    X1, X2, X3 = np.meshgrid(x1, x2, x3, indexing="ij")
    mT = (np.sin(X1) ** 2 + np.sin(X2) ** 2 + np.sin(X3) ** 2) / 3.0
    v = np.stack([np.sin(X3) * np.cos(X2) * np.sin(X2),
                  np.sin(X1) * np.cos(X3) * np.sin(X3),
                  np.sin(X2) * np.cos(X1) * np.sin(X1)])
    return mT, v
