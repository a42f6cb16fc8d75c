"""Pins of the multi-scale CLEAN minor cycle (Eq. 6-7)."""
import numpy as np
import pytest

from oracle import filters, msclean


def test_delta_psf_point_source_exact_flux_gain_one():
    n = 32
    x = np.zeros((n, n))
    x[11, 20] = 3.25
    psf_spec = np.ones((2 * n, 2 * n), dtype=complex)      # PSF = delta: every uv cell sampled
    res = msclean.clean(filters.image_spectrum(x), psf_spec, [0], 1.0, 10, 1e-12)
    assert res.iterations == 1
    assert res.components[0][:3] == (0, 11, 20)
    assert res.model[11, 20] == pytest.approx(3.25, rel=1e-14)
    assert np.max(np.abs(res.residuals[0])) < 1e-13


def _psf(n, seed=0):
    yy, xx = np.meshgrid(np.arange(2 * n) - n, np.arange(2 * n) - n, indexing="ij")
    p = np.exp(-(xx ** 2 + yy ** 2) / 6.0) + 0.05 * np.cos(0.7 * xx) * np.exp(-(xx ** 2 + yy ** 2) / 200.0)
    return p / p[n, n]


def test_single_scale_equals_hogbom_loop():
    n = 32
    rng = np.random.default_rng(1)
    psf = _psf(n)
    sky = np.zeros((n, n))
    sky[rng.integers(4, 28, 6), rng.integers(4, 28, 6)] = rng.uniform(0.5, 2.0, 6)
    dirty = filters.apply(sky, filters.psf_spectrum(psf))
    res = msclean.clean(filters.image_spectrum(dirty), filters.psf_spectrum(psf), [0], 0.2, 60, 1e-9)
    # hand-written Hogbom loop on the image domain
    r = dirty.copy()
    model = np.zeros((n, n))
    for _ in range(60):
        p = int(np.argmax(np.abs(r)))
        py, px = divmod(p, n)
        a = 0.2 * r[py, px]
        model[py, px] += a
        r -= a * psf[n - py:2 * n - py, n - px:2 * n - px]
    assert np.max(np.abs(res.model - model)) < 1e-12
    assert np.max(np.abs(res.residuals[0] - r)) < 1e-12


def test_scale_residual_invariant():
    """R_s = B_s (*) (D - P (*) model) after a run: with a compact PSF and
    interior sources no convolution reaches the image edge, so circular and
    linear convolutions agree and the identity is exact."""
    n = 32
    rng = np.random.default_rng(2)
    yy, xx = np.meshgrid(np.arange(2 * n) - n, np.arange(2 * n) - n, indexing="ij")
    r2 = xx ** 2 + yy ** 2
    psf = np.where(r2 <= 36, np.exp(-r2 / 6.0) + 0.05 * np.cos(0.7 * xx), 0.0)
    psf /= psf[n, n]
    sky = np.zeros((n, n))
    sky[14:18, 14:18] = rng.uniform(0.1, 1.0, (4, 4))
    ps = filters.psf_spectrum(psf)
    d = filters.apply(sky, ps)
    scales = [0, 2, 4]
    res = msclean.clean(filters.image_spectrum(d), ps, scales, 0.1, 40, 1e-9)
    rest = d - filters.apply(res.model, ps)
    for i, s in enumerate(scales):
        bs = filters.spectrum(msclean.scale_kernel(s, n).astype(complex))
        want = filters.apply(rest, bs)
        assert np.max(np.abs(res.residuals[i] - want)) < 1e-12
    assert {c[0] for c in res.components} - {0}       # larger scales get used


def test_allowed_scales_first_cycle():
    sc = [0, 3, 9]
    assert msclean.allowed_scales(sc, 128, 0, 1, [5.0], 1.0).all()
    a = msclean.allowed_scales(sc, 128, 1, 1, [5.0], 1.0)
    # N/(2s) >= ell - delta = 4: s=3 -> 21.3 yes, s=9 -> 7.1 yes
    assert a.tolist() == [True, True, True]
    a = msclean.allowed_scales(sc, 128, 1, 1, [20.0], 1.0)
    assert a.tolist() == [True, True, False]
    assert msclean.allowed_scales(sc, 128, 1, 2, [20.0], 1.0).all()
