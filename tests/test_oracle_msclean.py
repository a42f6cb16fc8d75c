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


def _hand_scale(s, n):
    """B_s on the 2N grid written out by loops: 1 - (r/s)^2 inside radius s,
    unit sum (B_0 = delta)."""
    b = np.zeros((2 * n, 2 * n))
    if s == 0:
        b[n, n] = 1.0
        return b
    tot = 0.0
    for y in range(2 * n):
        for x in range(2 * n):
            r2 = (y - n) ** 2 + (x - n) ** 2
            if r2 < s * s:
                b[y, x] = 1.0 - r2 / float(s * s)
                tot += b[y, x]
    return b / tot


def test_scale_choice_decided_by_the_bias():
    """Cornwell (2008) scale bias 1 - 0.6 s / s_max with peak normalisation by
    P_ss(0).  PSF = delta (every uv cell sampled) and D = a B_3 at pixel p:
    the unbiased criterion |R_s(p)| / P_ss(0) favours s = 9 (sum B_3 B_9 /
    sum B_9^2 > 1), the biased one s = 3 (0.8 against 0.4 x that ratio).  The
    first component is (s = 3, p, gain a) and the two best candidate values
    are the hand-computed ones."""
    n = 48
    a, gain = 2.5, 0.1
    py, px = 21, 26
    b3, b9 = _hand_scale(3, n), _hand_scale(9, n)
    sum33 = float((b3 * b3).sum())
    sum99 = float((b9 * b9).sum())
    sum39 = float((b3 * b9).sum())
    assert sum39 / sum99 > 1.0 and 0.8 > 0.4 * sum39 / sum99      # the bias flips the choice
    d = np.zeros((n, n))
    d[py - 2:py + 3, px - 2:px + 3] = a * b3[n - 2:n + 3, n - 2:n + 3]   # B_3 lies within radius 2.9
    psf_spec = np.ones((2 * n, 2 * n), dtype=complex)
    res = msclean.clean(filters.image_spectrum(d), psf_spec, [0, 3, 9], gain, 1, 0.0)
    s, y, x, amp = res.components[0]
    assert (s, y, x) == (1, py, px)
    assert amp == pytest.approx(gain * a, rel=1e-12)
    best, _ = res.gaps[0]
    assert best == pytest.approx(0.8 * a, rel=1e-12)
    # after the step R_s(p) = (1 - gain) a (B_s . B_3)(0) for every scale
    # (R_s -= amp P_{s,3}(. - p) with P_{s,3} = B_s * B_3 for a delta PSF)
    assert res.residuals[0][py, px] == pytest.approx((1 - gain) * a * b3[n, n], rel=1e-12)
    assert res.residuals[1][py, px] == pytest.approx((1 - gain) * a * sum33, rel=1e-12)
    assert res.residuals[2][py, px] == pytest.approx((1 - gain) * a * sum39, rel=1e-12)
    # the model is the scaled component: gain a B_3 centred on p
    want = np.zeros((n, n))
    want[py - 2:py + 3, px - 2:px + 3] = gain * a * b3[n - 2:n + 3, n - 2:n + 3]
    assert np.max(np.abs(res.model - want)) < 1e-14
    # the oracle's scale kernels and bias are the hand-written ones
    assert np.max(np.abs(msclean.scale_kernel(3, n) - b3)) < 1e-15
    assert np.max(np.abs(msclean.scale_kernel(9, n) - b9)) < 1e-15
    assert np.allclose(msclean.bias([0, 3, 9]), [1.0, 0.8, 0.4], rtol=0, atol=1e-15)
