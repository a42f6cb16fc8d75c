"""Pins of the direct-DFT operator (Eq. 1) against mathematics it must obey."""
import math

import numpy as np
import pytest

from oracle import dft, filters


def _tiny(rng, n=16, ns=50, wscale=200.0):
    u = rng.normal(0, 2.0 / (n * 1e-3) / 3, ns)
    v = rng.normal(0, 2.0 / (n * 1e-3) / 3, ns)
    w = rng.normal(0, wscale, ns)
    return u, v, w, 1e-3


@pytest.mark.parametrize("wterm", [False, True])
def test_adjointness(wterm):
    rng = np.random.default_rng(1)
    u, v, w, cell = _tiny(rng)
    x = rng.normal(size=(16, 16))
    y = rng.normal(size=50) + 1j * rng.normal(size=50)
    lhs = np.vdot(y, dft.degrid(x, u, v, w, cell, wterm)).real
    rhs = float(np.sum(x * dft.adjoint(y, u, v, w, 16, cell, wterm)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("wterm", [False, True])
def test_phase_centre_point_source_constant(wterm):
    rng = np.random.default_rng(2)
    u, v, w, cell = _tiny(rng)
    x = np.zeros((16, 16))
    x[8, 8] = 2.5
    vis = dft.degrid(x, u, v, w, cell, wterm)
    assert np.allclose(vis, 2.5, rtol=0, atol=1e-14)


@pytest.mark.parametrize("wterm", [False, True])
def test_brute_force_triple_loop(wterm):
    rng = np.random.default_rng(3)
    u, v, w, cell = _tiny(rng)
    x = rng.normal(size=(16, 16))
    ref = np.zeros(50, dtype=complex)
    for k in range(50):
        acc = 0j
        for b in range(16):
            for a in range(16):
                l = (a - 8) * cell
                m = (b - 8) * cell
                nn = math.sqrt(1 - l * l - m * m)
                ph = u[k] * l + v[k] * m + (w[k] * (nn - 1) if wterm else 0.0)
                acc += x[b, a] / (nn if wterm else 1.0) * complex(math.cos(-2 * math.pi * ph),
                                                                  math.sin(-2 * math.pi * ph))
        ref[k] = acc
    got = dft.degrid(x, u, v, w, cell, wterm)
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("wterm", [False, True])
def test_psf_peak_is_weight_sum(wterm):
    rng = np.random.default_rng(4)
    u, v, w, cell = _tiny(rng)
    wt = rng.uniform(0.5, 2.0, 50)
    unnorm = dft.adjoint(wt.astype(complex), u, v, w, 32, cell, wterm)
    assert unnorm[16, 16] == pytest.approx(wt.sum(), rel=1e-14)
    assert np.argmax(unnorm) == 16 * 32 + 16


def test_coplanar_psf_symmetric():
    rng = np.random.default_rng(5)
    u, v, w, cell = _tiny(rng)
    wt = np.ones(50)
    p = dft.psf(wt, u, v, w, 16, cell, False)
    # psf(-d) = psf(d) about the centre (16, 16)
    inner = p[1:, 1:]
    assert np.allclose(inner, inner[::-1, ::-1], atol=1e-13)


def test_coplanar_normal_operator_is_psf_convolution():
    """A^H(w . A x) = (sum w) psf_2N (*) x, exactly, in coplanar mode."""
    rng = np.random.default_rng(6)
    u, v, w, cell = _tiny(rng)
    wt = rng.uniform(0.5, 2.0, 50)
    x = rng.normal(size=(16, 16))
    lhs = dft.adjoint(wt * dft.degrid(x, u, v, w, cell, False), u, v, w, 16, cell, False)
    p = dft.psf(wt, u, v, w, 16, cell, False) * wt.sum()
    rhs = filters.apply(x, filters.psf_spectrum(p))
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(lhs))
