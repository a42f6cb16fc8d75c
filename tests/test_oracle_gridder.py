"""Pins of the FP64 ES gridder (G, G^H, F of Eq. 2) and its correction."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import dft, es, gridder


def test_es_fourier_quadrature_converged():
    f = np.linspace(-0.5, 0.5, 41)
    a = es.es_fourier(f, 8, es.beta_for(8))
    b = es.es_fourier(f, 8, es.beta_for(8), nodes=2 * es.QUAD_NODES)
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(a))


def test_es_fourier_reduces_to_sinc_at_beta_zero():
    # phi = 1 on [-1, 1]  =>  Phi(f) = sin(pi W f) / (pi f)
    f = np.array([0.013, 0.1, 0.25, 0.37, 0.5])
    W = 8
    exact = np.sin(np.pi * W * f) / (np.pi * f)
    # beta = 0 keeps the cos(t) Jacobian smooth; the integrand is analytic
    got = es.es_fourier(f, W, 0.0)
    assert np.allclose(got, exact, rtol=0, atol=1e-13)


def test_es_fourier_matches_adaptive_quadrature():
    for f in (0.0, 0.11, 0.3, 0.49):
        ref = 4.0 * quad(lambda z: np.exp(18.4 * (np.sqrt(1 - z * z) - 1)) * np.cos(np.pi * 8 * z * f),
                         -1, 1, epsabs=1e-14, epsrel=1e-13, limit=400)[0]
        assert es.es_fourier(np.array([f]), 8, 18.4)[0] == pytest.approx(ref, rel=1e-10, abs=1e-12)


@pytest.mark.parametrize("nw", [0, 16])
def test_grid_degrid_adjoint(obs_small, obs_wstack, nw):
    o = obs_small if nw == 0 else obs_wstack
    g = gridder.geometry(o.uvw, o.freq, o.n, o.cell_rad, W=8, nw=nw)
    rng = np.random.default_rng(7)
    x = rng.normal(size=(o.n, o.n))
    y = rng.normal(size=o.nvis) + 1j * rng.normal(size=o.nvis)
    y[~g.inside] = 0
    lhs = np.vdot(y, gridder.degrid(x, g)).real
    rhs = float(np.sum(x * gridder.grid_adjoint(y, g)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _subset(o, k, seed=0):
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(o.nrow, k, replace=False))
    return o.uvw[rows], rows


@pytest.mark.parametrize("nw", [0, 16])
def test_gridder_matches_direct_dft(obs_small, obs_wstack, nw):
    o = obs_small if nw == 0 else obs_wstack
    uvw, rows = _subset(o, 300)
    g = gridder.geometry(uvw, o.freq, o.n, o.cell_rad, W=8, nw=nw)
    assert g.inside.all()
    rng = np.random.default_rng(8)
    x = np.zeros((o.n, o.n))
    idx = rng.integers(int(0.1 * o.n), int(0.9 * o.n), (20, 2))
    x[idx[:, 0], idx[:, 1]] = rng.uniform(0.1, 1.0, 20)
    u, v, w = dft.uvw_lambda(uvw, o.freq)
    ref = dft.degrid(x, u, v, w, o.cell_rad, nw > 0)
    got = gridder.degrid(x, g)
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)
    y = rng.normal(size=u.shape) + 1j * rng.normal(size=u.shape)
    ref_i = dft.adjoint(y, u, v, w, o.n, o.cell_rad, nw > 0)
    got_i = gridder.grid_adjoint(y, g)
    assert np.linalg.norm(got_i - ref_i) <= 1e-6 * np.linalg.norm(ref_i)


def test_error_decreases_with_support(obs_small):
    o = obs_small
    uvw, _ = _subset(o, 200, seed=1)
    rng = np.random.default_rng(9)
    x = np.zeros((o.n, o.n))
    x[rng.integers(20, 108, 15), rng.integers(20, 108, 15)] = 1.0
    u, v, w = dft.uvw_lambda(uvw, o.freq)
    ref = dft.degrid(x, u, v, w, o.cell_rad, False)
    errs = []
    for W in (4, 6, 8):
        g = gridder.geometry(uvw, o.freq, o.n, o.cell_rad, W=W, nw=0)
        errs.append(np.linalg.norm(gridder.degrid(x, g) - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6


def test_wstacking_off_centre_point_large_w(obs_wstack):
    """A point far from the centre, samples with large |w|: the w-stacked
    gridder reproduces S n^-1 exp(-2 pi i (u l + v m + w (n-1)))."""
    o = obs_wstack
    g = gridder.geometry(o.uvw, o.freq, o.n, o.cell_rad, W=8, nw=16)
    u, v, w = g.ul, g.vl, g.wl
    big = np.argsort(-np.abs(w))[:200]
    x = np.zeros((o.n, o.n))
    b, a = 30, 220
    x[b, a] = 0.7
    l = (a - o.n // 2) * o.cell_rad
    m = (b - o.n // 2) * o.cell_rad
    nn = np.sqrt(1 - l * l - m * m)
    exact = 0.7 / nn * np.exp(-2j * np.pi * (u * l + v * m + w * (nn - 1)))
    got = gridder.degrid(x, g)
    assert np.abs(w[big]).min() * abs(nn - 1) > 1e-3      # the w-term matters here
    assert np.max(np.abs(got[big] - exact[big])) <= 1e-6 * 0.7
    # dropping the w-term would be far off
    assert np.max(np.abs(0.7 / nn * np.exp(-2j * np.pi * (u * l + v * m)) - exact)[big]) > 1e-3


def test_psf_peak_normalised(obs_small):
    o = obs_small
    g2 = gridder.geometry(o.uvw, o.freq, o.n, o.cell_rad, W=8, nw=0, image_scale=2)
    p = gridder.psf(o.weight.reshape(-1).astype(np.float64), g2)
    assert p.shape == (2 * o.n, 2 * o.n)
    assert p[o.n, o.n] == pytest.approx(1.0, abs=1e-6)
    assert np.unravel_index(np.argmax(p), p.shape) == (o.n, o.n)
