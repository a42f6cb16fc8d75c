"""Pins of the FISTA minor cycle (Eq. 4-5)."""
import numpy as np
import pytest

from oracle import filters, fista, wavelet


def _problem(seed=0, n=16, gamma_n=1.0):
    rng = np.random.default_rng(seed)
    psf = np.zeros((2 * n, 2 * n))
    yy, xx = np.meshgrid(np.arange(2 * n) - n, np.arange(2 * n) - n, indexing="ij")
    psf = np.exp(-(xx ** 2 + yy ** 2) / 4.0) * (1 + 0.1 * np.cos(xx))
    psf /= psf[n, n]
    h = filters.psf_spectrum(psf)
    gam = filters.gammas(n, np.array([5.0]), 1.0, 2)
    dirty = rng.normal(size=(n, n))
    rho = rng.normal(size=(n, n)) * 0.3
    prob = fista.problem(filters.image_spectrum(dirty), h, gam[0],
                         [(gam[1], filters.image_spectrum(rho))], gamma_n)
    return prob, n


def test_gradient_matches_finite_differences():
    prob, n = _problem()
    rng = np.random.default_rng(1)
    x = rng.normal(size=(n, n))
    d = rng.normal(size=(n, n))
    eps = 1e-6
    fd = (prob.data_term(x + eps * d) - prob.data_term(x - eps * d)) / (2 * eps)
    an = float(np.sum(prob.grad(x) * d))
    assert fd == pytest.approx(an, rel=1e-7)


def test_data_term_matches_image_domain_norms():
    """f(x) written with padded-grid images instead of spectra."""
    rng = np.random.default_rng(2)
    n = 16
    psf = rng.normal(size=(2 * n, 2 * n))
    h = filters.psf_spectrum(psf)
    gam = filters.gammas(n, np.array([5.0]), 1.0, 2)
    dirty, rho, x = (rng.normal(size=(n, n)) for _ in range(3))
    prob = fista.problem(filters.image_spectrum(dirty), h, gam[0],
                         [(gam[1], filters.image_spectrum(rho))], 1.0)
    t1 = filters.ispectrum(gam[0] * (filters.image_spectrum(dirty) - h * filters.image_spectrum(x)))
    t2 = filters.ispectrum(filters.image_spectrum(rho) - gam[1] * filters.image_spectrum(x))
    want = np.sum(np.abs(t1) ** 2) + np.sum(np.abs(t2) ** 2)
    assert prob.data_term(x) == pytest.approx(want, rel=1e-10)


def test_lipschitz_bounds_power_iteration():
    prob, n = _problem()
    rng = np.random.default_rng(3)
    v = rng.normal(size=(n, n))
    g0 = prob.grad(np.zeros((n, n)))
    for _ in range(200):
        hv = prob.grad(v) - g0
        v = hv / np.linalg.norm(hv)
    lam_max = np.linalg.norm(prob.grad(v) - g0)
    assert lam_max <= prob.lipschitz * (1 + 1e-9)
    assert lam_max >= 0.2 * prob.lipschitz


def test_kkt_after_many_iterations():
    prob, n = _problem(seed=4)
    lam = 0.5
    xbar, alpha = fista.solve(prob, lam, 5000, 2)
    g = wavelet.dwt2(prob.grad(wavelet.idwt2(alpha, 2)), 2)
    zero = alpha == 0
    assert zero.any() and (~zero).any()
    assert np.all(np.abs(g[zero]) <= lam * (1 + 1e-6))
    assert np.allclose(g[~zero], -lam * np.sign(alpha[~zero]), atol=1e-6 * lam)


def test_fista_beats_ista_after_50():
    prob, n = _problem(seed=5)
    lam = 0.2
    _, a_f = fista.solve(prob, lam, 50, 2, accelerate=True)
    _, a_i = fista.solve(prob, lam, 50, 2, accelerate=False)
    assert fista.objective(prob, a_f, lam, 2) <= fista.objective(prob, a_i, lam, 2)


def test_kkt_with_the_concatenated_dictionary():
    prob, n = _problem(seed=6, n=8)
    d = wavelet.Concatenation(2)
    lam = 0.3 * float(np.abs(d.analysis(prob.grad(np.zeros((n, n))))).max())
    _, alpha = fista.solve(prob, lam, 2000, 2, dictionary=d)
    g = d.analysis(prob.grad(d.synthesis(alpha)))
    zero = alpha == 0
    assert zero.any() and (~zero).any()
    assert np.all(np.abs(g[zero]) <= lam * (1 + 1e-6))
    assert np.allclose(g[~zero], -lam * np.sign(alpha[~zero]), atol=1e-5 * lam)


def test_fista_beats_ista_with_the_concatenated_dictionary():
    prob, n = _problem(seed=8)
    d = wavelet.Concatenation(2)
    lam = 0.2
    _, a_f = fista.solve(prob, lam, 50, 2, dictionary=d)
    _, a_i = fista.solve(prob, lam, 50, 2, accelerate=False, dictionary=d)
    assert fista.objective(prob, a_f, lam, 2, d) <= fista.objective(prob, a_i, lam, 2, d)


def test_lambda_at_the_kkt_threshold_gives_the_zero_solution():
    """alpha = 0 is optimal iff lambda >= max |W^T grad f(0)|; FISTA from 0
    stays at 0 above the threshold and moves below it (both dictionaries)."""
    prob, n = _problem(seed=9)
    for d in (None, wavelet.Concatenation(2)):
        W, WT, _ = fista._operators(2, d)
        thr = float(np.abs(WT(prob.grad(np.zeros((n, n))))).max())
        above, _ = fista.solve(prob, 1.001 * thr, 20, 2, dictionary=d)
        below, _ = fista.solve(prob, 0.99 * thr, 20, 2, dictionary=d)
        assert np.all(above == 0.0)
        assert np.abs(below).max() > 0.0
