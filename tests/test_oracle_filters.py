"""Pins of the filters Gamma_p and the padded convolutions."""
import numpy as np
import pytest
from scipy.signal import convolve2d

from oracle import filters


@pytest.mark.parametrize("nparts,ells", [(2, [10.3]), (4, [5.0, 9.5, 17.2])])
def test_gammas_partition_of_unity(nparts, ells):
    n = 64
    gam = filters.gammas(n, np.array(ells), 1.0, nparts)
    assert np.allclose(gam.sum(axis=0), 1.0, atol=1e-15)
    r = filters.radius_grid(n)
    lo = [-np.inf] + [e - 1.0 for e in ells]
    hi = [e + 1.0 for e in ells] + [np.inf]
    for p in range(nparts):
        assert np.all(gam[p] >= 0)
        core = (r >= (lo[p] + 2.0 if p else -1)) & (r <= (hi[p] - 2.0 if p < nparts - 1 else 1e9))
        assert np.all(gam[p][core] == 1.0)
        outside = (r < lo[p]) | (r > hi[p])
        assert np.all(gam[p][outside] == 0.0)


def test_padded_convolution_is_linear_convolution():
    rng = np.random.default_rng(0)
    n = 16
    x = rng.normal(size=(n, n))
    k2n = rng.normal(size=(2 * n, 2 * n))          # kernel, centre at (n, n)
    got = filters.apply(x, filters.psf_spectrum(k2n))
    full = convolve2d(x, k2n[1:, 1:])              # offsets -(n-1) .. (n-1)
    # output pixel p gets sum_q x[q] k[p - q]; in 'full' mode index p + (n-1)
    want = full[n - 1:2 * n - 1, n - 1:2 * n - 1]
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_band_limited_exchange_is_lossless_and_smaller():
    """Sec. 6.3: Phi_p is determined by Gamma_p F pad i_bar on the ring
    support of Gamma_p (half plane, by Hermitian symmetry): unpacking the
    packed coefficients gives Gamma_p i_bar as filters.apply does, to
    rounding; outside the support the filtered spectrum is exactly 0; the
    inner partition's message is much smaller than the N x N image."""
    n = 64
    rng = np.random.default_rng(3)
    ibar = rng.standard_normal((n, n))
    ells = np.array([9.5, 19.0])
    gam = filters.gammas(n, ells, 1.0, 3)
    for p in range(3):
        idx = filters.ring_support(gam[p])
        coef = filters.phi_pack(ibar, gam[p], idx)
        phi = filters.phi_unpack(coef, idx, n)
        want = filters.apply(ibar, gam[p])
        assert np.max(np.abs(phi - want)) < 1e-12 * np.max(np.abs(want))
        full = (gam[p] * filters.image_spectrum(ibar)).reshape(-1)
        outside = np.ones(full.shape[0], dtype=bool)
        ju = np.arange(full.shape[0]) // (2 * n)
        outside[idx] = False
        assert np.all(full[outside & (ju <= n)] == 0.0)
    # the inner ring's message: about the half disk of radius 2 (ell + delta)
    # grid cells, pi (2 (ell + delta))^2 / 2 complex values, against n^2 reals
    idx0 = filters.ring_support(gam[0])
    half_disk = np.pi * (2 * (ells[0] + 1.0)) ** 2 / 2
    assert abs(idx0.shape[0] - half_disk) < 0.05 * half_disk
    assert 2 * idx0.shape[0] < 0.35 * n * n
