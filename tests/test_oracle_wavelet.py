"""Pins of the Daubechies-4 filter and the periodic orthonormal 2D DWT."""
import numpy as np

from oracle import wavelet


def test_db4_filter_identities():
    h = wavelet.H_DB4
    assert h.shape == (8,)
    assert abs(h.sum() - np.sqrt(2.0)) < 1e-14
    assert abs((h * h).sum() - 1.0) < 1e-14
    for m in (1, 2, 3):                                  # double-shift orthogonality
        assert abs(np.dot(h[2 * m:], h[:8 - 2 * m])) < 1e-14
    i = np.arange(8)
    for k in range(4):                                   # 4 vanishing moments of g
        assert abs(np.sum(wavelet.G_DB4 * i ** k)) < 1e-10 * 8 ** k
    assert abs(np.sum(wavelet.G_DB4 * i ** 4)) > 1e-3     # and not 5
    assert h[0] > 0.2 and abs(h[7]) < 0.02                # minimum-phase ordering


def test_dwt_perfect_reconstruction_and_orthonormal():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(64, 64))
    c = wavelet.dwt2(x, 3)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    assert np.max(np.abs(wavelet.idwt2(c, 3) - x)) < 1e-12
    y = rng.normal(size=(64, 64))
    # <W^T x, y> = <x, W y>
    assert abs(np.sum(c * y) - np.sum(x * wavelet.idwt2(y, 3))) < 1e-11


def test_dwt_kills_low_order_polynomials_in_detail_bands():
    n = 32
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    # a cubic along rows, periodic wrap only affects the last taps: check interior details
    x = (xx.astype(float) / n) ** 3 + 0.0 * yy
    c = wavelet.dwt2(x, 1)
    detail_rows = c[:n // 2, n // 2:n // 2 + n // 2 - 4]  # row-detail band away from the wrap
    assert np.max(np.abs(detail_rows)) < 1e-12
