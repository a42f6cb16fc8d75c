"""Pins of the Daubechies filters (db1 .. db8), the periodic orthonormal 2D DWT
and the concatenated dictionary."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("p", range(1, 9))
def test_daubechies_family_identities(p):
    """db_p: 2p taps, sum sqrt 2, unit norm, double-shift orthogonality,
    exactly p vanishing moments of the high-pass filter, minimum phase."""
    h = wavelet.daubechies(p)
    g = wavelet.highpass(h)
    k = 2 * p
    assert h.shape == (k,)
    assert abs(h.sum() - np.sqrt(2.0)) < 1e-13
    assert abs((h * h).sum() - 1.0) < 1e-11
    for m in range(1, p):
        assert abs(np.dot(h[2 * m:], h[:k - 2 * m])) < 1e-11
    t = np.arange(k) / k
    for j in range(p):
        assert abs(np.sum(g * t ** j)) < 1e-12
    assert abs(np.sum(g * t ** p)) > 1e-7
    assert np.sum(h[:p] ** 2) >= np.sum(h[p:] ** 2)       # (equal for the symmetric Haar filter)


def test_db1_and_db2_closed_forms():
    assert np.max(np.abs(wavelet.daubechies(1) - np.array([1.0, 1.0]) / np.sqrt(2.0))) < 1e-15
    s3 = np.sqrt(3.0)
    want = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * np.sqrt(2.0))
    assert np.max(np.abs(wavelet.daubechies(2) - want)) < 1e-15


def test_concatenated_dictionary_is_a_tight_frame():
    """W = [Psi_1 .. Psi_8] / sqrt 8: W W^T = I, ||W^T x|| = ||x||, and
    synthesis is the adjoint of analysis."""
    rng = np.random.default_rng(7)
    d = wavelet.Concatenation(3)
    x = rng.normal(size=(64, 64))
    c = d.analysis(x)
    assert c.shape == (8, 64, 64)
    assert np.max(np.abs(d.synthesis(c) - x)) < 1e-11
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-11 * np.linalg.norm(x)
    y = rng.normal(size=(8, 64, 64))
    assert abs(np.sum(c * y) - np.sum(x * d.synthesis(y))) < 1e-10
    # each member is its own orthonormal basis: the frame is redundant, not a basis
    assert np.linalg.norm(d.analysis(d.synthesis(y)) - y) > 0.5 * np.linalg.norm(y)
