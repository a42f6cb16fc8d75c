"""Daubechies wavelets and the periodic orthonormal 2D DWT used as the
dictionary W of Eq. 4-5.

Two dictionaries: the Db4 member alone (8 taps, 4 vanishing moments; a single
orthonormal basis, W^T W = I), and the paper's concatenation of the first 8
Daubechies wavelets (Sec. 5.2): W = [Psi_1 ... Psi_8] / sqrt(8) with Psi_p the
orthonormal periodic DWT of db_p (2p taps, p vanishing moments), a tight frame
(W W^T = I, so ||W|| = 1 and the Lipschitz bound of the FISTA problem is
unchanged).  Each basis is transformed independently (Sec. 5.3).

Filter: Daubechies' construction.  With y = sin^2(w/2), the squared modulus
of the low-pass response is cos^{2N}(w/2) P(y), P(y) = sum_{k<N}
binom(N-1+k, k) y^k for N vanishing moments.  Substituting y = (2 - z - 1/z)/4 makes z^{N-1}
P a degree-2(N-1) polynomial whose roots come in pairs (r, 1/r); keeping the
roots inside the unit circle (spectral factorisation) and multiplying by
(1 + z)^N gives the filter, normalised to sum sqrt(2).  Coefficients are
ordered with the largest first (minimum phase).

Transform (periodic, analysis by correlation):
    a[k] = sum_i h[i] x[(2k + i) mod n],   d[k] = sum_i g[i] x[(2k + i) mod n],
    g[i] = (-1)^i h[7 - i];
2D level: along rows (last axis) then columns, outputs [a | d] in place; the
next level recurses on the top-left quadrant.  ``idwt2`` is the transpose.
"""
from __future__ import annotations

from math import comb

import numpy as np


def daubechies(nvm: int = 4) -> np.ndarray:
    pc = [comb(nvm - 1 + k, k) for k in range(nvm)]          # P(y) coefficients
    # P((2 - z - 1/z)/4) * z^(nvm-1) as a polynomial in z (highest power first)
    poly = np.zeros(2 * nvm - 1)
    base = np.array([-0.25, 0.5, -0.25])                      # z^1 * y(z) = (-z^2 + 2z - 1)/4
    term = np.array([1.0])
    for k in range(nvm):
        # y^k * z^k is a polynomial of degree 2k; shift to degree 2(nvm-1)
        padded = np.zeros(2 * nvm - 1)
        padded[nvm - 1 - k:nvm - 1 - k + term.shape[0]] = term
        poly += pc[k] * padded
        term = np.convolve(term, base)
    roots = np.roots(poly)
    inner = roots[np.abs(roots) < 1.0]
    h = np.real(np.poly(np.concatenate([inner, -np.ones(nvm)])))
    h = h * (np.sqrt(2.0) / h.sum())
    # choose the ordering with most energy first (minimum phase)
    if np.cumsum(h[::-1] ** 2)[nvm] > np.cumsum(h ** 2)[nvm]:
        h = h[::-1]
    return h.copy()


def highpass(h: np.ndarray) -> np.ndarray:
    """g[i] = (-1)^i h[K - 1 - i]."""
    k = h.shape[0]
    return np.array([(-1) ** i * h[k - 1 - i] for i in range(k)])


H_DB4 = daubechies(4)
G_DB4 = highpass(H_DB4)

# db1 .. db8, the members of the concatenated dictionary (Sec. 5.2)
SARA_ORDERS = tuple(range(1, 9))


def _analysis_last_axis(x: np.ndarray, h: np.ndarray, g: np.ndarray):
    n = x.shape[-1]
    idx = (2 * np.arange(n // 2)[:, None] + np.arange(h.shape[0])[None, :]) % n
    seg = x[..., idx]                                  # (..., n/2, taps)
    return seg @ h, seg @ g


def _synthesis_last_axis(a: np.ndarray, d: np.ndarray, h: np.ndarray, g: np.ndarray):
    half = a.shape[-1]
    n = 2 * half
    out = np.zeros(a.shape[:-1] + (n,))
    for i in range(h.shape[0]):
        idx = (2 * np.arange(half) + i) % n         # distinct indices for one tap i
        out[..., idx] += a * h[i] + d * g[i]
    return out


def dwt2(x: np.ndarray, levels: int, h: np.ndarray = H_DB4, g: np.ndarray = G_DB4) -> np.ndarray:
    c = np.array(x, dtype=np.float64, copy=True)
    n = c.shape[0]
    for _ in range(levels):
        blk = c[:n, :n]
        a, d = _analysis_last_axis(blk, h, g)
        blk = np.concatenate([a, d], axis=1)
        a, d = _analysis_last_axis(blk.T, h, g)
        c[:n, :n] = np.concatenate([a, d], axis=1).T
        n //= 2
    return c


def idwt2(c: np.ndarray, levels: int, h: np.ndarray = H_DB4, g: np.ndarray = G_DB4) -> np.ndarray:
    x = np.array(c, dtype=np.float64, copy=True)
    n0 = x.shape[0]
    for lev in reversed(range(levels)):
        n = n0 >> lev
        blk = x[:n, :n]
        cols = _synthesis_last_axis(blk.T[:, :n // 2], blk.T[:, n // 2:], h, g).T
        rows = _synthesis_last_axis(cols[:, :n // 2], cols[:, n // 2:], h, g)
        x[:n, :n] = rows
    return x


class Concatenation:
    """W = [Psi_p1 ... Psi_pm] / sqrt(m): coefficients of shape (m, n, n), one
    orthonormal periodic DWT (``levels`` levels) per member filter."""

    def __init__(self, levels: int, orders=SARA_ORDERS):
        self.levels = levels
        self.filters = [(h, highpass(h)) for h in (daubechies(p) for p in orders)]
        self.scale = 1.0 / np.sqrt(len(self.filters))

    def shape(self, n: int) -> tuple:
        return (len(self.filters), n, n)

    def synthesis(self, c: np.ndarray) -> np.ndarray:
        """x = W c = sum_p Psi_p c_p / sqrt(m)."""
        x = np.zeros(c.shape[1:])
        for k, (h, g) in enumerate(self.filters):
            x += idwt2(c[k], self.levels, h, g)
        return self.scale * x

    def analysis(self, x: np.ndarray) -> np.ndarray:
        """W^T x = [Psi_p^T x] / sqrt(m)."""
        return self.scale * np.stack([dwt2(x, self.levels, h, g) for h, g in self.filters])
