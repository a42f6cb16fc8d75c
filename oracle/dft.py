"""Direct (non-uniform) DFT measurement operator: the exact reference.

Eq. 1 with C = D = 1:  V(u, v, w) = sum_{pixels} I(l, m) / n
                                     * exp(-2 pi i (u l + v m + w (n - 1))),
n = sqrt(1 - l^2 - m^2).  Pixel (row b, column a) of an N x N image sits at
l = (a - N/2) dl, m = (b - N/2) dl (phase centre at pixel (N/2, N/2); l grows
with the column, m with the row).  In coplanar mode the w-term and the 1/n
factor are dropped (Sec. 2: "if we ignore ... the e^{-2 pi i w (n-1)} terms,
Eq. 1 simplifies to a two-dimensional Fourier transform").

``degrid``   = A x
``adjoint``  = Re(A^H y)            (unnormalised)
``dirty``    = Re(A^H (w . y)) / sum(w)
``psf``      = dirty image of unit visibilities on a 2N x 2N image
``residual`` = Eq. 2 with exact operators: Re(A^H (w . (v - A x))) / sum(w)

Coordinates u, v, w are in wavelengths (u_m * f / c).  Parity: pinned by
adjointness, the phase-centre point source, the PSF peak and a brute-force
triple loop (tests/test_oracle_dft.py).
"""
from __future__ import annotations

import numpy as np

C_LIGHT = 299792458.0


def lmn(n: int, cell: float):
    off = (np.arange(n) - n // 2) * cell
    m, l = np.meshgrid(off, off, indexing="ij")      # [row, col]
    r2 = l * l + m * m
    nn = np.sqrt(1.0 - r2)
    nm1 = -r2 / (1.0 + nn)                           # n - 1 without cancellation
    return l, m, nn, nm1


def uvw_lambda(uvw_m: np.ndarray, freq: np.ndarray):
    """(nrow*nchan,) u, v, w in wavelengths, row-major sample order."""
    s = freq / C_LIGHT
    u = (uvw_m[:, 0:1] * s[None, :]).reshape(-1)
    v = (uvw_m[:, 1:2] * s[None, :]).reshape(-1)
    w = (uvw_m[:, 2:3] * s[None, :]).reshape(-1)
    return u, v, w


def _phase(u, v, w, l, m, nm1, wterm):
    ph = np.outer(u, l.reshape(-1)) + np.outer(v, m.reshape(-1))
    if wterm:
        ph += np.outer(w, nm1.reshape(-1))
    return ph


def degrid(image: np.ndarray, u, v, w, cell: float, wterm: bool, chunk: int = 2048) -> np.ndarray:
    n = image.shape[0]
    l, m, nn, nm1 = lmn(n, cell)
    x = (image / nn if wterm else image).reshape(-1).astype(np.complex128)
    out = np.empty(u.shape[0], dtype=np.complex128)
    for i in range(0, u.shape[0], chunk):
        ph = _phase(u[i:i + chunk], v[i:i + chunk], w[i:i + chunk], l, m, nm1, wterm)
        out[i:i + chunk] = np.exp(-2j * np.pi * ph) @ x
    return out


def adjoint(y: np.ndarray, u, v, w, n: int, cell: float, wterm: bool, chunk: int = 2048) -> np.ndarray:
    l, m, nn, nm1 = lmn(n, cell)
    acc = np.zeros(n * n, dtype=np.complex128)
    for i in range(0, u.shape[0], chunk):
        ph = _phase(u[i:i + chunk], v[i:i + chunk], w[i:i + chunk], l, m, nm1, wterm)
        acc += y[i:i + chunk] @ np.exp(2j * np.pi * ph)
    img = acc.real.reshape(n, n)
    return img / nn if wterm else img


def dirty(vis, weight, u, v, w, n, cell, wterm):
    return adjoint(weight * vis, u, v, w, n, cell, wterm) / weight.sum()


def psf(weight, u, v, w, n, cell, wterm):
    """2N x 2N point spread function, normalised by the weight sum."""
    return adjoint(weight.astype(np.complex128), u, v, w, 2 * n, cell, wterm) / weight.sum()


def residual(vis, weight, model, u, v, w, cell, wterm):
    n = model.shape[0]
    r = vis - degrid(model, u, v, w, cell, wterm)
    return adjoint(weight * r, u, v, w, n, cell, wterm) / weight.sum()


def degrid_pixels_sparse(image: np.ndarray, u, v, w, cell, wterm) -> np.ndarray:
    """A x evaluated only over the non-zero pixels of x (same arithmetic as
    ``degrid``; for sparse models at large N)."""
    n = image.shape[0]
    rows, cols = np.nonzero(image)
    l = (cols - n // 2) * cell
    m = (rows - n // 2) * cell
    r2 = l * l + m * m
    nn = np.sqrt(1.0 - r2)
    nm1 = -r2 / (1.0 + nn)
    amp = image[rows, cols] / nn if wterm else image[rows, cols]
    ph = np.outer(u, l) + np.outer(v, m)
    if wterm:
        ph += np.outer(w, nm1)
    return np.exp(-2j * np.pi * ph) @ amp.astype(np.complex128)


def adjoint_at(y, u, v, w, n, cell, wterm, rows, cols) -> np.ndarray:
    """Re(A^H y) at the listed pixels only."""
    l = (np.asarray(cols) - n // 2) * cell
    m = (np.asarray(rows) - n // 2) * cell
    r2 = l * l + m * m
    nn = np.sqrt(1.0 - r2)
    nm1 = -r2 / (1.0 + nn)
    out = np.empty(l.shape[0])
    for k in range(l.shape[0]):
        ph = u * l[k] + v * m[k]
        if wterm:
            ph = ph + w * nm1[k]
        val = np.dot(y, np.exp(2j * np.pi * ph)).real
        out[k] = val / nn[k] if wterm else val
    return out
