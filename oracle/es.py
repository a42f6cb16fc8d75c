"""Exponential-of-semicircle (ES) gridding kernel and its Fourier transform.

The paper grids with "the improved w-gridder" (Sec. 2, Sec. 5.1; Ye et al.
2022), whose kernel is the ES function of Barnett, Magland & af Klinteberg
(2019):

    phi(z) = exp(beta * (sqrt(1 - z^2) - 1))   for |z| <= 1, 0 otherwise,

evaluated at z = 2 (j - x) / W for a support of W grid cells, with
beta = 2.30 W at oversampling 2.

Its continuous Fourier transform, over the cell-unit variable s = W z / 2,

    Phi(f) = int phi(2 s / W) exp(2 pi i s f) ds
           = (W / 2) int_{-1}^{1} phi(z) cos(pi W z f) dz,

is the gridding correction in u, v (at f = l-offset / Ng) and in w (at
f = dw (n - 1)).  The substitution z = sin(theta) removes the square-root
branch point at z = +-1,

    Phi(f) = (W / 2) int_{-pi/2}^{pi/2} exp(beta (cos t - 1)) cos(pi W f sin t) cos t dt,

an analytic integrand, evaluated by Gauss-Legendre quadrature with enough
nodes that doubling them changes the value by less than 1e-15 (pinned in the
tests).
"""
from __future__ import annotations

import numpy as np

BETA_PER_CELL = 2.30
QUAD_NODES = 128


def beta_for(support: int) -> float:
    return BETA_PER_CELL * support


def es_kernel(z: np.ndarray, beta: float) -> np.ndarray:
    z = np.asarray(z, dtype=np.float64)
    inside = np.abs(z) <= 1.0
    out = np.zeros_like(z)
    out[inside] = np.exp(beta * (np.sqrt(1.0 - z[inside] ** 2) - 1.0))
    return out


def es_fourier(f: np.ndarray, support: int, beta: float, nodes: int = QUAD_NODES) -> np.ndarray:
    """Phi(f) by Gauss-Legendre quadrature in theta on [-pi/2, pi/2]."""
    f = np.asarray(f, dtype=np.float64)
    x, wq = np.polynomial.legendre.leggauss(nodes)
    th = 0.5 * np.pi * x
    wt = 0.5 * np.pi * wq * np.exp(beta * (np.cos(th) - 1.0)) * np.cos(th)
    st = np.sin(th)
    shape = f.shape
    ff = f.reshape(-1)
    out = np.empty_like(ff)
    chunk = 1 << 14
    for i in range(0, ff.size, chunk):
        fc = ff[i:i + chunk]
        out[i:i + chunk] = (0.5 * support) * (np.cos(np.pi * support * np.outer(fc, st)) @ wt)
    return out.reshape(shape)
