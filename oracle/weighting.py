"""Uniform weighting of the visibilities (Sec. 5.1: every dataset is imaged
with uniform weighting).  Test infrastructure: only tests, the smoke check and
the benchmark's CPU baseline use this package.

Reading (the paper names the scheme only): the uv plane is divided into the
cells of the N x N image's Fourier grid (spacing 1 / (N dl)); sample k falls in
the cell nearest to it,
    a_k = floor(pu_k + 1/2),  b_k = floor(pv_k + 1/2),
    pu = u_lambda (N dl),  pv = v_lambda (N dl)   (float64, as for the radius),
and, because the sky is real, also counts in the Hermitian mirror cell
(-a_k, -b_k).  The density of a cell is the sum of the natural weights of
the samples counted in it,
    D(a, b) = sum_{j: (a_j, b_j) = (a, b)} w_j + sum_{j: (-a_j, -b_j) = (a, b)} w_j,
over the samples inside the grid, and the uniform weight is
    w_k^u = w_k / D(a_k, b_k),
rounded to float32 (the precision in which the weights are held).  Samples
outside the grid are excluded from imaging and keep their weight.
"""
from __future__ import annotations

import numpy as np

from .gridder import Geometry


def cells(g: Geometry) -> tuple[np.ndarray, np.ndarray]:
    ndl = g.cell * (g.ng // 2)
    return np.floor(g.ul * ndl + 0.5).astype(np.int64), np.floor(g.vl * ndl + 0.5).astype(np.int64)


def uniform_weights(g: Geometry, weight: np.ndarray) -> np.ndarray:
    n = g.ng // 2
    w = np.asarray(weight, dtype=np.float64).reshape(-1)
    a, b = cells(g)
    ins = g.inside
    dens = np.zeros((n, n))
    np.add.at(dens, (a[ins] + n // 2, b[ins] + n // 2), w[ins])
    np.add.at(dens, (-a[ins] + n // 2, -b[ins] + n // 2), w[ins])
    out = w.copy()
    out[ins] = w[ins] / dens[a[ins] + n // 2, b[ins] + n // 2]
    return out.astype(np.float32)
