"""Partition by |uv| (Sec. 3, Fig. 3) and the tile sort order of the samples.

Radius of a sample in pixels of the N x N image's Fourier grid:
    r = sqrt(pu^2 + pv^2),  pu = u_lambda * (N dl),  pv = v_lambda * (N dl),
evaluated in IEEE float64 with every product and sum rounded separately
(numpy never contracts to FMA), so the masks are reproducible bit for bit.

Overlapping domains (Sec. 3: "L and H are not mutually exclusive"; ell is the
radius bisecting the overlap, delta its half-width, delta = 1 px per Sec. 5.1):
with ring radii ell_1 < ... < ell_{P-1},
    sample in partition p  <=>  (p == 0   or r >= ell_p - delta)
                           and  (p == P-1 or r <= ell_{p+1} + delta),
both bounds inclusive.  For P = 2 this is L: r <= ell + delta, H: r >= ell - delta.
Default ring radii: ell_i = the lower i/P quantile of r over all samples,
element floor(i (n - 1) / P) of the ascending sort (the lower median for P = 2).
Samples whose kernel footprint leaves the grid get mask 0 and are excluded.

Sort order: every (sample s, partition p) pair is an entry with the key
    (p, first w-plane p0, tile row j0v >> log2 T, tile column j0u >> log2 T)
packed into one unsigned 32-bit integer; entries are stably sorted by key
(ties keep ascending sample order).  Parity: bit-exact against the CUDA path.
"""
from __future__ import annotations

import numpy as np

from .gridder import Geometry


def radius_px(g: Geometry) -> np.ndarray:
    ndl = g.cell * (g.ng // 2)       # N * dl for the N x N image
    pu = g.ul * ndl
    pv = g.vl * ndl
    return np.sqrt(pu * pu + pv * pv)


def ring_radii(r: np.ndarray, nparts: int) -> np.ndarray:
    rs = np.sort(r)
    n = rs.shape[0]
    return np.array([rs[(i * (n - 1)) // nparts] for i in range(1, nparts)], dtype=np.float64)


def masks(r: np.ndarray, ells: np.ndarray, delta: float, nparts: int, inside: np.ndarray) -> np.ndarray:
    m = np.zeros(r.shape[0], dtype=np.uint8)
    for p in range(nparts):
        ok = np.ones(r.shape[0], dtype=bool)
        if p > 0:
            ok &= r >= (ells[p - 1] - delta)
        if p < nparts - 1:
            ok &= r <= (ells[p] + delta)
        m |= (ok.astype(np.uint8) << p)
    m[~inside] = 0
    return m


def key_layout(g: Geometry, tile: int, nparts: int):
    bt = int(np.log2(g.ng // tile))
    nblk = g.nw - g.Ww + 1 if g.nw > 0 else 1
    bw = int(np.ceil(np.log2(nblk))) if nblk > 1 else 0
    bp = int(np.ceil(np.log2(nparts))) if nparts > 1 else 0
    assert 2 * bt + bw + bp <= 32
    return bt, bw, bp


def entries(g: Geometry, mask: np.ndarray, tile: int, nparts: int):
    """Entries (key, sample, partition) in generation order: ascending sample,
    then ascending partition."""
    bt, bw, bp = key_layout(g, tile, nparts)
    lt = int(np.log2(tile))
    keys, samples, parts = [], [], []
    for p in range(nparts):
        sel = np.nonzero((mask >> p) & 1)[0]
        k = ((np.uint64(p) << np.uint64(2 * bt + bw))
             | (g.p0[sel].astype(np.uint64) << np.uint64(2 * bt))
             | ((g.j0v[sel] >> lt).astype(np.uint64) << np.uint64(bt))
             | (g.j0u[sel] >> lt).astype(np.uint64))
        keys.append(k)
        samples.append(sel)
        parts.append(np.full(sel.shape[0], p))
    keys = np.concatenate(keys)
    samples = np.concatenate(samples)
    parts = np.concatenate(parts)
    # generation order: by sample, then partition
    order = np.lexsort((parts, samples))
    return keys[order].astype(np.uint32), samples[order].astype(np.uint32), parts[order]


def sort_entries(keys: np.ndarray, samples: np.ndarray):
    perm = np.argsort(keys, kind="stable")
    return keys[perm], samples[perm]


def partition_offsets(sorted_keys: np.ndarray, g: Geometry, tile: int, nparts: int) -> np.ndarray:
    bt, bw, _ = key_layout(g, tile, nparts)
    part = sorted_keys.astype(np.uint64) >> np.uint64(2 * bt + bw)
    return np.searchsorted(part, np.arange(nparts + 1), side="left")


def weight_sums(weight: np.ndarray, mask: np.ndarray, nparts: int) -> np.ndarray:
    w = weight.reshape(-1).astype(np.float64)
    return np.array([w[((mask >> p) & 1) == 1].sum() for p in range(nparts)])
