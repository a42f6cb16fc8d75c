"""Pins of the |uv| partition (Sec. 3) and the tile sort order."""
import math

import numpy as np
import pytest

from oracle import gridder, partition


def test_masks_match_plain_python_loop(obs_small):
    o = obs_small
    g = gridder.geometry(o.uvw, o.freq, o.n, o.cell_rad, W=8, nw=0)
    r = partition.radius_px(g)
    ells = partition.ring_radii(r, 2)
    m = partition.masks(r, ells, 1.0, 2, g.inside)
    c = 299792458.0
    ndl = o.cell_rad * o.n
    srt = sorted(r.tolist())
    ell = srt[(len(srt) - 1) // 2]
    assert ell == ells[0]
    for k in range(0, o.nvis, 7):
        row, ch = divmod(k, o.nchan)
        s = float(o.freq[ch]) / c
        pu = (float(o.uvw[row, 0]) * s) * ndl
        pv = (float(o.uvw[row, 1]) * s) * ndl
        rr = math.sqrt(pu * pu + pv * pv)
        want = (1 if rr <= ell + 1.0 else 0) | (2 if rr >= ell - 1.0 else 0)
        assert rr == r[k]
        assert m[k] == want


@pytest.mark.parametrize("nparts", [2, 4])
def test_every_sample_in_some_partition_and_balanced(obs_wstack, nparts):
    o = obs_wstack
    g = gridder.geometry(o.uvw, o.freq, o.n, o.cell_rad, W=8, nw=16)
    r = partition.radius_px(g)
    ells = partition.ring_radii(r, nparts)
    m = partition.masks(r, ells, 1.0, nparts, g.inside)
    assert np.all(m[g.inside] != 0)
    counts = np.array([((m >> p) & 1).sum() for p in range(nparts)])
    frac = counts / g.inside.sum()
    # ring radii are the i/P quantiles: each partition holds about 1/P
    assert np.all(np.abs(frac - 1.0 / nparts) < 0.1)
    overlap = (np.array([bin(int(v)).count("1") for v in m]) > 1).mean()
    assert 0.0 < overlap < 0.1 * (nparts - 1)


def test_sort_matches_python_sorted(obs_wstack):
    o = obs_wstack
    g = gridder.geometry(o.uvw, o.freq, o.n, o.cell_rad, W=8, nw=16)
    r = partition.radius_px(g)
    m = partition.masks(r, partition.ring_radii(r, 2), 1.0, 2, g.inside)
    keys, samples, parts = partition.entries(g, m, 16, 2)
    sk, ss = partition.sort_entries(keys, samples)
    ref = sorted(zip(parts.tolist(), g.p0[samples].tolist(), (g.j0v[samples] // 16).tolist(),
                     (g.j0u[samples] // 16).tolist(), samples.tolist()))
    assert [t[-1] for t in ref] == ss.tolist()
    off = partition.partition_offsets(sk, g, 16, 2)
    assert off[0] == 0 and off[-1] == keys.shape[0]
    assert off[1] - off[0] == ((m & 1) == 1).sum()


def test_outside_samples_masked():
    rng = np.random.default_rng(0)
    uvw = rng.normal(0, 1, (100, 3)) * 10.0
    uvw[3] = (1e7, 0, 0)                      # far outside the grid
    g = gridder.geometry(uvw, np.array([1e9]), 64, 1e-4, W=8, nw=0)
    r = partition.radius_px(g)
    m = partition.masks(r, partition.ring_radii(r, 2), 1.0, 2, g.inside)
    assert not g.inside[3] and m[3] == 0
    assert g.inside.sum() == 99
