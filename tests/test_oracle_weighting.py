"""Pins of uniform weighting (Sec. 5.1; reading in oracle/weighting.py)."""
import numpy as np

from oracle import framework, gridder, weighting


def _geometry(u, v, n=64, cell=1e-4):
    """Samples at given (u, v) in cells of the N x N uv grid, one channel."""
    ndl = cell * n
    lam = 299792458.0 / 1e9
    uvw = np.stack([np.asarray(u) / ndl * lam, np.asarray(v) / ndl * lam, np.zeros(len(u))], axis=1)
    return gridder.geometry(uvw, np.array([1e9]), n, cell, W=8, nw=0)


def test_hand_worked_cells_and_weights():
    # two samples in cell (3, -2), one in its mirror (-3, 2), one alone in (5, 5),
    # one at the origin: weights 1/3, 1/3, 1/3, 1, 1/2
    g = _geometry([3.2, 2.7, -3.4, 5.0, 0.1], [-2.1, -1.6, 2.4, 5.3, -0.2])
    a, b = weighting.cells(g)
    assert list(a) == [3, 3, -3, 5, 0] and list(b) == [-2, -2, 2, 5, 0]
    w = weighting.uniform_weights(g, np.ones(5, np.float32))
    assert w.dtype == np.float32
    assert np.array_equal(w, np.array([1 / 3, 1 / 3, 1 / 3, 1.0, 0.5], np.float32))


def test_cells_are_the_nearest_cell_centres():
    rng = np.random.default_rng(0)
    u, v = rng.uniform(-20, 20, 500), rng.uniform(-20, 20, 500)
    g = _geometry(u, v)
    a, b = weighting.cells(g)
    ndl = g.cell * (g.ng // 2)
    assert np.all(np.abs(g.ul * ndl - a) <= 0.5) and np.all(np.abs(g.vl * ndl - b) <= 0.5)


def test_each_occupied_cell_pair_carries_unit_weight():
    """Sum of the uniform weights over a cell and its mirror is 1 (1/2 for the
    self-mirrored origin), whatever the natural weights."""
    rng = np.random.default_rng(1)
    u, v = rng.normal(0, 6, 2000), rng.normal(0, 6, 2000)
    g = _geometry(u, v)
    w0 = rng.uniform(0.5, 2.0, 2000).astype(np.float32)
    w = weighting.uniform_weights(g, w0).astype(np.float64)
    a, b = weighting.cells(g)
    pairs = {}
    for k in range(2000):
        key = min((a[k], b[k]), (-a[k], -b[k]))
        pairs[key] = pairs.get(key, 0.0) + w[k]
    for key, tot in pairs.items():
        want = 0.5 if key == (0, 0) else 1.0
        assert abs(tot - want) < 1e-6


def test_uniform_setup_images_with_uniform_weights(obs_small):
    o = obs_small
    st = framework.setup(o.uvw, o.freq, o.weight, o.n, o.cell_rad, 0, 2, scheme="uniform")
    want = weighting.uniform_weights(st.geom, o.weight)
    assert np.array_equal(st.weight.reshape(-1), want)
    assert np.allclose(st.wsum, [want[((st.mask >> p) & 1) == 1].astype(np.float64).sum() for p in range(2)],
                       rtol=1e-12)
    # natural setup keeps the given weights
    st0 = framework.setup(o.uvw, o.freq, o.weight, o.n, o.cell_rad, 0, 2)
    assert np.array_equal(st0.weight, o.weight)
