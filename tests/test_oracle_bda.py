"""Pins of the baseline-dependent averaging oracle (Sec. 6.2 and Sec. 7 item d;
Wijnholds et al. 2018): windows by brute force, the identity at a vanishing
shift bound, exact averages of a constant field, weight conservation, the
closed-form decorrelation of a point source on linear tracks, and the
flattening of the partition imbalance it exists for."""
import math

import numpy as np
import pytest

from oracle import bda, gridder, partition
from paper_2507_22128_gb300 import synth


def _small(n_times=24, n_ant=8, seed=3):
    rng = np.random.default_rng(seed)
    enu = synth.layout_log_spiral(rng, n_ant, 20.0, 2000.0)
    ha = np.linspace(-1.0, 1.0, n_times) * (15.0 * math.pi / 180.0)
    uvw = synth.uvw_tracks(enu, -30 * math.pi / 180, -30 * math.pi / 180, ha)
    nbl = n_ant * (n_ant - 1) // 2
    freq = np.array([1.3e9, 1.4e9, 1.5e9])
    vis = rng.standard_normal((uvw.shape[0], 3)) + 1j * rng.standard_normal((uvw.shape[0], 3))
    w = rng.uniform(0.5, 2.0, (uvw.shape[0], 3))
    return uvw, vis, w, n_times, nbl, freq


def test_windows_match_a_loop_over_baselines_and_times():
    uvw, vis, w, nt, nbl, freq = _small()
    n, cell, shift = 256, 1.0 * math.pi / 180 / 3600, 0.7
    k = bda.windows(uvw, nt, nbl, freq.max(), n, cell, shift)
    s = freq.max() / bda.C_LIGHT
    for b in range(nbl):
        best = 0.0
        for t in range(nt - 1):
            du = (uvw[(t + 1) * nbl + b, 0] - uvw[t * nbl + b, 0]) * s
            dv = (uvw[(t + 1) * nbl + b, 1] - uvw[t * nbl + b, 1]) * s
            best = max(best, math.sqrt(du * du + dv * dv) * (n * cell))
        want = nt if best == 0.0 else min(nt, max(1, math.floor(shift / best)))
        assert k[b] == want
    assert k.min() >= 1 and k.max() > 1          # some baselines are averaged, not all alike
    assert len(set(k.tolist())) > 2


def test_vanishing_shift_bound_is_the_identity():
    uvw, vis, w, nt, nbl, freq = _small()
    r = bda.average(uvw, vis, w, nt, nbl, freq, 256, 4.85e-6, 1e-12)
    assert np.all(r.window == 1) and r.uvw.shape[0] == nt * nbl
    # baseline-major order of the time-major input
    perm = np.array([t * nbl + b for b in range(nbl) for t in range(nt)])
    assert np.array_equal(r.uvw, uvw[perm])
    assert np.max(np.abs(r.vis - vis[perm]) / np.abs(vis[perm])) < 4e-16   # (w v) / w
    assert np.array_equal(r.weight, w[perm])


def test_constant_field_averages_exactly_and_weights_are_conserved():
    uvw, vis, w, nt, nbl, freq = _small()
    const = np.full_like(vis, 0.75 - 0.25j)           # a point source at the phase centre
    r = bda.average(uvw, const, w, nt, nbl, freq, 256, 4.85e-6, 3.0)
    assert r.uvw.shape[0] < nt * nbl
    assert np.max(np.abs(r.vis - (0.75 - 0.25j))) < 1e-15
    wb = w.reshape(nt, nbl, 3).sum(axis=0)             # per baseline and channel
    for b in range(nbl):
        rows = slice(r.offsets[b], r.offsets[b + 1])
        assert np.allclose(r.weight[rows].sum(axis=0), wb[b], rtol=1e-14, atol=0)


def test_point_source_on_linear_tracks_decorrelates_by_the_dirichlet_kernel():
    """u, v linear in time within each window: the mean of S exp(-i(phi0 + t
    delta)) over k samples is the visibility at the mean (u, v) times
    sin(k delta / 2) / (k sin(delta / 2))."""
    nt, nbl = 30, 3
    a = np.array([40.0, 90.0, 170.0])          # metres per step (u)
    c = np.array([-25.0, 10.0, 60.0])          # metres per step (v)
    t = np.arange(nt)[:, None]
    uvw = np.zeros((nt, nbl, 3))
    uvw[:, :, 0] = 500.0 + t * a
    uvw[:, :, 1] = -300.0 + t * c
    uvw = uvw.reshape(-1, 3)
    freq = np.array([1.4e9])
    lam = freq[0] / bda.C_LIGHT
    l, m = 3e-4, -2e-4
    vis = np.exp(-2j * np.pi * (uvw[:, 0] * lam * l + uvw[:, 1] * lam * m))[:, None]
    n, cell, shift = 1024, 4.85e-6, 2.5
    r = bda.average(uvw, vis, None, nt, nbl, freq, n, cell, shift)
    for b in range(nbl):
        k = int(r.window[b])
        step = math.hypot(a[b] * lam, c[b] * lam) * n * cell
        assert k == max(1, math.floor(shift / step))
        delta = 2 * np.pi * (a[b] * lam * l + c[b] * lam * m)
        for g in range(int(r.counts[b])):
            row = int(r.offsets[b]) + g
            kk = min(nt, (g + 1) * k) - g * k
            ub, vb = r.uvw[row, 0] * lam, r.uvw[row, 1] * lam
            at_mean = np.exp(-2j * np.pi * (ub * l + vb * m))
            dirichlet = 1.0 if kk == 1 else math.sin(kk * delta / 2) / (kk * math.sin(delta / 2))
            assert abs(r.vis[row, 0] - at_mean * dirichlet) < 1e-12
            assert r.weight[row, 0] == kk


def test_averaging_flattens_the_partition_imbalance():
    """A fixed ring radius that leaves 80 % of the medium recipe's samples on
    the inner partition leaves far fewer there once the slowly moving short
    baselines are averaged (the dense uv centre is what unbalances Sgr B2's
    partitions)."""
    obs = synth.medium(seed=2, n_times=120, n=512, n_ant=32, n_chan=2, with_vis=False)
    nbl = 32 * 31 // 2
    g = gridder.geometry(obs.uvw, obs.freq, obs.n, obs.cell_rad, nw=0)
    r = partition.radius_px(g)
    ell = float(np.quantile(r, 0.8))
    inner_before = float(np.mean(r <= ell))
    av = bda.average(obs.uvw, obs.vis, obs.weight, 120, nbl, obs.freq, obs.n, obs.cell_rad, 1.0)
    g2 = gridder.geometry(av.uvw, obs.freq, obs.n, obs.cell_rad, nw=0)
    r2 = partition.radius_px(g2)
    inner_after = float(np.mean(r2 <= ell))
    assert inner_before == pytest.approx(0.8, abs=0.01)
    assert inner_after < 0.6
    assert av.uvw.shape[0] < 0.5 * obs.nrow
