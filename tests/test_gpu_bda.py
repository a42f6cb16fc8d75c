"""GPU parity of baseline-dependent averaging (Sec. 6.2, Sec. 7 item d) against
the oracle, through the C ABI: windows and row counts bit-exact (they are
integers decided by FP64 arithmetic taken in the same order on both sides),
averaged uvw and visibilities within the rounding of the summation order
(FP64 1e-12, FP32 visibilities 1e-6 relative), weights exact for unit
weights and within FP32 rounding otherwise; then the averaged data
partitioned by the library with a fixed ring radius split more evenly."""
import math

import numpy as np
import pytest

from gpu_util import need_gpu, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    from paper_2507_22128_gb300 import rix
    c = rix.create(0)
    yield c
    rix.destroy(c)


def _obs():
    from paper_2507_22128_gb300 import synth
    obs = synth.medium(seed=2, n_times=120, n=512, n_ant=32, n_chan=2)
    rng = np.random.default_rng(5)
    w = rng.uniform(0.5, 2.0, obs.weight.shape).astype(np.float32)
    return obs, 32 * 31 // 2, w


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("shift", [1e-9, 0.5, 3.0])
def test_averaging_matches_oracle(ctx, prec, shift):
    from oracle import bda
    from paper_2507_22128_gb300 import rix
    obs, nbl, w = _obs()
    nt = 120
    want = bda.average(obs.uvw, obs.vis, w, nt, nbl, obs.freq, obs.n, obs.cell_rad, shift)
    uvw = to_dev(obs.uvw, torch.float64)
    cdt = torch.complex128 if prec == 1 else torch.complex64
    nrow, win = rix.bda_rows(ctx, uvw, nt, nbl, list(obs.freq), obs.n, obs.cell_rad, shift)
    assert np.array_equal(win.astype(np.int64), want.window)
    assert nrow == want.uvw.shape[0]
    u, v, wo = rix.bda_average(ctx, uvw, to_dev(obs.vis.reshape(-1), cdt), to_dev(w.reshape(-1), torch.float32),
                               nt, nbl, list(obs.freq), obs.n, obs.cell_rad, shift)
    torch.cuda.synchronize()
    assert np.max(np.abs(u.cpu().numpy() - want.uvw)) <= 1e-12 * np.max(np.abs(want.uvw))
    gv = v.cpu().numpy().astype(np.complex128)
    rel = np.abs(gv - want.vis) / np.maximum(np.abs(want.vis), 1e-300)
    assert np.max(rel) < (1e-12 if prec == 1 else 1e-6)
    assert np.max(np.abs(wo.cpu().numpy() - want.weight) / want.weight) < 1e-6


def test_unit_weights_and_a_constant_field(ctx):
    from oracle import bda
    from paper_2507_22128_gb300 import rix
    obs, nbl, _ = _obs()
    nt = 120
    const = np.full(obs.vis.shape, 0.5 + 0.25j)
    u, v, wo = rix.bda_average(ctx, to_dev(obs.uvw, torch.float64), to_dev(const.reshape(-1), torch.complex128),
                               None, nt, nbl, list(obs.freq), obs.n, obs.cell_rad, 2.0)
    torch.cuda.synchronize()
    want = bda.average(obs.uvw, const, None, nt, nbl, obs.freq, obs.n, obs.cell_rad, 2.0)
    assert np.array_equal(wo.cpu().numpy().astype(np.float64), want.weight)      # window lengths
    assert np.max(np.abs(v.cpu().numpy() - (0.5 + 0.25j))) < 1e-15
    assert wo.cpu().numpy().sum() == obs.nvis                                   # every sample counted once


def test_averaged_data_split_more_evenly(ctx):
    """A ring radius leaving 80 % of the samples on the inner partition leaves
    far fewer there after averaging (the library's partition of the averaged
    rows against the oracle's count on its own averaged rows)."""
    from oracle import bda, gridder, partition
    from paper_2507_22128_gb300 import rix
    obs, nbl, w = _obs()
    nt = 120
    g = gridder.geometry(obs.uvw, obs.freq, obs.n, obs.cell_rad, nw=0)
    ell = float(np.quantile(partition.radius_px(g), 0.8))
    u, v, wo = rix.bda_average(ctx, to_dev(obs.uvw, torch.float64), to_dev(obs.vis.reshape(-1), torch.complex64),
                               to_dev(w.reshape(-1), torch.float32), nt, nbl, list(obs.freq), obs.n, obs.cell_rad, 1.0)
    nrow = u.shape[0]
    job = rix.job_create(ctx, obs.n, obs.cell_rad, 0, list(obs.freq), rix.FP32, 2, nrow)
    try:
        rix.set_uv_partition(job, u, wo.reshape(-1), [ell], 1.0)
        st = rix.job_get_stats(job)
        frac_gpu = st["part_count"][0] / (nrow * obs.nchan)
    finally:
        rix.job_destroy(job)
    want = bda.average(obs.uvw, obs.vis, w, nt, nbl, obs.freq, obs.n, obs.cell_rad, 1.0)
    g2 = gridder.geometry(want.uvw, obs.freq, obs.n, obs.cell_rad, nw=0)
    m2 = partition.masks(partition.radius_px(g2), np.array([ell]), 1.0, 2, g2.inside)
    frac_oracle = float(np.mean((m2 & 1) == 1))
    assert frac_gpu < 0.65
    assert abs(frac_gpu - frac_oracle) < 1e-3
