"""Host-side helpers of bench.py that decide what a run reports: the clock
summary (a run whose samples show a thermal or hardware slowdown must say
so), the gridder's traffic figure (only for the workload and source it was
measured on) and the roofline arithmetic.  CPU only."""
import hashlib
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    pytest.importorskip("torch")
    import bench as b
    return b


def _line(sm, mx, reasons=()):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    return ", ".join(["0", str(sm), str(mx), "900.5", "0x0"] + flags)


def test_clock_summary_median_max_and_reasons(bench):
    cs = bench.ClockSampler(0)
    cs.lines = [_line(2070, 2070), _line(1900, 2070, ("sw_power_cap",)), _line(2070, 2070),
                "garbage line", _line(2000, 2070, ("hw_thermal_slowdown",))]
    s = cs.summary()
    assert s["samples"] == 4
    assert s["sm_mhz"] == 2035.0            # median of 2070, 1900, 2070, 2000
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_unsampled(bench):
    cs = bench.ClockSampler(0)
    cs.lines = []
    assert cs.summary()["reasons"] == ["unsampled"]


def _args(**kw):
    a = dict(fp64=False, n=1024, n_times=1000, cycles=10, steps=5)
    a.update(kw)
    return types.SimpleNamespace(**a)


def test_tiles_traffic_only_for_the_measured_source_and_workload(bench):
    shas = []
    for name in ("k_tiles_fp.cu", "rix_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2507_22128_gb300", "csrc", name), "rb") as f:
            shas.append(hashlib.sha1(f.read()).hexdigest())
    t = bench.TILES_TRAFFIC
    got = bench.tiles_traffic(_args())
    if tuple(shas) != t["src_sha1"]:
        assert got is None
    else:
        # the mean over the two partitions' launches
        assert got == pytest.approx(sum(t["resid"]) / 2)
    assert bench.tiles_traffic(_args(fp64=True)) is None
    assert bench.tiles_traffic(_args(n=512)) is None
    assert bench.tiles_traffic(_args(n_times=300)) is None


def test_roofline_arithmetic(bench, monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: ({"sm_max_mhz": 2000.0, "hbm_gbs": 5000.0}, "measured"))
    st = {"window_size": [100, 200], "part_count": [600_000, 400_000]}
    a = _args()
    mc = {"per_partition_serial": {0: {"gridder_ms": 1.5}, 1: {"gridder_ms": 2.5}}}
    r = bench.roofline_gridder(mc, st, a)
    peak = 152 * 128 * 2 * 2000e6 / 1e12
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(4096.0 * 1e6 / 4e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    byt = 32.0 * 1e6 + 2 * 8.0 * 16 * (100 ** 2 + 200 ** 2)
    assert r["hbm"]["algorithmic_bytes_per_launch"] == pytest.approx(byt / 2)
    assert r["hbm"]["frac"] == pytest.approx(byt / 4e-3 / 1e9 / 5000.0)
    assert r["ms_per_launch"] == {"low": 1.5, "high": 2.5}
    mc0 = {"per_partition_serial": {0: {"gridder_ms": 0.0}, 1: {"gridder_ms": 0.0}}}
    assert bench.roofline_gridder(mc0, st, a) is None


def test_whole_job_value_is_the_aggregate_over_ranks(bench):
    # every rank processes the same units per step: the whole job's rate
    # scales with the ranks over the slowest rank's time
    assert bench.whole_job_value(82_466_880, 1, 140.0) == pytest.approx(82_466_880 / 0.140 / 1e6)
    assert bench.whole_job_value(1e6, 4, 10.0) == pytest.approx(4 * 1e6 / 0.010 / 1e6)


def test_serving_requests_follow_the_mix(bench):
    """The serving workload's requests: kinds drawn by the pools' shares
    (50/30/15/5 %), ms-CLEAN or FISTA with probability 1/2, each kind's cycle
    count and scale set, arrival times kept; the FP64 comparison subset
    leaves out the large recipe and keeps the order of the stream."""
    import numpy as np
    if not os.path.exists(os.path.join(ROOT, "paper_2507_22128_gb300", "librix.so")):
        from paper_2507_22128_gb300 import build
        build.build()
    from paper_2507_22128_gb300 import rix, serve
    obs = [types.SimpleNamespace(name=f"o{i}") for i in range(5)]
    pools = {"small": (0.50, obs[:2], 5, (0.0, 3.0, 9.0), 3), "medium": (0.30, obs[2:3], 10, (0.0, 4.0, 16.0), 4),
             "chunk": (0.15, obs[3:4], 5, (0.0, 4.0, 16.0), 4), "large": (0.05, obs[4:], 8, (0.0, 4.0, 16.0, 32.0), 4)}
    arr = serve.poisson_arrivals(np.random.default_rng(4), 4000, 20.0)
    reqs = bench.serve_requests(pools, arr, np.random.default_rng(40), rix.FP32)
    assert len(reqs) == 4000 and [q.arrival for q in reqs] == list(arr)
    for kind, (share, olist, n_major, scales, levels) in pools.items():
        mine = [q for q in reqs if q.kind.startswith(kind + " ")]
        assert abs(len(mine) / 4000 - share) < 0.02
        assert all(q.n_major == n_major and q.obs in olist for q in mine)
        assert all(tuple(q.method.scales) == scales for q in mine if q.method.kind == "msclean")
        assert all(q.method.levels == levels for q in mine if q.method.kind == "fista")
    assert abs(np.mean([q.method.kind == "msclean" for q in reqs]) - 0.5) < 0.03
    sub = [q for q in bench.serve_requests(pools, arr, np.random.default_rng(40), rix.FP64)
           if not q.kind.startswith("large")][:100]
    assert all(q.precision == rix.FP64 for q in sub)
    assert [q.rid for q in sub] == sorted(q.rid for q in sub)
    same = {q.rid: q.kind for q in reqs}
    assert all(same[q.rid] == q.kind for q in sub)
