"""Continuous-batching serving: a job gives the same image alone and in a mix
of concurrent jobs, and admission waits for the memory budget."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _reqs(obs_small, obs_wstack, base_id=0, arrivals=(0.0, 0.0, 0.0, 0.0)):
    """Request 0: FP64 ms-CLEAN; 1: FP32 FISTA; 2, 3: FP32 jobs that share the device.
    Greedy CLEAN can flip a near-tie under the last-bit differences of the
    gridder's cross-tile float atomics, so its alone/mix identity is checked
    in FP64; FISTA is continuous in its inputs and is checked in FP32."""
    from paper_2507_22128_gb300 import pipeline, rix, serve
    ms = pipeline.Method("msclean", (0.0, 3.0, 9.0), 0.1, 200, 1e-4)
    fi = pipeline.Method("fista", lam_rel=1e-3, iters=10, levels=3)
    kinds = [(obs_small, ms, 3, rix.FP64), (obs_wstack, fi, 2, rix.FP32), (obs_small, ms, 2, rix.FP32),
             (obs_wstack, fi, 3, rix.FP32)]
    return [serve.Request(base_id + i, o, m, nm, arrival=a, precision=pr)
            for i, ((o, m, nm, pr), a) in enumerate(zip(kinds, arrivals))]


def test_same_result_alone_and_in_the_mix(obs_small, obs_wstack):
    need_gpu()
    from paper_2507_22128_gb300 import rix, serve
    ctx = rix.create(0)
    try:
        alone = [serve.serve(ctx, [r], n_slots=1)[0].image for r in _reqs(obs_small, obs_wstack)[:2]]
        mix = serve.serve(ctx, _reqs(obs_small, obs_wstack, 10, arrivals=(0.0, 0.001, 0.002, 0.003)), n_slots=4)
        assert all(np.isfinite(q.image).all() for q in mix)
        # request 0 (ms-CLEAN) and 1 (FISTA) are the same jobs as the ones run alone
        assert rel_l2(mix[0].image, alone[0]) < 1e-9
        assert rel_l2(mix[1].image, alone[1]) < 1e-5
        # the jobs overlapped on the device: later arrivals were admitted before earlier ones finished
        assert mix[1].t_admit < mix[0].t_done
        s = serve.summary(mix)
        assert s["p99_latency_s"] >= s["p50_latency_s"] > 0
    finally:
        rix.destroy(ctx)


def test_admission_waits_for_memory_budget(obs_wstack):
    need_gpu()
    from paper_2507_22128_gb300 import pipeline, rix, serve
    o = obs_wstack
    need = rix.job_workspace_bytes(o.n, o.cell_rad, o.n_wplanes, list(o.freq), rix.FP32, 2, o.nrow)
    ctx = rix.create(0, int(need * 1.5))          # room for one job at a time
    try:
        fi = pipeline.Method("fista", lam_rel=1e-3, iters=5, levels=2)
        reqs = [serve.Request(i, o, fi, 1, arrival=0.0) for i in range(3)]
        serve.serve(ctx, reqs, n_slots=3)
        done = sorted(reqs, key=lambda q: q.t_admit)
        for a, b in zip(done, done[1:]):
            assert b.t_admit >= a.t_done - 1e-6      # admitted only after the previous job released its memory
        assert all(np.isfinite(q.image).all() for q in reqs)
    finally:
        rix.destroy(ctx)
