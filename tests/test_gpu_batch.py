"""GPU parity of the batched major cycle (rix_batch_*): several FP32
w-stacked jobs of different image sizes, every partition's degrid, residual
and grid in one gridder launch, against the oracle's major cycle (1e-5
relative L2, the FP32 operator bound), through a full loop with the minor
cycles (1e-4), replayed from a captured CUDA graph (equal to the uncaptured
call), and with the autotuner's choice applied and cached."""
import json

import numpy as np
import pytest

from gpu_util import need_gpu, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    from paper_2507_22128_gb300 import rix
    c = rix.create(0)
    yield c
    rix.destroy(c)


@pytest.fixture(scope="module")
def jobs_obs():
    from paper_2507_22128_gb300 import synth
    return [synth.medium(seed=21, n_times=30, n=256, n_ant=24, n_chan=2),
            synth.medium(seed=22, n_times=20, n=128, n_ant=20, n_chan=2),
            synth.medium(seed=23, n_times=40, n=256, n_ant=28, n_chan=1)]


def _recs(ctx, obs_list):
    from paper_2507_22128_gb300 import pipeline
    return [pipeline.observation_job(ctx, o, 2, 0) for o in obs_list]


def test_batched_major_cycles_match_oracle_and_a_full_loop(ctx, jobs_obs):
    from oracle import framework
    from paper_2507_22128_gb300 import pipeline, rix
    recs = _recs(ctx, jobs_obs)
    loops = [framework.Loop(framework.setup(o.uvw, o.freq, o.weight, o.n, o.cell_rad, o.n_wplanes, 2), o.vis, o.weight)
             for o in jobs_obs]
    bm = pipeline.BatchedMajor(ctx, recs)
    m = pipeline.Method("fista", lam_rel=1e-3, iters=10, levels=2)
    try:
        for c in range(1, 3):
            res = [torch.empty((r.n, r.n), dtype=torch.float32, device="cuda") for r, _ in bm.pairs]
            bm.run(residual_out=res)
            for r in recs:
                r.minor_all(m, torch.cuda.current_stream())
            torch.cuda.synchronize()
            for i, (r, p) in enumerate(bm.pairs):
                j = recs.index(r)
                want = loops[j].major(p)
                assert rel_l2(res[i].cpu().numpy(), want) < 1e-5
                assert r.stats()["cycle"][p] == c
            for j, o in enumerate(jobs_obs):
                for p in range(2):
                    loops[j].minor_fista(p, c, lam_rel=1e-3, n_iter=10, levels=2)
                loops[j].exchange()
        for j, r in enumerate(recs):
            img = r.combine().cpu().numpy()
            assert rel_l2(img, loops[j].combine()) < 1e-4
    finally:
        bm.close()
        for r in recs:
            r.close()


def test_captured_graph_replays_the_batched_cycle(ctx, jobs_obs):
    """Cycle 1 issued directly (it allocates the buffers), the minor cycles,
    then cycle 2 captured into a CUDA graph and replayed twice: both replays
    give the oracle's cycle-2 residuals."""
    from oracle import framework
    from paper_2507_22128_gb300 import pipeline
    recs = _recs(ctx, jobs_obs)
    loops = [framework.Loop(framework.setup(o.uvw, o.freq, o.weight, o.n, o.cell_rad, o.n_wplanes, 2), o.vis, o.weight)
             for o in jobs_obs]
    bm = pipeline.BatchedMajor(ctx, recs)
    m = pipeline.Method("fista", lam_rel=1e-3, iters=5, levels=2)
    s = torch.cuda.Stream()
    try:
        with torch.cuda.stream(s):
            bm.run(s)
            for r in recs:
                r.minor_all(m, s)
        torch.cuda.synchronize()
        for lp in loops:
            for p in range(2):
                lp.major(p)
            for p in range(2):
                lp.minor_fista(p, 1, lam_rel=1e-3, n_iter=5, levels=2)
            lp.exchange()
        got = [torch.full((r.n, r.n), np.nan, dtype=torch.float32, device="cuda") for r, _ in bm.pairs]
        bm.capture(s, residual_out=got)
        outs = []
        for _ in range(2):
            bm.replay()
            torch.cuda.synchronize()
            outs.append([g.cpu().numpy() for g in got])
        for i, (r, p) in enumerate(bm.pairs):
            want = loops[recs.index(r)].major(p)
            for o in outs:
                assert rel_l2(o[i], want) < 1e-5
            assert rel_l2(outs[1][i], outs[0][i]) < 1e-6
    finally:
        bm.close()
        for r in recs:
            r.close()


def test_autotuner_chooses_and_caches(ctx, jobs_obs, tmp_path):
    from paper_2507_22128_gb300 import autotune, pipeline
    rec = pipeline.observation_job(ctx, jobs_obs[0], 2, 0)
    path = str(tmp_path / "tune.json")
    try:
        vis = rec.vis.reshape(-1)
        first = autotune.tune(rec, vis, path)
        assert not first["cached"]
        assert (first["chunk_limit"], first["ctas_per_sm"]) in autotune.CANDIDATES
        assert len(first["timings"]) == len(autotune.CANDIDATES) and all(t["ms"] > 0 for t in first["timings"])
        table = json.load(open(path))
        assert first["key"] in table
        again = autotune.tune(rec, vis, path)
        assert again["cached"] and again["chunk_limit"] == first["chunk_limit"]
        # the tuned job still matches its own untuned result (same arithmetic, regrouped)
        a = torch.empty((rec.n, rec.n), dtype=torch.float32, device="cuda")
        rec.major(0, residual_out=a)
        torch.cuda.synchronize()
        from oracle import framework
        o = jobs_obs[0]
        loop = framework.Loop(framework.setup(o.uvw, o.freq, o.weight, o.n, o.cell_rad, o.n_wplanes, 2), o.vis,
                              o.weight)
        assert rel_l2(a.cpu().numpy(), loop.major(0)) < 1e-5
    finally:
        rec.close()
