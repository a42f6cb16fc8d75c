"""GPU parity of uniform weighting (Sec. 5.1): the weights the job images
with, bit for bit against the oracle, and a decentralized FISTA run imaged
with them."""
import numpy as np
import pytest

from gpu_util import need_gpu, real_dtype, rel_l2, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    from paper_2507_22128_gb300 import rix
    c = rix.create(0)
    yield c
    rix.destroy(c)


@pytest.mark.parametrize("natural", ["ones", "random"])
def test_uniform_weights_match_oracle(ctx, obs_wstack, natural):
    from oracle import gridder, weighting
    from paper_2507_22128_gb300 import rix
    o = obs_wstack
    w0 = o.weight if natural == "ones" else \
        np.random.default_rng(3).uniform(0.5, 2.0, o.weight.shape).astype(np.float32)
    job = rix.job_create(ctx, o.n, o.cell_rad, o.n_wplanes, list(o.freq), rix.FP32, 2, o.nrow, 0,
                         rix.WEIGHT_UNIFORM)
    try:
        rix.set_uv_partition(job, to_dev(o.uvw, torch.float64), to_dev(w0, torch.float32), None, 1.0, None)
        got = torch.empty(o.nvis, dtype=torch.float32, device="cuda")
        rix.get_weights(job, got)
        torch.cuda.synchronize()
        got = got.cpu().numpy()
        g = gridder.geometry(o.uvw, o.freq, o.n, o.cell_rad, nw=o.n_wplanes)
        want = weighting.uniform_weights(g, w0)
        if natural == "ones":
            # integer densities: exact in any summation order
            assert np.array_equal(got, want)
        else:
            # densities summed in a different order: at most one float32 ulp apart
            ulp = np.abs(got.view(np.int32).astype(np.int64) - want.view(np.int32).astype(np.int64))
            assert ulp.max() <= 1
        assert not np.array_equal(got, w0)
    finally:
        rix.job_destroy(job)


def test_fista_loop_with_uniform_weighting(ctx, obs_wstack):
    from oracle import framework
    from paper_2507_22128_gb300 import pipeline, rix
    o = obs_wstack
    st = framework.setup(o.uvw, o.freq, o.weight, o.n, o.cell_rad, o.n_wplanes, 2, scheme="uniform")
    loop = framework.Loop(st, o.vis)
    rec = pipeline.observation_job(ctx, o, 2, rix.FP64, weighting=rix.WEIGHT_UNIFORM)
    m = pipeline.Method("fista", lam_rel=1e-3, iters=10, levels=3)
    try:
        s = rix.job_get_stats(rec.job)
        assert np.allclose(s["part_weight"][:2], st.wsum, rtol=1e-12)
        for c in range(1, 3):
            for p in range(2):
                loop.major(p)
                rec.major(p)
            for p in range(2):
                loop.minor_fista(p, c, lam_rel=1e-3, n_iter=10, levels=3)
                rec.minor(p, m)
            loop.exchange()
        assert rel_l2(rec.combine().cpu().numpy(), loop.combine()) < 1e-9
    finally:
        rec.close()
