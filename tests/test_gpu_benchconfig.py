"""GPU parity in the configuration the benchmark times, at reduced row count.

The benchmark's step runs the medium recipe: 1024 x 1024 at 1", 16 w-planes,
4 channels over 1.3-1.5 GHz, 2 uv partitions, FISTA with the Db4 basis, 4
levels, 50 iterations, lambda = 1e-3 max |residual of cycle 1|, the two
partitions' minor cycles batched into one loop launch, each partition's
major cycle on its own stream.  Here the same recipe runs with 20 time
samples instead of 1000 (161,280 visibilities): the kernels are the same
template instances (the 2048-point transforms of the FISTA loop, the fused
degrid/residual/grid kernel and the PSF kernel at 1024^2 with 16 planes),
only the number of samples is smaller, so the oracle's cycles stay cheap.

Checked against the oracle's decentralized loop for two major cycles:
  the PSFs of both partitions (2048 x 2048) within 1e-5 (FP32) / 1e-10 (FP64);
  the cycle-1 residual images within 1e-5 / 1e-10;
  both partitions' models after each cycle and the combined image within
  1e-4 (FP32) / 1e-9 (FP64).
"""
import numpy as np
import pytest

from gpu_util import need_gpu, real_dtype, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_CYCLES = 2
TOL_OP = {0: 1e-5, 1: 1e-10}
TOL_IMG = {0: 1e-4, 1: 1e-9}


@pytest.fixture(scope="module")
def bench_case():
    """The oracle's two cycles of the benchmark recipe (run once for both
    precisions)."""
    need_gpu()
    from oracle import framework
    from paper_2507_22128_gb300 import synth
    obs = synth.medium(seed=1, n_times=20)
    st = framework.setup(obs.uvw, obs.freq, obs.weight, obs.n, obs.cell_rad, obs.n_wplanes, 2)
    loop = framework.Loop(st, obs.vis, obs.weight)
    models, residual1 = [], None
    for c in range(1, N_CYCLES + 1):
        for p in range(2):
            loop.major(p)
        if c == 1:
            residual1 = [r.copy() for r in loop.residual]
        for p in range(2):
            loop.minor_fista(p, c, lam_rel=1e-3, n_iter=50, levels=4)
        loop.exchange()
        models.append([m.copy() for m in loop.model])
    return obs, st, residual1, models, loop.combine()


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    from paper_2507_22128_gb300 import rix
    c = rix.create(0)
    yield c
    rix.destroy(c)


@pytest.mark.parametrize("prec", [0, 1])
def test_fista_job_in_the_benchmark_configuration(ctx, bench_case, prec):
    from paper_2507_22128_gb300 import pipeline, rix
    obs, st, residual1, models, combined = bench_case
    n = obs.n
    rdt = real_dtype(prec)
    rec = pipeline.observation_job(ctx, obs, 2, prec)
    m = pipeline.Method("fista", lam_rel=1e-3, iters=50, levels=4)
    stream = torch.cuda.current_stream()
    try:
        st_gpu = rec.stats()
        assert st_gpu["n_outside"] == 0
        for p in range(2):
            psf = torch.empty((2 * n, 2 * n), dtype=rdt, device="cuda")
            rix.psf(rec.job, p, psf)
            torch.cuda.synchronize()
            assert rel_l2(psf.cpu().numpy(), st.psf[p]) < TOL_OP[prec]
        for c in range(1, N_CYCLES + 1):
            if c == 1:
                # cycle 1 with the residual images read back, then the batched
                # minor cycles (one loop launch for both partitions)
                res = [torch.empty((n, n), dtype=rdt, device="cuda") for _ in range(2)]
                for p in range(2):
                    rec.major(p, residual_out=res[p], stream=stream)
                rec.minor_all(m, stream)
                torch.cuda.synchronize()
                for p in range(2):
                    assert rel_l2(res[p].cpu().numpy(), residual1[p]) < TOL_OP[prec]
            else:
                # the benchmark's schedule: partitions on their own streams,
                # batched minor cycles
                rec.cycles(m, 1, stream)
            for p in range(2):
                out = torch.empty((n, n), dtype=rdt, device="cuda")
                rix.get_model(rec.job, p, out, stream)
                torch.cuda.synchronize()
                want = models[c - 1][p]
                assert np.abs(want).max() > 0.0
                assert rel_l2(out.cpu().numpy(), want) < TOL_IMG[prec]
        img = rec.combine(stream=stream)
        torch.cuda.synchronize()
        assert rel_l2(img.cpu().numpy(), combined) < TOL_IMG[prec]
    finally:
        rec.close()
