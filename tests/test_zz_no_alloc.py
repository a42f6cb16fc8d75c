"""rix_grid_noalloc: gridding without device allocation at call time.

Callers that cannot allocate device memory while they grid (a latency-bound
host loop that must not stall on cudaMalloc's device synchronisation, or a
process whose GPU memory another allocator already holds) use this entry
point; it keeps its scratch in a fixed device array inside the library.
Checked here against rix_grid on the same job, two calls in a row, with the
library's own allocation counter unchanged across the calls.  The w-stacked
case (256^2, 16 w-planes) is one where the inverse transform splits its
planes into groups, whose images also come from the fixed scratch.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_l2, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["small", "wstack"])
def test_grid_noalloc_matches_grid_twice(obs_small, obs_wstack, which):
    need_gpu()
    from paper_2507_22128_gb300 import rix
    obs = obs_small if which == "small" else obs_wstack
    ctx = rix.create(0)
    job = rix.job_create(ctx, obs.n, obs.cell_rad, obs.n_wplanes, list(obs.freq), rix.FP32, 2, obs.nrow)
    try:
        rix.set_uv_partition(job, to_dev(obs.uvw, torch.float64), to_dev(obs.weight, torch.float32))
        vis = to_dev(obs.vis.reshape(-1), torch.complex64)
        for p in range(2):
            ref = torch.empty((obs.n, obs.n), dtype=torch.float32, device="cuda")
            rix.grid(job, p, vis, ref)
            outs = [torch.full((obs.n, obs.n), np.nan, dtype=torch.float32, device="cuda") for _ in range(2)]
            torch.cuda.synchronize()
            allocs = rix.device_allocations()
            for out in outs:                      # the shared scratch is re-zeroed by each call
                rix.grid_noalloc(job, p, vis, out)
            assert rix.device_allocations() == allocs
            torch.cuda.synchronize()
            for out in outs:
                assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) < 1e-5
    finally:
        rix.job_destroy(job)
        rix.destroy(ctx)


def test_grid_noalloc_then_destroy_without_sync(obs_wstack):
    """The call records its stream with the job, so destroying the job right
    after it (no synchronisation in between) waits for the gridding before
    the job's buffers are released: the output is complete and correct."""
    need_gpu()
    from paper_2507_22128_gb300 import rix
    obs = obs_wstack
    ctx = rix.create(0)
    job = rix.job_create(ctx, obs.n, obs.cell_rad, obs.n_wplanes, list(obs.freq), rix.FP32, 2, obs.nrow)
    side = torch.cuda.Stream()
    try:
        rix.set_uv_partition(job, to_dev(obs.uvw, torch.float64), to_dev(obs.weight, torch.float32))
        vis = to_dev(obs.vis.reshape(-1), torch.complex64)
        ref = torch.empty((obs.n, obs.n), dtype=torch.float32, device="cuda")
        rix.grid(job, 1, vis, ref)
        torch.cuda.synchronize()
        out = torch.full((obs.n, obs.n), np.nan, dtype=torch.float32, device="cuda")
        rix.grid_noalloc(job, 1, vis, out, side)
        rix.job_destroy(job)
        job = None
        side.synchronize()
        assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) < 1e-5
    finally:
        if job is not None:
            rix.job_destroy(job)
        rix.destroy(ctx)


def test_grid_noalloc_rejects_oversized_partition():
    need_gpu()
    from paper_2507_22128_gb300 import rix, synth
    # 1024^2 with 16 w-planes: the high partition's window needs more than the fixed scratch
    obs = synth.medium(seed=5, n_times=20, n=1024, n_wplanes=16, n_ant=64, n_chan=1)
    ctx = rix.create(0)
    job = rix.job_create(ctx, obs.n, obs.cell_rad, obs.n_wplanes, list(obs.freq), rix.FP32, 2, obs.nrow)
    try:
        rix.set_uv_partition(job, to_dev(obs.uvw, torch.float64), None)
        st = rix.job_get_stats(job)
        s = st["window_size"][1]
        need = 16 * s * (s + obs.n) * 8
        assert need > (32 << 20)
        out = torch.empty((obs.n, obs.n), dtype=torch.float32, device="cuda")
        allocs = rix.device_allocations()
        with pytest.raises(rix.RixError) as e:
            rix.grid_noalloc(job, 1, to_dev(obs.vis.reshape(-1), torch.complex64), out)
        assert e.value.code == rix.EINVAL
        assert rix.device_allocations() == allocs
    finally:
        rix.job_destroy(job)
        rix.destroy(ctx)
