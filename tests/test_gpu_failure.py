"""Failure detection without a GPU fault: a bounded device-side wait that runs
out reports RIX_ETIMEOUT and leaves the context usable; runs that should be
deterministic are bitwise repeatable."""
import time

import numpy as np
import pytest

from gpu_util import need_gpu, sparse_model, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_barrier_wait_runs_out_and_reports_timeout(obs_small):
    need_gpu()
    from paper_2507_22128_gb300 import rix
    ctx = rix.create(0)
    try:
        t0 = time.perf_counter()
        status, gave_up = rix.selftest_barrier_timeout(ctx)
        dt = time.perf_counter() - t0
        assert status == rix.ETIMEOUT
        assert gave_up == torch.cuda.get_device_properties(0).multi_processor_count - 1
        assert 1.5 < dt < 30.0
        # the context still works: a degrid after the timeout
        o = obs_small
        job = rix.job_create(ctx, o.n, o.cell_rad, o.n_wplanes, list(o.freq), rix.FP64, 1, o.nrow, 0)
        try:
            rix.set_uv_partition(job, to_dev(o.uvw, torch.float64), None, None, 1.0, None)
            vis = torch.zeros(o.nvis, dtype=torch.complex128, device="cuda")
            rix.degrid(job, 0, to_dev(sparse_model(o.n, 5, 3), torch.float64), vis)
            rix.job_sync(job)
            assert torch.isfinite(torch.view_as_real(vis)).all()
        finally:
            rix.job_destroy(job)
    finally:
        rix.destroy(ctx)


def test_partition_and_degrid_are_bitwise_repeatable(obs_wstack):
    """The sort, the masks and the degrid (no atomics) repeat bit for bit;
    gridding accumulates across work items with float atomics and is only
    repeatable to rounding."""
    need_gpu()
    from paper_2507_22128_gb300 import rix
    o = obs_wstack
    ctx = rix.create(0)
    try:
        outs = []
        for _ in range(2):
            job = rix.job_create(ctx, o.n, o.cell_rad, o.n_wplanes, list(o.freq), rix.FP32, 2, o.nrow, 0)
            try:
                mask = torch.zeros(o.nvis, dtype=torch.uint8, device="cuda")
                rix.set_uv_partition(job, to_dev(o.uvw, torch.float64), to_dev(o.weight, torch.float32), None, 1.0,
                                     mask)
                n = rix.job_get_stats(job)["n_entries"]
                keys = torch.empty(n, dtype=torch.int32, device="cuda")
                samples = torch.empty(n, dtype=torch.int32, device="cuda")
                rix.get_sorted_entries(job, keys, samples)
                vis = torch.zeros(o.nvis, dtype=torch.complex64, device="cuda")
                rix.degrid(job, 1, to_dev(sparse_model(o.n, 20, 4), torch.float32), vis)
                torch.cuda.synchronize()
                outs.append([t.cpu().numpy() for t in (mask, keys, samples, torch.view_as_real(vis))])
            finally:
                rix.job_destroy(job)
        for a, b in zip(*outs):
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
    finally:
        rix.destroy(ctx)
