"""GPU parity of a1-a7 (partition, sort, degrid, grid, PSF, major cycle)
against the CPU oracle, through the C ABI.

Tolerances: keys, permutation and masks bit-exact; FP32 operator within 1e-5
relative L2 of the FP64 oracle gridder with the same kernel and within 1e-4
of the direct DFT; FP64 operator within 1e-10 of the FP64 oracle gridder.
"""
import numpy as np
import pytest

from gpu_util import cplx_dtype, need_gpu, real_dtype, rel_l2, sparse_model, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-10}      # rix.FP32, rix.FP64


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    from paper_2507_22128_gb300 import rix
    c = rix.create(0)
    yield c
    rix.destroy(c)


def _job(ctx, obs, prec, nparts=2, tile=0):
    from paper_2507_22128_gb300 import rix
    job = rix.job_create(ctx, obs.n, obs.cell_rad, obs.n_wplanes, list(obs.freq), prec, nparts, obs.nrow, tile)
    mask = torch.zeros(obs.nvis, dtype=torch.uint8, device="cuda")
    rix.set_uv_partition(job, to_dev(obs.uvw, torch.float64), to_dev(obs.weight, torch.float32), None, 1.0, mask)
    torch.cuda.synchronize()
    return job, mask.cpu().numpy()


def _oracle(obs, nparts):
    from oracle import framework
    return framework.setup(obs.uvw, obs.freq, obs.weight, obs.n, obs.cell_rad, obs.n_wplanes, nparts)


CASES = [("small", 0, 2), ("small", 1, 2), ("wstack", 0, 2), ("wstack", 1, 2), ("wstack", 0, 4), ("wstack", 1, 8)]


def _obs(name, obs_small, obs_wstack):
    return obs_small if name == "small" else obs_wstack


@pytest.mark.parametrize("name,prec,nparts", CASES)
def test_partition_and_sort_bit_exact(ctx, obs_small, obs_wstack, name, prec, nparts):
    from oracle import partition
    from paper_2507_22128_gb300 import rix
    obs = _obs(name, obs_small, obs_wstack)
    job, mask = _job(ctx, obs, prec, nparts)
    try:
        st = _oracle(obs, nparts)
        assert np.array_equal(mask, st.mask)
        s = rix.job_get_stats(job)
        assert s["n_outside"] == int((~st.geom.inside).sum())
        for i in range(nparts - 1):
            assert s["ell_px"][i] == st.ells[i]
        if obs.n_wplanes:
            assert s["w_min"] == st.geom.w_min and s["dw"] == st.geom.dw
        keys, samples, _ = partition.entries(st.geom, st.mask, 16, nparts)
        sk, ss = partition.sort_entries(keys, samples)
        assert s["n_entries"] == sk.shape[0]
        gk = torch.empty(sk.shape[0], dtype=torch.int32, device="cuda")
        gs = torch.empty(sk.shape[0], dtype=torch.int32, device="cuda")
        rix.get_sorted_entries(job, gk, gs)
        torch.cuda.synchronize()
        assert np.array_equal(gk.cpu().numpy().view(np.uint32), sk)
        assert np.array_equal(gs.cpu().numpy().view(np.uint32), ss)
        for p in range(nparts):
            assert s["part_count"][p] == int(((st.mask >> p) & 1).sum())
            assert s["part_weight"][p] == pytest.approx(st.wsum[p], rel=1e-12)
    finally:
        rix.job_destroy(job)


@pytest.mark.parametrize("name,prec,nparts", CASES)
def test_degrid_matches_oracle_gridder(ctx, obs_small, obs_wstack, name, prec, nparts):
    from oracle import gridder
    from paper_2507_22128_gb300 import rix
    obs = _obs(name, obs_small, obs_wstack)
    job, _ = _job(ctx, obs, prec, nparts)
    try:
        st = _oracle(obs, nparts)
        x = sparse_model(obs.n, 40, seed=3) + 0.01 * np.random.default_rng(4).normal(size=(obs.n, obs.n))
        for p in range(nparts):
            vis = torch.zeros(obs.nvis, dtype=cplx_dtype(prec), device="cuda")
            rix.degrid(job, p, to_dev(x, real_dtype(prec)), vis)
            torch.cuda.synchronize()
            got = vis.cpu().numpy()
            g = st.gparts[p]
            want = gridder.degrid(x, g)
            sel = g.inside
            assert rel_l2(got[sel], want[sel]) < TOL[prec]
            assert np.all(got[~sel] == 0)          # samples outside the partition untouched
    finally:
        rix.job_destroy(job)


@pytest.mark.parametrize("name,prec,nparts", CASES)
def test_grid_matches_oracle_gridder(ctx, obs_small, obs_wstack, name, prec, nparts):
    from oracle import gridder
    from paper_2507_22128_gb300 import rix
    obs = _obs(name, obs_small, obs_wstack)
    job, _ = _job(ctx, obs, prec, nparts)
    try:
        st = _oracle(obs, nparts)
        w = obs.weight.reshape(-1).astype(np.float64)
        for p in range(nparts):
            img = torch.empty((obs.n, obs.n), dtype=real_dtype(prec), device="cuda")
            rix.grid(job, p, to_dev(obs.vis.reshape(-1), cplx_dtype(prec)), img)
            torch.cuda.synchronize()
            want = gridder.dirty(obs.vis.reshape(-1), w, st.gparts[p])
            assert rel_l2(img.cpu().numpy(), want) < TOL[prec]
    finally:
        rix.job_destroy(job)


@pytest.mark.parametrize("name,prec,nparts", CASES[:4])
def test_psf_matches_oracle(ctx, obs_small, obs_wstack, name, prec, nparts):
    from paper_2507_22128_gb300 import rix
    obs = _obs(name, obs_small, obs_wstack)
    job, _ = _job(ctx, obs, prec, nparts)
    try:
        st = _oracle(obs, nparts)
        for p in range(nparts):
            out = torch.empty((2 * obs.n, 2 * obs.n), dtype=real_dtype(prec), device="cuda")
            wsum = rix.psf(job, p, out)
            torch.cuda.synchronize()
            assert wsum == pytest.approx(st.wsum[p], rel=1e-12)
            assert rel_l2(out.cpu().numpy(), st.psf[p]) < TOL[prec]
    finally:
        rix.job_destroy(job)


# The tiled PSF grids on the image grid instead of the 2N image's own grid,
# so it matches the oracle's PSF to the gridding kernel's accuracy (the
# oracle's PSF is within 6e-8 of the direct DFT on these cases), not to
# rounding: 1e-6 in FP64, 1e-5 in FP32.
TOL_TILES = {0: 1e-5, 1: 1e-6}


@pytest.mark.parametrize("name,prec,nparts", CASES[:4])
def test_tiled_psf_matches_oracle(ctx, obs_small, obs_wstack, name, prec, nparts):
    """rix_psf with RIX_PSF_TILES (four N x N tiles on the image grid, the form
    N = 4096 jobs take): the whole 2N x 2N PSF, seams included, against the
    oracle's; then RIX_PSF_DOUBLE_GRID forms the PSF again, to the oracle's
    own tolerance."""
    from paper_2507_22128_gb300 import rix
    obs = _obs(name, obs_small, obs_wstack)
    job, _ = _job(ctx, obs, prec, nparts)
    try:
        st = _oracle(obs, nparts)
        rix.job_set_psf_method(job, rix.PSF_TILES)
        n = obs.n
        for p in range(nparts):
            out = torch.empty((2 * n, 2 * n), dtype=real_dtype(prec), device="cuda")
            wsum = rix.psf(job, p, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy().astype(np.float64)
            assert wsum == pytest.approx(st.wsum[p], rel=1e-12)
            assert rel_l2(got, st.psf[p]) < TOL_TILES[prec]
            assert got[n, n] == pytest.approx(1.0, abs=TOL_TILES[prec])
            # the rows and columns on both sides of the tile seams
            for sl in (np.s_[n - 1:n + 1, :], np.s_[:, n - 1:n + 1], np.s_[0:1, :], np.s_[:, 0:1]):
                assert rel_l2(got[sl], st.psf[p][sl]) < 10 * TOL_TILES[prec]
        rix.job_set_psf_method(job, rix.PSF_DOUBLE_GRID)
        for p in range(nparts):
            out = torch.empty((2 * n, 2 * n), dtype=real_dtype(prec), device="cuda")
            rix.psf(job, p, out)
            torch.cuda.synchronize()
            assert rel_l2(out.cpu().numpy(), st.psf[p]) < TOL[prec]
    finally:
        rix.job_destroy(job)


@pytest.mark.parametrize("name,prec,nparts", CASES)
def test_major_cycle_matches_oracle(ctx, obs_small, obs_wstack, name, prec, nparts):
    from oracle import gridder
    from paper_2507_22128_gb300 import rix
    obs = _obs(name, obs_small, obs_wstack)
    job, _ = _job(ctx, obs, prec, nparts)
    try:
        st = _oracle(obs, nparts)
        w = obs.weight.reshape(-1).astype(np.float64)
        model = sparse_model(obs.n, 30, seed=5)
        for p in range(nparts):
            res = torch.empty((obs.n, obs.n), dtype=real_dtype(prec), device="cuda")
            rix.major_cycle(job, p, to_dev(obs.vis.reshape(-1), cplx_dtype(prec)),
                            to_dev(model, real_dtype(prec)), res)
            torch.cuda.synchronize()
            want = gridder.residual(obs.vis.reshape(-1), w, model, st.gparts[p])
            assert rel_l2(res.cpu().numpy(), want) < TOL[prec]
    finally:
        rix.job_destroy(job)


def test_fp32_operator_vs_direct_dft(ctx, obs_wstack):
    """FP32 GPU degrid/grid within 1e-4 of the exact measurement operator."""
    from oracle import dft
    from paper_2507_22128_gb300 import rix
    obs = obs_wstack
    job, mask = _job(ctx, obs, rix.FP32, 2)
    try:
        x = sparse_model(obs.n, 25, seed=6)
        u, v, w = dft.uvw_lambda(obs.uvw, obs.freq)
        rng = np.random.default_rng(7)
        sel = np.nonzero((mask & 1) == 1)[0]
        sub = np.sort(rng.choice(sel, 2000, replace=False))
        vis = torch.zeros(obs.nvis, dtype=torch.complex64, device="cuda")
        rix.degrid(job, 0, to_dev(x, torch.float32), vis)
        torch.cuda.synchronize()
        want = dft.degrid_pixels_sparse(x, u[sub], v[sub], w[sub], obs.cell_rad, True)
        assert rel_l2(vis.cpu().numpy()[sub], want) < 1e-4
        # grid: sampled pixels of the dirty image of partition 0
        img = torch.empty((obs.n, obs.n), dtype=torch.float32, device="cuda")
        rix.grid(job, 0, to_dev(obs.vis.reshape(-1), torch.complex64), img)
        torch.cuda.synchronize()
        rows = rng.integers(0, obs.n, 64)
        cols = rng.integers(0, obs.n, 64)
        wt = np.where((mask & 1) == 1, obs.weight.reshape(-1), 0.0)
        want = dft.adjoint_at(wt * obs.vis.reshape(-1), u, v, w, obs.n, obs.cell_rad, True, rows, cols) / wt.sum()
        assert rel_l2(img.cpu().numpy()[rows, cols], want) < 1e-4
    finally:
        rix.job_destroy(job)


@pytest.fixture(scope="module")
def obs_outside(obs_small):
    """The small recipe with 2 % of its rows' uvw stretched 5-7x: the kernel
    footprints of many of those samples leave the 256 x 256 grid (they are
    dropped and counted by both sides), others stay inside near the edge."""
    import dataclasses
    rng = np.random.default_rng(17)
    uvw = obs_small.uvw.copy()
    rows = rng.choice(obs_small.nrow, obs_small.nrow // 50, replace=False)
    uvw[rows] *= rng.uniform(5.0, 7.0, (rows.shape[0], 1))
    return dataclasses.replace(obs_small, uvw=uvw)


@pytest.mark.parametrize("prec", [0, 1])
def test_samples_outside_the_grid(ctx, obs_outside, prec):
    """Samples whose footprint leaves the grid: counted and excluded
    identically (masks bit-exact, zero for them), and the operator on the rest
    matches the oracle gridder (degrid, grid, PSF, major cycle)."""
    from oracle import gridder
    from paper_2507_22128_gb300 import rix
    obs = obs_outside
    job, mask = _job(ctx, obs, prec, 2)
    try:
        st = _oracle(obs, 2)
        n_out = int((~st.geom.inside).sum())
        assert 0 < n_out < obs.nvis // 50
        s = rix.job_get_stats(job)
        assert s["n_outside"] == n_out
        assert np.array_equal(mask, st.mask)
        assert np.all(mask[~st.geom.inside] == 0)
        w = obs.weight.reshape(-1).astype(np.float64)
        x = sparse_model(obs.n, 30, seed=8)
        vis_d = to_dev(obs.vis.reshape(-1), cplx_dtype(prec))
        for p in range(2):
            g = st.gparts[p]
            vis = torch.zeros(obs.nvis, dtype=cplx_dtype(prec), device="cuda")
            rix.degrid(job, p, to_dev(x, real_dtype(prec)), vis)
            img = torch.empty((obs.n, obs.n), dtype=real_dtype(prec), device="cuda")
            rix.grid(job, p, vis_d, img)
            psf = torch.empty((2 * obs.n, 2 * obs.n), dtype=real_dtype(prec), device="cuda")
            rix.psf(job, p, psf)
            res = torch.empty((obs.n, obs.n), dtype=real_dtype(prec), device="cuda")
            rix.major_cycle(job, p, vis_d, to_dev(x, real_dtype(prec)), res)
            torch.cuda.synchronize()
            got = vis.cpu().numpy()
            assert rel_l2(got[g.inside], gridder.degrid(x, g)[g.inside]) < TOL[prec]
            assert np.all(got[~g.inside] == 0)
            assert rel_l2(img.cpu().numpy(), gridder.dirty(obs.vis.reshape(-1), w, g)) < TOL[prec]
            assert rel_l2(psf.cpu().numpy(), st.psf[p]) < TOL[prec]
            assert rel_l2(res.cpu().numpy(), gridder.residual(obs.vis.reshape(-1), w, x, g)) < TOL[prec]
    finally:
        rix.job_destroy(job)


@pytest.fixture(scope="module")
def obs_dense():
    """The medium recipe's 1" cell on a 128 x 128 field: 32 antennas x 100
    times x 2 channels (99,200 visibilities) land on a few hundred kernel
    footprints of the low partition (up to 3,440 samples share one), so the
    FP32 gridder's chunks span several batches of 32 and one footprint spans
    several chunks and work items."""
    from paper_2507_22128_gb300 import synth
    return synth.medium(seed=21, n_times=100, n=128, n_ant=32, n_chan=2)


@pytest.fixture(scope="module")
def dense_oracle(obs_dense):
    from oracle import gridder
    obs = obs_dense
    st = _oracle(obs, 2)
    w = obs.weight.reshape(-1).astype(np.float64)
    model = sparse_model(obs.n, 20, seed=9)
    vis = obs.vis.reshape(-1)
    res = [gridder.residual(vis, w, model, st.gparts[p]) for p in range(2)]
    dirty = [gridder.dirty(vis, w, st.gparts[p]) for p in range(2)]
    return st, model, res, dirty


@pytest.mark.parametrize("limit", [1, 7, 32, 33, 64, 256])
def test_fp32_gridder_at_every_chunk_limit(ctx, obs_dense, dense_oracle, limit):
    """The FP32 w-stacked gridder regrouped at chunk limits below, at and
    above its 32-entry batch (rix_job_tune): fused major cycle, grid and PSF
    (the same kernel on the PSF's grid) of both partitions within 1e-5 of the
    oracle."""
    from paper_2507_22128_gb300 import rix
    obs = obs_dense
    st, model, want_res, want_dirty = dense_oracle
    # the workload does put more samples than every tested limit on one footprint
    g = st.geom
    sel = np.nonzero(st.mask & 1)[0]
    _, per_tap = np.unique((g.p0[sel] * 4096 + g.j0u[sel]) * 4096 + g.j0v[sel], return_counts=True)
    assert per_tap.max() > 2048 and per_tap.max() > limit
    job, _ = _job(ctx, obs, rix.FP32, 2)
    try:
        rix.job_tune(job, limit, 0)
        vis = to_dev(obs.vis.reshape(-1), torch.complex64)
        for p in range(2):
            res = torch.empty((obs.n, obs.n), dtype=torch.float32, device="cuda")
            rix.major_cycle(job, p, vis, to_dev(model, torch.float32), res)
            img = torch.empty((obs.n, obs.n), dtype=torch.float32, device="cuda")
            rix.grid(job, p, vis, img)
            torch.cuda.synchronize()
            assert rel_l2(res.cpu().numpy(), want_res[p]) < TOL[rix.FP32]
            assert rel_l2(img.cpu().numpy(), want_dirty[p]) < TOL[rix.FP32]
            psf = torch.empty((2 * obs.n, 2 * obs.n), dtype=torch.float32, device="cuda")
            wsum = rix.psf(job, p, psf)
            torch.cuda.synchronize()
            assert abs(wsum - st.wsum[p]) <= 1e-9 * st.wsum[p]
            assert rel_l2(psf.cpu().numpy(), st.psf[p]) < TOL[rix.FP32]
        rix.job_sync(job)
    finally:
        rix.job_destroy(job)


def test_chunk_limit_range(ctx, obs_small):
    from paper_2507_22128_gb300 import rix
    job, _ = _job(ctx, obs_small, rix.FP32, 2)
    try:
        for bad in (0, 257):
            with pytest.raises(rix.RixError):
                rix.job_tune(job, bad, 0)
        rix.job_tune(job, 256, 0)
    finally:
        rix.job_destroy(job)
