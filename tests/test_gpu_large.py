"""Parity at the large recipe's geometry (4096 x 4096 at 0.5", 32 w-planes, 8
channels over 1.3-1.5 GHz, 128 antennas on a 10 km spiral) on a 1/64 subset
of its 4000 time samples (62 times: 4.03 M visibilities), FP32, 2 and 4 uv
partitions: masks, ring radii and the sort bit-exact in full; degrid on 10^4
sampled visibilities, grid and the fused major cycle on 64 sampled pixels
per partition against the direct DFT within the FP32 operator's 1e-4; the
major-cycle probe reproduces the major cycle's residual.

The PSF of a 4096^2 job is formed as four N x N tiles on the image grid (its
own 2N grid would need 16384-long transforms): the peak and 96 sampled pixels
(the centre, the tile seams, anywhere) against Re A^H w / W_p by direct DFT.
The minor cycles at this size (ms-CLEAN with the recipe's scales, FISTA with
2N = 8192 transforms), and those of the largest FP64 job (2048^2), have no
oracle run here; two full cycles of each are checked for what holds at any
size: components from the scales allowed in cycle 1, a finite non-zero
image, and a residual peak that falls from cycle 1 to 2."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_l2, sparse_model, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[2, 4])
def large(request):
    need_gpu()
    from oracle import gridder, partition
    from paper_2507_22128_gb300 import rix, synth
    P = request.param
    obs = synth.large(seed=3, n_times=62, with_vis=False)
    ctx = rix.create(0)
    job = rix.job_create(ctx, obs.n, obs.cell_rad, obs.n_wplanes, list(obs.freq), rix.FP32, P, obs.nrow)
    mask = torch.zeros(obs.nvis, dtype=torch.uint8, device="cuda")
    rix.set_uv_partition(job, to_dev(obs.uvw, torch.float64), to_dev(obs.weight, torch.float32), None, 1.0, mask)
    torch.cuda.synchronize()
    g = gridder.geometry(obs.uvw, obs.freq, obs.n, obs.cell_rad, nw=obs.n_wplanes)
    r = partition.radius_px(g)
    ells = partition.ring_radii(r, P)
    want_mask = partition.masks(r, ells, 1.0, P, g.inside)
    yield obs, rix, job, mask.cpu().numpy(), g, ells, want_mask, P
    rix.job_destroy(job)
    rix.destroy(ctx)


def test_partition_bit_exact(large):
    from oracle import partition
    obs, rix, job, mask, g, ells, want_mask, P = large
    assert np.array_equal(mask, want_mask)
    s = rix.job_get_stats(job)
    assert s["n_outside"] == int((~g.inside).sum())
    for i in range(P - 1):
        assert s["ell_px"][i] == ells[i]
    keys, samples, _ = partition.entries(g, want_mask, 16, P)
    sk, ss = partition.sort_entries(keys, samples)
    gk = torch.empty(sk.shape[0], dtype=torch.int32, device="cuda")
    gs = torch.empty(sk.shape[0], dtype=torch.int32, device="cuda")
    rix.get_sorted_entries(job, gk, gs)
    torch.cuda.synchronize()
    assert np.array_equal(gk.cpu().numpy().view(np.uint32), sk)
    assert np.array_equal(gs.cpu().numpy().view(np.uint32), ss)


def test_operator_sampled_vs_direct_dft(large):
    from oracle import dft
    obs, rix, job, mask, g, ells, want_mask, P = large
    u, v, w = dft.uvw_lambda(obs.uvw, obs.freq)
    rng = np.random.default_rng(91 + P)
    y = (rng.standard_normal(obs.nvis) + 1j * rng.standard_normal(obs.nvis)).astype(np.complex64)
    y_d = to_dev(y, torch.complex64)
    wt_all = obs.weight.reshape(-1).astype(np.float64)
    for part in (0, P - 1):
        sel = ((mask >> part) & 1) == 1
        idx = np.nonzero(sel)[0]
        x = sparse_model(obs.n, 25, seed=101 + part)
        # degrid on sampled visibilities
        vis = torch.zeros(obs.nvis, dtype=torch.complex64, device="cuda")
        rix.degrid(job, part, to_dev(x, torch.float32), vis)
        torch.cuda.synchronize()
        sub = np.sort(rng.choice(idx, 10000, replace=False))
        want = dft.degrid_pixels_sparse(x, u[sub], v[sub], w[sub], obs.cell_rad, True)
        assert rel_l2(vis.cpu().numpy()[sub], want) < 1e-4
        # grid and the fused major cycle on sampled pixels
        rows = rng.integers(0, obs.n, 64)
        cols = rng.integers(0, obs.n, 64)
        img = torch.empty((obs.n, obs.n), dtype=torch.float32, device="cuda")
        rix.grid(job, part, y_d, img)
        res = torch.empty((obs.n, obs.n), dtype=torch.float32, device="cuda")
        rix.major_cycle(job, part, y_d, to_dev(x, torch.float32), res)
        torch.cuda.synchronize()
        wt = wt_all[sel]
        us, vs, ws = u[sel], v[sel], w[sel]
        want = dft.adjoint_at(wt * y.astype(np.complex128)[sel], us, vs, ws, obs.n, obs.cell_rad, True,
                              rows, cols) / wt.sum()
        assert rel_l2(img.cpu().numpy()[rows, cols], want) < 1e-4
        ch = 1 << 18
        ax = np.concatenate([dft.degrid_pixels_sparse(x, us[i:i + ch], vs[i:i + ch], ws[i:i + ch], obs.cell_rad, True)
                             for i in range(0, us.shape[0], ch)])
        want = dft.adjoint_at(wt * (y.astype(np.complex128)[sel] - ax), us, vs, ws, obs.n, obs.cell_rad, True,
                              rows, cols) / wt.sum()
        assert rel_l2(res.cpu().numpy()[rows, cols], want) < 1e-4
        # the probe times the same operator without touching the job
        ms = rix.major_cycle_probe(job, part, y_d, 2)
        assert ms > 0.0
        assert rix.job_get_stats(job)["cycle"][part] == 1


def test_psf_tiles_sampled_vs_direct_dft(large):
    from oracle import dft
    obs, rix, job, mask, g, ells, want_mask, P = large
    n = obs.n
    n2 = 2 * n
    u, v, w = dft.uvw_lambda(obs.uvw, obs.freq)
    wt_all = obs.weight.reshape(-1).astype(np.float64)
    for part in (0, P - 1):
        psf = torch.empty((n2, n2), dtype=torch.float32, device="cuda")
        wsum = rix.psf(job, part, psf)
        torch.cuda.synchronize()
        sel = ((mask >> part) & 1) == 1
        wt = wt_all[sel]
        assert wsum == pytest.approx(wt.sum(), rel=1e-12)
        assert float(psf[n, n]) == pytest.approx(1.0, abs=1e-5)
        rng = np.random.default_rng(201 + 10 * P + part)
        k = 24
        rows = np.concatenate([rng.integers(0, n2, k), n + rng.integers(-48, 48, k),
                               rng.choice([n - 1, n, 0, n2 - 1], k), rng.integers(0, n2, k)])
        cols = np.concatenate([rng.integers(0, n2, k), n + rng.integers(-48, 48, k),
                               rng.integers(0, n2, k), rng.choice([n - 1, n, 0, n2 - 1], k)])
        got = psf[torch.as_tensor(rows, device="cuda"), torch.as_tensor(cols, device="cuda")].cpu().numpy()
        want = dft.adjoint_at(wt.astype(np.complex128), u[sel], v[sel], w[sel], n2, obs.cell_rad, True,
                              rows, cols) / wt.sum()
        assert rel_l2(got, want) < 1e-4


def _point_source_vis(obs, seed):
    from oracle import dft
    x = sparse_model(obs.n, 25, seed=seed)
    u, v, w = dft.uvw_lambda(obs.uvw, obs.freq)
    ch = 1 << 18
    return np.concatenate([dft.degrid_pixels_sparse(x, u[i:i + ch], v[i:i + ch], w[i:i + ch], obs.cell_rad, True)
                           for i in range(0, u.shape[0], ch)]).reshape(obs.nrow, obs.nchan)


@pytest.mark.parametrize("kind,prec", [("msclean", 0), ("fista", 0), ("msclean", 1), ("fista", 1)])
def test_minor_cycles_at_size(kind, prec):
    """Two major+minor cycles of the largest job of each precision (P = 2,
    visibilities of 25 point sources by direct DFT): FP32 at 4096^2 (the
    large recipe on 1/64 of its rows: FISTA with 8192-point transforms, the
    ms-CLEAN scales {0, 4, 16, 32}), FP64 at 2048^2 (the medium recipe's
    antennas, 100 times: FISTA with 4096-point transforms, scales {0, 4,
    16}); both PSFs are tiled.  The FP64 PSF also matches the direct DFT on
    sampled pixels: within 1e-6 near the centre, 1e-4 over the field."""
    need_gpu()
    from oracle import dft
    from paper_2507_22128_gb300 import pipeline, rix, synth
    if prec == 0:
        obs = synth.large(seed=3, n_times=62, with_vis=False)
        scales = (0.0, 4.0, 16.0, 32.0)
    else:
        obs = synth.medium(seed=5, n_times=100, n=2048, with_vis=False)
        scales = (0.0, 4.0, 16.0)
    n = obs.n
    vis = _point_source_vis(obs, 303)
    ctx = rix.create(0)
    rec = pipeline.Reconstruction(ctx, n, obs.cell_rad, obs.n_wplanes, obs.freq, obs.nrow, 2,
                                  rix.FP32 if prec == 0 else rix.FP64)
    try:
        rec.set_data(obs.uvw, vis, obs.weight)
        if kind == "msclean":
            m = pipeline.Method("msclean", scales, 0.1, 200, 1e-4)
        else:
            m = pipeline.Method("fista", lam_rel=1e-3, iters=20, levels=4)
        if prec == 1 and kind == "fista":
            mask = torch.zeros(obs.nvis, dtype=torch.uint8, device="cuda")
            rix.set_uv_partition(rec.job, rec.uvw, rec.weight, None, 1.0, mask)
            sel = ((mask.cpu().numpy() >> 1) & 1) == 1
            psf = torch.empty((2 * n, 2 * n), dtype=torch.float64, device="cuda")
            rix.psf(rec.job, 1, psf)
            torch.cuda.synchronize()
            rng = np.random.default_rng(17)
            rows = np.concatenate([n + rng.integers(-32, 32, 32), rng.integers(0, 2 * n, 32)])
            cols = np.concatenate([n + rng.integers(-32, 32, 32), rng.choice([n - 1, n, 0], 32)])
            u, v, w = dft.uvw_lambda(obs.uvw, obs.freq)
            wt = obs.weight.reshape(-1).astype(np.float64)[sel]
            want = dft.adjoint_at(wt.astype(np.complex128), u[sel], v[sel], w[sel], 2 * n, obs.cell_rad, True,
                                  rows, cols) / wt.sum()
            got = psf[torch.as_tensor(rows, device="cuda"), torch.as_tensor(cols, device="cuda")].cpu().numpy()
            # near the centre the kernel's accuracy; over the 2N field the
            # w-planes' spacing (set for the N field: dw |n - 1| reaches 0.36
            # at the PSF's corners, 0.09 at the image's) bounds it, as it
            # would on the PSF's own grid
            assert rel_l2(got[:32], want[:32]) < 1e-6
            assert rel_l2(got, want) < 1e-4
        peaks = []
        for c in range(2):
            res = [torch.empty((n, n), dtype=rec.rdtype, device="cuda") for _ in range(2)]
            for p in range(2):
                rec.major(p, res[p])
            torch.cuda.synchronize()
            peaks.append([float(r.abs().max()) for r in res])
            if kind == "fista":
                rec.minor_all(m, torch.cuda.current_stream())
            else:
                for p in range(2):
                    rec.minor(p, m)
            rix.job_sync(rec.job)
            if kind == "msclean" and c == 0:
                ell = rix.job_get_stats(rec.job)["ell_px"][0]
                for p in range(2):
                    sc, _, _ = rix.get_components(rec.job, p)
                    assert 0 < len(sc) <= 200
                    used = set(int(s) for s in sc)
                    # scales present in cycle 1: partition 0 all; partition 1
                    # s = 0 and those with N / (2 s) >= ell - delta
                    allowed = {0} | {i for i, s in enumerate(m.scales) if s > 0 and (p == 0 or n / (2 * s) >= ell - 1.0)}
                    assert used <= allowed
        img = rec.combine()
        torch.cuda.synchronize()
        assert bool(torch.isfinite(img).all())
        assert float(img.abs().max()) > 0.0
        for p in range(2):
            assert peaks[1][p] < peaks[0][p]
    finally:
        rec.close()
        rix.destroy(ctx)
