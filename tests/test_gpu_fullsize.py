"""Parity at the full 1024^2 workload (64 antennas x 1000 times x 4 channels,
16 w-planes, 2 uv partitions, FP32) in the launch configuration the benchmark
times.  The oracle cannot run the whole operator at this size, so:
  masks, keys and the sorted order are compared bit-exact in full;
  degrid is compared with the direct DFT on 10^4 sampled visibilities of each
  partition, grid on 128 sampled pixels of each partition's dirty image
  (the exact adjoint sum over all of the partition's samples), both within
  the FP32 operator's 1e-4 bound.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_l2, sparse_model, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    need_gpu()
    from oracle import gridder, partition
    from paper_2507_22128_gb300 import rix, synth
    obs = synth.medium(with_vis=False)
    ctx = rix.create(0)
    job = rix.job_create(ctx, obs.n, obs.cell_rad, obs.n_wplanes, list(obs.freq), rix.FP32, 2, obs.nrow, 0)
    mask = torch.zeros(obs.nvis, dtype=torch.uint8, device="cuda")
    rix.set_uv_partition(job, to_dev(obs.uvw, torch.float64), to_dev(obs.weight, torch.float32), None, 1.0, mask)
    torch.cuda.synchronize()
    g = gridder.geometry(obs.uvw, obs.freq, obs.n, obs.cell_rad, nw=obs.n_wplanes)
    r = partition.radius_px(g)
    ells = partition.ring_radii(r, 2)
    want_mask = partition.masks(r, ells, 1.0, 2, g.inside)
    yield obs, rix, job, mask.cpu().numpy(), g, ells, want_mask
    rix.job_destroy(job)
    rix.destroy(ctx)


def test_masks_keys_and_order_bit_exact(full):
    from oracle import partition
    obs, rix, job, mask, g, ells, want_mask = full
    assert np.array_equal(mask, want_mask)
    s = rix.job_get_stats(job)
    assert s["n_outside"] == 0 == int((~g.inside).sum())
    assert s["ell_px"][0] == ells[0]
    assert s["w_min"] == g.w_min and s["dw"] == g.dw
    keys, samples, _ = partition.entries(g, want_mask, 16, 2)
    sk, ss = partition.sort_entries(keys, samples)
    assert s["n_entries"] == sk.shape[0]
    gk = torch.empty(sk.shape[0], dtype=torch.int32, device="cuda")
    gs = torch.empty(sk.shape[0], dtype=torch.int32, device="cuda")
    rix.get_sorted_entries(job, gk, gs)
    torch.cuda.synchronize()
    assert np.array_equal(gk.cpu().numpy().view(np.uint32), sk)
    assert np.array_equal(gs.cpu().numpy().view(np.uint32), ss)


@pytest.mark.parametrize("part", [0, 1])
def test_degrid_sampled_vs_direct_dft(full, part):
    from oracle import dft
    obs, rix, job, mask, *_ = full
    x = sparse_model(obs.n, 25, seed=21 + part)
    u, v, w = dft.uvw_lambda(obs.uvw, obs.freq)
    rng = np.random.default_rng(31 + part)
    sel = np.nonzero(((mask >> part) & 1) == 1)[0]
    sub = np.sort(rng.choice(sel, 10000, replace=False))
    vis = torch.zeros(obs.nvis, dtype=torch.complex64, device="cuda")
    rix.degrid(job, part, to_dev(x, torch.float32), vis)
    torch.cuda.synchronize()
    want = dft.degrid_pixels_sparse(x, u[sub], v[sub], w[sub], obs.cell_rad, True)
    assert rel_l2(vis.cpu().numpy()[sub], want) < 1e-4


@pytest.mark.parametrize("part", [0, 1])
def test_grid_sampled_vs_direct_dft(full, part):
    from oracle import dft
    obs, rix, job, mask, *_ = full
    rng = np.random.default_rng(41 + part)
    y = (rng.standard_normal(obs.nvis) + 1j * rng.standard_normal(obs.nvis)).astype(np.complex64)
    img = torch.empty((obs.n, obs.n), dtype=torch.float32, device="cuda")
    rix.grid(job, part, to_dev(y, torch.complex64), img)
    torch.cuda.synchronize()
    rows = rng.integers(0, obs.n, 128)
    cols = rng.integers(0, obs.n, 128)
    sel = ((mask >> part) & 1) == 1
    u, v, w = dft.uvw_lambda(obs.uvw, obs.freq)
    wt = obs.weight.reshape(-1).astype(np.float64)[sel]
    want = dft.adjoint_at(wt * y.astype(np.complex128)[sel], u[sel], v[sel], w[sel], obs.n, obs.cell_rad, True,
                          rows, cols) / wt.sum()
    assert rel_l2(img.cpu().numpy()[rows, cols], want) < 1e-4


@pytest.mark.parametrize("part", [0, 1])
def test_major_cycle_sampled_vs_direct_dft(full, part):
    """rix_major_cycle at full size (the fused degrid/residual/grid kernel the
    benchmark times): residual Re A^H W (v - A x) / W_p of a sparse model x and
    random observed visibilities v, on 128 sampled pixels, against the direct
    DFT over all of the partition's samples."""
    from oracle import dft
    obs, rix, job, mask, *_ = full
    rng = np.random.default_rng(51 + part)
    y = (rng.standard_normal(obs.nvis) + 1j * rng.standard_normal(obs.nvis)).astype(np.complex64)
    x = sparse_model(obs.n, 25, seed=61 + part)
    res = torch.empty((obs.n, obs.n), dtype=torch.float32, device="cuda")
    rix.major_cycle(job, part, to_dev(y, torch.complex64), to_dev(x, torch.float32), res)
    torch.cuda.synchronize()
    sel = ((mask >> part) & 1) == 1
    u, v, w = dft.uvw_lambda(obs.uvw, obs.freq)
    us, vs, ws = u[sel], v[sel], w[sel]
    ch = 1 << 18
    ax = np.concatenate([dft.degrid_pixels_sparse(x, us[i:i + ch], vs[i:i + ch], ws[i:i + ch], obs.cell_rad, True)
                         for i in range(0, us.shape[0], ch)])
    r = y.astype(np.complex128)[sel] - ax
    wt = obs.weight.reshape(-1).astype(np.float64)[sel]
    rows = rng.integers(0, obs.n, 128)
    cols = rng.integers(0, obs.n, 128)
    want = dft.adjoint_at(wt * r, us, vs, ws, obs.n, obs.cell_rad, True, rows, cols) / wt.sum()
    assert rel_l2(res.cpu().numpy()[rows, cols], want) < 1e-4


@pytest.mark.parametrize("part", [0, 1])
def test_psf_sampled_vs_direct_dft(full, part):
    """rix_psf at full size (2048 x 2048, centre at pixel (1024, 1024)): the
    peak is 1, and 128 sampled pixels (half of them within 64 pixels of the
    centre, where the PSF is large) match Re A^H w / W_p by direct DFT."""
    from oracle import dft
    obs, rix, job, mask, *_ = full
    n2 = 2 * obs.n
    psf = torch.empty((n2, n2), dtype=torch.float32, device="cuda")
    wsum = rix.psf(job, part, psf)
    torch.cuda.synchronize()
    got = psf.cpu().numpy()
    sel = ((mask >> part) & 1) == 1
    wt = obs.weight.reshape(-1).astype(np.float64)[sel]
    assert wsum == pytest.approx(wt.sum(), rel=1e-12)
    assert got[obs.n, obs.n] == pytest.approx(1.0, abs=1e-5)
    rng = np.random.default_rng(71 + part)
    rows = np.concatenate([rng.integers(0, n2, 64), obs.n + rng.integers(-64, 64, 64)])
    cols = np.concatenate([rng.integers(0, n2, 64), obs.n + rng.integers(-64, 64, 64)])
    u, v, w = dft.uvw_lambda(obs.uvw, obs.freq)
    want = dft.adjoint_at(wt.astype(np.complex128), u[sel], v[sel], w[sel], n2, obs.cell_rad, True,
                          rows, cols) / wt.sum()
    assert rel_l2(got[rows, cols], want) < 1e-4
