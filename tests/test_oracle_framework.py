"""Pins of the decentralized loop (Sec. 3-4, Eq. 3, 5, 7) and the combine."""
import numpy as np
import pytest

from oracle import filters, fista, framework, gridder, msclean
from paper_2507_22128_gb300 import synth


@pytest.fixture(scope="module")
def small_setup2(obs_small):
    o = obs_small
    return o, framework.setup(o.uvw, o.freq, o.weight, o.n, o.cell_rad, 0, 2)


def test_single_partition_is_serial_msclean(obs_small):
    o = obs_small
    st = framework.setup(o.uvw, o.freq, o.weight, o.n, o.cell_rad, 0, 1)
    assert np.allclose(st.gam[0], 1.0)
    loop = framework.run(st, o.vis, o.weight, 2, "msclean", scales=[0, 3, 9], gain=0.1,
                         niter=100, threshold=1e-4)
    # serial: Eq. 2 residual, Eq. 6 ms-CLEAN with the full PSF, Eq. 3 update
    g = gridder.geometry(o.uvw, o.freq, o.n, o.cell_rad, W=8, nw=0)
    g2 = gridder.geometry(o.uvw, o.freq, o.n, o.cell_rad, W=8, nw=0, image_scale=2)
    w = o.weight.reshape(-1).astype(np.float64)
    hs = filters.psf_spectrum(gridder.psf(w, g2))
    model = np.zeros((o.n, o.n))
    for _ in range(2):
        res = gridder.residual(o.vis.reshape(-1), w, model, g)
        model = model + msclean.clean(filters.image_spectrum(res), hs, [0, 3, 9], 0.1, 100, 1e-4).model
    assert np.max(np.abs(loop.combine() - model)) < 1e-12


def test_single_partition_is_serial_fista(obs_small):
    o = obs_small
    st = framework.setup(o.uvw, o.freq, o.weight, o.n, o.cell_rad, 0, 1)
    loop = framework.run(st, o.vis, o.weight, 2, "fista", lam_rel=1e-3, n_iter=20, levels=3)
    g = gridder.geometry(o.uvw, o.freq, o.n, o.cell_rad, W=8, nw=0)
    g2 = gridder.geometry(o.uvw, o.freq, o.n, o.cell_rad, W=8, nw=0, image_scale=2)
    w = o.weight.reshape(-1).astype(np.float64)
    hs = filters.psf_spectrum(gridder.psf(w, g2))
    model = np.zeros((o.n, o.n))
    lam = None
    for _ in range(2):
        res = gridder.residual(o.vis.reshape(-1), w, model, g)
        lam = 1e-3 * np.abs(res).max() if lam is None else lam
        # Eq. 4: || i - H W alpha ||^2 + lambda ||alpha||_1
        prob = fista.problem(filters.image_spectrum(res), hs, np.ones_like(hs.real), [], 0.0)
        model = model + fista.solve(prob, lam, 20, 3)[0]
    assert np.max(np.abs(loop.combine() - model)) < 1e-12


def test_rho_in_place_equals_explicit_sums(small_setup2):
    o, st = small_setup2
    loop = framework.run(st, o.vis, o.weight, 3, "msclean", scales=[0, 3], gain=0.1,
                         niter=30, threshold=1e-5)
    P = st.nparts
    for p in range(P):
        for q in range(P):
            if q == p:
                continue
            # rho_{q->p} after cycle 3's publish, before cycle 4's ingest:
            # sum_{j<=2} Phi_q^j - Gamma_q sum_{j<=3} i_bar_p^j
            phis = [h[3] for h in loop.history if h[1] == q and h[0] <= 2]
            ibars = [h[2] for h in loop.history if h[1] == p and h[0] <= 3]
            want = sum(phis) - filters.apply(sum(ibars), st.gam[q])
            assert np.max(np.abs(loop.rho[p][q] - want)) < 1e-12
            # and Phi_q = Gamma_q i_bar_q
            for c, qq, ib, phi in loop.history:
                if qq == q:
                    assert np.max(np.abs(phi - filters.apply(ib, st.gam[q]))) < 1e-14


def test_combine_equal_weights(small_setup2):
    o, st = small_setup2
    loop = framework.run(st, o.vis, o.weight, 1, "msclean", scales=[0], gain=0.1, niter=10,
                         threshold=1e-5)
    assert np.allclose(loop.combine(), 0.5 * loop.model[0] + 0.5 * loop.model[1], atol=0)


def test_snr_improves_over_cycles(small_setup2):
    o, st = small_setup2
    truth = synth.sky_image(o.sky, o.n)
    loop = framework.Loop(st, o.vis, o.weight)
    snrs = []
    for c in range(1, 4):
        for p in range(2):
            loop.major(p)
        for p in range(2):
            loop.minor_msclean(p, c, [0, 3, 9], 0.1, 300, 1e-4)
        loop.exchange()
        snrs.append(framework.snr_db(truth, loop.combine()))
    assert snrs[-1] > snrs[0]


def test_single_partition_sara_with_lambda_schedule_is_serial(obs_small):
    """P = 1 with the concatenated db1..db8 dictionary and the paper's
    lambda_n = a ||i^n||_2 b^n is serial FISTA (Eq. 4) with that dictionary."""
    from oracle import wavelet
    o = obs_small
    a, b = 2e-4, 1.5
    st = framework.setup(o.uvw, o.freq, o.weight, o.n, o.cell_rad, 0, 1)
    loop = framework.run(st, o.vis, o.weight, 2, "fista", n_iter=8, levels=2, dictionary="sara", schedule=(a, b))
    g = gridder.geometry(o.uvw, o.freq, o.n, o.cell_rad, W=8, nw=0)
    g2 = gridder.geometry(o.uvw, o.freq, o.n, o.cell_rad, W=8, nw=0, image_scale=2)
    w = o.weight.reshape(-1).astype(np.float64)
    hs = filters.psf_spectrum(gridder.psf(w, g2))
    d = wavelet.Concatenation(2)
    model = np.zeros((o.n, o.n))
    for n in (1, 2):
        res = gridder.residual(o.vis.reshape(-1), w, model, g)
        prob = fista.problem(filters.image_spectrum(res), hs, np.ones_like(hs.real), [], 0.0)
        model = model + fista.solve(prob, a * np.linalg.norm(res) * b ** n, 8, 2, dictionary=d)[0]
    assert np.max(np.abs(loop.combine() - model)) < 1e-12
    assert np.abs(model).max() > 0.0
