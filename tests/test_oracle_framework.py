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


def _cycle_two_state(o, st, p):
    """The loop after cycle 1 (both nodes' major and ms-CLEAN minor cycles and
    the exchange), then node p's cycle-2 major cycle and ingest."""
    loop = framework.Loop(st, o.vis, o.weight)
    for q in range(st.nparts):
        loop.major(q)
    for q in range(st.nparts):
        loop.minor_msclean(q, 1, [0, 3], 0.1, 40, 1e-5)
    loop.exchange()
    loop.major(p)
    loop._ingest(p, 2)
    return loop


@pytest.mark.parametrize("nparts", [2, 4])
def test_composite_psf_is_the_same_on_every_node(obs_small, nparts):
    """Eq. 7 at n >= 2: node p's PSF gamma Gamma_p H_p + sum_q mu_q Gamma_q H_q
    with gamma = W_p / W and mu_q = W_q / W is sum_q W_q Gamma_q H_q / W for
    every p: each node solves against the same full-resolution PSF.  At n = 1
    node p's PSF is Gamma_p H_p alone."""
    o = obs_small
    st = framework.setup(o.uvw, o.freq, o.weight, o.n, o.cell_rad, 0, nparts)
    loop = framework.Loop(st, o.vis, o.weight)
    for q in range(nparts):
        loop.major(q)
    ps2 = [loop.msclean_problem(q, 2)[1] for q in range(nparts)]
    for q in range(1, nparts):
        assert np.max(np.abs(ps2[q] - ps2[0])) < 1e-14 * np.max(np.abs(ps2[0]))
    # not a trivial agreement: the nodes' own first-cycle PSFs differ
    ps1 = [loop.msclean_problem(q, 1)[1] for q in range(nparts)]
    for q in range(nparts):
        assert np.max(np.abs(ps1[q] - st.gam[q] * st.hspec[q])) == 0.0
    assert np.max(np.abs(ps1[1] - ps1[0])) > 0.1 * np.max(np.abs(ps1[0]))
    # its zero-frequency value is the weight-averaged PSF peak spectrum of the
    # partitions holding k = 0 (Gamma = 1 there for the innermost ring only)
    n = o.n
    assert ps2[0][n, n].real == pytest.approx(st.wsum[0] / st.wsum.sum() * st.hspec[0][n, n].real, rel=1e-12)


def test_composite_dirty_image_assembled_by_hand(small_setup2):
    """Eq. 7's dirty image at n = 2, gamma Gamma_p i_p + sum_q mu_q H_q rho_{q->p},
    against an assembly in the image domain that shares no code with the
    oracle's spectral one: Gamma_p applied with explicit centred DFT matrices on
    the 2N-padded grid, H_q rho as the linear convolution of rho with the
    2N x 2N PSF (scipy.signal.convolve2d), gamma and mu from the weight sums."""
    from scipy.signal import convolve2d
    o, st = small_setup2
    n = o.n
    m = 2 * n
    j = np.arange(m) - n
    E = np.exp(-2j * np.pi * np.outer(j, j) / m)     # centred DFT; E is symmetric

    def gamma_apply(x, gam):
        z = np.zeros((m, m), dtype=complex)
        z[n // 2:n // 2 + n, n // 2:n // 2 + n] = x
        spec = E @ z @ E
        back = np.conj(E) @ (gam * spec) @ np.conj(E) / (m * m)
        return back[n // 2:n // 2 + n, n // 2:n // 2 + n].real

    for p in range(2):
        loop = _cycle_two_state(o, st, p)
        d, _ = loop.msclean_problem(p, 2)
        got = filters.crop(filters.ispectrum(d)).real
        q = 1 - p
        wsum = st.wsum
        gam_n, mu_q = wsum[p] / wsum.sum(), wsum[q] / wsum.sum()
        h_rho = convolve2d(loop.rho[p][q], st.psf[q], mode="full")[n:2 * n, n:2 * n]
        want = gam_n * gamma_apply(loop.residual[p], st.gam[p]) + mu_q * h_rho
        assert np.max(np.abs(got - want)) < 1e-11 * np.max(np.abs(want))
        assert np.max(np.abs(loop.rho[p][q])) > 0.0      # the received term is present


def test_both_nodes_holding_all_data_sum_to_the_serial_problem(obs_small):
    """delta beyond every radius: both partitions hold every sample, so at
    n = 1 each node's residual and PSF are the serial ones (Eq. 2), and since
    Gamma_L + Gamma_H = 1 the two nodes' composite dirty images and PSFs
    (gamma = 1, mu = 0) add up to the serial dirty image and PSF."""
    o = obs_small
    st1 = framework.setup(o.uvw, o.freq, o.weight, o.n, o.cell_rad, 0, 1)
    big = 10.0 * o.n
    st2 = framework.setup(o.uvw, o.freq, o.weight, o.n, o.cell_rad, 0, 2, delta=big)
    assert np.all(st2.mask[st2.geom.inside] == 3)
    serial = framework.Loop(st1, o.vis, o.weight)
    serial.major(0)
    loop = framework.Loop(st2, o.vis, o.weight)
    for p in range(2):
        loop.major(p)
        assert np.max(np.abs(loop.residual[p] - serial.residual[0])) < 1e-13
        assert np.max(np.abs(st2.psf[p] - st1.psf[0])) < 1e-13
    d0, p0 = loop.msclean_problem(0, 1)
    d1, p1 = loop.msclean_problem(1, 1)
    ds, pss = serial.msclean_problem(0, 1)
    assert np.max(np.abs(d0 + d1 - ds)) < 1e-12 * np.max(np.abs(ds))
    assert np.max(np.abs(p0 + p1 - pss)) < 1e-12 * np.max(np.abs(pss))
    # neither node alone is the serial problem (Gamma ramps across the whole plane)
    assert np.max(np.abs(d0 - ds)) > 1e-3 * np.max(np.abs(ds))
