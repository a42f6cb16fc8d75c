"""GPU parity of the band-limited exchange (Sec. 6.3, Sec. 7 item a): each
partition sends the ring-support coefficients of Gamma_p F pad i_bar_p
instead of the image Phi_p.  The receivers rebuild Phi_p without loss, so a
job run with the spectral exchange matches the oracle's loop (which
exchanges images) within the same tolerances as the image exchange: FP64
1e-9, FP32 1e-4.  The message sizes are the oracle's support counts
exactly, and smaller than the image for every partition but the
outermost."""
import numpy as np
import pytest

from gpu_util import need_gpu, real_dtype, rel_l2, cplx_dtype

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    from paper_2507_22128_gb300 import rix
    c = rix.create(0)
    yield c
    rix.destroy(c)


@pytest.mark.parametrize("method,prec,nparts", [("fista", 1, 2), ("fista", 0, 2), ("fista", 1, 4),
                                                 ("msclean", 1, 2)])
def test_loop_with_spectral_exchange_matches_oracle(ctx, obs_small, obs_wstack, method, prec, nparts):
    from oracle import framework
    from paper_2507_22128_gb300 import pipeline, rix
    obs = obs_wstack if method == "fista" else obs_small
    st = framework.setup(obs.uvw, obs.freq, obs.weight, obs.n, obs.cell_rad, obs.n_wplanes, nparts)
    loop = framework.Loop(st, obs.vis, obs.weight)
    rec = pipeline.observation_job(ctx, obs, nparts, prec, exchange=rix.EXCHANGE_SPECTRAL)
    if method == "fista":
        m = pipeline.Method("fista", lam_rel=1e-3, iters=15, levels=3)
    else:
        m = pipeline.Method("msclean", (0.0, 3.0, 9.0), 0.1, 150, 1e-4)
    tol = 1e-9 if prec == 1 else 1e-4
    try:
        for c in range(1, 4):
            for p in range(nparts):
                loop.major(p)
                rec.major(p)
            for p in range(nparts):
                if method == "fista":
                    loop.minor_fista(p, c, lam_rel=1e-3, n_iter=15, levels=3)
                else:
                    loop.minor_msclean(p, c, [0.0, 3.0, 9.0], 0.1, 150, 1e-4)
                rec.minor(p, m)
            loop.exchange()
            for p in range(nparts):
                out = torch.empty((obs.n, obs.n), dtype=real_dtype(prec), device="cuda")
                rix.get_model(rec.job, p, out)
                torch.cuda.synchronize()
                assert rel_l2(out.cpu().numpy(), loop.model[p]) < tol
        assert rel_l2(rec.combine().cpu().numpy(), loop.combine()) < tol
    finally:
        rec.close()


@pytest.mark.parametrize("prec", [1, 0])
def test_pack_unpack_round_trip_and_message_size(ctx, obs_wstack, prec):
    from oracle import filters, framework
    from paper_2507_22128_gb300 import pipeline, rix
    obs = obs_wstack
    st = framework.setup(obs.uvw, obs.freq, obs.weight, obs.n, obs.cell_rad, obs.n_wplanes, 2)
    loop = framework.Loop(st, obs.vis, obs.weight)
    rec = pipeline.observation_job(ctx, obs, 2, prec)
    m = pipeline.Method("fista", lam_rel=1e-3, iters=15, levels=3)
    try:
        for p in range(2):
            loop.major(p)
            rec.major(p)
        for p in range(2):
            loop.minor_fista(p, 1, lam_rel=1e-3, n_iter=15, levels=3)
            rec.minor(p, m)
        n = obs.n
        for p in range(2):
            cnt = rix.phi_support(rec.job, p)
            assert cnt == filters.ring_support(st.gam[p]).shape[0]
            packed = torch.empty(cnt, dtype=cplx_dtype(prec), device="cuda")
            rix.phi_pack(rec.job, p, packed)
            phi = torch.empty((n, n), dtype=real_dtype(prec), device="cuda")
            rix.phi_unpack(rec.job, p, packed, phi)
            torch.cuda.synchronize()
            want = [h[3] for h in loop.history if h[1] == p][-1]      # Phi_p of cycle 1
            assert rel_l2(phi.cpu().numpy(), want) < (1e-9 if prec == 1 else 1e-4)
        # the inner partition's message is a fraction of the image
        assert 2 * rix.phi_support(rec.job, 0) < 0.5 * n * n
    finally:
        rec.close()
