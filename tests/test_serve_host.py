"""Host logic of the continuous-batching loop (serve.py), CPU only: the
GPU-facing run object and the streams are replaced by fakes that advance one
stage per call, so the test checks admission in arrival order, the slot
limit, slot reuse, waiting on a full memory budget (RIX_ENOMEM) while other
jobs run, latency bookkeeping and the summary."""
import sys
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")


class _Event:
    def query(self):
        return True


class _FakeRun:
    live = 0
    max_live = 0
    capacity = 10 ** 9
    admitted = []

    def __init__(self, ctx, req, stream):
        if _FakeRun.live >= _FakeRun.capacity:
            from paper_2507_22128_gb300 import rix
            raise rix.RixError(rix.ENOMEM, "fake memory budget")
        _FakeRun.live += 1
        _FakeRun.max_live = max(_FakeRun.max_live, _FakeRun.live)
        _FakeRun.admitted.append(req.rid)
        self.req = req
        self.stage = 0
        self.done_event = None
        self.out_host = None

    def issue_next(self):
        # upload/partition, n_major cycles, combine: n_major + 2 stages
        self.stage += 1
        if self.stage == self.req.n_major + 2:
            self.out_host = torch.full((2, 2), float(self.req.rid))
            self.done_event = _Event()

    @property
    def all_issued(self):
        return self.done_event is not None

    def close(self):
        _FakeRun.live -= 1


@pytest.fixture
def serve_mod(monkeypatch):
    if not os.path.exists(os.path.join(ROOT, "paper_2507_22128_gb300", "librix.so")):
        from paper_2507_22128_gb300 import build
        build.build()
    from paper_2507_22128_gb300 import serve
    monkeypatch.setattr(serve, "_Run", _FakeRun)
    monkeypatch.setattr(serve.torch.cuda, "Stream", lambda: object())
    _FakeRun.live = 0
    _FakeRun.max_live = 0
    _FakeRun.capacity = 10 ** 9
    _FakeRun.admitted = []
    return serve


def _reqs(serve, arrivals, n_major=3):
    from paper_2507_22128_gb300 import pipeline
    m = pipeline.Method("fista", lam_rel=1e-3, iters=5, levels=2)
    return [serve.Request(rid=i, obs=None, method=m, n_major=n_major, arrival=float(t))
            for i, t in enumerate(arrivals)]


def test_every_request_completes_in_arrival_order_within_the_slot_limit(serve_mod):
    serve = serve_mod
    arrivals = [0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.001, 0.002]
    reqs = _reqs(serve, list(reversed(arrivals)))        # given out of order
    out = serve.serve(None, reqs, n_slots=3, poll_s=1e-5)
    assert len(out) == len(arrivals)
    order = sorted(range(len(reqs)), key=lambda i: (reqs[i].arrival, i))
    assert _FakeRun.admitted == [reqs[i].rid for i in order]
    assert _FakeRun.max_live <= 3
    for q in out:
        assert q.t_admit >= q.arrival - 1e-9
        assert q.t_done >= q.t_admit
        assert q.latency == pytest.approx(q.t_done - q.arrival)
        assert np.all(q.image == q.rid)                # each job gets its own image back
    assert _FakeRun.live == 0                          # every job closed


def test_full_memory_budget_waits_for_running_jobs(serve_mod):
    serve = serve_mod
    _FakeRun.capacity = 2                              # the budget holds two jobs
    reqs = _reqs(serve, [0.0] * 5, n_major=2)
    out = serve.serve(None, reqs, n_slots=4, poll_s=1e-5)
    assert _FakeRun.max_live == 2
    assert sorted(_FakeRun.admitted) == list(range(5))
    assert all(q.t_done == q.t_done for q in out)      # no NaN: all finished


def test_full_budget_with_nothing_running_is_an_error(serve_mod):
    serve = serve_mod
    _FakeRun.capacity = 0
    from paper_2507_22128_gb300 import rix
    with pytest.raises(rix.RixError):
        serve.serve(None, _reqs(serve, [0.0]), n_slots=2, poll_s=1e-5)


def test_summary_and_arrivals(serve_mod):
    serve = serve_mod
    rng = np.random.default_rng(4)
    t = serve.poisson_arrivals(rng, 2000, 20.0)
    assert np.all(np.diff(t) > 0)
    assert np.mean(np.diff(t)) == pytest.approx(1 / 20.0, rel=0.1)
    reqs = _reqs(serve, [0.0, 1.0, 2.0])
    for q, (done, s) in zip(reqs, [(0.5, 10), (2.0, 20), (2.5, 30)]):
        q.t_done, q.samples = done, s
    sm = serve.summary(reqs)
    assert sm["jobs"] == 3
    assert sm["p50_latency_s"] == pytest.approx(0.5)
    assert sm["makespan_s"] == pytest.approx(2.5)
    assert sm["achieved_jobs_per_s"] == pytest.approx(3 / 2.5)
    assert sm["mvis_per_s"] == pytest.approx(60 / 2.5 / 1e6)
