"""Host orchestration of the decentralized loop (pipeline.py), CPU only: the
library calls and CUDA streams are replaced by recording fakes, so the test
checks what the pipeline issues and where -- every partition's major cycle
before the minor cycles of the same cycle, the FISTA minor cycles batched
into one call (or issued per partition), the dictionary and schedule passed
through, and the single-partition path."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")


class _Stream:
    n = 0

    def __init__(self, *a, **k):
        _Stream.n += 1
        self.name = f"s{_Stream.n}"

    def wait_event(self, ev):
        pass


class _Event:
    def record(self, stream=None):
        pass


MAIN = _Stream()        # the caller's stream


@pytest.fixture
def pl(monkeypatch):
    if not os.path.exists(os.path.join(ROOT, "paper_2507_22128_gb300", "librix.so")):
        from paper_2507_22128_gb300 import build
        build.build()
    from paper_2507_22128_gb300 import pipeline, rix
    calls = []
    monkeypatch.setattr(rix, "job_create", lambda *a, **k: "job")
    monkeypatch.setattr(rix, "job_destroy", lambda job: None)
    monkeypatch.setattr(rix, "major_cycle", lambda job, p, vis, a, b, st: calls.append(("major", p, st)))
    monkeypatch.setattr(rix, "minor_cycle_fista",
                        lambda job, p, lam, lam_rel, iters, levels, d_out, st, d, sched:
                        calls.append(("fista", p, st, d, sched)))
    monkeypatch.setattr(rix, "minor_cycle_fista_batch",
                        lambda job, parts, lam, lam_rel, iters, levels, st, d, sched:
                        calls.append(("fista_batch", tuple(parts), st, d, sched)))
    monkeypatch.setattr(rix, "minor_cycle_msclean",
                        lambda job, p, scales, gain, niter, thr, d_out, st: calls.append(("msclean", p, st)))
    monkeypatch.setattr(pipeline.torch.cuda, "Stream", _Stream)
    monkeypatch.setattr(pipeline.torch.cuda, "Event", _Event)
    monkeypatch.setattr(pipeline.torch.cuda, "current_stream", lambda dev=None: MAIN)
    return pipeline, rix, calls


def _rec(pipeline, n_part):
    return pipeline.Reconstruction(None, 64, 1e-5, 16, [1.4e9], 10, n_part=n_part, device="cpu")


def test_batched_fista_cycles(pl):
    pipeline, rix, calls = pl
    rec = _rec(pipeline, 3)
    m = pipeline.Method("fista", dictionary="db1-8", schedule=(0.5, 0.9))
    rec.cycles(m, 2, stream=MAIN, batch=True)
    streams = [s for (k, p, s) in [c[:3] for c in calls if c[0] == "major"]][:3]
    assert len(set(streams)) == 3 and MAIN not in streams   # one stream per partition
    want = []
    for _ in range(2):
        want += [("major", p, streams[p]) for p in range(3)]
        want += [("fista_batch", (0, 1, 2), streams[0], rix.DICT_DB1_8, (0.5, 0.9))]
    assert calls == want


def test_unbatched_cycles_issue_each_partition_on_its_stream(pl):
    pipeline, rix, calls = pl
    rec = _rec(pipeline, 2)
    rec.cycles(pipeline.Method("fista"), 1, stream=MAIN, batch=False)
    s0, s1 = calls[0][2], calls[1][2]
    assert calls == [("major", 0, s0), ("major", 1, s1),
                     ("fista", 0, s0, rix.DICT_DB4, None), ("fista", 1, s1, rix.DICT_DB4, None)]


def test_msclean_is_never_batched(pl):
    pipeline, rix, calls = pl
    rec = _rec(pipeline, 2)
    rec.cycles(pipeline.Method("msclean"), 1, stream=MAIN, batch=True)
    assert [c[0] for c in calls] == ["major", "major", "msclean", "msclean"]
    assert calls[2][2] == calls[0][2] and calls[3][2] == calls[1][2]


def test_single_partition_runs_on_the_callers_stream(pl):
    pipeline, rix, calls = pl
    rec = _rec(pipeline, 1)
    rec.cycles(pipeline.Method("fista"), 2, stream=MAIN)
    assert calls == [("major", 0, MAIN), ("fista", 0, MAIN, rix.DICT_DB4, None)] * 2


def test_one_cycle_with_and_without_concurrency(pl):
    pipeline, rix, calls = pl
    rec = _rec(pipeline, 2)
    rec.cycle(pipeline.Method("fista"), MAIN, concurrent=False)
    assert calls == [("major", 0, MAIN), ("major", 1, MAIN),
                     ("fista", 0, MAIN, rix.DICT_DB4, None), ("fista", 1, MAIN, rix.DICT_DB4, None)]
    calls.clear()
    rec.cycle(pipeline.Method("fista"), MAIN, concurrent=True, batch=True)
    assert calls[2] == ("fista_batch", (0, 1), MAIN, rix.DICT_DB4, None)
