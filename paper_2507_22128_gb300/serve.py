"""Continuous-batching request loop for reconstruction jobs on one GPU.

Requests (an observation, a minor-cycle method, a number of major cycles)
arrive over time.  The loop admits a request as soon as it has arrived, a
stream slot is free and the context's device-memory budget accepts the job
(rix_job_create fails with RIX_ENOMEM otherwise and the request waits).
Admitted jobs advance one stage at a time in round robin -- upload and
partition, each major+minor cycle, combine and read-back -- each on its own
CUDA stream, so the work of different jobs overlaps on the device and a job
that arrives while others run starts without waiting for them to finish.
Each job keeps its grids, images and minor-cycle state resident in its rix
job until it completes.  Latency is arrival to the read-back of the combined
image.  A request's inputs are page-locked host tensors (prepare_host, before
the run), copied to the device when the job is admitted.  Host-side
marshalling only; all arithmetic runs in librix.so.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np
import torch

from . import pipeline, rix


@dataclasses.dataclass
class Request:
    rid: int
    obs: object                       # synth.Observation (host arrays)
    method: pipeline.Method
    n_major: int
    arrival: float = 0.0              # seconds after the start of the run
    n_part: int = 2
    precision: int = rix.FP32
    kind: str = ""                    # label of the request's workload (summaries per kind)
    # filled in by the server
    t_admit: float = float("nan")
    t_done: float = float("nan")
    image: np.ndarray | None = None
    samples: int = 0                  # visibility samples gridded+degridded over all cycles

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


# page-locked host inputs per (observation, precision): uvw, vis, weight
_HOST: dict = {}


def host_inputs(obs, precision: int):
    """The observation's inputs as page-locked host tensors in the job's
    visibility type (made once per observation and precision)."""
    key = (id(obs), precision)
    if key not in _HOST:
        vdt = np.complex128 if precision == rix.FP64 else np.complex64
        _HOST[key] = (obs,   # keeps id(obs) valid while cached
                      torch.from_numpy(np.ascontiguousarray(obs.uvw, dtype=np.float64)).pin_memory(),
                      torch.from_numpy(np.ascontiguousarray(obs.vis.reshape(obs.nrow, obs.nchan), dtype=vdt)).pin_memory(),
                      torch.from_numpy(np.ascontiguousarray(obs.weight, dtype=np.float32)).pin_memory())
    return _HOST[key][1:]


def prepare_host(requests):
    for q in requests:
        host_inputs(q.obs, q.precision)


def clear_host():
    _HOST.clear()


class _Run:
    def __init__(self, ctx, req: Request, stream: torch.cuda.Stream):
        self.req = req
        self.stream = stream
        o = req.obs
        self.rec = pipeline.Reconstruction(ctx, o.n, o.cell_rad, o.n_wplanes, o.freq, o.nrow, req.n_part,
                                           req.precision)
        self.stage = 0
        self.done_event = None
        self.out_host = None

    def issue_next(self):
        r, o, st = self.req, self.req.obs, self.stream
        with torch.cuda.stream(st):
            if self.stage == 0:
                h_uvw, h_vis, h_w = host_inputs(o, r.precision)
                uvw = h_uvw.to("cuda", non_blocking=True)
                vis = h_vis.to("cuda", non_blocking=True)
                w = h_w.to("cuda", non_blocking=True)
                self.rec.uvw, self.rec.vis, self.rec.weight = uvw, vis, w
                rix.set_uv_partition(self.rec.job, uvw, w, None, 1.0, None, st)
                s = rix.job_get_stats(self.rec.job)
                r.samples = r.n_major * int(sum(s["part_count"][:r.n_part]))
            elif self.stage <= r.n_major:
                self.rec.cycle(r.method, st)
            else:
                img = self.rec.combine(stream=st)
                self.out_host = torch.empty(img.shape, dtype=img.dtype).pin_memory()
                self.out_host.copy_(img, non_blocking=True)
                self.done_event = torch.cuda.Event()
                self.done_event.record(st)
        self.stage += 1

    @property
    def all_issued(self) -> bool:
        return self.done_event is not None

    def close(self):
        self.rec.close()


def serve(ctx, requests: list[Request], n_slots: int = 4, poll_s: float = 2e-4, mem_probe=None):
    """Runs the requests; returns them with timings and images filled in.
    `mem_probe` (optional) is called about every 10 ms of the run (e.g. to
    record the device memory in use)."""
    streams = [torch.cuda.Stream() for _ in range(n_slots)]
    free = collections.deque(range(n_slots))
    pending = collections.deque(sorted(requests, key=lambda q: q.arrival))
    active: list[tuple[_Run, int]] = []
    t0 = time.perf_counter()
    t_probe = -1.0
    while pending or active:
        now = time.perf_counter() - t0
        if mem_probe is not None and now - t_probe >= 0.01:
            mem_probe()
            t_probe = now
        while pending and pending[0].arrival <= now and free:
            req = pending[0]
            slot = free[0]
            try:
                run = _Run(ctx, req, streams[slot])
            except rix.RixError as e:
                if e.code == rix.ENOMEM and active:
                    break                      # wait for memory to free up
                raise
            pending.popleft()
            free.popleft()
            req.t_admit = time.perf_counter() - t0
            active.append((run, slot))
        progressed = False
        for item in list(active):
            run, slot = item
            if run.all_issued:
                if run.done_event.query():
                    run.req.t_done = time.perf_counter() - t0
                    run.req.image = run.out_host.numpy().copy()
                    run.close()
                    active.remove(item)
                    free.append(slot)
                    progressed = True
            else:
                run.issue_next()
                progressed = True
        if not progressed:
            time.sleep(poll_s)
    return requests


def poisson_arrivals(rng: np.random.Generator, n: int, rate_per_s: float) -> np.ndarray:
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))


def summary(reqs: list[Request]) -> dict:
    """Latency percentiles, offered and achieved rates and visibility
    throughput of a finished run, overall and per request kind."""
    lat = np.array([q.latency for q in reqs])
    span = max(q.t_done for q in reqs) - min(q.arrival for q in reqs)
    arr = np.sort(np.array([q.arrival for q in reqs]))
    samples = sum(q.samples for q in reqs)
    out = {"jobs": len(reqs), "p50_latency_s": float(np.percentile(lat, 50)),
           "p99_latency_s": float(np.percentile(lat, 99)), "max_latency_s": float(lat.max()),
           "makespan_s": float(span),
           "offered_jobs_per_s": (len(reqs) / float(arr[-1] - arr[0])) if len(reqs) > 1 and arr[-1] > arr[0] else None,
           "achieved_jobs_per_s": len(reqs) / span, "mvis_per_s": samples / span / 1e6,
           "queue_wait_p50_s": float(np.percentile([q.t_admit - q.arrival for q in reqs], 50))}
    kinds = sorted({q.kind for q in reqs if q.kind})
    if kinds:
        per = {}
        for k in kinds:
            lk = np.array([q.latency for q in reqs if q.kind == k])
            per[k] = {"jobs": int(lk.size), "p50_latency_s": float(np.percentile(lk, 50)),
                      "p99_latency_s": float(np.percentile(lk, 99)),
                      "samples": int(sum(q.samples for q in reqs if q.kind == k))}
        out["per_kind"] = per
    return out
