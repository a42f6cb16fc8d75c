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
image.  Host-side marshalling only; all arithmetic runs in librix.so.
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
    # filled in by the server
    t_admit: float = float("nan")
    t_done: float = float("nan")
    image: np.ndarray | None = None
    samples: int = 0                  # visibility samples gridded+degridded over all cycles

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


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
                cdt = torch.complex128 if r.precision == rix.FP64 else torch.complex64
                uvw = torch.from_numpy(o.uvw).pin_memory().to("cuda", non_blocking=True)
                vis = torch.from_numpy(o.vis.reshape(o.nrow, o.nchan).astype(
                    np.complex128 if r.precision == rix.FP64 else np.complex64)).pin_memory().to(
                    "cuda", non_blocking=True)
                w = torch.from_numpy(o.weight).pin_memory().to("cuda", non_blocking=True)
                self.rec.uvw, self.rec.vis, self.rec.weight = uvw, vis.to(cdt), w
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


def serve(ctx, requests: list[Request], n_slots: int = 4, poll_s: float = 2e-4):
    """Runs the requests; returns them with timings and images filled in."""
    streams = [torch.cuda.Stream() for _ in range(n_slots)]
    free = collections.deque(range(n_slots))
    pending = collections.deque(sorted(requests, key=lambda q: q.arrival))
    active: list[tuple[_Run, int]] = []
    t0 = time.perf_counter()
    while pending or active:
        now = time.perf_counter() - t0
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
    lat = np.array([q.latency for q in reqs])
    span = max(q.t_done for q in reqs) - min(q.arrival for q in reqs)
    samples = sum(q.samples for q in reqs)
    return {"jobs": len(reqs), "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "makespan_s": float(span),
            "achieved_jobs_per_s": len(reqs) / span, "mvis_per_s": samples / span / 1e6}
