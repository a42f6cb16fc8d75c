"""Host driver of the decentralized major/minor loop (Sec. 3, Fig. 2).

Marshalling only: it uploads an observation, creates one rix job with its uv
partitions and issues, per major cycle, the major cycle of every partition,
then the minor cycle of every partition, and finally the combine.  All
arithmetic runs in librix.so.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import rix


@dataclasses.dataclass
class Method:
    kind: str = "msclean"                 # "msclean" or "fista"
    scales: tuple = (0.0, 3.0, 9.0)
    gain: float = 0.1
    niter: int = 2000
    threshold: float = 1e-4
    lam: float = 0.0
    lam_rel: float = 1e-3
    iters: int = 50
    levels: int = 4
    dictionary: str = "db4"               # "db4" or "db1-8" (the paper's concatenation, Sec. 5.2)
    schedule: tuple | None = None         # (a, b): lambda_n = a ||residual_n||_2 b^n


class Reconstruction:
    """One job on one device; partitions run on the caller's stream."""

    def __init__(self, ctx, n, cell_rad, n_wplanes, freq, nrow, n_part=2, precision=rix.FP32, tile=0,
                 device="cuda", weighting=rix.WEIGHT_NATURAL, exchange=rix.EXCHANGE_IMAGE):
        self.ctx = ctx
        self.n = n
        self.cell_rad = cell_rad
        self.n_wplanes = n_wplanes
        self.freq = list(freq)
        self.n_part = n_part
        self.precision = precision
        self.rdtype = torch.float64 if precision == rix.FP64 else torch.float32
        self.cdtype = torch.complex128 if precision == rix.FP64 else torch.complex64
        self.device = torch.device(device)
        self.job = rix.job_create(ctx, n, cell_rad, n_wplanes, list(freq), precision, n_part, nrow, tile, weighting,
                                  exchange)
        self.vis = None

    def close(self):
        if self.job:
            rix.job_destroy(self.job)
            self.job = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_data(self, uvw, vis, weight=None, ell_px=None, delta_px=1.0, stream=None):
        """uvw: (nrow, 3) float64; vis: (nrow, nchan) complex; device tensors or
        numpy arrays (copied to the device)."""
        dev = self.device
        self.uvw = torch.as_tensor(uvw, dtype=torch.float64, device=dev).contiguous()
        self.vis = torch.as_tensor(vis, device=dev).to(self.cdtype).contiguous()
        self.weight = None if weight is None else torch.as_tensor(weight, dtype=torch.float32,
                                                                  device=dev).contiguous()
        rix.set_uv_partition(self.job, self.uvw, self.weight, ell_px, delta_px, None, stream)

    def stats(self) -> dict:
        return rix.job_get_stats(self.job)

    def major(self, p, residual_out=None, stream=None):
        rix.major_cycle(self.job, p, self.vis, None, residual_out, stream)

    def minor(self, p, m: Method, delta_out=None, stream=None):
        if m.kind == "msclean":
            rix.minor_cycle_msclean(self.job, p, m.scales, m.gain, m.niter, m.threshold, delta_out, stream)
        else:
            d = rix.DICT_DB4 if m.dictionary == "db4" else rix.DICT_DB1_8
            rix.minor_cycle_fista(self.job, p, m.lam, m.lam_rel, m.iters, m.levels, delta_out, stream, d,
                                  m.schedule)

    def cycle(self, m: Method, stream=None, concurrent: bool = True, batch: bool = True):
        """One major cycle of every partition, then the minor cycles.  With
        `concurrent`, each partition's major cycle runs on its own stream (the
        partitions are concurrent instances on the device; the library orders
        the exchange between them with events); the minor cycles follow on the
        partitions' streams, or with `batch` the FISTA ones as one batched loop
        launch on `stream`; `stream` waits for them."""
        if not concurrent or self.n_part == 1:
            for p in range(self.n_part):
                self.major(p, stream=stream)
            for p in range(self.n_part):
                self.minor(p, m, stream=stream)
            return
        main = torch.cuda.current_stream(self.device) if stream is None else stream
        if not hasattr(self, "_pstreams"):
            self._pstreams = [torch.cuda.Stream(self.device) for _ in range(self.n_part)]
        start = torch.cuda.Event()
        start.record(main)
        for p, s in enumerate(self._pstreams):
            s.wait_event(start)
            self.major(p, stream=s)
        if batch and m.kind == "fista":
            # FISTA minor cycles of all partitions: one batched loop launch
            # (the library orders it after each partition's major cycle)
            self.minor_all(m, main)
            return
        for p, s in enumerate(self._pstreams):
            self.minor(p, m, stream=s)
        for s in self._pstreams:
            ev = torch.cuda.Event()
            ev.record(s)
            main.wait_event(ev)

    def minor_all(self, m: Method, stream):
        """The minor cycles of every partition on `stream`: FISTA as one batched
        loop launch (rix_minor_cycle_fista_batch), ms-CLEAN one call each."""
        if m.kind == "fista" and self.n_part > 1:
            d = rix.DICT_DB4 if m.dictionary == "db4" else rix.DICT_DB1_8
            rix.minor_cycle_fista_batch(self.job, list(range(self.n_part)), m.lam, m.lam_rel, m.iters, m.levels,
                                        stream, d, m.schedule)
        else:
            for p in range(self.n_part):
                self.minor(p, m, stream=stream)

    def cycles(self, m: Method, n_major: int, stream=None, batch: bool = True):
        """`n_major` major+minor cycles with each partition's major cycle on its
        own stream and no join between cycles: a partition starts its next major
        cycle as soon as its own minor cycle is done, while the library's events
        order the exchange with the other partitions.  With `batch`, FISTA minor
        cycles of a cycle run together (one loop launch for all partitions) on
        the first partition's stream; the library starts each partition's
        preparation as soon as that partition's major cycle is done and runs
        the loops as one dataflow-scheduled launch (the default).  Without it
        every minor cycle runs on its partition's stream.  `stream`
        waits for all."""
        if self.n_part == 1:
            for _ in range(n_major):
                self.cycle(m, stream)
            return
        main = torch.cuda.current_stream(self.device) if stream is None else stream
        if not hasattr(self, "_pstreams"):
            self._pstreams = [torch.cuda.Stream(self.device) for _ in range(self.n_part)]
        start = torch.cuda.Event()
        start.record(main)
        for s in self._pstreams:
            s.wait_event(start)
        for _ in range(n_major):
            for p, s in enumerate(self._pstreams):
                self.major(p, stream=s)
            if batch and m.kind == "fista":
                self.minor_all(m, self._pstreams[0])
            else:
                for p, s in enumerate(self._pstreams):
                    self.minor(p, m, stream=s)
        for s in self._pstreams:
            ev = torch.cuda.Event()
            ev.record(s)
            main.wait_event(ev)

    def combine(self, out=None, stream=None):
        if out is None:
            out = torch.empty((self.n, self.n), dtype=self.rdtype, device=self.device)
        rix.combine(self.job, out, stream)
        return out

    def run(self, m: Method, n_major: int, stream=None):
        self.cycles(m, n_major, stream)
        return self.combine(stream=stream)


class BatchedMajor:
    """The major cycles of every partition of several FP32 w-stacked
    reconstructions with one gridder launch (rix_batch_*), issued directly
    or replayed from a captured CUDA graph.  Marshalling only."""

    def __init__(self, ctx, recs):
        self.recs = list(recs)
        self.pairs = [(r, p) for r in self.recs for p in range(r.n_part)]
        self.batch = rix.batch_create(ctx, [r.job for r, _ in self.pairs], [p for _, p in self.pairs])
        self.graph = None

    def close(self):
        if self.batch:
            rix.batch_destroy(self.batch)
            self.batch = None
        self.graph = None

    def samples(self) -> int:
        return sum(r.stats()["part_count"][p] for r, p in self.pairs)

    def run(self, stream=None, residual_out=None):
        rix.batch_major_cycle(self.batch, [r.vis.reshape(-1) for r, _ in self.pairs], residual_out, stream)

    def capture(self, stream, residual_out=None):
        """Capture one batched major cycle (after an uncaptured one has run:
        the pairs' buffers exist) into a CUDA graph on `stream`."""
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            self.run(stream, residual_out)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()


def observation_job(ctx, obs, n_part=2, precision=rix.FP32, tile=0, ell_px=None, delta_px=1.0,
                    weighting=rix.WEIGHT_NATURAL, exchange=rix.EXCHANGE_IMAGE):
    """Reconstruction set up from a synth.Observation."""
    r = Reconstruction(ctx, obs.n, obs.cell_rad, obs.n_wplanes, obs.freq, obs.nrow, n_part, precision, tile,
                       weighting=weighting, exchange=exchange)
    r.set_data(obs.uvw, obs.vis, obs.weight, ell_px, delta_px)
    return r
