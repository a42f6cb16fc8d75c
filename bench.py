#!/usr/bin/env python
"""Throughput benchmark of the decentralized reconstruction path on GB300.

A step is one whole reconstruction job of the medium workload (1024 x 1024,
1" cells, 64 antennas x 1000 times x 4 channels = 8.06 M visibilities, 16
w-planes, 2 uv partitions, FISTA with Db4, lambda = 1e-3 max|dirty|, 50
iterations, 10 major cycles, FP32): partition + sort (a1-a3), PSF (a7), ten
major cycles of both partitions (a4-a6), the fill and FISTA minor cycles
(a8, a10) and the combine (a11).  The metric is grid+degrid Mvis/s: the
visibility samples the major cycles processed (overlap counted in each
partition, ten cycles) per second of step time.  Inputs are resident in HBM
for `value`; `e2e` adds the host->device copy of the inputs from pinned
memory and the device->host read of the final image.

Multi-GPU: independent replicas (one job per rank, no collective).
"""
from __future__ import annotations

import argparse
import collections
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "grid+degrid Mvis/s"
UNIT = "Mvis/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-times", type=int, default=1000, help="time samples (1000 = the full workload)")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--cycles", type=int, default=10)
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--fp64", action="store_true", help="FP64 operator (comparator)")
    ap.add_argument("--no-batch-minor", action="store_true",
                    help="run each partition's FISTA minor cycle as its own loop launch instead of one batched launch")
    ap.add_argument("--dictionary", default="db4", choices=["db4", "db1-8"],
                    help="FISTA dictionary: Db4 alone, or the concatenation of db1..db8")
    ap.add_argument("--method", default="fista", choices=["fista", "msclean"],
                    help="minor cycle of the medium workload: FISTA (the benchmark) or multi-scale CLEAN")
    ap.add_argument("--scales", default="0,4,16", help="ms-CLEAN scale radii in pixels")
    ap.add_argument("--clean-iters", type=int, default=2000, help="ms-CLEAN iterations per minor cycle")
    ap.add_argument("--schedule", default=None,
                    help="a,b: lambda_n = a ||residual_n||_2 b^n instead of 1e-3 max |residual_1|")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-phases", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 operator comparison")
    ap.add_argument("--job-only", action="store_true",
                    help="time the jobs only: no major-cycle metric, roofline, error, FP64 or cuFFT measurement "
                         "(for launch lists and profiles)")
    ap.add_argument("--serve-jobs", type=int, default=24, help="arrivals in the serving experiment (0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=20.0, help="Poisson arrival rate, jobs/s")
    ap.add_argument("--json-out", default=None)
    ap.add_argument("--workload", default="medium", choices=["medium", "batch", "large", "serve"],
                    help="medium: the whole-job benchmark; batch: the batching workload's batched major cycle; "
                         "large: the 4096^2 workload's major cycle; serve: the serving workload (Poisson "
                         "arrivals of the recipe mix under a memory budget)")
    ap.add_argument("--serve-budget-gb", type=float, default=150.0, help="device-memory budget of the serving runs")
    ap.add_argument("--serve-slots", type=int, default=16, help="streams (concurrent jobs at most) when serving")
    ap.add_argument("--serve-compare-jobs", type=int, default=100,
                    help="arrivals of the sustained-rate run and of the FP32-vs-FP64 runs (0 = skip them)")
    ap.add_argument("--parts", type=int, default=2, help="uv partitions of the large workload (2 or 4)")
    ap.add_argument("--batch-jobs", type=int, default=64)
    return ap.parse_args()


def max_over_ranks(x: float, device) -> float:
    """The largest x over all ranks of the process group (x itself without
    one): the timed region ends when the slowest rank does."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: float, world: int, ms_per_step: float) -> float:
    """Mvis/s of the whole job: every rank processes units_per_rank per step
    (weak scaling), divided by the slowest rank's time."""
    return units_per_rank * world / (ms_per_step * 1e-3) / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
            return self
        # nvidia-smi's start-up (NVML initialisation) runs before the timed
        # steps, not inside them: wait for its first sample
        t0 = time.time()
        while not self.lines and self.proc.poll() is None and time.time() - t0 < 10.0:
            time.sleep(0.02)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def flush_l2(buf):
    buf.add_(1.0)   # a write of 512 MiB, larger than the 129 MB L2


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# --------------------------------------------------------------------------
def reference_arm(a, rank, world):
    """The oracle as it stands, on the host cores, on a bounded sample of the
    same workload (one major cycle of one partition over a row subset)."""
    if rank != 0:
        return 0
    res = cpu_baseline(a, a.steps, a.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": res["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(a),
            "cpu_baseline": {"value": res["value"], "unit": UNIT, "cores": res["cores"], "kind": "oracle",
                             "sample": res["sample"], "cpu": res["cpu"], "nproc": res["nproc"]},
            "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _oracle_init(barrier):
    global _ORACLE_BARRIER
    _ORACLE_BARRIER = barrier


def _oracle_major_cycle(job):
    """One FP64 oracle major cycle (degrid + residual + grid, Eq. 2) of
    partition 0 on a row subset of the medium recipe; runs in a spawned
    process with one FFT thread.  Returns (samples, seconds)."""
    n_times, n, repeats = job
    from oracle import filters, gridder, partition
    filters.FFT_WORKERS = 1
    gridder.FFT_WORKERS = 1
    from paper_2507_22128_gb300 import synth
    obs = synth.medium(seed=1, n_times=n_times, n=n)
    g = gridder.geometry(obs.uvw, obs.freq, obs.n, obs.cell_rad, W=8, nw=obs.n_wplanes)
    r = partition.radius_px(g)
    m = partition.masks(r, partition.ring_radii(r, 2), 1.0, 2, g.inside)
    gp = gridder.subset(g, (m & 1) == 1)
    w = obs.weight.reshape(-1).astype(np.float64)
    model = np.zeros((obs.n, obs.n))
    out = []
    for _ in range(repeats):
        _ORACLE_BARRIER.wait()          # every process starts its cycle together
        t0 = time.perf_counter()
        gridder.residual(obs.vis.reshape(-1), w, model, gp)
        out.append(time.perf_counter() - t0)
    return int(gp.inside.sum()), out


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(a, steps=1, warmup=0):
    """The oracle on all host cores: one spawned process per core (bounded by
    host memory, about 4 GB per process at 1024^2 with 16 w-planes), each
    running the oracle's FP64 major cycle of partition 0 over 1/64 of the
    workload's time samples with one FFT thread, all started together;
    Mvis/s = the processes' samples / the slowest process's time (median
    over `steps` rounds after `warmup`)."""
    import multiprocessing as mp
    ncpu = os.cpu_count() or 1
    try:
        with open("/proc/meminfo") as f:
            avail_gb = next(int(ln.split()[1]) for ln in f if ln.startswith("MemAvailable")) / 2 ** 20
    except (OSError, StopIteration):
        avail_gb = 16.0
    nproc = max(1, min(ncpu, int(avail_gb // 4)))
    n_times = max(4, a.n_times // 64)
    ctx = mp.get_context("spawn")           # the parent holds a CUDA context: never fork it
    barrier = ctx.Barrier(nproc)
    with ctx.Pool(nproc, initializer=_oracle_init, initargs=(barrier,)) as pool:
        res = pool.map(_oracle_major_cycle, [(n_times, a.n, warmup + steps)] * nproc)
    nsamp = sum(r[0] for r in res)
    rounds = [max(r[1][i] for r in res) for i in range(warmup, warmup + steps)]
    t = statistics.median(rounds)
    return {"value": nsamp / t / 1e6, "ms_per_step": t * 1e3, "cores": nproc, "cpu": cpu_model(),
            "nproc": ncpu,
            "sample": f"{nproc} processes (one per host core, {ncpu} cores, {cpu_model()}), each one FP64 oracle "
                      f"major cycle of partition 0 over {n_times} of the {a.n_times} time samples x 4 channels "
                      f"({res[0][0]} samples each, 1/64 of the {a.n}^2 workload's rows; numpy, one FFT thread "
                      f"per process), started together; median of {steps} rounds"}


def config_dict(a):
    if a.method == "msclean":
        minor = f"ms-CLEAN scales {{{a.scales}}} gain 0.1 {a.clean_iters} it"
    else:
        minor = (f"FISTA {'Db4' if a.dictionary == 'db4' else 'db1..db8'} "
                 f"{a.iters} it{'' if a.schedule is None else ', lambda schedule ' + a.schedule}")
    return {"workload": f"medium: {a.n}x{a.n} 1as, 64 ant log-spiral x {a.n_times} times x 4 ch "
                        f"(1.3-1.5 GHz), 16 w-planes, 2 uv partitions, {minor}, "
                        f"{a.cycles} major cycles",
            "n": a.n, "n_wplanes": 16, "n_part": 2, "major_cycles": a.cycles, "minor_cycle": a.method,
            **({"clean_scales": a.scales, "clean_iters": a.clean_iters} if a.method == "msclean" else
               {"fista_iters": a.iters, "fista_dictionary": a.dictionary, "fista_batched": not a.no_batch_minor}),
            "l2": "flushed between steps (512 MiB write)", "precision": "fp64" if a.fp64 else "fp32"}


def main():
    a = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if a.impl == "ours" else "gloo")
    if a.impl == "reference":
        return reference_arm(a, rank, world)
    if a.workload == "batch":
        return batch_workload(a, rank, world, local)
    if a.workload == "large":
        return large_workload(a, rank, world, local)
    if a.workload == "serve":
        return serve_workload(a, rank, world, local)

    from paper_2507_22128_gb300 import pipeline, rix, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    obs = synth.medium(seed=1 + rank, n_times=a.n_times, n=a.n)
    prec = rix.FP64 if a.fp64 else rix.FP32
    cdt = torch.complex128 if a.fp64 else torch.complex64
    rdt = torch.float64 if a.fp64 else torch.float32
    uvw_h = torch.from_numpy(obs.uvw).pin_memory()
    vis_h = torch.from_numpy(obs.vis.astype(np.complex128 if a.fp64 else np.complex64)).pin_memory()
    w_h = torch.from_numpy(obs.weight).pin_memory()
    uvw_d = uvw_h.to(dev)
    vis_d = vis_h.to(dev)
    w_d = w_h.to(dev)
    img_h = torch.empty((obs.n, obs.n), dtype=rdt).pin_memory()
    ctx = rix.create(local)
    rec = pipeline.Reconstruction(ctx, obs.n, obs.cell_rad, obs.n_wplanes, obs.freq, obs.nrow, 2, prec)
    sched = None if a.schedule is None else tuple(float(v) for v in a.schedule.split(","))
    if a.method == "msclean":
        meth = pipeline.Method("msclean", tuple(float(v) for v in a.scales.split(",")), 0.1, a.clean_iters, 1e-4)
    else:
        meth = pipeline.Method("fista", lam_rel=1e-3, iters=a.iters, levels=4, dictionary=a.dictionary,
                               schedule=sched)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)
    out = torch.empty((obs.n, obs.n), dtype=rdt, device=dev)

    def one_job(uvw, vis, w):
        rec.uvw, rec.vis, rec.weight = uvw, vis, w
        rix.set_uv_partition(rec.job, uvw, w, None, 1.0, None, stream)
        rec.cycles(meth, a.cycles, stream, batch=not a.no_batch_minor)
        rix.combine(rec.job, out, stream)

    for _ in range(max(a.warmup, 1)):
        one_job(uvw_d, vis_d, w_d)
    torch.cuda.synchronize()
    st = rix.job_get_stats(rec.job)
    units = a.cycles * sum(st["part_count"][:2])

    # ---- timed steps: device-resident inputs ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    rix.timing_read(rix.TIME_TILES)
    rix.timing_read(rix.TIME_FFT)
    rix.timing_read(rix.TIME_MINOR_LOOP)
    rix.timing_enable(True)
    launches0 = rix.kernel_launches()
    with ClockSampler(local) as clk:
        for i in range(a.steps):
            flush_l2(flush)
            ev[i][0].record(stream)
            one_job(uvw_d, vis_d, w_d)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    launches = rix.kernel_launches() - launches0
    rix.timing_enable(False)
    tiles_ms, tiles_busy, tiles_n = rix.timing_read(rix.TIME_TILES)
    fft_ms, fft_busy, fft_n = rix.timing_read(rix.TIME_FFT)
    loop_ms, loop_busy, loop_n = rix.timing_read(rix.TIME_MINOR_LOOP)
    if world > 1:
        torch.distributed.barrier()
    step_ms = [s.elapsed_time(e) for s, e in ev]
    total_ms = max_over_ranks(sum(step_ms), dev)
    ms = total_ms / a.steps
    value = whole_job_value(units, world, ms)

    # ---- per-phase split of one job (diagnostic) ----
    phases = None if a.no_phases else phase_split(rec, rix, a, meth, stream, uvw_d, vis_d, w_d, out, flush)

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if not a.no_e2e:
        ts = []
        for i in range(max(2, min(a.steps, 3))):
            flush_l2(flush)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            uvw_x = uvw_h.to(dev, non_blocking=True)
            vis_x = vis_h.to(dev, non_blocking=True)
            w_x = w_h.to(dev, non_blocking=True)
            one_job(uvw_x, vis_x, w_x)
            img_h.copy_(out, non_blocking=True)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        t = statistics.median(ts)
        e2e = {"value": units / t / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(uvw_h.numel() * 8 + vis_h.numel() * vis_h.element_size() + w_h.numel() * 4),
               "d2h_bytes_per_step": int(img_h.numel() * img_h.element_size())}

    # ---- the survey's major-cycle metric, the gridder's roofline, the
    # stated error, the FP64 comparator and cuFFT ----
    mc = roof = err = fp64 = cufft = None
    if not a.job_only:
        mc = major_cycle_metric(rec, rix, meth, stream, vis_d, flush, st, obs.nchan)
        roof = roofline_gridder(mc, st, a)
        err = direct_dft_errors(rec, rix, obs, out, vis_d, w_d, 1)
        fp64 = None if (a.fp64 or a.no_fp64) else fp64_comparator(ctx, rix, pipeline, obs, a, flush)
        cufft = cufft_comparison(obs.n, obs.n_wplanes, st["window_size"][:2], flush)
        cufft["library_fft_ms_per_cycle"] = sum(mc["per_partition_serial"][p]["fft_ms"] for p in (0, 1))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if a.fp64 else "f32", "data": "synthetic",
            "config": config_dict(a), "clocks": clk.summary(), "e2e": e2e, "gpu_launches": int(launches),
            "roofline": roof, "major_cycle": mc, "operator_error": err, "fp64_operator": fp64, "cufft": cufft,
            "phases_ms": phases,
            "kernel_ms_per_step": {"grid_tiles_busy": tiles_busy / a.steps, "grid_tiles_sum": tiles_ms / a.steps,
                                   "fft_passes_busy": fft_busy / a.steps,
                                   "minor_loop_busy": loop_busy / a.steps, "minor_loop_sum": loop_ms / a.steps},
            "samples_per_cycle": int(sum(st["part_count"][:2])), "step_ms": step_ms}
    if a.serve_jobs > 0:
        line["serving"] = serving_experiment(ctx, a, rank)
    if rank == 0 and not a.no_cpu_baseline:
        cb = cpu_baseline(a)
        line["cpu_baseline"] = {"value": cb["value"], "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                                "sample": cb["sample"], "cpu": cb["cpu"], "nproc": cb["nproc"]}
    rec.close()
    rix.destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
        if a.json_out:
            with open(a.json_out, "w") as f:
                json.dump(line, f, indent=1)
    return 0


def batch_workload(a, rank, world, local):
    """The batching workload: n independent channel-chunk jobs (the medium
    recipe's generator per job, visibility counts log-uniform in 0.5-8 M,
    image sides from {256, 512, 1024, 2048}, 2 partitions each, FP32),
    every partition's degrid/residual/grid in one persistent gridder launch
    per major cycle, the cycle captured in a CUDA graph and replayed; the
    gridder's tuning per job shape from the autotuner's cache.  Visibilities
    are seeded complex Gaussian values drawn on the device (the operator's
    cost does not depend on them).  Compared with the same pairs as one
    batch each (one gridder launch per partition), also replayed from a
    graph."""
    from paper_2507_22128_gb300 import autotune, pipeline, rix, synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    obs_list = synth.batch_chunk_jobs(n_jobs=a.batch_jobs, base_seed=1000 + 1000 * rank, with_vis=False)
    ctx = rix.create(local)
    gen = torch.Generator(device=dev).manual_seed(1000 + rank)
    recs = []
    t0 = time.perf_counter()
    for o in obs_list:
        rec = pipeline.Reconstruction(ctx, o.n, o.cell_rad, o.n_wplanes, o.freq, o.nrow, 2, rix.FP32)
        vis = torch.complex(torch.randn(o.nvis, generator=gen, device=dev),
                            torch.randn(o.nvis, generator=gen, device=dev)).reshape(o.nrow, o.nchan)
        rec.set_data(o.uvw, vis, o.weight)
        recs.append(rec)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    cache = autotune.default_cache_path()
    tuned = [autotune.tune(r, r.vis.reshape(-1), cache) for r in recs]
    m = pipeline.Method("fista", lam_rel=1e-3, iters=1, levels=1)
    s = torch.cuda.Stream(dev)
    bm = pipeline.BatchedMajor(ctx, recs)
    singles = [pipeline.BatchedMajor.__new__(pipeline.BatchedMajor) for _ in bm.pairs]
    for sb, (r, p) in zip(singles, bm.pairs):
        sb.recs, sb.pairs, sb.graph = [r], [(r, p)], None
        sb.batch = rix.batch_create(ctx, [r.job], [p])
    units = bm.samples()
    with torch.cuda.stream(s):
        bm.run(s)                              # cycle 1, issued directly
        for r in recs:
            r.minor_all(m, s)
    torch.cuda.synchronize()
    g_b = bm.capture(s)                        # cycle 2: one gridder launch for all pairs
    g_s = torch.cuda.CUDAGraph()               # cycle 2: one gridder launch per pair
    with torch.cuda.graph(g_s, stream=s):
        for sb in singles:
            sb.run(s)

    def replay_ms(graph, reps):
        for _ in range(max(a.warmup, 1)):
            graph.replay()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            with torch.cuda.stream(s):
                graph.replay()
            e1.record(s)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), ts

    launches0 = rix.kernel_launches()
    with ClockSampler(local) as clk:
        ms_b, ts_b = replay_ms(g_b, a.steps)
        ms_s, _ = replay_ms(g_s, a.steps)
    launches = rix.kernel_launches() - launches0
    ms_b = max_over_ranks(ms_b, dev)
    value = whole_job_value(units, world, ms_b)
    shapes = collections.Counter(o.n for o in obs_list)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms_b, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (uvw of the medium recipe per job; seeded Gaussian visibilities)",
            "config": {"workload": f"batching: {len(obs_list)} channel-chunk jobs, 0.5-8 M visibilities each "
                                   f"(log-uniform), image sides {dict(sorted(shapes.items()))}, 16 w-planes, "
                                   f"2 uv partitions each; one batched major cycle per step, replayed from a "
                                   f"CUDA graph", "jobs": len(obs_list), "pairs": len(bm.pairs),
                       "samples_per_cycle": int(units), "l2": "inputs larger than L2 (5+ GB of entries)"},
            "clocks": clk.summary(), "gpu_launches": "graph replays (the library counts launches at capture)",
            "per_pair_graph": {"ms_per_cycle": ms_s, "value": units / (ms_s * 1e-3) / 1e6,
                               "note": "the same pairs, one gridder launch per partition, replayed from a graph"},
            "step_ms": ts_b, "setup_s": setup_s,
            "autotune": {"cache": cache,
                         "choices": dict(collections.Counter(f"{t['chunk_limit']}/{t['ctas_per_sm']}" for t in tuned)),
                         "tuned_now": sum(1 for t in tuned if not t["cached"])}}
    for sb in singles:
        sb.close()
    bm.close()
    for r in recs:
        r.close()
    rix.destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
        if a.json_out:
            with open(a.json_out, "w") as f:
                json.dump(line, f, indent=1)
    return 0


def large_workload(a, rank, world, local):
    """The large workload: 4096 x 4096 at 0.5", 128 antennas on a 10 km log
    spiral x 4000 times x 8 channels (1.3-1.5 GHz) = 260 M visibilities, 32
    w-planes, `--parts` uv partitions, FP32: partition and sort, then the
    fused major-cycle operator of every partition timed by
    rix_major_cycle_probe (its device time on the current model; the
    partitions one after another, so the cycle time is their sum).
    Visibilities are seeded complex Gaussian values drawn on the device (the
    operator's cost does not depend on them; analytic visibilities of 2100
    sources at 260 M samples take far longer to generate than to image)."""
    from paper_2507_22128_gb300 import pipeline, rix, synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    obs = synth.large(seed=3 + rank, with_vis=False)
    gen_s = time.perf_counter() - t0
    ctx = rix.create(local)
    P = a.parts
    rec = pipeline.Reconstruction(ctx, obs.n, obs.cell_rad, obs.n_wplanes, obs.freq, obs.nrow, P, rix.FP32)
    gen = torch.Generator(device=dev).manual_seed(3 + rank)
    vis = torch.complex(torch.randn(obs.nvis, generator=gen, device=dev),
                        torch.randn(obs.nvis, generator=gen, device=dev)).reshape(obs.nrow, obs.nchan)
    s = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    rec.set_data(obs.uvw, vis, obs.weight, stream=s)
    e1.record(s)
    torch.cuda.synchronize()
    part_ms = e0.elapsed_time(e1)
    st = rec.stats()
    flat = rec.vis.reshape(-1)
    with ClockSampler(local) as clk:
        per = {}
        for p in range(P):
            per[p] = {"major_cycle_ms": rix.major_cycle_probe(rec.job, p, flat, max(a.steps, 3)),
                      "gridder_ms": rix.gridder_probe(rec.job, p, flat, max(a.steps, 3)),
                      "entries": int(st["part_count"][p]), "window": int(st["window_size"][p])}
    units = sum(st["part_count"][:P])
    ms = max_over_ranks(sum(per[p]["major_cycle_ms"] for p in range(P)), dev)
    peaks, kind = measured_peaks()
    ng = 2 * obs.n
    byt = units * (24.0 / obs.nchan + 16.0) + P * obs.n_wplanes * 8 * ng * ng * 8.0
    mc = {"value": units / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_cycle": ms, "samples_per_cycle": int(units),
          "cycles_timed": max(a.steps, 3),
          "timing": "rix_major_cycle_probe per partition (one after another: the sum), mean of the timed runs",
          "hbm": {"algorithmic_bytes_per_cycle": byt, "achieved_gbs": byt / (ms * 1e-3) / 1e9,
                  "peak_gbs": float(peaks["hbm_gbs"]), "frac": byt / (ms * 1e-3) / 1e9 / float(peaks["hbm_gbs"]),
                  "peak_source": kind},
          "per_partition": per}
    value = whole_job_value(mc["samples_per_cycle"], world, mc["ms_per_cycle"])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": mc["cycles_timed"],
            "warmup": 1, "ms_per_step": mc["ms_per_cycle"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (uvw of the large recipe; seeded Gaussian visibilities)",
            "config": {"workload": f"large: 4096x4096 0.5as, 128 ant log-spiral 10 km x 4000 times x 8 ch "
                                   f"(1.3-1.5 GHz) = {obs.nvis / 1e6:.1f} M visibilities, 32 w-planes, {P} uv "
                                   f"partitions; one fused major cycle of every partition per step",
                       "n": obs.n, "n_wplanes": obs.n_wplanes, "n_part": P, "entries": int(st["n_entries"]),
                       "windows": st["window_size"][:P], "l2": "flushed before each cycle (512 MiB write)"},
            "clocks": clk.summary(), "major_cycle": mc, "partition_ms": part_ms, "generate_uvw_s": gen_s,
            "part_count": st["part_count"][:P], "n_outside": st["n_outside"]}
    rec.close()
    rix.destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
        if a.json_out:
            with open(a.json_out, "w") as f:
                json.dump(line, f, indent=1)
    return 0


def serve_pools(rank: int):
    """The serving workload's observations: four of the small recipe (seeds
    100-103), the medium recipe (seed 1: 8.06 M visibilities), four
    channel-chunk jobs of the batching recipe (seeds 1000-1003) and the large
    recipe's uvw (seed 3: 260 M visibilities) with seeded complex Gaussian
    visibilities (analytic visibilities of its 2100 sources at 260 M samples
    take far longer to make than to image).  Kind -> (share, [observations],
    major cycles, ms-CLEAN scales, FISTA levels)."""
    from paper_2507_22128_gb300 import synth
    small = [synth.plain_small(seed=100 + k + 10 * rank) for k in range(4)]
    medium = [synth.medium(seed=1 + rank)]
    chunk = synth.batch_chunk_jobs(n_jobs=4, base_seed=1000 + 100 * rank)
    large = synth.large(seed=3 + rank, with_vis=False)
    rng = np.random.default_rng(3 + rank)
    v = np.empty((large.nrow, large.nchan), np.complex64)
    v.real = rng.standard_normal(v.shape, dtype=np.float32)
    v.imag = rng.standard_normal(v.shape, dtype=np.float32)
    large.vis = v
    return {"small": (0.50, small, 5, (0.0, 3.0, 9.0), 3),
            "medium": (0.30, medium, 10, (0.0, 4.0, 16.0), 4),
            "chunk": (0.15, chunk, 5, (0.0, 4.0, 16.0), 4),
            "large": (0.05, [large], 8, (0.0, 4.0, 16.0, 32.0), 4)}


def serve_requests(pools, arrivals, rng, precision, only=None):
    """One request per arrival: kind by the pools' shares, observation
    uniform in its pool, ms-CLEAN or FISTA with probability 1/2 each
    (ms-CLEAN: gain 0.1, 2000 iterations, threshold 1e-4; FISTA: Db4, 50
    iterations, lambda = 1e-3 max |residual of cycle 1|)."""
    from paper_2507_22128_gb300 import pipeline, serve
    names = list(pools)
    probs = np.array([pools[k][0] for k in names])
    picks = rng.choice(len(names), arrivals.shape[0], p=probs / probs.sum())
    obs_pick = rng.random(arrivals.shape[0])
    meth_pick = rng.random(arrivals.shape[0]) < 0.5
    reqs = []
    for i, t in enumerate(arrivals):
        kind = names[picks[i]]
        _, obs_list, n_major, scales, levels = pools[kind]
        if only is not None and kind not in only:
            continue
        obs = obs_list[int(obs_pick[i] * len(obs_list))]
        if meth_pick[i]:
            m = pipeline.Method("msclean", scales, 0.1, 2000, 1e-4)
        else:
            m = pipeline.Method("fista", lam_rel=1e-3, iters=50, levels=levels)
        reqs.append(serve.Request(i, obs, m, n_major, arrival=float(t), precision=precision,
                                  kind=f"{kind} {m.kind}"))
    return reqs


def serve_workload(a, rank, world, local):
    """The serving workload (one process per GPU, each its own arrival
    stream): Poisson arrivals (seed 4) at --serve-rate jobs/s of jobs drawn
    50/30/15/5 % from the small, medium, channel-chunk and large recipes,
    half ms-CLEAN and half FISTA, admitted in arrival order under a
    --serve-budget-gb device-memory budget (the library's reservation per
    job) with each job's state resident until its combined image is read
    back, --serve-slots concurrent jobs at most.  Runs:
      offered:   --serve-jobs arrivals at --serve-rate, FP32;
      sustained: --serve-compare-jobs arrivals at 0.8 x the achieved rate of
                 the first run, FP32;
      fp32/fp64: the first --serve-compare-jobs arrivals of the first run's
                 stream whose jobs FP64 supports (N <= 2048: the large
                 recipe's are left out), at the same arrival times, served
                 in FP32 and then in FP64; per job the relative L2 distance
                 between the two combined images.
    Latency runs from a job's arrival to the read-back of its combined image;
    its inputs are copied from page-locked host memory when it is admitted."""
    from paper_2507_22128_gb300 import rix, serve
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    pools = serve_pools(rank)
    gen_s = time.perf_counter() - t0
    ctx = rix.create(local, int(a.serve_budget_gb * 1e9))
    peak = {"bytes": 0}

    def probe():
        free, total = torch.cuda.mem_get_info(dev)
        peak["bytes"] = max(peak["bytes"], total - free)

    def run(reqs, label):
        t1 = time.perf_counter()
        serve.prepare_host(reqs)
        prep = time.perf_counter() - t1
        torch.cuda.synchronize()
        peak["bytes"] = 0
        with ClockSampler(local) as clk:
            serve.serve(ctx, reqs, n_slots=a.serve_slots, mem_probe=probe)
        torch.cuda.synchronize()
        out = serve.summary(reqs)
        out.update({"run": label, "clocks": clk.summary(), "device_bytes_in_use_peak": int(peak["bytes"]),
                    "host_prepare_s": prep})
        serve.clear_host()
        return out

    rng = np.random.default_rng(4 + rank)
    arrivals = serve.poisson_arrivals(rng, a.serve_jobs, a.serve_rate)
    reqs = serve_requests(pools, arrivals, np.random.default_rng(40 + rank), rix.FP32)
    runs = {"offered": run(reqs, f"{a.serve_jobs} arrivals at {a.serve_rate} jobs/s, FP32")}
    runs["offered"]["arrival_rate_per_s"] = a.serve_rate
    k = a.serve_compare_jobs
    if k > 0:
        rate = max(0.8 * runs["offered"]["achieved_jobs_per_s"], 0.1)
        arr2 = serve.poisson_arrivals(np.random.default_rng(44 + rank), k, rate)
        runs["sustained"] = run(serve_requests(pools, arr2, np.random.default_rng(41 + rank), rix.FP32),
                                f"{k} arrivals at {rate:.2f} jobs/s (0.8 x the achieved rate), FP32")
        runs["sustained"]["arrival_rate_per_s"] = rate
        sub = [q for q in serve_requests(pools, arrivals, np.random.default_rng(40 + rank), rix.FP32)
               if not q.kind.startswith("large")][:k]
        r32 = run(sub, f"first {len(sub)} arrivals without the large recipe, FP32")
        img32 = {q.rid: q.image for q in sub}
        sub64 = [q for q in serve_requests(pools, arrivals, np.random.default_rng(40 + rank), rix.FP64)
                 if not q.kind.startswith("large")][:k]
        r64 = run(sub64, f"the same {len(sub64)} arrivals, FP64")
        diffs = {}
        for q in sub64:
            d = float(np.linalg.norm(img32[q.rid] - q.image) / max(np.linalg.norm(q.image), 1e-300))
            diffs.setdefault(q.kind, []).append(d)
        r64["fp32_vs_fp64_image_rel_l2"] = {kk: {"median": float(np.median(v)), "max": float(np.max(v)),
                                                 "jobs": len(v)} for kk, v in sorted(diffs.items())}
        runs["fp32"] = r32
        runs["fp64"] = r64
    rix.destroy(ctx)
    off = runs["offered"]
    line = {"metric": "p99 job latency", "value": off["p99_latency_s"], "unit": "s", "n_gpus": world,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (analytic visibilities of the small, medium and chunk recipes; the large recipe's "
                    "uvw with seeded Gaussian visibilities)",
            "config": {"workload": f"serving: Poisson arrivals at {a.serve_rate} jobs/s, {a.serve_jobs} arrivals, "
                                   "mix 50/30/15/5 % small/medium/chunk/large, half ms-CLEAN half FISTA",
                       "budget_gb": a.serve_budget_gb, "slots": a.serve_slots,
                       "pools": {kk: len(v[1]) for kk, v in pools.items()}},
            "generate_s": gen_s, "runs": runs}
    if rank == 0:
        print(json.dumps(line), flush=True)
        if a.json_out:
            with open(a.json_out, "w") as f:
                json.dump(line, f, indent=1)
    return 0


def serving_experiment(ctx, a, rank):
    """Continuous-batching run: Poisson arrivals of a job mix, p50/p99 latency."""
    from paper_2507_22128_gb300 import pipeline, serve, synth
    rng = np.random.default_rng(4 + rank)
    kinds = [
        ("small 128^2 coplanar ms-CLEAN 5 cycles", 0.5, synth.plain_small(seed=100),
         pipeline.Method("msclean", (0.0, 3.0, 9.0), 0.1, 500, 1e-4), 5),
        ("medium 1024^2 16 w-planes 2.0 M vis FISTA 10 cycles", 0.3, synth.medium(seed=101, n_times=250),
         pipeline.Method("fista", lam_rel=1e-3, iters=50, levels=4), 10),
        ("chunk 512^2 16 w-planes 1.0 M vis FISTA 5 cycles", 0.2, synth.medium(seed=102, n_times=125, n=512),
         pipeline.Method("fista", lam_rel=1e-3, iters=50, levels=4), 5),
    ]
    probs = np.array([k[1] for k in kinds])
    arrivals = serve.poisson_arrivals(rng, a.serve_jobs, a.serve_rate)
    picks = rng.choice(len(kinds), a.serve_jobs, p=probs / probs.sum())
    reqs = [serve.Request(i, kinds[k][2], kinds[k][3], kinds[k][4], arrival=float(t))
            for i, (k, t) in enumerate(zip(picks, arrivals))]
    torch.cuda.synchronize()
    serve.serve(ctx, reqs, n_slots=4)
    out = serve.summary(reqs)
    out.update({"arrival_rate_per_s": a.serve_rate, "slots": 4,
                "mix": {k[0]: int((picks == i).sum()) for i, k in enumerate(kinds)},
                "offered_jobs_per_s": a.serve_jobs / float(arrivals[-1])})
    return out


def phase_split(rec, rix, a, meth, stream, uvw, vis, w, out, flush):
    """Event-timed phases of one job on one stream (the timed steps overlap
    the partitions' work on their own streams): partition, major cycles,
    minor cycles (batched as in the steps unless --no-batch-minor; the first
    cycle's minor phase includes the PSFs)."""
    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e
    flush_l2(flush)
    e0 = ev()
    rix.set_uv_partition(rec.job, uvw, w, None, 1.0, None, stream)
    e1 = ev()
    maj, mnr = 0.0, 0.0
    for c in range(a.cycles):
        s0 = ev()
        for p in range(2):
            rix.major_cycle(rec.job, p, vis, None, None, stream)
        s1 = ev()
        if a.no_batch_minor:
            for p in range(2):
                rec.minor(p, meth, stream=stream)
        else:
            rec.minor_all(meth, stream)
        s2 = ev()
        torch.cuda.synchronize()
        maj += s0.elapsed_time(s1)
        mnr += s1.elapsed_time(s2)
    rix.combine(rec.job, out, stream)
    torch.cuda.synchronize()
    return {"partition_sort": e0.elapsed_time(e1), "major_cycles": maj, "minor_cycles_incl_psf": mnr}


def major_cycle_metric(rec, rix, meth, stream, vis, flush, st, nchan, n_cycles=7):
    """The survey's metric on the fused major-cycle operator alone: samples
    of both partitions (overlap counted in each) / the wall time of one major
    cycle of both partitions (a4-a6: model -> planes, degrid, residual,
    grid, planes -> residual image; each partition on its own stream as the
    pipeline issues them), median over cycles after the first, L2 flushed
    before each; %HBM against the survey's algorithmic bytes: per sample
    uvw 24/nchan + visibility 8 + weight 4 + index 4 B, per partition and
    w-plane 8 passes over the full (2N)^2 complex plane.  Then one more
    cycle with the partitions on one stream for the per-launch times of the
    gridder and the transforms."""
    main = stream
    ps = rec._pstreams if hasattr(rec, "_pstreams") else [torch.cuda.Stream() for _ in range(2)]
    times = []
    for c in range(n_cycles):
        flush_l2(flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(main)
        for p, s in enumerate(ps):
            s.wait_event(e0)
            rec.major(p, stream=s)
        for s in ps:
            j = torch.cuda.Event()
            j.record(s)
            main.wait_event(j)
        e1.record(main)
        rec.minor_all(meth, main)
        torch.cuda.synchronize()
        if c > 0:
            times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    units = sum(st["part_count"][:2])
    ng = 2 * rec.n
    nplanes = 16
    byt = units * (24.0 / nchan + 16.0) + 2 * nplanes * 8 * ng * ng * 8.0
    peaks, kind = measured_peaks()
    hbm = byt / (ms * 1e-3) / 1e9
    # serial pass: per-launch device times of the gridder and the transforms
    per = {}
    for p in range(2):
        flush_l2(flush)
        torch.cuda.synchronize()
        for cls in (rix.TIME_TILES, rix.TIME_FFT):
            rix.timing_read(cls)
        rix.timing_enable(True)
        rec.major(p, stream=main)
        torch.cuda.synchronize()
        rix.timing_enable(False)
        tt, tb, tn = rix.timing_read(rix.TIME_TILES)
        ft, fb, fn = rix.timing_read(rix.TIME_FFT)
        per[p] = {"gridder_ms": tt, "fft_ms": ft, "fft_launches": fn}
    rec.minor_all(meth, main)
    torch.cuda.synchronize()
    return {"value": units / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_cycle": ms, "cycles_timed": len(times),
            "samples_per_cycle": int(units),
            "hbm": {"algorithmic_bytes_per_cycle": byt, "achieved_gbs": hbm, "peak_gbs": float(peaks["hbm_gbs"]),
                    "frac": hbm / float(peaks["hbm_gbs"]), "peak_source": kind,
                    "bytes": "survey 8(d): per sample 24/nchan + 16 B; per partition and w-plane 8 x (2N)^2 x 8 B"},
            "per_partition_serial": per}


def direct_dft_errors(rec, rix, obs, image, vis_d, wt_d, part, n_vis=256, n_pix=64, seed=7):
    """Error of the library's operator against the exact measurement operator
    (Eq. 1 direct sums in FP64 on the device, independent of the library):
    degrid of `image` on n_vis sampled visibilities of partition `part`, and
    the partition's dirty image (grid of the observed visibilities) on n_pix
    sampled pixels; relative L2 over the samples."""
    dev = vis_d.device
    n, cell = obs.n, obs.cell_rad
    f = torch.as_tensor(obs.freq, dtype=torch.float64, device=dev) / 299792458.0
    uvw = torch.as_tensor(obs.uvw, dtype=torch.float64, device=dev)
    u = (uvw[:, 0:1] * f[None, :]).reshape(-1)
    v = (uvw[:, 1:2] * f[None, :]).reshape(-1)
    w = (uvw[:, 2:3] * f[None, :]).reshape(-1)
    mask = torch.zeros(obs.nvis, dtype=torch.uint8, device=dev)
    rix.set_uv_partition(rec.job, rec.uvw, rec.weight, None, 1.0, mask)
    sel = torch.nonzero(((mask >> part) & 1) == 1).reshape(-1)
    g = torch.Generator(device="cpu").manual_seed(seed)
    pick = sel[torch.randperm(sel.numel(), generator=g)[:n_vis].to(dev)]
    cdt = rec.cdtype
    # degrid
    out = torch.zeros(obs.nvis, dtype=cdt, device=dev)
    rix.degrid(rec.job, part, image.to(rec.rdtype).contiguous(), out)
    off = (torch.arange(n, dtype=torch.float64, device=dev) - n // 2) * cell
    mm, ll = torch.meshgrid(off, off, indexing="ij")
    r2 = ll * ll + mm * mm
    nn = torch.sqrt(1.0 - r2)
    nm1 = -r2 / (1.0 + nn)
    x = (image.to(torch.float64) / nn).reshape(-1)
    want = torch.zeros(n_vis, dtype=torch.complex128, device=dev)
    for c0 in range(0, n * n, 1 << 16):
        c1 = min(n * n, c0 + (1 << 16))
        ph = (torch.outer(u[pick], ll.reshape(-1)[c0:c1]) + torch.outer(v[pick], mm.reshape(-1)[c0:c1])
              + torch.outer(w[pick], nm1.reshape(-1)[c0:c1]))
        want += torch.exp(-2j * torch.pi * ph) @ x[c0:c1].to(torch.complex128)
    got = out[pick].to(torch.complex128)
    e_deg = float(torch.linalg.norm(got - want) / torch.linalg.norm(want))
    # grid: dirty image of the observed visibilities on sampled pixels
    img = torch.empty((n, n), dtype=rec.rdtype, device=dev)
    rix.grid(rec.job, part, vis_d, img)
    rows = torch.randint(0, n, (n_pix,), generator=g).to(dev)
    cols = torch.randint(0, n, (n_pix,), generator=g).to(dev)
    wt = wt_d.reshape(-1).to(torch.float64)[sel]
    y = wt * vis_d.reshape(-1).to(torch.complex128)[sel]
    lp, mp = off[cols], off[rows]
    rp = lp * lp + mp * mp
    np_ = torch.sqrt(1.0 - rp)
    nm1p = -rp / (1.0 + np_)
    acc = torch.zeros(n_pix, dtype=torch.float64, device=dev)
    us, vs, ws = u[sel], v[sel], w[sel]
    for s0 in range(0, sel.numel(), 1 << 18):
        s1 = min(sel.numel(), s0 + (1 << 18))
        ph = (torch.outer(us[s0:s1], lp) + torch.outer(vs[s0:s1], mp) + torch.outer(ws[s0:s1], nm1p))
        acc += (y[s0:s1] @ torch.exp(2j * torch.pi * ph)).real
    want_px = acc / np_ / wt.sum()
    got_px = img[rows, cols].to(torch.float64)
    e_grid = float(torch.linalg.norm(got_px - want_px) / torch.linalg.norm(want_px))
    return {"degrid_rel_l2": e_deg, "grid_rel_l2": e_grid, "partition": part, "visibilities": n_vis,
            "pixels": n_pix, "reference": "direct DFT of Eq. 1 in FP64 (sampled)"}


def fp64_comparator(ctx, rix, pipeline, obs, a, flush, n_cycles=4):
    """The plain FP64 GPU operator on the same workload: one FP64 job, the
    fused major cycle of both partitions timed as in major_cycle_metric, and
    its error against the direct DFT."""
    rec = pipeline.Reconstruction(ctx, obs.n, obs.cell_rad, obs.n_wplanes, obs.freq, obs.nrow, 2, rix.FP64)
    try:
        rec.set_data(obs.uvw, obs.vis, obs.weight)
        torch.cuda.synchronize()
        st = rec.stats()
        m = pipeline.Method("fista", lam_rel=1e-3, iters=2, levels=1)
        s = torch.cuda.current_stream()
        mc = major_cycle_metric(rec, rix, m, s, None, flush, st, obs.nchan, n_cycles=n_cycles)
        model = torch.empty((obs.n, obs.n), dtype=torch.float64, device="cuda")
        rix.get_model(rec.job, 1, model)
        wt = torch.as_tensor(obs.weight, device="cuda")
        err = direct_dft_errors(rec, rix, obs, model, rec.vis, wt, 1)
        return {"value": mc["value"], "unit": UNIT, "ms_per_cycle": mc["ms_per_cycle"], "error": err,
                "per_partition_serial": mc["per_partition_serial"]}
    finally:
        rec.close()


def cufft_comparison(n, nplanes, window, flush, reps=5):
    """cuFFT (through torch.fft) on the major cycle's plane transforms, as a
    comparison for the library's own passes: the forward transform of the
    zero-padded (2N)^2 planes of all w-planes and the inverse, full planes
    (cuFFT has no pruned window), complex64, median of `reps`."""
    ng = 2 * n
    x = torch.zeros((nplanes, ng, ng), dtype=torch.complex64, device="cuda")
    x[:, n // 2:n // 2 + n, n // 2:n // 2 + n] = 1.0
    times = []
    for _ in range(reps + 1):
        flush_l2(flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        y = torch.fft.fft2(x)
        z = torch.fft.ifft2(y)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    del x, y, z
    return {"cufft_fwd_plus_inv_ms": statistics.median(times[1:]), "planes": nplanes, "grid": ng,
            "note": "full (2N)^2 planes; the library transforms only each partition's uv window"}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# FP32 w-stacked gridder (k_tiles_fp<RESID>) at the default 1024^2 workload,
# from a one-pass ncu capture of the major cycles of both partitions: (low,
# high) partition.  Reported only for that workload and while the kernel's
# source is the one the counters were taken on.
# ncu dram__bytes_read.sum + dram__bytes_write.sum of the two k_tiles_fp<RESID>
# launches of the medium job's first major cycle (low, high partition), with
# the sha1 of the sources the kernel was built from (k_tiles_fp.cu,
# rix_internal.cuh): a changed source voids them
TILES_TRAFFIC = {"src_sha1": ("26627dc6d95a2554aad224fbd0f5828f69ef81e6", "f3856a35dfa300bce2539f3ed838fef54aba3c6c"),
                 "resid": (139.825408e6, 203.583488e6)}


def tiles_traffic(a):
    import hashlib
    shas = []
    for name in ("k_tiles_fp.cu", "rix_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2507_22128_gb300", "csrc", name), "rb") as f:
            shas.append(hashlib.sha1(f.read()).hexdigest())
    if tuple(shas) != TILES_TRAFFIC["src_sha1"] or a.fp64 or a.n != 1024 or a.n_times != 1000:
        return None
    return sum(TILES_TRAFFIC["resid"]) / 2


def roofline_gridder(mc, st, a):
    """Roofline of the major cycle's gridder (degrid + residual + grid), from
    its per-launch device times with the partitions on one stream.  Bound:
    FP32 issue (ALU): 4096 flops per (sample, partition) entry and major
    cycle (degrid 512 taps x 2 complex-by-real FMAs, grid 512 taps x 2) over
    152 SMs x 128 FP32 lanes x 2 flops x the maximum SM clock (a derived
    peak: the measured peaks hold no FP32 SIMT figure).  `hbm` adds its
    algorithmic bytes: per entry its geometry record and weighted visibility
    (16 + 16 B), and per w-plane of the partition's uv window one model read
    and one residual write (2 x 8 B per cell)."""
    per = mc["per_partition_serial"]
    ms = sum(per[p]["gridder_ms"] for p in (0, 1))
    if ms <= 0:
        return None
    peaks, kind = measured_peaks()
    clk = float(peaks.get("sm_max_mhz", 2070.0))
    lanes = 2 if a.fp64 else 128        # FP64 / FP32 results per SM per clock (GB300 unit counts)
    peak = 152 * lanes * 2 * clk * 1e6 / 1e12
    ent = float(sum(st["part_count"][:2]))
    ach = 4096.0 * ent / (ms * 1e-3) / 1e12
    win = st["window_size"][:2]
    byt = ent * 32.0 + sum(2 * 8.0 * 16 * w * w for w in win)
    hbm = byt / (ms * 1e-3) / 1e9
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    return {"bound": "alu",
            "kernel": "k_tiles_ws (FP64, shared-memory staging)" if a.fp64 else
                      "k_tiles_fp<RESID> (degrid + residual + grid, register-resident footprints, TMA tiles)",
            "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "ms_per_launch": {"low": per[0]["gridder_ms"], "high": per[1]["gridder_ms"]},
            "hbm": {"achieved_gbs": hbm, "peak_gbs": hbm_peak, "frac": hbm / hbm_peak,
                    "algorithmic_bytes_per_launch": byt / 2, "peak_source": kind},
            "traffic": tiles_traffic(a), "traffic_unit": "B per launch (ncu dram read + write)",
            "peak_source": f"152 SMs x {lanes} {'FP64' if a.fp64 else 'FP32'} lanes x 2 flop x {clk:.0f} MHz "
                           f"(max SM clock of {kind} peaks)"}


if __name__ == "__main__":
    sys.exit(main())
