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
    ap.add_argument("--schedule", default=None,
                    help="a,b: lambda_n = a ||residual_n||_2 b^n instead of 1e-3 max |residual_1|")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-phases", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=24, help="arrivals in the serving experiment (0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=20.0, help="Poisson arrival rate, jobs/s")
    ap.add_argument("--json-out", default=None)
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
                             "sample": res["sample"]},
            "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(a, steps=1, warmup=0):
    """FP64 oracle major cycle (degrid + residual + grid, Eq. 2) of partition 0
    on a 1/64 row subset of the workload; Mvis/s = samples / seconds."""
    from oracle import gridder, partition
    from paper_2507_22128_gb300 import synth
    obs = synth.medium(seed=1, n_times=max(4, a.n_times // 64), n=a.n)
    g = gridder.geometry(obs.uvw, obs.freq, obs.n, obs.cell_rad, W=8, nw=obs.n_wplanes)
    r = partition.radius_px(g)
    m = partition.masks(r, partition.ring_radii(r, 2), 1.0, 2, g.inside)
    gp = gridder.subset(g, (m & 1) == 1)
    w = obs.weight.reshape(-1).astype(np.float64)
    model = np.zeros((obs.n, obs.n))
    nsamp = int(gp.inside.sum())
    times = []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        gridder.residual(obs.vis.reshape(-1), w, model, gp)
        dt = time.perf_counter() - t0
        if i >= warmup:
            times.append(dt)
    t = statistics.median(times)
    return {"value": nsamp / t / 1e6, "ms_per_step": t * 1e3, "cores": 1,
            "sample": f"one FP64 major cycle of partition 0 over {obs.nrow} rows x {obs.nchan} channels "
                      f"({nsamp} samples; 1/64 of the {a.n}^2 workload's rows), numpy, median of {steps}"}


def config_dict(a):
    return {"workload": f"medium: {a.n}x{a.n} 1as, 64 ant log-spiral x {a.n_times} times x 4 ch "
                        f"(1.3-1.5 GHz), 16 w-planes, 2 uv partitions, FISTA {'Db4' if a.dictionary == 'db4' else 'db1..db8'} "
                        f"{a.iters} it{'' if a.schedule is None else ', lambda schedule ' + a.schedule}, "
                        f"{a.cycles} major cycles",
            "n": a.n, "n_wplanes": 16, "n_part": 2, "major_cycles": a.cycles, "fista_iters": a.iters,
            "fista_dictionary": a.dictionary, "fista_batched": not a.no_batch_minor,
            "l2": "flushed between steps (512 MiB write)", "precision": "fp64" if a.fp64 else "fp32"}


def main():
    a = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if a.impl == "ours" else "gloo")
    if a.impl == "reference":
        return reference_arm(a, rank, world)

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
    meth = pipeline.Method("fista", lam_rel=1e-3, iters=a.iters, levels=4, dictionary=a.dictionary, schedule=sched)
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

    # the gridder runs once per partition per major cycle and once per
    # partition for the PSF; the PSF launches carry (weights only) a fraction
    # of the work, so the flop count below is a lower bound of the work timed
    roof = roofline_tiles(tiles_busy, tiles_n, st, a, units * a.steps)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if a.fp64 else "f32", "data": "synthetic",
            "config": config_dict(a), "clocks": clk.summary(), "e2e": e2e, "gpu_launches": int(launches),
            "roofline": roof, "phases_ms": phases,
            "kernel_ms_per_step": {"grid_tiles_busy": tiles_busy / a.steps, "grid_tiles_sum": tiles_ms / a.steps,
                                   "fft_passes_busy": fft_busy / a.steps,
                                   "minor_loop_busy": loop_busy / a.steps, "minor_loop_sum": loop_ms / a.steps},
            "samples_per_cycle": int(sum(st["part_count"][:2])), "step_ms": step_ms}
    if a.serve_jobs > 0:
        line["serving"] = serving_experiment(ctx, a, rank)
    if rank == 0 and not a.no_cpu_baseline:
        cb = cpu_baseline(a)
        line["cpu_baseline"] = {"value": cb["value"], "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                                "sample": cb["sample"]}
    rec.close()
    rix.destroy(ctx)
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


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per k_tiles_ws
# launch at the default 1024^2 workload, from a one-pass ncu capture of one
# timed job: residual launches of
# partitions 0 and 1, PSF launches of partitions 0 and 1.  Reported only for
# that workload and while k_grid.cu is the source the counters were taken on.
TILES_TRAFFIC = {"k_grid_sha1": "dab75048113381c5baa1a22cc19111f811558f46",
                 "resid": (162.13e6, 261.79e6), "psf": (115.38e6, 237.54e6)}


def tiles_traffic(a):
    import hashlib
    src = os.path.join(ROOT, "paper_2507_22128_gb300", "csrc", "k_grid.cu")
    with open(src, "rb") as f:
        sha = hashlib.sha1(f.read()).hexdigest()
    if sha != TILES_TRAFFIC["k_grid_sha1"] or a.fp64 or a.n != 1024 or a.n_times != 1000:
        return None
    # a step: `cycles` residual launches per partition and one PSF launch each
    tot = a.cycles * sum(TILES_TRAFFIC["resid"]) + sum(TILES_TRAFFIC["psf"])
    return tot / (2 * a.cycles + 2)


def roofline_tiles(tiles_ms, tiles_n, st, a, entries_timed):
    """Roofline of the tiled degrid/residual/grid kernel, the gridder of the
    major cycle: FP32 (or FP64) arithmetic over its event-timed launches
    (`tiles_ms` is their busy time: the two partitions' launches overlap).
    Algorithmic work per (sample, partition) entry and major cycle: degrid
    8 x 64 taps x 2 FMA (2048 flops) + grid 8 x 64 taps x (2 mul + 2 add)
    (2048 flops) = 4096 flops; the PSF launches (weights only) are counted
    at zero, so `achieved` is a lower bound."""
    if not tiles_n or tiles_ms <= 0:
        return None
    peaks, kind = measured_peaks()
    clk = float(peaks.get("sm_max_mhz", 2070.0))
    lanes = 2 if a.fp64 else 128        # FP64 / FP32 results per SM per clock (GB300 unit counts)
    peak = 152 * lanes * 2 * clk * 1e6 / 1e12
    flops = 4096.0 * entries_timed
    ach = flops / (tiles_ms * 1e-3) / 1e12
    # secondary: HBM against the measured copy bandwidth, with the algorithmic
    # bytes of the residual launches (per entry: uvw 24/nchan + visibility 8 +
    # weight 4 + index 4 B; per w-plane of the partition's uv window: model
    # read + residual write, 2 x 8 B per cell)
    nchan = 4
    ent_b = (24.0 / nchan + 8 + 4 + 4) * entries_timed
    win = st["window_size"][:2]
    plane_b = a.steps * a.cycles * sum(2 * 8.0 * 16 * w * w for w in win)
    hbm = (ent_b + plane_b) / (tiles_ms * 1e-3) / 1e9
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    return {"bound": "alu", "kernel": "k_tiles (degrid + residual + grid, w-stacked, T=16)",
            "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "hbm": {"achieved_gbs": hbm, "peak_gbs": hbm_peak, "frac": hbm / hbm_peak,
                    "algorithmic_bytes_per_launch": (ent_b + plane_b) / tiles_n, "peak_source": kind},
            "traffic": tiles_traffic(a), "traffic_unit": "B per launch",
            "launches_timed": tiles_n, "busy_ms_per_launch": tiles_ms / tiles_n,
            "ncu_binding_unit": "shared memory: L1/shared throughput 86 % of peak, FMA pipe 20 % "
                                "(ncu --set full of one launch at the medium recipe)",
            "peak_source": f"152 SMs x {lanes} {'FP64' if a.fp64 else 'FP32'} lanes x 2 flop x {clk:.0f} MHz "
                           f"(max SM clock of {kind} peaks)"}


if __name__ == "__main__":
    sys.exit(main())
