"""Autotuner of the FP32 w-stacked gridder's per-job tuning.

Two knobs (rix_job_tune): the most samples with one kernel footprint a warp
grids between two flushes of its accumulators (chunk_limit) and the resident gridder CTAs per SM.  For a
job shape (GPU, image side, w-planes, channels, partitions, and the sample
count in powers of two) every candidate is applied and the partitions'
gridder is timed with rix_gridder_probe (device time, no change to the job's
results); the fastest candidate is cached in a JSON file and applied to
every later job of that shape without timing.  Host-side marshalling only.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import rix

# (chunk_limit, ctas_per_sm); ctas_per_sm 0 = as many as fit (two at 128 registers)
CANDIDATES = ((64, 0), (128, 0), (32, 0), (16, 0), (64, 1))


def default_cache_path() -> str:
    base = os.environ.get("RIX_AUTOTUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2507_22128_gb300", "autotune.json")


def shape_key(n: int, n_wplanes: int, nchan: int, n_part: int, n_samples: int, device: int = 0) -> str:
    gpu = torch.cuda.get_device_name(device) if torch.cuda.is_available() else "cpu"
    bucket = int(math.log2(max(n_samples, 1)))
    return f"{gpu}|N{n}|W{n_wplanes}|C{nchan}|P{n_part}|S2^{bucket}"


def load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(path: str, table: dict):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(rec, vis, cache_path: str | None = None, reps: int = 3, candidates=CANDIDATES) -> dict:
    """Tune one pipeline.Reconstruction (partitioned, FP32 w-stacked): the
    cached choice for its shape, else the fastest candidate by the summed
    gridder time of its partitions (then cached).  Returns the choice with
    its timings."""
    path = cache_path or default_cache_path()
    st = rec.stats()
    key = shape_key(rec.n, rec.n_wplanes, len(rec.freq), rec.n_part, int(st["n_samples"]), rec.device.index or 0)
    table = load(path)
    if key in table:
        c = table[key]
        rix.job_tune(rec.job, c["chunk_limit"], c["ctas_per_sm"])
        return dict(c, cached=True, key=key)
    timings = []
    for chunk, ctas in candidates:
        rix.job_tune(rec.job, chunk, ctas)
        ms = sum(rix.gridder_probe(rec.job, p, vis, reps) for p in range(rec.n_part))
        timings.append({"chunk_limit": chunk, "ctas_per_sm": ctas, "ms": ms})
    best = min(timings, key=lambda t: t["ms"])
    rix.job_tune(rec.job, best["chunk_limit"], best["ctas_per_sm"])
    table[key] = {"chunk_limit": best["chunk_limit"], "ctas_per_sm": best["ctas_per_sm"], "ms": best["ms"]}
    save(path, table)
    return dict(table[key], cached=False, key=key, timings=timings)

