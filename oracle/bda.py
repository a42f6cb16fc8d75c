"""Baseline-dependent averaging (BDA), the remedy the paper names for
unbalanced partitions (Sec. 6.2: a dense uv centre such as Sgr B2's leaves
the outer node idle; Sec. 7 item d), after Wijnholds et al. (2018).

Test infrastructure only: this module is the CPU oracle of the library's
averaging call and is imported by tests alone.

Short baselines move slowly through the uv plane, so consecutive time
samples of one baseline can be averaged with little decorrelation; long
baselines cannot.  Averaging each baseline over a window that shrinks with
its uv speed thins the dense centre of the uv plane and flattens the sample
density, so a fixed ring radius splits the samples more evenly.

Reading (the paper gives no parameters):
  * rows are time-major: row = t * n_baselines + b, t = 0 .. n_times - 1;
  * the uv shift of baseline b per time step is
        s_b = max_t  sqrt(du^2 + dv^2) * (N dl)
    with du, dv the change of (u, v) in wavelengths at the highest channel
    frequency between times t and t + 1 (the cells of the N x N image's
    Fourier grid, the unit of the partition radius);
  * the window is k_b = min(n_times, max(1, floor(max_shift / s_b))) time
    samples (n_times when s_b = 0): the uv track moves at most max_shift
    cells within a window;
  * baseline b's times are cut into consecutive windows of k_b samples, the
    last one shorter;
  * an averaged row holds the plain mean of the window's uvw, and per
    channel the weight sum W = sum w and the weighted mean visibility
    sum(w v) / W (0 when W = 0);
  * output rows are baseline-major: baseline b's windows in time order,
    after those of baselines 0 .. b-1.

Every step is FP64 with each product and sum rounded in the order written
(the window arithmetic decides an integer, so the library takes it in the
same order).
"""
from __future__ import annotations

import dataclasses

import numpy as np

C_LIGHT = 299792458.0


@dataclasses.dataclass
class Averaged:
    uvw: np.ndarray        # (nrow_out, 3) float64
    vis: np.ndarray        # (nrow_out, nchan) complex128
    weight: np.ndarray     # (nrow_out, nchan) float64
    window: np.ndarray     # (n_baselines,) int64: k_b
    counts: np.ndarray     # (n_baselines,) int64: windows per baseline
    offsets: np.ndarray    # (n_baselines + 1,) int64: first output row of each baseline


def uv_shift_cells(uvw_m: np.ndarray, n_times: int, n_bl: int, f_max: float, n: int, cell: float) -> np.ndarray:
    """s_b: the largest per-step (u, v) change of each baseline, in cells of
    the N-grid's Fourier plane at the highest frequency."""
    uv = uvw_m.reshape(n_times, n_bl, 3)
    s = f_max / C_LIGHT
    ncell = n * cell
    if n_times < 2:
        return np.zeros(n_bl)
    du = (uv[1:, :, 0] - uv[:-1, :, 0]) * s
    dv = (uv[1:, :, 1] - uv[:-1, :, 1]) * s
    step = np.sqrt(du * du + dv * dv) * ncell
    return step.max(axis=0)


def windows(uvw_m: np.ndarray, n_times: int, n_bl: int, f_max: float, n: int, cell: float,
            max_shift: float) -> np.ndarray:
    sb = uv_shift_cells(uvw_m, n_times, n_bl, f_max, n, cell)
    k = np.full(n_bl, n_times, dtype=np.int64)
    moving = sb > 0.0
    k[moving] = np.clip(np.floor(max_shift / sb[moving]), 1, n_times).astype(np.int64)
    return k


def average(uvw_m: np.ndarray, vis: np.ndarray, weight: np.ndarray | None, n_times: int, n_bl: int,
            freq: np.ndarray, n: int, cell: float, max_shift: float) -> Averaged:
    nchan = freq.shape[0]
    vis = vis.reshape(n_times, n_bl, nchan).astype(np.complex128)
    w = (np.ones((n_times, n_bl, nchan)) if weight is None
         else weight.reshape(n_times, n_bl, nchan).astype(np.float64))
    uv = uvw_m.reshape(n_times, n_bl, 3)
    k = windows(uvw_m, n_times, n_bl, float(np.max(freq)), n, cell, max_shift)
    counts = (n_times + k - 1) // k
    offsets = np.concatenate([[0], np.cumsum(counts)])
    nout = int(offsets[-1])
    out_uvw = np.zeros((nout, 3))
    out_vis = np.zeros((nout, nchan), dtype=np.complex128)
    out_w = np.zeros((nout, nchan))
    for b in range(n_bl):
        for g in range(int(counts[b])):
            t0, t1 = g * int(k[b]), min(n_times, (g + 1) * int(k[b]))
            row = int(offsets[b]) + g
            out_uvw[row] = uv[t0:t1, b].mean(axis=0)
            ws = w[t0:t1, b].sum(axis=0)
            sv = (w[t0:t1, b] * vis[t0:t1, b]).sum(axis=0)
            out_w[row] = ws
            out_vis[row] = np.where(ws > 0.0, sv / np.where(ws > 0.0, ws, 1.0), 0.0)
    return Averaged(out_uvw, out_vis, out_w, k, counts, offsets)
