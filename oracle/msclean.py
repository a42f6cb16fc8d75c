"""Multi-scale CLEAN minor cycle (Eq. 6 and Eq. 7; Cornwell 2008).

Inputs are the centred 2N-grid spectra of the dirty image D and of the PSF P
(for the decentralized form, Eq. 7's composite dirty image and PSF).

Scale functions (reading; the paper uses RASCIL's defaults): B_0 = delta,
B_s(r) = 1 - (r/s)^2 for r < s pixels, normalised to unit sum; scale bias
b_s = 1 - 0.6 s / s_max.

    R_s     = crop F^-1 [B_s D]                    (scale residuals, N x N)
    P_{s,t} = F^-1 [B_s B_t P]                     (cross PSFs, 2N x 2N, centre (N, N))
    repeat K times, or until max |R_0| < threshold:
        (s*, p*) = argmax_{s allowed, p} b_s |R_s(p)| / P_{s,s}(0)
                   (ties: smaller s, then smaller row-major index)
        a        = gain R_{s*}(p*) / P_{s*,s*}(0)
        model   += a B_{s*}(. - p*)                (clipped to the image)
        R_s     -= a P_{s,s*}(. - p*)   for every s
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import filters


def scale_kernel(s: float, n: int) -> np.ndarray:
    """B_s placed on the 2N x 2N grid, centre at (N, N)."""
    b = np.zeros((2 * n, 2 * n))
    if s == 0:
        b[n, n] = 1.0
        return b
    k = np.arange(2 * n) - n
    yy, xx = np.meshgrid(k, k, indexing="ij")
    r2 = (xx * xx + yy * yy).astype(np.float64)
    b = np.where(r2 < s * s, 1.0 - r2 / (s * s), 0.0)
    return b / b.sum()


def bias(scales) -> np.ndarray:
    smax = max(scales)
    return np.array([1.0 - 0.6 * s / smax if smax > 0 else 1.0 for s in scales])


@dataclasses.dataclass
class Result:
    model: np.ndarray
    components: list          # (scale index, row, col, amplitude)
    residuals: np.ndarray     # final R_s
    iterations: int
    gaps: list = dataclasses.field(default_factory=list)   # (best, runner-up) per iteration


def clean(dirty_spec: np.ndarray, psf_spec: np.ndarray, scales, gain: float, niter: int,
          threshold: float, allowed=None) -> Result:
    n = dirty_spec.shape[0] // 2
    ns = len(scales)
    allowed = np.ones(ns, dtype=bool) if allowed is None else np.asarray(allowed, dtype=bool)
    bk = [scale_kernel(s, n) for s in scales]
    bs = [filters.spectrum(b.astype(np.complex128)) for b in bk]
    R = np.stack([filters.crop(filters.ispectrum(bs[s] * dirty_spec)).real for s in range(ns)])
    P = np.empty((ns, ns, 2 * n, 2 * n))
    for s in range(ns):
        for t in range(ns):
            P[s, t] = filters.ispectrum(bs[s] * bs[t] * psf_spec).real
    peak = np.array([P[s, s, n, n] for s in range(ns)])
    b = bias(scales)
    model = np.zeros((n, n))
    comps = []
    gaps = []
    it = 0
    while it < niter:
        if np.abs(R[0]).max() < threshold:
            break
        best, bs_i, bp = -1.0, -1, -1
        second = -1.0
        for s in range(ns):
            if not allowed[s]:
                continue
            v = (b[s] * np.abs(R[s]) / peak[s]).reshape(-1)
            p = int(np.argmax(v))
            # runner-up over all candidates (for near-tie diagnostics only)
            top2 = np.partition(v, -2)[-2:] if v.size > 1 else np.array([-1.0, v[0]])
            if v[p] > best:
                second = max(best, float(top2[0]))
                best, bs_i, bp = float(v[p]), s, p
            else:
                second = max(second, float(v[p]))
        py, px = divmod(bp, n)
        a = gain * R[bs_i, py, px] / peak[bs_i]
        comps.append((bs_i, py, px, float(a)))
        gaps.append((best, second))
        # every pixel offset from p* lies in (-N, N): index the 2N-grid arrays
        model += a * bk[bs_i][n - py:2 * n - py, n - px:2 * n - px]
        for s in range(ns):
            R[s] -= a * P[s, bs_i, n - py:2 * n - py, n - px:2 * n - px]
        it += 1
    return Result(model, comps, R, it, gaps)


def allowed_scales(scales, n: int, p: int, cycle: int, ells, delta: float) -> np.ndarray:
    """psi^n of Eq. 7: every scale from cycle 2 on; at cycle 1 partition 0
    keeps all scales and partition p > 0 keeps s = 0 and the scales whose
    characteristic frequency N / (2 s) reaches its inner ring radius ell_p - delta."""
    if cycle > 1 or p == 0:
        return np.ones(len(scales), dtype=bool)
    inner = ells[p - 1] - delta
    return np.array([s == 0 or n / (2.0 * s) >= inner for s in scales])
