"""FP64 w-stacked ES gridder: the G, G^dagger and F, F^dagger of Eq. 2.

Conventions (shared by definition, not by code, with the CUDA path):

* grid side Ng = 2 N (oversampling 2); cell of the uv grid 1 / (Ng dl);
  uv-grid index j <-> spatial frequency k = j - Ng/2.
* sample grid coordinate  x = u_lambda * (dl * Ng) + Ng/2  (u_lambda = u_m f/c),
  first tap j0 = ceil(x - W/2), taps j0 .. j0+W-1 with weight
  phi(z), z = (d + i) * 2/W - 1, d = j0 - (x - W/2) in [0, 1).
* w-stacking with an ES kernel of the same support W_w = W over N_w planes:
  dw = (w_max - w_min) / (N_w - W_w), tw = (w_lambda - w_min) / dw,
  p0 = ceil(tw) (clamped to [0, N_w - W_w]), plane p weight
  phi((p0 - tw + i) * 2/W_w - 1), plane p sits at w_p = w_min + (p - W_w/2) dw.
  The identity  sum_p phi_g(t - p) exp(-2 pi i w_p (n-1))
               ~= exp(-2 pi i w (n-1)) Phi(dw (n-1))
  turns the w-term into a per-plane phase screen plus the image-domain
  correction 1 / Phi(dw (n-1)).
* model planes   G_p = F[ x / (n Phi(l/(dl Ng)) Phi(m/(dl Ng)) Phi(dw(n-1)))
                            * exp(-2 pi i w_p (n-1)) ]   (zero-padded, centred)
  degrid         V_k = sum_p phi_w sum_{i,j} phi_u phi_v G_p[j, i]
  grid (adjoint) planes accumulate y_k phi_w phi_u phi_v; image =
                 Re sum_p exp(+2 pi i w_p (n-1)) F^H[planes_p] / (n Phi Phi Phi_w)
  In coplanar mode (N_w = 0) there is one plane, no phase screen and no 1/n.
* samples whose footprint leaves [0, Ng) are dropped (flag ``inside``).

``grid`` and ``degrid`` are exact adjoints of each other by construction
(pinned to 1e-12) and approximate the direct DFT of ``oracle.dft`` to the ES
kernel's accuracy (pinned: <= 1e-6 relative L2 at W = 8).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.fft as _fft   # the 2D FFT primitive

# host threads of each 2D FFT (-1 = all); a caller running several oracle
# processes side by side sets 1
FFT_WORKERS = -1

from . import es

C_LIGHT = 299792458.0


@dataclasses.dataclass
class Geometry:
    n: int              # image side
    ng: int             # grid side
    cell: float
    W: int
    nw: int             # 0 = coplanar
    Ww: int
    beta: float
    w_min: float
    dw: float
    j0u: np.ndarray     # int64 per sample
    j0v: np.ndarray
    du: np.ndarray      # float64 offsets in [0, 1)
    dv: np.ndarray
    p0: np.ndarray      # first w-plane (0 in coplanar mode)
    dwo: np.ndarray     # p0 - tw
    inside: np.ndarray  # bool
    ul: np.ndarray
    vl: np.ndarray
    wl: np.ndarray

    @property
    def nplanes(self) -> int:
        return self.nw if self.nw > 0 else 1

    @property
    def wsupport(self) -> int:
        return self.Ww if self.nw > 0 else 1


def w_plane_params(wl: np.ndarray, nw: int, Ww: int):
    """w_min and plane spacing dw for N_w planes of kernel support W_w."""
    w_min = float(wl.min())
    w_max = float(wl.max())
    dw = (w_max - w_min) / (nw - Ww) if w_max > w_min else 1.0
    return w_min, dw


def geometry(uvw_m: np.ndarray, freq: np.ndarray, n: int, cell: float, W: int = 8,
             nw: int = 0, image_scale: int = 1, w_params=None) -> Geometry:
    """Per-sample grid geometry.  ``image_scale`` = 2 gives the 2N x 2N PSF
    image (grid 4N) over the same samples and w-planes."""
    s = freq / C_LIGHT
    ul = (uvw_m[:, 0:1] * s[None, :]).reshape(-1)
    vl = (uvw_m[:, 1:2] * s[None, :]).reshape(-1)
    wl = (uvw_m[:, 2:3] * s[None, :]).reshape(-1)
    nimg = n * image_scale
    ng = 2 * nimg
    scale = cell * ng
    half = ng / 2
    x = ul * scale + half
    y = vl * scale + half
    xs = x - W / 2
    ys = y - W / 2
    j0u = np.ceil(xs)
    j0v = np.ceil(ys)
    du = j0u - xs
    dv = j0v - ys
    j0u = j0u.astype(np.int64)
    j0v = j0v.astype(np.int64)
    inside = (j0u >= 0) & (j0u + W <= ng) & (j0v >= 0) & (j0v + W <= ng)
    Ww = W
    if nw > 0:
        w_min, dw = w_params if w_params is not None else w_plane_params(wl, nw, Ww)
        tw = (wl - w_min) / dw
        p0 = np.clip(np.ceil(tw), 0, nw - Ww)
        dwo = p0 - tw
        p0 = p0.astype(np.int64)
    else:
        w_min, dw = 0.0, 1.0
        p0 = np.zeros_like(j0u)
        dwo = np.zeros_like(du)
    return Geometry(nimg, ng, cell, W, nw, Ww, es.beta_for(W), w_min, dw, j0u, j0v, du, dv,
                    p0, dwo, inside, ul, vl, wl)


def _lmn(n, cell):
    off = (np.arange(n) - n // 2) * cell
    m, l = np.meshgrid(off, off, indexing="ij")
    r2 = l * l + m * m
    nn = np.sqrt(1.0 - r2)
    return nn, -r2 / (1.0 + nn)


def image_correction(g: Geometry) -> np.ndarray:
    """Real per-pixel factor 1 / (n Phi(a'/Ng) Phi(b'/Ng) Phi(dw (n-1)))."""
    n = g.n
    off = (np.arange(n) - n // 2) / g.ng
    ph1 = es.es_fourier(off, g.W, g.beta)
    c = 1.0 / np.outer(ph1, ph1)
    if g.nw > 0:
        nn, nm1 = _lmn(n, g.cell)
        c = c / (nn * es.es_fourier(g.dw * nm1, g.Ww, g.beta))
    return c


def plane_w(g: Geometry, p: int) -> float:
    return g.w_min + (p - g.Ww / 2) * g.dw


def _pad_center(z: np.ndarray, ng: int) -> np.ndarray:
    n = z.shape[0]
    out = np.zeros((ng, ng), dtype=np.complex128)
    o = ng // 2 - n // 2
    out[o:o + n, o:o + n] = z
    return out


def model_planes(image: np.ndarray, g: Geometry) -> np.ndarray:
    """Forward half of a4: correction, phase screen, zero-pad, FFT (centred)."""
    corr = image * image_correction(g)
    planes = np.empty((g.nplanes, g.ng, g.ng), dtype=np.complex128)
    if g.nw > 0:
        _, nm1 = _lmn(g.n, g.cell)
    for p in range(g.nplanes):
        z = corr.astype(np.complex128)
        if g.nw > 0:
            z = z * np.exp(-2j * np.pi * plane_w(g, p) * nm1)
        planes[p] = np.fft.fftshift(_fft.fft2(np.fft.ifftshift(_pad_center(z, g.ng)), workers=FFT_WORKERS))
    return planes


def planes_to_image(planes: np.ndarray, g: Geometry) -> np.ndarray:
    """Adjoint of ``model_planes``: F^H, crop, conjugate phase, sum, Re, correct."""
    acc = np.zeros((g.n, g.n), dtype=np.complex128)
    o = g.ng // 2 - g.n // 2
    if g.nw > 0:
        _, nm1 = _lmn(g.n, g.cell)
    for p in range(g.nplanes):
        z = np.fft.fftshift(_fft.ifft2(np.fft.ifftshift(planes[p]), workers=FFT_WORKERS)) * (g.ng * g.ng)
        z = z[o:o + g.n, o:o + g.n]
        if g.nw > 0:
            z = z * np.exp(2j * np.pi * plane_w(g, p) * nm1)
        acc += z
    return acc.real * image_correction(g)


def _weights(g: Geometry, sel: np.ndarray):
    W = g.W
    ar = np.arange(W)
    wu = es.es_kernel((g.du[sel][:, None] + ar) * (2.0 / W) - 1.0, g.beta)
    wv = es.es_kernel((g.dv[sel][:, None] + ar) * (2.0 / W) - 1.0, g.beta)
    if g.nw > 0:
        ww = es.es_kernel((g.dwo[sel][:, None] + np.arange(g.Ww)) * (2.0 / g.Ww) - 1.0, g.beta)
    else:
        ww = np.ones((sel.shape[0], 1))
    return wu, wv, ww


def _taps(g: Geometry, sel: np.ndarray):
    ar = np.arange(g.W)
    iu = g.j0u[sel][:, None] + ar
    iv = g.j0v[sel][:, None] + ar
    ip = g.p0[sel][:, None] + np.arange(g.wsupport)
    return ip, iv, iu


def degrid_planes(planes: np.ndarray, g: Geometry, chunk: int = 4096) -> np.ndarray:
    """V_k = sum_p phi_w sum_{j,i} phi_v phi_u G_p[j, i] for inside samples
    (0 elsewhere)."""
    idx = np.nonzero(g.inside)[0]
    out = np.zeros(g.j0u.shape[0], dtype=np.complex128)
    for c0 in range(0, idx.shape[0], chunk):
        sel = idx[c0:c0 + chunk]
        wu, wv, ww = _weights(g, sel)
        ip, iv, iu = _taps(g, sel)
        vals = planes[ip[:, :, None, None], iv[:, None, :, None], iu[:, None, None, :]]
        wt = ww[:, :, None, None] * wv[:, None, :, None] * wu[:, None, None, :]
        out[sel] = (vals * wt).sum(axis=(1, 2, 3))
    return out


def grid_planes(y: np.ndarray, g: Geometry, chunk: int = 4096) -> np.ndarray:
    """Adjoint of ``degrid_planes``: accumulate y_k * weights onto the planes."""
    planes = np.zeros((g.nplanes, g.ng, g.ng), dtype=np.complex128)
    flat = planes.reshape(-1)
    idx = np.nonzero(g.inside)[0]
    for c0 in range(0, idx.shape[0], chunk):
        sel = idx[c0:c0 + chunk]
        wu, wv, ww = _weights(g, sel)
        ip, iv, iu = _taps(g, sel)
        lin = (ip[:, :, None, None] * g.ng + iv[:, None, :, None]) * g.ng + iu[:, None, None, :]
        wt = ww[:, :, None, None] * wv[:, None, :, None] * wu[:, None, None, :]
        val = y[sel][:, None, None, None] * wt
        np.add.at(flat, lin.reshape(-1), val.reshape(-1))
    return planes


def degrid(image: np.ndarray, g: Geometry) -> np.ndarray:
    return degrid_planes(model_planes(image, g), g)


def grid_adjoint(y: np.ndarray, g: Geometry) -> np.ndarray:
    """Unnormalised adjoint Re(G^H y) on the N x N image."""
    return planes_to_image(grid_planes(y, g), g)


def dirty(vis: np.ndarray, weight: np.ndarray, g: Geometry) -> np.ndarray:
    wsum = weight[g.inside].sum()
    y = np.where(g.inside, weight * vis, 0.0)
    return grid_adjoint(y, g) / wsum


def residual(vis: np.ndarray, weight: np.ndarray, model: np.ndarray, g: Geometry) -> np.ndarray:
    """Eq. 2: F^H G (v - G^H F x), weighted and normalised by the weight sum."""
    r = vis - degrid(model, g)
    return dirty(r, weight, g)


def psf(weight: np.ndarray, g_psf: Geometry) -> np.ndarray:
    """2N x 2N PSF: grid the weights (unit visibilities), normalise by sum(w)."""
    return dirty(np.ones(weight.shape, dtype=np.complex128), weight, g_psf)


def subset(g: Geometry, keep: np.ndarray) -> Geometry:
    """Geometry restricted to a boolean sample selection (others dropped)."""
    return dataclasses.replace(g, inside=g.inside & keep)
