"""Seeded synthetic interferometric observations.

This module only produces inputs: antenna layouts, Earth-rotation uvw tracks,
a sky model (point sources and elliptical Gaussians), analytic visibilities of
that sky and Gaussian noise.  It holds none of the reconstruction arithmetic
(no gridding, no FFT, no partitioning, no deconvolution); both the CUDA path
and the CPU oracle consume what it returns.

Geometry: antennas in local East-North-Up on a plane at latitude -30 deg,
uvw from the standard hour-angle / declination rotation of the equatorial
baseline vector (Thompson, Moran & Swenson, "Interferometry and Synthesis in
Radio Astronomy", ch. 4).  Rows are time-major: for each time, every baseline
(i < j) in lexicographic order.

Visibilities follow the measurement equation of Eq. 1 with C = D = 1: a point
of flux S at direction cosines (l, m) contributes S/n exp(-2 pi i (u l + v m +
w (n - 1))) when the w-term is kept, S exp(-2 pi i (u l + v m)) when it is
dropped (coplanar configurations).  A Gaussian contributes its closed-form
Fourier transform times the phase term at its centre.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

C_LIGHT = 299792458.0
ARCSEC = math.pi / (180.0 * 3600.0)
DEG = math.pi / 180.0


@dataclasses.dataclass
class Sky:
    """Sky model.  Point and Gaussian positions are pixel offsets from the
    phase centre (column offset ``dx`` along l, row offset ``dy`` along m)."""
    pt_dx: np.ndarray
    pt_dy: np.ndarray
    pt_flux: np.ndarray
    g_dx: np.ndarray
    g_dy: np.ndarray
    g_flux: np.ndarray
    g_fwhm_a: np.ndarray   # pixels
    g_fwhm_b: np.ndarray   # pixels
    g_pa: np.ndarray       # radians


@dataclasses.dataclass
class Observation:
    name: str
    n: int                 # image side N
    cell_rad: float        # pixel size (radians)
    n_wplanes: int         # 0 = coplanar imaging
    uvw: np.ndarray        # (nrow, 3) float64, metres
    freq: np.ndarray       # (nchan,) float64, Hz
    vis: np.ndarray        # (nrow, nchan) complex128
    weight: np.ndarray     # (nrow, nchan) float32
    sky: Sky
    noise_sigma: float

    @property
    def nrow(self) -> int:
        return self.uvw.shape[0]

    @property
    def nchan(self) -> int:
        return self.freq.shape[0]

    @property
    def nvis(self) -> int:
        return self.nrow * self.nchan


# --------------------------------------------------------------------------
# Layouts and tracks
# --------------------------------------------------------------------------
def layout_disk(rng: np.random.Generator, n_ant: int, radius_m: float) -> np.ndarray:
    """Antennas uniform-random in a disk (ENU metres, U = 0)."""
    r = radius_m * np.sqrt(rng.random(n_ant))
    th = 2.0 * np.pi * rng.random(n_ant)
    return np.stack([r * np.cos(th), r * np.sin(th), np.zeros(n_ant)], axis=1)


def layout_log_spiral(rng: np.random.Generator, n_ant: int, r_min: float,
                      r_max: float, arms: int = 3) -> np.ndarray:
    """Antennas on a logarithmic spiral with ``arms`` arms, radii log-spaced
    from ``r_min`` to ``r_max``, plus a small random jitter."""
    per_arm = int(math.ceil(n_ant / arms))
    pos = []
    for a in range(arms):
        radii = np.geomspace(r_min, r_max, per_arm)
        th = 2.0 * np.pi * a / arms + 1.2 * np.log(radii / r_min)
        for r, t in zip(radii, th):
            pos.append((r * math.cos(t), r * math.sin(t)))
    pos = np.array(pos[:n_ant])
    pos += rng.normal(0.0, 0.01 * r_min, pos.shape)
    return np.concatenate([pos, np.zeros((n_ant, 1))], axis=1)


def baselines(n_ant: int) -> tuple[np.ndarray, np.ndarray]:
    i, j = np.triu_indices(n_ant, k=1)
    return i, j


def uvw_tracks(enu: np.ndarray, lat_rad: float, dec_rad: float,
               ha_rad: np.ndarray) -> np.ndarray:
    """uvw (metres) of every baseline at every hour angle, time-major rows."""
    a1, a2 = baselines(enu.shape[0])
    b = enu[a2] - enu[a1]                                  # ENU baseline vectors
    e, nn, uu = b[:, 0], b[:, 1], b[:, 2]
    sl, cl = math.sin(lat_rad), math.cos(lat_rad)
    x = -sl * nn + cl * uu                                 # equatorial frame
    y = e
    z = cl * nn + sl * uu
    sd, cd = math.sin(dec_rad), math.cos(dec_rad)
    h = ha_rad[:, None]
    sh, ch = np.sin(h), np.cos(h)
    u = sh * x + ch * y
    v = -sd * ch * x + sd * sh * y + cd * z
    w = cd * ch * x - cd * sh * y + sd * z
    return np.stack([u, v, w], axis=-1).reshape(-1, 3)


# --------------------------------------------------------------------------
# Sky
# --------------------------------------------------------------------------
def make_sky(rng: np.random.Generator, n: int, n_pts: int, n_gauss: int,
             pts_flux: str, fwhm_range=(3.0, 8.0)) -> Sky:
    """Point positions are pixel centres drawn uniformly over the inner 80 %
    of the field; Gaussian centres likewise.  ``pts_flux`` is ``"loguniform"``
    (0.01-1 Jy) or ``"powerlaw"`` (dN/dS ~ S^-1.6 on [1e-3, 1] Jy, inverse
    CDF)."""
    half = int(0.4 * n)
    pdx = rng.integers(-half, half, n_pts).astype(np.float64)
    pdy = rng.integers(-half, half, n_pts).astype(np.float64)
    if pts_flux == "loguniform":
        pf = np.exp(rng.uniform(np.log(0.01), np.log(1.0), n_pts))
    else:
        # dN/dS ~ S^-1.6 on [a, b]: CDF ~ S^-0.6
        a, b, k = 1e-3, 1.0, -0.6
        uu = rng.random(n_pts)
        pf = (a ** k + uu * (b ** k - a ** k)) ** (1.0 / k)
    gdx = rng.integers(-half, half, n_gauss).astype(np.float64)
    gdy = rng.integers(-half, half, n_gauss).astype(np.float64)
    gf = np.exp(rng.uniform(np.log(0.01), np.log(1.0), n_gauss))
    fa = rng.uniform(*fwhm_range, n_gauss)
    fb = rng.uniform(*fwhm_range, n_gauss)
    pa = rng.uniform(0.0, np.pi, n_gauss)
    return Sky(pdx, pdy, pf, gdx, gdy, gf, fa, fb, pa)


def sky_image(sky: Sky, n: int) -> np.ndarray:
    """Ground-truth image (Jy/pixel), row = m index, column = l index, phase
    centre at pixel (n/2, n/2).  Gaussians are sampled at pixel centres and
    scaled to their total flux."""
    img = np.zeros((n, n))
    c = n // 2
    for dx, dy, f in zip(sky.pt_dx, sky.pt_dy, sky.pt_flux):
        img[c + int(dy), c + int(dx)] += f
    yy, xx = np.mgrid[0:n, 0:n]
    for dx, dy, f, fa, fb, pa in zip(sky.g_dx, sky.g_dy, sky.g_flux,
                                     sky.g_fwhm_a, sky.g_fwhm_b, sky.g_pa):
        sa = fa / (2.0 * math.sqrt(2.0 * math.log(2.0)))
        sb = fb / (2.0 * math.sqrt(2.0 * math.log(2.0)))
        x = xx - (c + dx)
        y = yy - (c + dy)
        xr = x * math.cos(pa) + y * math.sin(pa)
        yr = -x * math.sin(pa) + y * math.cos(pa)
        g = np.exp(-0.5 * ((xr / sa) ** 2 + (yr / sb) ** 2))
        img += f * g / g.sum()
    return img


def _visibilities(uvw_m: np.ndarray, freq: np.ndarray, sky: Sky,
                  cell_rad: float, wterm: bool, chunk: int = 1 << 15) -> np.ndarray:
    """Analytic visibilities of ``sky`` (FP64)."""
    nrow = uvw_m.shape[0]
    out = np.zeros((nrow, freq.shape[0]), dtype=np.complex128)
    to_sig = cell_rad / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    groups = []
    for dx, dy, fl, fa, fb, pa in (
            (sky.pt_dx, sky.pt_dy, sky.pt_flux, None, None, None),
            (sky.g_dx, sky.g_dy, sky.g_flux, sky.g_fwhm_a, sky.g_fwhm_b, sky.g_pa)):
        if dx.shape[0] == 0:
            continue
        ls, ms = dx * cell_rad, dy * cell_rad
        nn = np.sqrt(1.0 - ls ** 2 - ms ** 2)
        amp = fl / nn if wterm else fl.copy()
        shape = None if fa is None else (fa * to_sig, fb * to_sig, pa)
        groups.append((ls, ms, nn, amp, shape))
    # The per-(row, source) phase sums run as multithreaded FP64 tensor ops on
    # the host (torch CPU); numpy's complex exp is an order of magnitude slower.
    for r0 in range(0, nrow, chunk):
        r1 = min(nrow, r0 + chunk)
        u_m = torch.from_numpy(np.ascontiguousarray(uvw_m[r0:r1, 0]))
        v_m = torch.from_numpy(np.ascontiguousarray(uvw_m[r0:r1, 1]))
        w_m = torch.from_numpy(np.ascontiguousarray(uvw_m[r0:r1, 2]))
        for ls, ms, nn, amp, shape in groups:
            ls_t, ms_t = torch.from_numpy(ls), torch.from_numpy(ms)
            amp_t = torch.from_numpy(amp)
            # geometric delay per (row, source), metres
            delay = torch.outer(u_m, ls_t) + torch.outer(v_m, ms_t)
            if wterm:
                delay += torch.outer(w_m, torch.from_numpy(nn - 1.0))
            for c, f in enumerate(freq):
                k = f / C_LIGHT
                ph = (-2.0 * math.pi * k) * delay
                re, im = torch.cos(ph), torch.sin(ph)
                if shape is not None:
                    # FT of a unit-flux elliptical Gaussian with axes rotated by
                    # pa: exp(-2 pi^2 (sa^2 ua^2 + sb^2 ub^2))
                    sa, sb, pa = (torch.from_numpy(a) for a in shape)
                    ua = k * (torch.outer(u_m, torch.cos(pa)) + torch.outer(v_m, torch.sin(pa)))
                    ub = k * (torch.outer(-u_m, torch.sin(pa)) + torch.outer(v_m, torch.cos(pa)))
                    env = torch.exp(-2.0 * math.pi ** 2 * (sa ** 2 * ua ** 2 + sb ** 2 * ub ** 2))
                    re, im = re * env, im * env
                out[r0:r1, c] += (re @ amp_t).numpy() + 1j * (im @ amp_t).numpy()
    return out


def _observe(name, rng_layout, rng_sky, rng_noise, enu, n_times, ha_span_h,
             freq, n, cell_arcsec, n_wplanes, n_pts, n_gauss, pts_flux, sigma,
             dec_deg=-30.0, lat_deg=-30.0, with_vis=True) -> Observation:
    freq = np.asarray(freq, dtype=np.float64)
    ha = np.linspace(-0.5 * ha_span_h, 0.5 * ha_span_h, n_times) * (15.0 * DEG)
    uvw = uvw_tracks(enu, lat_deg * DEG, dec_deg * DEG, ha)
    cell = cell_arcsec * ARCSEC
    sky = make_sky(rng_sky, n, n_pts, n_gauss, pts_flux)
    if with_vis:
        vis = _visibilities(uvw, freq, sky, cell, wterm=n_wplanes > 0)
        noise = rng_noise.normal(0.0, sigma, vis.shape) + 1j * rng_noise.normal(0.0, sigma, vis.shape)
        vis = vis + noise
    else:
        # geometry only (operator tests that bring their own visibilities)
        vis = np.zeros((uvw.shape[0], freq.shape[0]), dtype=np.complex128)
    weight = np.ones(vis.shape, dtype=np.float32)
    return Observation(name, n, cell, n_wplanes, uvw, freq,
                       vis, weight, sky, sigma)


def _streams(seed: int):
    ss = np.random.SeedSequence(seed)
    a, b, c = ss.spawn(3)
    return (np.random.Generator(np.random.PCG64(a)), np.random.Generator(np.random.PCG64(b)),
            np.random.Generator(np.random.PCG64(c)))


def plain_small(seed: int = 0) -> Observation:
    """128x128 at 2", one channel at 1.4 GHz, coplanar; 32 antennas uniform in
    a 1 km disk, 496 baselines x 40 times over 4 h at dec -30 deg = 19,840
    visibilities; 10 points (log-uniform 0.01-1 Jy) + 2 Gaussians; noise
    sigma 0.01 Jy."""
    rl, rs, rn = _streams(seed)
    enu = layout_disk(rl, 32, 1000.0)
    return _observe("plain_small_128", rl, rs, rn, enu, 40, 4.0, [1.4e9], 128, 2.0, 0,
                    10, 2, "loguniform", 0.01)


def medium(seed: int = 1, n_times: int = 1000, n: int = 1024, n_wplanes: int = 16,
           n_ant: int = 64, n_chan: int = 4, with_vis: bool = True) -> Observation:
    """1024x1024 at 1", 64 antennas on a 3-arm log spiral 50 m - 5 km (2016
    baselines) x 1000 times x 4 channels over 1.3-1.5 GHz = 8.06 M
    visibilities, 16 w-planes; 200 points (power-law counts) + 20 Gaussians;
    noise sigma 1e-3 Jy.  Smaller ``n_times`` / ``n`` / ``n_ant`` give the same
    recipe (same 1" cell, smaller field) at reduced size for parity tests."""
    rl, rs, rn = _streams(seed)
    enu = layout_log_spiral(rl, n_ant, 50.0, 5000.0)
    freq = np.linspace(1.3e9, 1.5e9, n_chan)
    cell = 1.0
    return _observe(f"medium_{n}", rl, rs, rn, enu, n_times, 4.0, freq, n, cell, n_wplanes,
                    200, 20, "powerlaw", 1e-3, with_vis=with_vis)


def large(seed: int = 3, n_times: int = 4000, n: int = 4096, n_wplanes: int = 32,
          n_chan: int = 8, with_vis: bool = True) -> Observation:
    """4096x4096 at 0.5", 128 antennas on a 10 km log spiral (8128
    baselines) x 4000 times x 8 channels = 260 M visibilities, 32 w-planes;
    2000 points + 100 Gaussians; noise sigma 5e-4 Jy."""
    rl, rs, rn = _streams(seed)
    enu = layout_log_spiral(rl, 128, 50.0, 10000.0)
    freq = np.linspace(1.3e9, 1.5e9, n_chan)
    cell = 0.5
    return _observe(f"large_{n}", rl, rs, rn, enu, n_times, 4.0, freq, n, cell, n_wplanes,
                    2000, 100, "powerlaw", 5e-4, with_vis=with_vis)


def batch_chunk_jobs(n_jobs: int = 64, base_seed: int = 1000, n_min: float = 0.5e6, n_max: float = 8e6,
                     sizes=(256, 512, 1024, 2048), n_ant: int = 64, n_chan: int = 4,
                     with_vis: bool = True) -> list[Observation]:
    """The batching workload: n_jobs independent channel-chunk jobs, job j
    the medium recipe's generator with its own seed base_seed + j, its
    visibility count log-uniform in [n_min, n_max] (the time samples scaled
    to reach it) and its image side drawn from `sizes` (1" cells, 16
    w-planes)."""
    out = []
    nbl = n_ant * (n_ant - 1) // 2
    for j in range(n_jobs):
        rng = np.random.default_rng(base_seed + j)
        nvis = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        n = int(rng.choice(np.asarray(sizes)))
        n_times = max(2, int(round(nvis / (nbl * n_chan))))
        out.append(medium(seed=base_seed + j, n_times=n_times, n=n, n_ant=n_ant, n_chan=n_chan, with_vis=with_vis))
    return out
