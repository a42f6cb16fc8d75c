"""The decentralized major/minor loop (Sec. 3-4, Fig. 2, Eq. 3, 5, 7).

Per major cycle n = 1, 2, ... and partition (node) p:
  major   i_p^n  = F^H G_p (v_p - G_p^H F model_p)        (Eq. 2, own visibilities)
  fill    from cycle 2 on, add the received filtered images of cycle n-1:
              rho_{q->p} += Phi_q^{n-1}
  minor   ms-CLEAN (Eq. 7) or FISTA (Eq. 5) on the pseudo-full-resolution
          problem built from i_p^n, the PSFs and rho_{q->p}; gives i_bar_p^n
  update  model_p += i_bar_p^n                             (Eq. 3)
          Phi_p^n  = Gamma_p i_bar_p^n                     (sent to every other node)
          rho_{q->p} -= Gamma_q i_bar_p^n                  (own half of Eq. 5's aggregate)
so that at cycle n, rho_{q->p} = sum_{j<n} Phi_q^j - Gamma_q sum_{j<n} i_bar_p^j
(Eq. 5, updated in place as Sec. 4.1 describes).  Final image: the equal-weight
mean of the node images (Sec. 5.2).

Readings (the paper is silent or garbled): gamma^n, mu^n of Eq. 7 are (1, 0) at
n = 1 and W_p / W, W_q / W afterwards (W_p = weight sum of partition p, W =
sum over partitions); lambda of FISTA is lam_rel * max |i_p^1| unless given.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import filters, fista, gridder, msclean, partition, wavelet, weighting


@dataclasses.dataclass
class Setup:
    n: int
    nparts: int
    ells: np.ndarray
    delta: float
    geom: gridder.Geometry
    mask: np.ndarray
    gparts: list
    wsum: np.ndarray
    psf: list            # 2N x 2N per partition
    hspec: list          # centred spectra of the PSFs
    gam: np.ndarray      # Gamma_p on the 2N grid
    weight: np.ndarray   # the weights imaged with (natural, or uniform per oracle.weighting)


def setup(uvw, freq, weight, n, cell, nw, nparts, delta=1.0, ells=None, W=8, scheme="natural") -> Setup:
    """``scheme``: "natural" (the given weights) or "uniform" (Sec. 5.1;
    oracle.weighting), applied before the partition's weight sums and PSFs."""
    g = gridder.geometry(uvw, freq, n, cell, W=W, nw=nw)
    if scheme == "uniform":
        weight = weighting.uniform_weights(g, weight).reshape(np.shape(weight))
    r = partition.radius_px(g)
    if ells is None:
        ells = partition.ring_radii(r, nparts)
    mask = partition.masks(r, np.asarray(ells, dtype=np.float64), delta, nparts, g.inside)
    gparts = [gridder.subset(g, ((mask >> p) & 1) == 1) for p in range(nparts)]
    gpsf = gridder.geometry(uvw, freq, n, cell, W=W, nw=nw, image_scale=2,
                            w_params=(g.w_min, g.dw))
    w = weight.reshape(-1).astype(np.float64)
    psfs, hs = [], []
    for p in range(nparts):
        gp = gridder.subset(gpsf, ((mask >> p) & 1) == 1)
        ps = gridder.psf(w, gp)
        psfs.append(ps)
        hs.append(filters.psf_spectrum(ps))
    wsum = partition.weight_sums(weight, mask, nparts)
    gam = filters.gammas(n, np.asarray(ells, dtype=np.float64), delta, nparts)
    return Setup(n, nparts, np.asarray(ells, dtype=np.float64), delta, g, mask, gparts, wsum,
                 psfs, hs, gam, np.asarray(weight))


class Loop:
    def __init__(self, st: Setup, vis: np.ndarray, weight: np.ndarray | None = None):
        """``weight`` None: the weights the setup images with (st.weight)."""
        self.st = st
        self.vis = vis.reshape(-1).astype(np.complex128)
        self.w = (st.weight if weight is None else weight).reshape(-1).astype(np.float64)
        P, n = st.nparts, st.n
        self.model = [np.zeros((n, n)) for _ in range(P)]
        self.rho = [[np.zeros((n, n)) for _ in range(P)] for _ in range(P)]   # rho[p][q]
        self.outbox = [np.zeros((n, n)) for _ in range(P)]
        self.inbox = [np.zeros((n, n)) for _ in range(P)]
        self.residual = [None] * P
        self.lam = [None] * P
        self.cycle = 0
        self.history = []          # (cycle, p, i_bar, Phi) for the explicit-sum pin

    # -- major cycle ---------------------------------------------------------
    def major(self, p: int) -> np.ndarray:
        self.residual[p] = gridder.residual(self.vis, self.w, self.model[p], self.st.gparts[p])
        return self.residual[p]

    # -- fill ------------------------------------------------------------------
    def _ingest(self, p: int, cycle: int):
        if cycle >= 2:
            for q in range(self.st.nparts):
                if q != p:
                    self.rho[p][q] = self.rho[p][q] + self.inbox[q]

    def gamma_mu(self, p: int, cycle: int):
        P = self.st.nparts
        if cycle == 1:
            return 1.0, np.zeros(P)
        tot = self.st.wsum.sum()
        return self.st.wsum[p] / tot, self.st.wsum / tot

    def msclean_problem(self, p: int, cycle: int):
        st = self.st
        g, mu = self.gamma_mu(p, cycle)
        ispec = filters.image_spectrum(self.residual[p])
        d = g * st.gam[p] * ispec
        ps = g * st.gam[p] * st.hspec[p]
        for q in range(st.nparts):
            if q == p or mu[q] == 0.0:
                continue
            d = d + mu[q] * st.hspec[q] * filters.image_spectrum(self.rho[p][q])
            ps = ps + mu[q] * st.gam[q] * st.hspec[q]
        return d, ps

    def fista_problem(self, p: int, cycle: int) -> fista.Problem:
        st = self.st
        gamma_n = 0.0 if cycle == 1 else 1.0
        others = [(st.gam[q], filters.image_spectrum(self.rho[p][q]))
                  for q in range(st.nparts) if q != p]
        return fista.problem(filters.image_spectrum(self.residual[p]), st.hspec[p], st.gam[p],
                             others, gamma_n)

    # -- minor cycles ------------------------------------------------------------
    def minor_msclean(self, p: int, cycle: int, scales, gain, niter, threshold):
        self._ingest(p, cycle)
        d, ps = self.msclean_problem(p, cycle)
        allowed = msclean.allowed_scales(scales, self.st.n, p, cycle, self.st.ells, self.st.delta)
        res = msclean.clean(d, ps, scales, gain, niter, threshold, allowed)
        self._publish(p, cycle, res.model)
        return res

    def minor_fista(self, p: int, cycle: int, lam_rel=1e-3, lam=None, n_iter=50, levels=4, dictionary="db4",
                    schedule=None):
        """lambda: ``lam`` if given; else with ``schedule`` = (a, b) the paper's
        lambda_n = a ||i_p^n||_2 b^n (Sec. 5.2; i_p^n the partition's residual
        image of this cycle, n the cycle number from 1); else lam_rel times
        max |i_p^1| of the partition's first residual.  ``dictionary``: "db4"
        or "sara" (db1 .. db8 concatenated)."""
        self._ingest(p, cycle)
        if lam is None and schedule is not None:
            a, b = schedule
            lam = a * float(np.linalg.norm(self.residual[p])) * b ** cycle
        if lam is None:
            if self.lam[p] is None:
                self.lam[p] = lam_rel * float(np.abs(self.residual[p]).max())
            lam = self.lam[p]
        prob = self.fista_problem(p, cycle)
        dic = None if dictionary == "db4" else wavelet.Concatenation(levels)
        ibar, alpha = fista.solve(prob, lam, n_iter, levels, dictionary=dic)
        self._publish(p, cycle, ibar)
        return ibar

    def _publish(self, p: int, cycle: int, ibar: np.ndarray):
        st = self.st
        self.model[p] = self.model[p] + ibar                    # Eq. 3
        phi = filters.apply(ibar, st.gam[p])                    # Phi_p = Gamma_p i_bar_p
        self.outbox[p] = phi
        for q in range(st.nparts):
            if q != p:
                self.rho[p][q] = self.rho[p][q] - filters.apply(ibar, st.gam[q])
        self.history.append((cycle, p, ibar, phi))

    def exchange(self):
        """End of a major cycle: every node's outbox becomes visible."""
        self.inbox = [o.copy() for o in self.outbox]

    def combine(self) -> np.ndarray:
        return sum(self.model) / self.st.nparts


def run(st: Setup, vis, weight, n_major: int, method: str, **params):
    loop = Loop(st, vis, weight)
    for c in range(1, n_major + 1):
        for p in range(st.nparts):
            loop.major(p)
        for p in range(st.nparts):
            if method == "msclean":
                loop.minor_msclean(p, c, **params)
            else:
                loop.minor_fista(p, c, **params)
        loop.exchange()
    return loop


def snr_db(truth: np.ndarray, est: np.ndarray) -> float:
    """Sec. 6.1: 10 log10(||i|| / ||i - i_hat||) (the paper's revised factor)."""
    return 10.0 * np.log10(np.linalg.norm(truth) / np.linalg.norm(truth - est))
