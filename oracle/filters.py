"""Fourier-domain filters Gamma_p and the padded convolutions of Eq. 4-7.

Every N x N image operator of the minor cycles (the PSF convolution H, the
filters Gamma, the scale functions B_s) acts on the 2N x 2N zero-padded grid:
the image is placed centred, transformed with a centred FFT (frequency index
j <-> k = j - N), multiplied by a spectrum, transformed back and cropped.
For the 2N x 2N PSF (centre at pixel (N, N)) this is the exact linear
convolution, since every offset between two pixels of an N x N image lies in
(-N, N).

Gamma_p (Sec. 4.1: each filter keeps its partition's spatial frequencies and
"the weights in L cap H sum to one"; its shape is not given): radial masks of
r = |k| / 2 (the radius in pixels of the N-grid's Fourier plane, the unit of
ell and delta), built from the ramps
    Lambda_i(r) = clip((ell_i + delta - r) / (2 delta), 0, 1),
    Lambda_0 = 0, Lambda_P = 1,   Gamma_p = Lambda_{p+1} - Lambda_p,
so that sum_p Gamma_p = 1 everywhere, Gamma_p = 1 inside its own ring and 0
outside its ring widened by delta.  For P = 2: Gamma_L = Lambda_1 and
Gamma_H = 1 - Gamma_L.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as _fft   # the 2D FFT primitive

# host threads of each 2D FFT (-1 = all); a caller running several oracle
# processes side by side sets 1
FFT_WORKERS = -1


def radius_grid(n: int) -> np.ndarray:
    """r = |k| / 2 on the centred 2N x 2N frequency grid."""
    k = np.arange(2 * n) - n
    ky, kx = np.meshgrid(k, k, indexing="ij")
    return np.sqrt((kx * kx + ky * ky).astype(np.float64)) / 2.0


def gammas(n: int, ells: np.ndarray, delta: float, nparts: int) -> np.ndarray:
    r = radius_grid(n)
    lam = [np.zeros_like(r)]
    for i in range(nparts - 1):
        lam.append(np.clip((ells[i] + delta - r) / (2.0 * delta), 0.0, 1.0))
    lam.append(np.ones_like(r))
    return np.stack([lam[p + 1] - lam[p] for p in range(nparts)])


def pad(x: np.ndarray) -> np.ndarray:
    n = x.shape[0]
    out = np.zeros((2 * n, 2 * n), dtype=np.complex128)
    out[n // 2:n // 2 + n, n // 2:n // 2 + n] = x
    return out


def crop(z: np.ndarray) -> np.ndarray:
    n = z.shape[0] // 2
    return z[n // 2:n // 2 + n, n // 2:n // 2 + n]


def spectrum(z2n: np.ndarray) -> np.ndarray:
    """Centred FFT of a 2N x 2N array whose centre is at index (N, N)."""
    return np.fft.fftshift(_fft.fft2(np.fft.ifftshift(z2n), workers=FFT_WORKERS))


def ispectrum(s: np.ndarray) -> np.ndarray:
    return np.fft.fftshift(_fft.ifft2(np.fft.ifftshift(s), workers=FFT_WORKERS))


def image_spectrum(x: np.ndarray) -> np.ndarray:
    return spectrum(pad(x))


def apply(x: np.ndarray, spec: np.ndarray) -> np.ndarray:
    """crop(F^-1(spec . F pad x)), real part."""
    return crop(ispectrum(spec * image_spectrum(x))).real


def psf_spectrum(psf2n: np.ndarray) -> np.ndarray:
    return spectrum(psf2n.astype(np.complex128))


# ---- band-limited exchange (Sec. 6.3, Sec. 7 item a) ------------------------
# Phi_p = crop F^-1 [Gamma_p F pad i_bar_p] is the crop of an image whose
# spectrum vanishes wherever Gamma_p does, and i_bar_p is real, so its
# spectrum is Hermitian: the coefficients of Gamma_p F pad i_bar_p on the
# ring support of Gamma_p in the half plane k_u <= 0 (centred index ju <= N,
# both halves of the self-mirrored columns ju = 0 and ju = N) determine
# Phi_p.  A receiver that scatters them back, completes the other half by
# conjugation, transforms and crops recovers Phi_p without loss.

def ring_support(gam_p: np.ndarray) -> np.ndarray:
    """Flat u-major indices ju * 2N + jv, ascending, of the half plane
    ju <= N where Gamma_p > 0."""
    n2 = gam_p.shape[0]
    mask = np.zeros_like(gam_p, dtype=bool)
    mask[: n2 // 2 + 1] = gam_p[: n2 // 2 + 1] > 0.0
    return np.nonzero(mask.reshape(-1))[0]


def phi_pack(ibar: np.ndarray, gam_p: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """The exchanged coefficients: Gamma_p F pad i_bar at the support."""
    return (gam_p * image_spectrum(ibar)).reshape(-1)[idx]


def phi_unpack(coef: np.ndarray, idx: np.ndarray, n: int) -> np.ndarray:
    """Phi = crop F^-1 of the spectrum rebuilt from the coefficients and
    their conjugate mirrors k -> -k (centred index j -> 2N - j mod 2N)."""
    n2 = 2 * n
    spec = np.zeros(n2 * n2, dtype=np.complex128)
    spec[idx] = coef
    spec = spec.reshape(n2, n2)
    ju, jv = np.divmod(idx, n2)
    mirror = (ju > 0) & (ju < n)
    spec[(n2 - ju[mirror]) % n2, (n2 - jv[mirror]) % n2] = np.conj(coef[mirror])
    return crop(ispectrum(spec)).real
