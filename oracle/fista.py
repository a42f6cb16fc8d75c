"""Sparsity-regularised minor cycle (Eq. 4 and Eq. 5) solved by FISTA.

Objective of node p at major cycle n (Eq. 5, P partitions; Eq. 4 when P = 1):
    f(x) = || Gamma_p (i_p - H_p x) ||^2 + gamma_n sum_{q != p} || rho_q - Gamma_q x ||^2,
    x = W alpha,   minimise f(W alpha) + lambda ||alpha||_1,
gamma_n = 0 at n = 1 and 1 afterwards.  Reading of the operators: H_p and
Gamma_q act on the 2N-padded grid and the norms are taken over that grid, so
in terms of centred spectra (X = F pad x, I_p = F pad i_p, R_q = F pad rho_q,
M = (2N)^2 points)
    f(x) = (1/M) sum_k [ Gamma_p^2 |I_p - H_p X|^2 + gamma_n sum_q |R_q - Gamma_q X|^2 ],
    grad f(x) = 2 crop F^-1 [ Mx X - C ],
    Mx = Gamma_p^2 |H_p|^2 + gamma_n sum_q Gamma_q^2,
    C  = Gamma_p^2 conj(H_p) I_p + gamma_n sum_q Gamma_q R_q,
and L = 2 max_k Mx bounds the Lipschitz constant (W orthonormal).

FISTA (Beck & Teboulle 2009), in coefficient space, alpha_0 = y_0 = 0, t_0 = 1:
    alpha_{k+1} = S_{lambda/L}( y_k - W^T grad f(W y_k) / L )
    t_{k+1}     = (1 + sqrt(1 + 4 t_k^2)) / 2
    y_{k+1}     = alpha_{k+1} + ((t_k - 1) / t_{k+1}) (alpha_{k+1} - alpha_k)
stopping after a fixed number of iterations (50 per major cycle, Sec. 5.2);
the deconvolved residual is i_bar = W alpha.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import filters, wavelet


@dataclasses.dataclass
class Problem:
    mx: np.ndarray       # real spectrum multiplying X
    c: np.ndarray        # complex constant spectrum
    const: float         # (1/M) sum of the constant part of f (for objective values)
    n: int

    @property
    def lipschitz(self) -> float:
        return 2.0 * float(self.mx.max())

    def grad(self, x: np.ndarray) -> np.ndarray:
        X = filters.image_spectrum(x)
        return 2.0 * filters.crop(filters.ispectrum(self.mx * X - self.c)).real

    def data_term(self, x: np.ndarray) -> float:
        X = filters.image_spectrum(x)
        m = (2 * self.n) ** 2
        # f = (1/M) sum [Mx |X|^2 - 2 Re(conj(X) C)] + const
        return float((np.sum(self.mx * np.abs(X) ** 2) - 2.0 * np.sum((np.conj(X) * self.c).real)) / m
                     + self.const)


def problem(i_spec: np.ndarray, h_spec: np.ndarray, gam_p: np.ndarray,
            others: list[tuple[np.ndarray, np.ndarray]], gamma_n: float) -> Problem:
    """``others`` = [(Gamma_q, R_q)] for the received aggregates."""
    n = i_spec.shape[0] // 2
    mx = gam_p ** 2 * np.abs(h_spec) ** 2
    c = gam_p ** 2 * np.conj(h_spec) * i_spec
    const = np.sum(gam_p ** 2 * np.abs(i_spec) ** 2)
    for gq, rq in others:
        mx = mx + gamma_n * gq ** 2
        c = c + gamma_n * gq * rq
        const = const + gamma_n * np.sum(np.abs(rq) ** 2)
    return Problem(mx, c, float(const) / (2 * n) ** 2, n)


def soft(x: np.ndarray, t: float) -> np.ndarray:
    return np.sign(x) * np.maximum(np.abs(x) - t, 0.0)


def _operators(levels: int, dictionary):
    """(W, W^T, coefficient shape) of the Db4 basis (dictionary None) or of a
    wavelet.Concatenation."""
    if dictionary is None:
        return (lambda c: wavelet.idwt2(c, levels)), (lambda x: wavelet.dwt2(x, levels)), (lambda n: (n, n))
    return dictionary.synthesis, dictionary.analysis, dictionary.shape


def solve(prob: Problem, lam: float, n_iter: int, levels: int, accelerate: bool = True, dictionary=None):
    """Returns (i_bar, alpha).  ``dictionary``: None for the Db4 basis, or a
    wavelet.Concatenation (the tight frame keeps L = 2 max Mx a bound)."""
    n = prob.n
    L = prob.lipschitz
    W, WT, shape = _operators(levels, dictionary)
    alpha = np.zeros(shape(n))
    y = alpha.copy()
    t = 1.0
    for _ in range(n_iter):
        g = WT(prob.grad(W(y)))
        alpha_new = soft(y - g / L, lam / L)
        if accelerate:
            t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
            y = alpha_new + ((t - 1.0) / t_new) * (alpha_new - alpha)
            t = t_new
        else:
            y = alpha_new
        alpha = alpha_new
    return W(alpha), alpha


def objective(prob: Problem, alpha: np.ndarray, lam: float, levels: int, dictionary=None) -> float:
    W, _, _ = _operators(levels, dictionary)
    return prob.data_term(W(alpha)) + lam * float(np.abs(alpha).sum())
