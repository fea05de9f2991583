"""Crack initiation and propagation (Sec. 2.4).

AT2 hybrid phase field (Eq. crack):
  -(Gc l0 / 2) div grad d + (Gc / (2 l0)) d + H d = H,
with the history field H = max over time of psi+ (Sec. 2.4) and the
degradation g(d) = (1 - d)^2 + kappa of the stiffness.

Eq. (crack-fft) applies the Laplacian in Fourier space through the symbol
"i xi . i xi". With the forward-difference gradient of Sec. 2.6 this is read
as -sum_alpha |D_alpha|^2 (minus the squared modulus of the gradient symbol,
the Galerkin product grad+^T grad+ of the weak form), which keeps the
operator symmetric positive definite; the paper's GMRES and this CG then reach
the same unique solution.
"""

import numpy as np

from . import spectral
from .krylov import cg, gmres


def coefficients(mat):
    """a = Gc / (2 l0) (reaction), b = Gc l0 / 2 (gradient), Eq. (crack)."""
    return mat.Gc / (2.0 * mat.l0), mat.Gc * mat.l0 / 2.0


def history_update(H_prev, psi_plus):
    """H = max(H_prev, psi+) (Sec. 2.4)."""
    return np.maximum(H_prev, psi_plus)


def degradation(d, kappa):
    """g(d) = (1 - d)^2 + kappa (Sec. 2.4)."""
    return (1.0 - d) ** 2 + kappa


def phasefield_solve(H, mat, h, tol=1e-12, max_iter=200000, d0=None, symbol="forward", literal=False):
    """Solve Eq. (crack-fft) for d given the history field H. symbol: the
    gradient operator of Sec. 2.6 (spectral.SYMBOLS; the paper's results use
    the forward difference). literal: the Laplacian as printed, "i xi . i
    xi" read as sum_alpha D_alpha^2 (not symmetric under a difference
    operator), solved by GMRES as the paper does, with the Galerkin
    operator's diagonal 1 / (a + <H> + b |D|^2) as right preconditioner."""
    H = np.asarray(H, dtype=np.float64)
    a, b = coefficients(mat)
    D = spectral.SYMBOLS[symbol](H.shape, h)
    lam = spectral.symbol_norm2(D)
    if literal:
        DD = sum(Da * Da for Da in D)

        def A_lit(x):
            return -b * spectral.ifft(DD * spectral.fft(x)).real + a * x + H * x

        m0 = a + H.mean()

        def M(v):
            return spectral.ifft(spectral.fft(v) / (m0 + b * lam)).real

        d, info = gmres(A_lit, H.copy(), tol=tol, max_iter=max_iter, apply_M=M)
        return d, info

    def A(x):
        lap = spectral.ifft(-lam * spectral.fft(x)).real  # F^-1(i xi . i xi x_hat)
        return -b * lap + a * x + H * x

    d, info = cg(A, H.copy(), x0=d0, tol=tol, max_iter=max_iter)
    return d, info
