"""Fourier-space gradient symbols and the compatibility projections.

Grid arrays are C-ordered with x fastest: shape (ny, nx) or (nz, ny, nx).
Direction alpha = 0, 1, 2 means x, y, z and lives on array axis
ndim - 1 - alpha. The FFT is numpy's: forward exp(-2 pi i j k / n),
unnormalised, inverse with 1/N.

Sec. 2.6 lists the gradient operators; the paper runs every result with the
forward difference, whose symbol is (exp(i xi_alpha Delta) - 1) / Delta. With
numpy's sign convention the mode k along an axis of n points has
xi_alpha Delta = 2 pi k / n and the symbol acts in real space as
(u(x + Delta e_alpha) - u(x)) / Delta on periodic fields.

App. A, Eq. (g-42): the inverse of the gradient symbol is
conj(D) / (D . conj(D)), taken as 0 where D . conj(D) = 0, and the
second-order projection is ghat_ij = D_i (D^-1)_j = D_i conj(D_j) / |D|^2.
The fourth-order projection applies ghat row-wise:
Ahat_ij = delta_im ghat_jl epshat_ml (App. A, second equation).
"""

import numpy as np


def direction_axis(alpha, ndim):
    """Array axis that carries spatial direction alpha (x = 0)."""
    return ndim - 1 - alpha


def phase_angles(shape):
    """theta_alpha = 2 pi k_alpha / n_alpha as broadcastable arrays, alpha = 0..d-1."""
    ndim = len(shape)
    out = []
    for alpha in range(ndim):
        ax = direction_axis(alpha, ndim)
        n = shape[ax]
        k = np.arange(n, dtype=np.float64)
        sh = [1] * ndim
        sh[ax] = n
        out.append((2.0 * np.pi * k / n).reshape(sh))
    return out


def forward_difference_symbol(shape, h):
    """D_alpha(k) = (exp(i theta_alpha) - 1) / h  (Sec. 2.6, forward difference)."""
    return [np.broadcast_to((np.exp(1j * th) - 1.0) / h, shape).copy()
            for th in phase_angles(shape)]


def fourier_symbol(shape, h):
    """The continuous Fourier gradient i xi_alpha (Sec. 2.6), with the
    wavenumber folded to (-n/2, n/2]; only used for operator comparisons."""
    ndim = len(shape)
    out = []
    for alpha in range(ndim):
        ax = direction_axis(alpha, ndim)
        n = shape[ax]
        k = np.fft.fftfreq(n, d=1.0 / n)
        sh = [1] * ndim
        sh[ax] = n
        out.append(np.broadcast_to(1j * 2 * np.pi * k.reshape(sh) / (n * h), shape).copy())
    return out


# Coefficients c_m of the 8th-order central first derivative
# u'(x) ~ sum_{m=1..4} c_m (u(x + m h) - u(x - m h)) / h: the solution of the
# moment conditions sum_m 2 m^(2j-1) c_m = delta_{j1}, j = 1..4 (Taylor
# expansion; the paper names the scheme without printing it, Sec. 2.6).
def central8_coefficients():
    A = np.array([[2.0 * m ** (2 * j - 1) for m in range(1, 5)] for j in range(1, 5)])
    return np.linalg.solve(A, np.array([1.0, 0.0, 0.0, 0.0]))


def central_difference_symbol(shape, h):
    """(u(x + h e_alpha) - u(x - h e_alpha)) / (2 h): symbol i sin(theta) / h
    (Sec. 2.6, the central difference; read as i sin(xi Delta) / Delta)."""
    return [np.broadcast_to(1j * np.sin(th) / h, shape).copy() for th in phase_angles(shape)]


def central8_symbol(shape, h):
    """The 8th-order central difference: i sum_m 2 c_m sin(m theta) / h."""
    c = central8_coefficients()
    return [np.broadcast_to(1j * sum(2.0 * c[m - 1] * np.sin(m * th) for m in range(1, 5)) / h, shape).copy()
            for th in phase_angles(shape)]


SYMBOLS = {"forward": forward_difference_symbol, "central": central_difference_symbol,
           "central8": central8_symbol, "fourier": fourier_symbol}


def symbol_norm2(D):
    """D . conj(D) = sum_alpha |D_alpha|^2 per mode (denominator of Eq. g-42)."""
    return sum((Da * np.conj(Da)).real for Da in D)


def gradient_inverse(D):
    """(i xi)^-1 of Eq. (g-42): conj(D_j) / (D . conj(D)), 0 where the
    denominator vanishes (the k = 0 mode)."""
    den = symbol_norm2(D)
    safe = np.where(den > 0, den, 1.0)
    return [np.where(den > 0, np.conj(Dj) / safe, 0.0) for Dj in D]


def projection_operator(D):
    """ghat[i][j] = D_i (D^-1)_j per mode (App. A): a d x d array of complex
    grids. Built explicitly, as the paper does."""
    Dinv = gradient_inverse(D)
    d = len(D)
    return [[D[i] * Dinv[j] for j in range(d)] for i in range(d)]


def fft(f):
    return np.fft.fftn(f)


def ifft(F):
    return np.fft.ifftn(F)


def apply_G(ghat, f):
    """Projection of a vector field f (shape (d, *grid)) onto periodic
    gradient fields: (G f)^_i = ghat_ij fhat_j (App. A, first equation)."""
    d = len(ghat)
    fh = [fft(f[j]) for j in range(d)]
    out = np.empty_like(f, dtype=np.float64)
    for i in range(d):
        acc = sum(ghat[i][j] * fh[j] for j in range(d))
        out[i] = ifft(acc).real
    return out


def apply_GG(ghat, A):
    """Fourth-order projection of a second-order tensor field A (shape
    (d, d, *grid), A[i, j] = d u_i / d x_j for a compatible field):
    (GG A)^_ij = delta_im ghat_jl Ahat_ml = ghat_jl Ahat_il (App. A)."""
    d = len(ghat)
    out = np.empty_like(A, dtype=np.float64)
    for i in range(d):
        Ah = [fft(A[i, l]) for l in range(d)]
        for j in range(d):
            acc = sum(ghat[j][l] * Ah[l] for l in range(d))
            out[i, j] = ifft(acc).real
    return out


def spectral_derivative(f, D):
    """F^-1(D_alpha F(f)) for each alpha: the gradient of a scalar field
    with the chosen symbol."""
    fh = fft(f)
    return np.stack([ifft(Da * fh).real for Da in D])


def solve_poisson_from_gradient(grad, D):
    """phi with grad phi = projection of `grad`: phihat = (D^-1) . gradhat
    (Alg. 1 fluctuation step, Eq. phi-fft with the inverse of Eq. g-42);
    zero mean."""
    Dinv = gradient_inverse(D)
    acc = sum(Dinv[j] * fft(grad[j]) for j in range(len(D)))
    return ifft(acc).real
