"""Ionic diffusion in the RVE (Sec. 2.1).

Homogenised (steady) problem, the paper's form: div j = 0 with
j = -D(x) grad c, <grad c> = grad c_mac (Eq. diffusion), D(x) =
omega D_solid I + (1 - omega) D_pore I. The unknown is the gradient field
grad c = grad c_mac + delta with delta compatible; the Galerkin equation
IFFT(G_hat . j_hat) = 0 (Eq. diffusion-final) is solved by CG on
G : (D delta) = -G : (D grad c_mac) (Algorithm 1, Diffusion of chemical
species). The fluctuation phi follows from Eq. (phi-fft) with the inverse
gradient of Eq. (g-42), and the concentration from Eq. (concentration) with
the two integration constants of Eq. (psi-two-values):
beta_pore = c(X)/eta - <grad c_mac . x>_pore - <phi>_pore,
beta_solid = - <grad c_mac . x>_solid - <phi>_solid
(Eq. concentration-correct for the pores; the solid uses beta_solid, so that
<c>_solid = 0).

Transient problem (NOT in the paper; the paper's RVE diffusion is static
and time enters only at the macroscale, Sec. 3.2): one backward-Euler step of
dc/dt = -grad+^T (D grad+ c) with grad+ the forward difference of Sec. 2.6,
on the voxels outside a Dirichlet mask, written out as a sparse matrix and
solved directly.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import spectral
from .krylov import cg


def diffusivity(phase, mat):
    w = (np.asarray(phase) == 1).astype(np.float64)
    return w * mat.D_solid + (1 - w) * mat.D_pore


def voxel_coordinates(shape, h):
    """x_alpha = k_alpha h for every voxel, alpha = 0 (x) .. d-1."""
    ndim = len(shape)
    out = []
    for alpha in range(ndim):
        ax = spectral.direction_axis(alpha, ndim)
        sh = [1] * ndim
        sh[ax] = shape[ax]
        out.append(np.broadcast_to(h * np.arange(shape[ax], dtype=np.float64).reshape(sh), shape))
    return out


def homogenise(phase, mat, grad_c_mac, c_macro, h, tol=1e-12, max_iter=200000, record=False, symbol="forward"):
    """Steady RVE diffusion (Eqs. diffusion, diffusion-final, phi-fft,
    psi-two-values, concentration-correct). Returns grad c, phi, c, the mean
    flux <j> and the CG info. symbol: the gradient operator of Sec. 2.6
    (forward, central, central8, fourier; the paper's results use forward)."""
    phase = np.asarray(phase)
    shape = phase.shape
    d = phase.ndim
    Dx = diffusivity(phase, mat)
    Dsym = spectral.SYMBOLS[symbol](shape, h)
    ghat = spectral.projection_operator(Dsym)
    gmac = np.array([grad_c_mac[a] for a in range(d)], dtype=np.float64)
    gradc = np.broadcast_to(gmac.reshape((d,) + (1,) * d), (d,) + shape).copy()

    def A(x):
        return spectral.apply_G(ghat, Dx[None] * x)

    b = -spectral.apply_G(ghat, Dx[None] * gradc)
    delta, info = cg(A, b, tol=tol, max_iter=max_iter, record=record)
    gradc = gradc + delta
    phi = spectral.solve_poisson_from_gradient(gradc, Dsym)
    x = voxel_coordinates(shape, h)
    ramp = sum(gmac[a] * x[a] for a in range(d))
    pore = phase == 0
    solid = ~pore
    c = ramp + phi
    eta = pore.mean()
    if pore.any():
        beta_pore = c_macro / eta - ramp[pore].mean() - phi[pore].mean()
        c = np.where(pore, c + beta_pore, c)
    if solid.any():
        beta_solid = -ramp[solid].mean() - phi[solid].mean()
        c = np.where(solid, c + beta_solid, c)
    j = -Dx[None] * gradc
    return {"grad_c": gradc, "phi": phi, "c": c,
            "mean_flux": j.reshape(d, -1).mean(axis=1), "info": info, "iters": info["iters"]}


def forward_difference_matrix(shape, alpha, h):
    """Sparse (u(x + h e_alpha) - u(x)) / h on the periodic grid."""
    ndim = len(shape)
    ax = spectral.direction_axis(alpha, ndim)
    N = int(np.prod(shape))
    idx = np.arange(N).reshape(shape)
    nxt = np.roll(idx, -1, axis=ax).ravel()
    rows = np.concatenate([np.arange(N), np.arange(N)])
    cols = np.concatenate([nxt, np.arange(N)])
    vals = np.concatenate([np.full(N, 1.0 / h), np.full(N, -1.0 / h)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def transient_matrix(phase, mat, dt, h):
    """(1/dt) I + sum_alpha B_alpha^T diag(D) B_alpha, B_alpha the forward
    difference: backward Euler for dc/dt = div(D grad c) in the Galerkin form
    of Sec. 2.1 (flux evaluated at each voxel with that voxel's D)."""
    phase = np.asarray(phase)
    shape = phase.shape
    N = phase.size
    Dx = sp.diags(diffusivity(phase, mat).ravel())
    A = sp.identity(N, format="csr") * (1.0 / dt)
    for alpha in range(phase.ndim):
        B = forward_difference_matrix(shape, alpha, h)
        A = A + B.T @ Dx @ B
    return A.tocsc()


def transient_step(phase, c_prev, mat, dt, h, mask=None, c_dirichlet=1.0):
    """One backward-Euler step; voxels with mask != 0 are held at c_dirichlet."""
    phase = np.asarray(phase)
    A = transient_matrix(phase, mat, dt, h)
    b = np.asarray(c_prev, dtype=np.float64).ravel() / dt
    if mask is None:
        c = spla.spsolve(A, b)
        return c.reshape(phase.shape)
    fixed = np.asarray(mask).ravel() != 0
    free = ~fixed
    cD = np.zeros(phase.size)
    cD[fixed] = c_dirichlet
    rhs = b[free] - (A[free][:, fixed] @ cD[fixed])
    c = cD.copy()
    c[free] = spla.spsolve(A[free][:, free].tocsc(), rhs)
    return c.reshape(phase.shape)
