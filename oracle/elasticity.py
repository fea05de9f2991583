"""Mechanical equilibrium with eigenstrain (Sec. 2.3) in the paper's
gradient form.

Unknown: the displacement gradient F[i, j] = d u_i / d x_j (shape
(d, d, *grid)), split as F = eps_mac + dF with dF compatible (in the range of
the fourth-order projection GG of App. A). Stress (Eq. solid):
sigma = g(d) C(x) : (eps - eps_eig), with C(x) = omega C_solid +
(1 - omega) C_pore, C_i = lambda_i I(x)I + 2 mu_i II (II the symmetric
fourth-order identity, so C : F = C : sym F), isotropic eigenstrain
eps_eig = e(x) I, and g(d) = (1 - d)^2 + kappa the degradation of Sec. 2.4.
2D is plane strain: in-plane components only, the eigenstrain identity is the
in-plane 2 x 2 identity.

Discrete weak form (Eq. solid-final): IFFT(GG_hat : sigma_hat) = 0, solved
with the Newton-Raphson loop of Algorithm 1 (Development of stresses), each
Newton correction by CG on GG : (g C : dF) = -GG : sigma(F).
"""

import numpy as np

from . import spectral
from .krylov import cg, dot

VOIGT = {2: [(0, 0), (1, 1), (0, 1)],
         3: [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]}


def lame(E, nu):
    """Lame constants of an isotropic solid; in plane strain the in-plane
    law uses the same lambda and mu."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def phase_lame(phase, mat):
    """Per-voxel (lambda, mu) from omega: C = omega C_s + (1 - omega) C_p."""
    ls, ms = lame(mat.E_solid, mat.nu_solid)
    lp, mp = lame(mat.E_pore, mat.nu_pore)
    w = (np.asarray(phase) == 1).astype(np.float64)
    return w * ls + (1 - w) * lp, w * ms + (1 - w) * mp


def sym(F):
    return 0.5 * (F + np.swapaxes(F, 0, 1))


def trace(T):
    return sum(T[i, i] for i in range(T.shape[0]))


def identity_field(d, shape):
    I = np.zeros((d, d) + tuple(shape))
    for i in range(d):
        I[i, i] = 1.0
    return I


def stress(F, e, g, lam, mu):
    """sigma = g [lambda tr(eps_el) I + 2 mu eps_el], eps_el = sym F - e I."""
    d = F.shape[0]
    eps_el = sym(F) - e[None, None] * identity_field(d, F.shape[2:])
    tr = trace(eps_el)
    return g[None, None] * (lam[None, None] * tr[None, None] * identity_field(d, F.shape[2:])
                            + 2.0 * mu[None, None] * eps_el)


def tangent(X, g, lam, mu):
    """g C : X (the linear law's tangent, no eigenstrain)."""
    d = X.shape[0]
    s = sym(X)
    tr = trace(s)
    return g[None, None] * (lam[None, None] * tr[None, None] * identity_field(d, X.shape[2:])
                            + 2.0 * mu[None, None] * s)


def macro_tensor(eps_mac_voigt, d):
    """Symmetric tensor from Voigt components (tensor shear, not engineering)."""
    E = np.zeros((d, d))
    for I, (i, j) in enumerate(VOIGT[d]):
        E[i, j] = eps_mac_voigt[I]
        E[j, i] = eps_mac_voigt[I]
    return E


def to_voigt(T):
    d = T.shape[0]
    return np.stack([T[i, j] for (i, j) in VOIGT[d]])


def equilibrium_solve(phase, eig, g, eps_mac, mat, h, tol=1e-12, newton_tol=1e-8,
                      max_newton=6, max_iter=200000, record=False, symbol="forward"):
    """Newton-Raphson + CG for Eq. (solid-final) (Algorithm 1, Development of
    stresses). eps_mac: Voigt components (len 3 in 2D, 6 in 3D). symbol:
    the gradient operator of Sec. 2.6 (spectral.SYMBOLS; the paper's results
    use the forward difference).
    Returns a dict with F, strain (Voigt), stress (Voigt), the CG info of the
    first Newton step and the total CG iterations."""
    phase = np.asarray(phase)
    shape = phase.shape
    d = phase.ndim
    lam, mu = phase_lame(phase, mat)
    e = np.asarray(eig, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    D = spectral.SYMBOLS[symbol](shape, h)
    ghat = spectral.projection_operator(D)
    E = macro_tensor(eps_mac, d)
    F = np.broadcast_to(E[:, :, None, None] if d == 2 else E[:, :, None, None, None],
                        (d, d) + shape).copy()

    def A(X):
        return spectral.apply_GG(ghat, tangent(X, g, lam, mu))

    # Newton-Raphson: residual tolerances are measured against the first
    # right-hand side, so with the linear law the second pass finds the
    # residual already below tol and stops (Algorithm 1's break test).
    infos = []
    total = 0
    b0 = None
    for _ in range(max_newton):
        b = -spectral.apply_GG(ghat, stress(F, e, g, lam, mu))
        bn = np.sqrt(dot(b, b))
        if b0 is None:
            b0 = bn
        elif bn <= tol * b0:
            break
        if bn == 0.0:
            infos.append({"iters": 0, "rel_res": 0.0, "history": [], "energy": []})
            break
        dF, info = cg(A, b, tol=tol * b0 / bn, max_iter=max_iter, record=record)
        infos.append(info)
        total += info["iters"]
        F = F + dF
        nF = np.sqrt(dot(F, F))
        if np.sqrt(dot(dF, dF)) <= newton_tol * max(nF, 1e-300):
            break
    sig = stress(F, e, g, lam, mu)
    strain = to_voigt(sym(F))
    return {"F": F, "strain": strain, "stress": to_voigt(sig), "sigma_tensor": sig,
            "info": infos[0], "newton": len(infos), "iters": total,
            "mean_stress": to_voigt(sig).reshape(len(VOIGT[d]), -1).mean(axis=1),
            "mean_strain": strain.reshape(len(VOIGT[d]), -1).mean(axis=1)}


def psi_plus(strain_voigt, eig, lam, mu):
    """Positive (tension + shear) energy density, Eq. (energy), of the elastic
    strain eps - e I with the undegraded phase constants. The printed form is
    2D: 1/2 (lambda + mu) [tr eps]_+^2 + mu eps_dev : eps_dev with
    eps_dev = eps - 1/2 tr(eps) I; in d dimensions the bulk factor is
    lambda + 2 mu / d and eps_dev = eps - tr(eps)/d I."""
    strain_voigt = np.asarray(strain_voigt)
    d = 2 if strain_voigt.shape[0] == 3 else 3
    T = np.zeros((d, d) + strain_voigt.shape[1:])
    for I, (i, j) in enumerate(VOIGT[d]):
        T[i, j] = strain_voigt[I]
        T[j, i] = strain_voigt[I]
    for i in range(d):
        T[i, i] = T[i, i] - eig
    tr = trace(T)
    dev = T - (tr / d)[None, None] * identity_field(d, T.shape[2:])
    K = lam + 2.0 * mu / d
    trp = 0.5 * (tr + np.abs(tr))
    return 0.5 * K * trp ** 2 + mu * np.einsum("ij...,ij...->...", dev, dev)


def elastic_energy(strain_voigt, stress_voigt, eig, h):
    """sum_x 1/2 (eps - e I) : sigma h^d (tensor contraction, shear twice)."""
    s = np.asarray(strain_voigt)
    t = np.asarray(stress_voigt)
    d = 2 if s.shape[0] == 3 else 3
    tot = 0.0
    for I, (i, j) in enumerate(VOIGT[d]):
        el = s[I] - (eig if i == j else 0.0)
        w = 1.0 if i == j else 2.0
        tot += w * float(np.sum(el * t[I]))
    return 0.5 * tot * h ** d


def effective_stiffness(phase, mat, h, g=None, tol=1e-12):
    """C_eff[I, J] = <sigma_I> under a unit macro strain in Voigt slot J
    (tensor components; shear slot J sets eps_ij = eps_ji = 1), e = 0."""
    phase = np.asarray(phase)
    d = phase.ndim
    nv = len(VOIGT[d])
    if g is None:
        g = np.ones(phase.shape)
    C = np.zeros((nv, nv))
    for J in range(nv):
        E = np.zeros(nv)
        E[J] = 1.0
        out = equilibrium_solve(phase, np.zeros(phase.shape), g, E, mat, h, tol=tol)
        C[:, J] = out["mean_stress"]
    return C


def reference_medium_preconditioner(r, lam0, mu0, h):
    """z = K0^-1 r for a displacement-space residual r (shape (d, *grid)),
    K0 = grad+^T C0 grad+ the Galerkin operator of a homogeneous isotropic
    reference medium C0 (lambda0, mu0): the Moulinec-Suquet reference medium
    (Sec. 1), per Fourier mode with the forward-difference symbol D (Sec. 2.6).
    From sigma_hat_ij = lambda0 delta_ij (D . u) + mu0 (D_j u_i + D_i u_j) and
    (K0 u)_i = sum_j conj(D_j) sigma_hat_ij, each mode solves the d x d system
        (mu0 |D|^2 I + lambda0 conj(D) D^T + mu0 D conj(D)^T) z_hat = r_hat
    (numpy.linalg.solve per mode); z_hat = 0 at k = 0."""
    r = np.asarray(r, dtype=np.float64)
    d = r.shape[0]
    shape = r.shape[1:]
    D = spectral.forward_difference_symbol(shape, h)
    rh = np.stack([spectral.fft(r[i]) for i in range(d)])
    zh = np.zeros_like(rh)
    for idx in np.ndindex(*shape):
        a = np.array([D[i][idx] for i in range(d)])
        n2 = float(np.sum(np.abs(a) ** 2))
        if n2 == 0.0:
            continue
        K = mu0 * n2 * np.eye(d) + lam0 * np.outer(np.conj(a), a) + mu0 * np.outer(a, np.conj(a))
        zh[(slice(None),) + idx] = np.linalg.solve(K, rh[(slice(None),) + idx])
    return np.stack([spectral.ifft(zh[i]).real for i in range(d)])
