"""Reverse-mode sensitivity of the staggered solve to the pore eigenstrain
(an extension: the paper solves forward only; Secs. 2.3-2.5 define the model
whose derivative is taken).

Forward model: S staggered steps of Algorithm 1 without the diffusion step,
the eigenstrain prescribed as e_s(x) = a_s e(x) with a load ramp a_s:
  equilibrium (Eqs. solid, solid-final) with the stiffness degraded by the
  previous damage, g(d_{s-1}) C : (eps_s - e_s I), <eps> = E (a fixed macro
  strain, zero in the paper's runs);
  psi_s = psi+(eps_s - e_s I)           (Eq. energy, undegraded Lame);
  H_s = max(H_{s-1}, psi_s)             (history, Sec. 2.4);
  A(H_s) d_s = H_s                      (Eq. crack-fft), A(H) = a + H + b L.
H_0 = d_0 = 0. Objectives at the last step S:
  'energy': the total elastic energy sum_x 1/2 (eps_S - e_S I) : sigma_S h^d;
  'damage': the summed damage sum_x d_S.

Gradient dJ/de(x) by the discrete adjoint, step by step backwards:
  phase field: A(H_s) lambda = dJ/dd_s (A symmetric), then
    dJ/dH_s += (1 - d_s) lambda;
  history max: dJ/dpsi_s = dJ/dH_s where psi_s >= H_{s-1} (ties count as
    the new value), the rest flows to H_{s-1};
  psi+: dJ/deps_el = dJ/dpsi_s (K [tr eps_el]_+ I + 2 mu dev eps_el),
    K = lambda + 2 mu / d; dJ/de_s gets -tr of it;
  equilibrium: the compatible field Lam with GG : (g C : Lam) = GG : G,
    G = dJ/deps through the history field (the paper's gradient-space CG on
    the same operator; the energy's own dJ/deps = sigma h^d is
    divergence-free at equilibrium and drops out);
    dJ/de_s += g (d lambda + 2 mu) tr Lam and
    dJ/dd_{s-1} = -g'(d_{s-1}) (C : (eps_s - e_s I)) : Lam, g' = -2 (1 - d);
  dJ/de(x) = sum_s a_s dJ/de_s.
"""

import numpy as np

from . import spectral, elasticity, phasefield
from .krylov import cg


def forward(phase, e_field, mat, h, ramp, tol=1e-12, eps_mac=None):
    """Runs the forward model and keeps every step's state. eps_mac: a fixed
    macro strain (Voigt; zero by default, as in the paper's runs)."""
    phase = np.asarray(phase)
    shape = phase.shape
    lam, mu = elasticity.phase_lame(phase, mat)
    d = np.zeros(shape)
    H = np.zeros(shape)
    steps = []
    for a_s in ramp:
        e_s = a_s * np.asarray(e_field, dtype=np.float64)
        g = phasefield.degradation(d, mat.kappa)
        nv = 3 if phase.ndim == 2 else 6
        E = [0.0] * nv if eps_mac is None else list(eps_mac)[:nv]
        eq = elasticity.equilibrium_solve(phase, e_s, g, E, mat, h, tol=tol)
        psi = elasticity.psi_plus(eq["strain"], e_s, lam, mu)
        H_new = phasefield.history_update(H, psi)
        d_new, _ = phasefield.phasefield_solve(H_new, mat, h, tol=tol, d0=d)
        steps.append({"e": e_s, "d_prev": d, "H_prev": H, "g_prev": g, "F": eq["F"], "strain": eq["strain"],
                      "stress": eq["stress"], "psi": psi, "H": H_new, "d": d_new})
        d, H = d_new, H_new
    return steps


def objective(steps, kind, h):
    last = steps[-1]
    if kind == "energy":
        return elasticity.elastic_energy(last["strain"], last["stress"], last["e"], h)
    if kind == "damage":
        return float(np.sum(last["d"]))
    raise ValueError(kind)


def _phasefield_adjoint(H, rhs, mat, h, tol):
    """A(H) x = rhs with the phase-field operator of Eq. (crack-fft)."""
    a, b = phasefield.coefficients(mat)
    D = spectral.forward_difference_symbol(H.shape, h)
    lam_k = spectral.symbol_norm2(D)

    def A(x):
        lap = spectral.ifft(-lam_k * spectral.fft(x)).real
        return -b * lap + a * x + H * x

    x, _ = cg(A, rhs.copy(), tol=tol)
    return x


def gradient(phase, e_field, mat, h, ramp, kind, tol=1e-12, steps=None, eps_mac=None):
    """dJ/de(x) of objective `kind` ('energy' or 'damage')."""
    phase = np.asarray(phase)
    shape = phase.shape
    dim = phase.ndim
    if steps is None:
        steps = forward(phase, e_field, mat, h, ramp, tol=tol, eps_mac=eps_mac)
    lam, mu = elasticity.phase_lame(phase, mat)
    K = lam + 2.0 * mu / dim
    I = elasticity.identity_field(dim, shape)
    Dsym = spectral.forward_difference_symbol(shape, h)
    ghat = spectral.projection_operator(Dsym)
    vol = h ** dim
    grad = np.zeros(shape)
    dJ_dd = np.ones(shape) if kind == "damage" else np.zeros(shape)  # seed of d_S
    dJ_dH = np.zeros(shape)
    S = len(steps)
    for s in range(S - 1, -1, -1):
        st = steps[s]
        eps = elasticity.sym(st["F"])
        eps_el = eps - st["e"][None, None] * I
        C_el = lam[None, None] * elasticity.trace(eps_el)[None, None] * I + 2.0 * mu[None, None] * eps_el
        g = st["g_prev"]
        gprime = -2.0 * (1.0 - st["d_prev"])
        G = np.zeros((dim, dim) + shape)  # dJ / d eps_s
        dJ_de = np.zeros(shape)
        dJ_dd_prev = np.zeros(shape)
        if s == S - 1 and kind == "energy":
            # dJ/deps = sigma h^d is divergence-free at equilibrium: the
            # energy is stationary in the displacement, so that term adds
            # nothing through the equilibrium adjoint and only the explicit
            # dependences on e and on d_{S-1} remain
            sig = g[None, None] * C_el
            dJ_de += -elasticity.trace(sig) * vol
            dJ_dd_prev += 0.5 * gprime * np.einsum("ij...,ij...->...", eps_el, C_el) * vol
        # phase field of step s
        if np.any(dJ_dd != 0.0):
            lam_pf = _phasefield_adjoint(st["H"], dJ_dd, mat, h, tol)
            dJ_dH = dJ_dH + (1.0 - st["d"]) * lam_pf
        # history max
        take = st["psi"] >= st["H_prev"]
        dJ_dpsi = np.where(take, dJ_dH, 0.0)
        dJ_dH = np.where(take, 0.0, dJ_dH)
        # psi+ of the elastic strain
        tr = elasticity.trace(eps_el)
        dev = eps_el - (tr / dim)[None, None] * I
        dpsi = K[None, None] * np.maximum(tr, 0.0)[None, None] * I + 2.0 * mu[None, None] * dev
        G += dJ_dpsi[None, None] * dpsi
        dJ_de += -dJ_dpsi * elasticity.trace(dpsi)
        # equilibrium of step s: compatible Lam with GG : (g C : Lam) = GG : G
        b_rhs = spectral.apply_GG(ghat, G)
        bn, Gn = np.linalg.norm(b_rhs), np.linalg.norm(G)
        if bn > tol * Gn:
            def A(X):
                return spectral.apply_GG(ghat, elasticity.tangent(X, g, lam, mu))

            Lam, _ = cg(A, b_rhs, tol=tol * Gn / bn)
            Ls = elasticity.sym(Lam)
            dJ_de += g * (dim * lam + 2.0 * mu) * elasticity.trace(Ls)
            dJ_dd_prev += -gprime * np.einsum("ij...,ij...->...", C_el, Ls)
        grad += ramp[s] * dJ_de
        dJ_dd = dJ_dd_prev
    return grad
