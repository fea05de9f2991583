"""One staggered load step in the order of Algorithm 1 (Sec. 2.5):
diffusion -> concentration -> precipitation -> eigenstrain -> equilibrium
(stiffness degraded by the damage of the previous step) -> history field ->
phase field. The degradation with the new damage (Algorithm 1, last line) is
applied at the start of the next step's equilibrium solve.
"""

import numpy as np

from . import diffusion, elasticity, phasefield, chemistry

DIFF_NONE, DIFF_HOMOGENISE, DIFF_TRANSIENT = 0, 1, 2
EIG_FROM_PRECIPITATE, EIG_PRESCRIBED = 0, 1


def initial_state(phase, c0=None):
    shape = np.asarray(phase).shape
    d = len(shape)
    nv = 3 if d == 2 else 6
    z = np.zeros(shape)
    return {"c": z.copy() if c0 is None else np.asarray(c0, dtype=np.float64).copy(),
            "c_ppt": z.copy(), "eig": z.copy(), "H": z.copy(), "d": z.copy(),
            "strain": np.zeros((nv,) + shape), "stress": np.zeros((nv,) + shape)}


def step(state, phase, mat, h, h_diff, diffusion_mode, eig_mode, eig_field=None,
         eig_scale=1.0, grad_c_mac=(0, 0, 0), c_macro=0.0, dt=0.0, mask=None,
         c_dirichlet=1.0, eps_mac=(0, 0, 0, 0, 0, 0), tol=1e-12):
    phase = np.asarray(phase)
    dim = phase.ndim
    nv = 3 if dim == 2 else 6
    s = {k: v.copy() for k, v in state.items()}
    info = {}
    # Diffusion of chemical species
    if diffusion_mode == DIFF_HOMOGENISE:
        out = diffusion.homogenise(phase, mat, grad_c_mac, c_macro, h_diff, tol=tol)
        s["c"] = out["c"]
        info["diffusion"] = out
    elif diffusion_mode == DIFF_TRANSIENT:
        s["c"] = diffusion.transient_step(phase, s["c"], mat, dt, h_diff, mask, c_dirichlet)
    # Pressurisation of pores
    if eig_mode == EIG_FROM_PRECIPITATE:
        s["c_ppt"] = chemistry.precipitate(s["c"], phase, mat.S_sol)
        s["eig"] = chemistry.eigenstrain(s["c_ppt"], phase, mat.M_ppt)
    else:
        s["eig"] = eig_scale * np.asarray(eig_field, dtype=np.float64)
    # Development of stresses, with the stiffness degraded by the current damage
    g = phasefield.degradation(s["d"], mat.kappa)
    eq = elasticity.equilibrium_solve(phase, s["eig"], g, list(eps_mac)[:nv], mat, h, tol=tol)
    s["strain"], s["stress"] = eq["strain"], eq["stress"]
    info["equilibrium"] = eq
    # Crack initiation and propagation
    lam, mu = elasticity.phase_lame(phase, mat)
    psi = elasticity.psi_plus(s["strain"], s["eig"], lam, mu)
    s["H"] = phasefield.history_update(s["H"], psi)
    s["d"], pinfo = phasefield.phasefield_solve(s["H"], mat, h, tol=tol, d0=s["d"])
    info["phasefield"] = pinfo
    solid = phase == 1
    info["frac_damaged"] = float((s["d"][solid] > 0.9).mean()) if solid.any() else 0.0
    return s, info
