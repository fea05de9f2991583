"""Pins of the oracle's adjoint (reverse-mode dJ/de(x) of the staggered solve
with a prescribed, ramped pore eigenstrain) against central finite
differences of the oracle's own forward model, for both objectives (total
elastic energy, summed damage), in 2D and 3D, over steps in which damage and
the history field evolve. The finite-difference step is 1e-6 on
eigenstrains of order 1e-2; every solve goes to a 1e-13 relative residual.
"""

import numpy as np
import pytest

from microstructures import random_carpet, random_sponge
from microstructures.workloads import Materials
from oracle import adjoint

H = 5e-6
MAT = Materials(E_pore=2e9)  # stiff pores: damage develops within a few steps
# load, unload, partial reload: the history max keeps H from the first step
# where the later psi+ is smaller, so both branches of the max are taken
RAMP = [1.0, 0.4, 0.9]
TOL = 1e-13


def case(dim):
    if dim == 2:
        phase, _ = random_carpet(27, 0.30, 5)
    else:
        phase, _ = random_sponge(9, 0.3, 6)
    rng = np.random.default_rng(3)
    e = np.where(phase == 0, 2e-2 * (1.0 + 0.2 * rng.standard_normal(phase.shape)), 0.0)
    return phase, e


def macro(dim, tension):
    """A fixed tensile macro strain (xx) puts part of the solid in volumetric
    tension, so the bulk branch [tr]_+ of psi+ is active; without it the
    pore expansion leaves every voxel in volumetric compression."""
    if not tension:
        return None
    return [3e-3, 0.0, 0.0] if dim == 2 else [3e-3, 0.0, 0.0, 0.0, 0.0, 0.0]


def fd(phase, e, kind, idx, step=1e-6, E=None):
    ep = e.copy()
    em = e.copy()
    ep[idx] += step
    em[idx] -= step
    jp = adjoint.objective(adjoint.forward(phase, ep, MAT, H, RAMP, tol=TOL, eps_mac=E), kind, H)
    jm = adjoint.objective(adjoint.forward(phase, em, MAT, H, RAMP, tol=TOL, eps_mac=E), kind, H)
    return (jp - jm) / (2 * step)


def voxels(phase, n, seed):
    rng = np.random.default_rng(seed)
    pores = np.argwhere(phase == 0)
    solid = np.argwhere(phase == 1)
    pick = list(pores[rng.choice(len(pores), n - 1, replace=False)]) + [solid[rng.integers(len(solid))]]
    return [tuple(p) for p in pick]


@pytest.mark.parametrize("tension", [False, True])
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("kind", ["energy", "damage"])
def test_adjoint_gradient_matches_central_differences(dim, kind, tension):
    phase, e = case(dim)
    E = macro(dim, tension)
    steps = adjoint.forward(phase, e, MAT, H, RAMP, tol=TOL, eps_mac=E)
    assert steps[-1]["d"].max() > 1e-3  # damage evolves
    takes = [st["psi"] >= st["H_prev"] for st in steps]
    assert takes[0].all() and not takes[1].all()  # both branches of the history max are taken
    if tension:
        from oracle import elasticity
        st = steps[-1]
        I = elasticity.identity_field(dim, phase.shape)
        assert (elasticity.trace(elasticity.sym(st["F"]) - st["e"][None, None] * I) > 0).mean() > 0.05
    g = adjoint.gradient(phase, e, MAT, H, RAMP, kind, tol=TOL, steps=steps)
    scale = np.abs(g).max()
    for idx in voxels(phase, 4 if dim == 2 else 3, 11):
        ref = fd(phase, e, kind, idx, E=E)
        assert abs(g[idx] - ref) <= 1e-5 * scale + 1e-6 * abs(ref), (kind, idx, g[idx], ref)


def test_adjoint_gradient_is_zero_without_load():
    """No eigenstrain: every field stays zero and the energy's gradient is
    the first-order term only (J is quadratic in e)."""
    phase, e = case(2)
    g = adjoint.gradient(phase, np.zeros_like(e), MAT, H, RAMP, "energy", tol=TOL)
    assert np.abs(g).max() == 0.0


MUTATIONS = {
    "drop (1 - d) of the phase-field adjoint": ('dJ_dH + (1.0 - st["d"]) * lam_pf', "dJ_dH + lam_pf"),
    "flip the degradation derivative": ('gprime = -2.0 * (1.0 - st["d_prev"])', 'gprime = 2.0 * (1.0 - st["d_prev"])'),
    "history max passes everything to psi+": ('take = st["psi"] >= st["H_prev"]', 'take = st["psi"] >= -1.0'),
    "2D bulk factor in 3D": ("K = lam + 2.0 * mu / dim", "K = lam + mu"),
    "eigenstrain drive without the trace factor": ("g * (dim * lam + 2.0 * mu)", "g * (lam + 2.0 * mu)"),
}


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_planted_mistakes_fail_the_finite_difference_pin(name):
    """Each mistake, planted in a copy of the oracle's adjoint, moves the
    gradient away from the finite differences of the (unchanged) forward."""
    import os
    import types
    src = open(os.path.join(os.path.dirname(adjoint.__file__), "adjoint.py")).read()
    old, new = MUTATIONS[name]
    assert old in src
    mod = types.ModuleType("oracle.adjoint_mutant")
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new), "adjoint_mutant", "exec"), mod.__dict__)
    worst = 0.0
    for dim in (2, 3):
        phase, e = case(dim)
        E = macro(dim, True)
        steps = adjoint.forward(phase, e, MAT, H, RAMP, tol=TOL, eps_mac=E)
        for kind in ("energy", "damage"):
            g = mod.gradient(phase, e, MAT, H, RAMP, kind, tol=TOL, steps=steps)
            g_ok = adjoint.gradient(phase, e, MAT, H, RAMP, kind, tol=TOL, steps=steps)
            scale = np.abs(g_ok).max()
            for idx in voxels(phase, 2, 12):
                worst = max(worst, abs(g[idx] - fd(phase, e, kind, idx, E=E)) / scale)
    assert worst > 1e-3, (name, worst)
