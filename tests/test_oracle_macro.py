"""Pins of the oracle's macroscale driver (oracle/macro.py, Sec. 3.2), CPU
only.

- Closed form: with RVEs whose effective diffusivity along the bar is known
  exactly (all pore: D_pore; a laminate of whole voxel columns normal to the
  bar: the harmonic mean of D over an x line; a laminate parallel to the
  bar: the arithmetic mean), c(X, t) = J t / L + J / (2 D L) (X - L)^2 solves
  the lumped scheme exactly at every node (quadratics have exact second
  differences; the end nodes' half masses balance the boundary fluxes), and
  forward Euler integrates its constant rate exactly. Starting from that
  profile, n steps must add n dt J / L at every node.
- Conservation: the lumped mass sum_m w_m c_m grows by dt J per step exactly,
  for any RVEs (random carpets here).
- Every RVE's mean concentration equals its element's c_macro (the two-value
  correction of Eq. psi-two-values keeps <c> = c(X)).
- dt above the explicit bound is rejected.
- Planted mistakes (flux sign, full end masses, node instead of element
  concentration, gradient across two elements) each fail one of these.
"""

import os
import types

import numpy as np
import pytest

from microstructures import random_carpet
from microstructures.workloads import Materials
from oracle import macro

MAT = Materials()
H = 5e-6
L = 400.0
M = 4
J_IN = 1e-3


def laminate(kind, n=9):
    ph = np.zeros((n, n), dtype=np.uint8)
    if kind == "normal":  # layers normal to x: the phase varies along x
        ph[:, n // 2 + 1:] = 1
    elif kind == "parallel":
        ph[n // 2 + 1:, :] = 1
    return ph


def d_eff(kind, n=9):
    """The exact effective diffusivity along x (the bar's direction)."""
    if kind == "pore":
        return MAT.D_pore
    D = np.where(laminate(kind, n) == 0, MAT.D_pore, MAT.D_solid)
    if kind == "normal":
        return 1.0 / np.mean(1.0 / D[0, :])  # resistances in series along x
    return float(np.mean(D[:, 0]))  # conductances in parallel


def quadratic_bar(mod, kind, dt_frac=0.4):
    D = d_eff(kind)
    dX = L / M
    X = dX * np.arange(M + 1)
    c0 = J_IN / (2.0 * D * L) * (X - L) ** 2
    dt = dt_frac * dX * dX / (2.0 * max(MAT.D_pore, MAT.D_solid))
    bar = mod.MacroBarOracle([laminate(kind)] * M, MAT, H, 1.0, L, dt, J_IN, c0=c0, tol=1e-13)
    return bar, c0, dt


@pytest.mark.parametrize("kind", ["pore", "normal", "parallel"])
def test_quadratic_profile_rises_uniformly(kind):
    bar, c0, dt = quadratic_bar(macro, kind)
    for n in range(1, 4):
        bar.step()
        want = c0 + n * dt * J_IN / L
        err = np.abs(bar.c - want).max() / np.abs(want).max()
        assert err < 1e-9, (kind, n, err)


def test_lumped_mass_grows_by_the_influx():
    phases = [random_carpet(9, 0.3, s)[0] for s in range(M)]
    dX = L / M
    c0 = np.linspace(1.2, 0.0, M + 1)
    dt = 0.4 * dX * dX / 2.0
    bar = macro.MacroBarOracle(phases, MAT, H, 1.0, L, dt, J_IN, c0=c0, tol=1e-12)
    m0 = bar.mass()
    for n in range(1, 4):
        bar.step()
        assert abs(bar.mass() - (m0 + n * dt * J_IN)) <= 1e-13 * m0
    # every RVE's mean concentration is its element's c_macro
    G, cbar = bar.element_inputs()
    bar2 = macro.MacroBarOracle(phases, MAT, H, 1.0, L, dt, J_IN, c0=bar.c, tol=1e-12)
    bar2.step()
    for e in range(M):
        assert abs(bar2.states[e]["c"].mean() - cbar[e]) <= 1e-12 * max(abs(cbar[e]), 1e-30)


def test_time_step_above_the_bound_is_rejected():
    dX = L / M
    with pytest.raises(ValueError):
        macro.MacroBarOracle([laminate("pore")] * M, MAT, H, 1.0, L, 0.51 * dX * dX, J_IN)


MUTATIONS = {
    "flux sign": ("(J[:-1] - J[1:])", "(J[1:] - J[:-1])"),
    "full end masses": ("self.w[0] = self.w[-1] = 0.5 * self.dX", "self.w[0] = self.w[-1] = self.dX"),
    "node concentration for the element": ("cbar = 0.5 * (self.c[1:] + self.c[:-1])", "cbar = self.c[:-1].copy()"),
    "gradient across two elements": ("G = (self.c[1:] - self.c[:-1]) / self.dX",
                                     "G = np.gradient(self.c, self.dX)[:-1]"),
}


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_planted_mistakes_fail_a_pin(name):
    src = open(os.path.join(os.path.dirname(macro.__file__), "macro.py")).read()
    old, new = MUTATIONS[name]
    assert old in src
    mod = types.ModuleType("oracle.macro_mutant")
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new), "macro_mutant", "exec"), mod.__dict__)
    failed = False
    for kind in ("normal", "parallel"):
        bar, c0, dt = quadratic_bar(mod, kind)
        bar.step()
        if np.abs(bar.c - (c0 + dt * J_IN / L)).max() > 1e-6 * np.abs(c0).max():
            failed = True
        for e in range(M):  # the element concentration reaches the RVEs only
            want = 0.5 * (c0[e] + c0[e + 1])
            if abs(bar.states[e]["c"].mean() - want) > 1e-9 * abs(want):
                failed = True
    assert failed, name
