"""Macroscale multiscale driver of Sec. 3.2 (test infrastructure: the oracle
of the library's macroscale driver; only tests/, smoke and the bench's CPU
baseline use it).

A bar along X whose lower face (X = 0, the steel-concrete interface) takes a
constant influx of ferrous ions and whose other faces are closed. Every
material point of the bar is coupled to an RVE: the macro concentration and
its gradient go down to the RVE, which solves the homogenised diffusion
(Eqs. diffusion, diffusion-final, phi-fft, concentration-correct) and returns
its mean flux <j>; the bar's diffusion (Eq. diffusion at the macroscale) is
advanced with those fluxes by a finite-difference scheme. All other processes
(precipitation, eigenstrain, equilibrium at zero macro strain, history, phase
field) run inside the RVEs only: one staggered step (Algorithm 1) per macro
time step.

The paper names neither the finite-difference scheme nor where the RVEs sit.
Reading taken here:
- nodes X_m = m dX (m = 0 .. M) carry the macro concentration c_m; element e
  spans nodes e and e + 1 and carries one RVE at its midpoint (one-point
  quadrature of linear elements), which sees
  grad c_mac = ((c_{e+1} - c_e) / dX, 0, 0) (the bar along the RVE's x axis)
  and c_macro = (c_e + c_{e+1}) / 2;
- lumped masses w_m = dX inside, dX / 2 at the two ends; forward Euler:
  c_m <- c_m + dt / w_m (J_{m-1/2} - J_{m+1/2}) with J_{e+1/2} = <j_x>_e,
  J_{-1/2} = the interface influx, J_{M+1/2} = 0;
- the RVE step of macro step n uses c^n (explicit coupling), then c^{n+1} is
  formed from its fluxes;
- dt <= dX^2 / (2 max(D_pore, D_solid)) (the scheme's stability bound with
  the Voigt bound on the effective diffusivity), else ValueError.
"""

import numpy as np

from . import staggered


class MacroBarOracle:
    """phases: list of M RVE phase arrays (one per element, same shape).
    length: bar length, in the RVE's length unit (h_diff per voxel);
    flux_in: influx at X = 0; c0: M + 1 initial nodal concentrations."""

    def __init__(self, phases, mat, h, h_diff, length, dt, flux_in, c0=None, tol=1e-12):
        self.phases = [np.asarray(p) for p in phases]
        self.M = len(self.phases)
        self.mat, self.h, self.h_diff, self.tol = mat, h, h_diff, tol
        self.dX = float(length) / self.M
        self.dt = float(dt)
        self.flux_in = float(flux_in)
        dmax = max(mat.D_pore, mat.D_solid)
        if self.dt > self.dX * self.dX / (2.0 * dmax):
            raise ValueError("dt above the explicit scheme's bound dX^2 / (2 D_max)")
        self.c = np.zeros(self.M + 1) if c0 is None else np.asarray(c0, dtype=np.float64).copy()
        self.w = np.full(self.M + 1, self.dX)
        self.w[0] = self.w[-1] = 0.5 * self.dX
        self.states = [staggered.initial_state(p) for p in self.phases]
        self.last_infos = None

    def element_inputs(self):
        """(grad c_mac along x, c_macro) of every element from the nodal c."""
        G = (self.c[1:] - self.c[:-1]) / self.dX
        cbar = 0.5 * (self.c[1:] + self.c[:-1])
        return G, cbar

    def step(self):
        G, cbar = self.element_inputs()
        fluxes = np.zeros(self.M)
        infos = []
        for e, ph in enumerate(self.phases):
            g = [G[e], 0.0, 0.0]
            self.states[e], info = staggered.step(
                self.states[e], ph, self.mat, self.h, self.h_diff, staggered.DIFF_HOMOGENISE,
                staggered.EIG_FROM_PRECIPITATE, grad_c_mac=g, c_macro=cbar[e], tol=self.tol)
            fluxes[e] = info["diffusion"]["mean_flux"][0]
            infos.append(info)
        J = np.concatenate([[self.flux_in], fluxes, [0.0]])  # faces -1/2 .. M + 1/2
        self.c = self.c + self.dt / self.w * (J[:-1] - J[1:])
        self.last_infos = infos
        return fluxes

    def mass(self):
        return float(np.dot(self.w, self.c))
