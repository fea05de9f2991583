"""Macroscale multiscale driver of Sec. 3.2 over the library's batched RVEs:
a bar whose lower face takes a constant influx of ferrous ions, one RVE per
bar element, the bar's nodal concentrations kept on the device and advanced
by the library (fftmech_bar_*, include/fftmech.h) from the RVEs' mean
fluxes. Each macro step is one library call: the element inputs, one
staggered step of every RVE (homogenised diffusion with the element's
c(X) and grad c(X), precipitation, eigenstrain, equilibrium at zero macro
strain, history, phase field) and the nodal update, as one CUDA graph.
Argument marshalling only: every step runs in the CUDA library.
"""

import numpy as np
import torch

from . import fftmech as fm


class MacroBar:
    """phases: M RVE phase arrays of one shape (uint8, 0 pore / 1 solid);
    length: bar length in the RVE's length unit (h_diff per voxel);
    flux_in: influx at X = 0; c0: M + 1 nodal concentrations (None = 0)."""

    def __init__(self, phases, materials, length, dt, flux_in, c0=None, precision=fm.FFTMECH_FP64, h=5e-6,
                 h_diff=1.0, tol=1e-10, max_iter=20000, device="cuda"):
        phases = [np.asarray(p, dtype=np.uint8) for p in phases]
        self.M = len(phases)
        shape = phases[0].shape
        self.shape = shape
        self.ctx = fm.Context(shape, materials, precision, h=h, h_diff=h_diff, tol=tol, max_iter=max_iter,
                              batch=self.M)
        N = int(np.prod(shape))
        dim = len(shape)
        nv = 3 if dim == 2 else 6
        ft = torch.float64 if precision == fm.FFTMECH_FP64 else torch.float32
        B = self.M
        self.bufs = {
            "phase": torch.as_tensor(np.concatenate([p.ravel() for p in phases])).to(device),
            "c": torch.zeros(B * N, dtype=torch.float64, device=device),
            "c_ppt": torch.zeros(B * N, dtype=ft, device=device),
            "eig": torch.zeros(B * N, dtype=ft, device=device),
            "u": torch.zeros(B * dim * N, dtype=torch.float64, device=device),
            "strain": torch.zeros(B * nv * N, dtype=ft, device=device),
            "stress": torch.zeros(B * nv * N, dtype=ft, device=device),
            "H": torch.zeros(B * N, dtype=ft, device=device),
            "damage": torch.zeros(B * N, dtype=torch.float64, device=device),
        }
        self.state = fm.fftmech_state()
        for k, v in self.bufs.items():
            setattr(self.state, k, v.data_ptr())
        self.params = fm.fftmech_step_params()
        self.params.diffusion_mode = fm.FFTMECH_DIFF_HOMOGENISE
        self.params.eig_mode = fm.FFTMECH_EIG_FROM_PRECIPITATE
        self.bar = fm.fftmech_bar_create(self.ctx.handle, length, dt, flux_in,
                                         None if c0 is None else list(np.asarray(c0, dtype=np.float64)))

    def step(self):
        """One macro time step; returns the RVEs' records (3 per RVE)."""
        return fm.fftmech_bar_step(self.bar, self.ctx.handle, self.state, self.params)

    def nodes(self):
        """Nodal macro concentrations c_0 .. c_M (host copy)."""
        return np.array(fm.fftmech_bar_read(self.bar, self.M + 1))

    def field(self, name, problem):
        """One RVE's field (host copy), reshaped to (components, *shape)."""
        N = int(np.prod(self.shape))
        v = self.bufs[name]
        per = v.numel() // self.M
        return v[problem * per:(problem + 1) * per].double().cpu().numpy().reshape((per // N,) + self.shape)

    def close(self):
        if self.bar:
            fm.fftmech_bar_destroy(self.bar)
            self.bar = None
        self.ctx.close()
