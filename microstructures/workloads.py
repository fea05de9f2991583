"""Workload recipes: materials, loads and seeded fields for the five benchmark
configurations of the hot path (all synthetic; the paper's scan, Sec. 3, is
not available, so seeded fractals stand in for it).

Units. Mechanics and the phase field use SI units with a voxel size
h = 5 um, so the regularisation length l0 = 2 voxels = 10 um matches the
paper's l0 = 0.01 mm on its 1 mm / 199 grid (Sec. 3). Diffusion is
nondimensional in grid units (h_diff = 1).

Numbers only: nothing here evaluates an operator or a constitutive law.
"""

from dataclasses import dataclass, asdict, field

import numpy as np

from .fractals import sierpinski_carpet, random_carpet, random_sponge, porosity
from .splitmix import derive_key, standard_normal, uniform01


@dataclass
class Materials:
    """Phase properties (Sec. 3) and model constants.

    kappa: residual stiffness of fully broken material (Sec. 2.4 leaves its
    value open; 1e-4 keeps the stiffness contrast below 1e7).
    S_sol, M_ppt: nondimensional solubility limit and molar volume used by the
    precipitation / eigenstrain step (Eqs. eigen, eigen-simplify); with these
    values a concentration of 1 gives an eigenstrain of 1e-3."""
    E_solid: float = 20e9
    nu_solid: float = 0.2
    E_pore: float = 20e6
    nu_pore: float = 0.2
    D_solid: float = 1e-3
    D_pore: float = 1.0
    Gc: float = 10.0
    l0: float = 10e-6
    kappa: float = 1e-4
    S_sol: float = 0.5
    M_ppt: float = 2.002

    def as_dict(self):
        return asdict(self)


H_MECH = 5e-6
H_DIFF = 1.0

# diffusion modes (shared numbering with the C interface)
DIFF_NONE = 0
DIFF_HOMOGENISE = 1
DIFF_TRANSIENT = 2

# eigenstrain modes
EIG_FROM_PRECIPITATE = 0
EIG_PRESCRIBED = 1


@dataclass
class Workload:
    name: str
    phase: np.ndarray
    materials: Materials
    h: float
    h_diff: float
    steps: int
    diffusion_mode: int
    eig_mode: int
    eig: np.ndarray            # prescribed eigenstrain field (scaled per step by eig_ramp)
    eig_ramp: list             # per-step scale of the prescribed field
    grad_c_mac: tuple = (0.0, 0.0, 0.0)
    c_macro: float = 0.0
    dt: float = 0.0
    dirichlet_mask: np.ndarray = None
    dirichlet_value: float = 0.0
    c0: np.ndarray = None
    eps_mac: tuple = (0.0,) * 6
    tol: float = 1e-8
    extra: dict = field(default_factory=dict)

    @property
    def dim(self):
        return self.phase.ndim

    @property
    def voxels(self):
        return int(self.phase.size)


def left_face_mask(phase):
    """Voxels of the x = 0 face (column 0 in 2D, plane x = 0 in 3D)."""
    mask = np.zeros_like(phase, dtype=np.uint8)
    mask[..., 0] = 1
    return mask


def sierpinski_static(levels=4, steps=10):
    """Sierpinski carpet 81^2 (4 levels, porosity 1-(8/9)^4), eigenstrain 1e-3
    in the pores, steady-state homogenised diffusion with grad c_mac = (1, 0)
    and c(X) = 1, `steps` staggered steps, all FP64."""
    phase = sierpinski_carpet(levels)
    eig = np.where(phase == 0, 1e-3, 0.0)
    return Workload(
        name=f"sierpinski-{phase.shape[0]}x{phase.shape[1]}", phase=phase,
        materials=Materials(), h=H_MECH, h_diff=H_DIFF, steps=steps,
        diffusion_mode=DIFF_HOMOGENISE, eig_mode=EIG_PRESCRIBED, eig=eig,
        eig_ramp=[1.0] * steps, grad_c_mac=(1.0, 0.0, 0.0), c_macro=1.0)


def carpet_transient(n=729, seed=2305, target_porosity=0.30, steps=200, tol=1e-8):
    """Random 3x3 fractal carpet on n^2 (n = 3^k), transient diffusion from a
    left-face source held at c = 1 (c = 0 initially), precipitate-driven
    eigenstrain, equilibrium CG and phase field every step.
    Time step dt = (n/4)^2 / steps in grid units, so the front reaches
    about a quarter of the width by the last step."""
    phase, _ = random_carpet(n, target_porosity, seed)
    return Workload(
        name=f"random-carpet-{n}x{n}", phase=phase, materials=Materials(),
        h=H_MECH, h_diff=H_DIFF, steps=steps, diffusion_mode=DIFF_TRANSIENT,
        eig_mode=EIG_FROM_PRECIPITATE, eig=np.zeros(phase.shape), eig_ramp=[1.0] * steps,
        dt=(n / 4.0) ** 2 / steps, dirichlet_mask=left_face_mask(phase),
        dirichlet_value=1.0, c0=np.zeros(phase.shape), tol=tol,
        extra={"seed": seed, "porosity": porosity(phase)})


def sponge_ramp(n=243, seed=13081, target_porosity=0.35, steps=50, e_final=5e-3):
    """Random Menger-type sponge on n^3, eigenstrain in the pores ramped
    linearly from e_final/steps to e_final over `steps`; no diffusion."""
    phase, _ = random_sponge(n, target_porosity, seed)
    eig = np.where(phase == 0, 1.0, 0.0)
    return Workload(
        name=f"random-sponge-{n}^3", phase=phase, materials=Materials(), h=H_MECH,
        h_diff=H_DIFF, steps=steps, diffusion_mode=DIFF_NONE, eig_mode=EIG_PRESCRIBED,
        eig=eig, eig_ramp=[e_final * (s + 1) / steps for s in range(steps)],
        extra={"seed": seed, "porosity": porosity(phase)})


def carpet_adjoint(n=2187, seed=7, e_seed=8, target_porosity=0.30, steps=30):
    """Random 3x3 carpet on n^2 with a per-voxel pore eigenstrain
    N(1e-3, (2e-4)^2) (seed e_seed), 0 in the solid, ramped linearly over
    `steps` staggered steps (scale (s + 1) / steps); no diffusion. The
    workload of the eigenstrain adjoint."""
    phase, _ = random_carpet(n, target_porosity, seed)
    return Workload(
        name=f"random-carpet-{n}x{n}-eigenstrain-adjoint", phase=phase, materials=Materials(), h=H_MECH,
        h_diff=H_DIFF, steps=steps, diffusion_mode=DIFF_NONE, eig_mode=EIG_PRESCRIBED,
        eig=gaussian_pore_eigenstrain(phase, e_seed), eig_ramp=[(s + 1) / steps for s in range(steps)],
        extra={"seed": seed, "e_seed": e_seed, "porosity": porosity(phase)})


def gaussian_pore_eigenstrain(phase, seed, mean=1e-3, std=2e-4):
    """Per-voxel eigenstrain N(mean, std^2) in the pores, 0 in the solid."""
    z = standard_normal(derive_key(seed, 0xE16), phase.size).reshape(phase.shape)
    return np.where(phase == 0, mean + std * z, 0.0)


def mixed_batch(n3=256, n2=64, steps=20, tol=1e-8, sizes3=(81, 243, 729), sizes2=(128, 256, 512, 1024),
                seed3=0, seed2=1000):
    """Batch of uneven 2D grids: n3 random 3x3 carpets with n drawn uniformly
    from sizes3 (seeds seed3 ..), n2 random 2x2 carpets with n drawn from
    sizes2 (seeds seed2 ..); target porosity uniform in [0.2, 0.45] per
    problem; each a transient-diffusion staggered workload as
    carpet_transient (left-face source, dt = (n/4)^2 / steps). The draws use
    the SplitMix64 stream of each seed."""
    out = []
    for base, count, sizes, s0 in ((3, n3, sizes3, seed3), (2, n2, sizes2, seed2)):
        for i in range(count):
            seed = s0 + i
            u = uniform01(derive_key(seed, 0xB47C), 2)
            n = sizes[min(int(u[0] * len(sizes)), len(sizes) - 1)]
            eta = 0.2 + 0.25 * float(u[1])
            phase, _ = random_carpet(n, eta, seed, base=base)
            out.append(Workload(
                name=f"random-carpet{base}-{n}x{n}", phase=phase, materials=Materials(),
                h=H_MECH, h_diff=H_DIFF, steps=steps, diffusion_mode=DIFF_TRANSIENT,
                eig_mode=EIG_FROM_PRECIPITATE, eig=np.zeros(phase.shape), eig_ramp=[1.0] * steps,
                dt=(n / 4.0) ** 2 / steps, dirichlet_mask=left_face_mask(phase),
                dirichlet_value=1.0, c0=np.zeros(phase.shape), tol=tol,
                extra={"seed": seed, "porosity": porosity(phase), "target_porosity": eta}))
    return out
