"""The z-slab decomposition of one 3D grid (paper_2305_13081_gb300.slab) on
two CPU ranks (torch.distributed, gloo, 127.0.0.1): halo exchange and
all-to-all transposes exact, and the slab-decomposed equilibrium PCG
(Sec. 2.3) on a random 3D sponge with a pore eigenstrain matching the
single-domain FP64 oracle on every rank's planes. Uneven splits (9 planes,
9 ky rows over 2 ranks) are exercised.

The per-slab arithmetic (forward-difference stencil, x-y and z transforms)
is plain CPU tensor arithmetic written here: the test checks the
decomposition, not the GPU kernels.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from microstructures import random_sponge
from microstructures.workloads import Materials
from oracle import elasticity

H = 5e-6
MAT = Materials(E_pore=2e9)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def case():
    phase, _ = random_sponge(9, 0.3, 6)
    rng = np.random.default_rng(3)
    e = np.where(phase == 0, 2e-2 * (1.0 + 0.2 * rng.standard_normal(phase.shape)), 0.0)
    return phase, e


class TorchSlabOps:
    """Per-slab arithmetic of 3D elasticity on planes [z0, z1) (plus the
    bottom halo plane for the stresses), E = 0, g = 1."""

    def __init__(self, phase, e, plan):
        from paper_2305_13081_gb300.slab import SlabPlan  # noqa: F401
        nz = phase.shape[0]
        zs = [(plan.z0 - 1 + k) % nz for k in range(plan.nzl + 2)]  # halo-extended planes
        lam, mu = elasticity.phase_lame(phase, MAT)
        self.lam = torch.as_tensor(lam[zs])
        self.mu = torch.as_tensor(mu[zs])
        self.e = torch.as_tensor(e[zs])
        self.plan = plan
        self.h = H

    def _stress(self, u_h, with_eig):
        """Stress on planes 0 .. nzl (z0 - 1 .. z1 - 1) of u_h (3, nzl + 2, ny, nx)."""
        ih = 1.0 / self.h
        ux, uy, uz = u_h[0], u_h[1], u_h[2]

        def dx(a):
            return (torch.roll(a, -1, dims=-1) - a) * ih

        def dy(a):
            return (torch.roll(a, -1, dims=-2) - a) * ih

        def dz(a):
            return (a[1:] - a[:-1]) * ih

        s = slice(0, -1)
        exx, eyy, ezz = dx(ux)[s], dy(uy)[s], dz(uz)
        eyz = 0.5 * (dz(uy) + dy(uz)[s])
        exz = 0.5 * (dz(ux) + dx(uz)[s])
        exy = 0.5 * (dy(ux) + dx(uy))[s]
        lam, mu = self.lam[:-1], self.mu[:-1]
        if with_eig:
            ee = self.e[:-1]
            exx, eyy, ezz = exx - ee, eyy - ee, ezz - ee
        tr = exx + eyy + ezz
        return (lam * tr + 2 * mu * exx, lam * tr + 2 * mu * eyy, lam * tr + 2 * mu * ezz,
                2 * mu * eyz, 2 * mu * exz, 2 * mu * exy)

    def _div_t(self, S):
        """grad+^T sigma on planes 1 .. nzl: -(backward differences)."""
        ih = 1.0 / self.h
        sxx, syy, szz, syz, sxz, sxy = S

        def bx(a):
            return (torch.roll(a, 1, dims=-1) - a)[1:] * ih

        def by(a):
            return (torch.roll(a, 1, dims=-2) - a)[1:] * ih

        def bz(a):
            return (a[:-1] - a[1:]) * ih

        return torch.stack([bx(sxx) + by(sxy) + bz(sxz), bx(sxy) + by(syy) + bz(syz), bx(sxz) + by(syz) + bz(szz)])

    def apply_K(self, p_h):
        return -self._div_t(self._stress(p_h, False))

    def residual(self, u_h):
        return self._div_t(self._stress(u_h, True))

    def fft_xy(self, x):
        return torch.fft.fft2(x)

    def ifft_xy(self, X):
        return torch.fft.ifft2(X)

    def z_multiply(self, Y, plan):
        nx, ny, nz = plan.nx, plan.ny, plan.nz
        kz = torch.arange(nz, dtype=torch.float64).reshape(nz, 1, 1)
        ky = torch.arange(plan.y0, plan.y1, dtype=torch.float64).reshape(1, -1, 1)
        kx = torch.arange(nx, dtype=torch.float64).reshape(1, 1, nx)
        lam = (2 - 2 * torch.cos(2 * np.pi * kx / nx)) + (2 - 2 * torch.cos(2 * np.pi * ky / ny)) + \
              (2 - 2 * torch.cos(2 * np.pi * kz / nz))
        m = torch.where(lam > 0, self.h * self.h / torch.where(lam > 0, lam, torch.ones_like(lam)), torch.zeros_like(lam))
        Z = torch.fft.fft(Y, dim=1)
        return torch.fft.ifft(Z * m, dim=1)


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2305_13081_gb300 import slab
        phase, e = case()
        nz, ny, nx = phase.shape
        plan = slab.SlabPlan(nx, ny, nz, world, rank)
        # exchanges against their definitions
        rng = np.random.default_rng(7)
        full = torch.as_tensor(rng.standard_normal((2, nz, ny, nx)))
        xh = torch.zeros(2, plan.nzl + 2, ny, nx, dtype=torch.float64)
        xh[:, 1:-1] = full[:, plan.z0:plan.z1]
        slab.halo_exchange(xh, plan)
        halo_ok = bool(torch.equal(xh[:, 0], full[:, (plan.z0 - 1) % nz]) and
                       torch.equal(xh[:, -1], full[:, plan.z1 % nz]))
        X = torch.fft.fft2(full[:, plan.z0:plan.z1].to(torch.complex128))
        Y = slab.transpose_z_to_y(X, plan)
        Yref = torch.fft.fft2(full.to(torch.complex128))[:, :, plan.y0:plan.y1]
        tr_ok = bool(torch.equal(Y, Yref)) and bool(torch.equal(slab.transpose_y_to_z(Y, plan), X))
        (tot,) = slab.allreduce_sum([float(rank + 1)])
        # the equilibrium solve
        ops = TorchSlabOps(phase, e, plan)
        u, iters, relres = slab.slab_pcg(ops, plan, torch.zeros(3, plan.nzl, ny, nx, dtype=torch.float64), tol=1e-12)
        uh = torch.zeros(3, plan.nzl + 2, ny, nx, dtype=torch.float64)
        uh[:, 1:-1] = u
        slab.halo_exchange(uh, plan)
        ih = 1.0 / H

        def d(a, axis):
            return (torch.roll(a, -1, dims=axis) - a) * ih

        interior = slice(1, -1)
        exx = d(uh[0], -1)[interior]
        eyy = d(uh[1], -2)[interior]
        ezz = ((uh[2][2:] - uh[2][1:-1]) * ih)
        eyz = 0.5 * ((uh[1][2:] - uh[1][1:-1]) * ih + d(uh[2], -2)[interior])
        exz = 0.5 * ((uh[0][2:] - uh[0][1:-1]) * ih + d(uh[2], -1)[interior])
        exy = 0.5 * (d(uh[0], -2) + d(uh[1], -1))[interior]
        strain = torch.stack([exx, eyy, ezz, eyz, exz, exy]).numpy()
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), strain=strain, z0=plan.z0, z1=plan.z1, iters=iters,
                 relres=relres, halo_ok=halo_ok, tr_ok=tr_ok, tot=tot)
    finally:
        dist.destroy_process_group()


def test_slab_decomposed_pcg_matches_single_domain_oracle(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)
    phase, e = case()
    ref = elasticity.equilibrium_solve(phase, e, np.ones(phase.shape), [0.0] * 6, MAT, H, tol=1e-12)
    planes = 0
    for r in range(world):
        out = np.load(os.path.join(str(tmp_path), f"rank{r}.npz"))
        assert bool(out["halo_ok"]) and bool(out["tr_ok"])
        assert float(out["tot"]) == 3.0
        z0, z1 = int(out["z0"]), int(out["z1"])
        planes += z1 - z0
        got = out["strain"]
        want = ref["strain"][:, z0:z1]
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err < 1e-9, (r, err)
        assert float(out["relres"]) <= 1e-12 and int(out["iters"]) > 5
    assert planes == phase.shape[0]
