"""Pins of the FP64 CPU oracle in three dimensions (d = 3: six strain
components, the 3D bulk factor and deviator of Eq. energy, the 3D Galerkin
operators of Secs. 2.1, 2.3 and 2.4), against what the mathematics fixes:
homogeneous media (a uniform load is the solution; the per-mode closed form
of the equilibrium with a heterogeneous eigenstrain), laminates (Reuss and
harmonic / arithmetic means exact), closed forms of the positive energy
density, the exact phase field of a uniform history, and the backward-Euler
decay of single Fourier modes; and brute-force dense solves of the same
discrete equations on a small two-phase grid."""

import numpy as np
import pytest

from microstructures.workloads import Materials
from oracle import spectral, elasticity, diffusion, phasefield

import dense_reference as dense

H = 5e-6
MAT = Materials()


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def roll_fwd(u, alpha, h):
    ax = u.ndim - 1 - alpha  # alpha = 0 is x, the last array axis
    return (np.roll(u, -1, axis=ax) - u) / h


def test_homogeneous_uniform_load_3d():
    """A uniform strain is the solution in a homogeneous medium: the
    projected right-hand side vanishes up to the FFT's rounding (the CG may
    take a step or two on that rounding), and the strain stays E."""
    shape = (4, 5, 6)
    phase = np.ones(shape, dtype=np.uint8)
    E = [1e-3, -2e-3, 5e-4, 3e-4, -1e-4, 2e-4]  # xx, yy, zz, yz, xz, xy
    out = elasticity.equilibrium_solve(phase, np.zeros(shape), np.ones(shape), E, MAT, H)
    for I in range(6):
        assert np.allclose(out["strain"][I], E[I], rtol=0, atol=1e-17)
    lam, mu = elasticity.lame(MAT.E_solid, MAT.nu_solid)
    assert np.allclose(out["stress"][0], lam * (E[0] + E[1] + E[2]) + 2 * mu * E[0], rtol=1e-13)
    assert np.allclose(out["stress"][3], 2 * mu * E[3], rtol=1e-13)
    dif = diffusion.homogenise(phase, MAT, (1.0, 0.5, -0.25), 1.0, 1.0)
    for a, g in enumerate((1.0, 0.5, -0.25)):
        assert np.allclose(dif["grad_c"][a], g, rtol=0, atol=1e-14)


def test_homogeneous_medium_heterogeneous_eigenstrain_closed_form_3d():
    """Per-mode closed form u_hat = K_hat^-1 f_hat with
    K_hat = mu lam_k I + lambda conj(D) D^T + mu D D^H for the forward
    differences D_a = (exp(i theta_a) - 1) / h, f_hat = conj(D) (3 lambda +
    2 mu) e_hat (an isotropic eigenstrain e I in three dimensions)."""
    shape = (6, 5, 4)  # (z, y, x)
    rng = np.random.default_rng(7)
    e = 1e-3 * rng.standard_normal(shape)
    phase = np.ones(shape, dtype=np.uint8)
    out = elasticity.equilibrium_solve(phase, e, np.ones(shape), [0] * 6, MAT, H, tol=1e-14)
    lam, mu = elasticity.lame(MAT.E_solid, MAT.nu_solid)
    D = spectral.forward_difference_symbol(shape, H)
    eh = np.fft.fftn(e)
    uh = np.zeros((3,) + shape, dtype=complex)
    for idx in np.ndindex(shape):
        Dk = np.array([D[a][idx] for a in range(3)])
        lk = float(np.sum(np.abs(Dk) ** 2))
        if lk == 0:
            continue
        K = mu * lk * np.eye(3) + lam * np.outer(np.conj(Dk), Dk) + mu * np.outer(Dk, np.conj(Dk))
        f = np.conj(Dk) * (3 * lam + 2 * mu) * eh[idx]
        uh[(slice(None),) + idx] = np.linalg.solve(K, f)
    u = np.fft.ifftn(uh, axes=(1, 2, 3)).real
    g = [[roll_fwd(u[i], j, H) for j in range(3)] for i in range(3)]
    ref = np.stack([g[0][0], g[1][1], g[2][2], 0.5 * (g[1][2] + g[2][1]), 0.5 * (g[0][2] + g[2][0]),
                    0.5 * (g[0][1] + g[1][0])])
    assert rel(out["strain"], ref) < 1e-11


def laminate3(shape=(3, 4, 12)):
    """Layers normal to x: the phase depends on x only."""
    col = np.array([1, 1, 0, 1, 0, 0, 1, 1, 1, 0, 1, 0], dtype=np.uint8)
    return np.broadcast_to(col, shape).copy()


def test_laminate_elastic_reuss_exact_3d():
    phase = laminate3()
    lam, mu = elasticity.phase_lame(phase, MAT)
    ones = np.ones(phase.shape)
    # uniaxial strain along the layer normal: sigma_xx = <1 / (lambda + 2 mu)>^-1 E_xx
    out = elasticity.equilibrium_solve(phase, 0 * ones, ones, [1.0, 0, 0, 0, 0, 0], MAT, H)
    assert np.allclose(out["stress"][0], 1.0 / np.mean(1.0 / (lam + 2 * mu)), rtol=1e-12)
    # shear across the layers (xy and xz): sigma = 2 <1 / mu>^-1 E (tensor shear)
    out = elasticity.equilibrium_solve(phase, 0 * ones, ones, [0, 0, 0, 0, 0, 1.0], MAT, H)
    assert np.allclose(out["stress"][5], 2.0 / np.mean(1.0 / mu), rtol=1e-12)
    out = elasticity.equilibrium_solve(phase, 0 * ones, ones, [0, 0, 0, 0, 1.0, 0], MAT, H)
    assert np.allclose(out["stress"][4], 2.0 / np.mean(1.0 / mu), rtol=1e-12)


def test_laminate_diffusion_harmonic_and_arithmetic_3d():
    phase = laminate3()
    Dx = diffusion.diffusivity(phase, MAT)
    out = diffusion.homogenise(phase, MAT, (1.0, 0.0, 0.0), 1.0, 1.0, tol=1e-14)
    assert out["mean_flux"][0] == pytest.approx(-1.0 / np.mean(1.0 / Dx), rel=1e-11)
    out = diffusion.homogenise(phase, MAT, (0.0, 0.0, 1.0), 1.0, 1.0, tol=1e-14)
    assert out["mean_flux"][2] == pytest.approx(-np.mean(Dx), rel=1e-12)


def test_psi_plus_closed_forms_3d():
    """Eq. energy in d = 3: psi+ = 1/2 K [tr eps]_+^2 + mu eps_dev : eps_dev
    with K = lambda + 2 mu / 3 and eps_dev = eps - tr(eps) / 3 I, of the
    elastic strain eps - e I."""
    lam, mu = 7.0, 3.0
    K = lam + 2 * mu / 3
    one = np.ones(1)
    a = 2e-3
    vol = np.array([a, a, a, 0, 0, 0])[:, None] * one
    assert elasticity.psi_plus(vol, 0.0, lam, mu)[0] == pytest.approx(0.5 * K * (3 * a) ** 2, rel=1e-14)
    assert elasticity.psi_plus(-vol, 0.0, lam, mu)[0] == pytest.approx(0.0, abs=1e-20)
    # an eigenstrain equal to the strain leaves no elastic strain
    assert elasticity.psi_plus(vol, a, lam, mu)[0] == pytest.approx(0.0, abs=1e-20)
    # pure shear (tensor component eps_xy = g, Voigt slot 5): dev:dev = 2 g^2
    g = 1e-3
    shear = np.array([0, 0, 0, 0, 0, g])[:, None] * one
    assert elasticity.psi_plus(shear, 0.0, lam, mu)[0] == pytest.approx(mu * 2 * g * g, rel=1e-14)
    # deviatoric uniaxial part of a compressive uniaxial strain still counts
    uni = np.array([-a, 0, 0, 0, 0, 0])[:, None] * one
    dev2 = (2 * a / 3) ** 2 + 2 * (a / 3) ** 2
    assert elasticity.psi_plus(uni, 0.0, lam, mu)[0] == pytest.approx(mu * dev2, rel=1e-13)


def test_phasefield_uniform_history_exact_3d():
    Hval = 3e4
    Hf = np.full((5, 4, 6), Hval)
    d, info = phasefield.phasefield_solve(Hf, MAT, H)
    a, b = phasefield.coefficients(MAT)
    assert np.allclose(d, Hval / (a + Hval), rtol=1e-13)
    assert info["iters"] <= 1


@pytest.mark.parametrize("k", [(0, 1, 2), (3, 0, 1), (1, 2, 0)])
def test_transient_single_mode_decay_3d(k):
    shape = (6, 5, 8)  # (z, y, x)
    Dc, dt, h = 0.7, 2.5, 1.0
    mat = Materials(D_solid=Dc, D_pore=Dc)
    z, y, x = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    kz, ky, kx = k
    c0 = np.cos(2 * np.pi * (kx * x / shape[2] + ky * y / shape[1] + kz * z / shape[0]))
    lam_k = sum(2 - 2 * np.cos(2 * np.pi * kk / n) for kk, n in zip((kx, ky, kz), (shape[2], shape[1], shape[0])))
    lam_k /= h ** 2
    c1 = diffusion.transient_step(np.ones(shape, np.uint8), c0, mat, dt, h)
    assert np.abs(c1 - c0 / (1 + Dc * dt * lam_k)).max() < 1e-13


# ---------------------------------------------------------------- dense direct solves in 3D
# The same discrete equations assembled from real-space forward differences
# and solved directly (tests/dense_reference.py), on a small two-phase grid
# with damage, eigenstrain and a full macro strain.


@pytest.fixture(scope="module")
def small_case_3d():
    rng = np.random.default_rng(11)
    phase = (rng.random((4, 5, 6)) > 0.35).astype(np.uint8)
    eig = np.where(phase == 0, 1e-3 + 2e-4 * rng.standard_normal(phase.shape), 0.0)
    dmg = np.clip(0.5 * rng.random(phase.shape), 0, 1)
    return phase, eig, dmg


def test_dense_equilibrium_3d(small_case_3d):
    phase, eig, dmg = small_case_3d
    g = phasefield.degradation(dmg, MAT.kappa)
    E = [2e-4, -1e-4, 3e-4, 5e-5, -4e-5, 6e-5]
    ref = dense.elastic(phase, eig, g, E, MAT, H)
    out = elasticity.equilibrium_solve(phase, eig, g, E, MAT, H, tol=1e-14)
    assert rel(out["strain"], ref["strain"]) < 1e-10
    assert rel(out["stress"], ref["stress"]) < 1e-10


def test_dense_diffusion_3d(small_case_3d):
    phase, _, _ = small_case_3d
    G = (1.0, 0.3, -0.2)
    ref = dense.homogenise(phase, MAT, G, 1.0, 1.0)
    out = diffusion.homogenise(phase, MAT, G, 1.0, 1.0, tol=1e-14)
    assert rel(out["c"], ref["c"]) < 1e-11
    assert rel(out["grad_c"], ref["grad_c"]) < 1e-11
    assert np.allclose(out["mean_flux"], ref["mean_flux"], rtol=1e-10)


def test_dense_phasefield_3d(small_case_3d):
    phase, _, _ = small_case_3d
    rng = np.random.default_rng(12)
    Hf = 1e5 * rng.random(phase.shape) ** 4
    ref = dense.phasefield(Hf, MAT, H)
    d, _ = phasefield.phasefield_solve(Hf, MAT, H, tol=1e-14)
    assert rel(d, ref) < 1e-11


def test_random_sponge_seeded_and_in_window():
    from microstructures import random_sponge, porosity

    p1, a1 = random_sponge(27, 0.35, 5)
    p2, a2 = random_sponge(27, 0.35, 5)
    assert p1.shape == (27, 27, 27) and p1.dtype == np.uint8
    assert a1 == a2 and np.array_equal(p1, p2)
    assert abs(porosity(p1) - 0.35) <= 0.02
    p3, _ = random_sponge(27, 0.35, 6)
    assert not np.array_equal(p1, p3)
