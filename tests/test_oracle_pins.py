"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix:
projection algebra (App. A), closed forms (homogeneous media, single Fourier
modes, the 1D phase-field profile, laminates), bounds (Voigt / Reuss),
averaging identities (Sec. 2.1, Eq. concentration-correct), invariants of the
phase field (Sec. 2.4), the CG energy decrease, brute-force dense solves of the
same discrete equations, and the equivalence of the paper's gradient-space CG
with a potential-space preconditioned CG.
"""

import os

import numpy as np
import pytest

from microstructures import sierpinski_carpet, random_carpet, porosity
from microstructures.splitmix import splitmix64_stream
from microstructures.workloads import Materials
from oracle import spectral, elasticity, diffusion, phasefield, chemistry, staggered
from oracle.krylov import dot

import dense_reference as dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
H = 5e-6
MAT = Materials()


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def roll_fwd(u, alpha, h):
    ax = u.ndim - 1 - alpha
    return (np.roll(u, -1, axis=ax) - u) / h


# ---------------------------------------------------------------- generators

def test_splitmix64_published_vector():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    got = [int(x) for x in splitmix64_stream(1234567, 5)]
    assert got == vals


def test_sierpinski_porosity_exact():
    for L in (1, 2, 3, 4):
        assert porosity(sierpinski_carpet(L)) == pytest.approx(1 - (8 / 9) ** L, abs=1e-15)
    assert porosity(sierpinski_carpet(2, dim=3)) == pytest.approx(1 - (26 / 27) ** 2, abs=1e-15)


def test_random_carpet_seeded_and_in_window():
    p1, a1 = random_carpet(81, 0.30, 5)
    p2, a2 = random_carpet(81, 0.30, 5)
    assert a1 == a2 and np.array_equal(p1, p2)
    assert abs(porosity(p1) - 0.30) <= 0.02
    p3, _ = random_carpet(81, 0.30, 6)
    assert not np.array_equal(p1, p3)


# ---------------------------------------------------------------- P1 projections

@pytest.mark.parametrize("shape", [(9, 9), (8, 12), (5, 6, 7)])
def test_projection_G_algebra(shape):
    rng = np.random.default_rng(1)
    d = len(shape)
    D = spectral.forward_difference_symbol(shape, 0.7)
    g = spectral.projection_operator(D)
    f = rng.standard_normal((d,) + shape)
    w = rng.standard_normal((d,) + shape)
    Gf = spectral.apply_G(g, f)
    # idempotent
    assert rel(spectral.apply_G(g, Gf), Gf) < 1e-13
    # self-adjoint in the l2 product
    assert abs(dot(spectral.apply_G(g, f), w) - dot(f, spectral.apply_G(g, w))) < 1e-12 * np.sqrt(dot(f, f) * dot(w, w))
    # leaves a real-space forward-difference gradient unchanged
    s = rng.standard_normal(shape)
    grad = np.stack([roll_fwd(s, a, 0.7) for a in range(d)])
    assert rel(spectral.apply_G(g, grad), grad) < 1e-13
    # kills constants
    c = np.ones((d,) + shape) * np.arange(1, d + 1).reshape((d,) + (1,) * d)
    assert np.abs(spectral.apply_G(g, c)).max() < 1e-13
    # curl-free output: the result is the forward gradient of some potential
    phi = spectral.solve_poisson_from_gradient(Gf, D)
    assert rel(np.stack([roll_fwd(phi, a, 0.7) for a in range(d)]), Gf) < 1e-12


def test_projection_GG_rowwise():
    shape = (9, 10)
    rng = np.random.default_rng(2)
    D = spectral.forward_difference_symbol(shape, 1.3)
    g = spectral.projection_operator(D)
    A = rng.standard_normal((2, 2) + shape)
    GA = spectral.apply_GG(g, A)
    assert rel(spectral.apply_GG(g, GA), GA) < 1e-13
    for i in range(2):
        assert rel(GA[i], spectral.apply_G(g, A[i])) < 1e-14
    u = rng.standard_normal((2,) + shape)
    F = np.stack([np.stack([roll_fwd(u[i], j, 1.3) for j in range(2)]) for i in range(2)])
    assert rel(spectral.apply_GG(g, F), F) < 1e-13


def test_symbol_sign_convention():
    # F^-1(D F(u)) must be the real-space forward difference (Sec. 2.6)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((6, 7))
    D = spectral.forward_difference_symbol(u.shape, 0.5)
    du = spectral.spectral_derivative(u, D)
    for a in range(2):
        assert np.abs(du[a] - roll_fwd(u, a, 0.5)).max() < 1e-12


# ---------------------------------------------------------------- P2 homogeneous

def test_homogeneous_uniform_load_zero_iterations():
    phase = np.ones((9, 9), dtype=np.uint8)
    out = elasticity.equilibrium_solve(phase, np.zeros((9, 9)), np.ones((9, 9)), [1e-3, -2e-3, 5e-4], MAT, H)
    assert out["iters"] == 0
    assert np.allclose(out["strain"][0], 1e-3) and np.allclose(out["strain"][2], 5e-4)
    dif = diffusion.homogenise(phase, MAT, (1.0, 0.5), 1.0, 1.0)
    assert dif["iters"] == 0
    assert np.allclose(dif["grad_c"][0], 1.0) and np.allclose(dif["grad_c"][1], 0.5)


def test_homogeneous_medium_heterogeneous_eigenstrain_closed_form():
    """Per-mode closed form u_hat = K_hat^-1 f_hat with
    K_hat = mu lam_k I + lambda conj(D) D^T + mu D D^H (forward differences)."""
    shape = (12, 9)
    rng = np.random.default_rng(4)
    e = 1e-3 * rng.standard_normal(shape)
    phase = np.ones(shape, dtype=np.uint8)
    out = elasticity.equilibrium_solve(phase, e, np.ones(shape), [0, 0, 0], MAT, H, tol=1e-14)
    lam, mu = elasticity.lame(MAT.E_solid, MAT.nu_solid)
    D = spectral.forward_difference_symbol(shape, H)
    eh = np.fft.fftn(e)
    uh = np.zeros((2,) + shape, dtype=complex)
    for idx in np.ndindex(shape):
        Dk = np.array([D[0][idx], D[1][idx]])
        lk = float(np.sum(np.abs(Dk) ** 2))
        if lk == 0:
            continue
        K = mu * lk * np.eye(2) + lam * np.outer(np.conj(Dk), Dk) + mu * np.outer(Dk, np.conj(Dk))
        f = np.conj(Dk) * (2 * lam + 2 * mu) * eh[idx]
        uh[(slice(None),) + idx] = np.linalg.solve(K, f)
    u = np.fft.ifftn(uh, axes=(1, 2)).real
    exx = roll_fwd(u[0], 0, H)
    eyy = roll_fwd(u[1], 1, H)
    exy = 0.5 * (roll_fwd(u[0], 1, H) + roll_fwd(u[1], 0, H))
    assert rel(out["strain"], np.stack([exx, eyy, exy])) < 1e-11


def test_homogeneous_diffusion_and_phasefield_one_pcg_iteration():
    """With a homogeneous coefficient the Fourier preconditioner is the exact
    inverse: the potential-form PCG converges in one iteration. Checked on the
    phase field with uniform H, whose exact solution is d = H / (a + H)."""
    Hval = 3e4
    Hf = np.full((8, 9), Hval)
    d, info = phasefield.phasefield_solve(Hf, MAT, H)
    a, b = phasefield.coefficients(MAT)
    assert np.allclose(d, Hval / (a + Hval), rtol=1e-13)
    assert info["iters"] <= 1


# ---------------------------------------------------------------- P3 mode decay

@pytest.mark.parametrize("k", [(0, 1), (2, 3), (4, 0)])
def test_transient_single_mode_decay(k):
    shape = (9, 12)
    Dc, dt, h = 0.7, 2.5, 1.0
    mat = Materials(D_solid=Dc, D_pore=Dc)
    y, x = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
    ky, kx = k
    c0 = np.cos(2 * np.pi * (kx * x / shape[1] + ky * y / shape[0]))
    lam_k = (2 - 2 * np.cos(2 * np.pi * kx / shape[1]) + 2 - 2 * np.cos(2 * np.pi * ky / shape[0])) / h ** 2
    c1 = diffusion.transient_step(np.ones(shape, np.uint8), c0, mat, dt, h)
    assert np.abs(c1 - c0 / (1 + Dc * dt * lam_k)).max() < 1e-13


def test_transient_converges_to_continuous_decay():
    """Backward Euler on the forward-difference Laplacian approaches
    exp(-D |xi|^2 t) as dt, h -> 0 (first order in dt)."""
    errs = []
    for n, steps in ((16, 8), (32, 32)):
        L, T, Dc = 1.0, 0.01, 1.0
        h = L / n
        mat = Materials(D_solid=Dc, D_pore=Dc)
        x = h * np.arange(n)
        c = np.tile(np.cos(2 * np.pi * x / L), (1, 1))
        for _ in range(steps):
            c = diffusion.transient_step(np.ones((1, n), np.uint8), c, mat, T / steps, h)
        exact = np.exp(-Dc * (2 * np.pi / L) ** 2 * T) * np.cos(2 * np.pi * x / L)
        errs.append(np.abs(c[0] - exact).max())
    assert errs[1] < errs[0] / 3.0


# ---------------------------------------------------------------- P4 1D profile

def test_phasefield_1d_profile_exact():
    n = 41
    hh = 2.5e-6
    Hf = np.zeros((1, n))
    hsrc = 7e5
    Hf[0, 0] = hsrc
    d, _ = phasefield.phasefield_solve(Hf, MAT, hh, tol=1e-14)
    a, b = phasefield.coefficients(MAT)
    q = 2 + (hh / MAT.l0) ** 2
    r = (q - np.sqrt(q * q - 4)) / 2
    i = np.arange(n)
    shape_fn = r ** i + r ** (n - i)
    A = hsrc / ((a + hsrc) * shape_fn[0] + (b / hh ** 2) * (2 * shape_fn[0] - shape_fn[1] - shape_fn[-1]))
    assert np.abs(d[0] - A * shape_fn).max() < 1e-13


# ---------------------------------------------------------------- P5 laminates

def laminate():
    shape = (6, 12)
    col = np.array([1, 1, 0, 1, 0, 0, 1, 1, 1, 0, 1, 0], dtype=np.uint8)
    return np.tile(col, (shape[0], 1))


def test_laminate_elastic_reuss_exact():
    phase = laminate()
    lam, mu = elasticity.phase_lame(phase, MAT)
    out = elasticity.equilibrium_solve(phase, np.zeros(phase.shape), np.ones(phase.shape), [1.0, 0, 0], MAT, H)
    M = lam + 2 * mu
    assert np.allclose(out["stress"][0], 1.0 / np.mean(1.0 / M), rtol=1e-12)
    out = elasticity.equilibrium_solve(phase, np.zeros(phase.shape), np.ones(phase.shape), [0, 0, 1.0], MAT, H)
    assert np.allclose(out["stress"][2], 2.0 / np.mean(1.0 / mu), rtol=1e-12)


def test_laminate_diffusion_harmonic_and_arithmetic():
    phase = laminate()
    Dx = diffusion.diffusivity(phase, MAT)
    out = diffusion.homogenise(phase, MAT, (1.0, 0.0), 1.0, 1.0, tol=1e-14)
    assert out["mean_flux"][0] == pytest.approx(-1.0 / np.mean(1.0 / Dx), rel=1e-11)
    out = diffusion.homogenise(phase, MAT, (0.0, 1.0), 1.0, 1.0, tol=1e-14)
    assert out["mean_flux"][1] == pytest.approx(-np.mean(Dx), rel=1e-12)


# ---------------------------------------------------------------- P6 bounds

def test_effective_stiffness_symmetric_and_bounded():
    phase = sierpinski_carpet(2)  # 9 x 9, square symmetry
    C = elasticity.effective_stiffness(phase, MAT, H)
    W = np.diag([1.0, 1.0, 2.0])
    A = W @ C
    assert np.abs(A - A.T).max() < 1e-10 * np.abs(A).max()
    assert C[0, 0] == pytest.approx(C[1, 1], rel=1e-10)
    lam, mu = elasticity.phase_lame(phase, MAT)
    Ax = np.zeros(phase.shape + (3, 3))
    Ax[..., 0, 0] = Ax[..., 1, 1] = lam + 2 * mu
    Ax[..., 0, 1] = Ax[..., 1, 0] = lam
    Ax[..., 2, 2] = 4 * mu  # W C for the shear slot
    voigt = Ax.reshape(-1, 3, 3).mean(axis=0)
    reuss = np.linalg.inv(np.linalg.inv(Ax.reshape(-1, 3, 3)).mean(axis=0))
    scale = np.abs(voigt).max()
    assert np.linalg.eigvalsh(voigt - 0.5 * (A + A.T)).min() > -1e-10 * scale
    assert np.linalg.eigvalsh(0.5 * (A + A.T) - reuss).min() > -1e-10 * scale


def test_effective_diffusivity_between_bounds():
    phase, _ = random_carpet(27, 0.35, 11)
    Dx = diffusion.diffusivity(phase, MAT)
    for gm in ((1.0, 0.0), (0.0, 1.0)):
        out = diffusion.homogenise(phase, MAT, gm, 1.0, 1.0)
        Deff = -out["mean_flux"][0] if gm[0] else -out["mean_flux"][1]
        assert 1 / np.mean(1 / Dx) * (1 - 1e-10) <= Deff <= np.mean(Dx) * (1 + 1e-10)


# ---------------------------------------------------------------- P7 dense solves

@pytest.fixture(scope="module")
def small_case():
    phase, _ = random_carpet(27, 0.30, 3)
    rng = np.random.default_rng(5)
    eig = np.where(phase == 0, 1e-3 + 2e-4 * rng.standard_normal(phase.shape), 0.0)
    dmg = np.clip(0.5 * rng.random(phase.shape), 0, 1)
    return phase, eig, dmg


def test_dense_equilibrium(small_case):
    phase, eig, dmg = small_case
    g = phasefield.degradation(dmg, MAT.kappa)
    E = [2e-4, -1e-4, 3e-4]
    ref = dense.elastic(phase, eig, g, E, MAT, H)
    out = elasticity.equilibrium_solve(phase, eig, g, E, MAT, H, tol=1e-14)
    assert rel(out["strain"], ref["strain"]) < 1e-10
    assert rel(out["stress"], ref["stress"]) < 1e-10


def test_dense_diffusion(small_case):
    phase, _, _ = small_case
    ref = dense.homogenise(phase, MAT, (1.0, 0.3), 1.0, 1.0)
    out = diffusion.homogenise(phase, MAT, (1.0, 0.3), 1.0, 1.0, tol=1e-14)
    assert rel(out["c"], ref["c"]) < 1e-11
    assert rel(out["grad_c"], ref["grad_c"]) < 1e-11
    assert np.allclose(out["mean_flux"], ref["mean_flux"], rtol=1e-10)


def test_dense_phasefield(small_case):
    phase, _, _ = small_case
    rng = np.random.default_rng(6)
    Hf = 1e5 * rng.random(phase.shape) ** 4
    ref = dense.phasefield(Hf, MAT, H)
    d, _ = phasefield.phasefield_solve(Hf, MAT, H, tol=1e-14)
    assert rel(d, ref) < 1e-11


def test_dense_staggered_step(small_case):
    phase, eig, _ = small_case
    mat = Materials(E_pore=20e9 * 1e-3)
    st = staggered.initial_state(phase)
    st["d"] = 0.2 * (phase == 1)
    st["H"] = np.full(phase.shape, 10.0)
    new, _ = staggered.step(st, phase, mat, H, 1.0, staggered.DIFF_HOMOGENISE,
                            staggered.EIG_PRESCRIBED, eig_field=eig, eig_scale=30.0,
                            grad_c_mac=(1.0, 0.0), c_macro=1.0, eps_mac=(1e-3, 0, 0), tol=1e-14)
    # the same step from dense solves
    dif = dense.homogenise(phase, mat, (1.0, 0.0), 1.0, 1.0)
    g = (1 - st["d"]) ** 2 + mat.kappa
    el = dense.elastic(phase, 30.0 * eig, g, [1e-3, 0, 0], mat, H)
    lam, mu = elasticity.phase_lame(phase, mat)
    # psi+ written out for 2D (Eq. energy) from the dense strain
    exx = el["strain"][0] - 30.0 * eig
    eyy = el["strain"][1] - 30.0 * eig
    exy = el["strain"][2]
    tr = exx + eyy
    dev2 = (exx - tr / 2) ** 2 + (eyy - tr / 2) ** 2 + 2 * exy ** 2
    psi = 0.5 * (lam + mu) * np.maximum(tr, 0) ** 2 + mu * dev2
    Hn = np.maximum(st["H"], psi)
    dn = dense.phasefield(Hn, mat, H)
    assert rel(new["c"], dif["c"]) < 1e-11
    assert rel(new["strain"], el["strain"]) < 1e-10
    assert rel(new["stress"], el["stress"]) < 1e-10
    assert rel(new["H"], Hn) < 1e-10
    assert rel(new["d"], dn) < 1e-10


# ---------------------------------------------------------------- P8 averages

def test_averages():
    phase, _ = random_carpet(27, 0.3, 8)
    E = [1e-3, -5e-4, 2e-4]
    eig = np.where(phase == 0, 1e-3, 0.0)
    out = elasticity.equilibrium_solve(phase, eig, np.ones(phase.shape), E, MAT, H)
    assert np.allclose(out["mean_strain"], E, atol=1e-15)
    dif = diffusion.homogenise(phase, MAT, (0.4, -0.2), 2.5, 1.0)
    eta = porosity(phase)
    assert np.allclose(dif["grad_c"].reshape(2, -1).mean(axis=1), [0.4, -0.2], atol=1e-14)
    assert dif["c"].mean() == pytest.approx(2.5, rel=1e-12)
    assert dif["c"][phase == 0].mean() == pytest.approx(2.5 / eta, rel=1e-12)
    assert abs(dif["c"][phase == 1].mean()) < 1e-12


# ---------------------------------------------------------------- P9 phase field

def test_phasefield_invariants():
    rng = np.random.default_rng(9)
    shape = (27, 27)
    H1 = 1e6 * rng.random(shape) ** 6
    d1, _ = phasefield.phasefield_solve(H1, MAT, H)
    assert d1.min() >= -1e-14 and d1.max() <= 1.0
    H2 = np.maximum(H1, 2e6 * rng.random(shape) ** 6)
    d2, _ = phasefield.phasefield_solve(H2, MAT, H)
    assert np.all(d2 >= d1 - 1e-13)
    d0, info = phasefield.phasefield_solve(np.zeros(shape), MAT, H)
    assert np.all(d0 == 0) and info["iters"] == 0


def test_chemistry_macaulay():
    phase = np.array([[0, 0, 1, 0]], dtype=np.uint8)
    c = np.array([[0.2, 0.9, 0.9, 0.5]])
    cp = chemistry.precipitate(c, phase, 0.5)
    assert np.allclose(cp, [[0, 0.4, 0, 0]])
    e = chemistry.eigenstrain(np.array([[0.5, 0.4, 0.6, 0.0]]), phase, 2.002)
    assert np.allclose(e, [[0.001, 0, 0, 0]], atol=1e-15)


# ---------------------------------------------------------------- P10 energy

def test_cg_energy_decreases():
    phase, _ = random_carpet(27, 0.3, 12)
    eig = np.where(phase == 0, 1e-3, 0.0)
    out = elasticity.equilibrium_solve(phase, eig, np.ones(phase.shape), [0, 0, 0], MAT, H, record=True)
    en = np.array(out["info"]["energy"])
    assert len(en) > 10
    assert np.all(np.diff(en) <= 1e-12 * np.abs(en).max())


# ---------------------------------------------------------------- P12 equivalence

def potential_pcg_history(phase, eig, mat, h, iters):
    """Preconditioned CG on the displacement potential: K u = f with
    K = B^T g C sym B (B forward differences), preconditioner the inverse of
    the per-component discrete Laplacian B^T B (zero mean). Written here
    independently of the oracle; returns sqrt(r.z / r0.z0) per iteration."""
    shape = phase.shape
    lam_s, mu_s = elasticity.lame(mat.E_solid, mat.nu_solid)
    lam_p, mu_p = elasticity.lame(mat.E_pore, mat.nu_pore)
    lam = np.where(phase == 1, lam_s, lam_p)
    mu = np.where(phase == 1, mu_s, mu_p)

    def bwd(f, a):
        ax = f.ndim - 1 - a
        return (np.roll(f, 1, axis=ax) - f) / h

    def sig(u, e):
        exx = roll_fwd(u[0], 0, h) - e
        eyy = roll_fwd(u[1], 1, h) - e
        exy = 0.5 * (roll_fwd(u[0], 1, h) + roll_fwd(u[1], 0, h))
        tr = exx + eyy
        return lam * tr + 2 * mu * exx, lam * tr + 2 * mu * eyy, 2 * mu * exy

    def Kop(u, e=0.0):
        sxx, syy, sxy = sig(u, e)
        return np.stack([bwd(sxx, 0) + bwd(sxy, 1), bwd(sxy, 0) + bwd(syy, 1)])

    ny, nx = shape
    L = ((2 - 2 * np.cos(2 * np.pi * np.arange(nx) / nx))[None] +
         (2 - 2 * np.cos(2 * np.pi * np.arange(ny) / ny))[:, None]) / h ** 2
    Minv = np.where(L > 0, 1 / np.where(L > 0, L, 1), 0)

    def prec(r):
        return np.stack([np.fft.ifft2(Minv * np.fft.fft2(ri)).real for ri in r])

    f = -Kop(np.zeros((2,) + shape), eig)
    u = np.zeros_like(f)
    r = f.copy()
    z = prec(r)
    rz = np.sum(r * z)
    rz0 = rz
    p = z.copy()
    hist = [1.0]
    for _ in range(iters):
        q = Kop(p)
        a = rz / np.sum(p * q)
        u += a * p
        r -= a * q
        z = prec(r)
        rzn = np.sum(r * z)
        hist.append(np.sqrt(rzn / rz0))
        p = z + (rzn / rz) * p
        rz = rzn
    return np.array(hist)


def test_gradient_cg_equals_potential_pcg():
    phase, _ = random_carpet(27, 0.3, 4)
    eig = np.where(phase == 0, 1e-3, 0.0)
    out = elasticity.equilibrium_solve(phase, eig, np.ones(phase.shape), [0, 0, 0], MAT, H,
                                       tol=1e-14, record=True)
    hist_grad = np.array(out["info"]["history"][:21])
    hist_pot = potential_pcg_history(phase, eig, MAT, H, 20)
    assert np.allclose(hist_grad, hist_pot, rtol=1e-9, atol=0)
