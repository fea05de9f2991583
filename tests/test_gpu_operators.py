"""Gradient-operator variants (Sec. 2.6 and Fig. 2) through the C ABI, of
the homogenised diffusion (fftmech_homogenise_operator) and of the
mechanical equilibrium (fftmech_equilibrium_operator):

- every operator (forward, central, 8th-order central, Fourier) against
  the FP64 oracle with the same symbol (oracle/diffusion.homogenise(symbol=))
  on a 2D random carpet and a 3D random sponge (odd sizes): phi and grad c
  within 1e-9 relative, the mean flux within 1e-10;
- the forward operator, solved by this spectral-operator PCG, agrees with
  the library's stencil-based HOMOGENISE diffusion (fftmech_diffusion_step):
  two independent GPU paths, one mean flux;
- laminates: every operator gives the harmonic mean of D across layers
  normal to the gradient and the arithmetic mean along them;
- elasticity: every operator against the FP64 oracle with the same symbol
  (oracle/elasticity.equilibrium_solve(symbol=)), 2D with a damage field
  and 3D; the forward operator against the library's stencil-based FP64
  solve; the laminate's closed form (uniform sigma_xx and eps_yy).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from microstructures import random_carpet, random_sponge
from microstructures.workloads import Materials
from oracle import diffusion
from paper_2305_13081_gb300 import build
from paper_2305_13081_gb300 import fftmech as fm

pytestmark = pytest.mark.gpu

MAT = Materials()
OPS = {"forward": fm.FFTMECH_GRAD_FORWARD, "central": fm.FFTMECH_GRAD_CENTRAL,
       "central8": fm.FFTMECH_GRAD_CENTRAL8, "fourier": fm.FFTMECH_GRAD_FOURIER}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    fm.load_library()


def gpu(phase, op, G, tol=1e-13):
    ctx = fm.Context(phase.shape, MAT, fm.FFTMECH_FP64, h_diff=1.0, tol=tol, max_iter=20000)
    N = phase.size
    d = phase.ndim
    ph = torch.as_tensor(phase.ravel()).cuda()
    phi = torch.zeros(N, dtype=torch.float64, device="cuda")
    gc = torch.zeros(d * N, dtype=torch.float64, device="cuda")
    info = fm.fftmech_homogenise_operator(ctx.handle, ph, OPS[op], G, phi, gc)
    ctx.close()
    return info, phi.cpu().numpy().reshape(phase.shape), gc.cpu().numpy().reshape((d,) + phase.shape)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("op", list(OPS))
@pytest.mark.parametrize("dim", [2, 3])
def test_operator_matches_oracle(op, dim):
    if dim == 2:
        phase = random_carpet(81, 0.30, 11)[0]
        G = [1.0, 0.5]
    else:
        phase = random_sponge(9, 0.35, 12)[0]
        G = [1.0, 0.5, -0.25]
    info, phi, gc = gpu(phase, op, G)
    ref = diffusion.homogenise(phase, MAT, G, 0.0, 1.0, tol=1e-13, symbol=op)
    e_phi, e_gc = rel(phi, ref["phi"]), rel(gc, ref["grad_c"])
    e_j = float(np.abs(np.array(info.mean_flux[:dim]) - ref["mean_flux"]).max() / np.abs(ref["mean_flux"]).max())
    print("operator", op, dim, "iterations", info.iters, "phi", e_phi, "grad c", e_gc, "mean flux", e_j)
    assert info.status == fm.FFTMECH_OK
    assert e_phi < 1e-9 and e_gc < 1e-9 and e_j < 1e-10


def test_forward_operator_agrees_with_the_stencil_path():
    phase = random_carpet(243, 0.30, 13)[0]
    G = [1.0, 0.0]
    info, _, _ = gpu(phase, "forward", G, tol=1e-12)
    ctx = fm.Context(phase.shape, MAT, fm.FFTMECH_FP64, h_diff=1.0, tol=1e-12, max_iter=20000)
    ph = torch.as_tensor(phase.ravel()).cuda()
    c = torch.zeros(phase.size, dtype=torch.float64, device="cuda")
    ref = fm.fftmech_diffusion_step(ctx.handle, ph, fm.FFTMECH_DIFF_HOMOGENISE, G, 0.3, 0.0, None, 0.0, c)
    ctx.close()
    a, b = np.array(info.mean_flux[:2]), np.array(ref.mean_flux[:2])
    assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max(), (a, b)


@pytest.mark.parametrize("op", list(OPS))
def test_laminates(op):
    n = 27
    normal = np.zeros((9, n), dtype=np.uint8)
    normal[:, 13:] = 1
    parallel = np.zeros((n, 9), dtype=np.uint8)
    parallel[13:, :] = 1
    D_n = np.where(normal[0] == 0, MAT.D_pore, MAT.D_solid)
    D_p = np.where(parallel[:, 0] == 0, MAT.D_pore, MAT.D_solid)
    i_n, _, _ = gpu(normal, op, [1.0, 0.0])
    i_p, _, _ = gpu(parallel, op, [1.0, 0.0])
    h = 1.0 / np.mean(1.0 / D_n)
    a = np.mean(D_p)
    assert abs(i_n.mean_flux[0] + h) <= 1e-9 * h and abs(i_p.mean_flux[0] + a) <= 1e-9 * a


# ---------------------------------------------------------------- elasticity

def gpu_el(phase, op, E, eig=None, damage=None, tol=1e-13):
    ctx = fm.Context(phase.shape, MAT, fm.FFTMECH_FP64, h=H_EL, tol=tol, max_iter=20000)
    N = phase.size
    d = phase.ndim
    nv = 3 if d == 2 else 6
    dev = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()
    strain = torch.zeros(nv * N, dtype=torch.float64, device="cuda")
    stress = torch.zeros(nv * N, dtype=torch.float64, device="cuda")
    info = fm.fftmech_equilibrium_operator(ctx.handle, torch.as_tensor(phase.ravel()).cuda(), dev(eig), dev(damage),
                                           E, OPS[op], strain, stress)
    ctx.close()
    return (info, strain.cpu().numpy().reshape((nv,) + phase.shape),
            stress.cpu().numpy().reshape((nv,) + phase.shape))


H_EL = 5e-6


@pytest.mark.parametrize("op", list(OPS))
@pytest.mark.parametrize("dim", [2, 3])
def test_elastic_operator_matches_oracle(op, dim):
    """Equilibrium with every gradient operator against the FP64 oracle
    (oracle/elasticity.equilibrium_solve(symbol=)): a carpet with a pore
    eigenstrain, a damage field (2D) and a macro strain with a shear."""
    from oracle import elasticity
    rng = np.random.default_rng(17)
    if dim == 2:
        phase = random_carpet(81, 0.30, 14)[0]
        E = [1e-3, -2e-4, 3e-4]
        damage = np.where(phase == 1, 0.6 * rng.random(phase.shape), 0.0)
    else:
        phase = random_sponge(9, 0.35, 15)[0]
        E = [1e-3, 0.0, -2e-4, 1e-4, 0.0, 3e-4]
        damage = None
    eig = np.where(phase == 0, 1e-3, 0.0)
    g = np.ones(phase.shape) if damage is None else (1.0 - damage) ** 2 + MAT.kappa
    info, strain, stress = gpu_el(phase, op, E, eig, damage)
    ref = elasticity.equilibrium_solve(phase, eig, g, E, MAT, H_EL, tol=1e-13, symbol=op)
    e_eps, e_sig = rel(strain, ref["strain"]), rel(stress, ref["stress"])
    e_mean = float(np.abs(np.array(info.mean_stress[:len(E)]) - ref["mean_stress"]).max()
                   / np.abs(ref["mean_stress"]).max())
    print("elastic operator", op, dim, "iterations", info.iters, "strain", e_eps, "stress", e_sig, "mean", e_mean)
    assert info.status == fm.FFTMECH_OK
    assert e_eps < 1e-9 and e_sig < 1e-9 and e_mean < 1e-10
    assert np.allclose(info.mean_strain[:len(E)], E, rtol=0, atol=1e-18)


def test_forward_elastic_operator_agrees_with_the_stencil_path():
    """The forward operator by this spectral-operator PCG and the library's
    stencil-based FP64 equilibrium solve: two independent GPU paths, one
    field."""
    phase = random_carpet(243, 0.30, 16)[0]
    eig = np.where(phase == 0, 1e-3, 0.0)
    E = [1e-3, 0.0, 2e-4]
    _, strain, _ = gpu_el(phase, "forward", E, eig, tol=1e-12)
    ctx = fm.Context(phase.shape, MAT, fm.FFTMECH_FP64, h=H_EL, tol=1e-12, max_iter=20000)
    N = phase.size
    u = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    s2 = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    fm.fftmech_equilibrium_solve(ctx.handle, torch.as_tensor(phase.ravel()).cuda(),
                                 torch.as_tensor(eig.ravel()).cuda(), None, E, u, s2, None)
    ctx.close()
    e = rel(strain, s2.cpu().numpy().reshape(strain.shape))
    assert e < 1e-9, e


@pytest.mark.parametrize("op", list(OPS))
def test_elastic_laminate_closed_form(op):
    """Layers normal to x under a macro strain E_yy (plane strain): eps_yy
    stays E_yy and sigma_xx is uniform, sigma_xx = <lam / M> / <1 / M> E_yy
    with M = lam + 2 mu, for every operator (odd size: no operator vanishes
    at a nonzero frequency)."""
    from oracle.elasticity import lame
    n = 27
    phase = np.zeros((9, n), dtype=np.uint8)
    phase[:, 13:] = 1
    Eyy = 1e-3
    _, strain, stress = gpu_el(phase, op, [0.0, Eyy, 0.0])
    ls, ms = lame(MAT.E_solid, MAT.nu_solid)
    lp, mp = lame(MAT.E_pore, MAT.nu_pore)
    lam = np.where(phase[0] == 1, ls, lp)
    mu = np.where(phase[0] == 1, ms, mp)
    M = lam + 2 * mu
    sxx = np.mean(lam / M) / np.mean(1.0 / M) * Eyy
    assert np.abs(strain[1] - Eyy).max() <= 1e-12 * Eyy
    assert np.abs(stress[0] - sxx).max() <= 1e-9 * abs(sxx)
    assert np.abs(strain[2]).max() <= 1e-12 * Eyy and np.abs(stress[2]).max() <= 1e-9 * abs(sxx)


# ---------------------------------------------------------------- phase field

def gpu_pf(phase, op, strain, Hin, h):
    ctx = fm.Context(phase.shape, MAT, fm.FFTMECH_FP64, h=h, tol=1e-13, max_iter=20000)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()
    H = dev(Hin)
    d = torch.zeros(phase.size, dtype=torch.float64, device="cuda")
    info = fm.fftmech_phasefield_operator(ctx.handle, torch.as_tensor(phase.ravel()).cuda(), dev(strain), None,
                                          OPS[op], H, d)
    ctx.close()
    return info, d.cpu().numpy().reshape(phase.shape), H.cpu().numpy().reshape(phase.shape)


@pytest.mark.parametrize("op", list(OPS))
@pytest.mark.parametrize("dim", [2, 3])
def test_phasefield_operator_matches_oracle(op, dim):
    """The phase field with every operator against the FP64 oracle
    (oracle/phasefield.phasefield_solve(symbol=)) for a given history field
    (zero strain leaves H unchanged); l0 = 2 voxels so that the gradient
    term weighs as much as the reaction."""
    from oracle import phasefield
    phase = random_carpet(81, 0.30, 18)[0] if dim == 2 else random_sponge(9, 0.35, 19)[0]
    nv = 3 if dim == 2 else 6
    h = MAT.l0 / 2
    a, _ = phasefield.coefficients(MAT)
    Hin = a * np.random.default_rng(20).random(phase.shape) * (phase == 1)
    info, d, Hout = gpu_pf(phase, op, np.zeros((nv,) + phase.shape), Hin, h)
    ref, _ = phasefield.phasefield_solve(Hin, MAT, h, tol=1e-13, symbol=op)
    e = rel(d, ref)
    print("phase field operator", op, dim, "iterations", info.iters, "d", e)
    assert info.status == fm.FFTMECH_OK
    assert np.array_equal(Hout, Hin) and e < 1e-10
    assert abs(info.total_damage - ref.sum()) <= 1e-10 * ref.sum()


def test_forward_phasefield_operator_agrees_with_the_library_solve():
    """History from a strain field and the phase field, forward operator:
    this spectral-operator path against the library's FP64
    fftmech_phasefield_solve (stencil PCG), two independent GPU paths."""
    phase = random_carpet(243, 0.30, 21)[0]
    N = phase.size
    h = MAT.l0 / 2
    ctx = fm.Context(phase.shape, MAT, fm.FFTMECH_FP64, h=h, tol=1e-13, max_iter=20000)
    ph = torch.as_tensor(phase.ravel()).cuda()
    u = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    strain = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    fm.fftmech_equilibrium_solve(ctx.handle, ph, None, None, [1e-2, 0.0, 0.0], u, strain, None)
    H1 = torch.zeros(N, dtype=torch.float64, device="cuda")
    d1 = torch.zeros(N, dtype=torch.float64, device="cuda")
    fm.fftmech_phasefield_solve(ctx.handle, strain, None, ph, H1, d1)
    ctx.close()
    _, d2, H2 = gpu_pf(phase, "forward", strain.cpu().numpy().reshape(3, *phase.shape), np.zeros(phase.shape), h)
    assert rel(H2, H1.cpu().numpy().reshape(phase.shape)) < 1e-14
    assert rel(d2, d1.cpu().numpy().reshape(phase.shape)) < 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_literal_phasefield_laplacian_by_gmres(dim):
    """The printed phase-field Laplacian read literally (sum_a D_a^2 with the
    forward difference: not symmetric), by the GPU's restarted GMRES,
    against the oracle's GMRES on the same equation; the symmetric Galerkin
    reading gives a different field. At h = 4 l0 every mode symbol of the
    literal operator has a positive real part (at the paper's h = l0 / 2 it
    does not, and neither GMRES converges: the reading of the oracle's
    phasefield module)."""
    from oracle import phasefield
    phase = random_carpet(81, 0.30, 22)[0] if dim == 2 else random_sponge(9, 0.35, 23)[0]
    nv = 3 if dim == 2 else 6
    h = 4 * MAT.l0
    a, _ = phasefield.coefficients(MAT)
    Hin = a * np.random.default_rng(24).random(phase.shape) * (phase == 1)
    ctx = fm.Context(phase.shape, MAT, fm.FFTMECH_FP64, h=h, tol=1e-12, max_iter=20000)
    dev = lambda x: torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64).ravel()).cuda()
    H = dev(Hin)
    d = torch.zeros(phase.size, dtype=torch.float64, device="cuda")
    info = fm.fftmech_phasefield_operator(ctx.handle, torch.as_tensor(phase.ravel()).cuda(),
                                          dev(np.zeros((nv,) + phase.shape)), None,
                                          fm.FFTMECH_GRAD_FORWARD | fm.FFTMECH_PF_LITERAL, H, d)
    ctx.close()
    got = d.cpu().numpy().reshape(phase.shape)
    ref, rinfo = phasefield.phasefield_solve(Hin, MAT, h, tol=1e-12, literal=True)
    gal, _ = phasefield.phasefield_solve(Hin, MAT, h, tol=1e-12)
    e = rel(got, ref)
    print("literal phase field", dim, "GMRES iterations", info.iters, "oracle", rinfo["iters"], "d", e,
          "vs Galerkin", rel(gal, ref))
    assert info.status == fm.FFTMECH_OK
    assert e < 1e-9 and rel(gal, ref) > 1e-3
