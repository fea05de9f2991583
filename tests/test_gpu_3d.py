"""3D path (Menger-type sponges and non-cubic random grids) against the FP64
CPU oracle through the C ABI: equilibrium with six strain components
(Sec. 2.3), homogenised and transient diffusion (Sec. 2.1), history and
phase field in d = 3 (Sec. 2.4), the staggered step with a ramped pore
eigenstrain (Algorithm 1), and uniform 3D batches.

Tolerances as in the 2D parity tests: FP64 within 1e-10 relative L2 of the
oracle (both at a 1e-12 relative residual); mixed within 1e-5 relative L2
on strain and stress, 1e-6 relative on concentration, 1e-4 max-abs on
damage. The non-cubic grid (12, 18, 24) has an even nx (the half-spectrum
column kx = nx/2 counts once) and radix-2 passes along every axis; the
(9, 9, 243) and (243, 9, 9) grids put a 243-point axis (compile-time
transform plans in the mixed path) along x and along z.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from microstructures import random_sponge
from microstructures.workloads import Materials, left_face_mask
from oracle import elasticity, diffusion, phasefield, staggered
from paper_2305_13081_gb300 import build
from paper_2305_13081_gb300 import fftmech as fm

pytestmark = pytest.mark.gpu

H = 5e-6
MAT = Materials()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    fm.load_library()


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def dev(x, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().contiguous()


def ftype(prec):
    return torch.float64 if prec == fm.FFTMECH_FP64 else torch.float32


def blob_phase(shape, seed, porosity=0.35):
    """Smooth random pores on any grid: threshold a periodic low-pass field."""
    rng = np.random.default_rng(seed)
    f = np.fft.fftn(rng.standard_normal(shape))
    k = np.meshgrid(*[np.fft.fftfreq(n) * n for n in shape], indexing="ij")
    f *= np.exp(-sum(kk ** 2 for kk in k) / 8.0)
    x = np.fft.ifftn(f).real
    return (x > np.quantile(x, porosity)).astype(np.uint8)


def case3(shape, seed):
    if len(set(shape)) == 1:
        phase, _ = random_sponge(shape[0], 0.35, seed)
    else:
        phase = blob_phase(shape, seed)
    rng = np.random.default_rng(seed)
    eig = np.where(phase == 0, 1e-3 * (1 + 0.2 * rng.standard_normal(shape)), 0.0)
    dmg = np.clip(0.6 * rng.random(shape) ** 3, 0, 1)
    return np.ascontiguousarray(phase), eig, dmg


def gpu_equilibrium3(phase, eig, dmg, E, prec, tol, batch_of=None):
    shape = phase.shape
    N = phase.size
    ctx = fm.Context(shape, MAT, prec, h=H, tol=tol, max_iter=50000)
    ft = ftype(prec)
    u = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    strain = torch.zeros(6 * N, dtype=ft, device="cuda")
    stress = torch.zeros(6 * N, dtype=ft, device="cuda")
    info = fm.fftmech_equilibrium_solve(ctx.handle, dev(phase, torch.uint8), dev(eig, ft),
                                        dev(dmg, torch.float64), E, u, strain, stress)
    torch.cuda.synchronize()
    ctx.close()
    return (strain.double().cpu().numpy().reshape((6,) + shape),
            stress.double().cpu().numpy().reshape((6,) + shape), info)


@pytest.mark.parametrize("shape", [(27, 27, 27), (12, 18, 24)])
def test_equilibrium3d_fp64_matches_oracle(shape):
    phase, eig, dmg = case3(shape, 21)
    g = phasefield.degradation(dmg, MAT.kappa)
    E = [2e-4, -1e-4, 5e-5, 3e-5, -2e-5, 1e-5]
    ref = elasticity.equilibrium_solve(phase, eig, g, E, MAT, H, tol=1e-12)
    strain, stress, info = gpu_equilibrium3(phase, eig, dmg, E, fm.FFTMECH_FP64, 1e-12)
    assert info.status == fm.FFTMECH_OK
    assert rel(strain, ref["strain"]) < 1e-10
    assert rel(stress, ref["stress"]) < 1e-10
    ms = np.array(info.mean_stress[:6])
    assert np.allclose(ms, ref["mean_stress"], rtol=1e-9, atol=1e-9 * np.abs(ref["mean_stress"]).max())
    assert np.allclose(info.mean_strain[:6], E, atol=1e-15)
    en = elasticity.elastic_energy(ref["strain"], ref["stress"], eig, H)
    assert info.elastic_energy == pytest.approx(en, rel=1e-9)


@pytest.mark.parametrize("shape", [(27, 27, 27), (12, 18, 24), (9, 9, 243), (243, 9, 9)])
def test_equilibrium3d_mixed_matches_oracle(shape):
    phase, eig, dmg = case3(shape, 22)
    g = phasefield.degradation(dmg, MAT.kappa)
    E = [0.0] * 6
    ref = elasticity.equilibrium_solve(phase, eig, g, E, MAT, H, tol=1e-12)
    strain, stress, info = gpu_equilibrium3(phase, eig, dmg, E, fm.FFTMECH_MIXED, 1e-8)
    assert info.status == fm.FFTMECH_OK
    assert rel(strain, ref["strain"]) < 1e-5
    assert rel(stress, ref["stress"]) < 1e-5
    assert info.true_rel_res < 1e-6


def test_equilibrium3d_homogeneous_one_iteration():
    """A homogeneous medium under a macro strain: the preconditioned
    residual is zero, so the solve takes no iteration and the strain is E."""
    shape = (9, 27, 18)
    phase = np.ones(shape, np.uint8)
    E = [1e-4, 2e-4, -3e-4, 0, 1e-5, 0]
    strain, stress, info = gpu_equilibrium3(phase, np.zeros(shape), np.zeros(shape), E, fm.FFTMECH_FP64, 1e-12)
    assert info.status == fm.FFTMECH_OK and info.iters == 0
    for k in range(6):
        assert np.allclose(strain[k], E[k], atol=1e-18)


@pytest.mark.parametrize("prec", [fm.FFTMECH_FP64, fm.FFTMECH_MIXED])
def test_diffusion3d_homogenise_matches_oracle(prec):
    shape = (12, 18, 24)
    phase = blob_phase(shape, 5)
    gmac = (1.0, -0.5, 0.25)
    ref = diffusion.homogenise(phase, MAT, gmac, 0.7, 1.0, tol=1e-12)
    ctx = fm.Context(shape, MAT, prec, h=H, h_diff=1.0, tol=1e-12 if prec == fm.FFTMECH_FP64 else 1e-9)
    c = torch.zeros(phase.size, dtype=torch.float64, device="cuda")
    info = fm.fftmech_diffusion_step(ctx.handle, dev(phase, torch.uint8), fm.FFTMECH_DIFF_HOMOGENISE, gmac, 0.7,
                                     0.0, None, 0.0, c)
    torch.cuda.synchronize()
    ctx.close()
    assert info.status == fm.FFTMECH_OK
    got = c.cpu().numpy().reshape(shape)
    tol = 1e-10 if prec == fm.FFTMECH_FP64 else 1e-6
    assert rel(got, ref["c"]) < tol
    assert np.allclose(info.mean_flux[:3], ref["mean_flux"], rtol=1e-8 if prec == fm.FFTMECH_FP64 else 1e-5,
                       atol=1e-12)
    assert info.porosity == pytest.approx(float((phase == 0).mean()), rel=1e-12)


@pytest.mark.parametrize("prec", [fm.FFTMECH_FP64, fm.FFTMECH_MIXED])
def test_diffusion3d_transient_matches_oracle(prec):
    shape = (18, 12, 24)
    phase = blob_phase(shape, 6)
    mask = left_face_mask(phase)
    dt = 4.0
    c0 = np.zeros(shape)
    ref = diffusion.transient_step(phase, c0, MAT, dt, 1.0, mask=mask, c_dirichlet=1.0)
    ctx = fm.Context(shape, MAT, prec, h=H, h_diff=1.0, tol=1e-12 if prec == fm.FFTMECH_FP64 else 1e-9)
    c = torch.zeros(phase.size, dtype=torch.float64, device="cuda")
    info = fm.fftmech_diffusion_step(ctx.handle, dev(phase, torch.uint8), fm.FFTMECH_DIFF_TRANSIENT, (0.0, 0.0, 0.0), 0.0, dt,
                                     dev(mask, torch.uint8), 1.0, c)
    torch.cuda.synchronize()
    ctx.close()
    assert info.status == fm.FFTMECH_OK
    got = c.cpu().numpy().reshape(shape)
    assert rel(got, ref) < (1e-10 if prec == fm.FFTMECH_FP64 else 1e-6)
    slack = 1e-9 if prec == fm.FFTMECH_FP64 else 1e-6
    assert got.max() <= 1.0 + slack and got.min() >= -slack  # discrete maximum principle


@pytest.mark.parametrize("prec", [fm.FFTMECH_FP64, fm.FFTMECH_MIXED])
def test_staggered3d_sponge_ramp_matches_oracle(prec):
    """27^3 sponge, prescribed pore eigenstrain ramped over two steps, no
    diffusion: equilibrium -> history -> phase field in d = 3."""
    phase, _ = random_sponge(27, 0.35, 7)
    mat = Materials(E_pore=2e9)
    eig = np.where(phase == 0, 1.0, 0.0)
    scales = [1e-2, 2e-2]
    ref = staggered.initial_state(phase)
    for s in scales:
        ref, _ = staggered.step(ref, phase, mat, H, 1.0, staggered.DIFF_NONE, staggered.EIG_PRESCRIBED,
                                eig_field=eig, eig_scale=s, eps_mac=(0, 0, 0, 0, 0, 0), tol=1e-12)
    N = phase.size
    ft = ftype(prec)
    ctx = fm.Context(phase.shape, mat, prec, h=H, h_diff=1.0, tol=1e-12 if prec == fm.FFTMECH_FP64 else 1e-9)
    bufs = {k: torch.zeros(n * N, dtype=dt, device="cuda") for k, n, dt in
            [("c", 1, torch.float64), ("c_ppt", 1, ft), ("eig", 1, ft), ("u", 3, torch.float64),
             ("strain", 6, ft), ("stress", 6, ft), ("H", 1, ft), ("damage", 1, torch.float64)]}
    bufs["phase"] = dev(phase, torch.uint8)
    st = fm.fftmech_state()
    for k, v in bufs.items():
        setattr(st, k, v.data_ptr())
    p = fm.fftmech_step_params()
    p.diffusion_mode = fm.FFTMECH_DIFF_NONE
    p.eig_mode = fm.FFTMECH_EIG_PRESCRIBED
    ef = dev(eig, ft)
    p.eig_field = ef.data_ptr()
    for s in scales:
        p.eig_scale = s
        infos = fm.fftmech_staggered_step(ctx.handle, st, p)
        assert infos[1].status == fm.FFTMECH_OK and infos[2].status == fm.FFTMECH_OK
    torch.cuda.synchronize()
    out = {k: v.double().cpu().numpy() for k, v in bufs.items()}
    ctx.close()
    shape = phase.shape
    assert ref["d"].max() > 1e-3
    if prec == fm.FFTMECH_FP64:
        assert rel(out["strain"].reshape((6,) + shape), ref["strain"]) < 1e-10
        assert rel(out["H"].reshape(shape), ref["H"]) < 1e-10
        assert rel(out["damage"].reshape(shape), ref["d"]) < 1e-10
    else:
        assert rel(out["strain"].reshape((6,) + shape), ref["strain"]) < 1e-5
        assert rel(out["stress"].reshape((6,) + shape), ref["stress"]) < 1e-5
        assert np.abs(out["damage"].reshape(shape) - ref["d"]).max() < 1e-4


def test_batched3d_equals_single_solves():
    shape = (12, 18, 24)
    probs = [case3(shape, s) for s in (31, 32)]
    N = probs[0][0].size
    E = [1e-4, 0, 0, 0, 0, 2e-5]
    single = [gpu_equilibrium3(ph, e, d, E, fm.FFTMECH_FP64, 1e-11) for ph, e, d in probs]
    ctx = fm.Context(shape, MAT, fm.FFTMECH_FP64, h=H, tol=1e-11, max_iter=50000, batch=2)
    u = torch.zeros(2 * 3 * N, dtype=torch.float64, device="cuda")
    strain = torch.zeros(2 * 6 * N, dtype=torch.float64, device="cuda")
    infos = fm.fftmech_equilibrium_solve(ctx.handle, dev(np.concatenate([p[0].ravel() for p in probs]), torch.uint8),
                                         dev(np.concatenate([p[1].ravel() for p in probs]), torch.float64),
                                         dev(np.concatenate([p[2].ravel() for p in probs]), torch.float64), E, u,
                                         strain, None)
    torch.cuda.synchronize()
    ctx.close()
    got = strain.cpu().numpy().reshape(2, 6, *shape)
    for b in range(2):
        assert infos[b].status == fm.FFTMECH_OK
        assert infos[b].iters == single[b][2].iters
        assert np.array_equal(got[b], single[b][0])
