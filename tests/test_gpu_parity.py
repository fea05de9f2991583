"""CUDA path against the FP64 CPU oracle, element by element, through the
C ABI: equilibrium (Sec. 2.3), homogenised and transient diffusion
(Sec. 2.1), history + phase field (Sec. 2.4) and the staggered step
(Algorithm 1), in FP64 and in the mixed path.

Tolerances: FP64 GPU path within 1e-10 relative L2 of the oracle (both
solved to a 1e-12 relative residual); mixed path (float fields, FP64
iterates and dot products) within 1e-5 relative L2 on strain and stress,
1e-6 relative on concentration and 1e-4 max-abs on damage.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from microstructures import random_carpet, sierpinski_carpet, porosity
from microstructures.workloads import Materials, left_face_mask
from oracle import elasticity, diffusion, phasefield, chemistry, staggered, spectral
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


def case(shape, seed, eig_mean=1e-3):
    n = max(shape)
    base = 2 if n & (n - 1) == 0 else 3  # 2x2 carpets for powers of two
    phase, _ = random_carpet(n, 0.30, seed, base=base)
    phase = np.ascontiguousarray(phase[:shape[0], :shape[1]])
    rng = np.random.default_rng(seed)
    eig = np.where(phase == 0, eig_mean * (1 + 0.2 * rng.standard_normal(shape)), 0.0)
    dmg = np.clip(0.6 * rng.random(shape) ** 3, 0, 1)
    return phase, eig, dmg


def gpu_equilibrium(phase, eig, dmg, E, prec, tol, mat=MAT, host=False, replace_residual=1):
    shape = phase.shape
    N = phase.size
    ctx = fm.Context(shape, mat, prec, h=H, tol=tol, max_iter=50000, replace_residual=replace_residual)
    ft = ftype(prec)
    if host:
        npt = np.float64 if prec == fm.FFTMECH_FP64 else np.float32
        u = np.zeros(2 * N)
        strain = np.zeros(3 * N, dtype=npt)
        stress = np.zeros(3 * N, dtype=npt)
        info = fm.fftmech_equilibrium_solve(ctx.handle, np.ascontiguousarray(phase, np.uint8),
                                            eig.astype(npt).ravel(),
                                            None if dmg is None else dmg.ravel().copy(), E, u,
                                            strain, stress)
        out = strain.reshape((3,) + shape).astype(np.float64), stress.reshape((3,) + shape).astype(np.float64), info
    else:
        u = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
        strain = torch.zeros(3 * N, dtype=ft, device="cuda")
        stress = torch.zeros(3 * N, dtype=ft, device="cuda")
        info = fm.fftmech_equilibrium_solve(ctx.handle, dev(phase, torch.uint8), dev(eig, ft),
                                            None if dmg is None else dev(dmg, torch.float64), E, u,
                                            strain, stress)
        torch.cuda.synchronize()
        out = (strain.double().cpu().numpy().reshape((3,) + shape),
               stress.double().cpu().numpy().reshape((3,) + shape), info)
    ctx.close()
    return out


# ---------------------------------------------------------------- equilibrium

@pytest.mark.parametrize("shape", [(27, 27), (81, 81), (729, 27), (81, 243)])
def test_equilibrium_fp64_matches_oracle(shape):
    phase, eig, dmg = case(shape, 11)
    g = phasefield.degradation(dmg, MAT.kappa)
    E = [2e-4, -1e-4, 5e-5]
    ref = elasticity.equilibrium_solve(phase, eig, g, E, MAT, H, tol=1e-12)
    strain, stress, info = gpu_equilibrium(phase, eig, dmg, E, fm.FFTMECH_FP64, 1e-12)
    assert info.status == fm.FFTMECH_OK
    assert rel(strain, ref["strain"]) < 1e-10
    assert rel(stress, ref["stress"]) < 1e-10
    assert np.allclose(info.mean_stress[:3], ref["mean_stress"], rtol=1e-9, atol=1e-9 * np.abs(ref["mean_stress"]).max())
    assert np.allclose(info.mean_strain[:3], E, atol=1e-15)
    en = elasticity.elastic_energy(ref["strain"], ref["stress"], eig, H)
    assert info.elastic_energy == pytest.approx(en, rel=1e-9)


@pytest.mark.parametrize("shape", [(81, 81), (729, 27), (128, 256), (81, 729)])
def test_equilibrium_mixed_matches_oracle(shape):
    phase, eig, dmg = case(shape, 12)
    g = phasefield.degradation(dmg, MAT.kappa)
    E = [0.0, 0.0, 0.0]
    ref = elasticity.equilibrium_solve(phase, eig, g, E, MAT, H, tol=1e-12)
    strain, stress, info = gpu_equilibrium(phase, eig, dmg, E, fm.FFTMECH_MIXED, 1e-8)
    assert info.status == fm.FFTMECH_OK
    assert rel(strain, ref["strain"]) < 1e-5
    assert rel(stress, ref["stress"]) < 1e-5
    assert info.true_rel_res < 1e-6


def test_equilibrium_host_buffers_match_device_buffers():
    phase, eig, dmg = case((81, 81), 13)
    E = [1e-4, 0, 0]
    a = gpu_equilibrium(phase, eig, dmg, E, fm.FFTMECH_FP64, 1e-10)
    b = gpu_equilibrium(phase, eig, dmg, E, fm.FFTMECH_FP64, 1e-10, host=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[2].iters == b[2].iters


def test_equilibrium_zero_rhs_and_homogeneous():
    phase = np.ones((27, 27), dtype=np.uint8)
    strain, stress, info = gpu_equilibrium(phase, np.zeros((27, 27)), None, [1e-3, 0, 0],
                                           fm.FFTMECH_FP64, 1e-12)
    assert info.iters == 0 and info.status == fm.FFTMECH_OK
    assert np.allclose(strain[0], 1e-3, rtol=1e-14) and np.allclose(strain[1:], 0, atol=1e-18)


def test_equilibrium_iteration_cap_and_nonfinite():
    phase, eig, _ = case((81, 81), 14)
    ctx = fm.Context(phase.shape, MAT, fm.FFTMECH_FP64, h=H, tol=1e-12, max_iter=5)
    N = phase.size
    u = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    info = fm.fftmech_equilibrium_solve(ctx.handle, dev(phase, torch.uint8), dev(eig, torch.float64),
                                        None, [0, 0, 0], u, None, None)
    assert info.status == fm.FFTMECH_ERR_NOT_CONVERGED and info.iters == 5
    bad = eig.copy()
    bad[3, 4] = np.nan
    u.zero_()
    info = fm.fftmech_equilibrium_solve(ctx.handle, dev(phase, torch.uint8), dev(bad, torch.float64),
                                        None, [0, 0, 0], u, None, None)
    assert info.status == fm.FFTMECH_ERR_NONFINITE
    ctx.close()


# ---------------------------------------------------------------- diffusion

@pytest.mark.parametrize("prec,tol", [(fm.FFTMECH_FP64, 1e-11), (fm.FFTMECH_MIXED, 1e-6)])
@pytest.mark.parametrize("shape", [(81, 81), (243, 27)])
def test_homogenise_matches_oracle(prec, tol, shape):
    phase, _, _ = case(shape, 21)
    gm, cX = (1.0, 0.25), 1.0
    ref = diffusion.homogenise(phase, MAT, gm, cX, 1.0, tol=1e-13)
    ctx = fm.Context(shape, MAT, prec, h=H, h_diff=1.0, tol=1e-12 if prec == fm.FFTMECH_FP64 else 1e-9)
    c = torch.zeros(phase.size, dtype=torch.float64, device="cuda")
    info = fm.fftmech_diffusion_step(ctx.handle, dev(phase, torch.uint8), fm.FFTMECH_DIFF_HOMOGENISE,
                                     gm, cX, 0.0, None, 0.0, c)
    ctx.close()
    got = c.cpu().numpy().reshape(shape)
    assert info.status == fm.FFTMECH_OK
    assert rel(got, ref["c"]) < tol
    assert np.allclose(info.mean_flux[:2], ref["mean_flux"], rtol=10 * tol, atol=10 * tol * np.abs(ref["mean_flux"]).max())
    assert info.porosity == pytest.approx(porosity(phase), abs=1e-15)


@pytest.mark.parametrize("prec,tol", [(fm.FFTMECH_FP64, 1e-11), (fm.FFTMECH_MIXED, 1e-6)])
def test_transient_matches_oracle(prec, tol):
    shape = (81, 81)
    phase, _, _ = case(shape, 22)
    mask = left_face_mask(phase)
    dt = (81 / 4.0) ** 2 / 20
    c_ref = np.zeros(shape)
    ctx = fm.Context(shape, MAT, prec, h=H, h_diff=1.0, tol=1e-12 if prec == fm.FFTMECH_FP64 else 1e-10)
    c = torch.zeros(phase.size, dtype=torch.float64, device="cuda")
    dmask = dev(mask, torch.uint8)
    for _ in range(3):
        c_ref = diffusion.transient_step(phase, c_ref, MAT, dt, 1.0, mask, 1.0)
        info = fm.fftmech_diffusion_step(ctx.handle, dev(phase, torch.uint8), fm.FFTMECH_DIFF_TRANSIENT,
                                         (0, 0, 0), 0.0, dt, dmask, 1.0, c)
        assert info.status == fm.FFTMECH_OK
    ctx.close()
    got = c.cpu().numpy().reshape(shape)
    assert rel(got, c_ref) < tol
    assert got.min() >= -tol and got.max() <= 1 + tol  # discrete maximum principle


# ---------------------------------------------------------------- phase field

@pytest.mark.parametrize("prec", [fm.FFTMECH_FP64, fm.FFTMECH_MIXED])
def test_phasefield_matches_oracle(prec):
    shape = (81, 81)
    phase, eig, _ = case(shape, 31, eig_mean=3e-2)
    mat = Materials(E_pore=2e9)
    ref_eq = elasticity.equilibrium_solve(phase, eig, np.ones(shape), [2e-3, 0, 0], mat, H, tol=1e-12)
    lam, mu = elasticity.phase_lame(phase, mat)
    rng = np.random.default_rng(3)
    H0 = 5e4 * rng.random(shape)
    psi = elasticity.psi_plus(ref_eq["strain"], eig, lam, mu)
    H1 = phasefield.history_update(H0, psi)
    d_ref, _ = phasefield.phasefield_solve(H1, mat, H, tol=1e-13)
    ctx = fm.Context(shape, mat, prec, h=H, tol=1e-12 if prec == fm.FFTMECH_FP64 else 1e-8)
    ft = ftype(prec)
    Hd = dev(H0, ft)
    d = torch.zeros(phase.size, dtype=torch.float64, device="cuda")
    info = fm.fftmech_phasefield_solve(ctx.handle, dev(ref_eq["strain"], ft), dev(eig, ft),
                                       dev(phase, torch.uint8), Hd, d)
    ctx.close()
    assert info.status == fm.FFTMECH_OK
    got_H = Hd.double().cpu().numpy().reshape(shape)
    got_d = d.cpu().numpy().reshape(shape)
    if prec == fm.FFTMECH_FP64:
        assert rel(got_H, H1) < 1e-12
        assert rel(got_d, d_ref) < 1e-10
    else:
        assert rel(got_H, H1) < 1e-6
        assert np.abs(got_d - d_ref).max() < 1e-4
    assert d_ref.max() > 1e-3  # the case exercises real damage
    assert info.total_damage == pytest.approx(got_d.sum(), rel=1e-12)


# ---------------------------------------------------------------- staggered step

def run_gpu_staggered(phase, prec, steps, params, eig_field=None, c0=None, tol=1e-12, mat=MAT):
    shape = phase.shape
    N = phase.size
    ft = ftype(prec)
    ctx = fm.Context(shape, mat, prec, h=H, h_diff=1.0, tol=tol)
    keep = []

    def t(x, dtype):
        v = dev(x, dtype)
        keep.append(v)
        return v

    st = fm.fftmech_state()
    bufs = {
        "phase": t(phase, torch.uint8),
        "c": t(np.zeros(N) if c0 is None else c0.ravel(), torch.float64),
        "c_ppt": torch.zeros(N, dtype=ft, device="cuda"),
        "eig": torch.zeros(N, dtype=ft, device="cuda"),
        "u": torch.zeros(2 * N, dtype=torch.float64, device="cuda"),
        "strain": torch.zeros(3 * N, dtype=ft, device="cuda"),
        "stress": torch.zeros(3 * N, dtype=ft, device="cuda"),
        "H": torch.zeros(N, dtype=ft, device="cuda"),
        "damage": torch.zeros(N, dtype=torch.float64, device="cuda"),
    }
    for k, v in bufs.items():
        setattr(st, k, v.data_ptr())
    if eig_field is not None:
        params.eig_field = t(eig_field, ft).data_ptr()
    infos = []
    for _ in range(steps):
        infos.append([i.as_dict() for i in fm.fftmech_staggered_step(ctx.handle, st, params)])
    torch.cuda.synchronize()
    out = {k: v.double().cpu().numpy() for k, v in bufs.items()}
    ctx.close()
    return out, infos


@pytest.mark.parametrize("prec", [fm.FFTMECH_FP64, fm.FFTMECH_MIXED])
def test_staggered_sierpinski_homogenise(prec):
    """Sierpinski 81^2 with prescribed pore eigenstrain (stiff pores so that
    damage develops) and homogenised diffusion, 2 steps, against the oracle."""
    phase = sierpinski_carpet(4)
    mat = Materials(E_pore=2e9)
    eig = np.where(phase == 0, 2e-2, 0.0)
    steps = 2
    ref = staggered.initial_state(phase)
    for s in range(steps):
        ref, _ = staggered.step(ref, phase, mat, H, 1.0, staggered.DIFF_HOMOGENISE, staggered.EIG_PRESCRIBED,
                                eig_field=eig, eig_scale=1.0 + s, grad_c_mac=(1.0, 0.0), c_macro=1.0,
                                eps_mac=(1e-3, 0, 0), tol=1e-12)
    p = fm.fftmech_step_params()
    p.diffusion_mode = fm.FFTMECH_DIFF_HOMOGENISE
    p.grad_c_mac = fm.c_double3(1.0, 0.0, 0.0)
    p.c_macro = 1.0
    p.eig_mode = fm.FFTMECH_EIG_PRESCRIBED
    p.eps_mac = fm.c_double6(1e-3, 0, 0, 0, 0, 0)
    # eig_scale ramps 1, 2: run step by step
    out = None
    shape = phase.shape
    N = phase.size
    ft = ftype(prec)
    ctx = fm.Context(shape, mat, prec, h=H, h_diff=1.0, tol=1e-12 if prec == fm.FFTMECH_FP64 else 1e-9)
    bufs = {k: torch.zeros(n * N, dtype=dt, device="cuda") for k, n, dt in
            [("c", 1, torch.float64), ("c_ppt", 1, ft), ("eig", 1, ft), ("u", 2, torch.float64),
             ("strain", 3, ft), ("stress", 3, ft), ("H", 1, ft), ("damage", 1, torch.float64)]}
    bufs["phase"] = dev(phase, torch.uint8)
    st = fm.fftmech_state()
    for k, v in bufs.items():
        setattr(st, k, v.data_ptr())
    ef = dev(eig, ft)
    p.eig_field = ef.data_ptr()
    for s in range(steps):
        p.eig_scale = 1.0 + s
        infos = fm.fftmech_staggered_step(ctx.handle, st, p)
        assert all(i.status == fm.FFTMECH_OK for i in infos)
    torch.cuda.synchronize()
    out = {k: v.double().cpu().numpy() for k, v in bufs.items()}
    ctx.close()
    d_ref = ref["d"]
    assert d_ref.max() > 1e-3
    if prec == fm.FFTMECH_FP64:
        assert rel(out["c"].reshape(shape), ref["c"]) < 1e-10
        assert rel(out["strain"].reshape((3,) + shape), ref["strain"]) < 1e-10
        assert rel(out["stress"].reshape((3,) + shape), ref["stress"]) < 1e-10
        assert rel(out["H"].reshape(shape), ref["H"]) < 1e-10
        assert rel(out["damage"].reshape(shape), d_ref) < 1e-10
    else:
        assert rel(out["c"].reshape(shape), ref["c"]) < 1e-6
        assert rel(out["strain"].reshape((3,) + shape), ref["strain"]) < 1e-5
        assert rel(out["stress"].reshape((3,) + shape), ref["stress"]) < 1e-5
        assert np.abs(out["damage"].reshape(shape) - d_ref).max() < 1e-4


@pytest.mark.parametrize("prec", [fm.FFTMECH_FP64, fm.FFTMECH_MIXED])
def test_staggered_transient_precipitation(prec):
    """Random carpet 81^2, left-face source, transient diffusion ->
    precipitate eigenstrain -> equilibrium -> phase field, 3 steps."""
    shape = (81, 81)
    phase, _ = random_carpet(81, 0.30, 2305)
    mat = Materials(E_pore=2e9, M_ppt=2.2)
    mask = left_face_mask(phase)
    dt = (81 / 4.0) ** 2 / 10
    ref = staggered.initial_state(phase)
    for _ in range(3):
        ref, _ = staggered.step(ref, phase, mat, H, 1.0, staggered.DIFF_TRANSIENT,
                                staggered.EIG_FROM_PRECIPITATE, dt=dt, mask=mask, c_dirichlet=1.0,
                                tol=1e-12)
    p = fm.fftmech_step_params()
    p.diffusion_mode = fm.FFTMECH_DIFF_TRANSIENT
    p.dt = dt
    dmask = dev(mask, torch.uint8)
    p.dirichlet_mask = dmask.data_ptr()
    p.dirichlet_value = 1.0
    p.eig_mode = fm.FFTMECH_EIG_FROM_PRECIPITATE
    out, infos = run_gpu_staggered(phase, prec, 3, p, tol=1e-12 if prec == fm.FFTMECH_FP64 else 1e-10, mat=mat)
    assert ref["eig"].max() > 0
    c = out["c"].reshape(shape)
    errs = {"c": rel(c, ref["c"]), "eig": rel(out["eig"].reshape(shape), ref["eig"]),
            "strain": rel(out["strain"].reshape((3,) + shape), ref["strain"]),
            "stress": rel(out["stress"].reshape((3,) + shape), ref["stress"]),
            "damage": rel(out["damage"].reshape(shape), ref["d"])}
    print("staggered transient", prec, errs)
    if prec == fm.FFTMECH_FP64:
        assert max(errs.values()) < 1e-10
    else:
        assert rel(c, ref["c"]) < 1e-6
        assert errs["strain"] < 1e-5 and errs["stress"] < 1e-5
        assert np.abs(out["damage"].reshape(shape) - ref["d"]).max() < 1e-4
    c_ppt = np.where(phase == 0, np.maximum(c - mat.S_sol, 0), 0)
    assert np.allclose(out["c_ppt"].reshape(shape), c_ppt, atol=1e-6 if prec else 1e-14)


# ---------------------------------------------------------------- full size

@pytest.mark.slow
def test_full_size_carpet_729_equilibrium_residual_by_oracle():
    """729^2 random carpet (the benchmark geometry): the oracle's own
    projection GG (App. A) applied to the GPU stress must vanish to the
    solver tolerance, and mixed must match FP64 within 1e-5."""
    phase, _ = random_carpet(729, 0.30, 2305)
    eig = np.where(phase == 0, 1e-3, 0.0)
    s64, t64, i64 = gpu_equilibrium(phase, eig, None, [0, 0, 0], fm.FFTMECH_FP64, 1e-8)
    s32, t32, i32 = gpu_equilibrium(phase, eig, None, [0, 0, 0], fm.FFTMECH_MIXED, 1e-8)
    assert i64.status == fm.FFTMECH_OK and i32.status == fm.FFTMECH_OK
    assert rel(s32, s64) < 1e-5 and rel(t32, t64) < 1e-5
    D = spectral.forward_difference_symbol(phase.shape, H)
    ghat = spectral.projection_operator(D)

    def tensor(v):
        return np.stack([np.stack([v[0], v[2]]), np.stack([v[2], v[1]])])

    lam, mu = elasticity.phase_lame(phase, MAT)
    sig0 = elasticity.stress(np.zeros((2, 2) + phase.shape), eig, np.ones(phase.shape), lam, mu)
    b0 = np.linalg.norm(spectral.apply_GG(ghat, sig0))
    for t in (t64, t32):
        r = np.linalg.norm(spectral.apply_GG(ghat, tensor(t)))
        assert r / b0 < (3e-8 if t is t64 else 1e-5)
    assert abs(i64.iters - i32.iters) <= max(3, 0.02 * i64.iters)
