"""The GPU adjoint of the staggered solve (fftmech_adjoint_eigenstrain) with
a prescribed, ramped pore eigenstrain: the gradient of the total elastic
energy and of the summed damage with respect to the per-voxel eigenstrain.

Checked through the C ABI:
- against the oracle's adjoint (itself pinned by central differences of the
  oracle's forward): FP64 path within 1e-8 relative L2, mixed path within
  1e-4, in 2D and 3D, with and without a tensile macro strain, over a load /
  unload / reload ramp (both branches of the history max);
- against central differences (step 1e-6) of the GPU's own FP64 forward at
  32 sampled voxels (28 pores, 4 solid) away from the kinks of the history
  max and the Macaulay bracket, within 1e-4 relative;
- the checkpoint interval changes nothing (bit for bit);
- torch.autograd through the EigenstrainObjective function gives the same
  gradient.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from microstructures import random_carpet, random_sponge
from microstructures.workloads import Materials
from oracle import adjoint
from paper_2305_13081_gb300 import build
from paper_2305_13081_gb300 import fftmech as fm

pytestmark = pytest.mark.gpu

H = 5e-6
MAT = Materials(E_pore=2e9)
RAMP = [1.0, 0.4, 0.9]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    fm.load_library()


def case(dim, n=None):
    if dim == 2:
        phase, _ = random_carpet(n or 27, 0.30, 5)
    else:
        phase, _ = random_sponge(n or 9, 0.3, 6)
    rng = np.random.default_rng(3)
    e = np.where(phase == 0, 2e-2 * (1.0 + 0.2 * rng.standard_normal(phase.shape)), 0.0)
    return phase, e


def macro(dim, tension):
    if not tension:
        return None
    return [3e-3, 0.0, 0.0] if dim == 2 else [3e-3, 0.0, 0.0, 0.0, 0.0, 0.0]


def gpu_grad(phase, e, prec, kind, E=None, k=2, tol=None):
    ctx = fm.Context(phase.shape, MAT, prec, h=H, tol=tol or (1e-13 if prec == fm.FFTMECH_FP64 else 1e-10),
                     max_iter=30000)
    ft = torch.float64 if prec == fm.FFTMECH_FP64 else torch.float32
    ph = torch.as_tensor(phase.ravel()).cuda()
    ef = torch.as_tensor(e.ravel()).to(ft).cuda()
    grad = torch.zeros(phase.size, dtype=torch.float64, device="cuda")
    obj = fm.FFTMECH_OBJ_ENERGY if kind == "energy" else fm.FFTMECH_OBJ_DAMAGE
    J, infos = fm.fftmech_adjoint_eigenstrain(ctx.handle, ph, ef, RAMP, E, obj, k, grad)
    ctx.close()
    return J, grad.cpu().numpy().reshape(phase.shape)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("prec", [fm.FFTMECH_FP64, fm.FFTMECH_MIXED])
@pytest.mark.parametrize("tension", [False, True])
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("kind", ["energy", "damage"])
def test_adjoint_matches_oracle_adjoint(kind, dim, tension, prec):
    phase, e = case(dim)
    E = macro(dim, tension)
    steps = adjoint.forward(phase, e, MAT, H, RAMP, tol=1e-13, eps_mac=E)
    ref = adjoint.gradient(phase, e, MAT, H, RAMP, kind, tol=1e-13, steps=steps, eps_mac=E)
    J_ref = adjoint.objective(steps, kind, H)
    J, g = gpu_grad(phase, e, prec, kind, E)
    err = rel(g, ref)
    print("adjoint", kind, dim, tension, prec, "J rel", abs(J - J_ref) / abs(J_ref), "grad rel", err)
    if prec == fm.FFTMECH_FP64:
        assert abs(J - J_ref) <= 1e-10 * abs(J_ref)
        assert err < 1e-8
    else:
        assert abs(J - J_ref) <= 1e-5 * abs(J_ref)
        assert err < 1e-4


def test_checkpoint_interval_changes_nothing():
    phase, e = case(2)
    _, g1 = gpu_grad(phase, e, fm.FFTMECH_FP64, "damage", k=1)
    _, g3 = gpu_grad(phase, e, fm.FFTMECH_FP64, "damage", k=3)
    assert np.array_equal(g1, g3)


@pytest.mark.parametrize("kind", ["energy", "damage"])
def test_adjoint_matches_central_differences_of_the_gpu_forward(kind):
    """81 x 81 carpet, FP64: central differences (step 1e-6) of J from the
    library's own forward steps at 32 sampled voxels (28 pores, 4 solid)
    away from the kinks: at every step the voxel's psi+ differs from H_prev
    and its elastic-strain trace from zero by at least 1 % of their field
    scales (the oracle's forward of the same case tells), far more than a
    1e-6 change of e moves them."""
    phase, e = case(2, 81)
    E = macro(2, True)
    J, g = gpu_grad(phase, e, fm.FFTMECH_FP64, kind, E)
    ctx = fm.Context(phase.shape, MAT, fm.FFTMECH_FP64, h=H, tol=1e-13, max_iter=30000)
    N = phase.size
    bufs = {k: torch.zeros(m * N, dtype=torch.float64, device="cuda") for k, m in
            [("c", 1), ("c_ppt", 1), ("eig", 1), ("u", 2), ("strain", 3), ("stress", 3), ("H", 1), ("damage", 1)]}
    bufs["phase"] = torch.as_tensor(phase.ravel()).cuda()
    st = fm.fftmech_state()
    for k, v in bufs.items():
        setattr(st, k, v.data_ptr())

    def forward(ev):
        for k in ("c", "u", "H", "damage"):
            bufs[k].zero_()
        ef = torch.as_tensor(ev.ravel()).cuda()
        p = fm.fftmech_step_params()
        p.diffusion_mode = fm.FFTMECH_DIFF_NONE
        p.eig_mode = fm.FFTMECH_EIG_PRESCRIBED
        p.eig_field = ef.data_ptr()
        p.eps_mac = fm.c_double6(*(E + [0, 0, 0]))
        for a in RAMP:
            p.eig_scale = a
            inf = fm.fftmech_staggered_step(ctx.handle, st, p)
        return inf[1].elastic_energy if kind == "energy" else inf[2].total_damage

    assert forward(e) == pytest.approx(J, rel=1e-12)
    rng = np.random.default_rng(17)
    ok = np.ones(phase.shape, dtype=bool)
    for st_ in adjoint.forward(phase, e, MAT, H, RAMP, tol=1e-13, eps_mac=E):
        el = st_["strain"][:2] - st_["e"]
        tr = el[0] + el[1]
        ok &= np.abs(st_["psi"] - st_["H_prev"]) > 1e-2 * np.abs(st_["psi"]).max()
        ok &= np.abs(tr) > 1e-2 * np.abs(tr).max()
    pores, solid = np.argwhere((phase == 0) & ok), np.argwhere((phase == 1) & ok)
    picks = [tuple(p) for p in pores[rng.choice(len(pores), 28, replace=False)]] + \
            [tuple(s) for s in solid[rng.choice(len(solid), 4, replace=False)]]
    scale = np.abs(g).max()
    for idx in picks:
        ep, em = e.copy(), e.copy()
        ep[idx] += 1e-6
        em[idx] -= 1e-6
        fd = (forward(ep) - forward(em)) / 2e-6
        print("fd", kind, idx, g[idx], fd)
        assert abs(g[idx] - fd) <= 1e-4 * max(abs(fd), 1e-3 * scale)
    ctx.close()


def test_autograd_function_gives_the_adjoint_gradient():
    from paper_2305_13081_gb300.autograd import eigenstrain_objective
    phase, e = case(2)
    ctx = fm.Context(phase.shape, MAT, fm.FFTMECH_FP64, h=H, tol=1e-13, max_iter=30000)
    ph = torch.as_tensor(phase.ravel()).cuda()
    ef = torch.as_tensor(e.ravel()).cuda().requires_grad_(True)
    J = eigenstrain_objective(ef, ctx, ph, RAMP, objective="damage", checkpoint_every=2)
    (g,) = torch.autograd.grad(2.0 * J, ef)
    ctx.close()
    _, ref = gpu_grad(phase, e, fm.FFTMECH_FP64, "damage")
    assert np.allclose(g.cpu().numpy().reshape(phase.shape), 2.0 * ref, rtol=1e-12, atol=0)
