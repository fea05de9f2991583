"""Programmatic dependent launches (the default launch mode) against plain
stream order: every kernel waits on the device for its predecessor, so both
modes must give bit-identical fields and the same iteration counts. A
missing wait would show up here as a race (a field that differs between the
modes or from run to run)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from microstructures import random_carpet, random_sponge
from microstructures.workloads import Materials, left_face_mask
from paper_2305_13081_gb300 import build
from paper_2305_13081_gb300 import fftmech as fm

pytestmark = pytest.mark.gpu

H = 5e-6
MAT = Materials(E_pore=2e9, M_ppt=2.2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    fm.load_library()


def transient_state(phases, prec, dt):
    n = phases[0].size
    d = phases[0].ndim
    nv = 3 if d == 2 else 6
    B = len(phases)
    ft = torch.float64 if prec == fm.FFTMECH_FP64 else torch.float32
    spec = [("c", 1, torch.float64), ("c_ppt", 1, ft), ("eig", 1, ft), ("u", d, torch.float64),
            ("strain", nv, ft), ("stress", nv, ft), ("H", 1, ft), ("damage", 1, torch.float64)]
    bufs = {k: torch.zeros(m * n * B, dtype=t, device="cuda") for k, m, t in spec}
    bufs["phase"] = torch.as_tensor(np.concatenate([p.ravel() for p in phases])).cuda()
    bufs["mask"] = torch.as_tensor(np.concatenate([left_face_mask(p).ravel() for p in phases])).cuda()
    st = fm.fftmech_state()
    for k in ("phase", "c", "c_ppt", "eig", "u", "strain", "stress", "H", "damage"):
        setattr(st, k, bufs[k].data_ptr())
    p = fm.fftmech_step_params()
    p.diffusion_mode = fm.FFTMECH_DIFF_TRANSIENT
    p.dt = dt
    p.dirichlet_mask = bufs["mask"].data_ptr()
    p.dirichlet_value = 1.0
    p.eig_mode = fm.FFTMECH_EIG_FROM_PRECIPITATE
    return bufs, st, p


def run_steps(phases, prec, launch_mode, steps=2, tol=1e-8):
    shape = phases[0].shape
    n = shape[0]
    ctx = fm.Context(shape, MAT, prec, h=H, h_diff=1.0, tol=tol, batch=len(phases), launch_mode=launch_mode)
    bufs, st, p = transient_state(phases, prec, (n / 4.0) ** 2 / 10)
    iters = []
    for _ in range(steps):
        infos = fm.fftmech_staggered_step(ctx.handle, st, p)
        k = len(phases) * 3
        assert all(infos[i].status == fm.FFTMECH_OK for i in range(k))
        iters.append([infos[i].iters for i in range(k)])
    torch.cuda.synchronize()
    ctx.close()
    return {k: bufs[k].cpu().numpy() for k in ("c", "u", "strain", "stress", "damage")}, iters


@pytest.mark.parametrize("prec", [fm.FFTMECH_MIXED, fm.FFTMECH_FP64])
@pytest.mark.parametrize("n,seeds", [(81, (7, 8)), (243, (9,))])
def test_dependent_launches_bit_identical_2d(prec, n, seeds):
    phases = [random_carpet(n, 0.30, s)[0] for s in seeds]
    a, ia = run_steps(phases, prec, 0)
    b, ib = run_steps(phases, prec, 1)
    assert ia == ib
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert a["damage"].max() > 0


def test_dependent_launches_bit_identical_3d():
    phases = [np.ascontiguousarray(random_sponge(27, 0.35, s)[0]) for s in (3, 4)]
    a, ia = run_steps(phases, fm.FFTMECH_MIXED, 0, steps=1)
    b, ib = run_steps(phases, fm.FFTMECH_MIXED, 1, steps=1)
    assert ia == ib
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_dependent_launches_repeatable():
    """Two runs in the default mode agree bit for bit (deterministic
    reductions; no read of a buffer that a still-running kernel writes)."""
    phases = [random_carpet(81, 0.30, s)[0] for s in (11, 12, 13)]
    a, ia = run_steps(phases, fm.FFTMECH_MIXED, 0)
    b, ib = run_steps(phases, fm.FFTMECH_MIXED, 0)
    assert ia == ib
    for k in a:
        assert np.array_equal(a[k], b[k]), k
