"""The transient carpet workload at full size (729 x 729 random carpet, seed
2305, left-face source, precipitate eigenstrain; Algorithm 1) against the
FP64 CPU oracle's first three staggered steps, stored in
tests/golden/carpet729_steps1to3.npz by tests/golden/make_carpet729_golden.py
(which calls only the oracle): per step and field, the values at 4096 fixed
voxels and the sum and L2 norm of every component over all voxels.

FP64 GPU path (solved to 1e-13; the oracle to 1e-12): sampled values within
1e-10 relative L2; norms within 1e-10 relative, sums within 1e-10 of
sqrt(N) times the norm (the strain's sum is the macro strain times N, zero
here, so it has no scale of its own). Mixed path at the
workload's tolerance 1e-8: strain and stress within 1e-5, concentration
within 1e-6 (relative L2 over the samples), damage within 1e-4 max-abs.
"""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from microstructures.workloads import carpet_transient
from paper_2305_13081_gb300 import build
from paper_2305_13081_gb300 import fftmech as fm

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "carpet729_steps1to3.npz")
FIELDS = {"c": ("c", 1), "c_ppt": ("c_ppt", 1), "eig": ("eig", 1), "strain": ("strain", 3),
          "stress": ("stress", 3), "H": ("H", 1), "d": ("damage", 1)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    fm.load_library()


def rel(a, b):
    nb = np.linalg.norm(np.ravel(b))
    return float(np.linalg.norm(np.ravel(a - b)) / nb) if nb > 0 else float(np.linalg.norm(np.ravel(a)))


def run(prec, tol, steps):
    w = carpet_transient(729)
    N = w.phase.size
    ft = torch.float64 if prec == fm.FFTMECH_FP64 else torch.float32
    ctx = fm.Context(w.phase.shape, w.materials, prec, h=w.h, h_diff=w.h_diff, tol=tol, max_iter=30000)
    bufs = {k: torch.zeros(m * N, dtype=dt, device="cuda") for k, m, dt in
            [("c", 1, torch.float64), ("c_ppt", 1, ft), ("eig", 1, ft), ("u", 2, torch.float64),
             ("strain", 3, ft), ("stress", 3, ft), ("H", 1, ft), ("damage", 1, torch.float64)]}
    bufs["phase"] = torch.as_tensor(w.phase.ravel()).cuda()
    mask = torch.as_tensor(w.dirichlet_mask.ravel()).cuda()
    st = fm.fftmech_state()
    for k, v in bufs.items():
        setattr(st, k, v.data_ptr())
    p = fm.fftmech_step_params()
    p.diffusion_mode = fm.FFTMECH_DIFF_TRANSIENT
    p.dt = w.dt
    p.dirichlet_mask = mask.data_ptr()
    p.dirichlet_value = w.dirichlet_value
    p.eig_mode = fm.FFTMECH_EIG_FROM_PRECIPITATE
    out = []
    for _ in range(steps):
        infos = fm.fftmech_staggered_step(ctx.handle, st, p)
        assert all(i.status == fm.FFTMECH_OK for i in infos)
        torch.cuda.synchronize()
        out.append({k: v.double().cpu().numpy().reshape(-1, N) for k, v in bufs.items() if k != "phase"})
    ctx.close()
    assert abs(float(np.load(GOLDEN)["dt"]) - w.dt) < 1e-12
    return out


@pytest.mark.parametrize("prec", [fm.FFTMECH_FP64, fm.FFTMECH_MIXED])
def test_carpet729_first_three_steps_match_oracle_golden(prec):
    if not os.path.exists(GOLDEN):
        pytest.fail("golden file missing: run tests/golden/make_carpet729_golden.py")
    g = np.load(GOLDEN)
    idx = g["idx"]
    steps = run(prec, 1e-13 if prec == fm.FFTMECH_FP64 else 1e-8, 3)
    for s, fields in enumerate(steps):
        errs = {}
        for name, (buf, _m) in FIELDS.items():
            ref_at = g[f"s{s}_{name}_at"]
            got = fields[buf]
            errs[name] = rel(got[:, idx], ref_at)
            if prec == fm.FFTMECH_FP64:
                # Sums on the scale sqrt(N) |a|_2 >= sum |a| (Cauchy-Schwarz):
                # a fluctuating field's sum can vanish (the strain's mean is
                # the macro strain, 0 here), so its own value is no scale.
                l2 = g[f"s{s}_{name}_l2"]
                N = got.shape[1]
                for stat, fn, scale in (("sum", lambda a: a.sum(axis=1), np.sqrt(N) * np.abs(l2).max()),
                                        ("l2", lambda a: np.sqrt((a * a).sum(axis=1)), np.abs(l2).max())):
                    ref = g[f"s{s}_{name}_{stat}"]
                    if scale > 0:
                        errs[f"{name}_{stat}"] = float(np.abs(fn(got) - ref).max() / scale)
        errs["d_maxabs"] = float(np.abs(steps[s]["damage"][:, idx] - g[f"s{s}_d_at"]).max())
        print("golden 729 step", s, "FP64" if prec == fm.FFTMECH_FP64 else "MIXED", errs)
        if prec == fm.FFTMECH_FP64:
            for k, e in errs.items():
                if k != "d_maxabs":
                    assert e < 1e-10, (s, k, e)
        else:
            assert errs["strain"] < 1e-5 and errs["stress"] < 1e-5, (s, errs)
            assert errs["c"] < 1e-6, (s, errs)
            assert errs["d_maxabs"] < 1e-4, (s, errs)
