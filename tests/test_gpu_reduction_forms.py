"""The two forms of the PCG reductions give the same solutions.

Launches of up to 2^21 voxels defer <p, K p> and <r, M^-1 r> to the kernel
that consumes them (every block of it sums the producer's partials); larger
launches finalise them in the producer's last block. A batch whose voxels
exceed 2^21 therefore runs the last-block form while each of its problems
solved alone runs the deferred form: the fields must agree within what two
solves stopped at the same relative residual can differ by, and the
iteration counts within 2 % (rounding in a different order can move the
stopping iteration)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from microstructures import random_carpet, random_sponge
from microstructures.workloads import Materials
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


def problems(phases, seed):
    rng = np.random.default_rng(seed)
    out = []
    for ph in phases:
        eig = np.where(ph == 0, 1e-3 * (1 + 0.2 * rng.standard_normal(ph.shape)), 0.0)
        dmg = np.clip(0.5 * rng.random(ph.shape) ** 3, 0, 1)
        out.append((np.ascontiguousarray(ph), eig, dmg))
    return out


def solve(probs, prec, tol, batched):
    shape = probs[0][0].shape
    d = len(shape)
    nv = 3 if d == 2 else 6
    N = probs[0][0].size
    ft = torch.float64 if prec == fm.FFTMECH_FP64 else torch.float32
    E = [1e-4, 0, 0] if d == 2 else [1e-4, 0, 0, 0, 0, 2e-5]
    groups = [probs] if batched else [[p] for p in probs]
    strains, iters = [], []
    for g in groups:
        B = len(g)
        ctx = fm.Context(shape, MAT, prec, h=H, tol=tol, max_iter=50000, batch=B)
        cat = lambda k, dt: torch.as_tensor(np.concatenate([p[k].ravel() for p in g])).to(dt).cuda()
        u = torch.zeros(d * N * B, dtype=torch.float64, device="cuda")
        strain = torch.zeros(nv * N * B, dtype=ft, device="cuda")
        infos = fm.fftmech_equilibrium_solve(ctx.handle, cat(0, torch.uint8), cat(1, ft), cat(2, torch.float64), E,
                                             u, strain, None)
        torch.cuda.synchronize()
        ctx.close()
        infos = [infos[b] for b in range(B)] if B > 1 else [infos]
        assert all(i.status == fm.FFTMECH_OK for i in infos)
        st = strain.double().cpu().numpy().reshape((B, nv) + shape)
        strains += [st[b] for b in range(B)]
        iters += [i.iters for i in infos]
    return strains, iters


@pytest.mark.parametrize("prec,tol,bound", [(fm.FFTMECH_FP64, 1e-11, 1e-8), (fm.FFTMECH_MIXED, 1e-8, 1e-5)])
def test_2d_last_block_batch_matches_deferred_single_solves(prec, tol, bound):
    # 8 x 729^2 = 4.25 M voxels per launch (last block); one 729^2 problem: deferred
    probs = problems([random_carpet(729, 0.30, s)[0] for s in range(40, 48)], 5)
    a, ia = solve(probs, prec, tol, batched=True)
    b, ib = solve(probs, prec, tol, batched=False)
    for sa, sb, na, nb in zip(a, b, ia, ib):
        assert abs(na - nb) <= max(2, nb // 50)
        assert rel(sa, sb) < bound


def test_3d_last_block_batch_matches_deferred_single_solves():
    # 4 x 81^3 = 2.13 M voxels per launch (last block); one 81^3 problem: deferred
    probs = problems([random_sponge(81, 0.35, s)[0] for s in (51, 52, 53, 54)], 6)
    a, ia = solve(probs, fm.FFTMECH_MIXED, 1e-8, batched=True)
    b, ib = solve(probs, fm.FFTMECH_MIXED, 1e-8, batched=False)
    for sa, sb, na, nb in zip(a, b, ia, ib):
        assert abs(na - nb) <= max(2, nb // 50)
        assert rel(sa, sb) < 1e-5
