"""Uniform batches (independent RVEs of one grid solved together): every
problem of a batch gives the fields and iteration counts it gets when solved
alone, and the batched staggered step matches the oracle per problem."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from microstructures import random_carpet
from microstructures.workloads import Materials, left_face_mask
from oracle import elasticity, phasefield, staggered
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


def problems(n, seeds):
    out = []
    for s in seeds:
        ph, _ = random_carpet(n, 0.30, s)
        rng = np.random.default_rng(s)
        eig = np.where(ph == 0, 1e-3 * (1 + 0.2 * rng.standard_normal(ph.shape)), 0.0)
        dmg = np.clip(0.5 * rng.random(ph.shape) ** 3, 0, 1)
        out.append((ph, eig, dmg))
    return out


def solve_equilibrium(probs, prec, tol, batch):
    n = probs[0][0].shape
    N = probs[0][0].size
    B = len(probs)
    ft = torch.float64 if prec == fm.FFTMECH_FP64 else torch.float32
    ctx = fm.Context(n, MAT, prec, h=H, tol=tol, batch=B if batch else 1)
    if batch:
        phase = torch.as_tensor(np.concatenate([p[0].ravel() for p in probs])).cuda()
        eig = torch.as_tensor(np.concatenate([p[1].ravel() for p in probs])).to(ft).cuda()
        dmg = torch.as_tensor(np.concatenate([p[2].ravel() for p in probs])).cuda()
        u = torch.zeros(2 * N * B, dtype=torch.float64, device="cuda")
        strain = torch.zeros(3 * N * B, dtype=ft, device="cuda")
        infos = fm.fftmech_equilibrium_solve(ctx.handle, phase, eig, dmg, [1e-4, 0, 0], u, strain, None)
        infos = [infos[b] for b in range(B)] if B > 1 else [infos]
        st = strain.double().cpu().numpy().reshape(B, 3, *n)
        out = [(st[b], infos[b].iters, infos[b].status) for b in range(B)]
    else:
        out = []
        for ph, e, d in probs:
            u = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
            strain = torch.zeros(3 * N, dtype=ft, device="cuda")
            info = fm.fftmech_equilibrium_solve(ctx.handle, torch.as_tensor(ph.ravel()).cuda(),
                                                torch.as_tensor(e.ravel()).to(ft).cuda(),
                                                torch.as_tensor(d.ravel()).cuda(), [1e-4, 0, 0], u, strain,
                                                None)
            out.append((strain.double().cpu().numpy().reshape(3, *n), info.iters, info.status))
    ctx.close()
    return out


@pytest.mark.parametrize("prec,tol", [(fm.FFTMECH_FP64, 1e-11), (fm.FFTMECH_MIXED, 1e-8)])
def test_batched_equilibrium_equals_single_solves(prec, tol):
    probs = problems(81, [3, 4, 5])
    a = solve_equilibrium(probs, prec, tol, batch=True)
    b = solve_equilibrium(probs, prec, tol, batch=False)
    for (sa, ia, ka), (sb, ib, kb) in zip(a, b):
        assert ka == fm.FFTMECH_OK and kb == fm.FFTMECH_OK
        assert ia == ib
        assert np.array_equal(sa, sb)


def test_batched_staggered_step_matches_oracle():
    """Three random carpets, transient diffusion -> precipitate eigenstrain ->
    equilibrium -> phase field, 2 steps, FP64, each against the oracle."""
    n = 81
    B = 3
    mat = Materials(E_pore=2e9, M_ppt=2.2)
    phases = [random_carpet(n, 0.30, s)[0] for s in (7, 8, 9)]
    masks = [left_face_mask(p) for p in phases]
    dt = (n / 4.0) ** 2 / 10
    refs = []
    for ph, mk in zip(phases, masks):
        r = staggered.initial_state(ph)
        for _ in range(2):
            r, _ = staggered.step(r, ph, mat, H, 1.0, staggered.DIFF_TRANSIENT,
                                  staggered.EIG_FROM_PRECIPITATE, dt=dt, mask=mk, c_dirichlet=1.0,
                                  tol=1e-12)
        refs.append(r)
    N = n * n
    ctx = fm.Context((n, n), mat, fm.FFTMECH_FP64, h=H, h_diff=1.0, tol=1e-12, batch=B)
    f64 = torch.float64
    bufs = {k: torch.zeros(m * N * B, dtype=f64, device="cuda") for k, m in
            [("c", 1), ("c_ppt", 1), ("eig", 1), ("u", 2), ("strain", 3), ("stress", 3), ("H", 1),
             ("damage", 1)]}
    bufs["phase"] = torch.as_tensor(np.concatenate([p.ravel() for p in phases])).cuda()
    mask = torch.as_tensor(np.concatenate([m.ravel() for m in masks])).cuda()
    st = fm.fftmech_state()
    for k, v in bufs.items():
        setattr(st, k, v.data_ptr())
    p = fm.fftmech_step_params()
    p.diffusion_mode = fm.FFTMECH_DIFF_TRANSIENT
    p.dt = dt
    p.dirichlet_mask = mask.data_ptr()
    p.dirichlet_value = 1.0
    p.eig_mode = fm.FFTMECH_EIG_FROM_PRECIPITATE
    for _ in range(2):
        infos = fm.fftmech_staggered_step(ctx.handle, st, p)
        assert all(infos[i].status == fm.FFTMECH_OK for i in range(3 * B))
    torch.cuda.synchronize()
    ctx.close()
    c = bufs["c"].cpu().numpy().reshape(B, n, n)
    strain = bufs["strain"].cpu().numpy().reshape(B, 3, n, n)
    d = bufs["damage"].cpu().numpy().reshape(B, n, n)
    for b in range(B):
        errs = (rel(c[b], refs[b]["c"]), rel(strain[b], refs[b]["strain"]), rel(d[b], refs[b]["d"]))
        print("batched staggered problem", b, errs)
        assert max(errs) < 1e-10
    assert refs[0]["eig"].max() > 0 and refs[0]["d"].max() > 1e-4


def _transient_state(ctx_shape, phases, mat, dt):
    """Device state of a uniform batch for a transient staggered step."""
    n = phases[0].size
    B = len(phases)
    f64 = torch.float64
    bufs = {k: torch.zeros(m * n * B, dtype=f64, device="cuda") for k, m in
            [("c", 1), ("c_ppt", 1), ("eig", 1), ("u", 2), ("strain", 3), ("stress", 3), ("H", 1),
             ("damage", 1)]}
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


def test_many_contexts_equal_separate_steps():
    """Uneven grids (27^2 x 2 and 81^2 x 1) stepped together through
    fftmech_staggered_step_many give the fields of separate steps."""
    mat = Materials(E_pore=2e9, M_ppt=2.2)
    groups = [[random_carpet(27, 0.30, s)[0] for s in (1, 2)], [random_carpet(81, 0.30, 3)[0]]]
    results = {}
    for mode in ("many", "separate"):
        ctxs, states, params, keep = [], [], [], []
        for phases in groups:
            n = phases[0].shape[0]
            ctx = fm.Context(phases[0].shape, mat, fm.FFTMECH_FP64, h=H, h_diff=1.0, tol=1e-12, batch=len(phases))
            bufs, st, p = _transient_state(phases[0].shape, phases, mat, (n / 4.0) ** 2 / 10)
            ctxs.append(ctx)
            states.append(st)
            params.append(p)
            keep.append(bufs)
        for _ in range(2):
            if mode == "many":
                infos = fm.fftmech_staggered_step_many([c.handle for c in ctxs], states, params)
                for inf in infos:
                    assert all(inf[i].status == fm.FFTMECH_OK for i in range(len(inf)))
            else:
                for c, st, p in zip(ctxs, states, params):
                    inf = fm.fftmech_staggered_step(c.handle, st, p)
        torch.cuda.synchronize()
        results[mode] = [{k: b[k].cpu().numpy() for k in ("c", "strain", "damage")} for b in keep]
        for c in ctxs:
            c.close()
    for a, b in zip(results["many"], results["separate"]):
        for k in a:
            assert np.array_equal(a[k], b[k])
    assert results["many"][1]["damage"].max() > 0


def test_group_graph_equals_separate_steps_and_matches_oracle():
    """A group of three contexts of uneven grids (27^2 x 2, 81^2, 128^2 2x2
    carpet) stepped as one graph (one launch per step, a parallel branch per
    context) gives bit for bit the fields of separate steps, and problem 0
    of the 27^2 context matches the oracle."""
    mat = Materials(E_pore=2e9, M_ppt=2.2)
    groups = [[random_carpet(27, 0.30, s)[0] for s in (1, 2)], [random_carpet(81, 0.30, 3)[0]],
              [random_carpet(128, 0.30, 4, base=2)[0]]]
    results = {}
    for mode in ("group", "separate"):
        ctxs, states, params, keep = [], [], [], []
        for phases in groups:
            n = phases[0].shape[0]
            ctx = fm.Context(phases[0].shape, mat, fm.FFTMECH_FP64, h=H, h_diff=1.0, tol=1e-12, batch=len(phases))
            bufs, st, p = _transient_state(phases[0].shape, phases, mat, (n / 4.0) ** 2 / 10)
            ctxs.append(ctx)
            states.append(st)
            params.append(p)
            keep.append(bufs)
        grp = fm.Group(ctxs) if mode == "group" else None
        for _ in range(2):
            if grp is not None:
                infos = grp.step(states, params)
                for inf in infos:
                    assert all(inf[i].status == fm.FFTMECH_OK for i in range(len(inf)))
            else:
                for c, st, p in zip(ctxs, states, params):
                    fm.fftmech_staggered_step(c.handle, st, p)
        torch.cuda.synchronize()
        if grp is not None:
            builds, launches, kernels = grp.stats()
            assert builds == 1 and launches == 2 and kernels > 0
            grp.close()
        results[mode] = [{k: b[k].cpu().numpy() for k in ("c", "strain", "damage")} for b in keep]
        for c in ctxs:
            c.close()
    for a, b in zip(results["group"], results["separate"]):
        for k in a:
            assert np.array_equal(a[k], b[k])
    ph = groups[0][0]
    ref = staggered.initial_state(ph)
    for _ in range(2):
        ref, _ = staggered.step(ref, ph, mat, H, 1.0, staggered.DIFF_TRANSIENT, staggered.EIG_FROM_PRECIPITATE,
                                dt=(27 / 4.0) ** 2 / 10, mask=left_face_mask(ph), c_dirichlet=1.0, tol=1e-12)
    N = ph.size
    assert rel(results["group"][0]["c"][:N].reshape(ph.shape), ref["c"]) < 1e-10
    assert rel(results["group"][0]["strain"][:3 * N].reshape((3,) + ph.shape), ref["strain"]) < 1e-10
