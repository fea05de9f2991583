"""The device-driven PCG as one CUDA graph: every loop decision
(convergence, iteration limit, reliable updates, restarts) is taken by the
kernels, so a staggered step (Algorithm 1) runs as one graph launch with
conditional WHILE / IF nodes and no host synchronisation inside it.

Checked here, through the C ABI:
- the graph execution and the host-driven execution (same kernels, the host
  polls the device's loop flags) give bit-identical fields and iteration
  counts: one problem (the direction kernel decides), a batch (the loop
  control kernel decides), 2D and 3D, FP64 and mixed;
- the graph path is the one that ran (graph launches counted, not disabled);
- fftmech_staggered_step_async + fftmech_step_info equal the synchronous call;
- a step captured by the caller into their own CUDA graph (stream capture on
  the context's stream) and replayed gives the fields of the uncaptured call.
"""

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


class Problem:
    """Device state of a (batched) transient carpet or prescribed-eigenstrain
    sponge, stepped through one context."""

    def __init__(self, phases, prec, tol, execution, stream=None, three=False):
        self.B = len(phases)
        shape = phases[0].shape
        N = phases[0].size
        dim = len(shape)
        nv = 3 if dim == 2 else 6
        ft = torch.float64 if prec == fm.FFTMECH_FP64 else torch.float32
        self.ctx = fm.Context(shape, MAT, prec, h=H, h_diff=1.0, tol=tol, batch=self.B, execution=execution,
                              stream=stream)
        B = self.B
        self.bufs = {k: torch.zeros(m * N * B, dtype=dt, device="cuda") for k, m, dt in
                     [("c", 1, torch.float64), ("c_ppt", 1, ft), ("eig", 1, ft), ("u", dim, torch.float64),
                      ("strain", nv, ft), ("stress", nv, ft), ("H", 1, ft), ("damage", 1, torch.float64)]}
        self.bufs["phase"] = torch.as_tensor(np.concatenate([p.ravel() for p in phases])).cuda()
        self.st = fm.fftmech_state()
        for k, v in self.bufs.items():
            setattr(self.st, k, v.data_ptr())
        self.p = fm.fftmech_step_params()
        if three:
            self.eigf = torch.as_tensor(np.concatenate([np.where(p == 0, 2e-2, 0.0).ravel() for p in phases])).to(ft).cuda()
            self.p.diffusion_mode = fm.FFTMECH_DIFF_NONE
            self.p.eig_mode = fm.FFTMECH_EIG_PRESCRIBED
            self.p.eig_field = self.eigf.data_ptr()
            self.p.eig_scale = 1.0
        else:
            n = shape[-1]
            self.mask = torch.as_tensor(np.concatenate([left_face_mask(p).ravel() for p in phases])).cuda()
            self.p.diffusion_mode = fm.FFTMECH_DIFF_TRANSIENT
            self.p.dt = (n / 4.0) ** 2 / 10
            self.p.dirichlet_mask = self.mask.data_ptr()
            self.p.dirichlet_value = 1.0
            self.p.eig_mode = fm.FFTMECH_EIG_FROM_PRECIPITATE

    def step(self):
        return [i.as_dict() for i in fm.fftmech_staggered_step(self.ctx.handle, self.st, self.p)]

    def fields(self):
        torch.cuda.synchronize()
        return {k: v.cpu().numpy().copy() for k, v in self.bufs.items()}

    def close(self):
        self.ctx.close()


def assert_same(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def carpets(n, seeds):
    return [random_carpet(n, 0.30, s)[0] for s in seeds]


CASES = [
    ("carpet81-fp64", lambda: carpets(81, [5]), fm.FFTMECH_FP64, 1e-11, False),
    ("carpet243-mixed", lambda: carpets(243, [6]), fm.FFTMECH_MIXED, 1e-8, False),
    ("carpet81x3-mixed", lambda: carpets(81, [7, 8, 9]), fm.FFTMECH_MIXED, 1e-8, False),
    ("sponge27-mixed", lambda: [random_sponge(27, 0.35, 3)[0]], fm.FFTMECH_MIXED, 1e-8, True),
    ("sponge27x2-fp64", lambda: [random_sponge(27, 0.35, s)[0] for s in (4, 5)], fm.FFTMECH_FP64, 1e-11, True),
]


@pytest.mark.parametrize("name,phases_fn,prec,tol,three", CASES, ids=[c[0] for c in CASES])
def test_graph_and_host_driven_execution_are_bit_identical(name, phases_fn, prec, tol, three):
    phases = phases_fn()
    out = {}
    for ex in (fm.FFTMECH_EXEC_GRAPH, fm.FFTMECH_EXEC_HOST):
        pr = Problem(phases, prec, tol, ex, three=three)
        infos = [pr.step() for _ in range(3)]
        out[ex] = (pr.fields(), infos)
        if ex == fm.FFTMECH_EXEC_GRAPH:
            builds, launches, kernels, disabled, why = fm.fftmech_graph_stats(pr.ctx.handle)
            assert disabled == 0, why
            assert launches == 3 and builds >= 1
            # at least stencil, update, column pass and direction per equilibrium iteration
            assert kernels >= 4 * sum(inf[1]["iters"] for inf in infos)
        pr.close()
    fg, ig = out[fm.FFTMECH_EXEC_GRAPH]
    fh, ih = out[fm.FFTMECH_EXEC_HOST]
    assert_same(fg, fh)
    for a, b in zip(ig, ih):
        for x, y in zip(a, b):
            assert x["status"] == y["status"] == fm.FFTMECH_OK
            assert x["iters"] == y["iters"]
            assert x["rel_res"] == y["rel_res"]
    assert fg["damage"].max() > 0


def test_async_step_and_step_info_equal_the_synchronous_step():
    phases = carpets(243, [11])
    a = Problem(phases, fm.FFTMECH_MIXED, 1e-8, fm.FFTMECH_EXEC_GRAPH)
    b = Problem(phases, fm.FFTMECH_MIXED, 1e-8, fm.FFTMECH_EXEC_GRAPH)
    for _ in range(2):
        ia = a.step()
        fm.fftmech_staggered_step_async(b.ctx.handle, b.st, b.p)
        ib = [i.as_dict() for i in fm.fftmech_step_info(b.ctx.handle)]
        for x, y in zip(ia, ib):
            assert x["iters"] == y["iters"] and x["status"] == y["status"]
            assert x["elastic_energy"] == y["elastic_energy"]
    assert_same(a.fields(), b.fields())
    a.close()
    b.close()


def test_async_step_rejects_host_pointers():
    phases = carpets(27, [1])
    pr = Problem(phases, fm.FFTMECH_FP64, 1e-10, fm.FFTMECH_EXEC_GRAPH)
    host_c = np.zeros(phases[0].size)
    pr.st.c = host_c.ctypes.data
    with pytest.raises(fm.FftmechError) as ei:
        fm.fftmech_staggered_step_async(pr.ctx.handle, pr.st, pr.p)
    assert ei.value.status == fm.FFTMECH_ERR_INVALID_ARG
    pr.close()


def test_step_captured_into_a_caller_graph_and_replayed():
    """The caller captures fftmech_staggered_step_async on the context's
    stream into a torch CUDA graph and replays it twice; the fields equal
    two uncaptured steps."""
    phases = carpets(243, [12])
    ref = Problem(phases, fm.FFTMECH_MIXED, 1e-8, fm.FFTMECH_EXEC_GRAPH)
    for _ in range(2):
        ref.step()
    s = torch.cuda.Stream()
    cap = Problem(phases, fm.FFTMECH_MIXED, 1e-8, fm.FFTMECH_EXEC_GRAPH, stream=s.cuda_stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        fm.fftmech_staggered_step_async(cap.ctx.handle, cap.st, cap.p)
    # capturing ran nothing
    assert torch.count_nonzero(cap.bufs["c"]).item() == 0
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    info = [i.as_dict() for i in fm.fftmech_step_info(cap.ctx.handle)]
    assert all(i["status"] == fm.FFTMECH_OK for i in info)
    assert_same(ref.fields(), cap.fields())
    del g
    ref.close()
    cap.close()


@pytest.mark.parametrize("shape,prec", [((243, 243), fm.FFTMECH_MIXED), ((27, 27, 27), fm.FFTMECH_MIXED),
                                        ((81, 81), fm.FFTMECH_FP64)])
def test_autotuner_keeps_results_and_caches_its_choice(shape, prec):
    """The autotuner's choice is no slower than the default shapes on its own
    timing, the solve with the tuned shapes still meets the oracle, a new
    context of the same grid starts from the rule-based shapes, and tuning
    it applies the cached choice without timing again."""
    from oracle import elasticity
    from microstructures import random_sponge as _sponge
    ph = random_carpet(shape[0], 0.30, 31)[0] if len(shape) == 2 else _sponge(shape[0], 0.35, 31)[0]
    eig = np.where(ph == 0, 1e-3, 0.0)
    ctx = fm.Context(shape, MAT, prec, h=H, tol=1e-12 if prec == fm.FFTMECH_FP64 else 1e-8, max_iter=20000)
    before, after, desc = fm.fftmech_autotune(ctx.handle, 20)
    print("autotune", shape, before, after, desc)
    assert after <= before * 1.0001 and after > 0
    N = ph.size
    d = len(shape)
    nv = 3 if d == 2 else 6
    ft = torch.float64 if prec == fm.FFTMECH_FP64 else torch.float32
    u = torch.zeros(d * N, dtype=torch.float64, device="cuda")
    strain = torch.zeros(nv * N, dtype=ft, device="cuda")
    info = fm.fftmech_equilibrium_solve(ctx.handle, torch.as_tensor(ph.ravel()).cuda(),
                                        torch.as_tensor(eig.ravel()).to(ft).cuda(), None, [0] * 6, u, strain, None)
    assert info.status == fm.FFTMECH_OK
    ref = elasticity.equilibrium_solve(ph, eig, np.ones(shape), [0] * nv, MAT, H, tol=1e-12)
    got = strain.double().cpu().numpy().reshape(ref["strain"].shape)
    err = np.linalg.norm(got - ref["strain"]) / np.linalg.norm(ref["strain"])
    assert err < (1e-10 if prec == fm.FFTMECH_FP64 else 1e-5), err
    ctx.close()
    ctx2 = fm.Context(shape, MAT, prec, h=H)
    _, _, desc0 = fm.fftmech_autotune(ctx2.handle, 0)  # the shapes it starts from
    b2, a2, desc2 = fm.fftmech_autotune(ctx2.handle, 20)
    ctx2.close()
    assert not desc0.endswith(")")
    assert desc2.endswith("(cached)") and desc2.startswith(desc), (desc, desc2)
    assert (b2, a2) == (before, after)


def test_carpet729_transient_workload_graph_equals_host_driven():
    """The headline workload itself (729^2 random carpet, seed 2305, left-face
    source, precipitate eigenstrain, tol 1e-8, mixed path): twelve staggered
    steps as one graph launch each give the fields and iteration counts of
    the host-driven execution bit for bit, with no host synchronisation
    inside a step (one graph launch per step, graph path not disabled)."""
    from microstructures.workloads import carpet_transient
    w = carpet_transient(729)
    N = w.phase.size
    out = {}
    for ex in (fm.FFTMECH_EXEC_GRAPH, fm.FFTMECH_EXEC_HOST):
        ctx = fm.Context(w.phase.shape, w.materials, fm.FFTMECH_MIXED, h=w.h, h_diff=w.h_diff, tol=w.tol,
                         execution=ex)
        f32 = torch.float32
        bufs = {k: torch.zeros(m * N, dtype=dt, device="cuda") for k, m, dt in
                [("c", 1, torch.float64), ("c_ppt", 1, f32), ("eig", 1, f32), ("u", 2, torch.float64),
                 ("strain", 3, f32), ("stress", 3, f32), ("H", 1, f32), ("damage", 1, torch.float64)]}
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
        iters = []
        for _ in range(12):
            infos = fm.fftmech_staggered_step(ctx.handle, st, p)
            iters.append([i.iters for i in infos])
            assert all(i.status == fm.FFTMECH_OK for i in infos)
        if ex == fm.FFTMECH_EXEC_GRAPH:
            builds, launches, _, disabled, why = fm.fftmech_graph_stats(ctx.handle)
            assert disabled == 0, why
            assert launches == 12 and builds == 1
        torch.cuda.synchronize()
        out[ex] = ({k: v.cpu().numpy() for k, v in bufs.items()}, iters)
        ctx.close()
    fg, ig = out[fm.FFTMECH_EXEC_GRAPH]
    fh, ih = out[fm.FFTMECH_EXEC_HOST]
    assert ig == ih
    assert sum(it[1] for it in ig) > 0  # the equilibrium solves ran
    assert_same(fg, fh)
