"""The library's macroscale bar (fftmech_bar_*, Sec. 3.2) through the C ABI:

- against the oracle's driver (oracle/macro.py) on 4 random-carpet RVEs of
  27 x 27 with a concentration profile that precipitates near the interface,
  3 macro steps: nodal concentrations, every RVE's mean flux and its
  concentration, eigenstrain, strain and damage fields (FP64 within 1e-10,
  mixed within 1e-6 / 1e-5);
- the closed form of a laminate bar: starting from the quadratic profile
  J / (2 D L) (X - L)^2 every node rises by dt J / L per step;
- the graph of a macro step is captured once and replayed.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from microstructures import random_carpet
from microstructures.workloads import Materials
from oracle import macro as omacro
from paper_2305_13081_gb300 import build
from paper_2305_13081_gb300 import fftmech as fm
from paper_2305_13081_gb300.macro import MacroBar

pytestmark = pytest.mark.gpu

MAT = Materials(E_pore=2e9)
H = 5e-6
L = 400.0
M = 4
J_IN = 1e-3
DT = 2000.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    fm.load_library()


def rel(a, b):
    nb = np.linalg.norm(np.ravel(b))
    return float(np.linalg.norm(np.ravel(a - b)) / nb) if nb > 0 else float(np.linalg.norm(np.ravel(a)))


@pytest.mark.parametrize("prec", [fm.FFTMECH_FP64, fm.FFTMECH_MIXED])
def test_bar_matches_oracle_driver(prec):
    phases = [random_carpet(27, 0.30, 40 + s)[0] for s in range(M)]
    c0 = np.array([0.31, 0.25, 0.15, 0.05, 0.0])
    ref = omacro.MacroBarOracle(phases, MAT, H, 1.0, L, DT, J_IN, c0=c0, tol=1e-12)
    bar = MacroBar(phases, MAT, L, DT, J_IN, c0=c0, precision=prec, h=H,
                   tol=1e-12 if prec == fm.FFTMECH_FP64 else 1e-9)
    fp64 = prec == fm.FFTMECH_FP64
    for s in range(3):
        c_prev = ref.c.copy()
        fluxes = ref.step()
        infos = bar.step()
        got_flux = np.array([infos[3 * e].mean_flux[0] for e in range(M)])
        errs = {"nodes": rel(bar.nodes(), ref.c), "flux": rel(got_flux, fluxes)}
        for e in range(M):
            st = ref.states[e]
            errs[f"c{e}"] = rel(bar.field("c", e)[0], st["c"])
            errs[f"eig{e}"] = rel(bar.field("eig", e)[0], st["eig"])
            errs[f"strain{e}"] = rel(bar.field("strain", e), st["strain"])
            errs[f"d{e}"] = float(np.abs(bar.field("damage", e)[0] - st["d"]).max())
            want_c = 0.5 * (c_prev[e] + c_prev[e + 1])  # the element's c_macro
            assert abs(infos[3 * e].mean_c - want_c) <= (1e-12 if fp64 else 1e-8) * abs(want_c) + 1e-30
        print("bar step", s, "FP64" if fp64 else "MIXED", {k: f"{v:.2e}" for k, v in errs.items()})
        assert errs["nodes"] < (1e-12 if fp64 else 1e-8), errs
        assert errs["flux"] < (1e-10 if fp64 else 1e-6), errs
        for e in range(M):
            assert errs[f"c{e}"] < (1e-10 if fp64 else 1e-6), (e, errs)
            assert errs[f"strain{e}"] < (1e-9 if fp64 else 1e-5), (e, errs)
            assert errs[f"d{e}"] < (1e-10 if fp64 else 1e-4), (e, errs)
    assert np.abs(ref.states[0]["eig"]).max() > 0  # the case precipitates
    bar.close()


def test_laminate_bar_closed_form_and_one_graph():
    n = 27
    ph = np.zeros((n, n), dtype=np.uint8)
    ph[:, n // 2 + 1:] = 1  # layers normal to the bar
    D = np.where(ph[0] == 0, MAT.D_pore, MAT.D_solid)
    Deff = 1.0 / np.mean(1.0 / D)
    dX = L / M
    X = dX * np.arange(M + 1)
    J = 1e-6  # keeps c below the solubility limit (no precipitation)
    c0 = J / (2.0 * Deff * L) * (X - L) ** 2
    bar = MacroBar([ph] * M, MAT, L, DT, J, c0=c0, precision=fm.FFTMECH_FP64, h=H, tol=1e-13)
    for s in range(1, 4):
        bar.step()
        want = c0 + s * DT * J / L
        assert np.abs(bar.nodes() - want).max() <= 1e-10 * np.abs(want).max()
    builds, launches, _, disabled, _ = fm.fftmech_graph_stats(bar.ctx.handle)
    assert disabled == 0 and builds == 1 and launches == 3
    bar.close()


def test_bar_rejects_unstable_dt_and_host_pointers():
    ph = random_carpet(27, 0.30, 40)[0]
    ctx = fm.Context(ph.shape, MAT, fm.FFTMECH_FP64, h=H, batch=M)
    with pytest.raises(fm.FftmechError):
        fm.fftmech_bar_create(ctx.handle, L, 0.51 * (L / M) ** 2, J_IN)
    ctx.close()
