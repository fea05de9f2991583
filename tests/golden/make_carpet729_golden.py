"""Writes tests/golden/carpet729_steps1to3.npz: the FP64 CPU oracle's first
three staggered steps (Algorithm 1) of the transient random-carpet workload on
729 x 729 (3^6, seed 2305, porosity 0.30 +/- 0.02, left-face source at c = 1,
dt = (729/4)^2 / 200, precipitate eigenstrain, equilibrium and phase field,
every solve to a 1e-12 relative residual).

The full fields are 42 MB a step, so the file keeps, per step and field:
- the values at 4096 fixed voxels (half drawn uniformly, half from the 40
  columns next to the source, where the concentration front and the
  eigenstrain are), and
- the sum and the L2 norm of every field component over all voxels.

Calls only the oracle and the seeded input generators. Run from the
repository root: python tests/golden/make_carpet729_golden.py
"""

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from microstructures.workloads import carpet_transient  # noqa: E402
from oracle import staggered  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "carpet729_steps1to3.npz")
FIELDS = ("c", "c_ppt", "eig", "strain", "stress", "H", "d")


def sample_indices(n, k=4096, seed=2305):
    rng = np.random.default_rng(seed)
    a = rng.choice(n * n, k // 2, replace=False)
    rows = rng.integers(0, n, k // 2)
    cols = rng.integers(0, 40, k // 2)
    b = rows * n + cols
    return np.unique(np.concatenate([a, b])).astype(np.int64)


def main(steps=3):
    w = carpet_transient(729)
    phase = w.phase
    n = phase.shape[0]
    idx = sample_indices(n)
    state = staggered.initial_state(phase, w.c0)
    out = {"idx": idx, "porosity": np.float64(w.extra["porosity"]), "dt": np.float64(w.dt)}
    for s in range(steps):
        t0 = time.time()
        state, info = staggered.step(state, phase, w.materials, w.h, w.h_diff, w.diffusion_mode, w.eig_mode,
                                     dt=w.dt, mask=w.dirichlet_mask, c_dirichlet=w.dirichlet_value, tol=1e-12)
        for f in FIELDS:
            v = np.asarray(state[f], dtype=np.float64)
            comps = v.reshape((-1, n * n))
            out[f"s{s}_{f}_at"] = comps[:, idx]
            out[f"s{s}_{f}_sum"] = comps.sum(axis=1)
            out[f"s{s}_{f}_l2"] = np.sqrt((comps * comps).sum(axis=1))
        out[f"s{s}_iters_eq"] = np.int64(info["equilibrium"]["iters"])
        out[f"s{s}_iters_pf"] = np.int64(info["phasefield"]["iters"])
        print(f"step {s}: {time.time() - t0:.1f} s, eq iters {info['equilibrium']['iters']}, "
              f"max eig {state['eig'].max():.3e}, max d {state['d'].max():.3e}", flush=True)
    np.savez_compressed(OUT, **out)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
