"""Fractal pore geometries on voxel grids.

The phase indicator follows the paper's omega (Sec. 2.1, the definition of the
diffusion tensor, and Sec. 2.3, the stiffness): omega = 1 in the solid, 0 in
the pores. Arrays are C-ordered with the x index fastest: shape (ny, nx) in 2D,
(nz, ny, nx) in 3D, dtype uint8.

The paper's own geometry is a 199^2 FIB-SEM scan (Sec. 3) that is not
available; these seeded fractals stand in for it with the porosity range it
reports (0.17 - 0.45).

Random fractals are built level by level: every solid block is split into
base^dim sub-blocks, of which k stay solid and the rest become pore for good.
k is drawn from {k_min, ..., base^dim} with weights proportional to exp(t k),
t tuned so that the expected solid fraction kept per level is
(1 - target)^(1/levels); a draw whose porosity misses the target by more than
`tol` is rejected and redrawn with the next attempt index.
"""

import numpy as np

from .splitmix import derive_key, uniform01


def porosity(phase):
    """Pore volume fraction eta = |Omega_p| / |Omega| (Sec. 2)."""
    phase = np.asarray(phase)
    return float(np.count_nonzero(phase == 0)) / phase.size


def _upsample(mask, factor):
    out = mask
    for ax in range(mask.ndim):
        out = np.repeat(out, factor, axis=ax)
    return out


def sierpinski_carpet(levels, dim=2):
    """Deterministic Sierpinski carpet (dim=2) or Menger sponge pattern
    (dim=3 keeps the 26 non-centre sub-cubes) on a 3^levels grid: the centre
    sub-block of every solid block is made pore at each level.
    Porosity is exactly 1 - ((3^dim - 1) / 3^dim)^levels."""
    solid = np.ones((1,) * dim, dtype=bool)
    centre = np.ones((3,) * dim, dtype=bool)
    centre[(1,) * dim] = False
    for _ in range(levels):
        solid = np.kron(solid, centre).astype(bool) & _upsample(solid, 3)
    return solid.astype(np.uint8)


def _tilt_for_mean(kmin, kmax, target_mean):
    ks = np.arange(kmin, kmax + 1, dtype=np.float64)
    if target_mean >= kmax:
        return np.inf
    if target_mean <= kmin:
        return -np.inf

    def mean(t):
        w = np.exp(t * (ks - kmax))
        return float((w * ks).sum() / w.sum())

    lo, hi = -60.0, 60.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mean(mid) < target_mean:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _keep_probs(kmin, kmax, t):
    ks = np.arange(kmin, kmax + 1, dtype=np.float64)
    if t == np.inf:
        p = np.zeros_like(ks)
        p[-1] = 1.0
    elif t == -np.inf:
        p = np.zeros_like(ks)
        p[0] = 1.0
    else:
        p = np.exp(t * (ks - kmax))
        p /= p.sum()
    return p


def _random_fractal_once(levels, base, dim, kmin, t, key):
    nsub = base ** dim
    probs = _keep_probs(kmin, nsub, t)
    cdf = np.cumsum(probs)
    cdf[-1] = 1.0
    solid = np.ones((1,) * dim, dtype=bool)
    for level in range(levels):
        nblocks = solid.size
        u = uniform01(derive_key(key, level), nblocks * (1 + nsub)).reshape(nblocks, 1 + nsub)
        kept = kmin + np.searchsorted(cdf, u[:, 0], side="right")
        kept = np.minimum(kept, nsub)
        # rank of each sub-block's uniform within its block; the (nsub - kept)
        # lowest-ranked sub-blocks turn into pore
        ranks = np.argsort(np.argsort(u[:, 1:], axis=1, kind="stable"), axis=1, kind="stable")
        keep = ranks >= (nsub - kept)[:, None]  # (nblocks, nsub)
        # scatter per-block sub-block masks into the refined grid
        side = base ** level
        keep = keep.reshape((side,) * dim + (base,) * dim)
        # interleave block axes with sub-block axes: (b0, s0, b1, s1, ...)
        order = []
        for ax in range(dim):
            order += [ax, dim + ax]
        keep = keep.transpose(order).reshape((side * base,) * dim)
        solid = _upsample(solid, base) & keep
    return solid


def random_carpet(n, target_porosity, seed, tol=0.02, base=3, levels=None,
                  kmin=None, dim=2, max_attempts=4000):
    """Seeded random fractal on an n^dim grid.

    n must be leaf * base^levels; by default levels = log_base(n) (leaf 1).
    Returns (phase uint8, attempt index that was accepted)."""
    if levels is None:
        levels = int(round(np.log(n) / np.log(base)))
    leaf = n // base ** levels
    if leaf * base ** levels != n:
        raise ValueError(f"n={n} is not a multiple of {base}^{levels}")
    nsub = base ** dim
    if kmin is None:
        kmin = {(3, 2): 6, (3, 3): 18, (2, 2): 2, (2, 3): 5}[(base, dim)]
    target_mean = nsub * (1.0 - target_porosity) ** (1.0 / levels)
    t = _tilt_for_mean(kmin, nsub, target_mean)
    for attempt in range(max_attempts):
        key = derive_key(seed, attempt, base, dim, n)
        solid = _random_fractal_once(levels, base, dim, kmin, t, key)
        eta = 1.0 - solid.mean()
        if abs(eta - target_porosity) <= tol:
            phase = _upsample(solid, leaf).astype(np.uint8)
            return phase, attempt
    raise RuntimeError("no seed attempt reached the porosity window")


def random_sponge(n, target_porosity, seed, tol=0.02, levels=None):
    """Seeded random Menger-type sponge on an n^3 grid (3x3x3 subdivision)."""
    return random_carpet(n, target_porosity, seed, tol=tol, base=3, levels=levels, dim=3)
