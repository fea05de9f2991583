"""Plain conjugate gradient: Algorithm 1's "linear iterative solver".

The operator is a Python callable on numpy arrays of any shape; the inner
product is the plain sum over every entry (the l2 product of the gradient
space in which the paper's unknowns live). Hestenes-Stiefel recurrences,
no preconditioner, zero initial guess unless one is given.
"""

import numpy as np


def dot(a, b):
    return float(np.vdot(a.ravel(), b.ravel()).real)


def cg(apply_A, b, x0=None, tol=1e-12, max_iter=100000, record=False):
    """Solve A x = b for a symmetric positive (semi)definite A whose range
    holds b. Stops when ||r|| <= tol ||b||. Returns (x, info) where info has
    the iteration count, the final relative residual and, when `record`, the
    relative residual and the energy 1/2 x.Ax - b.x after every iteration."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = np.sqrt(dot(b, b))
    info = {"iters": 0, "rel_res": 0.0, "history": [], "energy": []}
    if bnorm == 0.0:
        return x, info
    r = b - apply_A(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = dot(r, r)
    if record:
        info["history"].append(np.sqrt(rr) / bnorm)
    it = 0
    while np.sqrt(rr) > tol * bnorm and it < max_iter:
        Ap = apply_A(p)
        alpha = rr / dot(p, Ap)
        x += alpha * p
        r -= alpha * Ap
        rr_new = dot(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
        if record:
            info["history"].append(np.sqrt(rr) / bnorm)
            info["energy"].append(0.5 * dot(x, apply_A(x)) - dot(b, x))
    info["iters"] = it
    info["rel_res"] = np.sqrt(rr) / bnorm
    return x, info
