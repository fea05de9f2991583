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


def gmres(apply_A, b, tol=1e-12, restart=50, max_iter=100000, apply_M=None):
    """Restarted GMRES(m) (Saad and Schultz) for a general real operator A,
    with an optional right preconditioner M (A M y = b, x = M y): Arnoldi
    with modified Gram-Schmidt, Givens rotations on the Hessenberg matrix,
    the least-squares solution at the end of each cycle. Stops when
    ||b - A x|| <= tol ||b||. Returns (x, info) with the inner iteration
    count and the final relative residual of the recurrence."""
    M = apply_M if apply_M is not None else (lambda v: v)
    x = np.zeros_like(b)
    bnorm = np.sqrt(dot(b, b))
    info = {"iters": 0, "rel_res": 0.0}
    if bnorm == 0.0:
        return x, info
    r = b.copy()
    while True:
        beta = np.sqrt(dot(r, r))
        info["rel_res"] = beta / bnorm
        if beta <= tol * bnorm or info["iters"] >= max_iter:
            return x, info
        V = [r / beta]
        Hm = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        k = 0
        for j in range(restart):
            w = apply_A(M(V[j]))
            for i in range(j + 1):
                Hm[i, j] = dot(V[i], w)
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.sqrt(dot(w, w))
            V.append(w / Hm[j + 1, j] if Hm[j + 1, j] > 0 else w)
            for i in range(j):  # earlier rotations on the new column
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            den = np.hypot(Hm[j, j], Hm[j + 1, j])
            cs[j], sn[j] = Hm[j, j] / den, Hm[j + 1, j] / den
            Hm[j, j] = den
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            info["iters"] += 1
            if abs(g[j + 1]) <= tol * bnorm or info["iters"] >= max_iter:
                break
        y = np.linalg.solve(np.triu(Hm[:k, :k]), g[:k])
        x = x + M(sum(y[i] * V[i] for i in range(k)))
        r = b - apply_A(x)
