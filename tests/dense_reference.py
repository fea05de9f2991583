"""Brute-force reference for small grids: the same discrete equations as the
oracle, assembled as explicit matrices from real-space forward differences
(no FFT, no projection operator) and solved with a dense direct solver.

Used to pin the oracle (tests only). Real-space operator: B_alpha u(x) =
(u(x + h e_alpha) - u(x)) / h on the periodic grid; the Galerkin system of a
gradient-form law is B^T (law) B. The mean of a potential is fixed to zero
with Lagrange multipliers.
"""

import numpy as np
import scipy.sparse as sp


def fwd(shape, alpha, h):
    ndim = len(shape)
    ax = ndim - 1 - alpha
    N = int(np.prod(shape))
    idx = np.arange(N).reshape(shape)
    nxt = np.roll(idx, -1, axis=ax).ravel()
    M = sp.lil_matrix((N, N))
    M[np.arange(N), nxt] = 1.0 / h
    M[np.arange(N), np.arange(N)] = -1.0 / h
    return M.tocsr()


def lame(E, nu):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def solve_with_zero_mean(K, f, ncomp, N):
    """Solve K u = f with sum over each component block = 0 (Lagrange)."""
    n = K.shape[0]
    A = np.zeros((n + ncomp, n + ncomp))
    A[:n, :n] = K.toarray() if sp.issparse(K) else K
    for c in range(ncomp):
        A[n + c, c * N:(c + 1) * N] = 1.0
        A[c * N:(c + 1) * N, n + c] = 1.0
    rhs = np.concatenate([f, np.zeros(ncomp)])
    sol = np.linalg.solve(A, rhs)
    return sol[:n]


def elastic(phase, eig, g, eps_mac, mat, h):
    """Returns strain and stress in Voigt order (xx, yy, xy) / (xx, yy, zz, yz, xz, xy)."""
    phase = np.asarray(phase)
    shape = phase.shape
    d = phase.ndim
    N = phase.size
    ls, ms = lame(mat.E_solid, mat.nu_solid)
    lp, mp = lame(mat.E_pore, mat.nu_pore)
    lam = np.where(phase.ravel() == 1, ls, lp) * np.asarray(g).ravel()
    mu = np.where(phase.ravel() == 1, ms, mp) * np.asarray(g).ravel()
    e = np.asarray(eig, dtype=np.float64).ravel()
    B = [fwd(shape, a, h) for a in range(d)]
    delta = np.eye(d)

    def c4(i, j, k, l):
        return lam * delta[i, j] * delta[k, l] + mu * (delta[i, k] * delta[j, l] + delta[i, l] * delta[j, k])

    K = sp.lil_matrix((d * N, d * N)).tocsr()
    blocks = [[None] * d for _ in range(d)]
    for i in range(d):
        for k in range(d):
            acc = sp.csr_matrix((N, N))
            for j in range(d):
                for l in range(d):
                    c = c4(i, j, k, l)
                    if np.any(c != 0):
                        acc = acc + B[j].T @ sp.diags(c) @ B[l]
            blocks[i][k] = acc
    K = sp.bmat(blocks).tocsr()
    voigt = [(0, 0), (1, 1), (0, 1)] if d == 2 else [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    E = np.zeros((d, d))
    for I, (i, j) in enumerate(voigt):
        E[i, j] = E[j, i] = eps_mac[I]
    # sigma0 = g C : (E - e I)
    s0 = np.zeros((d, d, N))
    for i in range(d):
        for j in range(d):
            s0[i, j] = sum(c4(i, j, k, l) * (E[k, l] - e * delta[k, l]) for k in range(d) for l in range(d))
    f = np.concatenate([-sum(B[j].T @ s0[i, j] for j in range(d)) for i in range(d)])
    u = solve_with_zero_mean(K, f, d, N)
    U = u.reshape(d, N)
    F = np.zeros((d, d, N))
    for i in range(d):
        for j in range(d):
            F[i, j] = E[i, j] + B[j] @ U[i]
    eps = 0.5 * (F + F.transpose(1, 0, 2))
    sig = np.zeros((d, d, N))
    for i in range(d):
        for j in range(d):
            sig[i, j] = sum(c4(i, j, k, l) * (eps[k, l] - e * delta[k, l]) for k in range(d) for l in range(d))
    strain = np.stack([eps[i, j].reshape(shape) for (i, j) in voigt])
    stress = np.stack([sig[i, j].reshape(shape) for (i, j) in voigt])
    return {"u": U.reshape((d,) + shape), "strain": strain, "stress": stress}


def homogenise(phase, mat, grad_c_mac, c_macro, h):
    phase = np.asarray(phase)
    shape = phase.shape
    d = phase.ndim
    N = phase.size
    Dx = np.where(phase.ravel() == 1, mat.D_solid, mat.D_pore)
    B = [fwd(shape, a, h) for a in range(d)]
    K = sum(B[a].T @ sp.diags(Dx) @ B[a] for a in range(d))
    f = -sum(B[a].T @ (Dx * grad_c_mac[a]) for a in range(d))
    phi = solve_with_zero_mean(K, f, 1, N)
    gradc = np.stack([grad_c_mac[a] + B[a] @ phi for a in range(d)])
    # concentration: Eq. (concentration) with the two integration constants
    coords = np.meshgrid(*[h * np.arange(n) for n in shape], indexing="ij")
    # coords[axis]; direction alpha sits on axis d-1-alpha
    ramp = sum(grad_c_mac[a] * coords[d - 1 - a].ravel() for a in range(d))
    pore = phase.ravel() == 0
    c = ramp + phi
    eta = pore.mean()
    out = c.copy()
    if pore.any():
        out[pore] = c[pore] + c_macro / eta - c[pore].mean()
    if (~pore).any():
        out[~pore] = c[~pore] - c[~pore].mean()
    return {"phi": phi.reshape(shape), "c": out.reshape(shape), "grad_c": gradc.reshape((d,) + shape),
            "mean_flux": -(Dx[None] * gradc).mean(axis=1)}


def phasefield(H, mat, h):
    H = np.asarray(H, dtype=np.float64)
    shape = H.shape
    d = H.ndim
    a = mat.Gc / (2 * mat.l0)
    b = mat.Gc * mat.l0 / 2
    B = [fwd(shape, al, h) for al in range(d)]
    A = sp.diags(a + H.ravel()) + b * sum(Bi.T @ Bi for Bi in B)
    return np.linalg.solve(A.toarray(), H.ravel()).reshape(shape)
