"""Pin of the oracle's reference-medium preconditioner
(oracle.elasticity.reference_medium_preconditioner): for a homogeneous
isotropic medium it is the exact inverse of the Galerkin operator, so the
dense real-space operator K0 of tests/dense_reference.py (forward-difference
matrices, no FFT) applied to z = M r gives back r (zero-mean r) in 2D and 3D,
with lambda0 != mu0 so that swapping conj(D) D^T and D conj(D)^T, or
dropping a conjugate, fails. Also: z has zero mean, and M is symmetric
(<s, M r> = <r, M s>)."""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import elasticity
from tests.dense_reference import fwd

H = 5e-6


def dense_K0(shape, lam0, mu0, h):
    d = len(shape)
    N = int(np.prod(shape))
    B = [fwd(shape, a, h) for a in range(d)]
    delta = np.eye(d)
    blocks = [[None] * d for _ in range(d)]
    for i in range(d):
        for k in range(d):
            acc = sp.csr_matrix((N, N))
            for j in range(d):
                for l in range(d):
                    c = lam0 * delta[i, j] * delta[k, l] + mu0 * (delta[i, k] * delta[j, l] + delta[i, l] * delta[j, k])
                    if c != 0:
                        acc = acc + c * (B[j].T @ B[l])
            blocks[i][k] = acc
    return sp.bmat(blocks).tocsr()


@pytest.mark.parametrize("shape", [(6, 5), (4, 5, 3)])
def test_reference_medium_inverts_the_homogeneous_operator(shape):
    d = len(shape)
    lam0, mu0 = 0.7, 1.3
    rng = np.random.default_rng(5)
    r = rng.standard_normal((d,) + shape)
    r -= r.reshape(d, -1).mean(axis=1).reshape((d,) + (1,) * d)
    z = elasticity.reference_medium_preconditioner(r, lam0, mu0, H)
    K = dense_K0(shape, lam0, mu0, H)
    back = (K @ z.reshape(-1)).reshape(r.shape)
    assert np.abs(back - r).max() <= 1e-10 * np.abs(r).max()
    assert np.abs(z.reshape(d, -1).mean(axis=1)).max() <= 1e-12 * np.abs(z).max()
    s = rng.standard_normal((d,) + shape)
    zs = elasticity.reference_medium_preconditioner(s, lam0, mu0, H)
    assert abs(np.sum(s * z) - np.sum(r * zs)) <= 1e-10 * abs(np.sum(s * z))


MUTATIONS = {
    "conj(D) D^T and D conj(D)^T swapped": (
        "lam0 * np.outer(np.conj(a), a) + mu0 * np.outer(a, np.conj(a))",
        "lam0 * np.outer(a, np.conj(a)) + mu0 * np.outer(np.conj(a), a)"),
    "a conjugate dropped": ("np.outer(np.conj(a), a)", "np.outer(a, a)"),
}


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_planted_mistakes_fail_the_dense_pin(name):
    import os
    import types
    src = open(os.path.join(os.path.dirname(elasticity.__file__), "elasticity.py")).read()
    old, new = MUTATIONS[name]
    assert old in src
    mod = types.ModuleType("oracle.elasticity_mutant")
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new), "elasticity_mutant", "exec"), mod.__dict__)
    shape = (6, 5)
    rng = np.random.default_rng(5)
    r = rng.standard_normal((2,) + shape)
    r -= r.reshape(2, -1).mean(axis=1).reshape(2, 1, 1)
    z = mod.reference_medium_preconditioner(r, 0.7, 1.3, H)
    back = (dense_K0(shape, 0.7, 1.3, H) @ z.reshape(-1)).reshape(r.shape)
    assert np.abs(back - r).max() > 1e-3 * np.abs(r).max(), name
