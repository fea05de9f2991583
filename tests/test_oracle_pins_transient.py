"""Pins of the oracle's transient diffusion (the backward-Euler extension of
Sec. 2.1 used by the transient carpet workloads) with heterogeneous D and a
Dirichlet mask, and of the total elastic energy (the sum of 1/2 (eps - e I) :
sigma over the voxels, Sec. 2.3 / Eq. energy's companion), against statements
that do not go through the oracle's sparse B^T diag(D) B assembly:

- the finite-volume balance of every voxel, written face by face: the flux
  through the face between voxel x and x + e_a is -D(x) (c(x + e_a) - c(x)) / h
  (the forward-difference gradient of Sec. 2.6 evaluated at voxel x, with that
  voxel's diffusivity);
- a dense system assembled from those face conductances, the masked rows
  replaced by identity rows, solved by numpy.linalg.solve;
- closed forms: the steady limit dt -> inf with one Dirichlet value (c equals
  that value everywhere), the pinned-node profile on a periodic line
  c_i = (r^i + r^(n-i)) / (1 + r^n) with r + 1/r = 2 + h^2 / (D dt), and mass
  conservation without a mask;
- for the energy: the homogeneous medium under a uniform macro strain
  (1/2 lambda tr(E)^2 + mu E:E per unit volume) and the Hill-Mandel identity
  sum_x eps:sigma = V E:<sigma> for a compatible strain and an equilibrated
  stress, which gives the energy of a heterogeneous, damaged, eigenstrained
  RVE from its mean stress alone.

The last test plants mistakes in copies of the oracle functions (the
diffusivity taken from the neighbouring voxel, B D B^T instead of
B^T D B, a flipped Dirichlet elimination sign, a shear weight of 1 in the
energy) and checks that each one fails at least one of these pins.
"""

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from microstructures import sierpinski_carpet, random_carpet, random_sponge
from microstructures.workloads import Materials
from oracle import diffusion, elasticity

MAT = Materials()
H_MECH = 5e-6


# ---------------------------------------------------------------- helpers (no oracle code)

def neighbour(idx, shape, a, step):
    """Flat index of the voxel step * e_a away (periodic); a = 0 is x, the
    last (fastest) array axis."""
    coords = list(np.unravel_index(idx, shape))
    ax = len(shape) - 1 - a
    coords[ax] = (coords[ax] + step) % shape[ax]
    return int(np.ravel_multi_index(coords, shape))


def face_matrix(phase, mat, dt, h):
    """Dense (1/dt) I + sum over faces of the conductance D(x)/h^2 coupling
    voxel x and x + e_a, assembled face by face (finite-volume form)."""
    shape = phase.shape
    N = phase.size
    Dv = np.where(phase.ravel() == 1, mat.D_solid, mat.D_pore)
    A = np.eye(N) / dt
    for x in range(N):
        for a in range(phase.ndim):
            y = neighbour(x, shape, a, +1)
            k = Dv[x] / h ** 2
            A[x, x] += k
            A[y, y] += k
            A[x, y] -= k
            A[y, x] -= k
    return A


def balance_residual(phase, mat, dt, h, c_prev, c, mask=None):
    """Largest |(c - c_prev)/dt + (F_out - F_in)/h| over the free voxels,
    each face flux F = -D(x) (c(x + e_a) - c(x)) / h written out."""
    shape = phase.shape
    cf, cp = c.ravel(), c_prev.ravel()
    Dv = np.where(phase.ravel() == 1, mat.D_solid, mat.D_pore)
    worst = 0.0
    for x in range(phase.size):
        if mask is not None and mask.ravel()[x]:
            continue
        net_out = 0.0
        for a in range(phase.ndim):
            xp = neighbour(x, shape, a, +1)
            xm = neighbour(x, shape, a, -1)
            f_out = -Dv[x] * (cf[xp] - cf[x]) / h
            f_in = -Dv[xm] * (cf[x] - cf[xm]) / h
            net_out += (f_out - f_in) / h
        worst = max(worst, abs((cf[x] - cp[x]) / dt + net_out))
    return worst


def two_phase_27():
    return sierpinski_carpet(3)  # 27 x 27, pores and solid


def two_phase_456():
    rng = np.random.default_rng(11)
    return (rng.random((4, 5, 6)) < 0.6).astype(np.uint8)


def left_face_mask(shape):
    m = np.zeros(shape, np.uint8)
    m[..., 0] = 1
    return m


# ---------------------------------------------------------------- checks (return an error)

def err_matrix(matrix_fn, phase, dt, h):
    A = matrix_fn(phase, MAT, dt, h)
    A = A.toarray() if sp.issparse(A) else np.asarray(A)
    R = face_matrix(phase, MAT, dt, h)
    return np.abs(A - R).max() / np.abs(R).max()


def err_balance(step_fn, phase, dt, h, masked):
    rng = np.random.default_rng(3)
    c_prev = rng.random(phase.shape)
    mask = left_face_mask(phase.shape) if masked else None
    c = step_fn(phase, c_prev, MAT, dt, h, mask=mask, c_dirichlet=1.0)
    scale = np.abs(c_prev).max() / dt
    e = balance_residual(phase, MAT, dt, h, c_prev, c, mask) / scale
    if masked:
        e = max(e, np.abs(c[mask != 0] - 1.0).max())
    return e


def err_dirichlet_dense(step_fn, phase, dt, h):
    rng = np.random.default_rng(5)
    c_prev = rng.random(phase.shape)
    mask = left_face_mask(phase.shape)
    A = face_matrix(phase, MAT, dt, h)
    rhs = c_prev.ravel() / dt
    fixed = mask.ravel() != 0
    A[fixed, :] = 0.0
    A[fixed, fixed] = 1.0
    rhs[fixed] = 0.75
    ref = np.linalg.solve(A, rhs)
    got = step_fn(phase, c_prev, MAT, dt, h, mask=mask, c_dirichlet=0.75).ravel()
    return np.abs(got - ref).max() / np.abs(ref).max()


def err_steady_limit(step_fn, phase, h):
    rng = np.random.default_rng(7)
    c_prev = rng.random(phase.shape)
    c = step_fn(phase, c_prev, MAT, 1e14, h, mask=left_face_mask(phase.shape), c_dirichlet=1.0)
    return np.abs(c - 1.0).max()


def err_pinned_line(step_fn, n=33, Dc=0.8, dt=1.7, h=1.0):
    mat = Materials(D_solid=Dc, D_pore=Dc)
    phase = np.ones((1, n), np.uint8)
    mask = np.zeros((1, n), np.uint8)
    mask[0, 0] = 1
    c = step_fn(phase, np.zeros((1, n)), mat, dt, h, mask=mask, c_dirichlet=1.0)[0]
    s = 2.0 + h * h / (Dc * dt)
    r = (s - np.sqrt(s * s - 4.0)) / 2.0  # root of r + 1/r = s below 1
    i = np.arange(n)
    exact = (r ** i + r ** (n - i)) / (1.0 + r ** n)
    return np.abs(c - exact).max()


def err_energy_homogeneous(energy_fn, d):
    shape = (9, 9) if d == 2 else (5, 6, 7)
    nv = 3 if d == 2 else 6
    E = np.array([1.0e-3, -4.0e-4, 7.0e-4]) if d == 2 else np.array([1e-3, -4e-4, 2e-4, 3e-4, -5e-4, 6e-4])
    phase = np.ones(shape, np.uint8)
    out = elasticity.equilibrium_solve(phase, np.zeros(shape), np.ones(shape), E, MAT, H_MECH)
    lam, mu = elasticity.lame(MAT.E_solid, MAT.nu_solid)
    Et = elasticity.macro_tensor(E, d)
    w = 0.5 * lam * np.trace(Et) ** 2 + mu * np.sum(Et * Et)  # energy density, full tensor
    exact = w * phase.size * H_MECH ** d
    got = energy_fn(out["strain"], out["stress"], np.zeros(shape), H_MECH)
    assert out["strain"].shape[0] == nv
    return abs(got - exact) / exact


def err_energy_hill_mandel(energy_fn, d):
    if d == 2:
        phase, _ = random_carpet(27, 0.35, 3)
        E = np.array([2e-4, -1e-4, 3e-4])
    else:
        phase, _ = random_sponge(9, 0.3, 4)
        E = np.array([2e-4, -1e-4, 1e-4, 3e-4, -2e-4, 1.5e-4])
    rng = np.random.default_rng(9)
    eig = np.where(phase == 0, 1e-3 * (1.0 + 0.2 * rng.standard_normal(phase.shape)), 0.0)
    dmg = 0.4 * rng.random(phase.shape)
    g = (1 - dmg) ** 2 + MAT.kappa
    out = elasticity.equilibrium_solve(phase, eig, g, E, MAT, H_MECH, tol=1e-13)
    sig = out["sigma_tensor"]
    mean_sig = sig.reshape(d, d, -1).mean(axis=2)
    Et = elasticity.macro_tensor(E, d)
    tr_sig = sum(sig[i, i] for i in range(d))
    V = phase.size * H_MECH ** d
    exact = 0.5 * V * (np.sum(Et * mean_sig) - np.mean(eig * tr_sig))
    got = energy_fn(out["strain"], out["stress"], eig, H_MECH)
    return abs(got - exact) / abs(exact)


# ---------------------------------------------------------------- pins

TOL_MAT = 1e-13
TOL_BAL = 1e-10
TOL_DENSE = 1e-11
TOL_STEADY = 1e-8
TOL_LINE = 1e-13
TOL_ENERGY = 1e-9


@pytest.mark.parametrize("phase_fn,h", [(two_phase_27, 1.0), (two_phase_456, 0.8)])
def test_transient_matrix_equals_face_assembly(phase_fn, h):
    assert err_matrix(diffusion.transient_matrix, phase_fn(), 3.0, h) < TOL_MAT


@pytest.mark.parametrize("masked", [False, True])
@pytest.mark.parametrize("phase_fn,h", [(two_phase_27, 1.0), (two_phase_456, 0.8)])
def test_transient_step_satisfies_flux_balance(phase_fn, h, masked):
    assert err_balance(diffusion.transient_step, phase_fn(), 40.0, h, masked) < TOL_BAL


@pytest.mark.parametrize("phase_fn,h", [(two_phase_27, 1.0), (two_phase_456, 0.8)])
def test_transient_dirichlet_equals_identity_row_dense_solve(phase_fn, h):
    assert err_dirichlet_dense(diffusion.transient_step, phase_fn(), 25.0, h) < TOL_DENSE


@pytest.mark.parametrize("phase_fn", [two_phase_27, two_phase_456])
def test_transient_dirichlet_steady_limit(phase_fn):
    assert err_steady_limit(diffusion.transient_step, phase_fn(), 1.0) < TOL_STEADY


def test_transient_pinned_node_line_closed_form():
    assert err_pinned_line(diffusion.transient_step) < TOL_LINE


def test_transient_conserves_mass_without_mask():
    phase = two_phase_27()
    c_prev = np.random.default_rng(2).random(phase.shape)
    c = diffusion.transient_step(phase, c_prev, MAT, 13.0, 1.0)
    assert abs(c.sum() - c_prev.sum()) < 1e-11 * c_prev.sum()


@pytest.mark.parametrize("d", [2, 3])
def test_elastic_energy_homogeneous_closed_form(d):
    assert err_energy_homogeneous(elasticity.elastic_energy, d) < TOL_ENERGY


@pytest.mark.parametrize("d", [2, 3])
def test_elastic_energy_hill_mandel(d):
    assert err_energy_hill_mandel(elasticity.elastic_energy, d) < TOL_ENERGY


# ---------------------------------------------------------------- planted mistakes

def _matrix_neighbour_D(phase, mat, dt, h):
    """Mistake: the flux through the face x -> x + e_a uses D(x + e_a)."""
    shape = phase.shape
    N = phase.size
    A = sp.identity(N, format="csr") * (1.0 / dt)
    for a in range(phase.ndim):
        B = diffusion.forward_difference_matrix(shape, a, h)
        Dn = np.roll(diffusion.diffusivity(phase, mat), -1, axis=phase.ndim - 1 - a).ravel()
        A = A + B.T @ sp.diags(Dn) @ B
    return A.tocsc()


def _matrix_transposed(phase, mat, dt, h):
    """Mistake: B diag(D) B^T instead of B^T diag(D) B."""
    N = phase.size
    Dx = sp.diags(diffusion.diffusivity(phase, mat).ravel())
    A = sp.identity(N, format="csr") * (1.0 / dt)
    for a in range(phase.ndim):
        B = diffusion.forward_difference_matrix(phase.shape, a, h)
        A = A + B @ Dx @ B.T
    return A.tocsc()


def _step_with(matrix_fn, dirichlet_sign=-1.0):
    def step(phase, c_prev, mat, dt, h, mask=None, c_dirichlet=1.0):
        A = matrix_fn(phase, mat, dt, h)
        b = np.asarray(c_prev, dtype=np.float64).ravel() / dt
        if mask is None:
            return spla.spsolve(A, b).reshape(phase.shape)
        fixed = np.asarray(mask).ravel() != 0
        free = ~fixed
        cD = np.zeros(phase.size)
        cD[fixed] = c_dirichlet
        rhs = b[free] + dirichlet_sign * (A[free][:, fixed] @ cD[fixed])
        c = cD.copy()
        c[free] = spla.spsolve(A[free][:, free].tocsc(), rhs)
        return c.reshape(phase.shape)
    return step


def _energy_shear_weight_one(strain, stress, eig, h):
    s, t = np.asarray(strain), np.asarray(stress)
    d = 2 if s.shape[0] == 3 else 3
    tot = 0.0
    for I, (i, j) in enumerate(elasticity.VOIGT[d]):
        el = s[I] - (eig if i == j else 0.0)
        tot += float(np.sum(el * t[I]))
    return 0.5 * tot * h ** d


def _transient_pins_fail(matrix_fn, step_fn):
    errs = [
        err_matrix(matrix_fn, two_phase_27(), 3.0, 1.0) / TOL_MAT,
        err_balance(step_fn, two_phase_27(), 40.0, 1.0, True) / TOL_BAL,
        err_balance(step_fn, two_phase_456(), 40.0, 0.8, False) / TOL_BAL,
        err_dirichlet_dense(step_fn, two_phase_456(), 25.0, 0.8) / TOL_DENSE,
        err_steady_limit(step_fn, two_phase_27(), 1.0) / TOL_STEADY,
        err_pinned_line(step_fn) / TOL_LINE,
    ]
    return max(errs) > 1.0


def test_planted_mistakes_fail_the_pins():
    # the oracle itself passes
    assert not _transient_pins_fail(diffusion.transient_matrix, diffusion.transient_step)
    # diffusivity of the neighbouring voxel
    assert _transient_pins_fail(_matrix_neighbour_D, _step_with(_matrix_neighbour_D))
    # transposed operator
    assert _transient_pins_fail(_matrix_transposed, _step_with(_matrix_transposed))
    # flipped sign of the Dirichlet elimination
    assert _transient_pins_fail(diffusion.transient_matrix,
                                _step_with(diffusion.transient_matrix, dirichlet_sign=+1.0))
    # shear counted once in the energy
    assert max(err_energy_homogeneous(_energy_shear_weight_one, 2),
               err_energy_hill_mandel(_energy_shear_weight_one, 3)) > TOL_ENERGY
