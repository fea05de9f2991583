"""Pins of the gradient-operator symbols of Sec. 2.6 (oracle/spectral.py) and
of the oracle's homogenised diffusion with each of them
(oracle/diffusion.homogenise(symbol=...)):

- each symbol acts in real space as its stencil (np.roll): forward
  (u(x+h) - u(x))/h, central (u(x+h) - u(x-h))/(2h), 8th-order central
  sum_m c_m (u(x+mh) - u(x-mh))/h; the Fourier symbol differentiates a
  resolved sine exactly;
- the 8th-order coefficients: the textbook values 4/5, -1/5, 4/105, -1/280,
  and eighth-order convergence on a smooth periodic function;
- homogenisation of laminates (odd grids): every symbol gives the harmonic
  mean of D for layers normal to the gradient and the arithmetic mean for
  layers parallel to it (the flux of a 1D layered problem is constant);
- the oracle's phase field with each symbol
  (oracle/phasefield.phasefield_solve(symbol=...)) against a dense direct
  solve of (a + H) d + b G^T G d = H, G the operator's stencil matrix (the
  Fourier operator from the explicit DFT matrix);
- oracle/krylov.gmres (restarted, right-preconditioned) against a direct
  solve of a non-symmetric system; the literal reading of the printed
  phase-field Laplacian (sum_alpha D_alpha^2, non-symmetric for the forward
  difference) solved by it against the dense matrix diag(a + H) - b sum
  G_alpha G_alpha;
- the oracle's equilibrium with each symbol
  (oracle/elasticity.equilibrium_solve(symbol=...)) on a laminate normal to
  x under E_yy (plane strain): eps_yy = E_yy everywhere and a uniform
  sigma_xx = <lam / M> / <1 / M> E_yy, M = lam + 2 mu (the closed form of a
  1D layered problem); a homogeneous medium takes sigma = C : E exactly.
"""

import numpy as np
import pytest

from microstructures.workloads import Materials
from oracle import diffusion, spectral

H = 0.7


def apply(D, u):
    return np.fft.ifftn(D * np.fft.fftn(u)).real


def test_symbols_act_as_their_stencils():
    rng = np.random.default_rng(1)
    u = rng.standard_normal((9, 11))
    ax = 1  # x
    fwd = (np.roll(u, -1, ax) - u) / H
    cen = (np.roll(u, -1, ax) - np.roll(u, 1, ax)) / (2 * H)
    c = spectral.central8_coefficients()
    c8 = sum(c[m - 1] * (np.roll(u, -m, ax) - np.roll(u, m, ax)) for m in range(1, 5)) / H
    assert np.abs(apply(spectral.forward_difference_symbol(u.shape, H)[0], u) - fwd).max() < 1e-12
    assert np.abs(apply(spectral.central_difference_symbol(u.shape, H)[0], u) - cen).max() < 1e-12
    assert np.abs(apply(spectral.central8_symbol(u.shape, H)[0], u) - c8).max() < 1e-12
    # y direction of the central symbol
    ceny = (np.roll(u, -1, 0) - np.roll(u, 1, 0)) / (2 * H)
    assert np.abs(apply(spectral.central_difference_symbol(u.shape, H)[1], u) - ceny).max() < 1e-12


def test_fourier_symbol_differentiates_a_sine_exactly():
    n = 15
    x = H * np.arange(n)
    L = n * H
    u = np.tile(np.sin(2 * np.pi * 3 * x / L), (5, 1))
    du = np.tile(2 * np.pi * 3 / L * np.cos(2 * np.pi * 3 * x / L), (5, 1))
    assert np.abs(apply(spectral.fourier_symbol(u.shape, H)[0], u) - du).max() < 1e-12


def test_central8_coefficients_and_order():
    c = spectral.central8_coefficients()
    assert np.allclose(c, [4 / 5, -1 / 5, 4 / 105, -1 / 280], rtol=1e-13)
    errs = []
    for n in (32, 64):
        h = 2 * np.pi / n
        x = h * np.arange(n)
        u = np.exp(np.sin(x)).reshape(1, n)
        du = (np.cos(x) * np.exp(np.sin(x))).reshape(1, n)
        errs.append(np.abs(apply(spectral.central8_symbol(u.shape, h)[0], u) - du).max())
    rate = np.log2(errs[0] / errs[1])
    assert rate > 7.5, (errs, rate)


@pytest.mark.parametrize("symbol", ["forward", "central", "central8", "fourier"])
def test_laminates_give_harmonic_and_arithmetic_means(symbol):
    mat = Materials()
    n = 27
    normal = np.zeros((9, n), dtype=np.uint8)
    normal[:, 13:] = 1  # the phase varies along x
    parallel = np.zeros((n, 9), dtype=np.uint8)
    parallel[13:, :] = 1  # varies along y
    D_n = np.where(normal[0] == 0, mat.D_pore, mat.D_solid)
    D_p = np.where(parallel[:, 0] == 0, mat.D_pore, mat.D_solid)
    out_n = diffusion.homogenise(normal, mat, [1.0, 0.0], 0.3, 1.0, tol=1e-13, symbol=symbol)
    out_p = diffusion.homogenise(parallel, mat, [1.0, 0.0], 0.3, 1.0, tol=1e-13, symbol=symbol)
    assert abs(out_n["mean_flux"][0] + 1.0 / np.mean(1.0 / D_n)) <= 1e-9 / np.mean(1.0 / D_n)
    assert abs(out_p["mean_flux"][0] + np.mean(D_p)) <= 1e-9 * np.mean(D_p)


@pytest.mark.parametrize("symbol", ["forward", "central", "central8", "fourier"])
def test_elastic_laminate_and_homogeneous_medium(symbol):
    from oracle import elasticity
    mat = Materials()
    n = 27
    phase = np.zeros((9, n), dtype=np.uint8)
    phase[:, 13:] = 1
    Eyy = 1e-3
    out = elasticity.equilibrium_solve(phase, np.zeros(phase.shape), np.ones(phase.shape), [0.0, Eyy, 0.0], mat,
                                       H, tol=1e-13, symbol=symbol)
    ls, ms = elasticity.lame(mat.E_solid, mat.nu_solid)
    lp, mp = elasticity.lame(mat.E_pore, mat.nu_pore)
    lam = np.where(phase[0] == 1, ls, lp)
    M = lam + 2 * np.where(phase[0] == 1, ms, mp)
    sxx = np.mean(lam / M) / np.mean(1.0 / M) * Eyy
    assert np.abs(out["strain"][1] - Eyy).max() <= 1e-12 * Eyy
    assert np.abs(out["stress"][0] - sxx).max() <= 1e-9 * abs(sxx)
    solid = np.ones((9, 9), dtype=np.uint8)
    E = [1e-3, -2e-4, 3e-4]
    hom = elasticity.equilibrium_solve(solid, np.zeros(solid.shape), np.ones(solid.shape), E, mat, H, tol=1e-13,
                                       symbol=symbol)
    tr = E[0] + E[1]
    expect = [ls * tr + 2 * ms * E[0], ls * tr + 2 * ms * E[1], 2 * ms * E[2]]
    for v in range(3):
        assert np.abs(hom["stress"][v] - expect[v]).max() <= 1e-12 * abs(expect[0])


def stencil_matrix(shape, axis, symbol, h):
    """Dense periodic matrix of the gradient operator along `axis`, built
    from its stencil (Fourier: from the explicit DFT matrix), independent
    of the FFT-based symbols."""
    n = shape[axis]
    if symbol == "fourier":
        j = np.arange(n)
        F = np.exp(-2j * np.pi * np.outer(j, j) / n)
        k = np.where(j <= n // 2, j, j - n)
        M1 = np.real(np.conj(F).T @ np.diag(2j * np.pi * k / (n * h)) @ F / n)
    else:
        if symbol == "forward":
            coef = {1: 1.0, 0: -1.0}
        elif symbol == "central":
            coef = {1: 0.5, -1: -0.5}
        else:
            coef = {}
            for m, c in enumerate(spectral.central8_coefficients(), start=1):
                coef[m], coef[-m] = c, -c
        M1 = np.zeros((n, n))
        for i in range(n):
            for off, c in coef.items():
                M1[i, (i + off) % n] += c / h
    mats = [np.eye(s) for s in shape]
    mats[axis] = M1
    M = mats[0]
    for m in mats[1:]:
        M = np.kron(M, m)
    return M


@pytest.mark.parametrize("symbol", ["forward", "central", "central8", "fourier"])
def test_phasefield_with_each_symbol_matches_a_dense_solve(symbol):
    """(a + H) d + b G^T G d = H with G the operator's dense stencil matrix,
    solved directly, against oracle/phasefield.phasefield_solve(symbol=)."""
    from oracle import phasefield
    mat = Materials()
    shape = (5, 7)
    h = mat.l0 / 2  # the gradient term b |D|^2 ~ 4 a: a dropped or wrong term shows
    rng = np.random.default_rng(9)
    a, b = phasefield.coefficients(mat)
    Hf = a * rng.random(shape)
    A = np.diag(a + Hf.ravel())
    for ax in range(2):
        G = stencil_matrix(shape, ax, symbol, h)
        A = A + b * G.T @ G
    ref = np.linalg.solve(A, Hf.ravel()).reshape(shape)
    d, _ = phasefield.phasefield_solve(Hf, mat, h, tol=1e-14, symbol=symbol)
    assert np.abs(d - ref).max() <= 1e-10 * np.abs(ref).max()
    lapless = np.linalg.solve(np.diag(a + Hf.ravel()), Hf.ravel()).reshape(shape)
    assert np.abs(lapless - ref).max() > 1e-2 * np.abs(ref).max()  # the gradient term matters here


def test_gmres_solves_a_nonsymmetric_system():
    """oracle/krylov.gmres against numpy.linalg.solve on a random
    non-symmetric, well-conditioned system, with and without a right
    preconditioner, across restarts."""
    from oracle.krylov import gmres
    rng = np.random.default_rng(11)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    ref = np.linalg.solve(A, b)
    x, info = gmres(lambda v: A @ v, b, tol=1e-13, restart=7)
    assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max() and info["iters"] > 7
    d = 1.0 / np.diag(A)
    x2, _ = gmres(lambda v: A @ v, b, tol=1e-13, restart=10, apply_M=lambda v: d * v)
    assert np.abs(x2 - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("symbol", ["forward", "central"])
def test_literal_phasefield_laplacian_matches_a_dense_solve(symbol):
    """The printed "i xi . i xi" read literally as sum_alpha D_alpha^2: the
    dense matrix is diag(a + H) - b sum_alpha G_alpha G_alpha (not G^T G),
    non-symmetric for the forward difference; the oracle's GMRES solve
    matches its direct solution, and the literal and Galerkin readings
    differ where the gradient term matters."""
    from oracle import phasefield
    mat = Materials()
    shape = (5, 7)
    h = mat.l0 / 2
    rng = np.random.default_rng(12)
    a, b = phasefield.coefficients(mat)
    Hf = a * rng.random(shape)
    L = sum(stencil_matrix(shape, ax, symbol, h) @ stencil_matrix(shape, ax, symbol, h) for ax in range(2))
    A = np.diag(a + Hf.ravel()) - b * L
    if symbol == "forward":
        assert np.abs(A - A.T).max() > 1e-3 * np.abs(A).max()
    ref = np.linalg.solve(A, Hf.ravel()).reshape(shape)
    d, info = phasefield.phasefield_solve(Hf, mat, h, tol=1e-14, symbol=symbol, literal=True)
    assert np.abs(d - ref).max() <= 1e-10 * np.abs(ref).max(), info
    gal, _ = phasefield.phasefield_solve(Hf, mat, h, tol=1e-14, symbol=symbol)
    if symbol == "forward":
        assert np.abs(gal - ref).max() > 1e-3 * np.abs(ref).max()


def test_literal_laplacian_is_indefinite_at_the_papers_length_scale():
    """The literal mode symbol a + H - b sum_a D_a^2 of the forward
    difference has real part a + H + 4 b / h^2 sum_a sin^2(theta_a / 2)
    cos(theta_a): at the Nyquist corner a + H - 4 d b / h^2. With the
    paper's l0 = 2 h (b / h^2 = 4 a) that is negative for every H <= a,
    so the literal operator is indefinite there; at h = 4 l0 (b / h^2 =
    a / 16) every mode has a positive real part."""
    from oracle import phasefield
    mat = Materials()
    a, b = phasefield.coefficients(mat)
    for h, sign in ((mat.l0 / 2, -1), (4 * mat.l0, 1)):
        D = spectral.forward_difference_symbol((8, 8), h)
        sym = a + a - b * sum(Da * Da for Da in D)  # H = a, the largest history of the tests
        worst = sym.real.min()
        assert np.sign(worst) == sign, (h, worst)
