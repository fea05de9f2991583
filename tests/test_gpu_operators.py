"""Gradient-operator variants of the homogenised diffusion
(fftmech_homogenise_operator, Sec. 2.6 and Fig. 2) through the C ABI:

- every operator (forward, central, 8th-order central, Fourier) against
  the FP64 oracle with the same symbol (oracle/diffusion.homogenise(symbol=))
  on a 2D random carpet and a 3D random sponge (odd sizes): phi and grad c
  within 1e-9 relative, the mean flux within 1e-10;
- the forward operator, solved by this spectral-operator PCG, agrees with
  the library's stencil-based HOMOGENISE diffusion (fftmech_diffusion_step):
  two independent GPU paths, one mean flux;
- laminates: every operator gives the harmonic mean of D across layers
  normal to the gradient and the arithmetic mean along them.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from microstructures import random_carpet, random_sponge
from microstructures.workloads import Materials
from oracle import diffusion
from paper_2305_13081_gb300 import build
from paper_2305_13081_gb300 import fftmech as fm

pytestmark = pytest.mark.gpu

MAT = Materials()
OPS = {"forward": fm.FFTMECH_GRAD_FORWARD, "central": fm.FFTMECH_GRAD_CENTRAL,
       "central8": fm.FFTMECH_GRAD_CENTRAL8, "fourier": fm.FFTMECH_GRAD_FOURIER}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    fm.load_library()


def gpu(phase, op, G, tol=1e-13):
    ctx = fm.Context(phase.shape, MAT, fm.FFTMECH_FP64, h_diff=1.0, tol=tol, max_iter=20000)
    N = phase.size
    d = phase.ndim
    ph = torch.as_tensor(phase.ravel()).cuda()
    phi = torch.zeros(N, dtype=torch.float64, device="cuda")
    gc = torch.zeros(d * N, dtype=torch.float64, device="cuda")
    info = fm.fftmech_homogenise_operator(ctx.handle, ph, OPS[op], G, phi, gc)
    ctx.close()
    return info, phi.cpu().numpy().reshape(phase.shape), gc.cpu().numpy().reshape((d,) + phase.shape)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("op", list(OPS))
@pytest.mark.parametrize("dim", [2, 3])
def test_operator_matches_oracle(op, dim):
    if dim == 2:
        phase = random_carpet(81, 0.30, 11)[0]
        G = [1.0, 0.5]
    else:
        phase = random_sponge(9, 0.35, 12)[0]
        G = [1.0, 0.5, -0.25]
    info, phi, gc = gpu(phase, op, G)
    ref = diffusion.homogenise(phase, MAT, G, 0.0, 1.0, tol=1e-13, symbol=op)
    e_phi, e_gc = rel(phi, ref["phi"]), rel(gc, ref["grad_c"])
    e_j = float(np.abs(np.array(info.mean_flux[:dim]) - ref["mean_flux"]).max() / np.abs(ref["mean_flux"]).max())
    print("operator", op, dim, "iterations", info.iters, "phi", e_phi, "grad c", e_gc, "mean flux", e_j)
    assert info.status == fm.FFTMECH_OK
    assert e_phi < 1e-9 and e_gc < 1e-9 and e_j < 1e-10


def test_forward_operator_agrees_with_the_stencil_path():
    phase = random_carpet(243, 0.30, 13)[0]
    G = [1.0, 0.0]
    info, _, _ = gpu(phase, "forward", G, tol=1e-12)
    ctx = fm.Context(phase.shape, MAT, fm.FFTMECH_FP64, h_diff=1.0, tol=1e-12, max_iter=20000)
    ph = torch.as_tensor(phase.ravel()).cuda()
    c = torch.zeros(phase.size, dtype=torch.float64, device="cuda")
    ref = fm.fftmech_diffusion_step(ctx.handle, ph, fm.FFTMECH_DIFF_HOMOGENISE, G, 0.3, 0.0, None, 0.0, c)
    ctx.close()
    a, b = np.array(info.mean_flux[:2]), np.array(ref.mean_flux[:2])
    assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max(), (a, b)


@pytest.mark.parametrize("op", list(OPS))
def test_laminates(op):
    n = 27
    normal = np.zeros((9, n), dtype=np.uint8)
    normal[:, 13:] = 1
    parallel = np.zeros((n, 9), dtype=np.uint8)
    parallel[13:, :] = 1
    D_n = np.where(normal[0] == 0, MAT.D_pore, MAT.D_solid)
    D_p = np.where(parallel[:, 0] == 0, MAT.D_pore, MAT.D_solid)
    i_n, _, _ = gpu(normal, op, [1.0, 0.0])
    i_p, _, _ = gpu(parallel, op, [1.0, 0.0])
    h = 1.0 / np.mean(1.0 / D_n)
    a = np.mean(D_p)
    assert abs(i_n.mean_flux[0] + h) <= 1e-9 * h and abs(i_p.mean_flux[0] + a) <= 1e-9 * a
