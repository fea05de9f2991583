"""GPU Stockham FFT (the transform every solve uses) against numpy's FFT."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2305_13081_gb300 import build
from paper_2305_13081_gb300 import fftmech as fm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    fm.load_library()


SHAPES = [(1, 9), (1, 2187), (27, 9), (81, 81), (243, 81), (729, 729), (9, 1024), (64, 128),
          (12, 96), (6, 18), (2187, 27), (128, 256)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("precision", [fm.FFTMECH_FP64, fm.FFTMECH_MIXED])
@pytest.mark.parametrize("inverse", [0, 1])
def test_fft_matches_numpy(shape, precision, inverse):
    rng = np.random.default_rng(hash((shape, precision, inverse)) % 2**32)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = (np.fft.ifft2(x) * x.size) if inverse else np.fft.fft2(x)
    if shape[0] == 1:
        ref = (np.fft.ifft(x[0]) * x.shape[1] if inverse else np.fft.fft(x[0]))[None]
    dt = torch.complex128 if precision == fm.FFTMECH_FP64 else torch.complex64
    t = torch.tensor(x, dtype=dt, device="cuda")
    ndim = 1 if shape[0] == 1 else 2
    fm.fftmech_fft(ndim, [shape[1], shape[0]], precision, inverse, t)
    got = t.cpu().numpy()
    err = np.abs(got - ref).max() / np.abs(ref).max()
    tol = 1e-13 if precision == fm.FFTMECH_FP64 else 2e-6
    assert err < tol, err


def test_fft_rejects_host_pointer_and_bad_size():
    x = np.zeros((9, 9), dtype=np.complex128)
    with pytest.raises(fm.FftmechError):
        fm.fftmech_fft(2, [9, 9], fm.FFTMECH_FP64, 0, x)
    t = torch.zeros((5, 10), dtype=torch.complex128, device="cuda")
    with pytest.raises(fm.FftmechError):
        fm.fftmech_fft(2, [10, 5], fm.FFTMECH_FP64, 0, t)


SHAPES3 = [(9, 27, 81), (27, 27, 27), (16, 12, 8), (81, 9, 243), (4, 6, 2187)]


@pytest.mark.parametrize("shape", SHAPES3)
@pytest.mark.parametrize("precision", [fm.FFTMECH_FP64, fm.FFTMECH_MIXED])
@pytest.mark.parametrize("inverse", [0, 1])
def test_fft3d_matches_numpy(shape, precision, inverse):
    """3D transform (x lines, y columns of every plane, z columns) against
    numpy.fft.fftn / ifftn, called twice on the same length set so that the
    second call uses the cached plans."""
    rng = np.random.default_rng(sum(shape) + 7 * precision + inverse)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = (np.fft.ifftn(x) * x.size) if inverse else np.fft.fftn(x)
    dt = torch.complex128 if precision == fm.FFTMECH_FP64 else torch.complex64
    tol = 1e-13 if precision == fm.FFTMECH_FP64 else 3e-6
    for _ in range(2):
        t = torch.tensor(x, dtype=dt, device="cuda")
        fm.fftmech_fft(3, [shape[2], shape[1], shape[0]], precision, inverse, t)
        got = t.cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < tol, err
