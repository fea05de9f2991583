"""fftmech_fft_noalloc, the allocation-free transform, against fftmech_fft.

Some callers must not allocate device memory: code that runs while other
streams must keep running (cudaMalloc / cudaFree can synchronise the device),
code whose device memory belongs to another allocator or a fixed budget, or
code that must not hit an out-of-memory error in mid-run. For them the
library's FFT has a variant whose twiddle tables live in a fixed device array
inside the library instead of being allocated per call. This file checks,
through the C ABI, that the variant gives the same transform as fftmech_fft
(the FFT tests' tolerances) on two calls in a row, in both precisions and
both directions, and that sizes beyond the array are rejected up front.
"""

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


def _pair(shape, precision, inverse, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    dt = torch.complex128 if precision == fm.FFTMECH_FP64 else torch.complex64
    a = torch.tensor(x, dtype=dt, device="cuda")
    b = a.clone()
    ndim = 1 if shape[0] == 1 else 2
    n = [shape[1], shape[0]]
    fm.fftmech_fft(ndim, n, precision, inverse, a)
    fm.fftmech_fft_noalloc(ndim, n, precision, inverse, b)
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.abs(b - a).max() / np.abs(a).max()


@pytest.mark.parametrize("precision", [fm.FFTMECH_FP64, fm.FFTMECH_MIXED])
def test_noalloc_matches_fft_on_two_calls_in_a_row(precision):
    tol = 1e-13 if precision == fm.FFTMECH_FP64 else 2e-6
    # two consecutive calls with different sizes and directions: the second
    # call must not see stale twiddles of the first
    assert _pair((81, 729), precision, 0, 1) < tol
    assert _pair((128, 27), precision, 1, 2) < tol
    assert _pair((1, 2187), precision, 0, 3) < tol


@pytest.mark.parametrize("precision", [fm.FFTMECH_FP64, fm.FFTMECH_MIXED])
def test_noalloc_largest_plans_in_both_directions(precision):
    """The array's largest plan (2187 points) as the column and as the row
    transform, and a power of two near the limit (2048, so the slot is used
    up to its last pass multipliers), each against fftmech_fft."""
    tol = 1e-13 if precision == fm.FFTMECH_FP64 else 2e-6
    assert _pair((2187, 81), precision, 0, 4) < tol
    assert _pair((81, 2187), precision, 1, 5) < tol
    assert _pair((8, 2048), precision, 0, 6) < tol
    assert _pair((2048, 8), precision, 1, 7) < tol


def test_noalloc_rejects_sizes_beyond_its_array():
    t = torch.zeros((2, 4096), dtype=torch.complex128, device="cuda")
    with pytest.raises(fm.FftmechError) as ei:
        fm.fftmech_fft_noalloc(2, [4096, 2], fm.FFTMECH_FP64, 0, t)
    assert ei.value.status == fm.FFTMECH_ERR_UNSUPPORTED_SIZE
    assert torch.count_nonzero(t).item() == 0  # rejected before any work
