"""GB300-native FFT-Galerkin corrosion-fracture hot path (arXiv 2305.13081).

The product is the CUDA library libfftmech.so (C ABI in include/fftmech.h,
sources in csrc/); `fftmech` is its ctypes binding with the same names.
"""

from . import fftmech  # noqa: F401
from .fftmech import (  # noqa: F401
    Context,
    FftmechError,
    load_library,
    fftmech_create,
    fftmech_destroy,
    fftmech_set_solver_opts,
    fftmech_diffusion_step,
    fftmech_equilibrium_solve,
    fftmech_phasefield_solve,
    fftmech_staggered_step,
    fftmech_fft,
    fftmech_status_string,
    fftmech_last_error,
)
