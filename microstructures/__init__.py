"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This package holds input recipes only: the counter-based random generator,
the fractal pore geometries (phase indicator omega, 1 = solid, 0 = pore) and
the workload descriptions (materials, loads, seeds). It holds none of the
method's arithmetic: no operator, projection, solver or constitutive law. The
CPU oracle and the CUDA library each derive what they need (Lame constants,
symbols, stencils) from these raw inputs on their own.
"""

from .splitmix import splitmix64_stream, uniform01, standard_normal
from .fractals import (
    sierpinski_carpet,
    random_carpet,
    random_sponge,
    porosity,
)
from . import workloads

__all__ = [
    "splitmix64_stream",
    "uniform01",
    "standard_normal",
    "sierpinski_carpet",
    "random_carpet",
    "random_sponge",
    "porosity",
    "workloads",
]
