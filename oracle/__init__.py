"""Plain FP64 CPU oracle for the FFT-Galerkin corrosion-fracture hot path
(Pundir, Kammer & Angst, "An FFT-based framework for predicting
corrosion-driven damage in fractal porous media", arXiv 2305.13081).

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import this package. The CUDA library never
calls it and shares no code with it; the two meet only in the seeded input
generators of the `microstructures` package.

It follows the paper's literal form: the unknowns are gradient fields (the
concentration gradient, the displacement gradient), the compatibility
projections G and GG are built per Fourier mode from Eq. (g-42) of App. A with
the forward-difference gradient symbol of Sec. 2.6, the linear systems are
solved by a hand-written conjugate gradient in that gradient space
(Algorithm 1), and the staggered step runs in Algorithm 1's order.

Module map
- spectral:   gradient symbols, G and GG projections (App. A, Sec. 2.6)
- krylov:     plain conjugate gradient (Algorithm 1's linear iterative solver)
- elasticity: plane-strain / 3D isotropic law, equilibrium Newton + CG
              (Sec. 2.3, Eqs. solid, solid-final), psi+ (Eq. energy)
- diffusion:  homogenised diffusion (Eqs. diffusion, diffusion-final),
              fluctuation phi (Eq. phi-fft), concentration (Eqs.
              psi-two-values, concentration-correct); transient backward-Euler
              extension (not in the paper) by a sparse direct solve
- phasefield: history field and AT2 hybrid phase field (Eqs. crack,
              crack-fft), degradation (Sec. 2.4)
- chemistry:  precipitation and eigenstrain (Sec. 2.2, Eqs. eigen,
              eigen-simplify)
- staggered:  one staggered load step (Sec. 2.5, Algorithm 1)

Every function here is pinned by a `-m "not gpu"` test against closed forms,
invariants, brute-force dense solves or textbook special cases (tests/
test_oracle_*.py).
"""

from . import spectral, krylov, elasticity, diffusion, phasefield, chemistry, staggered

__all__ = ["spectral", "krylov", "elasticity", "diffusion", "phasefield", "chemistry", "staggered"]
