"""Precipitation of corrosion products and pore pressurisation (Sec. 2.2).

Precipitate concentration: the ferrous-ion concentration above the
solubility limit S(pH) precipitates (Sec. 3): c_ppt = (c - S)_+ in the pores,
0 in the solid (precipitates grow in the pores only, Sec. 2.2).

Isotropic eigenstrain from the precipitate's expansion (Eq. eigen-simplify):
eps_eig = (c_ppt M_ppt - 1)_+ I, Macaulay bracket, applied in the pores only.
"""

import numpy as np


def macaulay(x):
    """(x)_+ = x if x > 0 else 0 (Eq. eigen)."""
    return np.where(x > 0, x, 0.0)


def precipitate(c, phase, S):
    return np.where(np.asarray(phase) == 0, macaulay(np.asarray(c) - S), 0.0)


def eigenstrain(c_ppt, phase, M):
    """Scalar e(x) with eps_eig = e I (Eq. eigen-simplify)."""
    return np.where(np.asarray(phase) == 0, macaulay(np.asarray(c_ppt) * M - 1.0), 0.0)
