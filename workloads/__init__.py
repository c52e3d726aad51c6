"""Seeded synthetic workloads for the non-conforming DG atmosphere solver.

This package only *describes* inputs: base grids, per-cell refinement levels,
terrain, atmosphere and perturbation parameters, time-step sizes and seeded
random numbers.  It contains none of the discretisation's arithmetic (no
basis, quadrature, geometry map, flux or time-integration formula), so that
both the CUDA library and the independent CPU oracle can consume the same
case description without sharing any numerical code.
"""

from .cases import (  # noqa: F401
    Case,
    CONFIGS,
    make_case,
    tiny_case,
    noise,
    smooth_modes,
    GAMMA,
    R_GAS,
    GRAV,
)
