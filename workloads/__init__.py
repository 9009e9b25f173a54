"""Seeded synthetic plasmas shaped like the paper's runs (Sect. 4).

This module is shared by the CUDA path's tests/benchmark and by the FP64
oracle's tests.  It only draws initial conditions (positions, four-velocities,
initial fields); it contains none of the PIC step's arithmetic (no gather,
push, deposit, filter or field update).
"""
from .plasma import (  # noqa: F401
    Plasma,
    Species,
    mj_mean_gamma,
    charge_from_skin_depth,
    sample_mj_momenta,
    boost_flip,
    uniform_plasma,
    weibel_1d,
    turbulence_2d,
    shock_3d,
    shock_tube,
    injected_count,
    weibel_box,
    magnetic_modes,
    adjoint_box,
    weibel_ensemble,
    CONFIGS,
)
