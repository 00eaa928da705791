"""Seeded synthetic lattice inputs (gauge links, sources, gauge transforms).

This package is the one module that both the FP64 oracle tests and the CUDA path
draw their inputs from. It holds none of the Dirac-operator, solver or force
arithmetic; it only draws random numbers and shapes them into fields.
"""
from .generators import (  # noqa: F401
    BASE_SEED,
    config_seed,
    make_rng,
    haar_su3,
    exp_i_hermitian_su3,
    random_su3_algebra,
    gaussian_spinor,
    gauge_field,
    unit_gauge,
    lattice_volume,
    random_gauge_transform,
)
