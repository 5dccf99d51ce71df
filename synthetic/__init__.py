"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package only draws numbers: material density fields sampled at the nodal
points of a periodic grid, macroscopic load cases, and random vectors. It holds
none of the solver's arithmetic (no stiffness, no Green operator, no CG), so the
oracle and the CUDA path can both consume its output without sharing method code.
"""

from .fields import (  # noqa: F401
    smooth_density,
    smooth_density_device,
    laminate_density,
    cosine_density,
    random_field,
    mandel_unit_loads,
    mandel_dim,
    circular_inclusion,
    gaussian_filter,
)
