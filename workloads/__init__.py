"""Seeded synthetic inputs for the Method of Averaged Marginals.

This package only draws images and maps pixels to coordinates.  It holds none
of the method's arithmetic (no pruning, no cost, no projection), so that the
FP64 oracle and the CUDA path can both consume its output without sharing any
computation.
"""
from .generators import (  # noqa: F401
    Problem,
    grid_points,
    problem_from_images,
    tiny_problem,
    config1,
    config2,
    config3,
    config4,
    config5,
    config2_free_support,
    free_support_grid,
    CONFIGS,
)
