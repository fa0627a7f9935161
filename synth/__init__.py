"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only draws random numbers and builds grid topologies and
parameters; it holds none of the interior-point or KKT arithmetic.  Both the
CPU oracle and the CUDA path consume what it produces.
"""
from .grid import (Grid, make_grid, ring_grid, planar_grid, scale_loads, mixed_grid, batch_grids,
                   kkt_point, CONFIGS, config_grid, recipe_grid, recipe_batch)

__all__ = ["Grid", "make_grid", "ring_grid", "planar_grid", "scale_loads", "mixed_grid", "batch_grids",
           "kkt_point", "CONFIGS", "config_grid", "recipe_grid", "recipe_batch"]
