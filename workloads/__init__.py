"""Seeded synthetic OT problems shared by the oracle, the tests and the benchmark.

This package only draws inputs (points, grids, marginals, cost matrices).  It
holds none of the solver's arithmetic, so both the CPU oracle and the CUDA
path can consume the same bytes without sharing any method code.
"""

from .generators import (  # noqa: F401
    OTProblem,
    uniform_points_problem,
    gmm_points_problem,
    grid_problem,
    grid_marginals,
    batched_problems,
    batched_points,
    warmstart_gmm_problem,
    warmstart_init_params,
    WARMSTART_SHAPES,
    random_marginal,
    sq_euclidean_cost,
    grid_sq_cost,
    square_index_cost,
    paper_synthetic_problem,
    sphere_problem,
    workload,
)
