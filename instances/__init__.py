"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only *generates* agent MDPs, task DFAs, weight vectors and
threshold points.  It contains none of the method's arithmetic (no product
construction, no value iteration, no assignment, no projection), so the
oracle and the CUDA engine can both consume its output without sharing any
solver code.

All randomness comes from numpy's Philox counter-based generator, keyed by an
explicit seed, so every instance is reproducible on any machine.
"""

from .gen import (  # noqa: F401
    Agent,
    Task,
    Instance,
    grid_agent,
    moore_agent,
    sequence_task,
    fig2_agent,
    fig2_task,
    corridor_agent,
    chain_agent,
    tie_drift_agent,
    random_tiny_agent,
    random_tiny_task,
    weight_vectors,
    threshold_points,
    config_tiny,
    config_grid32,
    config_uneven,
    config_large,
    instance_footprint,
    GRID_AP,
    REGION_AP,
)
