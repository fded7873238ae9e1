"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This package only draws random numbers and lays them out; it holds none of the
transform's arithmetic (no eigenvalues, no DCT, no Cauchy products). Both the
CUDA path and the FP64 oracle consume what it returns.
"""
from .workloads import (  # noqa: F401
    SIZES_SMALL,
    MixedSegment,
    MixedWorkload,
    ar1_signals,
    edge_update_v,
    laplace_residuals,
    mixed_size_workload,
    normal_signals,
    random_unit_v,
    self_loop_v,
)
