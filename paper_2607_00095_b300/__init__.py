"""B300-native batched nonlinear constraint projection (the SNAP-FM hot path).

    from paper_2607_00095_b300 import Problem, SnapProject, project

The compute path is libsnap.so (hand-written sm_103a CUDA behind the C ABI of include/snap.h);
importing this package does not load it, the first call does, and fails loudly if it is missing.
"""
from .api import (Batch, Problem, SnapProject, decode_stats, measure_fp64_rate, options,  # noqa: F401
                  project, vorticity_problem)
