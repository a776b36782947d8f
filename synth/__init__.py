"""Seeded synthetic inputs for reverse k-ranks workloads.

This module is the one piece of code that both the FP64 oracle (``oracle/``)
and the CUDA path's tests and benchmark use.  It only draws random inputs
(user, item and query vectors, per-query k, sample positions, user subsets);
it holds none of the method's arithmetic.

The paper evaluates on matrix-factorisation embeddings of Amazon-Kindle,
MovieLens-25M and Netflix with d = 200 (Section 5, "Dataset").  Those datasets
are not available here, so these generators stand in for them: rows whose
direction is isotropic Gaussian (optionally clustered around Gaussian centres)
and whose norm is log-normal, matching the roughly Gaussian norm and inner
product distributions the paper reports (Section 4.2, Fig. 2).
"""

from .workloads import (  # noqa: F401
    Workload,
    WORKLOADS,
    disjoint_queries,
    gaussian_rows,
    mixture_rows,
    make_workload,
    sample_positions,
)
