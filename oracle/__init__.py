"""FP64 CPU oracle of the Method of Averaged Marginals (test infrastructure).

Only the tests, the package's ``smoke()`` check and the CPU-baseline leg of
``bench.py`` may import this package.  The library itself never calls it.
"""
from .mam_oracle import (  # noqa: F401
    project_simplex,
    proj_balanced,
    dist_balanced,
    prepare,
    Prepared,
    MamOracle,
    bundle_sequence,
    lower_bound,
)
