"""FP64 CPU oracle of the block-based multiresolution step (test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
import this package.  The product library never loads it.
"""
from .oracle import Oracle, OracleParams, build_oracle  # noqa: F401
