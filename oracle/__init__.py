"""FP64 CPU oracle of the LES time step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The product path (``paper_2301_04698_gb300``) never
imports, links or runs anything here.
"""
from .oracle import Oracle, build_oracle, FIELDS, NDIAG, DIAG_NAMES  # noqa: F401
