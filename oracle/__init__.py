"""FP64 oracle of the geometry-to-AMR hot path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The product path (``paper_2502_16310_gb300``) never
does, and the two share no code.

Parity: every function here is pinned by ``tests/test_oracle_*.py`` against
brute force on tiny inputs, independent exact-rational constructions
(polygon clipping, linear solves), closed forms for the circle and the sphere
and central finite differences.  Nothing in it is "parity unpinned".
"""
from .oracle import (  # noqa: F401
    Domain,
    OracleGeometry,
    build,
    lattice_dirs,
    run_pipeline,
)
