"""CPU oracle for HAMLS on S^2 (test infrastructure only).

This package is a slow, plain restatement of the paper's algorithm used to
check the CUDA library. Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it. The product path never calls it
and shares no code with it.
"""
from .hamls_oracle import *  # noqa: F401,F403
from .voronoi import voronoi_areas, voronoi_area_at  # noqa: F401
from .forward import complex_coeffs, forward, forward_full, global_lsq  # noqa: F401
