"""Plain FP64 CPU oracle of the Riccati sweep -- test infrastructure only.

Only tests/, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
import this package.  The product path (``paper_2205_15000_b300``) never does.
"""
from .oracle import (OracleGeom, STEPPERS, bulk_gap, greens, matsubara, norm_D, quad_weight, step,  # noqa: F401
                     step_midpoint, ozaki_poles, ozaki_energies)
