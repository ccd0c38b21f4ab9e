"""GB300 (sm_103a) lattice-spring hot path: image -> particle-spring network,
spring force, deterministic gather, irreversible breakage and damped velocity
Verlet under displacement control (arXiv 2201.04565), behind the C ABI of
include/lsm.h. ``lsm`` is the thin Python binding of that ABI.
"""
from . import lsm  # noqa: F401
