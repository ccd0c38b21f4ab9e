"""FP64 CPU oracle of the lattice-spring method -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the bench's CPU-baseline leg may import
this package. The CUDA library never loads it and shares no code with it.
"""
from .oracle import Oracle, build_oracle, ORACLE_SO  # noqa: F401
