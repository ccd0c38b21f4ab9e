"""Seeded synthetic inputs shared by the oracle, the CUDA path, the tests and the bench.

This package only draws images and material tables. It holds none of the
lattice-spring arithmetic (no springs, forces or integration).
"""
from .images import (  # noqa: F401
    inclusion_image,
    foam_volume,
    batch_specimens,
    warmstart_specimens,
    two_phase_materials,
    one_phase_materials,
    WORKLOADS,
)
