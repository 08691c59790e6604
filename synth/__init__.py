"""Seeded synthetic inputs: gapped model Hamiltonians in block-sparse (BSR) form.

This package only draws random geometries and matrix elements and stores them
in BSR layout.  It contains none of the purification arithmetic; both the CPU
oracle and the CUDA path consume what it produces.
"""

from .systems import (  # noqa: F401
    Bsr,
    System,
    make_chain,
    make_cluster,
    make_slab,
    make_config,
    make_batch_config,
    carve_sphere,
    make_overlap,
    CONFIGS,
)
