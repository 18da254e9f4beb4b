"""Seeded synthetic inputs: water-like block-sparse Kohn-Sham matrices.

This package only *draws inputs* (molecule positions, the block sparsity
pattern, random block values).  It holds none of the submatrix method's
arithmetic, so both the CPU oracle and the CUDA path may consume it.
"""
from .water import (  # noqa: F401
    bsr_to_dense,
    random_symmetric_bsr,
    summary,
    BSRMatrix,
    CONFIGS,
    make_config,
    make_water,
    make_slab,
    small_case,
)
