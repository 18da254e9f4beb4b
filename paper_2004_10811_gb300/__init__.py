"""GB300 (sm_103a) implementation of the submatrix method's sign path.

D = 1/2 (I - sign(K - mu I)) for a symmetric block-sparse K (Lass, Schade,
Kuehne, Plessl, "A Submatrix-Based Method for Approximate Matrix Function
Evaluation in the Quantum Chemistry Code CP2K", Section III), evaluated by
the CUDA library ``libsubmat.so`` behind the C ABI in ``include/submat.h``.
"""
from .submat import (  # noqa: F401
    EXPORTS,
    FP32,
    FP64,
    MIXED_BF16_REFINE,
    Plan,
    SubmatError,
    SubmatLibraryMissing,
    load,
    make_autograd_sign,
)
