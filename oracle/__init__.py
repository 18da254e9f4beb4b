"""CPU FP64 oracle of the submatrix method (TEST INFRASTRUCTURE ONLY).

This package is the independent reference that the CUDA path is checked
against.  Only the tests, the smoke check in ``__graft_entry__`` and the CPU
baseline leg of ``bench.py`` may import it; the library itself never does.
It shares no code with the CUDA path: it is plain NumPy/LAPACK in float64,
following the paper step by step (Section III-A, Eqs. eigendecompsym and
signevext, Algorithm 1).

Finite temperature (``oracle.fermi``): the Fermi function in place of
signum (Section IV-F, last paragraph), with its electron count, dN/dmu, a
bracketed Newton search for mu and the Daleckii-Krein gradient.

Groups of block columns sharing one submatrix (``oracle.grouped``, Section
IV-C): ``density_matrix_grouped``.

Parity unpinned: results that depend on eigenvalues of a submatrix lying
within about 1e-8 of the chemical potential (the answer there is
ill-conditioned, sensitivity ~ rounding / |lambda|); see the pins in
``tests/test_oracle_pins.py`` for everything else.
"""
from .submatrix import (  # noqa: F401
    column_structure,
    assemble_submatrix,
    sign_by_eigh,
    submatrix_sign,
    density_block_column,
    density_matrix,
    trace_bsr,
    decompose_all,
    n_elec_alg1,
    mu_search_alg1,
    frechet_sign,
    band_energy,
    band_energy_grad,
    sign_backward,
    dense_sign,
)
from .fermi import (  # noqa: F401
    fermi,
    fermi_deriv,
    fermi_by_eigh,
    density_matrix_T,
    n_elec_T,
    dn_dmu_T,
    mu_search_newton_T,
    frechet_fermi,
    fermi_backward,
)
from .grouped import density_matrix_grouped  # noqa: F401
