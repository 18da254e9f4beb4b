"""The finite-temperature polynomial (host code, through the host-only hook):
the Chebyshev series of tanh(c x) on [-1, 1] in the baby-step / giant-step
form that the GPU evaluates, checked against numpy's tanh on a dense grid.
The Fermi function is (1 - tanh(x / 2kT)) / 2 (Section IV-F, last
paragraph: the Fermi function in place of signum)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__ as g
    g.build()
    from paper_2004_10811_gb300 import submat
    return submat


def cheb_t(k, x):
    """T_k(x) = cos(k arccos x) on [-1, 1]."""
    return np.cos(k * np.arccos(np.clip(x, -1.0, 1.0)))


def evaluate(r, x):
    """p(x) = sum_j R_j(x) T_j(T_16(x)), R_j = sum_q r[j, q] T_{2q+1}(x)."""
    y = cheb_t(16, x)
    p = np.zeros_like(x)
    for j in range(r.shape[0]):
        rj = sum(r[j, q] * cheb_t(2 * q + 1, x) for q in range(8))
        p += rj * cheb_t(j, y)
    return p


@pytest.mark.parametrize("c,tol", [(0.5, 1e-13), (5.0, 1e-13), (40.0, 1e-13), (150.0, 1e-13), (40.0, 1e-8)])
def test_series_matches_tanh(sm, c, tol):
    r, m, trunc = sm.debug_fermi_poly(c, tol)
    assert m % 2 == 1 and trunc <= tol
    assert r.shape == ((m + 1 + 15) // 16, 8)
    x = np.linspace(-1.0, 1.0, 20001)
    err = np.max(np.abs(evaluate(r, x) - np.tanh(c * x)))
    # the truncation bound, plus the rounding of the coefficients and of this check
    assert err <= trunc + 2e-13 * max(1.0, m / 16), (c, m, err, trunc)


def test_degree_grows_with_c_and_is_capped(sm):
    ms = [sm.debug_fermi_poly(c)[1] for c in (1.0, 10.0, 100.0)]
    assert ms[0] < ms[1] < ms[2]
    # a geometric series: the degree grows about linearly in c for large c
    assert 5 < ms[2] / ms[1] < 15
    with pytest.raises(sm.SubmatError) as ei:
        sm.debug_fermi_poly(100.0, 1e-13, max_degree=101)
    assert ei.value.name == "UNSUPPORTED"


def test_bad_arguments(sm):
    for args in ((0.0, 1e-13), (-1.0, 1e-13), (5.0, 0.0)):
        with pytest.raises(sm.SubmatError):
            sm.debug_fermi_poly(*args)
