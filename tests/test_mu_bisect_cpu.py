"""Host logic of the mu search (Section IV-G, Algorithm 1's outer loop), checked
on the CPU through the library's host-only hook: the same bisection as
submat_mu_search, on the electron count N(mu) = sum_i (1 - sign(l_i - mu)) / 2
of a set of levels (the trace of D for a diagonal K), with the statuses the
zero-temperature staircase implies (reading R9)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__ as g
    g.build()
    from paper_2004_10811_gb300 import submat
    return submat


def gapped_levels(seed, n_occ=40, n_virt=60):
    rng = np.random.default_rng(seed)
    return np.sort(np.concatenate([rng.uniform(-1.0, -0.3, n_occ), rng.uniform(0.3, 1.5, n_virt)]))


def count(levels, mu):
    """N(mu) by its definition, sign(0) = 0."""
    return float(np.sum(levels < mu) + 0.5 * np.sum(levels == mu))


@pytest.mark.parametrize("mu0", [1.0, -0.9, 0.0, 0.31])
def test_target_on_a_plateau_ends_in_the_gap(sm, mu0):
    lv = gapped_levels(1)
    mu, steps, n, status = sm.debug_mu_bisect(lv, 40.0, mu0, tol=1e-9)
    assert status == "OK"
    assert n == 40.0 == count(lv, mu)
    assert lv[39] < mu < lv[40]
    assert steps <= 60
    if mu0 == 0.0:
        assert steps == 1 and mu == 0.0  # already on the plateau


def test_target_between_plateaus_reports_the_step(sm):
    """n_el = 40.5 lies on no plateau: the bracket shrinks onto the level where N
    jumps from 40 to 41 and the search reports MU_NO_ROOT there."""
    lv = gapped_levels(2)
    mu, steps, n, status = sm.debug_mu_bisect(lv, 40.5, 1.2, tol=1e-12)
    assert status == "MU_NO_ROOT"
    b = np.max(np.abs(lv - 1.2))
    assert abs(mu - lv[40]) <= 2e-10 * b
    assert n in (40.0, 41.0)
    # the bracket halves per step from 2 x 1.01 b down to 1e-10 b
    assert steps <= int(np.ceil(np.log2(2.02e10))) + 2


def test_step_cap_reports_not_converged(sm):
    lv = gapped_levels(3)
    mu, steps, n, status = sm.debug_mu_bisect(lv, 40.0, 1.4, tol=1e-9, max_steps=1)
    assert status == "NOT_CONVERGED" and steps == 1
    assert mu == 1.4 and n == count(lv, 1.4)


def test_degenerate_level_at_mu_counts_half(sm):
    """A level exactly at mu holds half an electron (sign(0) = 0), so a
    half-integer target on a dyadic level is met exactly."""
    lv = np.array([-0.5, 0.0, 0.5])
    mu, steps, n, status = sm.debug_mu_bisect(lv, 1.5, 0.0, tol=1e-12)
    assert status == "OK" and mu == 0.0 and n == 1.5 and steps == 1


def test_bad_arguments_rejected(sm):
    with pytest.raises(sm.SubmatError) as ei:
        sm.debug_mu_bisect([0.0, 1.0], 1.0, 0.5, tol=0.0)
    assert ei.value.name == "INVALID_ARG"


@pytest.mark.parametrize("scale", [0.5, 0.1, 0.01])
def test_underestimated_bound_grows_the_bracket(sm, scale):
    """A spectral bound below the true one starts the bracket short of the
    target; the far end is then evaluated and the bracket moves outward until
    it holds n_el, so the search still lands on the right plateau or step."""
    lv = gapped_levels(4)
    mu, steps, n, status = sm.debug_mu_bisect(lv, 40.0, -0.95, tol=1e-9, bound_scale=scale)
    assert status == "OK"
    assert n == 40.0 == count(lv, mu)
    assert lv[39] < mu < lv[40]
    mu, steps, n, status = sm.debug_mu_bisect(lv, 40.5, -0.95, tol=1e-12, max_steps=80,
                                              bound_scale=scale)
    assert status == "MU_NO_ROOT"
    assert abs(mu - lv[40]) <= 2e-10 * np.max(np.abs(lv + 0.95))
    assert n in (40.0, 41.0)


def test_unreachable_target_is_rejected(sm):
    """A target outside [0, n] can never be met: rejected before any evaluation."""
    lv = gapped_levels(5)
    for target in (100.5, -0.5):
        with pytest.raises(sm.SubmatError) as ei:
            sm.debug_mu_bisect(lv, target, 0.0, tol=1e-9)
        assert ei.value.name == "INVALID_ARG"


@pytest.mark.parametrize("target,mu0,tol", [(40.0, 1.2, 1e-9), (40.5, 1.2, 1e-12), (40.0, -0.95, 1e-9),
                                            (70.0, -0.9, 1e-9)])
def test_probes_keep_the_result_and_save_full_evaluations(sm, target, mu0, tol):
    """Probes off by up to 3 electrons (with that bound) decide the steps far
    from the target; the search ends at the same mu and status as without
    them, with fewer full evaluations, and the returned mu's N is full."""
    lv = gapped_levels(6)
    ref = sm.debug_mu_bisect(lv, target, mu0, tol=tol, max_steps=200)
    mu, steps, n, status, probes = sm.debug_mu_bisect(lv, target, mu0, tol=tol, max_steps=200, probe_err=3.0,
                                                      with_probes=True)
    assert status == ref[3]
    assert n == count(lv, mu)
    if status == "OK":
        assert abs(n - target) <= tol * target
    else:
        assert abs(mu - ref[0]) <= 1e-9 * np.max(np.abs(lv - mu0)) * 4
    assert probes > 0
    assert steps < ref[1]
