"""Host logic of the exact sliced residual products (mixed path), checked on
the CPU through the library's host-only hook: every kept slice pair appears
exactly once with its weight, and each launch stays inside the bounds that
make its FP32 and int32 sums exact.

The slice products compute sum_{p+q<=8} 2^(6 (8 - p - q)) X_p Y_q^T with 6-bit
integer slices |t| <= 63 (one 2^-48 scale left out).  A BF16 x BF16 -> FP32
product of such slices is exact while every partial sum stays below 2^24:
per_acc products of K <= 2048 terms give at most 2 * 63^2 * 2048 < 2^24.
With two accumulators per launch (256-wide tiles) they combine as
acc0 * 2^d + acc1 with d <= 6, below 2^31; with up to four (128-wide tiles)
as sum_k acc_k * 2^shift_k in 64-bit integers, shift_k <= 36.
"""
import itertools

import pytest

BITS, MAX_LEVEL = 6, 8


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__ as g
    g.build()
    from paper_2004_10811_gb300 import submat
    return submat


def expected(nx, ny, sym):
    """(p, q) -> shift for every kept slice product (the definition, by brute force)."""
    want = {}
    for p, q in itertools.product(range(1, nx + 1), range(1, ny + 1)):
        if p + q > MAX_LEVEL:
            continue
        shift = BITS * (MAX_LEVEL - p - q)
        if not sym:
            want[(p, q)] = shift
        elif p < q:
            want[(p, q)] = shift + 1  # s_p s_q + s_q s_p = 2 s_p s_q on the symmetric part
        elif p == q:
            want[(p, q)] = shift
    return want


@pytest.mark.parametrize("max_acc", [2, 4])
@pytest.mark.parametrize("nx,ny,sym,per_acc", [
    (4, 4, True, 2), (4, 6, False, 2),      # the first round: S on a 24-bit grid
    (6, 6, True, 2), (6, 6, False, 2),      # later rounds: 36 bits
    (4, 4, True, 1), (4, 6, False, 1),      # K extents above 2048
    (1, 1, True, 2), (2, 5, False, 2),
])
def test_every_kept_pair_once_with_its_weight(sm, nx, ny, sym, per_acc, max_acc):
    plan = sm.debug_slice_plan(nx, ny, sym, per_acc, max_acc)
    got = {}
    for _launch, _acc, p, q, shift in plan.tolist():
        assert (p, q) not in got, (p, q)
        got[(p, q)] = shift
    assert got == expected(nx, ny, sym)


@pytest.mark.parametrize("max_acc", [2, 4])
@pytest.mark.parametrize("nx,ny,sym,per_acc", [(4, 4, True, 2), (4, 6, False, 2), (6, 6, True, 2),
                                                (6, 6, False, 2), (4, 6, False, 1), (6, 6, True, 1)])
def test_launches_stay_inside_the_exactness_bounds(sm, nx, ny, sym, per_acc, max_acc):
    plan = sm.debug_slice_plan(nx, ny, sym, per_acc, max_acc)
    launches = {}
    for launch, acc, p, q, shift in plan.tolist():
        launches.setdefault(launch, {}).setdefault(acc, []).append((p, q, shift))
    assert sorted(launches) == list(range(len(launches)))
    assert 2 * 63 ** 2 * 2048 < 2 ** 24 and 2 ** 24 * 2 ** 6 + 2 ** 24 < 2 ** 31
    assert 4 * 2 ** 24 * 2 ** 36 < 2 ** 63
    for accs in launches.values():
        assert set(accs) <= set(range(max_acc)) and 0 in accs
        assert sorted(accs) == list(range(len(accs)))
        for prods in accs.values():
            # one exact accumulator: one weight, at most per_acc products
            assert len({s for _p, _q, s in prods}) == 1 and len(prods) <= per_acc
            assert prods[0][2] <= 36  # acc * 2^shift stays below 2^60
        shifts = [accs[k][0][2] for k in sorted(accs)]
        assert shifts == sorted(shifts, reverse=True)  # accumulator 0 the heaviest
        if max_acc == 2 and 1 in accs:
            d = accs[0][0][2] - accs[1][0][2]
            assert 0 <= d <= 6  # acc0 * 2^d + acc1 stays exact in 32 bits
        assert sum(len(v) for v in accs.values()) <= 2 * max_acc
        xs = {p for prods in accs.values() for p, _q, _s in prods}
        ys = {q for prods in accs.values() for _p, q, _s in prods}
        assert len(xs) + len(ys) <= 6  # operand tiles per pipeline stage
    # launches in decreasing weight, so the int64 sums grow from the top
    tops = [accs[0][0][2] for _l, accs in sorted(launches.items())]
    assert tops == sorted(tops, reverse=True)


def test_default_plans_use_the_expected_launch_counts(sm):
    """The first round: I - S^2 in 3 launches and S a in 4 with four
    accumulators per launch (5 and 6 with two); S a keeps 21 products."""
    assert len({r[0] for r in sm.debug_slice_plan(4, 4, True, 2).tolist()}) == 3
    assert len({r[0] for r in sm.debug_slice_plan(4, 6, False, 2).tolist()}) == 4
    assert len({r[0] for r in sm.debug_slice_plan(4, 4, True, 2, 2).tolist()}) == 5
    assert len({r[0] for r in sm.debug_slice_plan(4, 6, False, 2, 2).tolist()}) == 6
    assert len(sm.debug_slice_plan(4, 6, False, 2)) == 21


def test_bad_arguments_rejected(sm):
    for args in ((0, 4, False, 2), (4, 7, False, 2), (4, 6, True, 2), (4, 4, True, 3), (4, 4, True, 2, 3)):
        with pytest.raises(sm.SubmatError) as ei:
            sm.debug_slice_plan(*args)
        assert ei.value.name == "INVALID_ARG"
