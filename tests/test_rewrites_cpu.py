"""The CUDA path arranges the paper's iterations into products whose
epilogues load no second operand.  These FP64 NumPy checks pin each
rearrangement to the form it replaces, and the adjoint's arrangement to the
oracle's Daleckii-Krein derivative, so a dropped term, a wrong factor or a
transposed operand in the arrangement fails here on the CPU."""
import numpy as np

import oracle


def sym(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) * scale
    return 0.5 * (a + a.T)


def test_newton_schulz_as_x_times_z():
    """Section II-B: X (3I - X^2) / 2 = X Z with Z = 1.5 I - 0.5 X^2 (the squaring writes Z)."""
    x = sym(40, 1, 0.2)
    i = np.eye(40)
    z = 1.5 * i - 0.5 * x @ x
    assert np.allclose(x @ z, 0.5 * x @ (3 * i - x @ x), rtol=0, atol=1e-14)


def test_third_order_step_as_two_symmetric_products():
    """Section VI-A: X (15I - 10X^2 + 3X^4) / 8 = X Z, Z = 3/8 W^2 + 5/6 I, W = X^2 - 5/3 I."""
    x = sym(40, 2, 0.2)
    i = np.eye(40)
    x2 = x @ x
    w = x2 - 5.0 / 3.0 * i
    z = 0.375 * w @ w + 5.0 / 6.0 * i
    assert np.allclose(x @ z, x @ (15 * i - 10 * x2 + 3 * x2 @ x2) / 8.0, rtol=0, atol=1e-13)


def coupled_step_paper(x, e):
    """[[X, E], [0, X]] <- 1/2 M (3I - M^2), written out for the blocks."""
    i = np.eye(len(x))
    return 0.5 * x @ (3 * i - x @ x), 0.5 * (e @ (3 * i - x @ x) - x @ (x @ e + e @ x))


def upper_mirrored(c):
    """A symmetric result as the kernels write it: upper tiles, then the mirror."""
    return np.triu(c) + np.triu(c, 1).T


def coupled_step_tensor_cores(x, e):
    """The tensor-core adjoint's products, each C = A B^T with B read by rows:
    Z = 1.5 I - 0.5 X X^T; U = X (E^T)^T; T = E Z^T - 1.5 E; T += Z (E^T)^T;
    E' = T - 0.5 U X^T; X' = X Z^T.  Z and X' are symmetric results, written
    from their upper triangles: without that exact symmetry X X^T differs from
    X^2, and the antisymmetric part of X doubles every step."""
    i = np.eye(len(x))
    et = e.T.copy()                      # the transposed copy kept beside E
    z = upper_mirrored(-0.5 * (x @ x.T) + 1.5 * i)
    u = x @ et.T
    t = e @ z.T - 1.5 * e
    t = t + z @ et.T
    e_new = t - 0.5 * (u @ x.T)
    return upper_mirrored(x @ z.T), e_new


def test_without_exact_symmetry_the_antisymmetric_part_grows():
    """Why the symmetric products are mirrored: X <- X (1.5 I - 0.5 X X^T) doubles
    an antisymmetric perturbation of X at the fixed point sign(a)."""
    n = 20
    rng = np.random.default_rng(6)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = (q * np.where(np.arange(n) < 7, -1.0, 1.0)) @ q.T
    p = rng.standard_normal((n, n)) * 1e-12
    x = s + (p - p.T)
    i = np.eye(n)
    for _ in range(10):
        x = x @ (1.5 * i - 0.5 * x @ x.T)
    assert np.max(np.abs(x - x.T)) > 100 * 2e-12
    x = s + (p - p.T)
    for _ in range(10):
        x = upper_mirrored(x @ upper_mirrored(1.5 * i - 0.5 * x @ x.T))
    assert np.max(np.abs(x - x.T)) == 0.0


def test_adjoint_step_arrangement_equals_the_coupled_iteration():
    x = sym(30, 3, 0.15)
    rng = np.random.default_rng(4)
    e = rng.standard_normal((30, 30)) * 0.1   # nonsymmetric, like G
    xp, ep = coupled_step_paper(x, e)
    xt, et = coupled_step_tensor_cores(x, e)
    assert np.allclose(xt, xp, rtol=0, atol=1e-14)
    assert np.allclose(et, ep, rtol=0, atol=1e-14)


def test_adjoint_arrangement_converges_to_the_daleckii_krein_derivative():
    n = 24
    rng = np.random.default_rng(5)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(-1.0, -0.3, 8), rng.uniform(0.3, 1.2, n - 8)])
    a = (q * lam) @ q.T
    a = 0.5 * (a + a.T)
    g = rng.standard_normal((n, n))
    beta = 1.05 * np.max(np.abs(lam))
    x, e = a / beta, g / beta
    for _ in range(40):
        x, e = coupled_step_tensor_cores(x, e)
    lam_o, q_o = np.linalg.eigh(a)
    want = oracle.frechet_sign(lam_o, q_o, g)
    assert np.max(np.abs(e - want)) <= 1e-10 * np.max(np.abs(want))


def correction_round(a, s_tilde, fc_sign=1.0, keep_fc_commutator=True):
    """One correction round of the mixed path, in FP64 with exact products:
    F_c = -1/2 S (I - S^2); H = (S a + a S) / 2; C = ([S, a] - [F_c, a]) S;
    H F_a + F_a H = C (solved in H's eigenbasis); S <- S - F_c - F_a."""
    i = np.eye(len(a))
    fc = fc_sign * -0.5 * s_tilde @ (i - s_tilde @ s_tilde)
    h = 0.5 * (s_tilde @ a + a @ s_tilde)
    comm = s_tilde @ a - a @ s_tilde
    if keep_fc_commutator:
        comm = comm - (fc @ a - a @ fc)
    c = comm @ s_tilde
    w, q = np.linalg.eigh(h)
    fa = q @ ((q.T @ c @ q) / (w[:, None] + w[None, :])) @ q.T
    return s_tilde - fc - fa


def test_correction_round_squares_the_error():
    """The Newton step on {S^2 = I, [S, a] = 0}: an error delta of either symmetry
    type leaves O(delta^2 |a| / gap); a flipped F_c or a dropped [F_c, a] does not."""
    n = 60
    rng = np.random.default_rng(7)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(-1.0, -0.3, 20), rng.uniform(0.3, 1.4, n - 20)])
    a = (q * lam) @ q.T
    a = 0.5 * (a + a.T)
    s = (q * np.sign(lam)) @ q.T
    errs = []
    for delta in (1e-4, 1e-5):
        st = s + delta * sym(n, int(1e6 * delta))
        before = np.max(np.abs(st - s))
        after = np.max(np.abs(correction_round(a, st) - s))
        assert after <= 50 * before ** 2, (delta, before, after)
        errs.append(after)
        assert np.max(np.abs(correction_round(a, st, fc_sign=-1.0) - s)) > 0.5 * before
        assert np.max(np.abs(correction_round(a, st, keep_fc_commutator=False) - s)) > 50 * after
    assert errs[0] / errs[1] > 30  # quadratic, not linear, in delta


def six_bit_digits(m, k):
    """Signed base-64 digits of integers |m| < 2^(6k), most significant first."""
    s = np.sign(m)
    a = np.abs(m)
    return [s * ((a >> (6 * (k - p))) & 63) for p in range(1, k + 1)]


def test_sliced_residual_products_are_exact_where_the_method_needs_it():
    """The exact residual products of the mixed path (Section 5), in NumPy int64:
    S on a 24-bit grid as four 6-bit slices, a's rows scaled to their maxima
    and sliced six times, slice products of level p + q <= 8 summed with
    weights 2^(6 (8 - p - q)).  S^2 from the p <= q products (p < q doubled)
    plus an exact symmetrisation equals S_grid^2 exactly; S a comes within
    ~2e-10 of the FP64 product (level <= 7 alone would leave ~4e-9)."""
    n = 400
    rng = np.random.default_rng(3)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(-1.0, -0.3, 100), rng.uniform(0.3, 1.4, n - 100)])
    a = (q * lam) @ q.T
    a = 0.5 * (a + a.T)
    s = (q * np.sign(lam)) @ q.T
    e = int(np.ceil(np.log2(np.max(np.abs(s)))))
    m = np.round(s / 2.0 ** (e - 24)).astype(np.int64)
    m = (m + m.T) // 2 if not np.array_equal(m, m.T) else m
    sl = six_bit_digits(m, 4)
    assert np.array_equal(sum(d << (6 * (4 - p)) for p, d in enumerate(sl, 1)), m)
    # every slice product's sum stays exact in FP32 (below 2^24) for K <= 2048
    assert max(int(np.max(np.abs(x) @ np.abs(y).T)) for x in sl for y in sl) * (2048 // n) < 2 ** 24
    # S^2: p <= q with p < q doubled, then the exact symmetric part
    z = np.zeros((n, n), np.int64)
    for p in range(1, 5):
        for r in range(p, 5):
            w = 2 if p < r else 1
            z += w * (sl[p - 1] @ sl[r - 1].T) << (6 * (8 - p - r))
    z_sym = (z + z.T) // 2
    assert np.array_equal(z + z.T, 2 * z_sym)  # the symmetrisation is exact
    assert np.array_equal(z_sym, m @ m)
    # S a with a's rows scaled and sliced, levels <= 8 (and <= 7 for contrast)
    rexp = np.ceil(np.log2(np.max(np.abs(a), axis=1))).astype(int)
    ai = np.trunc(a / 2.0 ** (rexp[:, None] - 36)).astype(np.int64)
    tl = six_bit_digits(ai, 6)
    ref = (m * 2.0 ** (e - 24)) @ a

    def sliced(max_level):
        zz = np.zeros((n, n), np.int64)
        for p in range(1, 5):
            for r in range(1, 7):
                if p + r <= max_level:
                    zz += (sl[p - 1] @ tl[r - 1].T) << (6 * (8 - p - r))
        assert np.max(np.abs(zz)) < 2 ** 62
        return zz * 2.0 ** (e - 48) * 2.0 ** rexp[None, :]

    scale = np.max(np.abs(ref))
    err8 = np.max(np.abs(sliced(8) - ref)) / scale
    err7 = np.max(np.abs(sliced(7) - ref)) / scale
    assert err8 < 5e-10 and err7 > 1e-9, (err8, err7)


def test_one_round_with_an_inexact_lyapunov_solve_meets_the_acceptance_bound():
    """The one-round acceptance rule: with the Lyapunov solve to a relative 1e-3
    (the CG tolerance) and delta <= 1e-5, the remaining error
    delta^2 |a| / gap + delta 1e-3 stays below ~4e-8."""
    n = 60
    rng = np.random.default_rng(8)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(-1.0, -0.3, 20), rng.uniform(0.3, 1.4, n - 20)])
    a = (q * lam) @ q.T
    a = 0.5 * (a + a.T)
    s = (q * np.sign(lam)) @ q.T
    i = np.eye(n)
    p = sym(n, 9)
    st = s + 1e-5 * p / np.max(np.abs(p))
    delta = np.max(np.abs(st - s))
    assert delta <= 1.0000001e-5
    fc = -0.5 * st @ (i - st @ st)
    h = 0.5 * (st @ a + a @ st)
    c = ((st @ a - a @ st) - (fc @ a - a @ fc)) @ st
    w, qh = np.linalg.eigh(h)
    fa = qh @ ((qh.T @ c @ qh) / (w[:, None] + w[None, :])) @ qh.T
    noise = sym(n, 10)
    fa_cg = fa + 1e-3 * np.linalg.norm(fa) / np.linalg.norm(noise) * noise  # relative residual ~1e-3
    err = np.max(np.abs(st - fc - fa_cg - s))
    assert err < 4e-8, err


def lyapunov_cg(h, c, steps, upper_tiles=False, tile=32, weight=2.0):
    """CG on L -> H L + L H = C (H SPD, C symmetric), as the mixed path runs
    it.  With upper_tiles, R and X are updated on the tiles (a, b), a <= b,
    only (a diagonal tile whole); P is completed from its upper tiles; the
    inner product <R, R> counts an off-diagonal tile `weight` times."""
    n = len(h)
    nt = n // tile
    up = np.zeros((n, n), dtype=bool)
    for a in range(nt):
        for b in range(a, nt):
            up[a * tile:(a + 1) * tile, b * tile:(b + 1) * tile] = True
    # off-diagonal upper tiles: weight, diagonal tiles: 1, lower tiles: not stored
    wgt = np.where(up & ~up.T, weight, np.where(up, 1.0, 0.0))

    def inner(m):
        return float(np.sum(wgt * m * m)) if upper_tiles else float(np.sum(m * m))

    def full(m):  # the lower tiles from the upper ones
        return np.where(up, m, m.T) if upper_tiles else m

    x = np.zeros_like(c)
    r = c.copy()
    p = c.copy()
    rr = inner(r)
    for _ in range(steps):
        w = h @ full(p)
        tp = w + w.T
        alpha = rr / float(np.sum(full(p) * tp))  # <P, W + W^T>, from the full product
        x = x + alpha * full(p)
        r_new = r - alpha * tp
        if upper_tiles:
            r_new = np.where(up, r_new, 0.0)  # the lower tiles are never written
        rr_new = inner(r_new)
        p = r_new + (rr_new / rr) * full(p)
        r, rr = r_new, rr_new
    return full(x) if upper_tiles else x


def test_cg_on_upper_tiles_equals_the_full_cg():
    """R, X and P are symmetric, so updating the upper tiles only, completing
    P from them and counting off-diagonal tiles twice in <R, R> reproduces the
    full CG; counting them once does not."""
    n = 96
    rng = np.random.default_rng(11)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    h = (q * rng.uniform(0.2, 1.5, n)) @ q.T
    h = 0.5 * (h + h.T)
    c = sym(n, 12)
    full = lyapunov_cg(h, c, 12)
    upper = lyapunov_cg(h, c, 12, upper_tiles=True)
    assert np.max(np.abs(upper - full)) <= 1e-12 * np.max(np.abs(full))
    # the solution itself: H L + L H = C to the CG's accuracy after 40 steps
    lx = lyapunov_cg(h, c, 40, upper_tiles=True)
    assert np.max(np.abs(h @ lx + lx @ h - c)) <= 1e-8 * np.max(np.abs(c))
    wrong = lyapunov_cg(h, c, 12, upper_tiles=True, weight=1.0)
    assert np.max(np.abs(wrong - full)) > 1e-3 * np.max(np.abs(full))


def test_cg_tolerance_from_the_correction_size():
    """The one-round rule: a correction of size delta solved to a relative
    residual tol leaves ~delta * tol; CG stops at tol = 1e-2 where
    delta * 1e-2 <= 2e-8, and resumes at max(2e-8 / delta, 1e-3) otherwise.
    The remaining error then stays below 4e-8 for delta up to 2e-5."""
    n = 60
    rng = np.random.default_rng(13)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(-1.0, -0.3, 20), rng.uniform(0.3, 1.4, n - 20)])
    a = (q * lam) @ q.T
    a = 0.5 * (a + a.T)
    s = (q * np.sign(lam)) @ q.T
    i = np.eye(n)
    pert = sym(n, 14)
    for delta in (1e-6, 2e-6, 5e-6, 2e-5):
        st = s + delta * pert / np.max(np.abs(pert))
        fc = -0.5 * st @ (i - st @ st)
        h = 0.5 * (st @ a + a @ st)
        c = ((st @ a - a @ st) - (fc @ a - a @ fc)) @ st
        w, qh = np.linalg.eigh(h)
        fa = qh @ ((qh.T @ c @ qh) / (w[:, None] + w[None, :])) @ qh.T
        d = np.max(np.abs(fc + fa))
        tol = 1e-2 if d * 1e-2 <= 2e-8 else max(2e-8 / d, 1e-3)
        noise = sym(n, 15)
        fa_cg = fa + tol * np.linalg.norm(fa) / np.linalg.norm(noise) * noise
        err = np.max(np.abs(st - fc - fa_cg - s))
        assert err < 4e-8, (delta, tol, err)
