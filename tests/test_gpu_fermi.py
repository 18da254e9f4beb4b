"""Finite temperature on the GPU (Section IV-F, last paragraph: the Fermi
function in place of signum) against the finite-temperature oracle: D element
by element, the trace, dN/dmu, and the Newton search for mu."""
import numpy as np
import pytest

import oracle
from synth import make_config, random_symmetric_bsr, small_case
from synth.water import make_water

pytestmark = pytest.mark.gpu

# FP64 plans: the series is cut at 1e-13 and the products are FP64; FP32
# plans carry FP32 products (about 1e-6 relative per product)
TOL = {"fp64": 1e-10, "fp32": 2e-5}


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2004_10811_gb300 as p
    return p


def transpose_index(m):
    """perm such that vals[perm] lays out K_(c,r)^T in block (r, c)'s slots."""
    vp = m.val_ptr
    rows = np.repeat(np.arange(m.nblk), np.diff(m.row_ptr))
    pos = {(int(rows[p]), int(m.col_idx[p])): p for p in range(m.nnzb)}
    perm = np.empty(m.vals.shape[0], dtype=np.int64)
    for (r, c), p in pos.items():
        q = pos[(c, r)]
        br, bc = m.block_sizes[r], m.block_sizes[c]
        idx = np.arange(br * bc)
        perm[vp[p] + idx] = vp[q] + (idx % bc) * br + idx // bc
    return perm


def run(pkg, m, mu, kT, **kw):
    import torch
    K = torch.from_numpy(m.vals).cuda()
    with pkg.Plan.from_bsr(m, kT=kT, **kw) as plan:
        D = plan.sign(K, mu)
        tr = plan.trace(D)
        st = plan.stats()
    return D.cpu().numpy(), tr, st


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kT,mu", [(0.05, 0.0), (0.2, 0.1), (0.02, -0.05)])
def test_water_matches_oracle(pkg, prec, kT, mu):
    m = make_water(48, 6, 6.0, (3, -1.0, -0.3), (3, 0.3, 1.0), seed=12)
    want = oracle.density_matrix_T(m, mu, kT, workers=4)
    got, tr, st = run(pkg, m, mu, kT, prec=prec)
    err = float(np.max(np.abs(got - want)))
    assert err <= TOL[prec], (prec, kT, err, st["poly_degree"])
    assert abs(tr - oracle.trace_bsr(m, want)) <= TOL[prec] * m.n
    dec = oracle.decompose_all(m, mu)
    dn = oracle.dn_dmu_T(dec, 0.0, kT)
    # dN/dmu = sum_c (F - F^2)_cc / kT cancels to ~f (1 - f): the entries' own
    # error, summed over the n columns and divided by kT, bounds it absolutely
    eps = 1e-12 if prec == "fp64" else 2e-6
    assert abs(st["dn_dmu"] - dn) <= 1e-8 * dn + eps * m.n / kT
    assert st["poly_degree"] > 0 and st["poly_trunc"] <= (1e-13 if prec == "fp64" else 1e-8)


@pytest.mark.parametrize("sizes,density,seed", [
    ([2, 3, 1, 4, 2, 3], 0.45, 21),
    ([5, 7, 3, 9, 2, 8, 6, 4, 7, 5, 3, 6], 0.35, 24),
    ([1] * 70, 0.2, 25),
])
def test_uneven_blocks(pkg, sizes, density, seed):
    m = random_symmetric_bsr(sizes, density=density, seed=seed, scale=0.5)
    want = oracle.density_matrix_T(m, 0.05, 0.1)
    got, _tr, _st = run(pkg, m, 0.05, 0.1, prec="fp64")
    assert float(np.max(np.abs(got - want))) <= TOL["fp64"]


def test_waves_and_a_zero_submatrix(pkg):
    """Several waves (each with its own scale and polynomial); and a block
    whose submatrix is exactly mu I, where f(0) = 1/2 gives D = I / 2."""
    m = small_case(n_mol=40, block=4, r_c=5.5, seed=5)
    want = oracle.density_matrix_T(m, 0.0, 0.1)
    got, _tr, st = run(pkg, m, 0.0, 0.1, prec="fp64", workspace_cap_bytes=3_000_000)
    assert st["waves"] > 2
    assert float(np.max(np.abs(got - want))) <= TOL["fp64"]
    from synth.water import BSRMatrix
    bs = np.array([2, 2], dtype=np.int32)
    vals = np.array([0.3, 0.0, 0.0, 0.3, -1.0, 0.2, 0.2, 0.5])
    z = BSRMatrix(bs, np.array([0, 1, 2]), np.array([0, 1], dtype=np.int32), vals)
    got, _tr, _st = run(pkg, z, 0.3, 0.05, prec="fp64")
    want = oracle.density_matrix_T(z, 0.3, 0.05)
    assert got[:4].tolist() == [0.5, 0.0, 0.0, 0.5]
    assert float(np.max(np.abs(got - want))) <= 1e-12


def test_low_temperature_approaches_zero_temperature(pkg):
    """kT = gap / 20: the Fermi function differs from the step by at most
    e^-20 ~ 2e-9 on every eigenvalue, so D is the T = 0 result to that."""
    import torch
    m = small_case(n_mol=16, block=3, r_c=5.5, seed=102)
    dec = oracle.decompose_all(m, 0.0)
    gap = min(np.min(np.abs(lam)) for lam, _q in dec)
    got, _tr, st = run(pkg, m, 0.0, gap / 20.0, prec="fp64")
    with pkg.Plan.from_bsr(m, prec="fp64") as plan:
        d0 = plan.sign(torch.from_numpy(m.vals).cuda(), 0.0).cpu().numpy()
    assert float(np.max(np.abs(got - d0))) <= 5e-9
    assert float(np.max(np.abs(got - oracle.density_matrix_T(m, 0.0, gap / 20.0)))) <= TOL["fp64"]


@pytest.mark.parametrize("mu0", [0.5, -0.6, 0.0])
def test_newton_mu_search_matches_oracle(pkg, mu0):
    """Tr D(mu) = N_el by Newton steps with dN/dmu from the same evaluation;
    the oracle's bracketed Newton on its stored eigendecompositions agrees."""
    import torch
    m = make_water(48, 6, 6.0, (3, -1.0, -0.3), (3, 0.3, 1.0), seed=12)
    kT = 0.05
    dec = oracle.decompose_all(m, 0.0)
    mu_o, _n, _steps = oracle.mu_search_newton_T(dec, m.n_el, kT, -3.0, 3.0, tol=1e-14)
    K = torch.from_numpy(m.vals).cuda()
    with pkg.Plan.from_bsr(m, prec="fp64", kT=kT) as plan:
        mu, D, status = plan.mu_search(K, m.n_el, mu0=mu0, tol=1e-11, max_steps=40)
        steps = plan.stats()["mu_steps"]
        tr = plan.trace(D)
    assert status == "OK"
    assert abs(tr - m.n_el) <= 1e-11 * m.n_el
    # the oracle's count at the GPU's mu, and the two roots
    assert abs(oracle.n_elec_T(dec, mu, kT) - m.n_el) <= 1e-9 * m.n_el
    dn = oracle.dn_dmu_T(dec, mu_o, kT)
    assert abs(mu - mu_o) <= 2e-9 * m.n_el / dn
    assert steps <= 15


def test_dn_dmu_matches_central_differences_of_the_gpu_trace(pkg):
    import torch
    m = make_water(48, 6, 6.0, (3, -1.0, -0.3), (3, 0.3, 1.0), seed=12)
    kT, mu, h = 0.05, 0.03, 1e-4
    K = torch.from_numpy(m.vals).cuda()
    with pkg.Plan.from_bsr(m, prec="fp64", kT=kT) as plan:
        trs = [plan.trace(plan.sign(K, mu + d)) for d in (-h, h)]
        plan.sign(K, mu)
        dn = plan.stats()["dn_dmu"]
    fd = (trs[1] - trs[0]) / (2 * h)
    assert abs(dn - fd) <= 1e-5 * dn


def test_newton_mu_search_on_the_2048x23_recipe_at_128_molecules(pkg):
    """The 2048x23 workload's recipe (block 23, cutoff 8 A) at 128 molecules,
    FP32 plan at kT = 0.1: the search meets 1e-6 relative and lands where the
    oracle's count says N = N_el."""
    import torch
    m = make_water(128, 23, 8.0, (4, -1.0, -0.3), (19, 0.3, 1.5), seed=105)
    kT = 0.1
    K = torch.from_numpy(m.vals).cuda()
    with pkg.Plan.from_bsr(m, prec="fp32", kT=kT) as plan:
        mu, D, status = plan.mu_search(K, m.n_el, mu0=0.8, tol=1e-6, max_steps=30)
        steps = plan.stats()["mu_steps"]
    assert status == "OK" and steps <= 12
    dec = oracle.decompose_all(m, 0.0)
    n_o = oracle.n_elec_T(dec, mu, kT)
    assert abs(n_o - m.n_el) <= 2e-5 * m.n_el


@pytest.mark.parametrize("cfg", [3, 4])
def test_full_size_column_ranges(pkg, cfg):
    """The 2048x23 and 20736x6 workloads at kT = 0.1, FP64, on column ranges
    spread over the system."""
    import torch
    m = make_config(cfg)
    kT = 0.1
    q = m.nblk
    ranges = [(0, 2), (q // 2, q // 2 + 2), (q - 2, q)]
    cols = [j for a, b in ranges for j in range(a, b)]
    want = oracle.density_matrix_T(m, m.mu, kT, columns=cols, workers=6)
    K = torch.from_numpy(m.vals).cuda()
    D = torch.zeros_like(K)
    for a, b in ranges:
        with pkg.Plan.from_bsr(m, prec="fp64", kT=kT, columns=(a, b)) as plan:
            plan.sign(K, m.mu, out=D)
    got = D.cpu().numpy()
    mask = ~np.isnan(want)
    assert float(np.max(np.abs(got[mask] - want[mask]))) <= TOL["fp64"]


def test_mixed_plan_refused(pkg):
    m = small_case(n_mol=12, block=3, r_c=5.5, seed=9)
    with pytest.raises(pkg.SubmatError) as ei:
        pkg.Plan.from_bsr(m, prec="mixed", kT=0.1)
    assert ei.value.name == "UNSUPPORTED"


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 1e-4)])
@pytest.mark.parametrize("kT,mu", [(0.05, 0.02), (0.2, -0.1)])
def test_adjoint_matches_daleckii_krein(pkg, prec, tol, kT, mu):
    """Kbar from the polynomial on dual numbers against the oracle's
    Daleckii-Krein gradient with the Fermi function's divided differences;
    dN/dmu from the same pass against the oracle's."""
    import torch
    m = small_case(n_mol=20, block=4, r_c=5.5, seed=101)
    rng = np.random.default_rng(1)
    dbar = rng.standard_normal(m.vals.shape)
    want, dn_want = oracle.fermi_backward(m, dbar, mu, kT)
    with pkg.Plan.from_bsr(m, prec=prec, kT=kT) as plan:
        kbar, dn = plan.sign_backward(torch.from_numpy(m.vals).cuda(), mu, torch.from_numpy(dbar).cuda(),
                                      want_dn_dmu=True)
    got = kbar.cpu().numpy()
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    eps = 1e-12 if prec == "fp64" else 2e-6
    assert abs(dn - dn_want) <= 1e-8 * dn_want + eps * m.n / kT


def test_band_energy_gradient_matches_central_differences(pkg):
    """E = Tr(D K) at finite temperature through the autograd wrapper (the
    library's adjoint for the implicit part) against central differences of
    the GPU forward map, moving K_pq and K_qp together."""
    import torch
    m = small_case(n_mol=12, block=3, r_c=5.5, seed=33)
    kT, mu, h = 0.1, 0.0, 1e-5
    perm = torch.from_numpy(transpose_index(m)).cuda()
    with pkg.Plan.from_bsr(m, prec="fp64", kT=kT) as plan:
        K = torch.from_numpy(m.vals.copy()).cuda().requires_grad_(True)
        sign_fn = pkg.make_autograd_sign(plan)
        E = (sign_fn(K, mu) * K[perm]).sum()
        E.backward()
        grad = K.grad.cpu().numpy()
        rng = np.random.default_rng(4)
        tp = transpose_index(m)
        for p in rng.choice(m.vals.shape[0], 12, replace=False):
            q = int(tp[p])
            vals = []
            for d in (h, -h):
                v = m.vals.copy()
                v[p] += d
                if q != p:
                    v[q] += d
                Kd = torch.from_numpy(v).cuda()
                vals.append(float((plan.sign(Kd, mu) * Kd[perm]).sum()))
            fd = (vals[0] - vals[1]) / (2 * h)
            an = grad[p] + (grad[q] if q != p else 0.0)
            assert abs(an - fd) <= 1e-6 * max(1.0, abs(fd)), (p, an, fd)
