"""The oracle still reproduces its stored regression values."""
import json
import os

import numpy as np

import oracle
from synth import make_config, random_symmetric_bsr

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_oracle_regression_fixture():
    with open(os.path.join(HERE, "oracle_regression.json")) as f:
        gold = json.load(f)
    g = gold["uneven_blocks_seed21_mu0.1"]
    m = random_symmetric_bsr([2, 3, 1, 4, 2, 3], density=0.45, seed=21)
    d = oracle.density_matrix(m, 0.1)
    assert np.max(np.abs(d - np.array(g["D_vals"]))) < 1e-12
    assert abs(oracle.trace_bsr(m, d) - g["trace"]) < 1e-12
    g0 = gold["water32_b6_rc6_mu0"]
    m0 = make_config(0)
    d0 = oracle.density_matrix(m0, 0.0)
    assert abs(oracle.trace_bsr(m0, d0) - g0["trace"]) < 1e-9
    assert abs(oracle.band_energy(m0, d0) - g0["band_energy"]) < 1e-9
