"""Write the oracle regression fixtures in this folder.

Calls only ``oracle/`` (and the seeded input generator).  The paper prints no
worked example with values (its only numbers are timings and iteration
counts, Section VI-A, Table prec), so these fixtures pin the oracle against
later drift, not against the paper; the pins against the mathematics live
in ``tests/test_oracle_pins.py``.

Run: ``python tests/golden/make_golden.py`` from the repository root.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from synth import make_config, random_symmetric_bsr  # noqa: E402


def main():
    out = {}
    m = random_symmetric_bsr([2, 3, 1, 4, 2, 3], density=0.45, seed=21)
    d = oracle.density_matrix(m, 0.1)
    out["uneven_blocks_seed21_mu0.1"] = {
        "recipe": "synth.random_symmetric_bsr([2,3,1,4,2,3], density=0.45, seed=21), mu=0.1",
        "D_vals": [float(x) for x in d],
        "trace": oracle.trace_bsr(m, d),
    }
    m0 = make_config(0)
    d0 = oracle.density_matrix(m0, 0.0)
    out["water32_b6_rc6_mu0"] = {
        "recipe": "synth.make_config(0): 32 molecules, block 6, cutoff 6 A, seed 1000, mu=0",
        "trace": oracle.trace_bsr(m0, d0),
        "D_first_block_column_sum": float(np.nansum(d0[:36])),
        "band_energy": oracle.band_energy(m0, d0),
    }
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
