"""The oracle reproduces its stored fixture (tests/golden/oracle_small.json, written by
tests/golden/make_golden.py from oracle/ alone): a regression guard on the checker itself.
A change to the oracle's arithmetic that moves these values must be justified by the paper
and the fixture rewritten by the script."""
import json
import os
import sys

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)


def _c(a):
    a = np.asarray(a, dtype=np.float64)
    return a[..., 0] + 1j * a[..., 1]


def test_oracle_reproduces_fixture():
    import make_golden
    with open(os.path.join(GOLDEN, "oracle_small.json")) as f:
        stored = json.load(f)
    assert [tuple(c[k] for k in ("nk", "nocc", "nvir", "naux", "seed", "sigma_l")) for c in stored["cases"]] == \
        [tuple(c) for c in make_golden.CASES]
    for case, ref in zip(make_golden.CASES, stored["cases"]):
        got = make_golden.compute(case)
        assert abs(_c(got["energy_per_cell"]) - _c(ref["energy_per_cell"])) < 1e-10
        a, ar = _c(got["alpha"]), _c(ref["alpha"])
        assert np.abs(a - ar).max() < 1e-8 * np.abs(ar).max()
        w, wr = _c(got["excitation_energies"]), _c(ref["excitation_energies"])
        assert np.abs(w - wr).max() < 1e-9 * np.abs(wr).max()
        # alpha of a time-reversal-symmetric problem is real (Eq. 15)
        assert np.abs(ar.imag).max() < 1e-12 * np.abs(ar).max()
