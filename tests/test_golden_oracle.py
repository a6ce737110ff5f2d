"""The oracle reproduces its stored fixture (tests/golden/oracle_small.json, written by
tests/golden/make_golden.py from oracle/ alone): a regression guard on the checker itself.
A change to the oracle's arithmetic that moves these values must be justified by the paper
and the fixture rewritten by the script."""
import glob
import json
import os
import sys

import numpy as np
import pytest

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


@pytest.mark.parametrize("name", sorted(os.path.basename(p) for p in glob.glob(os.path.join(GOLDEN, "oracle_c2_alpha*.json"))))
def test_c2_fixture_is_consistent(name):
    """The stored Nk=5 chain results (tests/golden/oracle_c2_alpha*.json, make_c2_alpha.py; too
    slow to recompute here) describe the workload they name and obey what Eq. 15 fixes for a
    time-reversal-symmetric problem below its first excitation: alpha is real, symmetric in its
    two components, and grows with the frequency (normal dispersion)."""
    from synth import CONFIGS
    with open(os.path.join(GOLDEN, name)) as f:
        d = json.load(f)
    c = CONFIGS["c2"]
    assert (d["nk"], d["nocc"], d["nvir"], d["naux"], d["seed"]) == (c["nk"], c["nocc"], c["nvir"], c["naux"], 1266)
    a = _c(d["alpha"])
    assert a.shape == (len(d["omegas"]), len(d["comps"]), len(d["comps"]))
    assert np.abs(a.imag).max() < 1e-8 * np.abs(a).max()
    assert np.abs(a - a.transpose(0, 2, 1)).max() < 1e-8 * np.abs(a).max()
    order = np.argsort(d["omegas"])
    diag = np.einsum("wcc->wc", a.real)[order]
    assert (np.diff(diag, axis=0) > 0).all() and (diag > 0).all()
    assert _c(d["energy_per_cell"]).real < 0
    for name in ("t1", "t2", "l1", "l2"):
        assert len(d["ground_state_sample"][name]) == 64
