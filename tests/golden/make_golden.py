"""Writes oracle_small.json, the oracle regression fixture of this directory.

Every value in the fixture is computed by oracle/ on seeded synthetic inputs from synth/
(the paper prints no worked example that can be recomputed without its molecular
integrals).  The fixture pins nothing about the method; it freezes the oracle's output so
that a later change to the oracle's arithmetic shows up as a failing CPU test and must be
justified by the passage of the paper it follows.

    python tests/golden/make_golden.py     # from the repository root
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from synth import make_problem  # noqa: E402
from oracle import rcc  # noqa: E402

# (nk, nocc, nvir, naux, seed, sigma_l): a small periodic problem with interaction (two
# cells, four electrons in the supercell), alpha_zz only, cheap enough for the CPU suite
CASES = [(2, 1, 2, 3, 101, 0.2)]
COMPS = (2,)
OMEGAS = (0.0, 0.09)


def compute(case):
    nk, o, v, Q, seed, sig = case
    p = make_problem(nk, o, v, Q, seed=seed, sigma_l=sig)
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-12)
    e = complex(R.energy(t1, t2))
    a = rcc.polarizability(R, t1, t2, l1, l2, rcc.dipole_ops(p, COMPS), list(OMEGAS))
    w = np.sort_complex(np.asarray(rcc.excitation_energies(R, t1, t2)))[:4]
    return {"nk": nk, "nocc": o, "nvir": v, "naux": Q, "seed": seed, "sigma_l": sig,
            "comps": list(COMPS), "omegas": list(OMEGAS),
            "energy_per_cell": [e.real, e.imag],
            "alpha": [[[[complex(x).real, complex(x).imag] for x in row] for row in blk] for blk in np.asarray(a)],
            "excitation_energies": [[complex(x).real, complex(x).imag] for x in w]}


def main():
    out = {"source": "oracle/rcc.py on synth.make_problem inputs; written by tests/golden/make_golden.py",
           "units": "hartree (energies), a.u. per cell (alpha)",
           "cases": [compute(c) for c in CASES]}
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
