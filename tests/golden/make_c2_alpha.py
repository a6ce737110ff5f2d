"""Writes oracle_c2_alpha.json: the oracle's 3x3 polarizability of the Nk=5 chain workload.

Workload: Nk = 5, nocc = 8, nvir = 40, naux = 160, seed 1266 (synth.CONFIGS["c2"]), the full
3x3 alpha tensor at w = 0, 0.05 and 0.1 Ha in the symmetric form of Eq. 15, complex128
throughout.  Every value comes from oracle/rcc.py on synth/ inputs:

  * ground state: CCSD amplitudes (Eqs. 7-8) to max|Omega| <= 1e-10 and the Lambda
    multipliers (Eqs. 10-11) to max|grad L| <= 1e-10 (Jacobi + DIIS, Sec. II.D);
  * perturbed amplitudes (Eqs. 13-14) for the 15 systems (3 components x {0, +-0.05, +-0.1})
    to a relative residual <= 1e-11;
  * alpha from eta and F vectors (rcc.polarizability_vectors' formula, rcc.symmetric_alpha).

It takes hours of CPU time, so each stage is cached under tests/golden/cache/ (not part of
the repository) and a rerun resumes where the last one stopped.  Besides alpha the fixture
keeps the CCSD energy per cell and a seeded sample of T and Lambda elements in the paper's
normalization (t2 and lambda2 carry the factor Nk; lambda as the paper's multipliers), so
that a GPU ground state can be compared element by element.

    python tests/golden/make_c2_alpha.py [threads]      # from the repository root
"""
import json
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from synth import make_problem, CONFIGS  # noqa: E402
from oracle import rcc  # noqa: E402

CACHE = os.path.join(HERE, "cache", "c2_seed1266")
COMPS = (0, 1, 2)
OMEGAS = (0.0, 0.05, 0.1)
GS_TOL = 1e-10
RESP_TOL = 1e-11
NSAMPLE = 64


def _path(name):
    return os.path.join(CACHE, name + ".pt")


def staged(name, fn):
    """Run fn() once and keep its result (tensors / tuples of tensors) in the cache."""
    p = _path(name)
    if os.path.exists(p):
        return torch.load(p)
    t0 = time.time()
    out = fn()
    torch.save(out, p + ".tmp")
    os.replace(p + ".tmp", p)
    print(f"[{time.strftime('%H:%M:%S')}] {name}: {time.time() - t0:.0f} s", flush=True)
    return out


def paper_lambda(nk, l1, l2):
    """Oracle multipliers (plain pairing, supercell units) -> the paper's Lambda: the
    alpha-beta block of the spin-orbital multipliers, paper units."""
    sw = torch.zeros_like(l2)
    for ki in range(nk):
        for kj in range(nk):
            for ka in range(nk):
                sw[ki, kj, ka] = l2[ki, kj, (ki + kj - ka) % nk].transpose(2, 3)
    return l1 / 2.0, nk * (2.0 * l2 + sw) / 3.0


def _cplx(z):
    z = complex(z)
    return [z.real, z.imag]


def main():
    if len(sys.argv) > 1:
        torch.set_num_threads(int(sys.argv[1]))
    os.makedirs(CACHE, exist_ok=True)
    c = CONFIGS["c2"]
    nk, o, v, Q = c["nk"], c["nocc"], c["nvir"], c["naux"]
    p = make_problem(nk, o, v, Q, seed=1266)
    R = rcc.RCC(p)
    t0 = time.time()

    def ccsd():
        t1, t2, it = rcc.solve_ccsd(R, tol=GS_TOL, verbose=True)
        return t1, t2, torch.tensor(it)

    t1, t2, it_cc = staged("ccsd", ccsd)

    def lam():
        l1, l2, it = rcc.solve_lambda(R, t1, t2, tol=GS_TOL, verbose=True)
        return l1, l2, torch.tensor(it)

    l1, l2, it_l = staged("lambda", lam)
    mus = rcc.dipole_ops(p, COMPS)
    xis = [staged(f"xi{c}", lambda m=m: rcc.perturbation_rhs(R, t1, t2, m)) for c, m in zip(COMPS, mus)]
    etas = [staged(f"eta{c}", lambda m=m: rcc.eta_vector(R, t1, t2, l1, l2, m)) for c, m in zip(COMPS, mus)]

    iters = {}

    def resp(ic, w):
        def run():
            x1, x2, it = rcc.solve_response(R, t1, t2, *xis[ic], w, RESP_TOL, verbose=True)
            return x1, x2, torch.tensor(it)
        x1, x2, it = staged(f"t{COMPS[ic]}_w{w:+.3f}", run)
        iters[f"{COMPS[ic]},{w:+.3f}"] = int(it)
        return x1, x2

    def fvec(ic, w, x):
        return staged(f"F{COMPS[ic]}_w{w:+.3f}", lambda: rcc.F_vector(R, t1, t2, l1, l2, *x))

    alpha = []
    for w in OMEGAS:
        nc = len(COMPS)
        tp = [resp(ic, w) for ic in range(nc)]
        tm = [resp(ic, -w) for ic in range(nc)] if w != 0 else tp
        ftp = [fvec(ic, w, tp[ic]) for ic in range(nc)]
        ftm = [fvec(ic, -w, tm[ic]) for ic in range(nc)] if w != 0 else ftp
        alpha.append(rcc.symmetric_alpha(nk, etas, tp, tm, ftp, ftm))
    alpha = np.asarray(alpha)

    # seeded sample of ground-state elements, paper normalization
    rng = np.random.default_rng(2508)
    pl1, pl2 = paper_lambda(nk, l1, l2)
    T2 = t2 * nk
    s1 = [tuple(int(rng.integers(0, n)) for n in t1.shape) for _ in range(NSAMPLE)]
    s2 = [tuple(int(rng.integers(0, n)) for n in t2.shape) for _ in range(NSAMPLE)]
    sample = {
        "t1": [[list(i), _cplx(t1[i])] for i in s1],
        "t2": [[list(i), _cplx(T2[i])] for i in s2],
        "l1": [[list(i), _cplx(pl1[i])] for i in s1],
        "l2": [[list(i), _cplx(pl2[i])] for i in s2],
    }
    out = {
        "source": "oracle/rcc.py on synth.make_problem(5, 8, 40, 160, seed=1266); written by "
                  "tests/golden/make_c2_alpha.py",
        "units": "hartree (energy), a.u. per cell (alpha); amplitudes in the paper's normalization",
        "nk": nk, "nocc": o, "nvir": v, "naux": Q, "seed": 1266,
        "comps": list(COMPS), "omegas": list(OMEGAS),
        "tolerances": {"ccsd_max_abs_residual": GS_TOL, "lambda_max_abs_gradient": GS_TOL,
                       "response_relative_residual": RESP_TOL},
        "iterations": {"ccsd": int(it_cc), "lambda": int(it_l), "response": iters},
        "energy_per_cell": _cplx(R.energy(t1, t2) / nk),
        "alpha": [[[_cplx(x) for x in row] for row in blk] for blk in alpha],
        "ground_state_sample": sample,
        "cpu_seconds_this_run": round(time.time() - t0, 1),
        "threads": torch.get_num_threads(),
    }
    with open(os.path.join(HERE, "oracle_c2_alpha.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print("alpha", alpha.real)


if __name__ == "__main__":
    main()
