"""Writes oracle_c2_alpha.json: the oracle's 3x3 polarizability of the Nk=5 chain workload.

Workload: Nk = 5, nocc = 8, nvir = 40, naux = 160, seed 1266 (synth.CONFIGS["c2"]), the full
3x3 alpha tensor at w = 0, 0.05 and 0.1 Ha in the symmetric form of Eq. 15, complex128
throughout.  Every value comes from oracle/rcc.py on synth/ inputs:

  * ground state: CCSD amplitudes (Eqs. 7-8) to max|Omega| <= 1e-10 and the Lambda
    multipliers (Eqs. 10-11) to max|grad L| <= 1e-10 (Jacobi + DIIS, Sec. II.D);
  * perturbed amplitudes (Eqs. 13-14) for the 15 systems (3 components x {0, +-0.05, +-0.1})
    to a relative residual <= 1e-11 (rcc.solve_response);
  * eta^X vectors (rcc.eta_vector), the quadratic-term scalars F(t^x(-w), t^y(w))
    (rcc.F_dot), and alpha from them (rcc.symmetric_alpha_from_scalars).

It takes hours of CPU time.  The independent pieces (one response system, one F scalar) run
in a pool of worker processes (each needs about 14 GB), the memory-heavy gradient stages
(Lambda, eta: about 55 GB) alone; every result is cached under tests/golden/cache/ (not part
of the repository), so a rerun resumes where the last one stopped.  Besides alpha the
fixture keeps the CCSD energy per cell and a seeded sample of T and Lambda elements in the
paper's normalization (t2 and lambda2 carry the factor Nk; lambda as the paper's
multipliers), so that a GPU ground state can be compared element by element.

    python tests/golden/make_c2_alpha.py [workers] [threads per worker] [components] [omegas] [output]

from the repo root; components as letters (default xyz), frequencies in Ha separated by commas
(default 0,0.05,0.1), output file name under tests/golden (default oracle_c2_alpha.json).  A
subset (say z and 0,0.1) writes alpha for those components and frequencies only; the fixture
records which.  Runs with different subsets share the cache.
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

CACHE = os.path.join(HERE, "cache", "c2_seed1266")
COMPS = (0, 1, 2)
OMEGAS = (0.0, 0.05, 0.1)
GS_TOL = 1e-10
RESP_TOL = 1e-11
NSAMPLE = 64


def _path(name):
    return os.path.join(CACHE, name + ".pt")


def tname(c, w):
    """Cache name of the response solution of component c at frequency w (w = -0 is 0)."""
    return f"t{c}_w{w + 0.0:+.3f}"


def _log(msg):
    print(f"[{time.strftime('%H:%M:%S')}] {msg}", flush=True)


def staged(name, fn):
    """Run fn() once and keep its result in the cache."""
    import torch
    p = _path(name)
    if os.path.exists(p):
        return torch.load(p)
    t0 = time.time()
    out = fn()
    torch.save(out, p + ".tmp")
    os.replace(p + ".tmp", p)
    _log(f"{name}: {time.time() - t0:.0f} s")
    return out


_W = {}


def _system():
    """The problem and its oracle object (per process)."""
    if "R" not in _W:
        from synth import make_problem, CONFIGS
        from oracle import rcc
        c = CONFIGS["c2"]
        p = make_problem(c["nk"], c["nocc"], c["nvir"], c["naux"], seed=1266)
        _W["p"], _W["R"] = p, rcc.RCC(p)
    return _W["p"], _W["R"]


def _init_worker(threads):
    import torch
    torch.set_num_threads(threads)


def _resp_task_iters(args):
    """One perturbed-amplitude system, (A - w) t = -xi^X, with its iteration count."""
    c, w = args
    import torch
    from oracle import rcc
    name = tname(c, w)
    if os.path.exists(_path(name)):
        return name
    p, R = _system()
    t1, t2, _ = torch.load(_path("ccsd"))
    xi = torch.load(_path(f"xi{c}"))

    def run():
        x1, x2, it = rcc.solve_response(R, t1, t2, *xi, w, RESP_TOL)
        return x1, x2, torch.tensor(it)

    staged(name, run)
    return name


def _grad_task(args):
    """The gradient stages (Lambda, Eqs. 10-11; eta^X) in a child process of their own: they
    peak near 55 GB, and memory the parent kept after them would be missing for the F pool."""
    kind, c = args
    import torch
    from oracle import rcc
    p, R = _system()
    t1, t2, _ = torch.load(_path("ccsd"))
    if kind == "lambda":
        def lam():
            l1, l2, it = rcc.solve_lambda(R, t1, t2, tol=GS_TOL)
            return l1, l2, torch.tensor(it)
        staged("lambda", lam)
    else:
        l1, l2, _ = torch.load(_path("lambda"))
        m = rcc.dipole_ops(p, (c,))[0]
        staged(f"eta{c}", lambda: rcc.eta_vector(R, t1, t2, l1, l2, m))
    return kind


def _in_child(ctx, threads, args):
    """Run _grad_task(args) in one spawned worker unless its result is cached."""
    name = "lambda" if args[0] == "lambda" else f"eta{args[1]}"
    if os.path.exists(_path(name)):
        return
    with ctx.Pool(1, initializer=_init_worker, initargs=(threads,)) as pool:
        pool.map(_grad_task, [args])


def _F_task(args):
    """F(t^x(-w), t^y(+w)), the quadratic term of Eq. 15 (rcc.F_dot)."""
    x, y, w = args
    import torch
    from oracle import rcc
    name = f"F{x}{y}_w{w:.3f}"
    if os.path.exists(_path(name)):
        return name
    p, R = _system()
    t1, t2, _ = torch.load(_path("ccsd"))
    l1, l2, _ = torch.load(_path("lambda"))
    um = torch.load(_path(tname(x, -w)))
    wp = torch.load(_path(tname(y, w)))
    staged(name, lambda: torch.tensor(complex(rcc.F_dot(R, t1, t2, l1, l2, um[0], um[1], wp[0], wp[1]))))
    return name


def paper_lambda(nk, l1, l2):
    """Oracle multipliers (plain pairing, supercell units) -> the paper's Lambda: the
    alpha-beta block of the spin-orbital multipliers, paper units."""
    import torch
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
    import torch
    from oracle import rcc
    workers = int(sys.argv[1]) if len(sys.argv) > 1 else 3
    wthreads = int(sys.argv[2]) if len(sys.argv) > 2 else 2
    global COMPS, OMEGAS
    if len(sys.argv) > 3:
        COMPS = tuple("xyz".index(ch) for ch in sys.argv[3])
    if len(sys.argv) > 4:
        OMEGAS = tuple(float(w) for w in sys.argv[4].split(","))
    outname = sys.argv[5] if len(sys.argv) > 5 else "oracle_c2_alpha.json"
    torch.set_num_threads(os.cpu_count() or 8)
    os.makedirs(CACHE, exist_ok=True)
    p, R = _system()
    nk = p.nk
    t0 = time.time()

    def ccsd():
        t1, t2, it = rcc.solve_ccsd(R, tol=GS_TOL)
        return t1, t2, torch.tensor(it)

    t1, t2, it_cc = staged("ccsd", ccsd)
    mus = rcc.dipole_ops(p, COMPS)
    for c, m in zip(COMPS, mus):
        staged(f"xi{c}", lambda m=m: rcc.perturbation_rhs(R, t1, t2, m))
    ctx = mp.get_context("spawn")
    # response systems (need T only)
    jobs = [(c, w) for w in OMEGAS for c in COMPS]
    jobs += [(c, -w) for w in OMEGAS if w != 0 for c in COMPS]
    todo = [j for j in jobs if not os.path.exists(_path(tname(j[0], j[1])))]
    if todo:
        _log(f"response systems: {len(todo)} on {workers} workers x {wthreads} threads")
        with ctx.Pool(workers, initializer=_init_worker, initargs=(wthreads,)) as pool:
            for name in pool.imap_unordered(_resp_task_iters, todo):
                _log(f"done {name}")

    nthreads = os.cpu_count() or 8
    _in_child(ctx, nthreads, ("lambda", None))
    for c in COMPS:
        _in_child(ctx, nthreads, ("eta", c))
    l1, l2, it_l = torch.load(_path("lambda"))
    etas = [torch.load(_path(f"eta{c}")) for c in COMPS]
    nc = len(COMPS)
    fjobs = []
    for w in OMEGAS:
        for x in range(nc):
            for y in range(nc):
                if w == 0 and y < x:
                    continue  # F is symmetric: F(t^x, t^y) = F(t^y, t^x) at w = 0
                fjobs.append((COMPS[x], COMPS[y], w))
    todo = [j for j in fjobs if not os.path.exists(_path(f"F{j[0]}{j[1]}_w{j[2]:.3f}"))]
    if todo:
        _log(f"F scalars: {len(todo)} on {workers} workers x {wthreads} threads")
        with ctx.Pool(workers, initializer=_init_worker, initargs=(wthreads,)) as pool:
            for name in pool.imap_unordered(_F_task, todo):
                _log(f"done {name}")

    alpha, iters = [], {}
    for w in OMEGAS:
        tp, tm = [], []
        for ic in range(nc):
            a = torch.load(_path(tname(COMPS[ic], w)))
            b = torch.load(_path(tname(COMPS[ic], -w)))
            tp.append(a[:2])
            tm.append(b[:2])
            iters[f"{COMPS[ic]},{w + 0.0:+.3f}"] = int(a[2])
            iters[f"{COMPS[ic]},{-w + 0.0:+.3f}"] = int(b[2])

        def F(x, y):
            if w == 0 and y < x:
                x, y = y, x
            return complex(torch.load(_path(f"F{COMPS[x]}{COMPS[y]}_w{w:.3f}")))

        Fmp = [[F(x, y) for y in range(nc)] for x in range(nc)]
        alpha.append(rcc.symmetric_alpha_from_scalars(nk, etas, tp, tm, Fmp))
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
        "nk": nk, "nocc": p.nocc, "nvir": p.nvir, "naux": p.naux, "seed": 1266,
        "comps": list(COMPS), "omegas": list(OMEGAS),
        "tolerances": {"ccsd_max_abs_residual": GS_TOL, "lambda_max_abs_gradient": GS_TOL,
                       "response_relative_residual": RESP_TOL},
        "iterations": {"ccsd": int(it_cc), "lambda": int(it_l), "response": iters},
        "energy_per_cell": _cplx(R.energy(t1, t2) / nk),
        "alpha": [[[_cplx(x) for x in row] for row in blk] for blk in alpha],
        "ground_state_sample": sample,
    }
    with open(os.path.join(HERE, outname), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    _log(f"alpha written ({time.time() - t0:.0f} s this run)")
    print(alpha.real)


if __name__ == "__main__":
    main()
