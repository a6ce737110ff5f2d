"""Host-side test (no GPU): the comparison of the simulated op lists with the oracle
catches a wrong op anywhere in the library's programs.

For every op of the forward and transposed Jacobian programs, the perturbation
right-hand side, singles Hessian, zero-amplitude residual and energy-gradient programs,
and the ground-state program that builds their intermediates, the op list is simulated on
the CPU once without that op and once with its coefficient negated (zero ops: removed
only); each variant must disagree with the oracle.  Scratch and workspace start as NaN in
the simulation, so a missing zero op or W-block build shows up as a non-finite result.  A
passing run means every op is load-bearing and its sign is pinned by the oracle."""
import numpy as np
import pytest
import torch

from synth import make_problem, random_amplitudes
from oracle import rcc
import test_host_plan as th


def _deviation(pv, ar, which, prog, x1, x2p, r1, r2):
    save = pv.programs[which]
    pv.programs[which] = prog
    try:
        y1, y2 = th._sim_apply(pv, ar, x1, x2p, which)
    finally:
        pv.programs[which] = save
    if not (np.isfinite(y1).all() and np.isfinite(y2).all()):
        return float("inf")
    # one scale for both parts: some references have an identically zero part
    # (singles of the residual at zero amplitudes, doubles of the singles Hessian)
    scale = max(np.abs(r1).max(), np.abs(r2).max())
    return max(np.abs(y1 - r1).max(), np.abs(y2 - r2).max()) / scale


@pytest.mark.parametrize("nk,o,v,Q", [(2, 1, 2, 3), (3, 2, 3, 4)])
def test_every_op_is_pinned_by_the_oracle(nk, o, v, Q):
    import __graft_entry__ as g
    g.build()
    from paper_2508_01266_gb300._lib import lib
    p = make_problem(nk, o, v, Q, seed=3, sigma_l=0.2)
    R = rcc.RCC(p)
    T = torch.as_tensor
    t1, t2 = random_amplitudes(nk, o, v, seed=4, scale1=0.05, scale2=0.05)
    pv, ar = th._sim_setup(lib, p, t1, t2, 1 << 20)
    x1, x2 = random_amplitudes(nk, o, v, seed=5, scale1=1, scale2=1)
    f1, f2 = R.jacobian(T(t1), T(t2), T(x1), T(x2))
    g1, g2 = random_amplitudes(nk, o, v, seed=6, scale1=1, scale2=1)
    b1, b2 = R.transpose(T(t1), T(t2), T(g1), T(g2 * nk))
    cases = {1: (x1, x2 * nk, f1.numpy(), f2.numpy() * nk),   # A.X, paper units
             2: (g1, g2, b1.numpy(), b2.numpy() / nk)}        # P_sym A^T.G
    for which, (u1, u2, r1, r2) in cases.items():
        ops = pv.programs[which]
        assert _deviation(pv, ar, which, ops, u1, u2, r1, r2) < 1e-12
        missed = []
        for i, (kind, fixed, d) in enumerate(ops):
            for mut in ("drop", "negate"):
                if mut == "negate" and kind == "zero":
                    continue
                prog = list(ops)
                if mut == "drop":
                    del prog[i]
                else:
                    d2 = dict(d)
                    d2["alpha"] = -d["alpha"]
                    prog[i] = (kind, fixed, d2)
                if _deviation(pv, ar, which, prog, u1, u2, r1, r2) < 1e-9:
                    missed.append((which, i, kind, mut))
        assert len(ops) > 50
        assert not missed, missed


def _mutants(ops):
    for i, (kind, fixed, d) in enumerate(ops):
        for mut in ("drop", "negate"):
            if mut == "negate" and kind == "zero":
                continue
            prog = list(ops)
            if mut == "drop":
                del prog[i]
            else:
                d2 = dict(d)
                d2["alpha"] = -d["alpha"]
                prog[i] = (kind, fixed, d2)
            yield i, kind, mut, prog


@pytest.mark.parametrize("nk,o,v,Q", [(2, 2, 3, 3), (3, 1, 2, 4)])
def test_every_op_of_the_rhs_hessian_and_gradient_programs_is_pinned(nk, o, v, Q):
    """The same sweep over the perturbation right-hand side (Eq. 12), the singles energy
    Hessian, the residual at zero amplitudes and the energy gradient programs, each against
    the oracle's vector (the Hessian's by an exact central difference of the oracle's
    energy gradient, which is linear in the singles)."""
    import __graft_entry__ as g
    g.build()
    from paper_2508_01266_gb300._lib import lib
    T = torch.as_tensor
    p = make_problem(nk, o, v, Q, seed=8, sigma_l=0.2)
    R = rcc.RCC(p)
    t1, t2 = random_amplitudes(nk, o, v, seed=9, scale1=0.05, scale2=0.05)
    pv, ar = th._sim_setup(lib, p, t1, t2, 1 << 20)
    mu = p.dip[2]
    th._put_mu(pv, ar, mu, o)
    z1 = np.zeros((nk, o, v), complex)
    z2 = np.zeros((nk,) * 3 + (o, o, v, v), complex)
    x1, x2 = rcc.perturbation_rhs(R, T(t1), T(t2), T(mu))
    r1, r2 = R.residual(T(z1), T(z2))
    e1, e2 = R.energy_grad(T(t1), T(t2))
    u1, _ = random_amplitudes(nk, o, v, seed=10, scale1=1, scale2=1)
    h = 1e-2
    gp, _ = R.energy_grad(T(t1 + h * u1), T(t2))
    gm, _ = R.energy_grad(T(t1 - h * u1), T(t2))
    hu = ((gp - gm) / (2 * h)).numpy()
    cases = {3: (t1, t2 * nk, x1.numpy(), nk * x2.numpy()),
             4: (u1, z2, hu, np.zeros_like(z2)),
             5: (z1, z2, r1.numpy(), nk * r2.numpy()),
             6: (t1, t2 * nk, e1.numpy(), e2.numpy() / nk)}
    for which, (a1, a2, ref1, ref2) in cases.items():
        ops = pv.programs[which]
        assert _deviation(pv, ar, which, ops, a1, a2, ref1, ref2) < 1e-12
        missed = [(which, i, kind, mut) for i, kind, mut, prog in _mutants(ops)
                  if _deviation(pv, ar, which, prog, a1, a2, ref1, ref2) < 1e-9]
        assert not missed, missed


def _inputs(pv, p, t1, t2):
    """The fixed arena as the library receives it, before the ground-state program."""
    nk, o, v = p.nk, p.nocc, p.nvir
    ar = [np.zeros(int(s), np.complex128) for s in pv.arena_sizes]
    off, L, F = pv.offsets, p.L / np.sqrt(nk), ar[0]

    def put(o_, x):
        F[o_:o_ + x.size] = x.ravel()
    put(off[0], L[:, :, :, :o, :o])
    put(off[1], L[:, :, :, :o, o:])
    put(off[2], L[:, :, :, o:, :o])
    put(off[3], L[:, :, :, o:, o:])
    f0 = np.zeros((nk, o + v, o + v), complex)
    for k in range(nk):
        f0[k] = np.diag(p.eps[k])
    put(off[4], f0)
    put(off[5], t1)
    put(off[6], t2 * nk)
    put(off[7], np.eye(o))
    return ar


@pytest.mark.parametrize("nk,o,v,Q", [(2, 2, 3, 3), (3, 1, 2, 4)])
def test_every_ground_state_op_is_pinned(nk, o, v, Q):
    """The ground-state program (the T-dependent intermediates every other program reads):
    each op removed or negated in turn, the intermediates rebuilt and the Jacobian,
    transposed, right-hand-side and gradient programs compared with the oracle.  Ops that
    leave the state unchanged where they run (they add zeros for these inputs: the
    occupied-virtual blocks of the canonical Fock matrix diag(eps)) cannot be pinned and
    are exempt; they must be few and data movement only."""
    import __graft_entry__ as g
    g.build()
    from paper_2508_01266_gb300._lib import lib
    import plan_sim
    T = torch.as_tensor
    p = make_problem(nk, o, v, Q, seed=8, sigma_l=0.2)
    R = rcc.RCC(p)
    t1, t2 = random_amplitudes(nk, o, v, seed=9, scale1=0.05, scale2=0.05)
    pv, _ = th._sim_setup(lib, p, t1, t2, 1 << 20)
    mu = p.dip[2]
    x1, x2 = random_amplitudes(nk, o, v, seed=5, scale1=1, scale2=1)
    g1, g2 = random_amplitudes(nk, o, v, seed=6, scale1=1, scale2=1)
    f1, f2 = R.jacobian(T(t1), T(t2), T(x1), T(x2))
    b1, b2 = R.transpose(T(t1), T(t2), T(g1), T(g2 * nk))
    xi1, xi2 = rcc.perturbation_rhs(R, T(t1), T(t2), T(mu))
    e1, e2 = R.energy_grad(T(t1), T(t2))
    checks = [(1, x1, x2 * nk, f1.numpy(), f2.numpy() * nk), (2, g1, g2, b1.numpy(), b2.numpy() / nk),
              (3, t1, t2 * nk, xi1.numpy(), nk * xi2.numpy()), (6, t1, t2 * nk, e1.numpy(), e2.numpy() / nk)]
    base = _inputs(pv, p, t1, t2)

    def deviation(prog0):
        a = [x.copy() for x in base]
        a[3][:] = np.nan
        a[4][:] = np.nan
        plan_sim.run(prog0, a)
        th._put_mu(pv, a, mu, o)
        worst = 0.0
        for which, u1, u2, r1, r2 in checks:
            y1, y2 = th._sim_apply(pv, a, u1, u2, which)
            if not (np.isfinite(y1).all() and np.isfinite(y2).all()):
                return float("inf")
            worst = max(worst, np.abs(y1 - r1).max() / np.abs(r1).max(), np.abs(y2 - r2).max() / np.abs(r2).max())
        return worst

    ops = pv.programs[0]
    assert deviation(ops) < 1e-12
    # ops that change nothing where they run
    inert = set()
    state = [x.copy() for x in base]
    for i, op in enumerate(ops):
        before = [x.copy() for x in state]
        plan_sim.run([op], state)
        if all(np.array_equal(a_, b_, equal_nan=True) for a_, b_ in zip(before, state)):
            inert.add(i)
    assert len(inert) <= 2 * nk and all(ops[i][0] == "perm" for i in inert), sorted(inert)
    missed = [(i, kind, mut) for i, kind, mut, prog in _mutants(ops)
              if i not in inert and deviation(prog) < 1e-9]
    assert not missed, missed
