"""Host-side test (no GPU): the comparison of the simulated op list with the oracle
catches a wrong op anywhere in the Jacobian programs.

For every op of the forward and transposed Jacobian programs, the op list is simulated on
the CPU once without that op and once with its coefficient negated (zero ops: removed
only); each variant must disagree with the oracle's product.  Scratch and workspace start
as NaN in the simulation, so a missing zero op or W-block build shows up as a non-finite
result.  A passing run means every op is load-bearing and its sign is pinned by the
oracle."""
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
    return max(np.abs(y1 - r1).max() / np.abs(r1).max(), np.abs(y2 - r2).max() / np.abs(r2).max())


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
