"""LR excitation energies on the GPU (Davidson on Jacobian products) against the
oracle's dense Jacobian eigenvalues, and eigen-residuals of the returned vectors checked
with an independent product."""
import numpy as np
import pytest
import torch

from synth import make_problem, random_amplitudes, CONFIGS
from oracle import rcc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lr():
    import __graft_entry__ as g
    g.build()
    import paper_2508_01266_gb300 as m
    return m


@pytest.mark.parametrize("nk,o,v,Q,nroots", [(1, 1, 3, 4, 3), (2, 1, 3, 5, 4), (2, 2, 3, 4, 5), (3, 1, 2, 3, 2)])
def test_excitation_energies_vs_oracle(lr, nk, o, v, Q, nroots):
    p = make_problem(nk, o, v, Q, seed=81, sigma_l=0.15)
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
    ref = rcc.excitation_energies(R, t1, t2, nroots)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2 * nk)
    om, _, _, info = prob.excitation_energies(nroots, lr.default_options(conv_tol=1e-9, max_iter=200))
    assert info[1] == 0
    print("GPU", om, "oracle", ref)
    assert np.abs(om - ref).max() < 1e-8 * np.abs(ref).max()
    prob.close()


def test_excitation_vectors_c1(lr):
    """C1 workload: the returned right eigenvectors satisfy A x = omega x (checked with a
    separate product call) and the roots lie below the singles denominators' range."""
    c = CONFIGS["c1"]
    nk, o, v, Q = c["nk"], c["nocc"], c["nvir"], c["naux"]
    p = make_problem(nk, o, v, Q, seed=1266)
    t1, t2 = random_amplitudes(nk, o, v, seed=1267, scale1=0.01, scale2=0.01)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2 * nk)
    nroots = 4
    om, x1, x2, info = prob.excitation_energies(nroots, lr.default_options(conv_tol=1e-8, max_iter=200),
                                                vectors=True)
    assert info[1] == 0
    y1, y2 = prob.jacobian_apply(x1, x2)
    for r in range(nroots):
        res = torch.sqrt((y1[r] - om[r] * x1[r]).abs().pow(2).sum() + (y2[r] - om[r] * x2[r]).abs().pow(2).sum())
        assert float(res) < 1e-7
    d1 = np.array([[p.eps[k][o + a] - p.eps[k][i] for i in range(o) for a in range(v)] for k in range(nk)])
    assert om.real.min() > 0 and om.real.max() < d1.max()
    prob.close()
