"""Ground state on the GPU: the residual evaluated from Jacobian products (exact
two-point Gauss-Legendre identity), CCSD amplitudes and Lambda multipliers against the
oracle's converged ones, and alpha from a ground state solved entirely on the GPU."""
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


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("nk,o,v,Q", [(1, 2, 3, 4), (2, 2, 3, 4), (3, 4, 16, 48)])
def test_residual_vs_oracle(lr, nk, o, v, Q):
    p = make_problem(nk, o, v, Q, seed=71, sigma_l=0.15)
    t1, t2 = random_amplitudes(nk, o, v, seed=72, scale1=0.05, scale2=0.05)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    dev = torch.device("cuda")
    r1, r2 = prob.residual(torch.as_tensor(t1, device=dev), torch.as_tensor(t2 * nk, device=dev))
    R = rcc.RCC(p)
    T = torch.as_tensor
    o1, o2 = R.residual(T(t1), T(t2))
    assert _rel(r1.cpu().numpy(), o1.numpy()) < 1e-12
    assert _rel(r2.cpu().numpy(), nk * o2.numpy()) < 1e-12
    prob.close()


@pytest.mark.parametrize("nk,o,v,Q", [(2, 2, 3, 4), (3, 2, 5, 8)])
def test_ground_state_vs_oracle(lr, nk, o, v, Q):
    from test_gpu_alpha import paper_lambda
    p = make_problem(nk, o, v, Q, seed=73, sigma_l=0.15)
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-12)
    pl1, pl2 = paper_lambda(nk, l1, l2)
    e_ref = complex(R.energy(t1, t2)) / nk
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    g1, g2, h1, h2, e, info = prob.solve_ground_state(lr.default_options(conv_tol=1e-12, max_iter=300))
    assert info[1] == 0 and info[3] == 0
    assert _rel(g1.cpu().numpy(), t1.numpy()) < 1e-9
    assert _rel(g2.cpu().numpy(), nk * t2.numpy()) < 1e-9
    assert _rel(h1.cpu().numpy(), pl1.numpy()) < 1e-9
    assert _rel(h2.cpu().numpy(), pl2.numpy()) < 1e-9
    assert abs(e - e_ref.real) < 1e-11 * abs(e_ref)
    prob.close()


def test_alpha_c1_from_gpu_ground_state(lr):
    """C1 workload end to end on the GPU: T, Lambda and alpha_zz(0, 0.1) vs the oracle."""
    c = CONFIGS["c1"]
    nk, o, v, Q = c["nk"], c["nocc"], c["nvir"], c["naux"]
    p = make_problem(nk, o, v, Q, seed=1266)
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-10)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-10)
    ref = rcc.polarizability(R, t1, t2, l1, l2, rcc.dipole_ops(p, [2]), [0.0, 0.1], tol=1e-11)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    *_, e, info = prob.solve_ground_state(lr.default_options(conv_tol=1e-11, max_iter=300))
    assert info[1] == 0 and info[3] == 0
    got, info = prob.polarizability([2], [0.0, 0.1], lr.default_options(conv_tol=1e-11, max_iter=300))
    assert info[1] == 0
    rel = np.abs(got - ref).max() / np.abs(ref).max()
    print("C1 alpha_zz from GPU ground state", got.ravel(), "oracle", ref.ravel(), "rel", rel)
    assert rel < 1e-8
    prob.close()


@pytest.mark.parametrize("prec", [2, 1])
def test_mixed_precision_ground_state_vs_oracle(lr, prec):
    """Tensor-core inner solves (inexact Newton for T, iterative refinement for Lambda) reach
    the oracle's ground state to the FP64 tolerances given: the FP64 residual decides."""
    from test_gpu_alpha import paper_lambda
    nk, o, v, Q = 3, 2, 5, 8
    p = make_problem(nk, o, v, Q, seed=73, sigma_l=0.15)
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-12)
    pl1, pl2 = paper_lambda(nk, l1, l2)
    e_ref = complex(R.energy(t1, t2)) / nk
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    g1, g2, h1, h2, e, info = prob.solve_ground_state(
        lr.default_options(precision=prec, conv_tol=1e-11, refine_tol=1e-11, max_iter=300))
    print(f"precision {prec}: Newton steps {info[0]}, Lambda iterations {info[2]}")
    assert info[1] == 0 and info[3] == 0
    assert info[0] <= 8
    assert _rel(g1.cpu().numpy(), t1.numpy()) < 1e-8
    assert _rel(g2.cpu().numpy(), nk * t2.numpy()) < 1e-8
    assert _rel(h1.cpu().numpy(), pl1.numpy()) < 1e-8
    assert _rel(h2.cpu().numpy(), pl2.numpy()) < 1e-8
    assert abs(e - e_ref.real) < 1e-10 * abs(e_ref)
    prob.close()


def test_alpha_c1_mixed_end_to_end(lr):
    """C1 workload, everything in BF16x3 with FP64 refinement (ground state and alpha):
    alpha_zz(0, 0.1) within 1e-5 a.u. of the oracle."""
    c = CONFIGS["c1"]
    nk, o, v, Q = c["nk"], c["nocc"], c["nvir"], c["naux"]
    p = make_problem(nk, o, v, Q, seed=1266)
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-10)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-10)
    ref = rcc.polarizability(R, t1, t2, l1, l2, rcc.dipole_ops(p, [2]), [0.0, 0.1], tol=1e-11)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    opts = lr.default_options(precision=2, conv_tol=1e-9, refine_tol=1e-8, max_iter=300)
    *_, e, info = prob.solve_ground_state(opts)
    assert info[1] == 0 and info[3] == 0
    got, info = prob.polarizability([2], [0.0, 0.1], opts)
    assert info[1] == 0
    err = np.abs(got - ref).max()
    print("C1 alpha_zz, BF16x3 end to end", got.ravel(), "oracle", ref.ravel(), "|err|", err)
    assert err <= 1e-5
    prob.close()
