"""Adjoint path: the autograd.Function around the Jacobian product.

Its backward (the transpose product of the Lambda equations, as a complex VJP) is
checked against the oracle's transpose product, against central finite differences of
the forward product (h = 1e-5, FP64) on random probe vectors, and by torch's
gradcheck on a tiny case; at the adjoint workload's full size (Nk=7, nocc=10,
nvir=56, naux=240) by the finite-difference identity.
"""
import numpy as np
import pytest
import torch

from synth import make_problem, random_amplitudes, random_probe, CONFIGS
from oracle import rcc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lr():
    import __graft_entry__ as g
    g.build()
    import paper_2508_01266_gb300 as m
    return m


def _problem(lr, nk, o, v, Q, seed=21, sigma=0.1, tscale=0.02):
    p = make_problem(nk, o, v, Q, seed=seed, sigma_l=sigma)
    t1, t2 = random_amplitudes(nk, o, v, seed=seed + 1, scale1=tscale, scale2=tscale)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2 * nk)
    return p, prob, t1, t2


def _inner(a1, a2, b1, b2):
    """<a, b> = sum conj(a) b over both blocks."""
    return complex((a1.conj() * b1).sum() + (a2.conj() * b2).sum())


def _fd_check(lr, prob, nk, o, v, seed, h=1e-5):
    dev = torch.device("cuda")
    x1, x2 = random_probe(nk, o, v, seed=seed, nrhs=1)
    u1, u2 = random_probe(nk, o, v, seed=seed + 1, nrhs=1)
    g1, g2 = random_probe(nk, o, v, seed=seed + 2, nrhs=1)
    X1 = torch.as_tensor(x1, device=dev).requires_grad_(True)
    X2 = torch.as_tensor(x2 * nk, device=dev).requires_grad_(True)
    U1, U2 = torch.as_tensor(u1, device=dev), torch.as_tensor(u2 * nk, device=dev)
    G1, G2 = torch.as_tensor(g1, device=dev), torch.as_tensor(g2, device=dev)
    y1, y2 = lr.jacobian(prob, X1, X2)
    b1, b2 = torch.autograd.grad((y1, y2), (X1, X2), grad_outputs=(G1, G2))
    with torch.no_grad():
        p1, p2 = lr.jacobian(prob, X1 + h * U1, X2 + h * U2)
        m1, m2 = lr.jacobian(prob, X1 - h * U1, X2 - h * U2)
        fd1, fd2 = (p1 - m1) / (2 * h), (p2 - m2) / (2 * h)
    lhs = _inner(G1, G2, fd1, fd2)   # <g, (A(x+hu) - A(x-hu)) / 2h>
    rhs = _inner(b1, b2, U1, U2)     # <A^H g, u>
    return lhs, rhs


@pytest.mark.parametrize("nk,o,v,Q", [(2, 1, 3, 5), (3, 2, 4, 6), (3, 4, 16, 48)])
def test_backward_vs_oracle_transpose(lr, nk, o, v, Q):
    p, prob, t1, t2 = _problem(lr, nk, o, v, Q)
    dev = torch.device("cuda")
    x1, x2 = random_amplitudes(nk, o, v, seed=31, scale1=1.0, scale2=1.0)
    g1, g2 = random_amplitudes(nk, o, v, seed=32, scale1=1.0, scale2=1.0)
    X1 = torch.as_tensor(x1, device=dev)[None].requires_grad_(True)
    X2 = torch.as_tensor(x2 * nk, device=dev)[None].requires_grad_(True)
    y1, y2 = lr.jacobian(prob, X1, X2)
    G1 = torch.as_tensor(g1, device=dev)[None]
    G2 = torch.as_tensor(g2, device=dev)[None]
    b1, b2 = torch.autograd.grad((y1, y2), (X1, X2), grad_outputs=(G1, G2))
    # oracle: A_paper^T w = D_in A^T D_out w (supercell units: x2_paper = Nk x2), here with
    # w = conj(g) given in paper units
    R = rcc.RCC(p)
    T = torch.as_tensor
    o1, o2 = R.transpose(T(t1), T(t2), T(g1.conj()), T(g2.conj() * nk))
    r1, r2 = o1.numpy().conj(), (o2.numpy() / nk).conj()
    e1 = np.abs(b1[0].cpu().numpy() - r1).max() / np.abs(r1).max()
    e2 = np.abs(b2[0].cpu().numpy() - r2).max() / np.abs(r2).max()
    assert e1 < 1e-12 and e2 < 1e-12


@pytest.mark.parametrize("nk,o,v,Q", [(2, 1, 3, 5), (3, 4, 16, 48)])
def test_backward_central_differences(lr, nk, o, v, Q):
    _, prob, _, _ = _problem(lr, nk, o, v, Q)
    lhs, rhs = _fd_check(lr, prob, nk, o, v, seed=41)
    assert abs(lhs - rhs) < 1e-8 * abs(rhs)


def test_gradcheck_tiny(lr):
    nk, o, v, Q = 2, 1, 2, 3
    _, prob, _, _ = _problem(lr, nk, o, v, Q)
    dev = torch.device("cuda")
    x1, x2 = random_probe(nk, o, v, seed=51, nrhs=1)
    X1 = torch.as_tensor(x1, device=dev).requires_grad_(True)
    X2 = torch.as_tensor(x2, device=dev).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a, b: lr.jacobian(prob, a, b), (X1, X2), eps=1e-6, atol=1e-8, rtol=1e-6)


@pytest.mark.slow
def test_backward_central_differences_adjoint_workload(lr):
    """Full size of the adjoint workload (Nk=7, nocc=10, nvir=56, naux=240)."""
    c = CONFIGS["c5"]
    nk, o, v, Q = c["nk"], c["nocc"], c["nvir"], c["naux"]
    _, prob, _, _ = _problem(lr, nk, o, v, Q, seed=1266, sigma=0.02, tscale=0.01)
    lhs, rhs = _fd_check(lr, prob, nk, o, v, seed=61)
    print("adjoint workload: <g, FD> =", lhs, " <A^H g, u> =", rhs)
    assert abs(lhs - rhs) < 1e-8 * abs(rhs)
    prob.close()
