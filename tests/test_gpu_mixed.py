"""Tensor-core (tcgen05) Jacobian products against the FP64 products and the oracle.

TF32 keeps 10 mantissa bits per operand and BF16x3 about 16; both accumulate in FP32.
Bounds below are the expected rounding of the products relative to the largest
output element.
"""
import numpy as np
import pytest
import torch

from synth import make_problem, random_amplitudes, CONFIGS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lr():
    import __graft_entry__ as g
    g.build()
    import paper_2508_01266_gb300 as m
    return m


def _setup(lr, nk, o, v, Q, seed=11, sigma=0.1):
    p = make_problem(nk, o, v, Q, seed=seed, sigma_l=sigma)
    t1, t2 = random_amplitudes(nk, o, v, seed=seed + 1, scale1=0.02, scale2=0.02)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2 * nk)
    return prob


@pytest.mark.parametrize("nk,o,v,Q,sigma", [(2, 1, 3, 5, 0.1), (3, 2, 4, 6, 0.1), (3, 4, 16, 48, 0.1),
                                            (2, 8, 16, 40, 0.1), (5, 8, 40, 160, 0.02),
                                            (5, 4, 48, 60, 0.02)])
@pytest.mark.parametrize("prec,bound", [(1, 3e-3), (2, 5e-5)])
def test_mixed_products_vs_fp64(lr, nk, o, v, Q, sigma, prec, bound):
    """sigma: DF factor scale (0.02 is the workloads' value).  At (5, 4, 48, 60) the ladder
    contracts 5 x 48^2 = 11520 terms per output: the packed kernel sums it in two chunks."""
    prob = _setup(lr, nk, o, v, Q, sigma=sigma)
    dev = torch.device("cuda")
    x1, x2 = random_amplitudes(nk, o, v, seed=5, scale1=1.0, scale2=1.0)
    X1 = torch.as_tensor(x1, device=dev)[None].contiguous()
    X2 = torch.as_tensor(x2 * nk, device=dev)[None].contiguous()
    for tr in (False, True):
        r1, r2 = prob.jacobian_apply(X1, X2, transpose=tr)
        m1, m2 = prob.jacobian_apply(X1, X2, transpose=tr, options=lr.default_options(precision=prec))
        e1 = float((m1 - r1).abs().max() / r1.abs().max())
        e2 = float((m2 - r2).abs().max() / r2.abs().max())
        print(f"prec {prec} transpose {tr}: rel err singles {e1:.2e} doubles {e2:.2e}")
        assert e1 < bound and e2 < bound
    prob.close()


_ORACLE = {}


@pytest.mark.parametrize("nk,o,v,Q", [(3, 2, 4, 6), (3, 4, 16, 48), (2, 8, 16, 40)])
@pytest.mark.parametrize("prec,bound", [(1, 3e-3), (2, 5e-5)])
def test_mixed_products_vs_oracle(lr, nk, o, v, Q, prec, bound):
    """The tensor-core products against the oracle directly (A.X by the exact stencil, the
    transpose by reverse-mode differentiation), in both directions."""
    from oracle import rcc
    p = make_problem(nk, o, v, Q, seed=11, sigma_l=0.1)
    t1, t2 = random_amplitudes(nk, o, v, seed=12, scale1=0.02, scale2=0.02)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2 * nk)
    x1, x2 = random_amplitudes(nk, o, v, seed=5, scale1=1.0, scale2=1.0)
    dev = torch.device("cuda")
    X1 = torch.as_tensor(x1, device=dev)[None].contiguous()
    X2 = torch.as_tensor(x2 * nk, device=dev)[None].contiguous()
    opt = lr.default_options(precision=prec)
    y1, y2 = prob.jacobian_apply(X1, X2, options=opt)
    z1, z2 = prob.jacobian_apply(X1, X2, transpose=True, options=opt)
    prob.close()
    key = (nk, o, v, Q)
    if key not in _ORACLE:  # shared by both precisions
        R = rcc.RCC(p)
        T = torch.as_tensor
        a1, a2 = R.jacobian(T(t1), T(t2), T(x1), T(x2))
        b1, b2 = R.transpose(T(t1), T(t2), T(x1), T(x2 * nk * nk))  # A_paper^T = D_in A^T D_out
        _ORACLE[key] = (a1, a2, b1, b2)
    a1, a2, b1, b2 = _ORACLE[key]
    for got, want in ((y1[0], a1), (y2[0], nk * a2), (z1[0], b1), (z2[0], b2 / nk)):
        got, want = got.cpu().numpy(), want.numpy()
        err = float(np.abs(got - want).max() / np.abs(want).max())
        print(f"prec {prec}: rel err vs oracle {err:.2e}")
        assert err < bound
