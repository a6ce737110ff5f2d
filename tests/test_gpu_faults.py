"""Failure handling without a GPU fault: rejected inputs, allocation failure, non-
convergence and a bounded device wait that runs out.  After each, the context and the
problem stay usable (a product still matches the oracle-checked reference)."""
import numpy as np
import pytest
import torch

from synth import make_problem, random_amplitudes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lr():
    import __graft_entry__ as g
    g.build()
    import paper_2508_01266_gb300 as m
    return m


def _small(lr):
    nk, o, v, Q = 2, 2, 3, 4
    p = make_problem(nk, o, v, Q, seed=91, sigma_l=0.1)
    t1, t2 = random_amplitudes(nk, o, v, seed=92, scale1=0.02, scale2=0.02)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2 * nk, t1, t2 * nk)
    x1, x2 = random_amplitudes(nk, o, v, seed=93, scale1=1.0, scale2=1.0)
    dev = torch.device("cuda")
    X = (torch.as_tensor(x1, device=dev)[None].contiguous(), torch.as_tensor(x2 * nk, device=dev)[None].contiguous())
    return p, prob, X, prob.jacobian_apply(*X)


def _same(prob, X, ref):
    y = prob.jacobian_apply(*X)
    return torch.equal(y[0], ref[0]) and torch.equal(y[1], ref[1])


def test_rejected_inputs_leave_problem_usable(lr):
    p, prob, X, ref = _small(lr)
    L = p.L.copy()
    L[0, 1, 0, 0, 1] += 0.3  # breaks L(k2,k1) = L(k1,k2)^H
    for bad in ({"L": L}, {"L": np.where(np.isfinite(p.L), p.L, 0) * np.nan}, {"eps": p.eps[:, ::-1].copy()},
                {"dip": p.dip * np.nan}):
        args = {"L": p.L, "eps": p.eps, "dip": p.dip}
        args.update(bad)
        with pytest.raises(lr.LrccError) as e:
            prob.set_integrals(args["L"], args["eps"], args["dip"])
        assert e.value.status == 1
        assert _same(prob, X, ref)
    t1, t2 = random_amplitudes(2, 2, 3, seed=94, scale1=0.02, scale2=0.02)
    t2[0, 0, 0, 0, 0, 0, 0] = np.nan
    with pytest.raises(lr.LrccError) as e:
        prob.set_ground_state(t1, t2 * 2)
    assert e.value.status == 1
    assert _same(prob, X, ref)
    prob.close()


def test_allocation_failure_is_reported(lr):
    with pytest.raises(lr.LrccError) as e:
        lr.Problem(9, 16, 100, 400)  # fixed arena of about 0.5 TB
    assert e.value.status == 2
    with pytest.raises(lr.LrccError) as e:
        lr.Problem(3, 40, 400, 2000)  # a single extent beyond 32-bit layout dimensions
    assert e.value.status == 1 and "too large" in str(e.value)
    p, prob, X, ref = _small(lr)  # the context is still usable
    assert _same(prob, X, ref)
    prob.close()


def test_non_convergence_is_reported(lr):
    p, prob, X, ref = _small(lr)
    with pytest.raises(lr.LrccError) as e:
        prob.polarizability([2], [0.05], lr.default_options(max_iter=1, conv_tol=1e-14))
    assert e.value.status == 4
    assert _same(prob, X, ref)
    prob.close()


def test_bounded_wait_runs_out(lr):
    p, prob, X, ref = _small(lr)
    from paper_2508_01266_gb300._lib import lib
    st = lib.lrcc_wait_selftest(prob.h, 1000)
    assert st == 5  # LRCC_ETIMEOUT
    assert _same(prob, X, ref)
    # the flag was cleared: a tensor-core product still succeeds
    y = prob.jacobian_apply(*X, options=lr.default_options(precision=2))
    assert float((y[1] - ref[1]).abs().max() / ref[1].abs().max()) < 1e-4
    prob.close()
