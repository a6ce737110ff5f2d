"""Batched multi-problem polarizability: chains of different sizes in one call.

Each problem's alpha from the batch call must equal, bit for bit, the alpha of the
same problem solved alone (the kernels are deterministic; only the interleaving on the
GPU differs), and the FP64 result must match the oracle.
"""
import numpy as np
import pytest
import torch

from synth import make_problem, random_amplitudes
from oracle import rcc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lr():
    import __graft_entry__ as g
    g.build()
    import paper_2508_01266_gb300 as m
    return m


def _prob(lr, nk, o, v, Q, seed):
    p = make_problem(nk, o, v, Q, seed=seed, sigma_l=0.1)
    t1, t2 = random_amplitudes(nk, o, v, seed=seed + 1, scale1=0.02, scale2=0.02)
    l1, l2 = random_amplitudes(nk, o, v, seed=seed + 2, scale1=0.02, scale2=0.02)
    pr = lr.Problem(nk, o, v, Q)
    pr.set_integrals(p.L, p.eps, p.dip)
    pr.set_ground_state(t1, t2 * nk, l1, l2 * nk)
    return pr


def test_batch_equals_individual_solves(lr):
    shapes = [(2, 2, 3, 4), (3, 1, 2, 3), (3, 2, 6, 12)]
    comps, omegas = [0, 2], [0.0, 0.08]
    opts = lr.default_options(conv_tol=1e-11, max_iter=300)
    probs = [_prob(lr, *s, seed=100 + 10 * i) for i, s in enumerate(shapes)]
    alone = [pr.polarizability(comps, omegas, opts)[0] for pr in probs]
    res = lr.batch_polarizability(probs, comps, omegas, opts)
    for (a, info), b in zip(res, alone):
        assert info[1] == 0
        assert np.array_equal(a, b)
    for pr in probs:
        pr.close()


def test_batch_vs_oracle_converged(lr):
    """Two chains with converged oracle T/Lambda: FP64 alpha within 1e-8 relative."""
    from test_gpu_alpha import paper_lambda
    shapes = [(2, 1, 3, 4), (1, 2, 3, 5)]
    comps, omegas = [2], [0.0, 0.05]
    probs, refs = [], []
    for i, (nk, o, v, Q) in enumerate(shapes):
        p = make_problem(nk, o, v, Q, seed=200 + i, sigma_l=0.15)
        R = rcc.RCC(p)
        t1, t2, _ = rcc.solve_ccsd(R, tol=1e-11)
        l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-11)
        refs.append(rcc.polarizability(R, t1, t2, l1, l2, rcc.dipole_ops(p, comps), omegas, tol=1e-11))
        pl1, pl2 = paper_lambda(nk, l1, l2)
        pr = lr.Problem(nk, o, v, Q)
        pr.set_integrals(p.L, p.eps, p.dip)
        pr.set_ground_state(t1, t2 * nk, pl1, pl2)
        probs.append(pr)
    res = lr.batch_polarizability(probs, comps, omegas, lr.default_options(conv_tol=1e-11, max_iter=300))
    for (a, info), ref in zip(res, refs):
        assert info[1] == 0
        assert np.abs(a - ref).max() < 1e-8 * np.abs(ref).max()
    for pr in probs:
        pr.close()


def test_batch_at_real_shapes_smallest_vs_oracle(lr):
    """Two chains of the mixed-size batch at their real shapes, (Nk, nocc, nvir, naux) =
    (3, 4, 24, 96) and (5, 6, 32, 128), in one FP64 batch call: the smaller, given the oracle's
    converged T and Lambda, matches the oracle's alpha_zz(0, 0.1) to 1e-8 relative (Eq. 15),
    and each problem's alpha equals its solo solve bit for bit.  The larger one takes a seeded
    weakly correlated ground state (amplitudes of size 0.01): the oracle would need hours for
    it on the host."""
    from test_gpu_alpha import paper_lambda
    comps, omegas = [2], [0.0, 0.1]
    p = make_problem(3, 4, 24, 96, seed=1266)
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-10)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-10)
    ref = rcc.polarizability(R, t1, t2, l1, l2, rcc.dipole_ops(p, comps), omegas, tol=1e-11)
    pl1, pl2 = paper_lambda(3, l1, l2)
    small = lr.Problem(3, 4, 24, 96)
    small.set_integrals(p.L, p.eps, p.dip)
    small.set_ground_state(t1, t2 * 3, pl1, pl2)
    q = make_problem(5, 6, 32, 128, seed=1267)
    u1, u2 = random_amplitudes(5, 6, 32, seed=1268, scale1=0.01, scale2=0.01)
    m1, m2 = random_amplitudes(5, 6, 32, seed=1269, scale1=0.01, scale2=0.01)
    big = lr.Problem(5, 6, 32, 128)
    big.set_integrals(q.L, q.eps, q.dip)
    big.set_ground_state(u1, u2 * 5, m1, m2 * 5)
    opts = lr.default_options(conv_tol=1e-11, max_iter=300)
    res = lr.batch_polarizability([small, big], comps, omegas, opts)
    alone = [pr.polarizability(comps, omegas, opts)[0] for pr in (small, big)]
    for (a, info), b in zip(res, alone):
        assert info[1] == 0
        assert np.array_equal(a, b)
    rel = np.abs(res[0][0] - ref).max() / np.abs(ref).max()
    print("(3,4,24,96) alpha_zz batch", res[0][0].ravel(), "oracle", ref.ravel(), "rel", rel)
    assert rel < 1e-8
    small.close()
    big.close()


def test_batch_rejects_duplicate_handles(lr):
    pr = _prob(lr, 1, 1, 2, 3, seed=300)
    with pytest.raises(lr.LrccError):
        lr.batch_polarizability([pr, pr], [2], [0.0])
    pr.close()
