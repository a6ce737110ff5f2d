"""GPU polarizability (FP64 path) against the CPU oracle.

The oracle converges T and Lambda; the GPU receives them (paper normalization) and
solves the perturbed-amplitude equations and assembles alpha(w) itself.
Tolerance: 1e-8 relative on alpha (FP64 path).
"""
import numpy as np
import pytest
import torch

from synth import make_problem, CONFIGS
from oracle import rcc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lr():
    import __graft_entry__ as g
    g.build()
    import paper_2508_01266_gb300 as m
    return m


def paper_lambda(nk, l1, l2):
    """Oracle multipliers (plain pairing, supercell units) -> the paper's Lambda
    (alpha-beta block of the spin-orbital multipliers, paper units)."""
    kb = lambda i, j, a: (i + j - a) % nk  # noqa: E731
    sw = torch.zeros_like(l2)
    for ki in range(nk):
        for kj in range(nk):
            for ka in range(nk):
                sw[ki, kj, ka] = l2[ki, kj, kb(ki, kj, ka)].transpose(2, 3)
    return l1 / 2.0, nk * (2.0 * l2 + sw) / 3.0


def _run(lr, p, comps, omegas, tol=1e-10):
    nk, o, v, Q = p.nk, p.nocc, p.nvir, p.naux
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=tol)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=tol)
    ref = rcc.polarizability(R, t1, t2, l1, l2, rcc.dipole_ops(p, comps), omegas, tol=1e-11)
    pl1, pl2 = paper_lambda(nk, l1, l2)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2 * nk, pl1, pl2)
    opts = lr.default_options(conv_tol=1e-11, max_iter=300)
    got, info = prob.polarizability(comps, omegas, opts)
    prob.close()
    return got, ref, info


def test_alpha_small_vs_oracle(lr):
    p = make_problem(2, 2, 3, 4, seed=5, sigma_l=0.15)
    got, ref, info = _run(lr, p, [0, 2], [0.0, 0.07])
    assert info[1] == 0
    assert np.abs(got - ref).max() < 1e-8 * np.abs(ref).max()


def test_alpha_skips_vanishing_component(lr):
    p = make_problem(1, 1, 3, 4, seed=6, sigma_l=0.15)
    p.dip[1] = 0.0
    got, ref, info = _run(lr, p, [1, 2], [0.05])
    assert info[2] == 1 and info[3] == 0
    assert np.abs(got[0, 0, :]).max() == 0.0 and np.abs(got[0, :, 0]).max() == 0.0
    assert abs(got[0, 1, 1] - ref[0, 1, 1]) < 1e-8 * abs(ref[0, 1, 1])


@pytest.fixture(scope="module")
def c1_ref():
    """C1 workload (Nk=3, nocc=4, nvir=16, naux=48): oracle T, Lambda and alpha_zz at w = 0, 0.1 Ha."""
    c = CONFIGS["c1"]
    p = make_problem(c["nk"], c["nocc"], c["nvir"], c["naux"], seed=1266)
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-10)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-10)
    ref = rcc.polarizability(R, t1, t2, l1, l2, rcc.dipole_ops(p, [2]), [0.0, 0.1], tol=1e-11)
    return p, t1, t2, l1, l2, ref


def _c1_gpu(lr, c1_ref, options):
    p, t1, t2, l1, l2, ref = c1_ref
    nk, o, v, Q = p.nk, p.nocc, p.nvir, p.naux
    pl1, pl2 = paper_lambda(nk, l1, l2)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2 * nk, pl1, pl2)
    got, info = prob.polarizability([2], [0.0, 0.1], options)
    prob.close()
    return got, ref, info


def test_alpha_c1_vs_oracle(lr, c1_ref):
    got, ref, info = _c1_gpu(lr, c1_ref, lr.default_options(conv_tol=1e-11, max_iter=300))
    assert info[1] == 0
    rel = np.abs(got - ref).max() / np.abs(ref).max()
    print("C1 alpha_zz gpu", got.ravel(), "oracle", ref.ravel(), "rel", rel)
    assert rel < 1e-8


@pytest.mark.parametrize("prec", [2, 1])
def test_alpha_mixed_precision_c1(lr, c1_ref, prec):
    """Tensor-core inner solves + FP64 iterative refinement: |alpha - alpha_oracle| <= 1e-5 a.u."""
    got, ref, info = _c1_gpu(lr, c1_ref, lr.default_options(precision=prec, refine_tol=1e-8))
    err = np.abs(got - ref).max()
    print(f"C1 alpha_zz prec {prec}: {got.ravel()} oracle {ref.ravel()} |err| {err:.2e} iterations {info[0]}")
    assert info[1] == 0
    assert err <= 1e-5


@pytest.mark.parametrize("form", [1, 2])
def test_left_response_alpha_vs_oracle(lr, form):
    """Asymmetric (left-response) alpha on the GPU vs the oracle's asymmetric form
    (form 2, as computed) and its symmetrisation (form 1); non-TR data so that the
    two differ."""
    p = make_problem(2, 2, 3, 4, seed=7, sigma_l=0.15, tr=False)
    nk, o, v, Q = p.nk, p.nocc, p.nvir, p.naux
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-11)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-11)
    comps, omegas = [0, 2], [0.0, 0.06]
    sym, asym = rcc.polarizability_left(R, t1, t2, l1, l2, rcc.dipole_ops(p, comps), omegas, tol=1e-11)
    ref = sym if form == 1 else asym
    pl1, pl2 = paper_lambda(nk, l1, l2)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2 * nk, pl1, pl2)
    got, info = prob.polarizability(comps, omegas, lr.default_options(conv_tol=1e-11, max_iter=300,
                                                                      response_form=form))
    sym_gpu, _ = prob.polarizability(comps, omegas, lr.default_options(conv_tol=1e-11, max_iter=300))
    prob.close()
    assert info[1] == 0
    assert np.abs(got - ref).max() < 1e-8 * np.abs(ref).max()
    if form == 2:  # at convergence the asymmetric form equals the symmetric one element by element
        assert np.abs(got - sym_gpu).max() < 1e-8 * np.abs(sym_gpu).max()


def test_left_response_alpha_mixed_c1(lr, c1_ref):
    """Left-response form with tensor-core inner solves: within 1e-5 a.u. of the oracle."""
    got, ref, info = _c1_gpu(lr, c1_ref, lr.default_options(precision=2, refine_tol=1e-8, response_form=1))
    err = np.abs(got - ref).max()
    print(f"C1 left-response alpha_zz BF16x3: {got.ravel()} oracle {ref.ravel()} |err| {err:.2e}")
    assert info[1] == 0
    assert err <= 1e-5


def test_alpha_host_history_and_chunks_bitwise(lr):
    """DIIS history in pinned host memory (read by the kernels over the CPU-GPU link) and
    chunked products give bitwise the alpha of the all-device, single-launch solve."""
    p = make_problem(2, 2, 3, 4, seed=5, sigma_l=0.15)
    nk, o, v, Q = p.nk, p.nocc, p.nvir, p.naux
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-10)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-10)
    pl1, pl2 = paper_lambda(nk, l1, l2)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2 * nk, pl1, pl2)
    base = dict(conv_tol=1e-11, max_iter=300)
    ref, _ = prob.polarizability([0, 2], [0.0, 0.07], lr.default_options(host_history=-1, **base))
    got, info = prob.polarizability([0, 2], [0.0, 0.07], lr.default_options(host_history=1, max_batch=2, **base))
    prob.close()
    assert info[1] == 0
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("form", [0, 2])
def test_response_function_general_operators(lr, form):
    """lrcc_response_function with operators other than the dipole (a magnetic-dipole-like
    time-reversal-odd operator, a quadrupole-like even one, a dipole component) against the
    oracle's response function <<X;Y>> = -alpha_XY, symmetric (form 0) and asymmetric
    (form 2) forms, X != Y included; non-TR data so that every element is non-trivial."""
    from synth import make_operator
    p = make_problem(2, 2, 3, 4, seed=8, sigma_l=0.15, tr=False)
    nk, o, v, Q = p.nk, p.nocc, p.nvir, p.naux
    n = o + v
    ops = np.stack([make_operator(nk, n, seed=301, parity=-1), make_operator(nk, n, seed=302, parity=1),
                    p.dip[0]])
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-11)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-11)
    mus = [torch.as_tensor(X) for X in ops]
    om = [0.0, 0.06]
    if form == 0:
        ref = -rcc.polarizability(R, t1, t2, l1, l2, mus, om, tol=1e-11)
    else:
        ref = -rcc.polarizability_left(R, t1, t2, l1, l2, mus, om, tol=1e-11)[1]
    pl1, pl2 = paper_lambda(nk, l1, l2)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2 * nk, pl1, pl2)
    got, info = prob.response_function(ops, om, lr.default_options(conv_tol=1e-11, max_iter=300,
                                                                    response_form=form))
    prob.close()
    assert info[1] == 0
    rel = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"form {form}: <<X;Y>> rel err {rel:.2e}; odd-even element {got[1, 0, 1]}")
    assert rel < 1e-8
    assert np.abs(got[1, 0, 1]) > 1e-3 * np.abs(got).max()  # X != Y coupling present


def test_response_function_rejects_non_hermitian(lr):
    p = make_problem(1, 1, 2, 3, seed=9, sigma_l=0.1)
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-10)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-10)
    pl1, pl2 = paper_lambda(1, l1, l2)
    prob = lr.Problem(1, 1, 2, 3)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2, pl1, pl2)
    bad = np.zeros((1, 1, 3, 3), dtype=np.complex128)
    bad[0, 0, 0, 1] = 1.0
    with pytest.raises(lr.LrccError) as e:
        prob.response_function(bad, [0.0])
    assert "not Hermitian" in str(e.value)
    prob.close()


def test_polarizability_both_forms_from_one_solve(lr):
    """lrcc_polarizability_forms: the symmetric and the asymmetric form from one set of
    right-hand solutions, each against the oracle's, non-TR data."""
    p = make_problem(2, 2, 3, 4, seed=7, sigma_l=0.15, tr=False)
    nk, o, v, Q = p.nk, p.nocc, p.nvir, p.naux
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-11)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-11)
    mus = rcc.dipole_ops(p, [0, 2])
    om = [0.0, 0.08]
    ref_sym = rcc.polarizability(R, t1, t2, l1, l2, mus, om, tol=1e-11)
    ref_asym = rcc.polarizability_left(R, t1, t2, l1, l2, mus, om, tol=1e-11)[1]
    pl1, pl2 = paper_lambda(nk, l1, l2)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2 * nk, pl1, pl2)
    sym, asym, info = prob.polarizability_forms([0, 2], om, lr.default_options(conv_tol=1e-11, max_iter=300))
    prob.close()
    assert info[1] == 0
    assert np.abs(sym - ref_sym).max() < 1e-8 * np.abs(ref_sym).max()
    assert np.abs(asym - ref_asym).max() < 1e-8 * np.abs(ref_asym).max()
    assert np.abs(asym - asym.transpose(0, 2, 1)).max() > 1e-6 * np.abs(asym).max()  # forms differ element-wise
