"""Pins of the CPU oracle against facts that do not come from the oracle itself.

P0 generator invariants; P1 spin-orbital residual vs determinant-space brute force;
P2 Jacobian stencil vs brute-force commutator; P3 adjoint identity; P4/P9 closed-shell
k-blocked residual vs the dense spin-orbital one (Nk = 1 molecular case included);
P5 decoupled replicas; P6 two electrons = FCI (energy and sum-over-states alpha,
with and without time-reversal symmetry); P7 finite field; P8 symmetries and
momentum zeros; P10 left-response (asymmetric) alpha = symmetric alpha, and = FCI
for two electrons; P11 zero interaction closed form; P12 first Jacobi step = MP2.
"""
import numpy as np
import pytest
import torch

from synth import make_problem, random_amplitudes, kmesh_neg
from oracle import spinorb, fci, rcc

T = lambda x: torch.as_tensor(x)  # noqa: E731


# P0 ---------------------------------------------------------------------------
@pytest.mark.parametrize("nk,kmesh", [(3, 0), (4, 1), (4, 2), (1, 0)])
def test_generator_invariants(nk, kmesh):
    p = make_problem(nk, 2, 3, 5, seed=7, kmesh=kmesh)
    neg = kmesh_neg(nk, kmesh)
    for k1 in range(nk):
        assert np.allclose(p.dip[:, k1], np.conj(np.swapaxes(p.dip[:, k1], 1, 2)))
        assert np.allclose(p.dip[:, neg[k1]], np.conj(p.dip[:, k1]))
        assert np.allclose(p.eps[neg[k1]], p.eps[k1])
        for k2 in range(nk):
            assert np.allclose(p.L[k2, k1], np.conj(np.swapaxes(p.L[k1, k2], 1, 2)))
            assert np.allclose(p.L[neg[k1], neg[k2]], np.conj(p.L[k1, k2]))
    # Coulomb matrix V[(p,q),(s,r)] = (pq|rs) over momentum-conserving pairs is PSD
    S = spinorb.SpinOrbitalSystem(p)
    g = S.g  # <PQ|RS> = (PR|QS)
    chem = g.transpose(0, 2, 1, 3)  # (PR|QS) -> [P,R,Q,S]
    N = S.N
    M = chem.transpose(0, 1, 3, 2).reshape(N * N, N * N)  # rows (P,R), cols (S,Q)
    assert np.allclose(M, M.conj().T, atol=1e-14)
    assert np.linalg.eigvalsh(M).min() > -1e-12


# P1 ---------------------------------------------------------------------------
@pytest.mark.parametrize("nk,o,v,seed", [(1, 2, 2, 1), (2, 1, 2, 2), (3, 1, 2, 3)])
def test_spinorb_residual_vs_bruteforce(nk, o, v, seed):
    p = make_problem(nk, o, v, 4, seed=seed, sigma_l=0.3)
    S = spinorb.SpinOrbitalSystem(p)
    t1k, t2k = random_amplitudes(nk, o, v, seed=seed + 10, scale1=0.1, scale2=0.1)
    t1, t2 = spinorb.to_spinorb(S, t1k, t2k)
    a1, a2 = spinorb.residual(S, t1, t2)
    b1, b2 = fci.cc_residual(S, t1, t2)
    assert np.abs(a1 - b1).max() < 1e-13
    assert np.abs(a2 - b2).max() < 1e-13
    assert np.abs(b2).max() > 0.1


def test_spinorb_residual_nonspinadapted_bruteforce():
    """Random spin-orbital amplitudes (not spin-adapted) also match: no closed-shell
    assumption hides inside the spin-orbital equations."""
    p = make_problem(2, 1, 1, 3, seed=4, sigma_l=0.3, tr=False)
    S = spinorb.SpinOrbitalSystem(p)
    rng = np.random.default_rng(0)
    O, V = S.O, S.V
    t1 = 0.1 * (rng.normal(size=(O, V)) + 1j * rng.normal(size=(O, V)))
    t2 = 0.1 * (rng.normal(size=(O, O, V, V)) + 1j * rng.normal(size=(O, O, V, V)))
    t2 = t2 - t2.transpose(1, 0, 2, 3)
    t2 = t2 - t2.transpose(0, 1, 3, 2)
    a1, a2 = spinorb.residual(S, t1, t2)
    b1, b2 = fci.cc_residual(S, t1, t2)
    assert np.abs(a1 - b1).max() < 1e-13 and np.abs(a2 - b2).max() < 1e-13


# P4 / P9 -------------------------------------------------------------------------
@pytest.mark.parametrize("nk,o,v,seed,tr", [(1, 2, 3, 1, True), (2, 1, 2, 2, False),
                                           (3, 1, 2, 3, True), (2, 2, 2, 4, True),
                                           (4, 1, 1, 5, True)])
def test_closed_shell_vs_spinorb(nk, o, v, seed, tr):
    p = make_problem(nk, o, v, 5, seed=seed, sigma_l=0.3, tr=tr)
    S = spinorb.SpinOrbitalSystem(p)
    R = rcc.RCC(p)
    t1k, t2k = random_amplitudes(nk, o, v, seed=seed + 3, scale1=0.1, scale2=0.1)
    t1, t2 = spinorb.to_spinorb(S, t1k, t2k)
    c1, c2 = spinorb.from_spinorb(S, *spinorb.residual(S, t1, t2))
    b1, b2 = R.residual(T(t1k), T(t2k))
    assert np.abs(c1 - b1.numpy()).max() < 1e-13
    assert np.abs(c2 - b2.numpy()).max() < 1e-13
    assert abs(spinorb.energy(S, t1, t2) - complex(R.energy(T(t1k), T(t2k)))) < 1e-14
    # sampled blocks equal the full evaluation
    blocks = [(0, nk - 1, min(1, nk - 1))]
    _, s2 = R.residual(T(t1k), T(t2k), blocks=blocks)
    for bk in blocks:
        assert torch.allclose(s2[bk], b2[bk], atol=1e-15)
    s1, _ = R.residual(T(t1k), T(t2k), blocks=blocks, singles=True)
    assert torch.allclose(s1, b1, atol=1e-15)


# P2 ---------------------------------------------------------------------------
def test_jacobian_stencil_vs_commutator():
    """A.X from the stencil equals <mu| exp(-T) [H, X] exp(T) |0> by brute force."""
    nk, o, v = 2, 1, 2
    p = make_problem(nk, o, v, 4, seed=21, sigma_l=0.3)
    S = spinorb.SpinOrbitalSystem(p)
    R = rcc.RCC(p)
    t1k, t2k = random_amplitudes(nk, o, v, seed=22, scale1=0.1, scale2=0.1)
    x1k, x2k = random_amplitudes(nk, o, v, seed=23, scale1=1.0, scale2=1.0)
    a1, a2 = R.jacobian(T(t1k), T(t2k), T(x1k), T(x2k))
    t1, t2 = spinorb.to_spinorb(S, t1k, t2k)
    x1, x2 = spinorb.to_spinorb(S, x1k, x2k)
    # commutator by brute force: exp(-T) (H X - X H) exp(T) |0>
    O, N = S.O, S.N
    ds = fci.DetSpace(N, O)
    g = S.g
    h = S.f - np.einsum("piqi->pq", (g - g.transpose(0, 1, 3, 2))[:, :O, :, :O])
    psi = fci._exp_T(ds, O, t1, t2, ds.ref(), 1.0)
    hx = fci._apply_H(ds, h, g, fci._apply_T(ds, O, x1, x2, psi))
    xh = fci._apply_T(ds, O, x1, x2, fci._apply_H(ds, h, g, psi))
    om = fci._exp_T(ds, O, t1, t2, hx - xh, -1.0)
    ref = ds.ref()
    V = N - O
    b1 = np.zeros((O, V), complex)
    b2 = np.zeros((O, O, V, V), complex)
    for I in range(O):
        for A in range(V):
            b1[I, A] = np.vdot(ds.E(O + A, I) @ ref, om)
            for J in range(O):
                for B in range(V):
                    if I != J and A != B:
                        b2[I, J, A, B] = np.vdot(ds.E(O + A, I) @ (ds.E(O + B, J) @ ref), om)
    c1, c2 = spinorb.from_spinorb(S, b1, b2)
    assert np.abs(c1 - a1.numpy()).max() < 1e-12
    assert np.abs(c2 - a2.numpy()).max() < 1e-12


# P3 ---------------------------------------------------------------------------
def test_transpose_adjoint_identity():
    nk, o, v = 3, 1, 2
    p = make_problem(nk, o, v, 4, seed=31, sigma_l=0.2)
    R = rcc.RCC(p)
    t1, t2 = map(T, random_amplitudes(nk, o, v, seed=32, scale1=0.05, scale2=0.05))
    for s in range(3):
        x1, x2 = map(T, random_amplitudes(nk, o, v, seed=40 + s, scale1=1, scale2=1))
        y1, y2 = map(T, random_amplitudes(nk, o, v, seed=50 + s, scale1=1, scale2=1))
        a1, a2 = R.jacobian(t1, t2, x1, x2)
        b1, b2 = R.transpose(t1, t2, y1, y2)
        lhs = (y1 * a1).sum() + (y2 * a2).sum()
        rhs = (b1 * x1).sum() + (b2 * x2).sum()
        assert abs(complex(lhs - rhs)) < 1e-12 * abs(complex(lhs))


# P6 ---------------------------------------------------------------------------
@pytest.mark.parametrize("tr", [True, False])
def test_two_electrons_equal_fci(tr):
    p = make_problem(1, 1, 3, 4, seed=61, sigma_l=0.15, tr=tr)
    R = rcc.RCC(p)
    S = spinorb.SpinOrbitalSystem(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-12)
    comps = (0, 2)
    mus = rcc.dipole_ops(p, comps)
    ops = [spinorb.one_body_to_spinorb(S, p.dip[c]) for c in comps]
    for w in (0.0, 0.07):
        ecorr, a_fci = fci.sos_polarizability(S, ops, w)
        assert abs(complex(R.energy(t1, t2)) - ecorr) < 1e-10
        a_cc = rcc.polarizability(R, t1, t2, l1, l2, mus, [w])[0]
        assert np.abs(a_cc - a_fci).max() < 1e-9 * np.abs(a_fci).max()
        if tr:
            assert np.abs(a_cc.imag).max() < 1e-10
        else:  # exact alpha is Hermitian, not symmetric, for complex operators
            assert np.allclose(a_cc, a_cc.conj().T, atol=1e-10)


# P10 --------------------------------------------------------------------------
@pytest.mark.parametrize("tr", [True, False])
def test_left_response_alpha_equals_fci_two_electrons(tr):
    """Two electrons: the asymmetric form (left perturbed multipliers from transpose
    products) reproduces the FCI sum over states, with and without TR symmetry."""
    p = make_problem(1, 1, 3, 4, seed=61, sigma_l=0.15, tr=tr)
    R = rcc.RCC(p)
    S = spinorb.SpinOrbitalSystem(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-12)
    comps = (0, 2)
    mus = rcc.dipole_ops(p, comps)
    ops = [spinorb.one_body_to_spinorb(S, p.dip[c]) for c in comps]
    for w in (0.0, 0.07):
        _, a_fci = fci.sos_polarizability(S, ops, w)
        _, a_left = rcc.polarizability_left(R, t1, t2, l1, l2, mus, [w])
        assert np.abs(a_left[0] - a_fci).max() < 1e-9 * np.abs(a_fci).max()


def test_left_response_alpha_equals_symmetric_form():
    """Beyond two electrons (Nk = 2: four electrons in the two-cell supercell): asymmetric
    alpha = symmetric alpha element by element at convergence, two components at +-w."""
    p = make_problem(2, 1, 2, 3, seed=101, sigma_l=0.2)
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-12)
    mus = rcc.dipole_ops(p, (0, 2))
    om = [0.09]
    a_sym = rcc.polarizability(R, t1, t2, l1, l2, mus, om)
    a_ls, a_left = rcc.polarizability_left(R, t1, t2, l1, l2, mus, om)
    assert np.abs(a_left - a_sym).max() < 1e-9 * np.abs(a_sym).max()
    assert np.abs(a_ls - 0.5 * (a_sym + a_sym.transpose(0, 2, 1))).max() < 1e-9 * np.abs(a_sym).max()


def test_eta_and_F_vectors_match_scalar_stencils():
    """eta^X . w and (F u) . w from the vector forms equal the scalar stencils."""
    nk, o, v = 2, 1, 2
    p = make_problem(nk, o, v, 3, seed=103, sigma_l=0.2)
    R = rcc.RCC(p)
    t1, t2 = (T(x) for x in random_amplitudes(nk, o, v, seed=104, scale1=0.05, scale2=0.05))
    l1, l2 = (T(x) for x in random_amplitudes(nk, o, v, seed=105, scale1=0.05, scale2=0.05))
    u1, u2 = (T(x) for x in random_amplitudes(nk, o, v, seed=106, scale1=1.0, scale2=1.0))
    w1, w2 = (T(x) for x in random_amplitudes(nk, o, v, seed=107, scale1=1.0, scale2=1.0))
    mu = rcc.dipole_ops(p, (1,))[0]
    e1, e2 = rcc.eta_vector(R, t1, t2, l1, l2, mu)
    ref = complex(rcc.eta_dot(R, t1, t2, l1, l2, mu, w1, w2))
    assert abs(complex((e1 * w1).sum() + (e2 * w2).sum()) - ref) < 1e-10 * abs(ref)
    f1, f2 = rcc.F_vector(R, t1, t2, l1, l2, u1, u2)
    ref = complex(rcc.F_dot(R, t1, t2, l1, l2, u1, u2, w1, w2))
    assert abs(complex((f1 * w1).sum() + (f2 * w2).sum()) - ref) < 1e-9 * abs(ref)


def test_vector_form_alpha_equals_fci_and_stencil_form():
    """alpha assembled from eta and F vectors (the form the large-workload fixture uses)
    equals the FCI sum over states for two electrons, and the per-element scalar-stencil
    form element by element for four electrons in two cells, with and without TR."""
    p = make_problem(1, 1, 3, 4, seed=61, sigma_l=0.15)
    R = rcc.RCC(p)
    S = spinorb.SpinOrbitalSystem(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-12)
    comps = (0, 2)
    ops = [spinorb.one_body_to_spinorb(S, p.dip[c]) for c in comps]
    _, a_fci = fci.sos_polarizability(S, ops, 0.07)
    a_vec = rcc.polarizability_vectors(R, t1, t2, l1, l2, rcc.dipole_ops(p, comps), [0.07])[0]
    assert np.abs(a_vec - a_fci).max() < 1e-9 * np.abs(a_fci).max()
    for tr in (True, False):
        p = make_problem(2, 1, 2, 3, seed=101, sigma_l=0.2, tr=tr)
        R = rcc.RCC(p)
        t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
        l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-12)
        mus = rcc.dipole_ops(p, (0, 1, 2))
        a = rcc.polarizability(R, t1, t2, l1, l2, mus, [0.0, 0.09])
        b = rcc.polarizability_vectors(R, t1, t2, l1, l2, mus, [0.0, 0.09])
        assert np.abs(a - b).max() < 1e-10 * np.abs(a).max()
        # eta vectors with the F scalars F(t^x(-w), t^y(w))
        etas = [rcc.eta_vector(R, t1, t2, l1, l2, m) for m in mus]
        xis = [rcc.perturbation_rhs(R, t1, t2, m) for m in mus]
        tp = [rcc.solve_response(R, t1, t2, *xi, 0.09)[:2] for xi in xis]
        tm = [rcc.solve_response(R, t1, t2, *xi, -0.09)[:2] for xi in xis]
        Fmp = [[complex(rcc.F_dot(R, t1, t2, l1, l2, *tm[x], *tp[y])) for y in range(3)] for x in range(3)]
        c = rcc.symmetric_alpha_from_scalars(R.nk, etas, tp, tm, Fmp)
        assert np.abs(c - a[1]).max() < 1e-10 * np.abs(a).max()


@pytest.mark.parametrize("tr", [True, False])
def test_mixed_operator_response_equals_fci_two_electrons(tr):
    """Response functions between different one-body operators (a magnetic-dipole-like
    time-reversal-odd operator, a quadrupole-like even one and a dipole component): the
    symmetric form of Eq. 15 and the asymmetric (left-response) form with arbitrary
    Hermitian operators both equal the FCI sum over states for two electrons."""
    from synth import make_operator
    p = make_problem(1, 1, 3, 4, seed=61, sigma_l=0.15, tr=tr)
    R = rcc.RCC(p)
    S = spinorb.SpinOrbitalSystem(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-12)
    ops = [make_operator(1, 4, seed=201, parity=-1), make_operator(1, 4, seed=202, parity=1), p.dip[2]]
    assert np.abs(ops[0].real).max() == 0.0 and np.abs(ops[1].imag).max() == 0.0
    mus = [T(X) for X in ops]
    for w in (0.0, 0.07):
        _, a_fci = fci.sos_polarizability(S, [spinorb.one_body_to_spinorb(S, X) for X in ops], w)
        a_cc = rcc.polarizability(R, t1, t2, l1, l2, mus, [w])[0]
        assert np.abs(a_cc - a_fci).max() < 1e-9 * np.abs(a_fci).max()
        _, a_left = rcc.polarizability_left(R, t1, t2, l1, l2, mus, [w])
        assert np.abs(a_left[0] - a_fci).max() < 1e-9 * np.abs(a_fci).max()
    # the odd-even response is imaginary, antisymmetric and vanishes in the static limit
    # under time reversal; a sanity check that the operators are what they claim to be
    if tr:
        _, a0 = fci.sos_polarizability(S, [spinorb.one_body_to_spinorb(S, X) for X in ops[:2]], 0.0)
        assert abs(a0[0, 1]) < 1e-12 * np.abs(a0).max()


# excitation energies (Jacobian eigenvalues) -------------------------------------
@pytest.mark.parametrize("tr", [True, False])
def test_excitation_energies_are_fci_two_electrons(tr):
    """Two electrons: CCSD is exact, so every eigenvalue of its Jacobian on the
    closed-shell space is an FCI excitation energy."""
    p = make_problem(1, 1, 3, 4, seed=61, sigma_l=0.15, tr=tr)
    R = rcc.RCC(p)
    S = spinorb.SpinOrbitalSystem(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
    w = rcc.excitation_energies(R, t1, t2)
    _, e, _ = fci.fci_states(S)
    ex = e[1:] - e[0]
    assert np.abs(w.imag).max() < 1e-9
    for x in w.real:
        assert np.abs(ex - x).min() < 1e-9


def test_excitation_energies_replicas():
    """Decoupled replicas: every excitation energy of one cell is also one of the
    two-cell chain (the replicated excitation at zero crystal momentum)."""
    p1 = make_problem(1, 1, 2, 3, seed=62, sigma_l=0.2, kind="replica")
    p2 = make_problem(2, 1, 2, 3, seed=62, sigma_l=0.2, kind="replica")
    w = []
    for p in (p1, p2):
        R = rcc.RCC(p)
        t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
        w.append(rcc.excitation_energies(R, t1, t2))
    for x in w[0]:
        assert np.abs(w[1] - x).min() < 1e-9


# P5 ---------------------------------------------------------------------------
def test_decoupled_replicas_independent_of_nk():
    vals = []
    for nk in (1, 2, 3):
        p = make_problem(nk, 1, 2, 3, seed=71, sigma_l=0.2, kind="replica")
        R = rcc.RCC(p)
        t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
        l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-12)
        e = complex(R.energy(t1, t2)) / nk
        a = rcc.polarizability(R, t1, t2, l1, l2, rcc.dipole_ops(p, (2,)), [0.05])[0, 0, 0]
        vals.append((e, a))
    for e, a in vals[1:]:
        assert abs(e - vals[0][0]) < 1e-12
        assert abs(a - vals[0][1]) < 1e-10 * abs(vals[0][1])


# P7 ---------------------------------------------------------------------------
def test_static_alpha_is_finite_field_second_derivative():
    p = make_problem(2, 1, 2, 3, seed=81, sigma_l=0.2)
    R = rcc.RCC(p)
    mu = rcc.dipole_ops(p, (2,))[0]
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-13)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-12)
    a = rcc.polarizability(R, t1, t2, l1, l2, [mu], [0.0])[0, 0, 0]
    hf = 1e-3

    def E(eps):
        hh = R.h + eps * mu
        s1, s2, _ = rcc.solve_ccsd(R, tol=1e-14, h=hh)
        return complex(R.energy(s1, s2, hh)) / R.nk

    d2 = (-E(2 * hf) + 16 * E(hf) - 30 * E(0.0) + 16 * E(-hf) - E(-2 * hf)) / (12 * hf * hf)
    # the reference energy is linear in eps, so only the correlation part contributes
    assert abs(a.real - (-d2.real)) < 1e-7 * abs(a.real)
    assert a.real > 0


# P8 ---------------------------------------------------------------------------
def test_alpha_symmetries_tr():
    p = make_problem(2, 1, 2, 3, seed=91, sigma_l=0.2)
    R = rcc.RCC(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-12)
    mus = rcc.dipole_ops(p, (0, 2))
    a = rcc.polarizability(R, t1, t2, l1, l2, mus, [0.06, -0.06])
    assert np.abs(a.imag).max() < 1e-10
    assert np.allclose(a[0], a[0].T, atol=1e-10)
    assert np.allclose(a[0], a[1], atol=1e-10)


def test_momentum_forbidden_blocks_stay_zero():
    nk, o, v = 3, 1, 2
    p = make_problem(nk, o, v, 4, seed=95, sigma_l=0.3)
    S = spinorb.SpinOrbitalSystem(p)
    t1, t2 = spinorb.to_spinorb(S, *random_amplitudes(nk, o, v, seed=96, scale1=0.1, scale2=0.1))
    r1, r2 = spinorb.residual(S, t1, t2)
    ko, kv = S.kk[:S.O], S.kk[S.O:]
    bad1 = ko[:, None] != kv[None, :]
    bad2 = ((ko[:, None, None, None] + ko[None, :, None, None]
             - kv[None, None, :, None] - kv[None, None, None, :]) % nk) != 0
    assert np.abs(r1[bad1]).max() == 0.0
    assert np.abs(r2[bad2]).max() == 0.0
    assert np.abs(r2[~bad2]).max() > 1e-3


# P11 --------------------------------------------------------------------------
def test_zero_interaction_closed_form():
    nk, o, v = 2, 2, 3
    p = make_problem(nk, o, v, 2, seed=101, kind="zero")
    R = rcc.RCC(p)
    t1, t2, it = rcc.solve_ccsd(R, tol=1e-14)
    assert it == 0
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-14)
    comps = (0, 1)
    w = 0.09
    a = rcc.polarizability(R, t1, t2, l1, l2, rcc.dipole_ops(p, comps), [w])[0]
    ref = np.zeros((2, 2), complex)
    for x, cx in enumerate(comps):
        for y, cy in enumerate(comps):
            s = 0.0
            for k in range(nk):
                for i in range(o):
                    for aa in range(v):
                        d = p.eps[k, o + aa] - p.eps[k, i]
                        xia, xai = p.dip[cx, k, i, o + aa], p.dip[cx, k, o + aa, i]
                        yia, yai = p.dip[cy, k, i, o + aa], p.dip[cy, k, o + aa, i]
                        s += 2 * (xia * yai / (d - w) + yia * xai / (d + w))
            ref[x, y] = s / nk
    assert np.abs(a - ref).max() < 1e-12 * np.abs(ref).max()


# P12 --------------------------------------------------------------------------
def test_first_jacobi_step_is_mp2():
    nk, o, v = 3, 1, 2
    p = make_problem(nk, o, v, 4, seed=111, sigma_l=0.2)
    R = rcc.RCC(p)
    S = spinorb.SpinOrbitalSystem(p)
    z1 = torch.zeros((nk, o, v), dtype=torch.complex128)
    z2 = torch.zeros((nk,) * 3 + (o, o, v, v), dtype=torch.complex128)
    r1, r2 = R.residual(z1, z2)
    d1, d2 = R.denominators()
    e = complex(R.energy(z1 - r1 / d1, z2 - r2 / d2))
    assert abs(e - spinorb.mp2_energy(S)) < 1e-14
