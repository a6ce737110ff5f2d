"""Planted mistakes in the CPU oracle are caught by its pins.

Each test patches one plausible mistake into oracle/rcc.py (on the CPU, for the duration
of the test) and checks that the pin meant to guard that part fails, after checking that
the same comparison passes unpatched:

  P9  closed-shell k-blocked residual and energy = spin-orbital ones: a sign error in
      the T1 similarity transform, a Fock build without exchange, an energy without the
      T1 terms (Eq. 6);
  P6  two electrons: alpha = FCI sum over states: the quadratic F term dropped from the
      response function (Eq. 15), the perturbation right-hand side (Eq. 12) off by its
      factor 1/2, a wrong sign of eta, Lambda with the wrong sign of dE/dt;
  P5  decoupled replicas: alpha per cell independent of Nk: the 1/Nk of alpha per cell
      missing;
  P2  A.X vs the brute-force commutator: a 3-point stencil, inexact for the quartic residual;
  P3  adjoint identity: a transpose that forgets to undo the conjugation of the autograd
      gradient;
  P9, term by term: every contraction of the closed-shell residual, dressing, Fock build
      and energy dropped, sign-flipped or index-transposed in turn (mutations that cannot
      change the compared quantities are listed with their reason); the energy's singles
      term, zero at the canonical reference, through P6.
"""
import numpy as np
import pytest
import torch

from synth import make_problem, random_amplitudes
from oracle import spinorb, fci, rcc

T = lambda x: torch.as_tensor(x)  # noqa: E731


def _p9_deviation():
    """max deviation of the closed-shell residual / energy from the spin-orbital ones."""
    nk, o, v, seed = 2, 1, 2, 2
    p = make_problem(nk, o, v, 5, seed=seed, sigma_l=0.3, tr=False)
    S = spinorb.SpinOrbitalSystem(p)
    R = rcc.RCC(p)
    t1k, t2k = random_amplitudes(nk, o, v, seed=seed + 3, scale1=0.1, scale2=0.1)
    t1, t2 = spinorb.to_spinorb(S, t1k, t2k)
    c1, c2 = spinorb.from_spinorb(S, *spinorb.residual(S, t1, t2))
    b1, b2 = R.residual(T(t1k), T(t2k))
    de = abs(spinorb.energy(S, t1, t2) - complex(R.energy(T(t1k), T(t2k))))
    return max(np.abs(c1 - b1.numpy()).max(), np.abs(c2 - b2.numpy()).max(), de)


def _p6_deviation():
    """relative deviation of CC alpha_zz(0.07) from FCI for two electrons."""
    p = make_problem(1, 1, 3, 4, seed=61, sigma_l=0.15)
    R = rcc.RCC(p)
    S = spinorb.SpinOrbitalSystem(p)
    t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
    l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-12)
    w = 0.07
    _, a_fci = fci.sos_polarizability(S, [spinorb.one_body_to_spinorb(S, p.dip[2])], w)
    a_cc = rcc.polarizability(R, t1, t2, l1, l2, rcc.dipole_ops(p, (2,)), [w])[0]
    return np.abs(a_cc - a_fci).max() / np.abs(a_fci).max()


def _p5_deviation():
    """relative change of alpha_zz(0.05) per cell between Nk = 1 and Nk = 2 replicas."""
    vals = []
    for nk in (1, 2):
        p = make_problem(nk, 1, 2, 3, seed=71, sigma_l=0.2, kind="replica")
        R = rcc.RCC(p)
        t1, t2, _ = rcc.solve_ccsd(R, tol=1e-12)
        l1, l2, _ = rcc.solve_lambda(R, t1, t2, tol=1e-12)
        vals.append(rcc.polarizability(R, t1, t2, l1, l2, rcc.dipole_ops(p, (2,)), [0.05])[0, 0, 0])
    return abs(vals[1] - vals[0]) / abs(vals[0])


P9_TOL, P6_TOL, P5_TOL = 1e-13, 1e-9, 1e-10


# P9 ---------------------------------------------------------------------------
def _dress_wrong_sign(orig):
    # L~ = (1 + tau) L (1 - tau) instead of (1 - tau) L (1 + tau)
    return lambda self, t1, h=None: orig(self, -t1, h)


def _G_without_exchange(self, L):
    nk, o = self.nk, self.o
    G = torch.zeros((nk, self.n, self.n), dtype=L.dtype)
    for k in range(nk):
        for kk in range(nk):
            G[k] = G[k] + 2.0 * torch.einsum("Qpq,Qii->pq", L[k, k], L[kk, kk][:, :o, :o])
    return G


def _energy_without_t1(orig):
    return lambda self, t1, t2, h=None: orig(self, torch.zeros_like(t1), t2, h)


@pytest.mark.parametrize("mutation", ["dress_sign", "fock_exchange", "energy_t1"])
def test_p9_catches_planted_mistake(monkeypatch, mutation):
    assert _p9_deviation() < P9_TOL
    if mutation == "dress_sign":
        monkeypatch.setattr(rcc.RCC, "dress", _dress_wrong_sign(rcc.RCC.dress))
    elif mutation == "fock_exchange":
        monkeypatch.setattr(rcc.RCC, "_G", _G_without_exchange)
    else:
        monkeypatch.setattr(rcc.RCC, "energy", _energy_without_t1(rcc.RCC.energy))
    assert _p9_deviation() > 1e3 * P9_TOL


# P6 ---------------------------------------------------------------------------
@pytest.mark.parametrize("mutation", ["no_F_term", "xi_factor", "eta_sign"])
def test_p6_catches_planted_mistake(monkeypatch, mutation):
    assert _p6_deviation() < P6_TOL
    if mutation == "no_F_term":
        monkeypatch.setattr(rcc, "F_dot", lambda *a, **k: 0.0)
    elif mutation == "xi_factor":
        orig = rcc.perturbation_rhs
        monkeypatch.setattr(rcc, "perturbation_rhs", lambda *a, **k: tuple(2.0 * x for x in orig(*a, **k)))
    else:
        orig = rcc.eta_dot
        monkeypatch.setattr(rcc, "eta_dot", lambda *a, **k: -orig(*a, **k))
    assert _p6_deviation() > 1e3 * P6_TOL


# P5 ---------------------------------------------------------------------------
def test_p5_catches_missing_per_cell_factor(monkeypatch):
    assert _p5_deviation() < P5_TOL
    orig = rcc.polarizability
    monkeypatch.setattr(rcc, "polarizability", lambda R, *a, **k: orig(R, *a, **k) * R.nk)
    assert _p5_deviation() > 1e3 * P5_TOL


# P9, term by term -------------------------------------------------------------------
def _p9_case():
    nk, o, v, seed = 2, 2, 3, 4
    p = make_problem(nk, o, v, 5, seed=seed, sigma_l=0.3, tr=False)
    S = spinorb.SpinOrbitalSystem(p)
    t1k, t2k = random_amplitudes(nk, o, v, seed=seed + 3, scale1=0.1, scale2=0.1)
    t1, t2 = spinorb.to_spinorb(S, t1k, t2k)
    ref = spinorb.from_spinorb(S, *spinorb.residual(S, t1, t2)), spinorb.energy(S, t1, t2)
    return p, t1k, t2k, ref


def _p9_case_deviation(case):
    p, t1k, t2k, ((c1, c2), e) = case
    R = rcc.RCC(p)
    b1, b2 = R.residual(T(t1k), T(t2k))
    de = abs(e - complex(R.energy(T(t1k), T(t2k))))
    return max(np.abs(c1 - b1.numpy()).max(), np.abs(c2 - b2.numpy()).max(), de)


def _swap_first_equal_pair(spec, r):
    """Transpose the first two output indices of equal extent (a wrong-index mistake)."""
    out = spec.split("->")[1]
    for a in range(len(out)):
        for b in range(a + 1, len(out)):
            if r.shape[a] == r.shape[b] and r.shape[a] > 1:
                return r.transpose(a, b)
    return None


# Mutations that cannot change the compared quantities, with the reason:
EQUIVALENT = {
    # the dressed DF factors enter every integral in pairs, so L~ -> -L~ is exact
    ("pr,Qrs,sq->Qpq", "sign"): "DF factors enter in pairs",
    # 2 f_ia t1_ia vanishes for the canonical reference (f_ia = 0); the term matters once
    # the one-body part is perturbed (eta of Eq. 15) and P6 guards it there
    ("ia,ia->", "drop"): "f_ia = 0 (canonical)",
    ("ia,ia->", "sign"): "f_ia = 0 (canonical)",
}


def test_p9_guards_every_contraction_of_the_closed_shell_residual(monkeypatch):
    """Every contraction the closed-shell residual, its T1 dressing, its Fock build and
    its energy evaluate is planted, one at a time, with a dropped term, a flipped sign and
    (where two output indices have equal extent) transposed output indices; the
    comparison with the independent spin-orbital oracle fails for each, except the
    mutations listed in EQUIVALENT, which leave the compared quantities unchanged."""
    case = _p9_case()
    shapes = {}
    orig = rcc.ein

    def record(spec, *ops):
        r = orig(spec, *ops)
        shapes.setdefault(spec, tuple(r.shape))
        return r

    monkeypatch.setattr(rcc, "ein", record)
    assert _p9_case_deviation(case) < P9_TOL
    assert len(shapes) >= 20, sorted(shapes)
    missed, tried = [], 0
    for target, shape in shapes.items():
        for kind in ("drop", "sign", "swap"):
            if kind == "swap" and _swap_first_equal_pair(target, torch.zeros(shape)) is None:
                continue  # no two output indices of equal extent: nothing to transpose

            def mutated(spec, *ops, _t=target, _k=kind):
                r = orig(spec, *ops)
                if spec != _t:
                    return r
                if _k == "drop":
                    return torch.zeros_like(r)
                if _k == "sign":
                    return -r
                return _swap_first_equal_pair(spec, r)

            monkeypatch.setattr(rcc, "ein", mutated)
            tried += 1
            if _p9_case_deviation(case) <= 1e3 * P9_TOL:
                missed.append((target, kind))
    assert tried >= 50
    assert sorted(missed) == sorted(EQUIVALENT), sorted(set(missed) ^ set(EQUIVALENT))


def test_p6_catches_energy_singles_term(monkeypatch):
    """The singles term of the energy (Eq. 6), invisible to P9 at the canonical reference,
    enters alpha through eta (the one-body part perturbed by the dipole): dropping it
    fails P6."""
    assert _p6_deviation() < P6_TOL
    orig = rcc.ein
    monkeypatch.setattr(rcc, "ein", lambda spec, *ops: torch.zeros_like(orig(spec, *ops)) if spec == "ia,ia->"
                        else orig(spec, *ops))
    assert _p6_deviation() > 1e3 * P6_TOL


# P1, term by term ---------------------------------------------------------------------
def test_p1_guards_every_contraction_of_the_spin_orbital_residual(monkeypatch):
    """Every contraction of the spin-orbital residual (Oracle-A, the paper's arrangement of
    Eqs. 7-8) is planted in turn with a dropped term, a flipped sign and transposed output
    indices; the determinant-space brute force detects each.  A non-canonical one-body
    part (random Hermitian shift) and amplitudes that are neither spin-adapted nor
    momentum-conserving keep every term alive."""
    nk, o, v = 2, 1, 2
    p = make_problem(nk, o, v, 4, seed=5, sigma_l=0.3, tr=False)
    rng = np.random.default_rng(3)
    n = o + v
    F = 0.05 * (rng.normal(size=(nk, n, n)) + 1j * rng.normal(size=(nk, n, n)))
    F = F + F.conj().transpose(0, 2, 1)
    S = spinorb.SpinOrbitalSystem(p, fock_shift=F)
    O, V = S.O, S.V
    t1 = 0.1 * (rng.normal(size=(O, V)) + 1j * rng.normal(size=(O, V)))
    t2 = 0.1 * (rng.normal(size=(O, O, V, V)) + 1j * rng.normal(size=(O, O, V, V)))
    t2 = t2 - t2.transpose(1, 0, 2, 3)
    t2 = t2 - t2.transpose(0, 1, 3, 2)
    b1, b2 = fci.cc_residual(S, t1, t2)

    def deviation():
        a1, a2 = spinorb.residual(S, t1, t2)
        return max(np.abs(a1 - b1).max(), np.abs(a2 - b2).max())

    shapes = {}
    orig = spinorb.einsum

    def record(spec, *ops):
        r = orig(spec, *ops)
        shapes.setdefault(spec, r.shape)
        return r

    monkeypatch.setattr(spinorb, "einsum", record)
    assert deviation() < 1e-13
    assert len(shapes) >= 25, sorted(shapes)
    missed, tried = [], 0
    for target, shape in shapes.items():
        for kind in ("drop", "sign", "swap"):
            if kind == "swap" and _swap_first_equal_pair(target, torch.zeros(shape)) is None:
                continue

            def mutated(spec, *ops, _t=target, _k=kind):
                r = orig(spec, *ops)
                if spec != _t:
                    return r
                if _k == "drop":
                    return np.zeros_like(r)
                if _k == "sign":
                    return -r
                return np.asarray(_swap_first_equal_pair(spec, torch.as_tensor(r)))

            monkeypatch.setattr(spinorb, "einsum", mutated)
            tried += 1
            if deviation() <= 1e-10:
                missed.append((target, kind))
    assert tried >= 60
    assert not missed, missed


# P2, P3 -------------------------------------------------------------------------------
def _p2_deviation():
    """max deviation of the oracle's A.X from the brute-force commutator
    <mu| exp(-T) [H, X] exp(T) |0> (the P2 pin's comparison)."""
    nk, o, v = 2, 1, 2
    p = make_problem(nk, o, v, 4, seed=21, sigma_l=0.3)
    S = spinorb.SpinOrbitalSystem(p)
    R = rcc.RCC(p)
    t1k, t2k = random_amplitudes(nk, o, v, seed=22, scale1=0.1, scale2=0.1)
    x1k, x2k = random_amplitudes(nk, o, v, seed=23, scale1=1.0, scale2=1.0)
    a1, a2 = R.jacobian(T(t1k), T(t2k), T(x1k), T(x2k))
    t1, t2 = spinorb.to_spinorb(S, t1k, t2k)
    x1, x2 = spinorb.to_spinorb(S, x1k, x2k)
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
    return max(np.abs(c1 - a1.numpy()).max(), np.abs(c2 - a2.numpy()).max())


def _p3_deviation():
    """relative violation of <Y, A X> = <A^T Y, X> (the P3 pin's comparison), complex data."""
    nk, o, v = 3, 1, 2
    p = make_problem(nk, o, v, 4, seed=31, sigma_l=0.2, tr=False)
    R = rcc.RCC(p)
    t1, t2 = map(T, random_amplitudes(nk, o, v, seed=32, scale1=0.05, scale2=0.05))
    x1, x2 = map(T, random_amplitudes(nk, o, v, seed=40, scale1=1, scale2=1))
    y1, y2 = map(T, random_amplitudes(nk, o, v, seed=50, scale1=1, scale2=1))
    a1, a2 = R.jacobian(t1, t2, x1, x2)
    b1, b2 = R.transpose(t1, t2, y1, y2)
    lhs = complex((y1 * a1).sum() + (y2 * a2).sum())
    rhs = complex((b1 * x1).sum() + (b2 * x2).sum())
    return abs(lhs - rhs) / abs(lhs)


def _jacobian_three_point(self, t1, t2, x1, x2, h=None, blocks=None, singles=None):
    # central difference [f(s) - f(-s)] / 2s: not exact for the quartic CCSD residual
    s = max(float(torch.max(torch.abs(x1))), float(torch.max(torch.abs(x2))), 1e-300)
    hh = 1e-2 / s
    rp = self.residual(t1 + hh * x1, t2 + hh * x2, h, blocks, singles)
    rm = self.residual(t1 - hh * x1, t2 - hh * x2, h, blocks, singles)
    return (rp[0] - rm[0]) / (2 * hh), (rp[1] - rm[1]) / (2 * hh)


def _transpose_without_conj(orig):
    # the autograd gradient of a holomorphic function comes back conjugated; forgetting to
    # undo it turns the bilinear transpose into a sesquilinear one
    return lambda self, t1, t2, y1, y2, h=None: tuple(z.conj().resolve_conj() for z in orig(self, t1, t2, y1, y2, h))


def test_p2_catches_inexact_stencil(monkeypatch):
    assert _p2_deviation() < 1e-12
    monkeypatch.setattr(rcc.RCC, "jacobian", _jacobian_three_point)
    assert _p2_deviation() > 1e-9


def test_p3_catches_missing_conjugation(monkeypatch):
    assert _p3_deviation() < 1e-12
    monkeypatch.setattr(rcc.RCC, "transpose", _transpose_without_conj(rcc.RCC.transpose))
    assert _p3_deviation() > 1e-6


def test_p6_catches_lambda_sign(monkeypatch):
    """Lambda solved from A^T lam = +dE/dt instead of -dE/dt (Eqs. 10-11): alpha, which
    sees Lambda through eta and F, no longer equals FCI."""
    assert _p6_deviation() < P6_TOL
    orig = rcc.lagrangian_grad

    def wrong_sign(R, t1, t2, l1, l2, h=None):
        g1, g2 = orig(R, t1, t2, l1, l2, h)
        e1, e2 = R.energy_grad(t1, t2, h)
        return g1 - 2 * e1, g2 - 2 * e2

    monkeypatch.setattr(rcc, "lagrangian_grad", wrong_sign)
    assert _p6_deviation() > 1e3 * P6_TOL
