"""Planted mistakes in the CPU oracle are caught by its pins.

Each test patches one plausible mistake into oracle/rcc.py (on the CPU, for the duration
of the test) and checks that the pin meant to guard that part fails, after checking that
the same comparison passes unpatched:

  P9  closed-shell k-blocked residual and energy = spin-orbital ones: a sign error in
      the T1 similarity transform, a Fock build without exchange, an energy without the
      T1 terms (Eq. 6);
  P6  two electrons: alpha = FCI sum over states: the quadratic F term dropped from the
      response function (Eq. 15), the perturbation right-hand side (Eq. 12) off by its
      factor 1/2, a wrong sign of eta;
  P5  decoupled replicas: alpha per cell independent of Nk: the 1/Nk of alpha per cell
      missing.
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
