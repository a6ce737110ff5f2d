"""Host-side tests (no GPU): the library loads and exports every declared symbol,
the plan validates for every workload shape, and the op list reproduces the
oracle's Jacobian products when simulated on the CPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest
import torch

from synth import make_problem, random_amplitudes, CONFIGS
from oracle import rcc
import plan_sim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2508_01266_gb300 import _lib
    return _lib.lib


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "lrcc.h")).read()
    names = set(re.findall(r"\b(lrcc_[a-z_0-9]+)\s*\(", hdr))
    assert len(names) >= 15
    for n in sorted(names):
        assert hasattr(lib, n), n


@pytest.mark.parametrize("cfg", sorted(CONFIGS))
def test_plan_validates_for_workloads(lib, cfg):
    c = CONFIGS[cfg]
    pv = plan_sim.PlanView(lib, c["nk"], c["nocc"], c["nvir"], c["naux"], 1 << 26)
    msg = C.create_string_buffer(512)
    st = lib.lrcc_plan_validate(pv.h, msg, 512)
    assert st == 0, msg.value
    assert pv.flops[0] > 0 and pv.flops[1] > 0


def test_first_writes_fold_zeroing_at_c2(lib):
    """At the Nk=5 workload the permutations and GEMMs that are first writers of a whole
    scratch buffer store into it (no zero op ahead of them): 5 permutations and 21 GEMMs of
    the Jacobian program, 9 and 17 of its transpose; two zero ops remain in each (the ladder's
    half-filled pair-pair buffer and a singles transpose).  A store permutation never reads the
    buffer it writes."""
    c = CONFIGS["c2"]
    pv = plan_sim.PlanView(lib, c["nk"], c["nocc"], c["nvir"], c["naux"], 1 << 30)
    for which, want, want_g in ((1, 5, 21), (2, 9, 17)):
        ops = pv.programs[which]
        stores = [d for k, _, d in ops if k == "perm" and d["ints"][18]]
        assert len(stores) == want
        assert sum(1 for k, _, d in ops if k == "gemm" and d["ints"][15]) == want_g
        assert sum(1 for k, _, d in ops if k == "zero") == 2
        for d in stores:
            v = d["ints"]
            n = int(np.prod(v[8:12])) * int(v[7]) ** 3
            offS, offD = map(int, d["offs"])
            assert v[17] == 3  # scratch
            assert v[16] != v[17] or offS + n <= offD or offD + n <= offS


def _sim_setup(lib, prob, t1, t2sc, ws):
    nk, o, v, Q = prob.nk, prob.nocc, prob.nvir, prob.naux
    pv = plan_sim.PlanView(lib, nk, o, v, Q, ws)
    ar = [np.zeros(int(s), np.complex128) for s in pv.arena_sizes]
    off = pv.offsets
    L = prob.L / np.sqrt(nk)
    F = ar[0]

    def put(o_, x):
        F[o_:o_ + x.size] = x.ravel()
    put(off[0], L[:, :, :, :o, :o])
    put(off[1], L[:, :, :, :o, o:])
    put(off[2], L[:, :, :, o:, :o])
    put(off[3], L[:, :, :, o:, o:])
    n = o + v
    f0 = np.zeros((nk, n, n), complex)
    for k in range(nk):
        f0[k] = np.diag(prob.eps[k])
    put(off[4], f0)
    put(off[5], t1)
    put(off[6], t2sc * nk)
    put(off[7], np.eye(o))
    plan_sim.run(pv.programs[0], ar)
    return pv, ar


def _sim_apply(pv, ar, x1, x2p, which):
    a = [x.copy() for x in ar]
    for i in (1, 2):
        a[i][:] = 0
    # scratch and workspace start as garbage: the programs' own zero ops (scratch) and
    # overwriting W builds (workspace) must make every value they read defined
    for i in (3, 4):
        a[i][:] = np.nan
    off = pv.offsets
    fwd = which != 2  # the transposed program reads OUT and writes IN
    src = a[1] if fwd else a[2]
    src[off[8]:off[8] + x1.size] = x1.ravel()
    src[off[9]:off[9] + x2p.size] = x2p.ravel()
    plan_sim.run(pv.programs[which], a)
    r = a[2] if fwd else a[1]
    return r[off[8]:off[8] + x1.size].reshape(x1.shape), r[off[9]:off[9] + x2p.size].reshape(x2p.shape)


@pytest.mark.parametrize("nk,o,v,Q,ws", [(2, 1, 2, 3, 1 << 20), (3, 2, 3, 4, 1 << 20), (2, 3, 2, 3, 1),
                                          (4, 2, 2, 2, 40)])
def test_plan_simulation_matches_oracle(lib, nk, o, v, Q, ws):
    p = make_problem(nk, o, v, Q, seed=3, sigma_l=0.2)
    R = rcc.RCC(p)
    t1, t2 = random_amplitudes(nk, o, v, seed=4, scale1=0.05, scale2=0.05)
    x1, x2 = random_amplitudes(nk, o, v, seed=5, scale1=1, scale2=1)
    pv, ar = _sim_setup(lib, p, t1, t2, ws)
    y1, y2 = _sim_apply(pv, ar, x1, x2 * nk, 1)
    T = torch.as_tensor
    o1, o2 = R.jacobian(T(t1), T(t2), T(x1), T(x2))
    o1, o2 = o1.numpy(), o2.numpy() * nk
    assert np.abs(y1 - o1).max() < 1e-12 * np.abs(o1).max()
    assert np.abs(y2 - o2).max() < 1e-12 * np.abs(o2).max()
    g1, g2 = random_amplitudes(nk, o, v, seed=6, scale1=1, scale2=1)
    z1, z2 = _sim_apply(pv, ar, g1, g2, 2)
    b1, b2 = R.transpose(T(t1), T(t2), T(g1), T(g2 * nk))
    b1, b2 = b1.numpy(), b2.numpy() / nk
    assert np.abs(z1 - b1).max() < 1e-12 * np.abs(b1).max()
    assert np.abs(z2 - b2).max() < 1e-12 * np.abs(b2).max()


def _put_mu(pv, ar, mu, o):
    """One-body operator blocks oo, ov, vo, vv and ov^T into the FIX arena."""
    nk = mu.shape[0]
    off = int(pv.offsets[10])
    blocks = [mu[:, :o, :o], mu[:, :o, o:], mu[:, o:, :o], mu[:, o:, o:], np.swapaxes(mu[:, :o, o:], 1, 2)]
    for b in blocks:
        ar[0][off:off + b.size] = np.ascontiguousarray(b).ravel()
        off += b.size


@pytest.mark.parametrize("nk,o,v,Q", [(2, 2, 3, 3), (3, 1, 2, 4)])
def test_xi_and_egrad_programs(lib, nk, o, v, Q):
    """Perturbation right-hand side xi^X(t) and the singles energy Hessian, simulated."""
    p = make_problem(nk, o, v, Q, seed=8, sigma_l=0.2)
    R = rcc.RCC(p)
    t1, t2 = random_amplitudes(nk, o, v, seed=9, scale1=0.05, scale2=0.05)
    pv, ar = _sim_setup(lib, p, t1, t2, 1 << 20)
    mu = p.dip[2]
    _put_mu(pv, ar, mu, o)
    y1, y2 = _sim_apply(pv, ar, t1, t2 * nk, 3)
    T = torch.as_tensor
    x1, x2 = rcc.perturbation_rhs(R, T(t1), T(t2), T(mu))
    assert np.abs(y1 - x1.numpy()).max() < 1e-13 * np.abs(x1.numpy()).max()
    assert np.abs(y2 - nk * x2.numpy()).max() < 1e-13 * np.abs(nk * x2.numpy()).max()
    # egrad: <w, egrad(u)> = d^2 E / dt^2 [u, w] restricted to singles
    u1, _ = random_amplitudes(nk, o, v, seed=10, scale1=1, scale2=1)
    w1, _ = random_amplitudes(nk, o, v, seed=11, scale1=1, scale2=1)
    z = np.zeros((nk,) * 3 + (o, o, v, v), complex)
    g1, _ = _sim_apply(pv, ar, u1, z, 4)
    lhs = np.sum(w1 * g1)

    def E(a):
        return complex(R.energy(T(t1 + a[0] * u1 + a[1] * w1), T(t2)))
    h = 1e-2
    ref = (E((h, h)) - E((h, -h)) - E((-h, h)) + E((-h, -h))) / (4 * h * h)  # exact: E quadratic in t1
    assert abs(lhs - ref) < 1e-11 * abs(ref)


@pytest.mark.parametrize("nk,o,v,Q", [(2, 2, 3, 3), (3, 1, 2, 4)])
def test_omega0_and_tgrad_programs(lib, nk, o, v, Q):
    """Residual at zero amplitudes and the energy gradient, simulated, against the oracle
    (paper units: doubles of the residual times Nk, doubles of the gradient over Nk)."""
    p = make_problem(nk, o, v, Q, seed=12, sigma_l=0.2)
    R = rcc.RCC(p)
    t1, t2 = random_amplitudes(nk, o, v, seed=13, scale1=0.05, scale2=0.05)
    pv, ar = _sim_setup(lib, p, t1, t2, 1 << 20)
    z1 = np.zeros((nk, o, v), complex)
    z2 = np.zeros((nk,) * 3 + (o, o, v, v), complex)
    y1, y2 = _sim_apply(pv, ar, z1, z2, 5)
    T = torch.as_tensor
    r1, r2 = R.residual(T(z1), T(z2))
    assert np.abs(y1 - r1.numpy()).max() <= 1e-15
    assert np.abs(y2 - nk * r2.numpy()).max() < 1e-13 * np.abs(nk * r2.numpy()).max()
    g1, g2 = _sim_apply(pv, ar, t1, t2 * nk, 6)
    e1, e2 = R.energy_grad(T(t1), T(t2))
    assert np.abs(g1 - e1.numpy()).max() < 1e-13 * np.abs(e1.numpy()).max()
    assert np.abs(g2 - e2.numpy() / nk).max() < 1e-13 * np.abs(e2.numpy() / nk).max()


def test_residual_by_gauss_legendre_identity(lib):
    """Omega(t) = Omega(0) + 1/2 [A(s1 t) t + A(s2 t) t], s1,2 = (1 -+ 1/sqrt 3)/2: exact
    (A(s t) t is cubic in s); the GPU ground-state solver evaluates the residual this way."""
    nk, o, v, Q = 2, 2, 3, 3
    p = make_problem(nk, o, v, Q, seed=14, sigma_l=0.2)
    R = rcc.RCC(p)
    t1, t2 = random_amplitudes(nk, o, v, seed=15, scale1=0.1, scale2=0.1)
    z1 = np.zeros((nk, o, v), complex)
    z2 = np.zeros((nk,) * 3 + (o, o, v, v), complex)
    pv, ar = _sim_setup(lib, p, 0 * t1, 0 * t2, 1 << 20)
    w1, w2 = _sim_apply(pv, ar, z1, z2, 5)
    for s in (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)):
        pv, ar = _sim_setup(lib, p, s * t1, s * t2, 1 << 20)
        a1, a2 = _sim_apply(pv, ar, t1, t2 * nk, 1)
        w1, w2 = w1 + 0.5 * a1, w2 + 0.5 * a2
    T = torch.as_tensor
    r1, r2 = R.residual(T(t1), T(t2))
    assert np.abs(w1 - r1.numpy()).max() < 1e-12 * np.abs(r1.numpy()).max()
    assert np.abs(w2 - nk * r2.numpy()).max() < 1e-12 * np.abs(nk * r2.numpy()).max()
