"""Oracle-B: closed-shell, k-blocked CCSD and LR-CCSD (test infrastructure only).

Plain CPU FP64/complex128 code (PyTorch CPU tensors, so that the transpose products
can be taken by reverse-mode differentiation).  Everything is written with explicit
loops over momentum blocks and one small contraction per block; nothing is fused or
reordered for speed.

Method (see also oracle/spinorb.py for the spin-orbital form of Eqs. 6-8):
  * Supercell reading: the Nk-point problem is a molecular CCSD on the supercell with
    two-electron integrals <pq|rs>_paper / Nk, so the code uses L_sc = L / sqrt(Nk) and
    supercell amplitudes s1 = t1, s2 = t2_paper / Nk.  Cell quantities are supercell
    quantities / Nk (Eq. 6 and Eq. 15 weights).
  * Closed shell: amplitudes are the alpha (singles) and alpha-beta (doubles) blocks of
    the spin-orbital amplitudes of Sec. II.A (the paper keeps all spin blocks with
    zeros; they are determined by these for a singlet).
  * T1 dressing: exp(-T1) H exp(T1) has the same form as H with one-body factors
    transformed as X -> (1 - tau) X (1 + tau), tau[a,i] = t1[i,a].  Applied to the DF
    factors this is L~ = (1 - tau) L (1 + tau) (so L~_ab = L_ab - sum_m t_m^a L_mb), and
    the CCSD residual becomes the CCD residual of the dressed Hamiltonian.
  * Residual Omega(t1, t2) = <mu| exp(-T) H exp(T) |0> (full Fock matrix, so Omega = 0
    at the solution; the D t terms of Eqs. 7-8 are included).
  * Right Jacobian product  A.X = d/dh Omega(t + h X)|_0, taken with the 5-point
    central stencil, which is exact for the degree-4 polynomial Omega (rounding only).
  * Transpose product  Y^T.A = grad_t <Y, Omega(t)> (bilinear, plain array pairing),
    projected onto pair-symmetric doubles.
  * Lambda (Eqs. 10-11): P_sym(A^T lam + grad E) = 0 with the plain pairing; lam is the
    multiplier of <lam, Omega>_plain, which equals the spin-orbital pairing of Eq. 6 /
    Eq. 15 (weights 1/Nk, 1/(4 Nk^3) in paper units) applied to the paper's lambda.
  * Perturbed amplitudes (Eqs. 13-14): (A - w) t^X(w) = -xi^X, xi^X = dOmega/d eps_X.
  * Linear response (Eq. 15, symmetric form):
      <<X;Y>>_w = 1/2 C^{+-w} P(X(-w), Y(w)) [eta^X t^Y(w) + 1/2 F t^X(-w) t^Y(w)],
      eta^X = d^2 L/d eps_X dt, F = d^2 L / dt^2, L = E + <lam, Omega>,
    alpha_XY(w) = -<<X;Y>>_w / Nk  (per cell; static alpha_zz > 0).
    All directional derivatives are exact polynomial stencils.
"""
from __future__ import annotations

import math

import numpy as np
import torch

DT = torch.complex128


def _t(x):
    return torch.as_tensor(np.asarray(x), dtype=DT)


def ein(spec, *ops):
    return torch.einsum(spec, *ops)


def blocks_of(t2):
    """Nested lists of the momentum blocks t2[ki][kj][ka] (views)."""
    return [[list(x.unbind(0)) for x in y.unbind(0)] for y in t2.unbind(0)]


class RCC:
    """Closed-shell k-point CCSD system built from a synth.Problem."""

    def __init__(self, prob, fock_shift=None):
        self.prob = prob
        nk, o, v = prob.nk, prob.nocc, prob.nvir
        self.nk, self.o, self.v, self.n = nk, o, v, o + v
        self.naux = prob.naux
        self.L = _t(prob.L) / math.sqrt(nk)                  # supercell units
        f = torch.zeros((nk, self.n, self.n), dtype=DT)
        for k in range(nk):
            f[k] = torch.diag(_t(prob.eps[k]))
        self.f0 = f
        self.h = f - self._G(self.L)                          # bare one-body part
        if fock_shift is not None:
            self.h = self.h + _t(fock_shift)

    # -- helpers -----------------------------------------------------------------
    def kb(self, ki, kj, ka):
        return (ki + kj - ka) % self.nk

    def _G(self, L):
        """Closed-shell two-electron Fock contribution sum_i 2(pq|ii) - (pi|iq)."""
        nk, o = self.nk, self.o
        G = torch.zeros((nk, self.n, self.n), dtype=DT)
        for k in range(nk):
            for kk in range(nk):
                G[k] = G[k] + 2.0 * ein("Qpq,Qii->pq", L[k, k], L[kk, kk][:, :o, :o])
                G[k] = G[k] - ein("Qpi,Qiq->pq", L[k, kk][:, :, :o], L[kk, k][:, :o, :])
        return G

    def dress(self, t1, h=None):
        """Dressed DF factors L~ and dressed Fock f~ for singles t1[k,i,a]."""
        nk, o = self.nk, self.o
        h = self.h if h is None else h
        eye = torch.eye(self.n, dtype=DT)
        Xl, Xr = [], []
        t1b = t1.unbind(0)
        for k in range(nk):
            tau = torch.zeros((self.n, self.n), dtype=DT)
            tau[o:, :o] = t1b[k].T
            Xl.append(eye - tau)
            Xr.append(eye + tau)
        Lt = torch.stack([torch.stack([ein("pr,Qrs,sq->Qpq", Xl[k1], self.L[k1, k2], Xr[k2])
                                       for k2 in range(nk)]) for k1 in range(nk)])
        ht = torch.stack([Xl[k] @ h[k] @ Xr[k] for k in range(nk)])
        ft = ht + self._G(Lt)
        return Lt, ft

    # -- residual ----------------------------------------------------------------
    def residual(self, t1, t2, h=None, blocks=None, singles=None):
        """Closed-shell CCSD residual (supercell units).

        Returns (omega1[k,i,a], omega2[ki,kj,ka,i,j,a,b]).  With `blocks` (a list of
        (ki, kj, ka)), only those doubles blocks are computed (the others stay zero)
        and the singles are skipped unless `singles` is True; used to sample large problems.
        """
        nk, o = self.nk, self.o
        O, Vs = slice(0, o), slice(o, self.n)
        Lt, ft = self.dress(t1, h)

        memo = {}

        def eri(kp, kq, kr, ks, sp, sq, sr, ss):
            # (pq|rs) = sum_Q L~_pq L~_rs, built once per call and block (the same block is
            # asked for by several amplitude blocks; the value does not depend on which)
            key = (kp, kq, kr, ks, sp.start, sq.start, sr.start, ss.start)
            if key not in memo:
                memo[key] = ein("Qpq,Qrs->pqrs", Lt[kp, kq][:, sp, sq], Lt[kr, ks][:, sr, ss])
            return memo[key]

        v = self.v

        def vvvv(ka, kc, kb_, kd):
            # (ac|bd) as the matrix [(c,d), (a,b)], built once per call and block: the same
            # block serves every (ki, kj) pair with ki + kj = ka + kb
            key = ("vvvv", ka, kc, kb_, kd)
            if key not in memo:
                blk = ein("Qac,Qbd->cdab", Lt[ka, kc][:, Vs, Vs], Lt[kb_, kd][:, Vs, Vs])
                memo[key] = blk.reshape(v * v, v * v)
            return memo[key]

        kb = self.kb
        # amplitude blocks t2[ki][kj][ka] taken apart once (one stacked gradient per level
        # under reverse-mode differentiation, instead of a full-size one per block read)
        t2b = blocks_of(t2)
        T = lambda ki, kj, ka: t2b[ki][kj][ka]                                      # noqa: E731
        U = lambda ki, kj, ka: 2.0 * t2b[ki][kj][ka] - t2b[ki][kj][kb(ki, kj, ka)].transpose(2, 3)  # noqa: E731
        K = range(nk)
        Ct, Dt, Ev, Eo = {}, {}, {}, {}

        def ct(kk, ki, ka):
            """(ki|ac) - 1/2 sum_ld t_li^ad (kd|lc), as [k,i,a,c]; kc = kk - ki + ka."""
            if (kk, ki, ka) not in Ct:
                kc = (kk - ki + ka) % nk
                c = eri(kk, ki, ka, kc, O, O, Vs, Vs)
                for kl in K:
                    kd = (kl + ki - ka) % nk
                    c = c - 0.5 * ein("liad,kdlc->kiac", T(kl, ki, ka), eri(kk, kd, kl, kc, O, Vs, O, Vs))
                Ct[kk, ki, ka] = c
            return Ct[kk, ki, ka]

        def dt(ka, ki, kk):
            """L_aikc + 1/2 sum_ld u_il^ad L_ldkc, as [a,i,k,c]; L_pqrs = 2(pq|rs) - (ps|rq)."""
            if (ka, ki, kk) not in Dt:
                kc = (ka - ki + kk) % nk
                d = 2.0 * eri(ka, ki, kk, kc, Vs, O, O, Vs) - eri(ka, kc, kk, ki, Vs, Vs, O, O).permute(0, 3, 2, 1)
                for kl in K:
                    kd = (ki + kl - ka) % nk
                    Lldkc = 2.0 * eri(kl, kd, kk, kc, O, Vs, O, Vs) - eri(kl, kc, kk, kd, O, Vs, O, Vs).permute(0, 3, 2, 1)
                    d = d + 0.5 * ein("ilad,ldkc->aikc", U(ki, kl, ka), Lldkc)
                Dt[ka, ki, kk] = d
            return Dt[ka, ki, kk]

        def ev(kb_):
            """f~_bc - sum_kld u_kl^bd (ld|kc)."""
            if kb_ not in Ev:
                e = ft[kb_][Vs, Vs].clone()
                for kk in K:
                    for kl in K:
                        kd = (kk + kl - kb_) % nk
                        e = e - ein("klbd,ldkc->bc", U(kk, kl, kb_), eri(kl, kd, kk, kb_, O, Vs, O, Vs))
                Ev[kb_] = e
            return Ev[kb_]

        def eo(kj):
            """f~_kj + sum_lcd u_lj^cd (kd|lc)."""
            if kj not in Eo:
                e = ft[kj][O, O].clone()
                for kl in K:
                    for kc in K:
                        kd = (kl + kj - kc) % nk
                        e = e + ein("ljcd,kdlc->kj", U(kl, kj, kc), eri(kj, kd, kl, kc, O, Vs, O, Vs))
                Eo[kj] = e
            return Eo[kj]

        def sym_part(ki, kj, ka):
            """C + D + E terms for one block (to be pair-symmetrized)."""
            kb_ = kb(ki, kj, ka)
            y = torch.zeros((o, o, self.v, self.v), dtype=DT)
            for kk in K:
                y = y - 0.5 * ein("kjbc,kiac->ijab", T(kk, kj, kb_), ct(kk, ki, ka))
                y = y - ein("kibc,kjac->ijab", T(kk, ki, kb_), ct(kk, kj, ka))
                y = y + 0.5 * ein("jkbc,aikc->ijab", U(kj, kk, kb_), dt(ka, ki, kk))
            y = y + ein("ijac,bc->ijab", T(ki, kj, ka), ev(kb_))
            y = y - ein("ikab,kj->ijab", T(ki, kj, ka), eo(kj))
            return y

        out_blocks = [(ki, kj, ka) for ki in K for kj in K for ka in K] if blocks is None else list(blocks)
        zero2 = torch.zeros((o, o, v, v), dtype=DT)
        r2b = [[[zero2 for _ in K] for _ in K] for _ in K]
        for (ki, kj, ka) in out_blocks:
            kb_ = kb(ki, kj, ka)
            # (ai|bj)
            r = eri(ka, ki, kb_, kj, Vs, O, Vs, O).permute(1, 3, 0, 2).clone()
            # A: particle-particle ladder, sum_cd t_ij^cd (ac|bd)
            for kc in K:
                kd = (ki + kj - kc) % nk
                r = r + (T(ki, kj, kc).reshape(o * o, v * v) @ vvvv(ka, kc, kb_, kd)).reshape(o, o, v, v)
            # B: hole-hole ladder with the quadratic tau-like piece
            for kk in K:
                kl = (ki + kj - kk) % nk
                W = eri(kk, ki, kl, kj, O, O, O, O)                                  # (ki|lj)[k,i,l,j]
                for kc in K:
                    kd = (ki + kj - kc) % nk
                    W = W + ein("ijcd,kcld->kilj", T(ki, kj, kc), eri(kk, kc, kl, kd, O, Vs, O, Vs))
                r = r + ein("klab,kilj->ijab", T(kk, kl, ka), W)
            # C, D, E with the pair symmetrizer P_ij^ab
            r = r + sym_part(ki, kj, ka) + sym_part(kj, ki, kb_).permute(1, 0, 3, 2)
            r2b[ki][kj][ka] = r
        r2 = torch.stack([torch.stack([torch.stack(r2b[ki][kj]) for kj in K]) for ki in K])

        r1b = [torch.zeros((o, self.v), dtype=DT) for _ in K]
        if (blocks is None) if singles is None else singles:
            for k in K:
                r = ft[k][Vs, O].T.clone()
                for km in K:
                    r = r + ein("imae,me->ia", U(k, km, k), ft[km][O, Vs])
                    for ke in K:
                        kf = (k + km - ke) % nk
                        r = r + ein("imef,aemf->ia", U(k, km, ke), eri(k, ke, km, kf, Vs, Vs, O, Vs))
                    for kn in K:
                        ke = (km + kn - k) % nk
                        r = r - ein("mnae,nemi->ia", U(km, kn, k), eri(kn, ke, km, k, O, Vs, O, O))
                r1b[k] = r
        return torch.stack(r1b), r2

    def energy(self, t1, t2, h=None):
        """Closed-shell supercell correlation energy (Eq. 6); divide by Nk per cell."""
        nk, o = self.nk, self.o
        O, Vs = slice(0, o), slice(o, self.n)
        h = self.h if h is None else h
        f = h + self._G(self.L)
        L = self.L
        e = 0.0
        t1b = t1.unbind(0)
        t2b = blocks_of(t2)
        for k in range(nk):
            e = e + 2.0 * ein("ia,ia->", f[k][O, Vs], t1b[k])
        for ki in range(nk):
            for kj in range(nk):
                for ka in range(nk):
                    kb = self.kb(ki, kj, ka)
                    iajb = ein("Qia,Qjb->iajb", L[ki, ka][:, O, Vs], L[kj, kb][:, O, Vs])
                    ibja = ein("Qib,Qja->iajb", L[ki, kb][:, O, Vs], L[kj, ka][:, O, Vs])
                    tau = t2b[ki][kj][ka]
                    if ka == ki:
                        tau = tau + ein("ia,jb->ijab", t1b[ki], t1b[kj])
                    e = e + ein("iajb,ijab->", 2.0 * iajb - ibja, tau)
        return e

    # -- products --------------------------------------------------------------
    def sym(self, x2):
        """Projection onto pair-symmetric doubles: (x + S x)/2, (Sx)_ij^ab = x_ji^ba."""
        nk = self.nk
        out = torch.zeros_like(x2)
        for ki in range(nk):
            for kj in range(nk):
                for ka in range(nk):
                    out[ki, kj, ka] = 0.5 * (x2[ki, kj, ka] + x2[kj, ki, self.kb(ki, kj, ka)].permute(1, 0, 3, 2))
        return out

    def jacobian(self, t1, t2, x1, x2, h=None, blocks=None, singles=None):
        """A.X by the exact 5-point stencil of the residual (supercell units).

        The stencil f'(0) = [f(-2s) - 8 f(-s) + 8 f(s) - f(2s)] / (12 s) is exact for
        polynomials of degree <= 4, which the CCSD residual is in (t1, t2).
        """
        s = max(float(torch.max(torch.abs(x1))) if x1.numel() else 0.0, float(torch.max(torch.abs(x2))), 1e-300)
        hh = 1e-2 / s
        r = [self.residual(t1 + c * hh * x1, t2 + c * hh * x2, h, blocks, singles) for c in (-2.0, -1.0, 1.0, 2.0)]
        y1 = (r[0][0] - 8.0 * r[1][0] + 8.0 * r[2][0] - r[3][0]) / (12.0 * hh)
        y2 = (r[0][1] - 8.0 * r[1][1] + 8.0 * r[2][1] - r[3][1]) / (12.0 * hh)
        return y1, y2

    def transpose(self, t1, t2, y1, y2, h=None):
        """P_sym(A^T Y) with the plain bilinear pairing <Y, Omega> = sum y1 o1 + sum y2 o2."""
        a1 = t1.detach().clone().requires_grad_(True)
        a2 = t2.detach().clone().requires_grad_(True)
        r1, r2 = self.residual(a1, a2, h)
        f = (y1 * r1).sum() + (y2 * r2).sum()
        g1, g2 = torch.autograd.grad(f, (a1, a2), grad_outputs=torch.ones((), dtype=DT))
        return g1.conj().resolve_conj().detach(), self.sym(g2.conj().resolve_conj().detach())

    def energy_grad(self, t1, t2, h=None):
        a1 = t1.detach().clone().requires_grad_(True)
        a2 = t2.detach().clone().requires_grad_(True)
        e = self.energy(a1, a2, h)
        g1, g2 = torch.autograd.grad(e, (a1, a2), grad_outputs=torch.ones((), dtype=DT))
        return g1.conj().resolve_conj().detach(), self.sym(g2.conj().resolve_conj().detach())

    # -- denominators and solvers ------------------------------------------------
    def denominators(self):
        """Diagonal orbital-energy differences eps_a - eps_i (Eq. 9 with the opposite sign)."""
        nk, o = self.nk, self.o
        e = torch.stack([torch.diagonal(self.f0[k]).real for k in range(nk)])
        d1 = torch.zeros((nk, o, self.v), dtype=torch.float64)
        d2 = torch.zeros((nk, nk, nk, o, o, self.v, self.v), dtype=torch.float64)
        for k in range(nk):
            d1[k] = e[k, o:][None, :] - e[k, :o][:, None]
        for ki in range(nk):
            for kj in range(nk):
                for ka in range(nk):
                    kb = self.kb(ki, kj, ka)
                    d2[ki, kj, ka] = (e[ka, o:][None, None, :, None] + e[kb, o:][None, None, None, :]
                                      - e[ki, :o][:, None, None, None] - e[kj, :o][None, :, None, None])
        return d1, d2


# -- units ---------------------------------------------------------------------
def to_paper(nk, x1, x2):
    """Supercell -> paper units for amplitude-like vectors (t2_paper = Nk s2)."""
    return x1, x2 * nk


def from_paper(nk, x1, x2):
    return x1, x2 / nk


# -- iterative solvers (Jacobi + DIIS, Sec. II.D) ------------------------------
class DIIS:
    """Direct inversion in the iterative subspace with a Hermitian error matrix."""

    def __init__(self, nvec=8):
        self.nvec = nvec
        self.x, self.e = [], []

    def update(self, x, e):
        self.x.append(x.clone())
        self.e.append(e.clone())
        if len(self.x) > self.nvec:
            self.x.pop(0)
            self.e.pop(0)
        m = len(self.x)
        if m < 2:
            return x
        B = torch.zeros((m + 1, m + 1), dtype=DT)
        for i in range(m):
            for j in range(m):
                B[i, j] = torch.vdot(self.e[i], self.e[j])
        # the coefficients minimise |sum c_i e_i| subject to sum c_i = 1 and do not change
        # when the error block is scaled; scaling it to O(1) keeps the bordered system
        # well conditioned when the errors are tiny near convergence
        B[:m, :m] = B[:m, :m] / torch.max(torch.abs(torch.diagonal(B[:m, :m])))
        B[m, :m] = -1.0
        B[:m, m] = -1.0
        rhs = torch.zeros(m + 1, dtype=DT)
        rhs[m] = -1.0
        c = torch.linalg.lstsq(B, rhs.unsqueeze(1)).solution[:, 0]
        return sum(c[i] * self.x[i] for i in range(m))


def _flat(a, b):
    return torch.cat([a.reshape(-1), b.reshape(-1)])


def _unflat(x, s1, s2):
    n1 = int(np.prod(s1))
    return x[:n1].reshape(s1), x[n1:].reshape(s2)


def _maxabs(a, b):
    return max(float(torch.max(torch.abs(a))) if a.numel() else 0.0, float(torch.max(torch.abs(b))))


def solve_ccsd(R: RCC, tol=1e-10, maxit=200, h=None, verbose=False):
    """Ground-state amplitudes with max|Omega| <= tol (supercell units)."""
    d1, d2 = R.denominators()
    t1 = torch.zeros((R.nk, R.o, R.v), dtype=DT)
    t2 = torch.zeros((R.nk,) * 3 + (R.o, R.o, R.v, R.v), dtype=DT)
    diis = DIIS()
    for it in range(maxit):
        r1, r2 = R.residual(t1, t2, h)
        err = _maxabs(r1, r2)
        if verbose:
            print("ccsd", it, err)
        if err <= tol:
            return t1, t2, it
        n1, n2 = t1 - r1 / d1, t2 - r2 / d2
        x = diis.update(_flat(n1, n2), _flat(n1 - t1, n2 - t2))
        t1, t2 = _unflat(x, t1.shape, t2.shape)
        t2 = R.sym(t2)
    raise RuntimeError("CCSD did not converge")


def lagrangian_grad(R: RCC, t1, t2, l1, l2, h=None):
    """P_sym grad_t [E + <lam, Omega>] = grad E + A^T lam (plain pairing)."""
    a1 = t1.detach().clone().requires_grad_(True)
    a2 = t2.detach().clone().requires_grad_(True)
    r1, r2 = R.residual(a1, a2, h)
    f = R.energy(a1, a2, h) + (l1 * r1).sum() + (l2 * r2).sum()
    g1, g2 = torch.autograd.grad(f, (a1, a2), grad_outputs=torch.ones((), dtype=DT))
    return g1.conj().resolve_conj().detach(), R.sym(g2.conj().resolve_conj().detach())


def solve_lambda(R: RCC, t1, t2, tol=1e-10, maxit=200, verbose=False):
    """Lambda multipliers (Eqs. 10-11) in the plain pairing, max|grad L| <= tol."""
    d1, d2 = R.denominators()
    e1, e2 = R.energy_grad(t1, t2)
    l1, l2 = -e1 / d1, -e2 / d2
    diis = DIIS()
    for it in range(maxit):
        g1, g2 = lagrangian_grad(R, t1, t2, l1, l2)
        err = _maxabs(g1, g2)
        if verbose:
            print("lambda", it, err)
        if err <= tol:
            return l1, l2, it
        n1, n2 = l1 - g1 / d1, l2 - g2 / d2
        x = diis.update(_flat(n1, n2), _flat(n1 - l1, n2 - l2))
        l1, l2 = _unflat(x, l1.shape, l2.shape)
    raise RuntimeError("Lambda did not converge")


def perturbation_rhs(R: RCC, t1, t2, mu):
    """xi^X = dOmega/d eps for h -> h + eps * mu (mu[k,p,q] k-diagonal).  Exact central
    difference with eps = 1 (Omega is linear in the one-body part)."""
    p1, p2 = R.residual(t1, t2, R.h + mu)
    m1, m2 = R.residual(t1, t2, R.h - mu)
    return 0.5 * (p1 - m1), 0.5 * (p2 - m2)


def solve_response(R: RCC, t1, t2, xi1, xi2, omega, tol=1e-11, maxit=300, verbose=False):
    """(A - w) x = -xi with relative residual <= tol (Jacobi + DIIS)."""
    d1, d2 = R.denominators()
    p1, p2 = d1 - omega, d2 - omega
    x1, x2 = -xi1 / p1, -xi2 / p2
    nrm = _maxabs(xi1, xi2)
    if nrm == 0.0:  # vanishing perturbation (Sec. II.C): the response amplitudes are zero
        return x1, x2, 0
    diis = DIIS()
    for it in range(maxit):
        a1, a2 = R.jacobian(t1, t2, x1, x2)
        r1, r2 = a1 - omega * x1 + xi1, a2 - omega * x2 + xi2
        err = _maxabs(r1, r2) / nrm
        if verbose:
            print("resp", it, err)
        if err <= tol:
            return x1, x2, it
        n1, n2 = x1 - r1 / p1, x2 - r2 / p2
        x = diis.update(_flat(n1, n2), _flat(n1 - x1, n2 - x2))
        x1, x2 = _unflat(x, x1.shape, x2.shape)
        x2 = R.sym(x2)
    raise RuntimeError("response equations did not converge")


def _d1(f, hh):
    """Exact first derivative of a degree<=4 polynomial from 4 samples."""
    return (f(-2 * hh) - 8 * f(-hh) + 8 * f(hh) - f(2 * hh)) / (12 * hh)


def _d2(f, hh):
    """Exact second derivative of a degree<=5 polynomial from 5 samples."""
    return (-f(2 * hh) + 16 * f(hh) - 30 * f(0.0) + 16 * f(-hh) - f(-2 * hh)) / (12 * hh * hh)


def lagrangian(R: RCC, t1, t2, l1, l2, h=None):
    r1, r2 = R.residual(t1, t2, h)
    return R.energy(t1, t2, h) + (l1 * r1).sum() + (l2 * r2).sum()


def eta_dot(R: RCC, t1, t2, l1, l2, mu, w1, w2):
    """eta^X . w = d/ds [dL/d eps_X](t + s w)."""
    def g(s):
        a1, a2 = t1 + s * w1, t2 + s * w2
        return 0.5 * (lagrangian(R, a1, a2, l1, l2, R.h + mu) - lagrangian(R, a1, a2, l1, l2, R.h - mu))
    sc = max(_maxabs(w1, w2), 1e-300)
    return _d1(g, 1e-2 / sc)


def F_dot(R: RCC, t1, t2, l1, l2, u1, u2, w1, w2):
    """F(u, w) = d^2 L / dt^2 [u, w] by polarization of exact line second derivatives."""
    def Q(z1, z2):
        sc = max(_maxabs(z1, z2), 1e-300)
        return _d2(lambda s: lagrangian(R, t1 + s * z1, t2 + s * z2, l1, l2), 1e-2 / sc)
    return 0.25 * (Q(u1 + w1, u2 + w2) - Q(u1 - w1, u2 - w2))


def polarizability(R: RCC, t1, t2, l1, l2, mus, omegas, tol=1e-11, verbose=False):
    """alpha_XY(w) per cell, symmetric LR-CCSD form (Eq. 15); mus[c] = [k,p,q]."""
    nc = len(mus)
    out = np.zeros((len(omegas), nc, nc), dtype=np.complex128)
    xis = [perturbation_rhs(R, t1, t2, m) for m in mus]
    for iw, w in enumerate(omegas):
        tp = [solve_response(R, t1, t2, *xis[c], w, tol)[:2] for c in range(nc)]      # t^X(+w)
        tm = [solve_response(R, t1, t2, *xis[c], -w, tol)[:2] for c in range(nc)] if w != 0 else tp
        for x in range(nc):
            for y in range(nc):
                a = (eta_dot(R, t1, t2, l1, l2, mus[x], *tp[y])
                     + eta_dot(R, t1, t2, l1, l2, mus[y], *tm[x])
                     + F_dot(R, t1, t2, l1, l2, *tm[x], *tp[y]))
                b = (eta_dot(R, t1, t2, l1, l2, mus[x], *tm[y])
                     + eta_dot(R, t1, t2, l1, l2, mus[y], *tp[x])
                     + F_dot(R, t1, t2, l1, l2, *tp[x], *tm[y]))
                lr = 0.5 * (complex(a) + np.conj(complex(b)))
                out[iw, x, y] = -lr / R.nk
    return out


def symmetric_alpha(nk, etas, tp, tm, ftp, ftm):
    """alpha_XY(w) per cell in the symmetric form of Eq. 15, assembled from vectors under the
    plain pairing: etas[c] = eta^X (eta_vector), tp[c] / tm[c] = t^X(+w) / t^X(-w)
    (solve_response), ftp[c] / ftm[c] = F t^X(+w) / F t^X(-w) (F_vector).  Same formula as
    `polarizability`, whose scalar stencils eta^X . w and F(u, w) are the pairings
    <eta^X, w> and <F u, w> of these vectors (all vectors pair-symmetric)."""
    nc = len(etas)
    out = np.zeros((nc, nc), dtype=np.complex128)
    for x in range(nc):
        for y in range(nc):
            a = _pair(*etas[x], *tp[y]) + _pair(*etas[y], *tm[x]) + _pair(*ftm[x], *tp[y])
            b = _pair(*etas[x], *tm[y]) + _pair(*etas[y], *tp[x]) + _pair(*ftp[x], *tm[y])
            out[x, y] = -0.5 * (a + np.conj(b)) / nk
    return out


def symmetric_alpha_from_scalars(nk, etas, tp, tm, Fmp):
    """alpha_XY(w) per cell in the symmetric form of Eq. 15 from eta vectors and the scalars
    Fmp[x][y] = F(t^x(-w), t^y(+w)) (F_dot); F is symmetric, so F(t^x(+w), t^y(-w)) =
    Fmp[y][x].  Same formula as `polarizability`."""
    nc = len(etas)
    out = np.zeros((nc, nc), dtype=np.complex128)
    for x in range(nc):
        for y in range(nc):
            a = _pair(*etas[x], *tp[y]) + _pair(*etas[y], *tm[x]) + complex(Fmp[x][y])
            b = _pair(*etas[x], *tm[y]) + _pair(*etas[y], *tp[x]) + complex(Fmp[y][x])
            out[x, y] = -0.5 * (a + np.conj(b)) / nk
    return out


def polarizability_vectors(R: RCC, t1, t2, l1, l2, mus, omegas, tol=1e-11):
    """`polarizability` (symmetric form, Eq. 15) evaluated through eta and F vectors: one
    eta vector per component and one F vector per response solution instead of one scalar
    stencil per (X, Y, w) pair, so that large problems need far fewer Lagrangian
    evaluations.  Mathematically identical; per cell."""
    nc = len(mus)
    out = np.zeros((len(omegas), nc, nc), dtype=np.complex128)
    xis = [perturbation_rhs(R, t1, t2, m) for m in mus]
    etas = [eta_vector(R, t1, t2, l1, l2, m) for m in mus]
    for iw, w in enumerate(omegas):
        tp = [solve_response(R, t1, t2, *xis[c], w, tol)[:2] for c in range(nc)]
        tm = [solve_response(R, t1, t2, *xis[c], -w, tol)[:2] for c in range(nc)] if w != 0 else tp
        ftp = [F_vector(R, t1, t2, l1, l2, *tp[c]) for c in range(nc)]
        ftm = [F_vector(R, t1, t2, l1, l2, *tm[c]) for c in range(nc)] if w != 0 else ftp
        out[iw] = symmetric_alpha(R.nk, etas, tp, tm, ftp, ftm)
    return out


def eta_vector(R: RCC, t1, t2, l1, l2, mu):
    """eta^X = P_sym grad_t dL/d eps_X in the plain pairing (Eq. 15 ingredients).  L is
    linear in the one-body operator, so the central difference with eps = 1 is exact."""
    p1, p2 = lagrangian_grad(R, t1, t2, l1, l2, R.h + mu)
    m1, m2 = lagrangian_grad(R, t1, t2, l1, l2, R.h - mu)
    return 0.5 * (p1 - m1), 0.5 * (p2 - m2)


def F_vector(R: RCC, t1, t2, l1, l2, u1, u2):
    """F u = d/ds [grad_t L](t + s u): exact 4-point stencil (grad L has degree <= 3 in t)."""
    sc = max(_maxabs(u1, u2), 1e-300)
    hh = 1e-2 / sc
    g = [lagrangian_grad(R, t1 + c * hh * u1, t2 + c * hh * u2, l1, l2) for c in (-2.0, -1.0, 1.0, 2.0)]
    f1 = (g[0][0] - 8.0 * g[1][0] + 8.0 * g[2][0] - g[3][0]) / (12.0 * hh)
    f2 = (g[0][1] - 8.0 * g[1][1] + 8.0 * g[2][1] - g[3][1]) / (12.0 * hh)
    return f1, f2


def solve_left_response(R: RCC, t1, t2, b1, b2, omega, tol=1e-11, maxit=300, verbose=False):
    """Left perturbed multipliers: y (A + w) = -b, i.e. (A^T + w) y = -b on the pair-symmetric
    subspace (transpose products), Jacobi + DIIS, relative residual <= tol."""
    d1, d2 = R.denominators()
    p1, p2 = d1 + omega, d2 + omega
    y1, y2 = -b1 / p1, -b2 / p2
    nrm = _maxabs(b1, b2)
    if nrm == 0.0:
        return y1, y2, 0
    diis = DIIS()
    for it in range(maxit):
        a1, a2 = R.transpose(t1, t2, y1, y2)
        r1, r2 = a1 + omega * y1 + b1, a2 + omega * y2 + b2
        err = _maxabs(r1, r2) / nrm
        if verbose:
            print("left", it, err)
        if err <= tol:
            return y1, y2, it
        n1, n2 = y1 - r1 / p1, y2 - r2 / p2
        x = diis.update(_flat(n1, n2), _flat(n1 - y1, n2 - y2))
        y1, y2 = _unflat(x, y1.shape, y2.shape)
        y2 = R.sym(y2)
    raise RuntimeError("left response equations did not converge")


def _pair(a1, a2, b1, b2):
    return complex((a1 * b1).sum() + (a2 * b2).sum())


def polarizability_left(R: RCC, t1, t2, l1, l2, mus, omegas, tol=1e-11):
    """alpha_XY(w) per cell from the asymmetric (left-response) form of the CC linear-
    response function:
        <<X;Y>>_w = 1/2 C^{+-w} [eta^Y t^X(-w) + tbar^X(-w) xi^Y],
        tbar^X(w) (A + w) = -(eta^X + F t^X(w)).
    Returns (symmetrised alpha = (alpha_XY + alpha_YX)/2, unsymmetrised alpha)."""
    nc = len(mus)
    out = np.zeros((len(omegas), nc, nc), dtype=np.complex128)
    xis = [perturbation_rhs(R, t1, t2, m) for m in mus]
    etas = [eta_vector(R, t1, t2, l1, l2, m) for m in mus]

    def left(c, tc, ws):
        f1, f2 = F_vector(R, t1, t2, l1, l2, *tc)
        return solve_left_response(R, t1, t2, etas[c][0] + f1, etas[c][1] + f2, ws, tol)[:2]

    for iw, w in enumerate(omegas):
        tp = [solve_response(R, t1, t2, *xis[c], w, tol)[:2] for c in range(nc)]
        tm = [solve_response(R, t1, t2, *xis[c], -w, tol)[:2] for c in range(nc)] if w != 0 else tp
        lm = [left(c, tm[c], -w) for c in range(nc)]
        lp = [left(c, tp[c], w) for c in range(nc)] if w != 0 else lm
        for x in range(nc):
            for y in range(nc):
                a = _pair(*etas[y], *tm[x]) + _pair(*lm[x], *xis[y])
                b = _pair(*etas[y], *tp[x]) + _pair(*lp[x], *xis[y])
                out[iw, x, y] = -0.5 * (a + np.conj(b)) / R.nk
    return 0.5 * (out + out.transpose(0, 2, 1)), out


def symmetric_basis(R: RCC):
    """Orthonormal basis of the amplitude space with pair-symmetric doubles: singles unit
    vectors, then one vector per orbit of the pair swap (ki,kj,ka,i,j,a,b) -> (kj,ki,kb,j,i,b,a):
    e_p for fixed points, (e_p + e_Sp)/sqrt 2 otherwise.  Returned as index lists."""
    nk, o, v = R.nk, R.o, R.v
    n1 = nk * o * v
    shape2 = (nk, nk, nk, o, o, v, v)
    seen = np.zeros(shape2, dtype=bool)
    pairs = []
    for idx in np.ndindex(*shape2):
        if seen[idx]:
            continue
        ki, kj, ka, i, j, a, b = idx
        sw = (kj, ki, R.kb(ki, kj, ka), j, i, b, a)
        seen[idx] = True
        seen[sw] = True
        pairs.append((idx, sw if sw != idx else None))
    return n1, shape2, pairs


def jacobian_matrix(R: RCC, t1, t2):
    """Dense Jacobian on the pair-symmetric subspace in the orthonormal basis of
    symmetric_basis (supercell units; columns are A applied to the basis vectors).
    Its eigenvalues are the linear-response excitation energies (poles of Eq. 15)."""
    n1, shape2, pairs = symmetric_basis(R)
    dim = n1 + len(pairs)
    s1 = (R.nk, R.o, R.v)
    A = np.zeros((dim, dim), dtype=np.complex128)

    def vec(c):
        x1 = np.zeros(s1, dtype=np.complex128)
        x2 = np.zeros(shape2, dtype=np.complex128)
        if c < n1:
            x1.reshape(-1)[c] = 1.0
        else:
            p, q = pairs[c - n1]
            if q is None:
                x2[p] = 1.0
            else:
                x2[p] = x2[q] = 1.0 / np.sqrt(2.0)
        return x1, x2

    def coords(y1, y2):
        out = np.zeros(dim, dtype=np.complex128)
        out[:n1] = y1.reshape(-1)
        for r, (p, q) in enumerate(pairs):
            out[n1 + r] = y2[p] if q is None else (y2[p] + y2[q]) / np.sqrt(2.0)
        return out

    for c in range(dim):
        x1, x2 = vec(c)
        y1, y2 = R.jacobian(t1, t2, torch.as_tensor(x1), torch.as_tensor(x2))
        A[:, c] = coords(y1.numpy(), y2.numpy())
    return A


def excitation_energies(R: RCC, t1, t2, nroots=None):
    """Eigenvalues of the Jacobian (LR-CCSD excitation energies), sorted by real part."""
    w = np.linalg.eigvals(jacobian_matrix(R, t1, t2))
    w = w[np.argsort(w.real)]
    return w if nroots is None else w[:nroots]


def dipole_ops(prob, comps=(0, 1, 2)):
    """k-diagonal dipole matrices mu[k,p,q] for the chosen components."""
    return [_t(prob.dip[c]) for c in comps]
