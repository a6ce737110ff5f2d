"""Brute force in determinant space (test infrastructure, tiny sizes only).

Gives values that do not depend on any CC algebra:
  * the CC residual  omega_mu = <mu| exp(-T) H exp(T) |0>  for arbitrary amplitudes,
    with H and T built as sparse matrices on the N-electron determinant space;
  * the exact (FCI) energy and the sum-over-states polarizability
        alpha_XY(w) = sum_n [ X_0n Y_n0 / (w_n - w) + Y_0n X_n0 / (w_n + w) ],
    which CCSD reproduces exactly for two electrons (Sec. II, Eq. 4 and the
    linear-response function of Eq. 15 are exact in that case).

Fermionic sign convention: a determinant is a bit string; a_p^dagger acting on it
carries (-1)^(number of occupied spin-orbitals with index < p).
"""
from __future__ import annotations

from itertools import combinations

import numpy as np
import scipy.sparse as sp


class DetSpace:
    def __init__(self, nso: int, nel: int):
        self.nso, self.nel = nso, nel
        dets = [sum(1 << p for p in c) for c in combinations(range(nso), nel)]
        self.dets = np.array(dets, dtype=np.int64)
        self.index = {d: i for i, d in enumerate(dets)}
        self.D = len(dets)
        self._E = {}

    def _popcount_below(self, d, p):
        mask = (1 << p) - 1
        x = d & mask
        c = np.zeros_like(x)
        while np.any(x):
            c += x & 1
            x = x >> 1
        return c

    def E(self, p: int, q: int) -> sp.csr_matrix:
        """Sparse matrix of a_p^dagger a_q on the determinant space."""
        key = (p, q)
        if key in self._E:
            return self._E[key]
        d = self.dets
        has_q = (d >> q) & 1 == 1
        d1 = np.where(has_q, d & ~(1 << q), 0)
        s1 = self._popcount_below(d1, q)          # sign from a_q on original d (bits below q)
        ok = has_q & ((((d1 >> p) & 1) == 0))
        d2 = d1 | (1 << p)
        s2 = self._popcount_below(d1, p)
        sign = np.where(((s1 + s2) % 2) == 0, 1.0, -1.0)
        rows, cols, vals = [], [], []
        for col in np.nonzero(ok)[0]:
            rows.append(self.index[int(d2[col])])
            cols.append(col)
            vals.append(sign[col])
        m = sp.csr_matrix((np.array(vals, dtype=np.complex128), (rows, cols)), shape=(self.D, self.D))
        self._E[key] = m
        return m

    def ref(self) -> np.ndarray:
        v = np.zeros(self.D, dtype=np.complex128)
        v[self.index[(1 << self.nel) - 1]] = 1.0
        return v


def _apply_H(ds: DetSpace, h, g, psi):
    """H psi with H = sum h_pq p+q + 1/2 sum g_pqrs p+q+sr, g_pqrs = <pq|rs>."""
    N = ds.nso
    out = np.zeros_like(psi)
    Y = {}
    for q in range(N):
        for s in range(N):
            y = ds.E(q, s) @ psi
            if np.any(y):
                Y[(q, s)] = y
    keys = list(Y.keys())
    Ymat = np.array([Y[k] for k in keys]) if keys else np.zeros((0, ds.D))
    for p in range(N):
        for r in range(N):
            coef = np.array([g[p, k[0], r, k[1]] for k in keys])
            if np.any(coef):
                out += 0.5 * (ds.E(p, r) @ (coef @ Ymat))
    hh = h - 0.5 * np.einsum("pqqs->ps", g)
    for p in range(N):
        for q in range(N):
            if hh[p, q] != 0:
                out += hh[p, q] * (ds.E(p, q) @ psi)
    return out


def _apply_T(ds: DetSpace, O, t1, t2, psi):
    """T psi, T = sum t1[I,A] a_A^+ a_I + 1/4 sum t2[I,J,A,B] a_A^+ a_I a_B^+ a_J."""
    N = ds.nso
    V = N - O
    out = np.zeros_like(psi)
    EB = {}
    for J in range(O):
        for B in range(V):
            EB[(J, B)] = ds.E(O + B, J) @ psi
    for I in range(O):
        for A in range(V):
            phi = t1[I, A] * psi
            for J in range(O):
                for B in range(V):
                    c = t2[I, J, A, B]
                    if c != 0:
                        phi = phi + 0.25 * c * EB[(J, B)]
            out += ds.E(O + A, I) @ phi
    return out


def _exp_T(ds, O, t1, t2, psi, sign=1.0):
    out = psi.copy()
    term = psi.copy()
    for n in range(1, ds.nel + 2):
        term = sign * _apply_T(ds, O, t1, t2, term) / n
        if not np.any(np.abs(term) > 0):
            break
        out = out + term
    return out


def cc_residual(sysA, t1, t2):
    """<mu| exp(-T) H exp(T) |0> for singles and doubles, spin-orbital amplitudes.

    sysA supplies the Fock matrix f and <PQ|RS> (g); the bare one-body part is
    h = f - sum_i <pi||qi>.  Returns (omega1[I,A], omega2[I,J,A,B]).
    """
    O, N = sysA.O, sysA.N
    V = N - O
    ds = DetSpace(N, O)
    g = sysA.g
    vas = g - g.transpose(0, 1, 3, 2)
    h = sysA.f - np.einsum("piqi->pq", vas[:, :O, :, :O])
    psi = _exp_T(ds, O, t1, t2, ds.ref(), 1.0)
    phi = _apply_H(ds, h, g, psi)
    om = _exp_T(ds, O, t1, t2, phi, -1.0)
    ref = ds.ref()
    r1 = np.zeros((O, V), dtype=np.complex128)
    r2 = np.zeros((O, O, V, V), dtype=np.complex128)
    for I in range(O):
        for A in range(V):
            mu = ds.E(O + A, I) @ ref
            r1[I, A] = np.vdot(mu, om)
    for I in range(O):
        for J in range(O):
            if J == I:
                continue
            for A in range(V):
                for B in range(V):
                    if B == A:
                        continue
                    mu = ds.E(O + A, I) @ (ds.E(O + B, J) @ ref)
                    r2[I, J, A, B] = np.vdot(mu, om)
    return r1, r2


def fci_states(sysA):
    """All eigenpairs of H on the N-electron space (dense; tiny sizes)."""
    O, N = sysA.O, sysA.N
    ds = DetSpace(N, O)
    g = sysA.g
    vas = g - g.transpose(0, 1, 3, 2)
    h = sysA.f - np.einsum("piqi->pq", vas[:, :O, :, :O])
    H = np.zeros((ds.D, ds.D), dtype=np.complex128)
    for c in range(ds.D):
        e = np.zeros(ds.D, dtype=np.complex128)
        e[c] = 1.0
        H[:, c] = _apply_H(ds, h, g, e)
    w, U = np.linalg.eigh(0.5 * (H + H.conj().T))
    return ds, w, U


def one_body_op(ds, m):
    """Sparse matrix of sum_pq m[p,q] a_p^+ a_q (m given on spin-orbitals)."""
    N = ds.nso
    out = sp.csr_matrix((ds.D, ds.D), dtype=np.complex128)
    for p in range(N):
        for q in range(N):
            if m[p, q] != 0:
                out = out + m[p, q] * ds.E(p, q)
    return out


def sos_polarizability(sysA, ops, omega):
    """alpha_XY(w) = sum_n [X_0n Y_n0/(w_n - w) + Y_0n X_n0/(w_n + w)], FCI states.

    ops: list of spin-orbital one-body matrices (Hermitian).  Returns (E0 - E_ref,
    alpha[len(ops), len(ops)]) where E_ref is the reference-determinant energy.
    """
    ds, w, U = fci_states(sysA)
    psi0 = U[:, 0]
    M = [one_body_op(ds, m) for m in ops]
    Xn = [U.conj().T @ (m @ psi0) for m in M]      # <n|X|0>
    dw = w - w[0]
    a = np.zeros((len(ops), len(ops)), dtype=np.complex128)
    for x in range(len(ops)):
        for y in range(len(ops)):
            s = 0.0
            for n in range(1, ds.D):
                x0n = np.conj(Xn[x][n])
                y0n = np.conj(Xn[y][n])
                s += x0n * Xn[y][n] / (dw[n] - omega) + y0n * Xn[x][n] / (dw[n] + omega)
            a[x, y] = s
    O = sysA.O
    eref = np.sum(np.real(np.diag(sysA.f)[:O])) - 0.5 * np.real(
        np.einsum("ijij->", (sysA.g - sysA.g.transpose(0, 1, 3, 2))[:O, :O, :O, :O]))
    return w[0] - eref, a
