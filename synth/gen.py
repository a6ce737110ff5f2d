"""Seeded generators for periodic (1D, k-point) LR-CCSD inputs.

Shapes follow the k-point layout of the method (paper Sec. II.A, Eq. 5 and Table I):
  L[k1, k2, Q, p, q]   density-fitting factors, paper units:
                       <pq|rs> = (pr|qs) = sum_Q L[kp,kr,Q,p,r] * L[kq,ks,Q,q,s]
                       defined when kp + kq = kr + ks (mod Nk)
  eps[k, p]            orbital energies (occupied first, then virtual)
  dip[c, k, p, q]      dipole integrals, k-diagonal, Hermitian per k, c in (x, y, z)
Amplitudes:
  t1[k, i, a]          (k_a = k_i)
  t2[ki, kj, ka, i, j, a, b]   (kb = ki + kj - ka mod Nk), closed-shell alpha-beta block
                       with the pair symmetry t2[ki,kj,ka,i,j,a,b] = t2[kj,ki,kb,j,i,b,a].

Random draws: one numpy Generator(PCG64(seed)), drawn in a fixed order
(eps_occ, eps_vir, L, dip).  Complex Gaussians are circular: real and imaginary
parts each N(0, sigma^2/2); diagonal entries of Hermitian blocks are real N(0, sigma^2).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

# Workload shapes (Nk, nocc, nvir, naux) of the synthetic 1D chains.
CONFIGS = {
    "c1": dict(nk=3, nocc=4, nvir=16, naux=48),
    "c2": dict(nk=5, nocc=8, nvir=40, naux=160),
    "c3": dict(nk=7, nocc=8, nvir=48, naux=200),
    "c4": dict(nk=9, nocc=12, nvir=64, naux=320),
    "c5": dict(nk=7, nocc=10, nvir=56, naux=240),
}


def kmesh_neg(nk: int, kmesh: int = 0) -> np.ndarray:
    """Index of -k for each k index.

    kmesh 0: Gamma-centred mesh k_m = 2 pi m / Nk.
    kmesh 1: NRecip=N with N odd (Nk = N-1 points, Gamma and the zone edge included).
    kmesh 2: NRecip=N with N even (Nk = N points shifted by half a step).
    (Sec. II.A and Fig. 1.)  Momentum conservation in index space is the same for
    every mesh: k_a + k_b = k_i + k_j (mod Nk); only the -k partner differs.
    """
    m = np.arange(nk)
    if kmesh in (0, 1):
        return (-m) % nk
    if kmesh == 2:
        return nk - 1 - m
    raise ValueError("kmesh must be 0, 1 or 2")


def pair_index(nk: int) -> np.ndarray:
    """kb for each (ki, kj, ka): kb = ki + kj - ka mod Nk, shape [Nk, Nk, Nk]."""
    k = np.arange(nk)
    return (k[:, None, None] + k[None, :, None] - k[None, None, :]) % nk


@dataclass
class Problem:
    nk: int
    nocc: int
    nvir: int
    naux: int
    L: np.ndarray
    eps: np.ndarray
    dip: np.ndarray
    kmesh: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nmo(self) -> int:
        return self.nocc + self.nvir


def _circ(rng, shape, sigma):
    return (rng.normal(0.0, sigma / np.sqrt(2.0), shape)
            + 1j * rng.normal(0.0, sigma / np.sqrt(2.0), shape))


def _hermitian_block(rng, naux, n, sigma, real):
    """[naux, n, n] blocks, Hermitian in (p, q); real symmetric when `real`."""
    iu = np.triu_indices(n, 1)
    out = np.zeros((naux, n, n), dtype=np.complex128)
    if real:
        up = rng.normal(0.0, sigma, (naux, len(iu[0])))
    else:
        up = _circ(rng, (naux, len(iu[0])), sigma)
    dg = rng.normal(0.0, sigma, (naux, n))
    out[:, iu[0], iu[1]] = up
    out[:, iu[1], iu[0]] = np.conj(up)
    out[:, np.arange(n), np.arange(n)] = dg
    return out


def _symmetric_block(rng, naux, n, sigma):
    """[naux, n, n] complex symmetric blocks (L_pq = L_qp)."""
    iu = np.triu_indices(n, 1)
    out = np.zeros((naux, n, n), dtype=np.complex128)
    up = _circ(rng, (naux, len(iu[0])), sigma)
    out[:, iu[0], iu[1]] = up
    out[:, iu[1], iu[0]] = up
    out[:, np.arange(n), np.arange(n)] = _circ(rng, (naux, n), sigma)
    return out


def _draw_L(rng, nk, naux, n, sigma, neg, tr):
    """Density-fitting factors with L[k2,k1,Q] = L[k1,k2,Q]^H (Hermiticity) and,
    when `tr`, L[-k1,-k2,Q] = conj(L[k1,k2,Q]) (time reversal)."""
    L = np.zeros((nk, nk, naux, n, n), dtype=np.complex128)
    done = np.zeros((nk, nk), dtype=bool)
    for k1 in range(nk):
        for k2 in range(nk):
            if done[k1, k2]:
                continue
            h = (k2, k1)
            t = (neg[k1], neg[k2]) if tr else None
            ht = (neg[k2], neg[k1]) if tr else None
            fix_h = h == (k1, k2)
            fix_t = tr and t == (k1, k2)
            fix_ht = tr and ht == (k1, k2)
            if fix_h and fix_t:
                blk = _hermitian_block(rng, naux, n, sigma, real=True)
            elif fix_h:
                blk = _hermitian_block(rng, naux, n, sigma, real=False)
            elif fix_t:
                blk = rng.normal(0.0, sigma, (naux, n, n)).astype(np.complex128)
            elif fix_ht:
                blk = _symmetric_block(rng, naux, n, sigma)
            else:
                blk = _circ(rng, (naux, n, n), sigma)
            L[k1, k2] = blk
            done[k1, k2] = True
            L[h] = np.conj(np.swapaxes(blk, 1, 2))
            done[h] = True
            if tr:
                L[t] = np.conj(blk)
                done[t] = True
                L[ht] = np.swapaxes(blk, 1, 2)
                done[ht] = True
    return L


def _draw_dip(rng, nk, n, sigma, neg, tr):
    dip = np.zeros((3, nk, n, n), dtype=np.complex128)
    for c in range(3):
        done = np.zeros(nk, dtype=bool)
        for k in range(nk):
            if done[k]:
                continue
            real = tr and neg[k] == k
            blk = _hermitian_block(rng, 1, n, sigma, real=real)[0]
            dip[c, k] = blk
            done[k] = True
            if tr:
                dip[c, neg[k]] = np.conj(blk)
                done[neg[k]] = True
    return dip


def make_problem(nk: int, nocc: int, nvir: int, naux: int, seed: int = 1266, *,
                 sigma_l: float = 0.02, sigma_mu: float = 0.5, kmesh: int = 0,
                 tr: bool = True, kind: str = "random") -> Problem:
    """Synthetic periodic problem.

    kind="random":  independent draws with the symmetries above.
    kind="replica": decoupled replicas of one molecule: L[k1,k2] = L_mol (real
                    symmetric) for every k pair, eps[k] = eps_mol, dip[:,k] = dip_mol
                    (real symmetric).  Each cell is then an isolated molecule.
    kind="zero":    L = 0 (no two-electron interaction).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n = nocc + nvir
    neg = kmesh_neg(nk, kmesh)
    if kind == "replica":
        eo = np.sort(rng.uniform(-1.5, -0.3, nocc))
        ev = np.sort(rng.uniform(0.2, 3.0, nvir))
        eps = np.tile(np.concatenate([eo, ev])[None, :], (nk, 1))
        lm = _hermitian_block(rng, naux, n, sigma_l, real=True)
        L = np.broadcast_to(lm[None, None], (nk, nk, naux, n, n)).copy()
        dm = np.stack([_hermitian_block(rng, 1, n, sigma_mu, real=True)[0] for _ in range(3)])
        dip = np.broadcast_to(dm[:, None], (3, nk, n, n)).copy()
        return Problem(nk, nocc, nvir, naux, L, eps, dip, kmesh,
                       dict(seed=seed, kind=kind, sigma_l=sigma_l, sigma_mu=sigma_mu, tr=True))
    eps = np.zeros((nk, n))
    reps = [k for k in range(nk) if (not tr) or k <= neg[k]]
    eo = rng.uniform(-1.5, -0.3, (len(reps), nocc))
    ev = rng.uniform(0.2, 3.0, (len(reps), nvir))
    for r, k in enumerate(reps):
        e = np.concatenate([np.sort(eo[r]), np.sort(ev[r])])
        eps[k] = e
        if tr:
            eps[neg[k]] = e
    if kind == "zero":
        L = np.zeros((nk, nk, naux, n, n), dtype=np.complex128)
    elif kind == "random":
        L = _draw_L(rng, nk, naux, n, sigma_l, neg, tr)
    else:
        raise ValueError(kind)
    dip = _draw_dip(rng, nk, n, sigma_mu, neg, tr)
    return Problem(nk, nocc, nvir, naux, L, eps, dip, kmesh,
                   dict(seed=seed, kind=kind, sigma_l=sigma_l, sigma_mu=sigma_mu, tr=tr))


def make_operator(nk: int, n: int, seed: int, parity: int = 1, sigma: float = 0.5, kmesh: int = 0) -> np.ndarray:
    """A k-diagonal one-body operator X[k, p, q], Hermitian per k, with time-reversal parity
    X(-k) = parity * conj(X(k)): +1 for electric-multipole-like operators (dipole, quadrupole;
    real symmetric at self-conjugate k), -1 for magnetic-dipole-like ones (purely imaginary
    at self-conjugate k)."""
    if parity not in (1, -1):
        raise ValueError("parity must be +1 or -1")
    rng = np.random.Generator(np.random.PCG64(seed))
    neg = kmesh_neg(nk, kmesh)
    X = np.zeros((nk, n, n), dtype=np.complex128)
    done = np.zeros(nk, dtype=bool)
    for k in range(nk):
        if done[k]:
            continue
        if neg[k] == k:  # X = parity conj(X) and Hermitian: real symmetric or imaginary antisymmetric
            if parity == 1:
                blk = _hermitian_block(rng, 1, n, sigma, real=True)[0]
            else:
                a = rng.normal(0.0, sigma, (n, n))
                blk = 1j * (a - a.T) / np.sqrt(2.0)
        else:
            blk = _hermitian_block(rng, 1, n, sigma, real=False)[0]
        X[k] = blk
        done[k] = True
        if neg[k] != k:
            X[neg[k]] = parity * np.conj(blk)
            done[neg[k]] = True
    return X


def symmetrize_pairs(t2: np.ndarray) -> np.ndarray:
    """Impose t2[ki,kj,ka,i,j,a,b] = t2[kj,ki,kb,j,i,b,a] by averaging."""
    nk = t2.shape[0]
    kb = pair_index(nk)
    sw = np.empty_like(t2)
    for ki in range(nk):
        for kj in range(nk):
            for ka in range(nk):
                sw[ki, kj, ka] = t2[kj, ki, kb[ki, kj, ka]].transpose(1, 0, 3, 2)
    return 0.5 * (t2 + sw)


def random_amplitudes(nk: int, nocc: int, nvir: int, seed: int, scale1: float = 1e-2,
                      scale2: float = 1e-2, symmetric: bool = True):
    """Random complex (t1, t2) with the momentum layout above; t2 pair-symmetric."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t1 = _circ(rng, (nk, nocc, nvir), scale1)
    t2 = _circ(rng, (nk, nk, nk, nocc, nocc, nvir, nvir), scale2)
    if symmetric:
        t2 = symmetrize_pairs(t2)
    return t1, t2


def random_probe(nk: int, nocc: int, nvir: int, seed: int, nrhs: int = 1,
                 scale: float = 1.0):
    """nrhs random probe vectors (x1 [nrhs,Nk,o,v], x2 [nrhs,Nk,Nk,Nk,o,o,v,v])."""
    x1s, x2s = [], []
    for r in range(nrhs):
        a, b = random_amplitudes(nk, nocc, nvir, seed + 7919 * r, scale, scale)
        x1s.append(a)
        x2s.append(b)
    return np.stack(x1s), np.stack(x2s)
