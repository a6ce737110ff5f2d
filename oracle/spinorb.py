"""Oracle-A: dense spin-orbital CCSD with collective indices (test infrastructure).

Follows the paper's formulation: spin-orbitals with collective index P = (p, k_p, spin),
forbidden spin and momentum blocks kept as explicit zeros (Sec. II.A, Table I), the
energy of Eq. 6 and the amplitude equations of Eqs. 7-8 in that arrangement (no W_abef
intermediate: <AB||EF> contracted directly plus the t1 * (tau <MB||EF>) term, and the
tau <MN||EF> part carried twice in W_MNIJ).  The intermediates of Eqs. S1-S6 are not in
the paper; they are the standard spin-orbital Hbar elements (Stanton-Gauss type) that
the text says they are based on.

Normalization (supercell reading of Sec. II.B): the Nk-point problem is one molecular
CCSD on the Born-von Karman supercell with v = <PQ||RS>_paper / Nk.  Every 1/Nk factor
of Eqs. 6-8 follows from t2_paper = Nk * s2, lambda2_paper = Nk * l2 and
E_cell = E_supercell / Nk.  This module works in supercell units (s1, s2, v) and the
wrappers convert.

Residual convention: omega = <mu| exp(-T) H exp(T) |0> with the full Fock matrix
(diagonal included), so omega = 0 at the CCSD solution; Eq. 7-8's left-hand D t terms
are part of it.  Integrals carry their physical index order: excitation integrals
<ab||ij>, f_ai appear where the paper writes <IJ||AB>*, f_IA under its stated
assumption <PQ|RS>* = <RS|PQ> (Sec. II.C), which holds exactly for Hermitian DF factors.
"""
from __future__ import annotations

import numpy as np

einsum = lambda *a: np.einsum(*a, optimize=True)  # noqa: E731


class SpinOrbitalSystem:
    """Dense spin-orbital Fock matrix and antisymmetrized integrals of a Problem.

    Spin-orbital order: occupied (k, i, spin) first, then virtual (k, a, spin); index
    within each group = (k * n_per_k + orbital) * 2 + spin.
    """

    def __init__(self, prob, fock_shift=None):
        nk, o, v = prob.nk, prob.nocc, prob.nvir
        n = o + v
        self.nk, self.o, self.v = nk, o, v
        self.O, self.V = 2 * nk * o, 2 * nk * v
        N = self.O + self.V
        self.N = N
        # spatial collective labels for each spin-orbital
        lab = []
        for k in range(nk):
            for i in range(o):
                for s in range(2):
                    lab.append((k, i, s))
        for k in range(nk):
            for a in range(v):
                for s in range(2):
                    lab.append((k, o + a, s))
        self.lab = lab
        kk = np.array([l[0] for l in lab])
        pp = np.array([l[1] for l in lab])
        ss = np.array([l[2] for l in lab])
        self.kk, self.pp, self.ss = kk, pp, ss
        # Fock: diagonal orbital energies (canonical), optional one-body shift
        f = np.zeros((N, N), dtype=np.complex128)
        f[np.arange(N), np.arange(N)] = prob.eps[kk, pp]
        if fock_shift is not None:  # fock_shift[k, p, q], k-diagonal, spin-free
            same = (kk[:, None] == kk[None, :]) & (ss[:, None] == ss[None, :])
            f = f + np.where(same, fock_shift[kk[:, None], pp[:, None], pp[None, :]], 0.0)
        self.f = f
        # <PQ|RS> = (PR|QS), supercell units (1/Nk)
        L = prob.L / np.sqrt(nk)
        Lg = L[kk[:, None], kk[None, :], :, pp[:, None], pp[None, :]]  # [N, N, naux]
        spin_pr = (ss[:, None] == ss[None, :])
        Lg = Lg * spin_pr[:, :, None]
        g = einsum("prQ,qsQ->pqrs", Lg, Lg)
        mom = ((kk[:, None, None, None] + kk[None, :, None, None]
                - kk[None, None, :, None] - kk[None, None, None, :]) % nk) == 0
        g = np.where(mom, g, 0.0)
        self.g = g
        self.v_as = g - g.transpose(0, 1, 3, 2)   # <PQ||RS>

    def blocks(self):
        O = self.O
        o_, v_ = slice(0, O), slice(O, self.N)
        return o_, v_


def residual(sys: SpinOrbitalSystem, t1, t2):
    """Spin-orbital CCSD residual (supercell units), Eqs. 7-8 arrangement.

    t1[I, A], t2[I, J, A, B]; returns (omega1[I, A], omega2[I, J, A, B]).
    """
    o, v = sys.blocks()
    f = sys.f
    w = sys.v_as
    fov, fvo, foo, fvv = f[o, v], f[v, o], f[o, o], f[v, v]
    oooo, ooov, oovv = w[o, o, o, o], w[o, o, o, v], w[o, o, v, v]
    ovvv, ovov, ovvo = w[o, v, v, v], w[o, v, o, v], w[o, v, v, o]
    vvoo, vvvv, vvvo, ovoo = w[v, v, o, o], w[v, v, v, v], w[v, v, v, o], w[o, v, o, o]
    vovv = w[v, o, v, v]
    ooij_ie = ooov                      # <mn||ie>
    tau = t2 + einsum("ia,jb->ijab", t1, t1) - einsum("ib,ja->ijab", t1, t1)
    taut = t2 + 0.5 * (einsum("ia,jb->ijab", t1, t1) - einsum("ib,ja->ijab", t1, t1))

    # Hbar-type intermediates (the roles of Eqs. S1-S6)
    Fae = (fvv - 0.5 * einsum("me,ma->ae", fov, t1)
           + einsum("mf,mafe->ae", t1, w[o, v, v, v])
           - 0.5 * einsum("mnaf,mnef->ae", taut, oovv))
    Fmi = (foo + 0.5 * einsum("ie,me->mi", t1, fov)
           + einsum("ne,mnie->mi", t1, ooij_ie)
           + 0.5 * einsum("inef,mnef->mi", taut, oovv))
    Fme = fov + einsum("nf,mnef->me", t1, oovv)
    Wmnij = (oooo + einsum("je,mnie->mnij", t1, ooij_ie)
             - einsum("ie,mnje->mnij", t1, ooij_ie)
             + 0.5 * einsum("ijef,mnef->mnij", tau, oovv))
    Wmbej = (ovvo + einsum("jf,mbef->mbej", t1, ovvv)
             - einsum("nb,mnej->mbej", t1, w[o, o, v, o])
             - einsum("jnfb,mnef->mbej", 0.5 * t2 + einsum("jf,nb->jnfb", t1, t1), oovv))

    # Eq. 7 (singles)
    r1 = (fvo.T.copy()
          + einsum("ie,ae->ia", t1, Fae)
          - einsum("ma,mi->ia", t1, Fmi)
          + einsum("imae,me->ia", t2, Fme)
          - 0.5 * einsum("imef,maef->ia", t2, ovvv)
          + 0.5 * einsum("mnae,nmie->ia", t2, ooij_ie)
          + einsum("nf,nafi->ia", t1, w[o, v, v, o]))

    # Eq. 8 (doubles)
    vvij = vvoo.transpose(2, 3, 0, 1)                   # <ab||ij> as [i,j,a,b]
    r2 = vvij.copy()
    Fbe = Fae - 0.5 * einsum("mb,me->be", t1, Fme)
    tmp = einsum("ijae,be->ijab", t2, Fbe) - einsum("ma,mbij->ijab", t1, ovoo)
    r2 += tmp - tmp.transpose(0, 1, 3, 2)
    Fmj = Fmi + 0.5 * einsum("je,me->mj", t1, Fme)
    tmp = einsum("imab,mj->ijab", t2, Fmj) - einsum("ie,abej->ijab", t1, vvvo)
    r2 -= tmp - tmp.transpose(1, 0, 2, 3)
    tmp = (einsum("imae,mbej->ijab", t2, Wmbej)
           - einsum("ie,ma,mbej->ijab", t1, t1, ovvo))
    r2 += tmp - tmp.transpose(1, 0, 2, 3) - tmp.transpose(0, 1, 3, 2) + tmp.transpose(1, 0, 3, 2)
    r2 += 0.5 * einsum("ijef,abef->ijab", tau, vvvv)
    r2 += 0.5 * einsum("mnab,mnij->ijab", tau, Wmnij)
    tmp = einsum("ma,ijmb->ijab", t1, 0.5 * einsum("ijef,mbef->ijmb", tau, ovvv))
    r2 -= tmp - tmp.transpose(0, 1, 3, 2)
    return r1, r2


def energy(sys: SpinOrbitalSystem, t1, t2):
    """Eq. 6 in supercell units: E = f_IA t_I^A + 1/4 tau_IJ^AB <IJ||AB>."""
    o, v = sys.blocks()
    tau = t2 + einsum("ia,jb->ijab", t1, t1) - einsum("ib,ja->ijab", t1, t1)
    return einsum("ia,ia->", sys.f[o, v], t1) + 0.25 * einsum("ijab,ijab->", tau, sys.v_as[o, o, v, v])


# ---- closed-shell k-blocked <-> spin-orbital maps ---------------------------------

def to_spinorb(sys: SpinOrbitalSystem, t1k, t2k):
    """Spin-orbital amplitudes from closed-shell k-blocked ones (supercell units).

    t1_so[(ki,i,s),(ka,a,s)] = t1k[ki,i,a] (ka = ki);
    t2_so[I,J,A,B] = d(sI,sA) d(sJ,sB) t_ij^ab - d(sI,sB) d(sJ,sA) t_ij^ba.
    """
    nk, o, v = sys.nk, sys.o, sys.v
    O, V = sys.O, sys.V
    ko, io, so = sys.kk[:O], sys.pp[:O], sys.ss[:O]
    kv, av, sv = sys.kk[O:], sys.pp[O:] - o, sys.ss[O:]
    t1 = np.where((ko[:, None] == kv[None, :]) & (so[:, None] == sv[None, :]),
                  t1k[ko[:, None], io[:, None], av[None, :]], 0.0)
    # spatial collective t2[I,J,A,B] = t2k[ki,kj,ka,i,j,a,b] if momentum conserved
    KI, KJ, KA, KB = np.ix_(ko, ko, kv, kv)
    II, JJ, AA, BB = np.ix_(io, io, av, av)
    mom = ((KI + KJ - KA - KB) % nk) == 0
    tsp = np.where(mom, t2k[KI, KJ, KA, II, JJ, AA, BB], 0.0)
    SI, SJ, SA, SB = np.ix_(so, so, sv, sv)
    t2 = np.where((SI == SA) & (SJ == SB), tsp, 0.0) - np.where((SI == SB) & (SJ == SA),
                                                               tsp.transpose(0, 1, 3, 2), 0.0)
    return t1, t2


def from_spinorb(sys: SpinOrbitalSystem, r1, r2):
    """Closed-shell k-blocked (alpha / alpha-beta) blocks of spin-orbital tensors."""
    nk, o, v = sys.nk, sys.o, sys.v
    O = sys.O
    idx_o = lambda k, i, s: (k * o + i) * 2 + s          # noqa: E731
    idx_v = lambda k, a, s: (k * v + a) * 2 + s          # noqa: E731
    r1k = np.zeros((nk, o, v), dtype=np.complex128)
    r2k = np.zeros((nk, nk, nk, o, o, v, v), dtype=np.complex128)
    oi = np.array([[idx_o(k, i, 0) for i in range(o)] for k in range(nk)])
    ob = np.array([[idx_o(k, i, 1) for i in range(o)] for k in range(nk)])
    va = np.array([[idx_v(k, a, 0) for a in range(v)] for k in range(nk)])
    vb = np.array([[idx_v(k, a, 1) for a in range(v)] for k in range(nk)])
    for k in range(nk):
        r1k[k] = r1[np.ix_(oi[k], va[k])]
    for ki in range(nk):
        for kj in range(nk):
            for ka in range(nk):
                kb = (ki + kj - ka) % nk
                r2k[ki, kj, ka] = r2[np.ix_(oi[ki], ob[kj], va[ka], vb[kb])]
    return r1k, r2k


def one_body_to_spinorb(sys: SpinOrbitalSystem, m):
    """Spin-orbital matrix of a spin-free, k-diagonal one-body operator m[k,p,q]."""
    kk, pp, ss = sys.kk, sys.pp, sys.ss
    same = (kk[:, None] == kk[None, :]) & (ss[:, None] == ss[None, :])
    return np.where(same, m[kk[:, None], pp[:, None], pp[None, :]], 0.0)


def mp2_energy(sys: SpinOrbitalSystem):
    """Closed form  E = 1/4 sum <IJ||AB><AB||IJ> / (e_I + e_J - e_A - e_B)  (supercell)."""
    o, v = sys.blocks()
    e = np.real(np.diag(sys.f))
    D = (e[o][:, None, None, None] + e[o][None, :, None, None]
         - e[v][None, None, :, None] - e[v][None, None, None, :])
    w = sys.v_as
    num = w[o, o, v, v] * w[v, v, o, o].transpose(2, 3, 0, 1)
    return 0.25 * np.sum(num / D)
