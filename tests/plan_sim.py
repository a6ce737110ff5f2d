"""CPU simulator of a liblrcc op list (test infrastructure only).

Executes the ops exposed by the plan-introspection entry points of include/lrcc.h
on numpy arrays, so that the plan builder's index arithmetic (momentum blocks,
layouts, segment lists, transposition) can be checked against the oracle on a
machine without a GPU.  The library never uses this file.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

I32P = C.POINTER(C.c_int32)
I64P = C.POINTER(C.c_int64)
F64P = C.POINTER(C.c_double)


def _p(a, t):
    return a.ctypes.data_as(t)


class PlanView:
    """Reads the complete op list of a plan through the C introspection calls."""

    def __init__(self, lib, nk, o, v, Q, ws_budget=1 << 22):
        self.lib = lib
        lib.lrcc_plan_create.restype = C.c_int
        lib.lrcc_plan_num_ops.restype = C.c_int32

        at = getattr(lib.lrcc_plan_create, "argtypes", None)
        if at:
            Dims = at[0]._type_
        else:
            class Dims(C.Structure):
                _fields_ = [("nk", C.c_int32), ("nocc", C.c_int32), ("nvir", C.c_int32),
                            ("naux", C.c_int32), ("kmesh", C.c_int32)]
        d = Dims(nk, o, v, Q, 0)
        h = C.c_void_p()
        st = lib.lrcc_plan_create(C.byref(d), ws_budget, C.byref(h))
        assert st == 0, st
        self.h = h
        self.dims = (nk, o, v, Q)
        ar = np.zeros(5, np.int64)
        off = np.zeros(11, np.int64)
        fl = np.zeros(3, np.float64)
        lib.lrcc_plan_info(h, _p(ar, I64P), _p(off, I64P), _p(fl, F64P))
        self.arena_sizes, self.offsets, self.flops = ar, off, fl
        self.programs = [self._read(w) for w in range(7)]

    def _read(self, which):
        lib, h = self.lib, self.h
        n = lib.lrcc_plan_num_ops(h, which)
        ops = []
        kif = np.zeros(3, np.int32)
        for i in range(n):
            lib.lrcc_plan_op(h, which, i, _p(kif, I32P))
            kind, idx, fixed = map(int, kif)
            if kind == 0:
                ints = np.zeros(16, np.int32)
                lds = np.zeros(3, np.int64)
                al = np.zeros(2)
                lib.lrcc_plan_gemm(h, idx, _p(ints, I32P), _p(lds, I64P), _p(al, F64P), None, None, None, None)
                nb, ns = int(ints[13]), int(ints[14])
                coff = np.zeros(nb, np.int64)
                sbeg = np.zeros(nb + 1, np.int32)
                aoff = np.zeros(ns, np.int64)
                boff = np.zeros(ns, np.int64)
                lib.lrcc_plan_gemm(h, idx, None, None, None, _p(coff, I64P), _p(sbeg, I32P),
                                   _p(aoff, I64P), _p(boff, I64P))
                ops.append(("gemm", fixed, dict(ints=ints.copy(), lds=lds.copy(), alpha=complex(al[0], al[1]),
                                                coff=coff, sbeg=sbeg, aoff=aoff, boff=boff)))
            elif kind == 1:
                ints = np.zeros(19, np.int32)
                offs = np.zeros(2, np.int64)
                al = np.zeros(2)
                lib.lrcc_plan_perm(h, idx, _p(ints, I32P), _p(offs, I64P), _p(al, F64P))
                ops.append(("perm", fixed, dict(ints=ints.copy(), offs=offs.copy(), alpha=complex(al[0], al[1]))))
            elif kind == 3:
                ar = np.zeros(1, np.int32)
                on = np.zeros(2, np.int64)
                lib.lrcc_plan_zero(h, idx, _p(ar, I32P), _p(on, I64P))
                ops.append(("zero", fixed, dict(arena=int(ar[0]), off=int(on[0]), n=int(on[1]))))
            else:
                ints = np.zeros(5, np.int32)
                offs = np.zeros(2, np.int64)
                al = np.zeros(2)
                lib.lrcc_plan_btrans(h, idx, _p(ints, I32P), _p(offs, I64P), _p(al, F64P))
                ops.append(("btrans", fixed, dict(ints=ints.copy(), offs=offs.copy(), alpha=complex(al[0], al[1]))))
        return ops

    def __del__(self):
        try:
            self.lib.lrcc_plan_destroy(self.h)
        except Exception:
            pass


def layout_offsets(kind, nk, n, k1, k2, k3, i1, i2, i3, i4):
    """Vectorized element offsets (mirrors the layout definitions in include/lrcc.h's plan section)."""
    n0, n1, n2, n3 = n
    if kind == 0:
        return ((k1 * nk + k2) * nk + k3) * (n0 * n1 * n2 * n3) + ((i1 * n1 + i2) * n2 + i3) * n3 + i4
    if kind == 1:
        P = (k1 + k2) % nk
        rows, cols = nk * n0 * n1, nk * n2 * n3
        return P * rows * cols + ((k1 * n0 + i1) * n1 + i2) * cols + (k3 * n2 + i3) * n3 + i4
    if kind == 2:
        q = (k3 - k1) % nk
        k4 = (k1 + k2 - k3) % nk
        rows, cols = nk * n0 * n2, nk * n3 * n1
        return q * rows * cols + ((k1 * n0 + i1) * n2 + i3) * cols + (k4 * n3 + i4) * n1 + i2
    if kind == 3:
        return ((k1 * nk + k3) * nk + k2) * (n0 * n1 * n2 * n3) + ((i1 * n2 + i3) * n1 + i2) * n3 + i4
    raise ValueError(kind)


def _mat(buf, off, rows, cols, ld):
    if rows == 0 or cols == 0:
        return np.zeros((rows, cols), buf.dtype)
    end = off + (rows - 1) * ld + cols
    assert off >= 0 and end <= buf.size, (off, end, buf.size)
    return np.lib.stride_tricks.as_strided(buf[off:], shape=(rows, cols), strides=(ld * buf.itemsize, buf.itemsize))


def run(ops, arenas):
    for kind, _fixed, d in ops:
        if kind == "gemm":
            M, N, K, ta, tb, arA, arB, arC, epi, e0, e1, e2, e3, nb, ns, store = map(int, d["ints"])
            lda, ldb, ldc = map(int, d["lds"])
            al = d["alpha"]
            A, Bm, Cm = arenas[arA], arenas[arB], arenas[arC]
            for b in range(nb):
                acc = np.zeros((M, N), np.complex128)
                for s in range(d["sbeg"][b], d["sbeg"][b + 1]):
                    a = _mat(A, int(d["aoff"][s]), K if ta else M, M if ta else K, lda)
                    bb = _mat(Bm, int(d["boff"][s]), N if tb else K, K if tb else N, ldb)
                    acc += (a.T if ta else a) @ (bb.T if tb else bb)
                c0 = int(d["coff"][b])
                if epi == 0:
                    cm = _mat(Cm, c0, M, N, ldc)
                    if store:  # first writer: the old contents are not read
                        cm[...] = al * acc
                    else:
                        cm += al * acc
                else:
                    na, nbb, nc, nd = e0, e1, e2, e3
                    m = np.arange(M)[:, None]
                    n = np.arange(N)[None, :]
                    a_, c_ = m // nc, m % nc
                    b_, d_ = n // nd, n % nd
                    addr = c0 + ((a_ * nbb + b_) * nc + c_) * nd + d_
                    Cm[addr.ravel()] = (al * acc).ravel()
        elif kind == "perm":
            v = list(map(int, d["ints"]))
            skind, snk, sn = v[0], v[1], v[2:6]
            dkind, dnk, dn = v[6], v[7], v[8:12]
            pi = v[12:16]
            arS, arD = v[16], v[17]
            offS, offD = map(int, d["offs"])
            nk = dnk
            K = np.arange(nk)
            k1, k2, k3 = np.meshgrid(K, K, K, indexing="ij")
            k4 = (k1 + k2 - k3) % nk
            ks = [k1.ravel(), k2.ravel(), k3.ravel(), k4.ravel()]
            ii = np.meshgrid(*[np.arange(x) for x in dn], indexing="ij")
            ii = [x.ravel() for x in ii]
            # combine: all k-combos x all orbital combos
            kk = [x[:, None] for x in ks]
            io = [x[None, :] for x in ii]
            od = layout_offsets(dkind, nk, dn, kk[0], kk[1], kk[2], io[0], io[1], io[2], io[3])
            sk = [kk[pi[s]] for s in range(4)]
            si = [io[pi[s]] for s in range(4)]
            os_ = layout_offsets(skind, snk, sn, sk[0], sk[1], sk[2], si[0], si[1], si[2], si[3])
            Dst, Src = arenas[arD], arenas[arS]
            vals = d["alpha"] * Src[offS + os_.ravel()]
            if v[18]:  # store: every destination element written once, old values not read
                idx = offD + od.ravel()
                assert np.unique(idx).size == idx.size
                Dst[idx] = vals
            else:
                np.add.at(Dst, offD + od.ravel(), vals)
        elif kind == "zero":
            arenas[d["arena"]][d["off"]:d["off"] + d["n"]] = 0
        elif kind == "btrans":
            nb, R, Cc, arS, arD = map(int, d["ints"])
            offS, offD = map(int, d["offs"])
            src = arenas[arS][offS:offS + nb * R * Cc].reshape(nb, R, Cc)
            arenas[arD][offD:offD + nb * R * Cc] += d["alpha"] * src.transpose(0, 2, 1).reshape(-1)
    return arenas
