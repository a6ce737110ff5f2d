"""GB300-native periodic LR-CCSD: k-point Jacobian products and polarizability.

Thin Python layer over liblrcc.so (include/lrcc.h).  The functions below carry the
C entry points' names without the `lrcc_` prefix and only marshal arguments:
torch tensors supply device memory and streams, the library runs every step.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._lib import lib, lrcc_dims, lrcc_options, STATUS, LIB_PATH

__all__ = ["LrccError", "Problem", "default_options", "create", "set_integrals", "set_ground_state",
           "jacobian_apply", "polarizability", "last_error", "destroy", "kernel_launches", "profile",
           "profile_query", "profile_report", "batch_polarizability", "residual", "solve_ground_state", "excitation_energies", "LRCCJacobian", "jacobian", "LIB_PATH"]


class LrccError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(st, h):
    if st != 0:
        msg = lib.lrcc_last_error(h) if h else b""
        raise LrccError(st, (msg or b"").decode())


def default_options(**kw) -> lrcc_options:
    o = lrcc_options()
    lib.lrcc_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v.encode() if k == "log_path" and isinstance(v, str) else v)
    return o


def _ptr(t: torch.Tensor):
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if t.is_conj() or t.is_neg():
        raise ValueError("tensor has a lazy conjugate/negation bit: resolve it first")
    return C.c_void_p(t.data_ptr())


def _dense(t: torch.Tensor) -> torch.Tensor:
    """Contiguous tensor whose memory holds its values (lazy conj/neg views resolved)."""
    return t.resolve_conj().resolve_neg().contiguous()


def _c128(x, device):
    t = torch.as_tensor(x) if not isinstance(x, torch.Tensor) else x
    return _dense(t.to(device=device, dtype=torch.complex128))


def create(nk, nocc, nvir, naux, kmesh=0):
    d = lrcc_dims(nk, nocc, nvir, naux, kmesh)
    h = C.c_void_p()
    st = lib.lrcc_create(C.byref(d), C.byref(h))
    if st != 0:
        msg = lib.lrcc_last_error(h) if h else b""
        if h:
            lib.lrcc_destroy(h)
        raise LrccError(st, (msg or b"").decode())
    return h


def destroy(h):
    lib.lrcc_destroy(h)


def last_error(h) -> str:
    return (lib.lrcc_last_error(h) or b"").decode()


def kernel_launches(h) -> int:
    return int(lib.lrcc_kernel_launches(h))


def profile(h, enable=True):
    _check(lib.lrcc_profile(h, int(bool(enable))), h)


def profile_query(h, tag=""):
    ms, fl = C.c_double(), C.c_double()
    cnt = C.c_int64()
    _check(lib.lrcc_profile_query(h, tag.encode(), C.byref(ms), C.byref(cnt), C.byref(fl)), h)
    return ms.value, cnt.value, fl.value


def profile_report(h):
    """Per-tag totals of the recorded ops, slowest first: [(tag, ms, count, flops)]."""
    buf = C.create_string_buffer(1 << 20)
    _check(lib.lrcc_profile_report(h, buf, len(buf)), h)
    rows = []
    for line in buf.value.decode().splitlines():
        tag, ms, n, fl = line.split("\t")
        rows.append((tag, float(ms), int(n), float(fl)))
    return rows


def set_integrals(h, L, eps, dip):
    dev = torch.device("cuda")
    Lt, dt = _c128(L, dev), _c128(dip, dev)
    et = torch.as_tensor(eps).to(device=dev, dtype=torch.float64).contiguous()
    _check(lib.lrcc_set_integrals(h, _ptr(Lt), _ptr(et), _ptr(dt), 1), h)


def set_ground_state(h, t1, t2, l1=None, l2=None):
    dev = torch.device("cuda")
    a, b = _c128(t1, dev), _c128(t2, dev)
    c = _c128(l1, dev) if l1 is not None else None
    d = _c128(l2, dev) if l2 is not None else None
    _check(lib.lrcc_set_ground_state(h, _ptr(a), _ptr(b), _ptr(c) if c is not None else None,
                                     _ptr(d) if d is not None else None, 1), h)


def jacobian_apply(h, x1: torch.Tensor, x2: torch.Tensor, transpose=False, y1=None, y2=None, options=None,
                   stream=None):
    """y = A x (or P_sym A^T x) for a batch of vectors x1[nrhs,...], x2[nrhs,...] (CUDA complex128)."""
    if x1.device.type != "cuda" or x2.device.type != "cuda":
        raise ValueError("jacobian_apply takes CUDA tensors")
    x1 = _dense(x1)
    x2 = _dense(x2)
    nrhs = x1.shape[0]
    y1 = torch.empty_like(x1) if y1 is None else y1
    y2 = torch.empty_like(x2) if y2 is None else y2
    opt = options if options is not None else default_options()
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib.lrcc_jacobian_apply(h, int(bool(transpose)), nrhs, _ptr(x1), _ptr(x2), _ptr(y1), _ptr(y2),
                                   C.byref(opt), C.c_void_p(st.cuda_stream)), h)
    return y1, y2


def polarizability(h, comps, omegas, options=None):
    comps = np.ascontiguousarray(comps, dtype=np.int32)
    om = np.ascontiguousarray(omegas, dtype=np.float64)
    out = np.zeros((len(om), len(comps), len(comps)), dtype=np.complex128)
    info = np.zeros(2 + len(comps), dtype=np.int32)
    opt = options if options is not None else default_options()
    _check(lib.lrcc_polarizability(h, comps.ctypes.data_as(C.POINTER(C.c_int32)), len(comps),
                                   om.ctypes.data_as(C.POINTER(C.c_double)), len(om), C.byref(opt),
                                   C.c_void_p(out.ctypes.data), info.ctypes.data_as(C.POINTER(C.c_int32))), h)
    return out, info


def polarizability_forms(h, comps, omegas, options=None):
    """Symmetric and asymmetric (left-response) alpha from one solve: (sym, asym, info)."""
    comps = np.ascontiguousarray(comps, dtype=np.int32)
    om = np.ascontiguousarray(omegas, dtype=np.float64)
    sym = np.zeros((len(om), len(comps), len(comps)), dtype=np.complex128)
    asym = np.zeros_like(sym)
    info = np.zeros(2 + len(comps), dtype=np.int32)
    opt = options if options is not None else default_options()
    _check(lib.lrcc_polarizability_forms(h, comps.ctypes.data_as(C.POINTER(C.c_int32)), len(comps),
                                         om.ctypes.data_as(C.POINTER(C.c_double)), len(om), C.byref(opt),
                                         C.c_void_p(sym.ctypes.data), C.c_void_p(asym.ctypes.data),
                                         info.ctypes.data_as(C.POINTER(C.c_int32))), h)
    return sym, asym, info


def response_function(h, ops, omegas, options=None):
    """<<X;Y>>_w per cell for one-body operators ops[c][k][p][q] (Hermitian per k):
    returns (out[nomega][nops][nops], info)."""
    X = np.ascontiguousarray(ops, dtype=np.complex128)
    om = np.ascontiguousarray(omegas, dtype=np.float64)
    nops = X.shape[0]
    out = np.zeros((len(om), nops, nops), dtype=np.complex128)
    info = np.zeros(2 + nops, dtype=np.int32)
    opt = options if options is not None else default_options()
    _check(lib.lrcc_response_function(h, nops, C.c_void_p(X.ctypes.data), om.ctypes.data_as(C.POINTER(C.c_double)),
                                      len(om), C.byref(opt), C.c_void_p(out.ctypes.data),
                                      info.ctypes.data_as(C.POINTER(C.c_int32))), h)
    return out, info


def residual(h, t1: torch.Tensor, t2: torch.Tensor):
    """CCSD residual Omega(t) (paper units) of CUDA complex128 amplitudes t1, t2."""
    t1 = _dense(t1)
    t2 = _dense(t2)
    r1, r2 = torch.empty_like(t1), torch.empty_like(t2)
    _check(lib.lrcc_residual(h, _ptr(t1), _ptr(t2), _ptr(r1), _ptr(r2)), h)
    return r1, r2


def solve_ground_state(h, nk, nocc, nvir, options=None):
    """CCSD T and Lambda on the GPU; returns (t1, t2, l1, l2, energy_per_cell, info) with
    CUDA tensors in the paper's normalization.  They become the problem's ground state."""
    dev = torch.device("cuda")
    t1 = torch.empty((nk, nocc, nvir), dtype=torch.complex128, device=dev)
    t2 = torch.empty((nk, nk, nk, nocc, nocc, nvir, nvir), dtype=torch.complex128, device=dev)
    l1, l2 = torch.empty_like(t1), torch.empty_like(t2)
    e = C.c_double()
    info = np.zeros(4, dtype=np.int32)
    opt = options if options is not None else default_options()
    _check(lib.lrcc_solve_ground_state(h, C.byref(opt), _ptr(t1), _ptr(t2), _ptr(l1), _ptr(l2), 1, C.byref(e),
                                       info.ctypes.data_as(C.POINTER(C.c_int32))), h)
    return t1, t2, l1, l2, e.value, info


def excitation_energies(h, nroots, nk, nocc, nvir, options=None, vectors=False):
    """Lowest nroots LR excitation energies (complex; Jacobian eigenvalues) and, if
    vectors, the right eigenvectors (CUDA tensors, paper units).  Returns (omegas, x1, x2, info)."""
    om = np.zeros(nroots, dtype=np.complex128)
    info = np.zeros(2, dtype=np.int32)
    x1 = x2 = None
    if vectors:
        dev = torch.device("cuda")
        x1 = torch.empty((nroots, nk, nocc, nvir), dtype=torch.complex128, device=dev)
        x2 = torch.empty((nroots, nk, nk, nk, nocc, nocc, nvir, nvir), dtype=torch.complex128, device=dev)
    opt = options if options is not None else default_options()
    _check(lib.lrcc_excitation_energies(h, nroots, C.byref(opt), C.c_void_p(om.ctypes.data),
                                        _ptr(x1) if vectors else None, _ptr(x2) if vectors else None,
                                        info.ctypes.data_as(C.POINTER(C.c_int32))), h)
    return om, x1, x2, info


def batch_polarizability(problems, comps, omegas, options=None):
    """alpha for several independent problems in one call (one host thread and stream
    each); returns a list of (alpha, info) in the order of `problems`."""
    comps = np.ascontiguousarray(comps, dtype=np.int32)
    om = np.ascontiguousarray(omegas, dtype=np.float64)
    n = len(problems)
    outs = [np.zeros((len(om), len(comps), len(comps)), dtype=np.complex128) for _ in range(n)]
    infos = [np.zeros(2 + len(comps), dtype=np.int32) for _ in range(n)]
    hs = (C.c_void_p * n)(*[pr.h if isinstance(pr, Problem) else pr for pr in problems])
    ap = (C.c_void_p * n)(*[o.ctypes.data for o in outs])
    ip = (C.c_void_p * n)(*[i.ctypes.data for i in infos])
    opt = options if options is not None else default_options()
    st = lib.lrcc_batch_polarizability(hs, n, comps.ctypes.data_as(C.POINTER(C.c_int32)), len(comps),
                                       om.ctypes.data_as(C.POINTER(C.c_double)), len(om), C.byref(opt), ap, ip)
    if st != 0:
        msgs = "; ".join((lib.lrcc_last_error(h) or b"").decode() for h in hs)
        raise LrccError(st, msgs)
    return list(zip(outs, infos))


class Problem:
    """Owning wrapper around an lrcc_problem handle."""

    def __init__(self, nk, nocc, nvir, naux, kmesh=0):
        self.nk, self.nocc, self.nvir, self.naux = nk, nocc, nvir, naux
        self.h = create(nk, nocc, nvir, naux, kmesh)

    def set_integrals(self, L, eps, dip):
        set_integrals(self.h, L, eps, dip)

    def set_ground_state(self, t1, t2, l1=None, l2=None):
        set_ground_state(self.h, t1, t2, l1, l2)

    def jacobian_apply(self, x1, x2, transpose=False, **kw):
        return jacobian_apply(self.h, x1, x2, transpose, **kw)

    def polarizability(self, comps, omegas, options=None):
        return polarizability(self.h, comps, omegas, options)

    def polarizability_forms(self, comps, omegas, options=None):
        return polarizability_forms(self.h, comps, omegas, options)

    def response_function(self, ops, omegas, options=None):
        return response_function(self.h, ops, omegas, options)

    def residual(self, t1, t2):
        return residual(self.h, t1, t2)

    def solve_ground_state(self, options=None):
        return solve_ground_state(self.h, self.nk, self.nocc, self.nvir, options)

    def excitation_energies(self, nroots, options=None, vectors=False):
        return excitation_energies(self.h, nroots, self.nk, self.nocc, self.nvir, options, vectors)

    def profile(self, enable=True):
        profile(self.h, enable)

    def profile_query(self, tag=""):
        return profile_query(self.h, tag)

    def profile_report(self):
        return profile_report(self.h)

    @property
    def kernel_launches(self):
        return kernel_launches(self.h)

    def close(self):
        if self.h:
            destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


from .autograd import LRCCJacobian, jacobian  # noqa: E402
