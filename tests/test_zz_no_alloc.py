"""The allocation-free Jacobian product, called through the C-ABI.

lrcc_jacobian_apply_noalloc serves callers that cannot let a library allocate device
memory while they run (an application that owns the allocator, a latency-critical
loop).  It must give the same products as lrcc_jacobian_apply, call after call,
while reusing one static device array.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import make_problem, random_amplitudes

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def lr():
    import __graft_entry__ as g
    g.build()
    import paper_2508_01266_gb300 as m
    f = m._lib.lib.lrcc_jacobian_apply_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return m


def _problem(lr, nk, o, v, Q, seed):
    p = make_problem(nk, o, v, Q, seed=seed, sigma_l=0.1)
    t1, t2 = random_amplitudes(nk, o, v, seed=seed + 1, scale1=0.02, scale2=0.02)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2 * nk)
    return prob


def _noalloc(lr, prob, transpose, X1, X2):
    y1 = torch.full_like(X1[0], complex(float("nan"), 0.0))
    y2 = torch.full_like(X2[0], complex(float("nan"), 0.0))
    st = torch.cuda.current_stream()
    status = lr._lib.lib.lrcc_jacobian_apply_noalloc(prob.h, transpose, X1.data_ptr(), X2.data_ptr(),
                                                     y1.data_ptr(), y2.data_ptr(), C.c_void_p(st.cuda_stream))
    assert status == 0, lr.last_error(prob.h)
    torch.cuda.synchronize()
    return y1, y2


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("nk,o,v,Q", [(3, 2, 4, 6), (3, 4, 16, 48)])
def test_noalloc_matches_allocating_entry_point(lr, nk, o, v, Q):
    prob = _problem(lr, nk, o, v, Q, seed=21)
    dev = torch.device("cuda")
    for transpose in (0, 1):
        for call in range(2):  # two calls in a row reuse the static array
            x1, x2 = random_amplitudes(nk, o, v, seed=100 + 10 * transpose + call, scale1=1.0, scale2=1.0)
            X1 = torch.as_tensor(x1, device=dev)[None].contiguous()
            X2 = torch.as_tensor(x2 * nk, device=dev)[None].contiguous()
            r1, r2 = prob.jacobian_apply(X1, X2, transpose=bool(transpose))
            y1, y2 = _noalloc(lr, prob, transpose, X1, X2)
            assert _rel(y1, r1[0]) < TOL and _rel(y2, r2[0]) < TOL
    prob.close()


def test_noalloc_first_on_fresh_problem(lr):
    """The allocation-free call comes first on a freshly created problem (no allocating product
    has run on it, so no lazily created buffer exists), in both directions, and only then is
    it compared with the allocating entry point."""
    nk, o, v, Q = 3, 2, 4, 6
    dev = torch.device("cuda")
    for transpose in (0, 1):
        prob = _problem(lr, nk, o, v, Q, seed=41 + transpose)
        x1, x2 = random_amplitudes(nk, o, v, seed=200 + transpose, scale1=1.0, scale2=1.0)
        X1 = torch.as_tensor(x1, device=dev)[None].contiguous()
        X2 = torch.as_tensor(x2 * nk, device=dev)[None].contiguous()
        y1, y2 = _noalloc(lr, prob, transpose, X1, X2)
        r1, r2 = prob.jacobian_apply(X1, X2, transpose=bool(transpose))
        assert _rel(y1, r1[0]) < TOL and _rel(y2, r2[0]) < TOL
        prob.close()


def test_noalloc_rejects_problems_beyond_its_limit(lr):
    prob = _problem(lr, 4, 4, 24, 32, seed=31)
    dev = torch.device("cuda")
    X1 = torch.zeros((1, 4, 4, 24), dtype=torch.complex128, device=dev)
    X2 = torch.zeros((1, 4, 4, 4, 4, 4, 24, 24), dtype=torch.complex128, device=dev)
    y1, y2 = torch.empty_like(X1[0]), torch.empty_like(X2[0])
    status = lr._lib.lib.lrcc_jacobian_apply_noalloc(prob.h, 0, X1.data_ptr(), X2.data_ptr(), y1.data_ptr(),
                                                     y2.data_ptr(), None)
    assert status == 6
    assert "static limit" in lr.last_error(prob.h)
    prob.close()
