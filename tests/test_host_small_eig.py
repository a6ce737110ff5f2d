"""Host-side small complex eigensolver of the Davidson iteration (no GPU), against
numpy's LAPACK eigenvalues and the eigen-equation itself."""
import ctypes as C

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2508_01266_gb300 import _lib
    return _lib.lib


@pytest.mark.parametrize("n,seed,kind", [(1, 0, "gen"), (2, 1, "gen"), (5, 2, "gen"), (17, 3, "gen"),
                                          (40, 4, "gen"), (24, 5, "herm"), (30, 6, "nearsym"), (12, 7, "triangular")])
def test_small_eig(lib, n, seed, kind):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    if kind == "herm":
        A = A + A.conj().T
    elif kind == "nearsym":  # a Davidson-like subspace matrix: dominant real diagonal
        A = np.diag(np.sort(rng.uniform(0.2, 3.0, n))) + 1e-2 * A
    elif kind == "triangular":
        A = np.triu(A)
    A = np.ascontiguousarray(A, dtype=np.complex128)
    w = np.zeros(n, np.complex128)
    V = np.zeros((n, n), np.complex128)
    st = lib.lrcc_small_eig(n, A.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p),
                            V.ctypes.data_as(C.c_void_p))
    assert st == 0
    ref = np.linalg.eigvals(A)
    for x in ref:
        assert np.abs(w - x).min() < 1e-9 * max(1.0, np.abs(ref).max())
    res = A @ V - V * w[None, :]
    assert np.abs(res).max() < 1e-9 * max(1.0, np.abs(A).max())
    assert np.allclose(np.linalg.norm(V, axis=0), 1.0)
