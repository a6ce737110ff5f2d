"""Host-side tests (no GPU) of the executor's default kernel choices, read through the plan
introspection call lrcc_plan_choice: in the mixed-precision modes every FP32 accumulation
chain stays within 8192 complex terms (longer contractions go through K splits whose
partials are summed in FP64, or through the packed kernel's chunks, each added into the
FP64 destination), and FP64 products use FP64 arithmetic only.

The chain lengths are recomputed here from each kernel's split rule and the plan's own
segment lists, not from the library's split formulas."""
import ctypes as C

import numpy as np
import pytest

from synth import CONFIGS

CHAIN_MAX = 8192  # complex terms summed in one FP32 accumulator
TC_BK = 16        # complex K per iteration of the unpacked tensor-core kernel
TILE_BK = 8       # complex K per iteration of the tiled kernel
LANES = 32        # lanes of the reduction kernel's warp sums
PK_STEP = 16      # complex K per k-step of the packed kernel (32 real K)
PK_CHUNK = 512    # k-steps the packed kernel sums in one FP32 accumulator before adding it to C

SHAPES = dict(CONFIGS)
SHAPES.update({"chain_a": dict(nk=3, nocc=4, nvir=24, naux=60),
               "chain_b": dict(nk=5, nocc=6, nvir=32, naux=100),
               "tiny": dict(nk=2, nocc=1, nvir=3, naux=5)})


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2508_01266_gb300 import _lib
    return _lib.lib


def _plan(lib, s):
    from paper_2508_01266_gb300._lib import lrcc_dims
    d = lrcc_dims(s["nk"], s["nocc"], s["nvir"], s["naux"], 0)
    h = C.c_void_p()
    assert lib.lrcc_plan_create(C.byref(d), 1 << 26, C.byref(h)) == 0
    return h


def _gemm_ops(lib, h, epi=None):
    """(gemm index, M, N, K, most segments of a batch entry) of every GEMM op of every program;
    `epi` (a dict) receives each op's epilogue kind (1: storing W-block build)."""
    seen = {}
    kif = (C.c_int32 * 3)()
    for which in range(7):
        for i in range(lib.lrcc_plan_num_ops(h, which)):
            assert lib.lrcc_plan_op(h, which, i, kif) == 0
            if kif[0] != 0 or kif[1] in seen:
                continue
            idx = kif[1]
            ints = (C.c_int32 * 16)()
            assert lib.lrcc_plan_gemm(h, idx, ints, None, None, None, None, None, None) == 0
            nb = ints[13]
            sbeg = np.zeros(nb + 1, np.int32)
            assert lib.lrcc_plan_gemm(h, idx, None, None, None, None,
                                      sbeg.ctypes.data_as(C.c_void_p), None, None) == 0
            maxseg = int(np.diff(sbeg).max()) if nb > 0 else 0
            seen[idx] = (ints[0], ints[1], ints[2], maxseg)
            if epi is not None:
                epi[idx] = ints[8]
    return seen


def _choice(lib, h, idx, prec):
    out = (C.c_int32 * 7)()
    assert lib.lrcc_plan_choice(h, idx, prec, out) == 0
    return dict(zip(("packed", "special", "tc", "f32", "tile", "nsplit", "max_seg"), list(out)))


def _fp32_chain(c, K, maxseg):
    """Longest run of complex terms one FP32 accumulator sums under choice c (None: FP64)."""
    cdiv = lambda a, b: -(-a // b)
    if c["packed"]:
        # one TMEM accumulator per chunk of at most PK_CHUNK k-steps of a tile's contraction
        return min(maxseg * cdiv(K, PK_STEP), PK_CHUNK) * PK_STEP
    if c["tc"]:
        iters = maxseg * cdiv(K, TC_BK)
        return cdiv(iters, c["nsplit"]) * TC_BK
    if not c["f32"]:
        return None
    if c["special"] == 1:
        return maxseg * K
    if c["special"] == 2:  # splits take whole segments; a lane sums every 32nd element
        return LANES * cdiv(K, LANES) * cdiv(maxseg, c["nsplit"])
    iters = maxseg * cdiv(K, TILE_BK)
    return cdiv(iters, c["nsplit"]) * TILE_BK


@pytest.mark.parametrize("shape", sorted(SHAPES))
def test_fp32_chains_capped_and_fp64_pure(lib, shape):
    h = _plan(lib, SHAPES[shape])
    try:
        epi = {}
        ops = _gemm_ops(lib, h, epi)
        assert ops
        for idx, (M, N, K, maxseg) in ops.items():
            c0 = _choice(lib, h, idx, 0)
            assert not (c0["packed"] or c0["tc"] or c0["f32"]), (shape, idx, c0)
            assert c0["nsplit"] >= 1
            for prec in (1, 2):
                c = _choice(lib, h, idx, prec)
                assert c["max_seg"] == max(maxseg, 1)
                assert c["nsplit"] >= 1
                assert not (c["packed"] and c["tc"])
                if c["packed"] and maxseg * K > CHAIN_MAX:  # chunked: only an accumulating epilogue
                    assert epi[idx] == 0, (shape, idx)
                chain = _fp32_chain(c, K, max(maxseg, 1))
                if chain is not None:
                    assert chain <= CHAIN_MAX, (shape, idx, (M, N, K, maxseg), prec, c, chain)
    finally:
        lib.lrcc_plan_destroy(h)


def test_long_contractions_leave_the_packed_kernel(lib):
    """At Nk=5, nocc=8, nvir=40 the v x v and o x o intermediates summed over three momenta
    contract up to 64000 complex terms per output into a few small tiles; none of them may run
    on the packed kernel (its chunks of one tile run one after the other), while the
    ladder-sized GEMMs (K >= 16) still do."""
    h = _plan(lib, SHAPES["c2"])
    try:
        ops = _gemm_ops(lib, h)
        long_ops = [i for i, (M, N, K, ms) in ops.items() if ms * K > CHAIN_MAX and M >= 32 and N >= 32]
        assert len(long_ops) >= 2
        for prec in (1, 2):
            for i in long_ops:
                assert not _choice(lib, h, i, prec)["packed"]
            big = [i for i, (M, N, K, ms) in ops.items()
                   if M >= 1600 and N >= 1600 and K >= 16 and ms * K <= CHAIN_MAX]
            assert big and all(_choice(lib, h, i, prec)["packed"] for i in big)
    finally:
        lib.lrcc_plan_destroy(h)


def test_long_ladder_chains_take_the_packed_kernel_in_chunks(lib):
    """At Nk=7, nocc=8, nvir=48 the ladder contracts 7 x 48^2 = 16128 complex terms per output;
    its GEMMs stay on the packed kernel (two chunks of at most 8192 terms per tile), which
    the tile counts fill."""
    h = _plan(lib, SHAPES["c3"])
    try:
        ops = _gemm_ops(lib, h)
        ladder = [i for i, (M, N, K, ms) in ops.items() if (M, N, K) == (448, 2304, 2304)]
        assert ladder
        for prec in (1, 2):
            for i in ladder:
                M, N, K, ms = ops[i]
                c = _choice(lib, h, i, prec)
                assert c["packed"] == 1, (i, c)
                if ms * K > CHAIN_MAX:
                    assert _fp32_chain(c, K, ms) <= CHAIN_MAX
    finally:
        lib.lrcc_plan_destroy(h)


def test_plan_choice_rejects_bad_arguments(lib):
    h = _plan(lib, SHAPES["tiny"])
    try:
        out = (C.c_int32 * 7)()
        assert lib.lrcc_plan_choice(h, -1, 0, out) != 0
        assert lib.lrcc_plan_choice(h, 1 << 20, 0, out) != 0
        assert lib.lrcc_plan_choice(h, 0, 3, out) != 0
        assert lib.lrcc_plan_choice(h, 0, 0, None) != 0
        assert lib.lrcc_plan_choice(None, 0, 0, out) != 0
    finally:
        lib.lrcc_plan_destroy(h)


def test_small_shapes_take_fp32_kernels_in_mixed_precision(lib):
    """At nvir = 40 the mixed modes run the Fock-like 8 x 1600 x 8 blocks on the FP32
    short-contraction kernel, and the 40 x 40 blocks that the packed path does not take
    (K < 16, or contractions over the FP32 chain cap) on the FP32 tiled kernel with the
    48 x 48 tile; FP64 products keep FP64 kernels for both."""
    h = _plan(lib, SHAPES["c2"])
    try:
        ops = _gemm_ops(lib, h)
        skinny = [i for i, (M, N, K, ms) in ops.items() if (M, N, K) == (8, 1600, 8) and ms == 1]
        small = [i for i, (M, N, K, ms) in ops.items()
                 if (M, N) == (40, 40) and K <= 40 and (K < 16 or ms * K > CHAIN_MAX)]
        assert skinny and small
        for prec in (1, 2):
            for i in skinny:
                c = _choice(lib, h, i, prec)
                assert (c["special"], c["f32"]) == (1, 1), c
            for i in small:
                c = _choice(lib, h, i, prec)
                assert c["f32"] == 1 and not (c["tc"] or c["packed"] or c["special"]), c
                assert c["tile"] == 10, c  # the 48 x 48 tile
        for i in skinny + small:
            assert _choice(lib, h, i, 0)["f32"] == 0
    finally:
        lib.lrcc_plan_destroy(h)
