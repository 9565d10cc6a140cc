"""CPU-side checks of the boundary: the library loads, exports every symbol
that include/sma.h declares, and rejects invalid problems on the host before
any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2105_01170_gb300 as S
from sma_inputs import generators as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "sma.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const char\*|sma_status)\s+(sma_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2105_01170_gb300 import _build
    _build.build()
    return S.lib()


def test_every_declared_symbol_is_exported(lib):
    decl = declared_symbols()
    assert len(decl) >= 10
    for name in decl:
        assert hasattr(lib, name), name
    assert set(decl) >= set(S.EXPORTED)


def test_version_and_status_strings(lib):
    assert "sm_103a" in S.sma_version()
    assert S.sma_status_string(S.SMA_ERR_STRUCT) == "invalid structure map"
    assert S.sma_status_string(99) == "unknown status"


def _create(problems, **kw):
    opt = S.sma_options(kw.get("prec", S.SMA_FP64), kw.get("decomp", S.SMA_TSVDM),
                        kw.get("mkind", S.SMA_M_DCT2), kw.get("layout", S.SMA_INPUT_DENSE),
                        None, kw.get("fixed_rank", 0), kw.get("rel_tol", 1e-6), 0, None, 0, 0,
                        kw.get("precondition", S.SMA_PRECOND_AUTO), kw.get("autotune", 0))
    structs, keep = [], []
    for ell, q, m, n, p, bm in problems:
        b = np.ascontiguousarray(np.asarray(bm, dtype=np.int32).ravel(order="F"))
        keep.append(b)
        structs.append(S.sma_problem(ell, q, m, n, p, b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     1, None, None, None, None))
    st, h = S.sma_create(structs, opt)
    return st, h


def test_rejects_map_out_of_range(lib):
    bm = G.toeplitz_map(4)
    bad = bm.copy()
    bad[0, 0] = 7          # p = 7 -> valid range [0, 6]
    st, h = _create([(4, 4, 3, 3, 7, bad)])
    assert st == S.SMA_ERR_STRUCT and not h.value


def test_rejects_uncovered_index(lib):
    bm = G.toeplitz_map(4)
    st, _ = _create([(4, 4, 3, 3, 8, bm)])        # index 7 never occurs
    assert st == S.SMA_ERR_STRUCT


def test_rejects_bad_sizes_and_options(lib):
    bm = G.toeplitz_map(3)
    assert _create([(3, 3, 0, 2, 5, bm)])[0] == S.SMA_ERR_ARG
    assert _create([(3, 3, 2, 2, 5, bm)], rel_tol=-1.0)[0] == S.SMA_ERR_ARG
    assert _create([(3, 3, 2, 3, 5, bm)], decomp=S.SMA_TUCKER_SHARED_U)[0] == S.SMA_ERR_ARG
    assert _create([(3, 3, 2, 2, 5, bm)], mkind=S.SMA_M_USER)[0] == S.SMA_ERR_ARG
    assert _create([(3, 3, 2, 2, 5, bm)], prec=7)[0] == S.SMA_ERR_ARG
    assert _create([(3, 3, 2, 2, 5, bm)], precondition=4)[0] == S.SMA_ERR_ARG
    assert _create([(3, 3, 2, 2, 5, bm)], precondition=-1)[0] == S.SMA_ERR_ARG
    assert _create([(3, 3, 2, 2, 5, bm)], autotune=2)[0] == S.SMA_ERR_ARG
    assert S.sma_create([], S.sma_options())[0] == S.SMA_ERR_ARG


def test_spd_split_is_validated_before_any_device_call(lib):
    """Section 5.2 needs T = I (x) T_0 + sum_k E_k (x) T_k: one distinct block
    on the whole diagonal and nowhere else, square blocks, p >= 2."""
    spd = dict(decomp=S.SMA_TUCKER_SPD)
    bm = G.toeplitz_map(4)                                    # lag 0 on the diagonal only
    assert S.sma_status_string(S.SMA_ERR_NOT_SPD) == "diagonal block not positive definite"
    assert _create([(4, 4, 3, 2, 7, bm)], **spd)[0] == S.SMA_ERR_ARG      # m != n
    assert _create([(4, 4, 3, 3, 4, G.block_diagonal_map(4))], **spd)[0] == S.SMA_ERR_STRUCT
    off = bm.copy()
    off[1, 0] = off[0, 0]              # T_0 also off the diagonal (lag 1 still occurs below)
    assert _create([(4, 4, 3, 3, 7, off)], **spd)[0] == S.SMA_ERR_STRUCT
    one = np.where(np.eye(3, dtype=bool), 0, -1).astype(np.int32)
    assert _create([(3, 3, 2, 2, 1, one)], **spd)[0] == S.SMA_ERR_STRUCT  # p = 1
    assert _create([(3, 3, 2, 2, 5, G.toeplitz_map(3))], decomp=6)[0] == S.SMA_ERR_ARG


def test_sketch_options_are_validated(lib):
    """The randomized block-index factor needs block-index mode, both maps, a
    fixed rank the sketch can hold (<= s^2 and <= p) and one (m, n)."""
    bm = G.toeplitz_map(4)
    om = np.zeros((3, 2))
    keep = []

    def create(probs, s=2, omega=True, psi=True, **kw):
        opt = S.sma_options(kw.get("prec", S.SMA_FP64), kw.get("decomp", S.SMA_TUCKER_BLOCKMODE),
                            S.SMA_M_DCT2, S.SMA_INPUT_DENSE, None, kw.get("fixed_rank", 2), 0.0, 0,
                            None, 0, 0, S.SMA_PRECOND_AUTO, 0, s,
                            om.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if omega else None,
                            om.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if psi else None)
        structs = []
        for ell, m, n, p, b in probs:
            b = np.ascontiguousarray(np.asarray(b, dtype=np.int32).ravel(order="F"))
            keep.append(b)
            structs.append(S.sma_problem(ell, ell, m, n, p,
                                         b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                         1, None, None, None, None))
        return S.sma_create(structs, opt)[0]

    one = [(4, 3, 3, 7, bm)]
    assert create(one, decomp=S.SMA_TSVDM) == S.SMA_ERR_ARG
    assert create(one, decomp=S.SMA_TUCKER_SHARED_U) == S.SMA_ERR_ARG
    assert create(one, fixed_rank=0) == S.SMA_ERR_ARG
    assert create(one, fixed_rank=5) == S.SMA_ERR_ARG          # s^2 = 4 < 5
    assert create(one, omega=False) == S.SMA_ERR_ARG
    assert create(one, psi=False) == S.SMA_ERR_ARG
    assert create(one, s=-1) == S.SMA_ERR_ARG
    assert create(one + [(4, 2, 3, 7, bm)]) == S.SMA_ERR_ARG  # another m


def test_cp_options_are_validated(lib):
    """CP-ALS needs a rank in 1..64 (and <= p), iterations and both initial
    factors, and one (m, n) for all problems."""
    bm = G.toeplitz_map(4)
    x0 = np.zeros((3, 70))
    keep = []

    def create(probs, r=2, iters=3, ix=True, iz=True):
        dp = ctypes.POINTER(ctypes.c_double)
        opt = S.sma_options(S.SMA_FP64, S.SMA_CP_ALS, S.SMA_M_DCT2, S.SMA_INPUT_DENSE, None, r, 0.0,
                            0, None, 0, 0, S.SMA_PRECOND_AUTO, 0, 0, None, None, iters,
                            x0.ctypes.data_as(dp) if ix else None,
                            x0.ctypes.data_as(dp) if iz else None)
        structs = []
        for ell, m, n, p, b in probs:
            b = np.ascontiguousarray(np.asarray(b, dtype=np.int32).ravel(order="F"))
            keep.append(b)
            structs.append(S.sma_problem(ell, ell, m, n, p,
                                         b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                         1, None, None, None, None))
        return S.sma_create(structs, opt)[0]

    one = [(4, 3, 3, 7, bm)]
    assert create(one, r=0) == S.SMA_ERR_ARG
    assert create(one, r=65) == S.SMA_ERR_ARG
    assert create(one, iters=0) == S.SMA_ERR_ARG
    assert create(one, ix=False) == S.SMA_ERR_ARG
    assert create(one, iz=False) == S.SMA_ERR_ARG
    assert create(one + [(4, 3, 2, 7, bm)]) == S.SMA_ERR_ARG


def test_null_handle_calls(lib):
    assert S.sma_destroy(None) == S.SMA_ERR_ARG
    assert S.sma_apply(None, 0, 0, 1, 0, 1, 1) == S.SMA_ERR_ARG
    assert S.sma_reconstruct(None, 0, 0, 1) == S.SMA_ERR_ARG


def test_binding_requires_colmajor():
    with pytest.raises(ValueError):
        S._ptr_ld(np.zeros((3, 2)))          # C-ordered numpy matrix
    assert S._ptr_ld(np.zeros((3, 2), order="F"))[1] == 3
