"""Degenerate and ragged cases of the Section 5.2, 6.3 (sketch), 2.3 (CP) and
Section 7 (two levels) paths against the FP64 oracle: one remaining block
after the SPD split, a single distinct block for CP, a one-block level,
a one-column sketch, odd block sizes."""
import numpy as np
import pytest

from oracle import sma_oracle as O
from sma_inputs import generators as G

from _util import gpu_tensor, np_dtype, oracle_tensor, rel, to_dev, torch_dtype

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
S = pytest.importorskip("paper_2105_01170_gb300")

PRECS = [S.SMA_FP64, S.SMA_MIXED]
PNAME = {S.SMA_FP64: "fp64", S.SMA_MIXED: "mixed"}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_01170_gb300 import _build
    _build.build()


def tol(prec):
    return 1e-10 if prec == S.SMA_FP64 else 1e-5


def stored(X, prec):
    return X if prec == S.SMA_FP64 else X.astype(np.float32).astype(np.float64)


def dense_of(h, rows, cols, prec):
    Ah = torch.empty(cols, rows, dtype=torch_dtype(prec), device="cuda").t()
    h.reconstruct(0, Ah)
    return Ah.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_spd_with_one_remaining_block(prec):
    """Symmetric block-tridiagonal Toeplitz (T_0 on the diagonal, one
    symmetric T_1 on both off-diagonals, p = 2): after the split the tensor
    has a single slice."""
    g = np.random.default_rng(31)
    m, ell = 7, 5
    B = g.standard_normal((m, m))
    T0 = B @ B.T + 4 * m * np.eye(m)
    C = g.standard_normal((m, m))
    T1 = C + C.T
    pr = G.Problem("spd_p2", np.stack([T0, T1]), G.symmetric_banded_toeplitz_map(ell, 1))
    A = pr.dense().astype(np_dtype(prec))
    h = S.Handle([pr], prec=prec, decomp=S.SMA_TUCKER_SPD, fixed_rank=3)
    res = h.compress([to_dev(np.asfortranarray(A))])[0]
    assert res["device_status"] == 0
    s = O.spd_preserving(A.astype(np.float64), pr.block_map, pr.p, m, rank=3)
    assert s.X.shape == (m, m, 1)
    Th = dense_of(h, ell * m, ell * m, prec)
    assert rel(Th, s.dense()) < tol(prec)
    assert np.linalg.eigvalsh((Th + Th.T) / 2).min() > 0
    h.close()


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_cp_single_block_rank_one_odd_sizes(prec):
    """One distinct block (p = 1, r = 1) of odd size 7 x 5: rank-1 CP of an
    m x n x 1 tensor is the leading singular pair's outer product reached by
    the ALS iterate."""
    g = np.random.default_rng(32)
    pr = G.Problem("single", g.standard_normal((1, 7, 5)), np.zeros((1, 1), dtype=np.int32))
    X0, Z0 = g.standard_normal((7, 1)), g.standard_normal((5, 1))
    A = pr.dense().astype(np_dtype(prec))
    h = S.Handle([pr], prec=prec, decomp=S.SMA_CP_ALS, fixed_rank=1, cp_init=(X0, Z0), cp_iters=6)
    res = h.compress([to_dev(np.asfortranarray(A))])[0]
    X = stored(oracle_tensor(A.astype(np.float64), pr), prec)
    c = O.cp_als(X, stored(X0, prec), stored(Z0, prec), 6)
    T = gpu_tensor(h, S.EXPORT_T, X.shape, prec)
    assert rel(T, c.tensor_approx()) < tol(prec)
    assert abs(res["tensor_err"] - c.err) <= tol(prec) * np.linalg.norm(X)
    h.close()


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_two_level_with_one_block_level_and_odd_blocks(prec):
    """Level 2 holds one block everywhere (p2 = 1); blocks 5 x 3."""
    map1 = G.toeplitz_map(4)
    map2 = np.zeros((2, 2), dtype=np.int32)
    pr = G.two_level_problem(map1, map2, 5, 3)
    mp = S.MultilevelProblem([map1, map2], [7, 1], 5, 3)
    A = np.asfortranarray(pr.dense().astype(np_dtype(prec)))
    h = S.Handle([mp], prec=prec, decomp=S.SMA_HOSVD_MULTILEVEL, fixed_rank=2)
    res = h.compress([to_dev(A)])[0]
    X = stored(O.two_level_tensor(A.astype(np.float64), map1, map2, 5, 3), prec)
    ho = O.hosvd4(X, ranks=(2, 2, 2, 1))
    assert tuple(res["ranks"]) == ho.ranks
    Ah = dense_of(h, 8 * 5, 8 * 3, prec)
    assert rel(Ah, O.two_level_matrix(ho.tensor_approx(), map1, map2)) < tol(prec)
    h.close()


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_one_column_sketch(prec):
    """s = 1: the sketch of each block is a scalar and V is its rank-1 factor."""
    pr = G.planted_kron_toeplitz(ell=9, m=5, terms=1, seed_index=2)
    Om, Ps = G.gaussian_sketch(pr.m, pr.n, 1)
    A = np.asfortranarray(pr.dense().astype(np_dtype(prec)))
    h = S.Handle([pr], prec=prec, decomp=S.SMA_TUCKER_BLOCKMODE, fixed_rank=1, sketch=(Om, Ps))
    res = h.compress([to_dev(A)])[0]
    X = stored(oracle_tensor(A.astype(np.float64), pr), prec)
    t = O.tucker1_blockmode_sketch(X, stored(Om, prec), stored(Ps, prec), 1)
    assert res["ranks"][0] == 1
    assert abs(res["tensor_err"] - t.err) <= 1e-6 * t.err + tol(prec) * np.linalg.norm(X)
    V = gpu_tensor(h, S.EXPORT_FACTOR, (pr.p, pr.p), prec)[:, :1]
    assert np.linalg.norm(V @ V.T - t.V @ t.V.T, 2) < (1e-9 if prec == S.SMA_FP64 else 1e-5)
    h.close()


def test_create_rejects_slice_without_jacobi_plan():
    """A 30000 x 4 block: two of its stacked Jacobi columns do not fit in
    shared memory, so sma_create reports SMA_ERR_UNSUPPORTED (host-side plan
    check; no kernel runs)."""
    pr = G.Problem("tall", np.zeros((1, 30000, 4)), G.block_diagonal_map(1))
    with pytest.raises(S.SmaError) as e:
        S.Handle([pr], prec=S.SMA_MIXED, rel_tol=1e-6)
    assert e.value.status == S.SMA_ERR_UNSUPPORTED
