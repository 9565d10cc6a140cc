"""Seeded random structures against the FP64 oracle: arbitrary block maps
(random distinct-block assignment with empty positions, every index used),
non-square and degenerate block sizes (m or n = 1), fixed per-slice rank
t-SVDM and fixed-rank block-index Tucker-1; the dense approximation and the
Kronecker-sum matvec must match."""
import numpy as np
import pytest

from oracle import sma_oracle as O
from sma_inputs import generators as G

from _util import apply, input_matrix, oracle_tensor, reconstruct, rel, to_dev, tol_for, np_dtype

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


def random_problem(seed):
    g = np.random.default_rng(1000 + seed)
    ell, q = int(g.integers(1, 7)), int(g.integers(1, 7))
    m, n = int(g.integers(1, 41)), int(g.integers(1, 41))
    cells = ell * q
    p = int(g.integers(1, cells + 1))
    bm = -np.ones(cells, dtype=np.int32)
    pos = g.permutation(cells)
    bm[pos[:p]] = np.arange(p)                          # every index at least once
    extra = pos[p:]
    fill = extra[g.random(len(extra)) < 0.6]            # some repeats, the rest empty
    bm[fill] = g.integers(0, p, len(fill))
    bm = bm.reshape((ell, q), order="F")
    return G.Problem(f"random_{seed}", g.standard_normal((p, m, n)), bm)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("seed", range(8))
def test_random_map_tsvdm_fixed_rank(prec, seed):
    pr = random_problem(seed)
    r = max(1, min(pr.m, pr.n) // 2)
    A = input_matrix(pr, prec)
    h = S.Handle([pr], prec=prec, fixed_rank=r)
    res = h.compress([to_dev(A)])[0]
    assert res["device_status"] == 0
    X = oracle_tensor(A, pr)
    ora = O.tsvdm(X, O.dct2_matrix(pr.p), fixed_rank=r)
    assert np.array_equal(h.ranks(0), ora.ranks)
    Ao = O.M_E(ora.tensor_approx(), pr.block_map)
    assert rel(reconstruct(h, pr, prec), Ao) < tol_for(prec)
    x = G.random_rhs(pr.q * pr.n, 3, seed).astype(np_dtype(prec)).astype(np.float64)
    assert rel(apply(h, pr, x, prec), Ao @ x) < tol_for(prec)
    h.close()


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("seed", range(8, 14))
def test_random_map_blockmode_fixed_rank(prec, seed):
    pr = random_problem(seed)
    r = max(1, pr.p // 2)
    A = input_matrix(pr, prec)
    h = S.Handle([pr], prec=prec, decomp=S.SMA_TUCKER_BLOCKMODE, fixed_rank=r)
    res = h.compress([to_dev(A)])[0]
    assert res["device_status"] == 0
    X = oracle_tensor(A, pr)
    if prec == S.SMA_MIXED:
        X = X.astype(np.float32).astype(np.float64)
    t = O.tucker1_blockmode(X, rank=r)
    Ao = O.M_E(t.tensor_approx(), pr.block_map)
    assert rel(reconstruct(h, pr, prec), Ao) < tol_for(prec)
    x = G.random_rhs(pr.q * pr.n, 3, seed).astype(np_dtype(prec)).astype(np.float64)
    assert rel(apply(h, pr, x, prec), Ao @ x) < tol_for(prec)
    h.close()
