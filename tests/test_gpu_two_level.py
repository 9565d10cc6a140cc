"""Section 7 with two levels and m x n blocks on the GPU: the fourth-order
tensor's truncated HOSVD over four modes and the Kronecker sum over the two
level structures, against the FP64 oracle (hosvd4, two_level_kron_terms):
ranks, error (the multilevel Lemma), the dense approximation and the matvec,
for both input layouts and both precisions; a planted multilinear rank is
recovered."""
import numpy as np
import pytest

from oracle import sma_oracle as O
from sma_inputs import generators as G

from _util import np_dtype, rel, to_dev, torch_dtype

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


def run(map1, map2, pr, prec, layout, **kw):
    p1, p2 = int(map1.max()) + 1, int(map2.max()) + 1
    mp = S.MultilevelProblem([map1, map2], [p1, p2], pr.m, pr.n)
    if layout == S.SMA_INPUT_DENSE:
        A = pr.dense()
    else:
        A = np.concatenate(list(pr.blocks), axis=1)
    A = np.asfortranarray(A.astype(np_dtype(prec)))
    h = S.Handle([mp], prec=prec, decomp=S.SMA_HOSVD_MULTILEVEL, layout=layout, **kw)
    res = h.compress([to_dev(A)])[0]
    Ad = pr.dense().astype(np_dtype(prec)).astype(np.float64)
    X = O.two_level_tensor(Ad, map1, map2, pr.m, pr.n)
    if prec == S.SMA_MIXED:
        X = X.astype(np.float32).astype(np.float64)     # the tensor as the path stores it
    return h, res, X


def check(h, res, X, ho, map1, map2, pr, prec):
    assert res["device_status"] == 0
    assert tuple(res["ranks"]) == ho.ranks
    assert res["n_kron_terms"] == ho.ranks[2] * ho.ranks[3]
    tol = 1e-10 if prec == S.SMA_FP64 else 1e-5
    floor = (1e-12 if prec == S.SMA_FP64 else 1e-5) * np.linalg.norm(X)
    assert abs(res["tensor_err"] - ho.err) <= 1e-6 * ho.err + floor
    rows = pr.block_map.shape[0] * pr.m
    cols = pr.block_map.shape[1] * pr.n
    Ah = torch.empty(cols, rows, dtype=torch_dtype(prec), device="cuda").t()
    h.reconstruct(0, Ah)
    Ao = O.two_level_matrix(ho.tensor_approx(), map1, map2)
    assert rel(Ah.cpu().numpy(), Ao) < tol
    terms = O.two_level_kron_terms(ho, map1, map2)
    x = G.random_rhs(cols, 3, 6).astype(np_dtype(prec))
    Y = torch.empty(3, rows, dtype=torch_dtype(prec), device="cuda").t()
    h.apply(0, to_dev(x), Y)
    assert rel(Y.cpu().numpy(), O.apply_kron(terms, x.astype(np.float64))) < tol


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("layout", [S.SMA_INPUT_DENSE, S.SMA_INPUT_BLOCKS], ids=["dense", "blocks"])
def test_running_example_fixed_rank(prec, layout):
    """4 x 4 block-pentadiagonal symmetric Toeplitz of 5 x 5 block-diagonal
    blocks of 4 x 3 (15 distinct blocks), rank 2 in every mode."""
    map1 = G.symmetric_banded_toeplitz_map(4, 2)
    map2 = G.block_diagonal_map(5)
    pr = G.two_level_problem(map1, map2, 4, 3)
    h, res, X = run(map1, map2, pr, prec, layout, fixed_rank=2)
    ho = O.hosvd4(X, ranks=(2, 2, 2, 2))
    check(h, res, X, ho, map1, map2, pr, prec)
    h.close()


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_planted_multilinear_rank_recovered(prec):
    """Block Toeplitz (8 blocks, p1 = 15) of symmetric banded Toeplitz (6
    blocks, half-band 2, p2 = 3) blocks of 16 x 12 whose tensor has
    multilinear rank (3, 2, 4, 2) plus 1e-9 noise: tolerance 1e-6 finds it."""
    map1 = G.toeplitz_map(8)
    map2 = G.symmetric_banded_toeplitz_map(6, 2)
    pr = G.two_level_problem(map1, map2, 16, 12, ranks=(3, 2, 4, 2), noise=1e-9)
    tol = 1e-6 if prec == S.SMA_FP64 else 1e-4
    h, res, X = run(map1, map2, pr, prec, S.SMA_INPUT_BLOCKS, rel_tol=tol)
    ho = O.hosvd4(X, rel_tol=tol)
    assert ho.ranks == (3, 2, 4, 2)
    check(h, res, X, ho, map1, map2, pr, prec)
    assert res["rel_err"] < tol
    h.close()
