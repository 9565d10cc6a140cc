"""The global truncation rule (step 4; Lemma 1) over many slices.

The slices are diagonal matrices with chosen singular values (powers of two,
so that fp32 and fp64 hold them exactly and exact ties across slices are
common), placed on the diagonal of a block-diagonal matrix and compressed
with the identity transform, so the slice SVDs return the chosen values and
the ranks depend on the truncation rule alone.  Slice counts cover the three
forms of the device truncation: one warp (at most 32 slices), one warp with
fp32 keys in shared memory (33 to 256), and the block form (more).  The ranks
must equal the oracle's exactly, ties at the budget boundary included
(dropped from the highest slice index first).
"""
import numpy as np
import pytest

from oracle import sma_oracle as O
from sma_inputs import generators as G

from _util import input_matrix, oracle_tensor, to_dev

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


def diagonal_slices(p, m, case, seed):
    g = np.random.default_rng(seed)
    if case == "ties":      # few distinct values: exact ties across slices
        e = g.integers(0, 6, size=(p, m))
    else:                   # many distinct values over twenty octaves
        e = g.integers(0, 40, size=(p, m)) / 2.0
        e = np.floor(e)
    d = -np.sort(-(2.0 ** (-e)), axis=1)
    d[g.random(p) < 0.1, :] = 0.0           # some all-zero slices
    return np.stack([np.diag(d[k]) for k in range(p)])


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("p", [20, 33, 100, 127, 256, 300])
@pytest.mark.parametrize("case", ["ties", "spread"])
@pytest.mark.parametrize("tol", [0.05, 0.3])
def test_global_truncation_ranks_equal_oracle(prec, p, case, tol):
    m = 8
    blocks = diagonal_slices(p, m, case, seed=p + (7 if case == "ties" else 0))
    pr = G.Problem("diagonal_slices", blocks, G.block_diagonal_map(p))
    A = input_matrix(pr, prec)
    h = S.Handle([pr], prec=prec, rel_tol=tol, mkind=S.SMA_M_IDENTITY)
    res = h.compress([to_dev(A)])[0]
    assert res["device_status"] == 0
    ora = O.tsvdm(oracle_tensor(A, pr), np.eye(p), rel_tol=tol)
    assert np.array_equal(h.ranks(0), np.asarray(ora.ranks))
    assert res["total_rank"] == int(np.sum(ora.ranks))
    # the reported error is the discarded energy (Lemma 1), exact here
    assert abs(res["tensor_err"] - ora.err) <= 1e-12 * max(ora.normX, 1.0)
