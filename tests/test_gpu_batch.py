"""Many problems in one handle (uneven block-tridiagonal matrices of four
block sizes: the slice SVDs of all problems run in one launch per slice size)
and CUDA-graph replay of sma_compress, against the FP64 oracle."""
import numpy as np
import pytest

from oracle import sma_oracle as O
from sma_inputs import generators as G

from _util import (apply, gpu_tensor, input_matrix, np_dtype, oracle_at_gpu_ranks, reconstruct,
                   rel, to_dev, tol_for)

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


def batch(count=8):
    return G.block_tridiag_batch(count=count, ell_range=(4, 12), m_choices=(8, 16, 32, 64))


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("tune", [False, True], ids=["default_plan", "autotuned"])
def test_batched_tsvdm_matches_oracle(prec, tune):
    prs = batch()
    assert len({pr.m for pr in prs}) >= 3
    tol = 1e-3
    As = [input_matrix(pr, prec) for pr in prs]
    h = S.Handle(prs, prec=prec, rel_tol=tol, autotune=tune)
    res = h.compress([to_dev(A) for A in As])
    for i, (pr, A) in enumerate(zip(prs, As)):
        X = O.T_E(np.asarray(A, dtype=np.float64), pr.block_map, pr.p, pr.m, pr.n)
        M = O.dct2_matrix(pr.p)
        ora = O.tsvdm(X, M, rel_tol=tol)
        ranks = h.ranks(i)
        cmp = oracle_at_gpu_ranks(ranks, ora, X, M, tol, prec, f"batch problem {i} tune {tune}")
        if prec == S.SMA_FP64:
            assert abs(res[i]["tensor_err"] - ora.err) <= 1e-9 * ora.err
        assert res[i]["device_status"] == 0
        sig = gpu_tensor(h, S.EXPORT_SIGMA, (pr.m, pr.p), prec, i=i)
        smax = max(float(np.max(s)) for s in ora.sigma)
        assert max(np.max(np.abs(sig[:, k] - ora.sigma[k])) for k in range(pr.p)) <= \
            (1e-12 if prec == S.SMA_FP64 else 2e-5) * smax
        x = G.random_rhs(pr.q * pr.n, 2, i).astype(np_dtype(prec)).astype(np.float64)
        y = apply(h, pr, x, prec, i=i)
        Ah = reconstruct(h, pr, prec, i=i)
        e_apply = rel(y, Ah @ x)                  # the factored matvec itself
        assert e_apply < tol_for(prec), e_apply
        Ao = O.M_E(cmp.tensor_approx(), pr.block_map)
        e_op = rel(Ah, Ao)                        # the compressed operator
        e_tot = rel(y, O.apply_kron(O.tsvdm_kron_terms(cmp, pr.block_map), x))
        print(f"problem {i} m={pr.m}: apply {e_apply:.2e} operator {e_op:.2e} total {e_tot:.2e}")
        assert e_op < tol_for(prec) and e_tot < tol_for(prec), (e_apply, e_op, e_tot)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_batched_kronecker_rank(prec):
    prs = batch(6)
    tol = 1e-3
    As = [input_matrix(pr, prec) for pr in prs]
    h = S.Handle(prs, prec=prec, decomp=S.SMA_TUCKER_BLOCKMODE, rel_tol=tol)
    res = h.compress([to_dev(A) for A in As])
    for i, pr in enumerate(prs):
        X = O.T_E(np.asarray(As[i], dtype=np.float64), pr.block_map, pr.p, pr.m, pr.n)
        t = O.tucker1_blockmode(X, rel_tol=tol)
        assert res[i]["ranks"][0] == t.rank == pr.extra["K"]


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_graph_replay_is_identical(prec):
    prs = batch(5)
    st = torch.cuda.Stream()
    As = [to_dev(input_matrix(pr, prec)) for pr in prs]
    h = S.Handle(prs, prec=prec, rel_tol=1e-3, stream=st.cuda_stream, graph=True, profile=True)
    with torch.cuda.stream(st):
        outs = []
        for _ in range(4):              # run, capture, replay, replay
            res = h.compress(As)
            T = [gpu_tensor(h, S.EXPORT_X, None, prec, i=i) for i in range(len(prs))]
            sig = [gpu_tensor(h, S.EXPORT_SIGMA, None, prec, i=i) for i in range(len(prs))]
            outs.append((res, T, sig))
    for res, T, sig in outs[1:]:
        for i in range(len(prs)):
            assert res[i]["total_rank"] == outs[0][0][i]["total_rank"]
            assert res[i]["tensor_err"] == outs[0][0][i]["tensor_err"]
            assert np.array_equal(T[i], outs[0][1][i])
            assert np.array_equal(sig[i], outs[0][2][i])
    assert h.profile()["launches"] > 0
