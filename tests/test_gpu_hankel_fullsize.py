"""The block-Hankel workload at full size (64 x 64 blocks of 32 x 32 Markov
parameters of a 40-state system, p = 127): rows-and-columns Tucker block
low rank at ranks 5, 10 and 20, the dense approximation and the matvec on
256 right-hand sides, against the FP64 oracle; host-buffer inputs for the
CP and two-level paths."""
import numpy as np
import pytest

from oracle import sma_oracle as O
from sma_inputs import generators as G

from _util import input_matrix, np_dtype, oracle_tensor, rel, to_dev, tol_for, torch_dtype

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


@pytest.fixture(scope="module")
def hankel():
    return G.lti_hankel()


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("r", [5, 10, 20])
def test_hankel_rowcol_full_size(prec, r, hankel):
    pr = hankel
    A = input_matrix(pr, prec)
    h = S.Handle([pr], prec=prec, decomp=S.SMA_TUCKER_ROWCOL, fixed_rank=r)
    res = h.compress([to_dev(A)])[0]
    assert res["device_status"] == 0 and res["ranks"][:2] == [r, r]
    X = oracle_tensor(A, pr)
    t = O.tucker2_rows_cols(X, r, r)
    N = pr.ell * pr.m
    Ah = torch.empty(N, N, dtype=torch_dtype(prec), device="cuda").t()
    h.reconstruct(0, Ah)
    Ao = O.M_E(t.tensor_approx(), pr.block_map)
    assert rel(Ah.cpu().numpy(), Ao) < tol_for(prec)
    x = G.random_rhs(N, 256, 3).astype(np_dtype(prec))
    Y = torch.empty(256, N, dtype=torch_dtype(prec), device="cuda").t()
    h.apply(0, to_dev(x), Y)
    assert rel(Y.cpu().numpy(), Ao @ x.astype(np.float64)) < tol_for(prec)
    assert abs(res["tensor_err"] - t.err) <= 1e-6 * t.err + (1e-12 if prec == S.SMA_FP64 else 1e-5) * np.linalg.norm(X)
    h.close()


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_host_inputs_cp_and_two_level(prec):
    """Host (pageable) inputs give the same results as device inputs."""
    pr, f = G.planted_cp_toeplitz(ell=6, m=9, n=7, r=2, noise=1e-3)
    X0, Z0 = G.cp_initial_factors(pr.m, pr.n, 2)
    A = np.asfortranarray(pr.dense().astype(np_dtype(prec)))
    out = []
    for src in (A, to_dev(A)):
        h = S.Handle([pr], prec=prec, decomp=S.SMA_CP_ALS, fixed_rank=2, cp_init=(X0, Z0), cp_iters=5)
        out.append(h.compress([src])[0]["tensor_err"])
        h.close()
    assert out[0] == out[1]
    map1, map2 = G.toeplitz_map(3), G.block_diagonal_map(4)
    pr2 = G.two_level_problem(map1, map2, 5, 4)
    mp = S.MultilevelProblem([map1, map2], [5, 4], 5, 4)
    A2 = np.asfortranarray(pr2.dense().astype(np_dtype(prec)))
    out = []
    for src in (A2, to_dev(A2)):
        h = S.Handle([mp], prec=prec, decomp=S.SMA_HOSVD_MULTILEVEL, fixed_rank=2)
        out.append(h.compress([src])[0]["tensor_err"])
        h.close()
    assert out[0] == out[1]
