"""Parity at the benchmark's full size (space-time covariance, 16384^2,
tensor 256 x 256 x 127, tolerance 1e-6), in the launch configuration the
benchmark times: every singular value and rank, the error report, and the
Kronecker-sum matvec on sampled right-hand sides, against the FP64 oracle."""
import numpy as np
import pytest

from oracle import sma_oracle as O
from sma_inputs import generators as G

from _util import gpu_tensor, oracle_at_gpu_ranks, rel, to_dev, tol_for

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
def workload():
    pr = G.spacetime_covariance()
    Ad = pr.dense()
    return pr, Ad


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_spacetime_full_size(prec, workload):
    pr, Ad = workload
    A = Ad if prec == S.SMA_FP64 else Ad.astype(np.float32)
    dA = to_dev(A)
    st = torch.cuda.Stream()
    h = S.Handle([pr], prec=prec, rel_tol=1e-6, stream=st.cuda_stream)
    with torch.cuda.stream(st):
        res = h.compress([dA])[0]
    del dA
    X = O.T_E(np.asarray(A, dtype=np.float64), pr.block_map, pr.p, pr.m, pr.n)
    M = O.dct2_matrix(pr.p)
    ora = O.tsvdm(X, M, rel_tol=1e-6)
    assert res["device_status"] == 0
    sig = gpu_tensor(h, S.EXPORT_SIGMA, (pr.m, pr.p), prec)
    smax = max(float(np.max(s)) for s in ora.sigma)
    diff = max(float(np.max(np.abs(sig[:, k] - ora.sigma[k]))) for k in range(pr.p))
    assert diff <= (1e-12 if prec == S.SMA_FP64 else 2e-5) * smax
    ranks = h.ranks(0)
    cmp = oracle_at_gpu_ranks(ranks, ora, X, M, 1e-6, prec, "spacetime full size")
    if prec == S.SMA_FP64:
        assert abs(res["tensor_err"] - ora.err) <= 1e-9 * ora.err
    assert res["rel_err"] <= 1e-6
    # the whole approximation tensor T (filled by sma_reconstruct), element
    # by element
    dt = torch.float64 if prec == S.SMA_FP64 else torch.float32
    rows = pr.ell * pr.m
    Ah = torch.empty(rows, rows, dtype=dt, device="cuda").t()
    with torch.cuda.stream(st):
        h.reconstruct(0, Ah)
    st.synchronize()
    del Ah
    T = gpu_tensor(h, S.EXPORT_T, (pr.m, pr.n, pr.p), prec)
    e_T = rel(T, cmp.tensor_approx())
    print(f"full size {'fp64' if prec == S.SMA_FP64 else 'mixed'}: T rel err {e_T:.2e}")
    assert e_T < tol_for(prec), e_T
    del T
    # sampled matvec: two of the benchmark's right-hand sides
    x = G.random_rhs(pr.q * pr.n, 2, 1)
    xin = x if prec == S.SMA_FP64 else x.astype(np.float32)
    X_d = to_dev(xin)
    dt = torch.float64 if prec == S.SMA_FP64 else torch.float32
    Y_d = torch.empty(2, pr.ell * pr.m, dtype=dt, device="cuda").t()
    with torch.cuda.stream(st):
        h.apply(0, X_d, Y_d)
    st.synchronize()
    y = Y_d.cpu().numpy().astype(np.float64)
    yo = O.apply_kron(O.tsvdm_kron_terms(cmp, pr.block_map), np.asarray(xin, dtype=np.float64))
    assert rel(y, yo) < tol_for(prec), rel(y, yo)
    # the compressed operator reproduces A x: per column,
    # ||y - A x|| <= ||A - A_hat||_2 ||x|| + (matvec rounding)
    #             <= tensor_err ||x|| + tol ||A x||     (Lemma 1: ||A - A_hat||_F = tensor_err)
    xa = np.asarray(xin, dtype=np.float64)
    ya = np.asarray(A, dtype=np.float64) @ xa
    for s in range(2):
        lhs = np.linalg.norm(y[:, s] - ya[:, s])
        bound = res["tensor_err"] * np.linalg.norm(xa[:, s]) + tol_for(prec) * np.linalg.norm(ya[:, s])
        assert lhs <= bound, (s, lhs, bound)
