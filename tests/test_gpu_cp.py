"""CP by alternating least squares on the GPU (Section 2.3 with the matrix
forms of Theorem tildeA / Corollary kronsumcp), against the FP64 oracle's
cp_als from the same initial factors and iteration count: the Kruskal
tensor, the error, the dense Kronecker sum and its matvec; a planted exact
CP tensor is recovered; a singular normal-equations system is reported."""
import numpy as np
import pytest

from oracle import sma_oracle as O
from sma_inputs import generators as G

from _util import (apply, gpu_tensor, input_matrix, np_dtype, oracle_tensor, reconstruct, rel,
                   to_dev)

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


def stored_tensor(A, pr, prec):
    X = oracle_tensor(A, pr)
    return X if prec == S.SMA_FP64 else X.astype(np.float32).astype(np.float64)


def rounded(a, prec):
    return a if prec == S.SMA_FP64 else a.astype(np.float32).astype(np.float64)


def run_cp(pr, prec, r, X0, Z0, iters, check=True):
    A = input_matrix(pr, prec)
    h = S.Handle([pr], prec=prec, decomp=S.SMA_CP_ALS, fixed_rank=r, cp_init=(X0, Z0),
                 cp_iters=iters)
    res = h.compress([to_dev(A)], check=check)[0]
    return h, A, res


def compare(h, A, res, pr, prec, c, tol):
    X = stored_tensor(A, pr, prec)
    T = gpu_tensor(h, S.EXPORT_T, (pr.m, pr.n, pr.p), prec)
    assert rel(T, c.tensor_approx()) < tol
    assert abs(res["tensor_err"] - c.err) <= tol * np.linalg.norm(X)
    Ah = reconstruct(h, pr, prec)
    assert rel(Ah, O.kron_dense(O.cp_kron_terms(c, pr.block_map))) < tol
    x = G.random_rhs(pr.q * pr.n, 3, 9).astype(np_dtype(prec)).astype(np.float64)
    assert rel(apply(h, pr, x, prec), O.apply_kron(O.cp_kron_terms(c, pr.block_map), x)) < tol


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_planted_cp_is_recovered(prec):
    pr, f = G.planted_cp_toeplitz(ell=8, m=12, n=10, r=3)
    g = np.random.default_rng(5)
    X0 = f["Xf"] + 0.05 * g.standard_normal(f["Xf"].shape)
    Z0 = f["Zf"] + 0.05 * g.standard_normal(f["Zf"].shape)
    h, A, res = run_cp(pr, prec, 3, X0, Z0, 30)
    assert res["device_status"] == 0 and res["ranks"][0] == 3 and res["n_kron_terms"] == 3
    X = stored_tensor(A, pr, prec)
    c = O.cp_als(X, rounded(X0, prec), rounded(Z0, prec), 30)
    tol = 1e-10 if prec == S.SMA_FP64 else 1e-5
    compare(h, A, res, pr, prec, c, tol)
    assert res["rel_err"] < (1e-12 if prec == S.SMA_FP64 else 1e-6)
    h.close()


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_cp_on_covariance_follows_the_oracle(prec):
    """Not an exact CP tensor: 8 iterations of rank 4 from N(0,1) factors on
    the small space-time covariance; the same iterate as the oracle."""
    pr = G.spacetime_covariance(npts=12, T=6, seed_index=1)
    X0, Z0 = G.cp_initial_factors(pr.m, pr.n, 4)
    h, A, res = run_cp(pr, prec, 4, X0, Z0, 8)
    assert res["device_status"] == 0
    X = stored_tensor(A, pr, prec)
    c = O.cp_als(X, rounded(X0, prec), rounded(Z0, prec), 8)
    tol = 1e-10 if prec == S.SMA_FP64 else 1e-4
    compare(h, A, res, pr, prec, c, tol)
    Xf = gpu_tensor(h, S.EXPORT_CP_X, (pr.m, 4), prec)
    assert rel(Xf, c.Xf) < tol
    h.close()


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_singular_normal_equations_are_reported(prec):
    pr, _ = G.planted_cp_toeplitz(ell=4, m=6, n=5, r=2)
    X0, Z0 = G.cp_initial_factors(pr.m, pr.n, 2)
    X0[:, 1] = X0[:, 0]
    Z0[:, 1] = Z0[:, 0]           # equal columns in both: (X0^T X0) .* (Z0^T Z0) is singular
    h, A, res = run_cp(pr, prec, 2, X0, Z0, 2, check=False)
    assert h.last_status == S.SMA_ERR_NONFINITE
    assert res["device_status"] & (1 << S.SMA_ERR_NONFINITE)
    assert np.isfinite(res["tensor_err"])
    h.close()
