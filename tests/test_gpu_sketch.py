"""Section 6.3's randomized block-index factor on the GPU: V from the sketch
Y_k = Omega^T X_k Psi (Gaussian maps passed in), compared with the FP64
oracle's tucker1_blockmode_sketch on the same maps: the subspace of V, the
error, the reconstruction and the Kronecker-sum matvec; with identity maps it
must agree with the deterministic block-index factor."""
import numpy as np
import pytest

from oracle import sma_oracle as O
from sma_inputs import generators as G

from _util import (TOL_MIXED, gpu_tensor, input_matrix, np_dtype, oracle_tensor, reconstruct,
                   rel, to_dev, tol_for, apply)

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


def projector_gap(Ug, Uo):
    return float(np.linalg.norm(Ug @ Ug.T - Uo @ Uo.T, 2))


def run_sketch(pr, prec, r, Om, Ps):
    A = input_matrix(pr, prec)
    h = S.Handle([pr], prec=prec, decomp=S.SMA_TUCKER_BLOCKMODE, fixed_rank=r, sketch=(Om, Ps))
    res = h.compress([to_dev(A)])[0]
    return h, A, res


def check_against_oracle(h, A, res, pr, prec, r, Om, Ps):
    X = stored_tensor(A, pr, prec)
    # the oracle takes the maps as the path rounds them (fp32 on the mixed path)
    if prec == S.SMA_MIXED:
        Om = Om.astype(np.float32).astype(np.float64)
        Ps = Ps.astype(np.float32).astype(np.float64)
    t = O.tucker1_blockmode_sketch(X, Om, Ps, r)
    assert res["device_status"] == 0
    assert res["ranks"][0] == r and res["n_kron_terms"] == r
    V = gpu_tensor(h, S.EXPORT_FACTOR, (pr.p, pr.p), prec)[:, :r]
    assert projector_gap(V, t.V) < (1e-9 if prec == S.SMA_FP64 else 1e-5)
    assert res["orth_defect"] < (1e-11 if prec == S.SMA_FP64 else 1e-5)
    floor = (1e-12 if prec == S.SMA_FP64 else TOL_MIXED) * np.linalg.norm(X)
    assert abs(res["tensor_err"] - t.err) <= 1e-6 * t.err + floor
    Ah = reconstruct(h, pr, prec)
    assert rel(Ah, O.M_E(t.tensor_approx(), pr.block_map)) < tol_for(prec)
    x = G.random_rhs(pr.q * pr.n, 3, 8).astype(np_dtype(prec)).astype(np.float64)
    y = apply(h, pr, x, prec)
    assert rel(y, O.apply_kron(O.tucker1_kron_terms(t, pr.block_map), x)) < tol_for(prec)
    return t


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_sketch_recovers_planted_kronecker_sum(prec):
    pr = G.planted_kron_toeplitz(ell=50, m=6, terms=4, seed_index=5)      # p = 99
    Om, Ps = G.gaussian_sketch(pr.m, pr.n, 3)
    h, A, res = run_sketch(pr, prec, 4, Om, Ps)
    t = check_against_oracle(h, A, res, pr, prec, 4, Om, Ps)
    X = stored_tensor(A, pr, prec)
    assert t.err <= 1e-6 * np.linalg.norm(X)          # the planted sum is recovered
    h.close()


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_sketch_block_tridiagonal(prec):
    """The matrix with the most blocks among those of a small batch of the
    block-tridiagonal workload whose dense form stays small (order <= 2048;
    Kron rank K plus 1e-4 noise and a 30% zero pattern), rank K from a sketch
    with s^2 >= K."""
    prs = G.block_tridiag_batch(count=12)
    pr = max((q for q in prs if q.block_map.shape[0] * q.m <= 2048), key=lambda q: q.p)
    K = int(pr.extra["K"])
    Om, Ps = G.gaussian_sketch(pr.m, pr.n, 3, seed_index=8)
    h, A, res = run_sketch(pr, prec, K, Om, Ps)
    check_against_oracle(h, A, res, pr, prec, K, Om, Ps)
    h.close()


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_identity_maps_give_the_deterministic_factor(prec):
    pr = G.planted_kron_toeplitz(ell=12, m=5, terms=3, noise=1e-3, seed_index=3)
    r = 3
    h, A, res = run_sketch(pr, prec, r, np.eye(pr.m), np.eye(pr.n))
    hd = S.Handle([pr], prec=prec, decomp=S.SMA_TUCKER_BLOCKMODE, fixed_rank=r)
    resd = hd.compress([to_dev(A)])[0]
    V = gpu_tensor(h, S.EXPORT_FACTOR, (pr.p, pr.p), prec)[:, :r]
    Vd = gpu_tensor(hd, S.EXPORT_FACTOR, (pr.p, pr.p), prec)[:, :r]
    assert projector_gap(V, Vd) < (1e-10 if prec == S.SMA_FP64 else 1e-5)
    assert abs(res["tensor_err"] - resd["tensor_err"]) <= 1e-6 * resd["tensor_err"]
    check_against_oracle(h, A, res, pr, prec, r, np.eye(pr.m), np.eye(pr.n))
    h.close()
    hd.close()
