"""GPU parity of the C-ABI path against the FP64 oracle (same seeded inputs).

Bars: bit-exact for the gather (a scaling by sqrt(eta_k) in fp64, rounded
once to the path's type), identical ranks on the fp64 path, relative
Frobenius error <= 1e-10 (fp64) / 1e-5 (mixed) for every floating-point
result.  Singular vectors are never compared directly (signs and rotations
inside repeated singular values are not unique): the tests compare singular
values, ranks, the approximation tensor T, the dense M_E[T] and the matvec."""
import math

import numpy as np
import pytest

from oracle import sma_oracle as O
from sma_inputs import generators as G

from _util import (TOL_FP64, TOL_MIXED, apply, gpu_tensor, input_matrix, np_dtype,
                   oracle_at_gpu_ranks, oracle_tensor, reconstruct, rel, to_dev, tol_for)

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


def problem(kind):
    g = np.random.default_rng(11)
    if kind == "toeplitz_ragged":          # 5 x 5 blocks of 7 x 5, p = 9
        bm = G.toeplitz_map(5)
        return G.Problem(kind, g.standard_normal((9, 7, 5)), bm)
    if kind == "wide_trans":               # m < n: transposed Jacobi path
        bm = G.hankel_map(4)
        return G.Problem(kind, g.standard_normal((7, 6, 11)), bm)
    if kind == "tridiag_zero_blocks":      # -1 entries in the map
        bm = G.block_banded_map(6, 1)
        return G.Problem(kind, g.standard_normal((16, 9, 9)), bm)
    if kind == "planted_cfg1":
        return G.planted_kron_toeplitz()
    if kind == "single_block":
        return G.Problem(kind, g.standard_normal((1, 13, 9)), np.zeros((1, 1), dtype=np.int32))
    if kind == "block_mode_fp64":          # 192 x 192 fp64 exceeds shared memory
        bm = G.toeplitz_map(2)
        return G.Problem(kind, g.standard_normal((3, 192, 192)), bm)
    if kind == "block_mode_fp32":          # 256 x 256 fp32 exceeds shared memory
        bm = G.toeplitz_map(2)
        return G.Problem(kind, g.standard_normal((3, 256, 256)), bm)
    if kind == "p300":                     # more than 256 distinct blocks: N-tiled transform
        bm = G.block_diagonal_map(300)
        return G.Problem(kind, g.standard_normal((300, 8, 6)), bm)
    if kind == "wide_128":                 # n = 128 blocks: the matvec's staged epilogue
        bm = G.toeplitz_map(3)
        return G.Problem(kind, g.standard_normal((5, 24, 128)), bm)
    if kind == "tall_300x40":              # QR reflectors longer than 256 rows
        bm = G.toeplitz_map(2)
        return G.Problem(kind, g.standard_normal((3, 300, 40)), bm)
    # short columns: the fp32 Jacobi's partial-warp groups (16 lanes up to 64
    # rows, 8 lanes up to 32), with full and ragged tiles and float4 rows
    if kind == "short_64x64":
        bm = G.block_banded_map(4, 1)
        return G.Problem(kind, g.standard_normal((10, 64, 64)), bm)
    if kind == "short_48x40":
        bm = G.toeplitz_map(3)
        return G.Problem(kind, g.standard_normal((5, 48, 40)), bm)
    if kind == "short_32x32":
        bm = G.toeplitz_map(3)
        return G.Problem(kind, g.standard_normal((5, 32, 32)), bm)
    raise KeyError(kind)


def run(pr, prec, decomp=S.SMA_TSVDM, **kw):
    A = input_matrix(pr, prec)
    h = S.Handle([pr], prec=prec, decomp=decomp, **kw)
    dA = to_dev(A)
    res = h.compress([dA])[0]
    return h, A, res


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("kind", ["toeplitz_ragged", "wide_trans", "tridiag_zero_blocks"])
def test_gather_is_exact(prec, kind):
    pr = problem(kind)
    h, A, res = run(pr, prec, rel_tol=1e-3)
    X = gpu_tensor(h, S.EXPORT_X, (pr.m, pr.n, pr.p), prec)
    Xo = oracle_tensor(A, pr).astype(np_dtype(prec)).astype(np.float64)
    assert np.array_equal(X, Xo)
    assert abs(res["norm"] - np.linalg.norm(Xo)) <= 1e-13 * np.linalg.norm(Xo)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("kind", ["toeplitz_ragged", "wide_trans", "planted_cfg1", "p300"])
def test_transform_matches(prec, kind):
    pr = problem(kind)
    h, A, _ = run(pr, prec, rel_tol=1e-3)
    Xh = gpu_tensor(h, S.EXPORT_XHAT, (pr.m, pr.n, pr.p), prec)
    Xho = O.mode3(oracle_tensor(A, pr), O.dct2_matrix(pr.p))
    assert rel(Xh, Xho) < (1e-14 if prec == S.SMA_FP64 else 2e-6)


PRECONDS = [S.SMA_PRECOND_NONE, S.SMA_PRECOND_QRCP, S.SMA_PRECOND_QRCP2]
QNAME = {S.SMA_PRECOND_NONE: "plain", S.SMA_PRECOND_QRCP: "qrcp", S.SMA_PRECOND_QRCP2: "qrcp2"}


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("kind", ["toeplitz_ragged", "wide_trans", "tridiag_zero_blocks",
                                  "planted_cfg1", "single_block", "block_mode_fp64",
                                  "block_mode_fp32", "tall_300x40", "p300", "short_64x64",
                                  "short_48x40", "short_32x32"])
@pytest.mark.parametrize("tol", [1e-2, 1e-6])
@pytest.mark.parametrize("pre", PRECONDS, ids=QNAME.get)
def test_tsvdm_end_to_end(prec, kind, tol, pre):
    pr = problem(kind)
    h, A, res = run(pr, prec, rel_tol=tol, precondition=pre)
    X = oracle_tensor(A, pr)
    M = O.dct2_matrix(pr.p)
    ora = O.tsvdm(X, M, rel_tol=tol)
    assert res["device_status"] == 0
    # singular values per slice
    rc = min(pr.m, pr.n)
    sig = gpu_tensor(h, S.EXPORT_SIGMA, (rc, pr.p), prec)
    smax = max(float(np.max(s)) for s in ora.sigma)
    diff = max(float(np.max(np.abs(sig[:, i] - ora.sigma[i]))) for i in range(pr.p))
    assert diff <= (1e-12 if prec == S.SMA_FP64 else 2e-5) * smax
    # ranks (step 4)
    ranks = h.ranks(0)
    cmp = oracle_at_gpu_ranks(ranks, ora, X, M, tol, prec, f"tsvdm {kind} tol {tol:g} pre {pre}")
    assert res["total_rank"] == int(ranks.sum())
    # error report (step 5) and Lemma 1
    if prec == S.SMA_FP64:
        assert abs(res["tensor_err"] - ora.err) <= 1e-9 * max(ora.err, 1e-12 * ora.normX)
    assert res["tensor_err"] <= tol * ora.normX * (1 + 1e-9)
    Ah = reconstruct(h, pr, prec)
    T = gpu_tensor(h, S.EXPORT_T, (pr.m, pr.n, pr.p), prec)
    tolp = tol_for(prec)
    assert rel(T, cmp.tensor_approx()) < tolp
    Ao = O.M_E(cmp.tensor_approx(), pr.block_map)
    assert rel(Ah, Ao) < tolp
    # Section 6.2 report: trace error of the square cases, storage ratio
    A64 = np.asarray(A, dtype=np.float64)
    if pr.m == pr.n and pr.ell == pr.q:
        tr_o = abs(np.trace(A64) - np.trace(Ao)) / abs(np.trace(A64))
        assert abs(res["trace_relerr"] - tr_o) <= tolp * np.linalg.norm(A64) / abs(np.trace(A64))
    else:
        assert res["trace_relerr"] == 0.0
    assert abs(res["storage_ratio"] - ranks.sum() * (pr.m + pr.n + 1) / (pr.m * pr.n * pr.p)) < 1e-15
    if prec == S.SMA_MIXED:
        assert abs(res["tensor_err"] - cmp.err) <= 1e-6 * cmp.err + tolp * ora.normX
    lemma = np.linalg.norm(np.asarray(A, dtype=np.float64) - Ah)
    assert abs(lemma - res["tensor_err"]) <= tolp * ora.normX + 1e-6 * res["tensor_err"]
    assert res["orth_defect"] < (1e-12 if prec == S.SMA_FP64 else 1e-4)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("kind", ["toeplitz_ragged", "wide_trans", "tridiag_zero_blocks",
                                  "block_mode_fp32", "wide_128", "short_64x64", "short_32x32"])
@pytest.mark.parametrize("pre", PRECONDS, ids=QNAME.get)
def test_kron_sum_apply(prec, kind, pre):
    pr = problem(kind)
    h, A, res = run(pr, prec, rel_tol=1e-2, precondition=pre)
    X = oracle_tensor(A, pr)
    M = O.dct2_matrix(pr.p)
    ora = O.tsvdm(X, M, rel_tol=1e-2)
    cmp = oracle_at_gpu_ranks(h.ranks(0), ora, X, M, 1e-2, prec, f"apply {kind} pre {pre}")
    x = G.random_rhs(pr.q * pr.n, 5, 0).astype(np_dtype(prec)).astype(np.float64)
    y = apply(h, pr, x, prec)
    yo = O.apply_kron(O.tsvdm_kron_terms(cmp, pr.block_map), x)
    # against the oracle's factored matvec, and against dense A_hat x
    assert rel(y, yo) < tol_for(prec)
    Ah = reconstruct(h, pr, prec)
    assert rel(y, Ah @ x) < (1e-12 if prec == S.SMA_FP64 else 1e-5)


def test_planted_rank_ranks_equal_with_margin():
    pr = problem("planted_cfg1")
    h, A, res = run(pr, S.SMA_FP64, rel_tol=1e-6)
    ora = O.tsvdm(oracle_tensor(A, pr), O.dct2_matrix(pr.p), rel_tol=1e-6)
    assert np.array_equal(h.ranks(0), ora.ranks)
    # each transformed 16 x 16 slice is a generic mix of three B_k: full rank
    assert np.all(ora.ranks == 16)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("pre", PRECONDS, ids=QNAME.get)
def test_planted_slice_ranks_and_zero_rank_slices(prec, pre):
    m, n, p = 12, 9, 6
    ranks = [3, 0, 1, 5, 2, 0]
    L, R = G.planted_tsvdm_tensor(m, n, p, ranks)
    Xh = np.stack([L[i] @ R[i] for i in range(p)], axis=2)
    M = O.dct2_matrix(p)
    X = O.mode3(Xh, M.T)
    # a block-diagonal matrix whose distinct blocks are the slices of X
    blocks = np.transpose(X, (2, 0, 1)).copy()
    pr = G.Problem("planted_tsvdm", blocks, G.block_diagonal_map(p))
    h, A, res = run(pr, prec, rel_tol=1e-4, precondition=pre)
    ora = O.tsvdm(oracle_tensor(A, pr), M, rel_tol=1e-4)
    assert list(ora.ranks) == ranks
    assert list(h.ranks(0)) == ranks
    assert res["n_kron_terms"] == 4
    T = gpu_tensor(h, S.EXPORT_T, None, prec)
    reconstruct(h, pr, prec)
    T = gpu_tensor(h, S.EXPORT_T, (m, n, p), prec)
    assert rel(T, ora.tensor_approx()) < tol_for(prec)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("pre", PRECONDS, ids=QNAME.get)
def test_fixed_rank_and_user_transform(prec, pre):
    pr = problem("toeplitz_ragged")
    Mu = G.random_orthogonal(pr.p, 5)
    h, A, res = run(pr, prec, fixed_rank=2, mkind=S.SMA_M_USER, M_user=Mu, precondition=pre)
    ora = O.tsvdm(oracle_tensor(A, pr), Mu, fixed_rank=2)
    assert list(h.ranks(0)) == [2] * pr.p
    Ah = reconstruct(h, pr, prec)
    assert rel(Ah, O.M_E(ora.tensor_approx(), pr.block_map)) < tol_for(prec)
    assert abs(res["tensor_err"] - ora.err) <= 1e-5 * ora.err


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_identity_transform_is_slicewise_svd(prec):
    pr = problem("toeplitz_ragged")
    h, A, res = run(pr, prec, fixed_rank=3, mkind=S.SMA_M_IDENTITY)
    X = oracle_tensor(A, pr)
    for k in range(pr.p):
        s = np.linalg.svd(X[:, :, k], compute_uv=False)
        sig = gpu_tensor(h, S.EXPORT_SIGMA, (5, pr.p), prec)[:, k]
        assert np.max(np.abs(sig - s)) <= (1e-12 if prec == S.SMA_FP64 else 1e-5) * s[0]


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_host_pointer_inputs_match_device(prec):
    pr = problem("toeplitz_ragged")
    A = np.asfortranarray(input_matrix(pr, prec))
    h = S.Handle([pr], prec=prec, rel_tol=1e-3)
    r_host = h.compress([A])[0]
    Ah_host = reconstruct(h, pr, prec)
    x = np.asfortranarray(G.random_rhs(pr.q * pr.n, 3, 1).astype(np_dtype(prec)))
    y_host = np.zeros((pr.ell * pr.m, 3), dtype=np_dtype(prec), order="F")
    h.apply(0, x, y_host)
    h2, _, r_dev = run(pr, prec, rel_tol=1e-3)
    assert r_host["total_rank"] == r_dev["total_rank"]
    assert np.array_equal(Ah_host, reconstruct(h2, pr, prec))
    assert rel(y_host, apply(h2, pr, x.astype(np.float64), prec)) < 1e-12


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_blocks_layout_equals_dense(prec):
    pr = problem("tridiag_zero_blocks")
    blocks = np.concatenate([b for b in pr.blocks], axis=1)   # m x (n p)
    Bl = blocks if prec == S.SMA_FP64 else blocks.astype(np.float32)
    h = S.Handle([pr], prec=prec, rel_tol=1e-3, layout=S.SMA_INPUT_BLOCKS)
    h.compress([to_dev(Bl)])
    X = gpu_tensor(h, S.EXPORT_X, (pr.m, pr.n, pr.p), prec)
    h2, A, _ = run(pr, prec, rel_tol=1e-3)
    assert np.array_equal(X, gpu_tensor(h2, S.EXPORT_X, (pr.m, pr.n, pr.p), prec))


# ------------------------------------------------------------------ Tucker family

@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_tucker_blockmode_recovers_kronecker_rank(prec):
    pr = problem("planted_cfg1")
    tol = 1e-6 if prec == S.SMA_FP64 else 1e-4
    h, A, res = run(pr, prec, decomp=S.SMA_TUCKER_BLOCKMODE, rel_tol=tol)
    X = oracle_tensor(A, pr)
    t = O.tucker1_blockmode(X, rel_tol=tol)
    assert t.rank == 3 and res["ranks"][0] == 3 and res["n_kron_terms"] == 3
    Ah = reconstruct(h, pr, prec)
    To = t.tensor_approx()
    assert rel(Ah, O.M_E(To, pr.block_map)) < tol_for(prec)
    # the error is measured directly as ||X - T||_F on the device
    floor = (1e-13 if prec == S.SMA_FP64 else TOL_MIXED) * np.linalg.norm(X)
    assert abs(res["tensor_err"] - t.err) <= 1e-6 * t.err + floor
    x = G.random_rhs(pr.q * pr.n, 4, 2).astype(np_dtype(prec)).astype(np.float64)
    y = apply(h, pr, x, prec)
    assert rel(y, O.apply_kron(O.tucker1_kron_terms(t, pr.block_map), x)) < tol_for(prec)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_shared_u_spsd_blr(prec):
    pr = G.spacetime_covariance(npts=24, T=6, seed_index=1)
    h, A, res = run(pr, prec, decomp=S.SMA_TUCKER_SHARED_U, fixed_rank=8)
    X = oracle_tensor(A, pr)
    su = O.shared_u(X, rank=8)
    Ah = reconstruct(h, pr, prec)
    Ao = O.M_E(su.tensor_approx(), pr.block_map)
    assert rel(Ah, Ao) < tol_for(prec)
    ev = np.linalg.eigvalsh((Ah + Ah.T) / 2)
    assert ev.min() > -(1e-12 if prec == S.SMA_FP64 else 1e-5) * ev.max()
    x = G.random_rhs(pr.q * pr.n, 3, 3).astype(np_dtype(prec)).astype(np.float64)
    assert rel(apply(h, pr, x, prec), Ao @ x) < tol_for(prec)
    floor = (1e-13 if prec == S.SMA_FP64 else TOL_MIXED) * np.linalg.norm(X)
    assert abs(res["tensor_err"] - su.err) <= 1e-6 * su.err + floor


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_rowcol_tucker_blr(prec):
    pr = G.lti_hankel(s=8, d=6, n_in=7, n_out=5, seed_index=2)
    h, A, res = run(pr, prec, decomp=S.SMA_TUCKER_ROWCOL, fixed_rank=3)
    X = oracle_tensor(A, pr)
    t = O.tucker2_rows_cols(X, 3, 3)
    Ah = reconstruct(h, pr, prec)
    Ao = O.M_E(t.tensor_approx(), pr.block_map)
    assert rel(Ah, Ao) < tol_for(prec)
    x = G.random_rhs(pr.q * pr.n, 3, 4).astype(np_dtype(prec)).astype(np.float64)
    assert rel(apply(h, pr, x, prec), Ao @ x) < tol_for(prec)
    floor = (1e-13 if prec == S.SMA_FP64 else TOL_MIXED) * np.linalg.norm(X)
    assert abs(res["tensor_err"] - t.err) <= 1e-6 * t.err + floor


@pytest.mark.parametrize("kind", ["block_mode_fp32", "toeplitz_ragged", "wide_128", "short_64x64",
                                  "short_32x32"])
def test_autotuned_plan_gives_the_same_compression(kind):
    """The autotuner only changes the Jacobi plan (tile, block width, warps):
    the retained ranks, singular values and rebuilt tensor stay those of the
    default plan to fp32 accuracy, and a second handle reuses the choice."""
    pr = problem(kind)
    prec = S.SMA_MIXED
    h0, A, r0 = run(pr, prec, rel_tol=1e-6)
    h1, _, r1 = run(pr, prec, rel_tol=1e-6, autotune=True)
    h2, _, r2 = run(pr, prec, rel_tol=1e-6, autotune=True)
    rc = min(pr.m, pr.n)
    s0, s1 = (gpu_tensor(h, S.EXPORT_SIGMA, (rc, pr.p), prec) for h in (h0, h1))
    assert np.max(np.abs(s0 - s1)) <= 2e-5 * np.max(s0)
    assert np.array_equal(h1.ranks(0), h2.ranks(0))
    assert abs(r1["tensor_err"] - r0["tensor_err"]) <= 1e-4 * r0["norm"]
    for r in (r1, r2):
        assert r["device_status"] == 0
    T0, T1 = (reconstruct(h, pr, prec) for h in (h0, h1))
    assert rel(T1, T0) < TOL_MIXED

