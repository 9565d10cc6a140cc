"""Pins for the FP64 oracle: checks against values the paper prints, closed
forms, invariants the paper proves and brute force on tiny inputs.  Each test
is chosen so that a plausible slip in the oracle (a dropped sqrt(eta), a
transposed transform, a wrong truncation order, a swapped mode) fails it."""
import json
import math
import os

import numpy as np
import pytest
import scipy.fft

from oracle import sma_oracle as O
from sma_inputs import generators as G

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def random_problem(bm, m, n, seed=0):
    g = np.random.default_rng(seed)
    p = int(bm.max()) + 1
    blocks = g.standard_normal((p, m, n))
    return G.Problem("t", blocks, bm)


# ---------------------------------------------------------------- Section 3 maps

def test_tridiagonal_example_counts():
    gold = GOLDEN["tridiagonal_symmetric_ell4"]
    bm = G.symmetric_tridiagonal_map(gold["ell"])
    assert int(bm.max()) + 1 == gold["p"]
    for ell in (2, 4, 9):
        assert int(G.block_banded_map(ell, 1).max()) + 1 == 3 * ell - 2
        assert int(G.symmetric_tridiagonal_map(ell).max()) + 1 == 2 * ell - 1
    for ell, b in ((7, 2), (10, 3)):
        assert int(G.block_banded_map(ell, b).max()) + 1 == ell * (2 * b + 1) - b * (b + 1)
        sym = sum(1 for a in range(ell) for c in range(ell) if 0 <= a - c <= b)
        assert sym == ell * (b + 1) - b * (b + 1) // 2


def test_mapping_matrices_unit_norm_and_partition():
    for bm in (G.toeplitz_map(6), G.hankel_map(5), G.block_banded_map(5, 1),
               G.block_diagonal_map(4), G.symmetric_tridiagonal_map(5)):
        p = int(bm.max()) + 1
        E = O.mapping_matrices(bm, p)
        for Ek in E:
            assert abs(np.linalg.norm(Ek) - 1.0) < 1e-15
        supp = sum((Ek != 0).astype(int) for Ek in E)
        assert np.array_equal(supp, (bm >= 0).astype(int))


def test_toeplitz_weights_match_shift_powers():
    ell = 7
    bm = G.toeplitz_map(ell)
    E = O.mapping_matrices(bm, 2 * ell - 1)
    Ed = np.eye(ell, k=-1)
    Eu = Ed.T
    for j in range(ell):
        assert np.allclose(E[j], np.linalg.matrix_power(Ed, j) / math.sqrt(ell - j), atol=0, rtol=1e-15)
    for j in range(1, ell):
        assert np.allclose(E[ell - 1 + j], np.linalg.matrix_power(Eu, j) / math.sqrt(ell - j), atol=0, rtol=1e-15)


def test_block_diagonal_example():
    ell = 5
    E = O.mapping_matrices(G.block_diagonal_map(ell), ell)
    for k in range(ell):
        e = np.zeros(ell)
        e[k] = 1
        assert np.array_equal(E[k], np.outer(e, e))


def test_hankel_multiplicities_rule():
    s = 6
    eta = O.multiplicities(G.hankel_map(s), 2 * s - 1)
    expect = [k if k <= s else 2 * s - k for k in range(1, 2 * s)]
    assert list(eta) == expect
    gold = GOLDEN["era_tensor_size"]
    assert 2 * gold["s"] - 1 == gold["tensor"][1]


def test_multilevel_running_example_eta():
    gold = GOLDEN["multilevel_running_example"]
    # lower block triangle of a 4x4 block-pentadiagonal Toeplitz matrix
    bm = -np.ones((4, 4), dtype=np.int32)
    for a in range(4):
        for b in range(4):
            if 0 <= a - b <= 2:
                bm[a, b] = a - b
    assert list(O.multiplicities(bm, gold["p1"])) == gold["eta1"]
    assert list(O.multiplicities(G.block_diagonal_map(5), gold["p2"])) == gold["eta2"]
    assert gold["p1"] * gold["p2"] == gold["stored_blocks"]


def test_storage_ratio_reading():
    gold = GOLDEN["spacetime_storage_ratio"]
    N, T, r = gold["N"], gold["T"], gold["r"]
    printed = O.storage_ratio_blr(N, T, r)
    # the printed 0.002 is reproduced when the core holds all p = 2T-1 slices
    core_all = (r * r * (2 * T - 1) + N * r) / (N * N * T)
    assert round(core_all, 3) == gold["printed"]
    assert round(printed, 3) != gold["printed"]


@pytest.mark.parametrize("kind", ["toeplitz", "hankel", "tridiag", "blockdiag", "symtri"])
def test_struct_identity_and_inverse(kind):
    bm = {"toeplitz": G.toeplitz_map(5), "hankel": G.hankel_map(4),
          "tridiag": G.block_banded_map(5, 1), "blockdiag": G.block_diagonal_map(4),
          "symtri": G.symmetric_tridiagonal_map(4)}[kind]
    pr = random_problem(bm, 3, 2, seed=1)
    A = pr.dense()
    eta = O.multiplicities(bm, pr.p)
    # eq. (kronsum): sum_k E_k (x) sqrt(eta_k) A_k = A
    S = O.struct_E([math.sqrt(eta[k]) * pr.blocks[k] for k in range(pr.p)], bm, pr.p)
    assert rel(S, A) < 1e-15
    # M_E[T_E[A]] = A
    X = O.T_E(A, bm, pr.p, pr.m, pr.n)
    assert rel(O.M_E(X, bm), A) < 1e-15
    # on structured input the adjoint gather equals the gather
    assert rel(O.T_E_adjoint(A, bm, pr.p, pr.m, pr.n), X) < 1e-15
    # norm preservation: ||X||_F = ||A||_F
    assert abs(np.linalg.norm(X) - np.linalg.norm(A)) < 1e-13 * np.linalg.norm(A)


def test_adjoint_is_orthogonal_projection():
    bm = G.toeplitz_map(4)
    g = np.random.default_rng(3)
    A = g.standard_normal((4 * 3, 4 * 2))      # unstructured
    Xa = O.T_E_adjoint(A, bm, 7, 3, 2)
    R = A - O.M_E(Xa, bm)
    for _ in range(3):
        Y = g.standard_normal((3, 2, 7))
        assert abs(np.sum(R * O.M_E(Y, bm))) < 1e-13


def test_trace_orthogonality_remark():
    bm = G.hankel_map(4)
    E = O.mapping_matrices(bm, 7)
    g = np.random.default_rng(4)
    K, L = g.standard_normal((2, 3, 3))
    for j in range(7):
        for k in range(7):
            ip = np.sum(np.kron(E[j], K) * np.kron(E[k], L))
            if j != k:
                assert abs(ip) < 1e-14
            else:
                assert abs(ip - np.sum(K * L)) < 1e-13


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lemma1_error_transfer(seed):
    bm = G.toeplitz_map(5) if seed != 1 else G.hankel_map(5)
    pr = random_problem(bm, 4, 3, seed=seed)
    A = pr.dense()
    X = O.T_E(A, bm, pr.p, pr.m, pr.n)
    T = X + np.random.default_rng(seed + 10).standard_normal(X.shape) * 0.1
    lhs = np.linalg.norm(A - O.M_E(T, bm))
    rhs = np.linalg.norm(X - T)
    assert abs(lhs - rhs) < 1e-13 * rhs


def test_greedy_discovery_reproduces_partition():
    for bm in (G.toeplitz_map(5), G.hankel_map(4), G.block_banded_map(6, 1)):
        pr = random_problem(bm, 2, 3, seed=5)
        A = pr.dense()
        found = O.greedy_structure(A, bm.shape[0], bm.shape[1], 2, 3)
        # same partition of block positions (labels may differ)
        pairs = {(int(a), int(b)) for a, b in zip(bm.ravel(), found.ravel())}
        assert len(pairs) == len({a for a, _ in pairs}) == len({b for _, b in pairs})


# ---------------------------------------------------------------- transform

def test_dct2_matches_scipy_and_is_orthogonal():
    for p in (1, 2, 15, 127):
        M = O.dct2_matrix(p)
        ref = scipy.fft.dct(np.eye(p), type=2, norm="ortho", axis=0)
        assert np.max(np.abs(M - ref)) < 1e-13
        assert np.max(np.abs(M @ M.T - np.eye(p))) < 1e-13


def test_mode3_and_unfoldings():
    g = np.random.default_rng(6)
    X = g.standard_normal((3, 4, 5))
    M = g.standard_normal((2, 5))
    Y = O.mode3(X, M)
    assert Y.shape == (3, 4, 2)
    # X x3 M == M X_(3) in unfolded form
    assert rel(O.unfold(Y, 3), M @ O.unfold(X, 3)) < 1e-14
    assert O.unfold(X, 1).shape == (3, 20) and O.unfold(X, 2).shape == (4, 15)
    assert np.array_equal(O.unfold(X, 1)[:, 4:8], X[:, :, 1])
    assert np.array_equal(O.unfold(X, 2)[:, 3:6], X[:, :, 1].T)


# ---------------------------------------------------------------- t-SVDM

def test_global_truncation_hand_example():
    sig = [np.array([3.0, 2.0, 1.0]), np.array([4.0, 0.5, 0.1])]
    normX2 = 9 + 4 + 1 + 16 + 0.25 + 0.01
    tol = math.sqrt(1.3 / normX2)
    assert list(O.truncate_global(sig, tol, normX2)) == [2, 1]
    tol = math.sqrt(1.2 / normX2)          # 1 can no longer be dropped
    assert list(O.truncate_global(sig, tol, normX2)) == [3, 1]
    # ties: equal values are dropped from the highest slice index first
    sig = [np.array([2.0, 1.0]), np.array([2.0, 1.0])]
    assert list(O.truncate_global(sig, math.sqrt(1.0 / 10), 10.0)) == [2, 1]
    assert list(O.truncate_global(sig, 0.0, 10.0)) == [2, 2]


def test_tsvdm_identity_transform_diagonal_slices():
    # with M = I and diagonal slices the singular values are the diagonals
    X = np.zeros((3, 3, 2))
    X[:, :, 0] = np.diag([3.0, 2.0, 1.0])
    X[:, :, 1] = np.diag([4.0, 0.5, 0.1])
    res = O.tsvdm(X, np.eye(2), rel_tol=math.sqrt(1.3 / 30.26))
    assert list(res.ranks) == [2, 1]
    assert abs(res.err - math.sqrt(1.26)) < 1e-14
    T = res.tensor_approx()
    assert np.allclose(T[:, :, 0], np.diag([3.0, 2.0, 0.0]), atol=1e-14)
    assert np.allclose(T[:, :, 1], np.diag([4.0, 0.0, 0.0]), atol=1e-14)


def test_tsvdm_given_rank_vector():
    """The per-slice rank option: planted slices U diag(s) V^T under M = I
    truncate to the closed form U_r diag(s_r) V_r^T with error
    sqrt(sum of the dropped s^2); uniform ranks equal fixed_rank; the
    tolerance rule's own ranks reproduce the tolerance result."""
    g = np.random.default_rng(5)
    m, n, p = 7, 5, 4
    svals = [np.array([5.0, 3.0, 2.0, 0.5, 0.25]) * (i + 1) for i in range(p)]
    X = np.zeros((m, n, p))
    bases = []
    for i in range(p):
        U, _ = np.linalg.qr(g.standard_normal((m, n)))
        V, _ = np.linalg.qr(g.standard_normal((n, n)))
        X[:, :, i] = (U * svals[i]) @ V.T
        bases.append((U, V))
    r = [0, 2, 5, 1]
    res = O.tsvdm(X, np.eye(p), ranks=r)
    assert list(res.ranks) == r
    T = res.tensor_approx()
    for i in range(p):
        U, V = bases[i]
        want = (U[:, :r[i]] * svals[i][:r[i]]) @ V[:, :r[i]].T
        assert np.allclose(T[:, :, i], want, atol=1e-13)
    disc = sum(float(np.sum(svals[i][r[i]:] ** 2)) for i in range(p))
    assert abs(res.err - math.sqrt(disc)) < 1e-13
    # a uniform vector is fixed_rank; the tolerance rule's ranks reproduce it
    M = O.dct2_matrix(p)
    a = O.tsvdm(X, M, fixed_rank=3)
    b = O.tsvdm(X, M, ranks=[3] * p)
    assert np.array_equal(a.ranks, b.ranks) and rel(b.tensor_approx(), a.tensor_approx()) < 1e-15
    t = O.tsvdm(X, M, rel_tol=0.05)
    u = O.tsvdm(X, M, ranks=t.ranks)
    assert np.array_equal(t.ranks, u.ranks) and rel(u.tensor_approx(), t.tensor_approx()) < 1e-15
    assert u.err == t.err
    with pytest.raises(ValueError):
        O.tsvdm(X, M, ranks=[6, 0, 0, 0])


def test_blockwise_M_E_matvec_equals_the_dense_map():
    """apply_M_E (block by block, with the -1 zero blocks of a banded map)
    against the dense M_E[T] times x, and M_E[T_E(A)] x = A x."""
    for bm in (G.toeplitz_map(4), G.block_banded_map(5, 1), G.hankel_map(3)):
        pr = random_problem(bm, 3, 2, seed=4)
        A = pr.dense()
        T = O.T_E(A, bm, pr.p, pr.m, pr.n)
        x = np.random.default_rng(2).standard_normal((bm.shape[1] * 2, 3))
        assert rel(O.apply_M_E(T, bm, x), A @ x) < 1e-14
        T2 = np.random.default_rng(3).standard_normal(T.shape)
        assert rel(O.apply_M_E(T2, bm, x), O.M_E(T2, bm) @ x) < 1e-14


def test_tsvdm_full_rank_reproduces_A():
    pr = G.planted_kron_toeplitz(ell=5, m=4, terms=2, seed_index=0)
    A = pr.dense()
    X = O.T_E(A, pr.block_map, pr.p, pr.m, pr.n)
    res = O.tsvdm(X, O.dct2_matrix(pr.p), rel_tol=0.0)
    assert all(res.ranks == 4)
    assert rel(res.tensor_approx(), X) < 1e-14
    terms = O.tsvdm_kron_terms(res, pr.block_map)
    assert rel(O.kron_dense(terms), A) < 1e-14


@pytest.mark.parametrize("Mkind", ["dct", "haar"])
def test_tsvdm_planted_slice_ranks(Mkind):
    m, n, p = 9, 7, 6
    ranks = [3, 0, 1, 5, 2, 4]
    L, R = G.planted_tsvdm_tensor(m, n, p, ranks)
    Xh = np.stack([L[i] @ R[i] for i in range(p)], axis=2)
    M = O.dct2_matrix(p) if Mkind == "dct" else G.random_orthogonal(p, 0)
    X = O.mode3(Xh, M.T)
    res = O.tsvdm(X, M, rel_tol=1e-10)
    assert list(res.ranks) == ranks
    assert res.rel_err < 1e-13
    assert rel(res.tensor_approx(), X) < 1e-13


def test_tsvdm_error_is_parseval_and_lemma1():
    pr = G.planted_kron_toeplitz(ell=6, m=5, terms=2, noise=1e-3, seed_index=0)
    A = pr.dense()
    X = O.T_E(A, pr.block_map, pr.p, pr.m, pr.n)
    M = O.dct2_matrix(pr.p)
    res = O.tsvdm(X, M, rel_tol=1e-2)
    assert 0 < res.ranks.sum() < pr.p * 5
    T = res.tensor_approx()
    # Parseval: the error measured in the transform domain equals the direct one
    assert abs(np.linalg.norm(X - T) - res.err) < 1e-12 * max(res.err, 1e-300) + 1e-14
    # Lemma 1 end to end through the Kronecker-sum form
    Ahat = O.kron_dense(O.tsvdm_kron_terms(res, pr.block_map))
    assert abs(np.linalg.norm(A - Ahat) - res.err) < 1e-12 * res.err
    assert res.err <= 1e-2 * np.linalg.norm(X) * (1 + 1e-12)


def test_p1_reduces_to_eckart_young():
    g = np.random.default_rng(7)
    A = g.standard_normal((6, 5))
    X = A[:, :, None]
    res = O.tsvdm(X, np.ones((1, 1)), fixed_rank=2)
    s = np.linalg.svd(A, compute_uv=False)
    assert abs(res.err - math.sqrt(np.sum(s[2:] ** 2))) < 1e-13
    # no rank-2 matrix from random search beats it
    best = res.err
    for _ in range(200):
        B = g.standard_normal((6, 2)) @ g.standard_normal((2, 5))
        c = np.sum(A * B) / np.sum(B * B)
        assert np.linalg.norm(A - c * B) >= best - 1e-12


def test_kron_terms_preserve_structure_and_blr_agrees():
    pr = G.planted_kron_toeplitz(ell=6, m=4, terms=2, noise=1e-3, seed_index=0)
    A = pr.dense()
    X = O.T_E(A, pr.block_map, pr.p, pr.m, pr.n)
    res = O.tsvdm(X, O.dct2_matrix(pr.p), rel_tol=1e-3)
    terms = O.tsvdm_kron_terms(res, pr.block_map)
    for C, _ in terms:          # C_i Toeplitz for a Toeplitz map
        for d in range(-5, 6):
            diag = np.diagonal(C, offset=d)
            assert np.ptp(diag) < 1e-14
    K = O.kron_dense(terms)
    assert rel(K, O.M_E(res.tensor_approx(), pr.block_map)) < 1e-13
    U, F, V = O.tsvdm_blr(res)
    assert rel(O.blr_dense(U, F, V, pr.block_map), K) < 1e-13
    x = G.random_rhs(pr.q * pr.n, 3, 0)
    assert rel(O.apply_kron(terms, x), K @ x) < 1e-13
    assert rel(O.apply_blr(U, F, V, pr.block_map, x), K @ x) < 1e-13


def test_tridiagonal_terms_stay_tridiagonal():
    pr = G.block_tridiag_batch(count=1, ell_range=(6, 6), m_choices=(4,), seed_index=3)[0]
    A = pr.dense()
    X = O.T_E(A, pr.block_map, pr.p, pr.m, pr.n)
    t = O.tucker1_blockmode(X, rel_tol=1e-3)
    for C, _ in O.tucker1_kron_terms(t, pr.block_map):
        assert np.all(np.triu(C, 2) == 0) and np.all(np.tril(C, -2) == 0)
    assert t.rank == pr.extra["K"]


# ---------------------------------------------------------------- Tucker family

def test_planted_kronecker_rank_three():
    pr = G.planted_kron_toeplitz()            # 8x8 blocks of 16x16, 3 terms
    A = pr.dense()
    X = O.T_E(A, pr.block_map, pr.p, pr.m, pr.n)
    t = O.tucker1_blockmode(X, rel_tol=1e-6)
    assert t.rank == 3
    assert t.rel_err < 1e-6
    # span{C_j} equals span{T_k} (principal angles ~ 0)
    terms = O.tucker1_kron_terms(t, pr.block_map)
    Cs = np.stack([C.ravel() for C, _ in terms], axis=1)
    Ts = np.stack([O.struct_E([pr.extra["tvals"][k, j] * math.sqrt(O.multiplicities(pr.block_map, pr.p)[j])
                               for j in range(pr.p)], pr.block_map, pr.p).ravel()
                   for k in range(3)], axis=1)
    Qc, _ = np.linalg.qr(Cs)
    Qt, _ = np.linalg.qr(Ts)
    cosines = np.linalg.svd(Qc.T @ Qt, compute_uv=False)
    assert np.min(cosines) > 1 - 1e-12
    assert abs(np.linalg.norm(A - O.kron_dense(terms)) - t.err) < 1e-9 * np.linalg.norm(A)


def test_tucker_exact_multilinear_rank():
    g = np.random.default_rng(8)
    Gc = g.standard_normal((2, 3, 2))
    U1, U2, U3 = (np.linalg.qr(g.standard_normal((d, r)))[0] for d, r in ((6, 2), (5, 3), (7, 2)))
    X = np.einsum("ijk,ai,bj,ck->abc", Gc, U1, U2, U3)
    h = O.hosvd3(X, rel_tol=1e-10)
    assert h.ranks == (2, 3, 2)
    assert h.rel_err < 1e-13


def test_shared_u_spsd_and_trace_identity():
    pr = G.spacetime_covariance(npts=12, T=5, seed_index=1)
    A = pr.dense()
    X = O.T_E(A, pr.block_map, pr.p, pr.m, pr.n)
    su = O.shared_u(X, rank=4)
    Ah = O.M_E(su.tensor_approx(), pr.block_map)
    # Section 5.1: M_E[T] = (I (x) P) A (I (x) P), hence SPSD
    P = su.U @ su.U.T
    IP = np.kron(np.eye(pr.ell), P)
    assert rel(Ah, IP @ A @ IP) < 1e-13
    assert np.min(np.linalg.eigvalsh((Ah + Ah.T) / 2)) > -1e-12 * np.linalg.norm(A, 2)
    assert np.min(np.linalg.eigvalsh(A)) > 0            # the input is SPD
    # Section 6.2 trace identity
    trh = np.trace(Ah)
    assert abs(trh - pr.ell * np.trace(su.U.T @ pr.blocks[0] @ su.U)) < 1e-12 * trh
    rel_tr = O.trace_relerr_shared_u(pr.blocks[0], su.U, pr.ell)
    assert abs(rel_tr - abs(np.trace(A) - trh) / np.trace(A)) < 1e-12
    # Lemma 1 for the shared-U compression
    assert abs(np.linalg.norm(A - Ah) - su.err) < 1e-12 * np.linalg.norm(A)


def test_tucker2_blr_form():
    pr = G.lti_hankel(s=6, d=5, n_in=4, n_out=3, seed_index=2)
    A = pr.dense()
    X = O.T_E(A, pr.block_map, pr.p, pr.m, pr.n)
    t = O.tucker2_rows_cols(X, 2, 3)
    Ah = O.blr_dense(t.U, [t.F[:, :, k] for k in range(pr.p)], t.W, pr.block_map)
    assert rel(Ah, O.M_E(t.tensor_approx(), pr.block_map)) < 1e-13
    assert abs(np.linalg.norm(A - Ah) - t.err) < 1e-12 * np.linalg.norm(A)
    # the Hankel of a d=5 system has mode ranks <= 5 -> exact at full (3, 4)
    t_full = O.tucker2_rows_cols(X, 3, 4)
    assert t_full.rel_err < 1e-13


# ---------------------------------------------------------------- Section 7

def vlp_nearest_kron_error(A, m1, n1, m2, n2):
    """Van Loan-Pitsianis: min ||A - B (x) C||_F via the rearrangement R(A)."""
    R = np.empty((m1 * n1, m2 * n2))
    for i in range(m1):
        for j in range(n1):
            R[i + m1 * j, :] = A[i * m2:(i + 1) * m2, j * n2:(j + 1) * n2].ravel(order="F")
    s = np.linalg.svd(R, compute_uv=False)
    return math.sqrt(np.sum(s[1:] ** 2))


def test_kamm_nagy_bttb_special_case():
    # L = 2, m = n = 1: BTTB with a 2-D PSF; the weighted rank-1 SVD gives the
    # optimal Kronecker approximation among ALL Kronecker products.
    K, half = 9, 2
    s = 2 * half + 1
    g = np.random.default_rng(9)
    Pm = g.random((s, s))
    bm = O.banded_toeplitz_map(K, half)
    eta = O.multiplicities(bm, s).astype(float)
    X = np.sqrt(eta)[:, None] * np.sqrt(eta)[None, :] * Pm.T     # X[i1, i2] = w w P[i2, i1]
    E = O.mapping_matrices(bm, s)
    A = sum(np.kron(E[i1], E[i2]) * X[i1, i2] for i1 in range(s) for i2 in range(s))
    u, sv, vt = np.linalg.svd(X)
    C1 = O.struct_E(list(sv[0] * u[:, 0]), bm, s)
    C2 = O.struct_E(list(vt[0]), bm, s)
    err = np.linalg.norm(A - np.kron(C1, C2))
    assert abs(err - math.sqrt(np.sum(sv[1:] ** 2))) < 1e-12
    assert abs(err - vlp_nearest_kron_error(A, K, K, K, K)) < 1e-10


def test_psf_weighting_and_lemma2():
    K, half = 6, 2
    P = G.gaussian_psf3(support=2 * half + 1, sig=(1.0, 1.5, 2.0))
    A = O.blur_matrix(P, K)
    X = O.psf_tensor(P, K)
    bm = O.banded_toeplitz_map(K, half)
    s = 2 * half + 1
    E = O.mapping_matrices(bm, s)
    Am = sum(np.kron(np.kron(E[i], E[j]), E[k]) * X[i, j, k]
             for i in range(s) for j in range(s) for k in range(s))
    assert rel(Am, A) < 1e-14
    h = O.hosvd3(X, rel_tol=1e-2)
    Gc, C1, C2, C3 = O.multilevel_kron_terms(h, K, half)
    Ah = sum(Gc[a, b, c] * np.kron(np.kron(C1[a], C2[b]), C3[c])
             for a in range(len(C1)) for b in range(len(C2)) for c in range(len(C3)))
    assert abs(np.linalg.norm(A - Ah) - h.err) < 1e-12 * np.linalg.norm(A)
    # the unweighted PSF HOSVD (Nagy-Kilmer) does not transfer its error
    Pz = np.transpose(P, (2, 1, 0))
    hu = O.hosvd3(Pz, ranks=h.ranks)
    w = np.sqrt(O.multiplicities(bm, s).astype(float))
    Xu = np.einsum("i,j,k,ijk->ijk", w, w, w, hu.tensor_approx())
    Ahu = sum(np.kron(np.kron(E[i], E[j]), E[k]) * Xu[i, j, k]
              for i in range(s) for j in range(s) for k in range(s))
    assert abs(np.linalg.norm(A - Ahu) - hu.err) > 1e-6 * np.linalg.norm(A)
    vols = G.random_volumes(2, K)
    y = O.multilevel_apply(Gc, C1, C2, C3, vols)
    yd = np.stack([(Ah @ v.ravel(order="F")).reshape((K, K, K), order="F") for v in vols])
    assert rel(y, yd) < 1e-13


# ---------------------------------------------------------------- Section 5.2 (SPD)

def _spd_case():
    pr = G.spacetime_covariance(npts=12, T=6)
    T = pr.dense()
    assert np.linalg.eigvalsh(T)[0] > 0          # a covariance: SPD
    return pr, T


def test_spd_split_of_block_toeplitz():
    pr, _ = _spd_case()
    k0, inner = O.spd_split(pr.block_map)
    assert k0 == 0 and inner.max() == pr.p - 2
    assert np.all(np.diag(inner) == -1)
    with pytest.raises(ValueError):
        O.spd_split(G.block_diagonal_map(3))      # distinct diagonal blocks


def test_spd_full_rank_reproduces_T():
    pr, T = _spd_case()
    s = O.spd_preserving(T, pr.block_map, pr.p, pr.m, rank=pr.m)
    assert np.linalg.norm(s.dense() - T) <= 1e-12 * np.linalg.norm(T)


def test_spd_every_rank_positive_definite_where_spsd_form_is_singular():
    """The theorem of Section 5.2, against Section 5.1's SPSD construction
    (I (x) P) T (I (x) P) on T itself, which is only semidefinite for r < m."""
    pr, T = _spd_case()
    X = O.T_E(T, pr.block_map, pr.p, pr.m, pr.n)
    for r in range(1, pr.m):
        s = O.spd_preserving(T, pr.block_map, pr.p, pr.m, rank=r)
        ev = np.linalg.eigvalsh(s.dense())
        assert ev[0] > 1e-6 * ev[-1], (r, ev[0])
        su = O.shared_u(X, rank=r)
        ev2 = np.linalg.eigvalsh(O.M_E(su.tensor_approx(), pr.block_map))
        assert abs(ev2[0]) < 1e-10 * ev2[-1], (r, ev2[0])


def test_spd_equals_the_rearranged_form():
    """T_hat = I (x) T_0 + (I (x) L P L^-1)(T - I (x) T_0)(I (x) L^-T P L^T),
    P = U U^T: the identity stated after the theorem of Section 5.2, whose
    right factor is the transpose of the left one (reading R15)."""
    pr, T = _spd_case()
    s = O.spd_preserving(T, pr.block_map, pr.p, pr.m, rank=3)
    L, P = s.L, s.su.U @ s.su.U.T
    Li = np.linalg.inv(L)
    I = np.eye(pr.ell)
    T0 = np.kron(I, L @ L.T)
    alt = T0 + np.kron(I, L @ P @ Li) @ (T - T0) @ np.kron(I, Li.T @ P @ L.T)
    assert np.linalg.norm(s.dense() - alt) <= 1e-12 * np.linalg.norm(T)
    # the factor as printed (L^T P L^-T) does not give the construction
    printed = T0 + np.kron(I, L @ P @ Li) @ (T - T0) @ np.kron(I, L.T @ P @ Li.T)
    assert np.linalg.norm(s.dense() - printed) > 1e-6 * np.linalg.norm(T)


def test_spd_inner_error_is_lemma_1():
    pr, T = _spd_case()
    s = O.spd_preserving(T, pr.block_map, pr.p, pr.m, rel_tol=1e-3)
    A = O.M_E(s.X, s.inner_map)
    e = np.linalg.norm(A - s.inner_approx())
    assert abs(e - s.su.err) <= 1e-12 * np.linalg.norm(A)
    assert s.su.err <= 1e-3 * np.linalg.norm(s.X) * (1 + 1e-12)



# ------------------------------------------- Section 6.3, randomized block-index factor

def test_sketch_with_identity_maps_is_the_deterministic_factor():
    """Omega = I_m, Psi = I_n make the sketch the tensor itself: the same
    subspace, core and error as the deterministic Tucker-1 at that rank."""
    pr = G.planted_kron_toeplitz(ell=6, m=5, terms=3, noise=1e-3, seed_index=3)
    X = O.T_E(pr.dense(), pr.block_map, pr.p, pr.m, pr.n)
    r = 4
    t = O.tucker1_blockmode(X, rank=r)
    s = O.tucker1_blockmode_sketch(X, np.eye(pr.m), np.eye(pr.n), r)
    assert np.allclose(s.V @ s.V.T, t.V @ t.V.T, atol=1e-12)
    assert abs(s.err - t.err) <= 1e-12 * np.linalg.norm(X)
    assert np.allclose(s.tensor_approx(), t.tensor_approx(), atol=1e-12 * np.abs(X).max())


def test_sketch_recovers_a_planted_kronecker_sum_exactly():
    """A noise-free sum of 3 Kronecker products has a rank-3 block-index
    unfolding; Gaussian sketches with s^2 >= 3 keep its row space, so the
    sketched factor spans it and the error vanishes."""
    pr = G.planted_kron_toeplitz(ell=7, m=6, terms=3, noise=0.0, seed_index=4)
    X = O.T_E(pr.dense(), pr.block_map, pr.p, pr.m, pr.n)
    g = np.random.default_rng(11)
    for sk in (2, 3, 5):
        s = O.tucker1_blockmode_sketch(X, g.standard_normal((pr.m, sk)),
                                       g.standard_normal((pr.n, sk)), 3)
        assert s.err <= 1e-12 * np.linalg.norm(X)
        t = O.tucker1_blockmode(X, rank=3)
        assert np.allclose(s.V @ s.V.T, t.V @ t.V.T, atol=1e-10)


def test_sketch_error_is_a_projection_residual_and_not_below_the_optimum():
    """V has orthonormal columns, so the error is the Pythagorean remainder
    sqrt(||X||^2 - ||X x3 V^T||^2); no rank-r factor beats the leading
    singular vectors of the unfolding (Eckart-Young)."""
    pr = G.planted_kron_toeplitz(ell=8, m=6, terms=5, noise=1e-2, seed_index=6)
    X = O.T_E(pr.dense(), pr.block_map, pr.p, pr.m, pr.n)
    g = np.random.default_rng(12)
    for r, sk in ((2, 3), (4, 3), (5, 6)):
        s = O.tucker1_blockmode_sketch(X, g.standard_normal((pr.m, sk)),
                                       g.standard_normal((pr.n, sk)), r)
        assert np.allclose(s.V.T @ s.V, np.eye(r), atol=1e-12)
        pyth = np.sqrt(max(np.sum(X * X) - np.sum(s.G * s.G), 0.0))
        assert abs(s.err - pyth) <= 1e-9 * np.linalg.norm(X)
        assert s.err >= O.tucker1_blockmode(X, rank=r).err * (1 - 1e-12)


# ------------------------------------------- Sections 2.3, 4.1, 5: CP by alternating least squares

def _planted_cp(m, n, p, r, seed, noise=0.0):
    g = np.random.default_rng(seed)
    Xf, Yf, Zf = g.standard_normal((m, r)), g.standard_normal((p, r)), g.standard_normal((n, r))
    X = np.einsum("aj,kj,bj->abk", Xf, Yf, Zf)
    if noise:
        X = X + noise * g.standard_normal(X.shape)
    return X, Xf, Yf, Zf, g


def test_cp_als_recovers_a_planted_kruskal_tensor():
    """An exact rank-3 Kruskal tensor, started near its factors: the fit
    reaches rounding level and the product tensor is the planted one."""
    X, Xf, Yf, Zf, g = _planted_cp(7, 6, 9, 3, 21)
    c = O.cp_als(X, Xf + 0.05 * g.standard_normal(Xf.shape), Zf + 0.05 * g.standard_normal(Zf.shape), 40)
    assert c.err <= 1e-10 * np.linalg.norm(X)
    assert np.allclose(c.tensor_approx(), X, atol=1e-10 * np.abs(X).max())


def test_cp_als_rank_one_is_exact_in_one_iteration():
    """For a rank-1 tensor each least-squares step is exact once the other two
    factors are parallel to the true ones: from the true Xf, Zf one iteration
    reproduces X."""
    X, Xf, Yf, Zf, _ = _planted_cp(5, 4, 6, 1, 22)
    c = O.cp_als(X, 2.0 * Xf, -0.5 * Zf, 1)
    assert c.err <= 1e-12 * np.linalg.norm(X)


def test_cp_als_fit_never_increases():
    """Every ALS step solves its least-squares problem exactly, so the error
    after each iteration is non-increasing."""
    X, _, _, _, g = _planted_cp(8, 7, 10, 4, 23, noise=0.3)
    c = O.cp_als(X, g.standard_normal((8, 3)), g.standard_normal((7, 3)), 25)
    f = np.asarray(c.fit_err)
    assert np.all(np.diff(f) <= 1e-12 * f[0])
    assert c.err == f[-1]


def test_cp_kronecker_sum_and_block_form_equal_M_E():
    """Corollary kronsumcp and Theorem blockCP both reproduce M_E of the
    Kruskal tensor (block Toeplitz map, so the C_j are Toeplitz)."""
    ell, m, n = 5, 4, 3
    bm = G.toeplitz_map(ell)
    p = int(bm.max()) + 1
    X, _, _, _, g = _planted_cp(m, n, p, 3, 24, noise=0.1)
    c = O.cp_als(X, g.standard_normal((m, 2)), g.standard_normal((n, 2)), 5)
    dense = O.M_E(c.tensor_approx(), bm)
    terms = O.cp_kron_terms(c, bm)
    assert np.allclose(O.kron_dense(terms), dense, atol=1e-12 * np.abs(dense).max())
    assert np.allclose(O.cp_blr(c, bm), dense, atol=1e-12 * np.abs(dense).max())
    for C, _ in terms:       # each C_j keeps the block-Toeplitz structure
        assert np.allclose(C[1:, 1:], C[:-1, :-1])


# ------------------------------------------- Section 7 with two levels and m x n blocks

def _two_level(ranks=None, noise=0.0, m=3, n=2):
    map1 = G.symmetric_banded_toeplitz_map(4, 2)   # 4 x 4 block pentadiagonal, block symmetric
    map2 = G.block_diagonal_map(5)                 # 5 x 5 block diagonal
    pr = G.two_level_problem(map1, map2, m, n, ranks=ranks, noise=noise)
    return map1, map2, pr


def test_two_level_running_example_sizes():
    """The example of Section 7.1: 4 x 4 block-pentadiagonal symmetric Toeplitz
    of 5 x 5 block-diagonal blocks is stored as 3 x 5 = 15 distinct m x n
    blocks, a fourth-order m x 3 x 5 x n tensor (ours: m x n x 3 x 5)."""
    map1, map2, pr = _two_level()
    assert (int(map1.max()) + 1, int(map2.max()) + 1) == (3, 5)
    assert pr.p == 15
    X = O.two_level_tensor(pr.dense(), map1, map2, pr.m, pr.n)
    assert X.shape == (pr.m, pr.n, 3, 5)


def test_two_level_map_round_trip_and_product_form():
    """M_E(T_E(A)) = A for an exactly two-level structured A; the tensor is
    the one-level tensor of the product map with the block index split as
    i1 + p1 i2, so the weights multiply (eta = eta1 eta2)."""
    map1, map2, pr = _two_level()
    A = pr.dense()
    X = O.two_level_tensor(A, map1, map2, pr.m, pr.n)
    assert np.allclose(O.two_level_matrix(X, map1, map2), A, atol=1e-13)
    bm = O.product_map(map1, map2)
    assert np.array_equal(bm, pr.block_map)
    X3 = O.T_E(A, bm, pr.p, pr.m, pr.n)
    assert np.allclose(X3, X.reshape(pr.m, pr.n, -1, order="F"), atol=1e-13)
    eta = O.multiplicities(bm, pr.p)
    assert np.array_equal(eta, np.outer(O.multiplicities(map1, 3), O.multiplicities(map2, 5)).ravel(order="F"))


def test_two_level_kron_sum_is_M_E_and_lemma_holds():
    """Section 7.3: the sum over (j1, j2) of struct1 (x) struct2 (x)
    Xf G_j1j2 Zf^T equals M_E of the Tucker tensor, and its Frobenius error
    equals the tensor error (the multilevel Lemma)."""
    map1, map2, pr = _two_level(m=4, n=3)
    A = pr.dense()
    X = O.two_level_tensor(A, map1, map2, pr.m, pr.n)
    h = O.hosvd4(X, ranks=(3, 2, 2, 3))
    dense = O.two_level_matrix(h.tensor_approx(), map1, map2)
    assert np.allclose(O.kron_dense(O.two_level_kron_terms(h, map1, map2)), dense,
                       atol=1e-12 * np.abs(dense).max())
    assert abs(np.linalg.norm(A - dense) - h.err) <= 1e-12 * np.linalg.norm(A)
    assert h.err > 0.1 * np.linalg.norm(X)        # a real truncation


def test_two_level_planted_multilinear_rank_is_exact():
    map1, map2, pr = _two_level(ranks=(2, 2, 2, 3), m=4, n=3)
    X = O.two_level_tensor(pr.dense(), map1, map2, pr.m, pr.n)
    h = O.hosvd4(X, rel_tol=1e-10)
    assert h.ranks == (2, 2, 2, 3)
    assert h.err <= 1e-12 * np.linalg.norm(X)
    full = O.hosvd4(X, ranks=X.shape)
    assert full.err <= 1e-12 * np.linalg.norm(X)


# ------------------------------------------------ truncation helpers, brute force

def test_rank_for_tolerance_is_the_smallest_feasible_rank():
    g = np.random.default_rng(21)
    for trial in range(200):
        n = int(g.integers(1, 9))
        # integer singular values: every square and tail sum is exact
        sig = g.integers(0, 5, size=n).astype(np.float64)
        sq = sig ** 2
        budget = float(g.integers(0, int(sq.sum()) + 2))
        s = np.sort(sq)[::-1]
        feasible = [r for r in range(n + 1) if s[r:].sum() <= budget]
        assert O.rank_for_tolerance(g.permutation(sig), budget) == min(feasible)


def test_representatives_are_first_in_column_major_order():
    g = np.random.default_rng(22)
    for trial in range(50):
        ell, q = int(g.integers(1, 7)), int(g.integers(1, 7))
        p = int(g.integers(1, ell * q + 1))
        bm = np.concatenate([np.arange(p), g.integers(-1, p, size=ell * q - p)])
        bm = g.permutation(bm).reshape(ell, q).astype(np.int32)
        rep = O.representatives(bm, p)
        flat = bm.T.ravel()            # column-major: index b * ell + a
        for k in range(p):
            first = int(np.flatnonzero(flat == k)[0])
            assert rep[k] == (first % ell, first // ell)
            assert bm[rep[k]] == k


def test_truncation_margin_brackets_the_decision():
    """Budgets inside (1 - margin, 1 + margin) times the budget keep the global
    rule's ranks; just past either end the ranks change."""
    g = np.random.default_rng(23)
    checked = 0
    for trial in range(100):
        sig = [np.sort(g.random(int(g.integers(2, 6))))[::-1] for _ in range(3)]
        normX2 = sum(float(np.sum(s ** 2)) for s in sig)
        tol = float(g.uniform(0.05, 0.6))
        ranks = O.truncate_global(sig, tol, normX2)
        margin = O.truncation_margin(sig, ranks, tol, normX2)
        assert margin >= 0
        if not (1e-6 < margin < 0.5):
            continue
        checked += 1
        for f in (1 - 0.9 * margin, 1 + 0.9 * margin):
            assert np.array_equal(O.truncate_global(sig, tol * math.sqrt(f), normX2), ranks)
        moved = [not np.array_equal(O.truncate_global(sig, tol * math.sqrt(f), normX2), ranks)
                 for f in (1 - 1.1 * margin, 1 + 1.1 * margin)]
        assert any(moved)
    assert checked > 20


def test_leading_left_singular_spans_the_top_eigenspace_of_the_gram():
    g = np.random.default_rng(24)
    Y = g.standard_normal((9, 30)) * np.geomspace(1, 1e-3, 9)[:, None]
    ev, Q = np.linalg.eigh(Y @ Y.T)            # ascending
    ev, Q = ev[::-1], Q[:, ::-1]
    for r in (1, 3, 6):
        U, s, rr = O.leading_left_singular(Y, r=r)
        assert rr == r and U.shape == (9, r)
        assert np.allclose(U.T @ U, np.eye(r), atol=1e-12)
        assert np.linalg.norm(U @ U.T - Q[:, :r] @ Q[:, :r].T, 2) < 1e-8
        assert np.allclose(s ** 2, ev, rtol=1e-10, atol=1e-14)
    # budget form: the rank leaves a tail energy within the budget, one less would not
    budget = float(np.sum(ev[4:])) * 1.0001
    U, s, rr = O.leading_left_singular(Y, budget=budget)
    assert rr == 4
