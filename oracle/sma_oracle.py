"""FP64 CPU oracle for the structured-matrix-approximation hot path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this module; the library itself never
does, and this module imports nothing from the library.

It is a plain, slow, direct transcription of the definitions of
Kilmer & Saibaba, "Structured Matrix Approximations via Tensor Decompositions"
(arXiv 2105.01170), in float64 with numpy.  The per-slice and per-unfolding
SVDs are LAPACK's (numpy.linalg.svd), used as a library step.

Orientation.  The paper stores the mapped tensor as m x p x n with the
distinct-block index in mode 2 (Section 3).  Here it is stored frontal-slice,
X of shape (m, n, p) with X[:, :, k] = sqrt(eta_k) A_k: the paper's mode 2 is
our mode 3, its modes 1 and 3 (block rows / block columns) are our modes 1 and 2.

Readings of points the paper leaves open (each also listed in the design notes):
  R1  representative occurrence of block k: smallest column-major block index
      b*ell + a among the positions with block_map == k;
  R2  tensor-to-matrix map M_E uses struct_E without the sqrt(eta) factor
      (Section 3 definition of M_E), so C_j = sum_k v_kj E_k;
  R3  t-SVDM (not defined in the paper; Kernfeld-Kilmer-Aeron M-product):
      Xhat = X x3 M, SVD of every frontal slice, truncation, T = That x3 M^T;
  R4  tolerance truncation is global over all slices: sort every singular
      value descending (ties: slice ascending, index ascending) and keep the
      shortest prefix whose discarded energy sum sigma^2 <= tol^2 ||X||_F^2;
      fixed rank keeps min(rank, m, n) per slice;
  R5  HOSVD with t truncated modes gives each mode the budget tol^2||X||^2/t;
  R6  eq. (blockTuck) sums j = 1..r2 (the printed upper limit ell is a typo);
  R7  orthonormal DCT-II: M[k, j] = a_k cos(pi (2j+1) k / (2p)),
      a_0 = sqrt(1/p), a_k = sqrt(2/p);
  R15 Section 5.2: T_0 is the one distinct block on the whole diagonal; the
      tolerance of the SPD-preserving form applies to the tensor of
      A = sum_k E_k (x) L^-1 T_k L^-T; in the rearranged form printed after
      the theorem the right factor is (I (x) L^-T P L^T), the transpose of the
      left one (as printed, L^T P L^-T, the result would not be symmetric).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# ---------------------------------------------------------------------------
# Section 3: E_k, eta_k, struct_E, T_E and M_E
# ---------------------------------------------------------------------------


def multiplicities(block_map: np.ndarray, p: int) -> np.ndarray:
    """eta_k = number of block positions holding A_k (Section 3)."""
    eta = np.zeros(p, dtype=np.int64)
    for k in block_map.ravel():
        if k >= 0:
            eta[int(k)] += 1
    if np.any(eta == 0):
        raise ValueError("block_map does not cover every k in [0, p)")
    return eta


def mapping_matrices(block_map: np.ndarray, p: int) -> list[np.ndarray]:
    """E_k in R^{ell x q}: 1/sqrt(eta_k) where A_k occurs, else 0 (Section 3)."""
    eta = multiplicities(block_map, p)
    ell, q = block_map.shape
    E = [np.zeros((ell, q)) for _ in range(p)]
    for a in range(ell):
        for b in range(q):
            k = int(block_map[a, b])
            if k >= 0:
                E[k][a, b] = 1.0 / math.sqrt(eta[k])
    return E


def representatives(block_map: np.ndarray, p: int) -> list[tuple[int, int]]:
    """Reading R1: occurrence of A_k with the smallest column-major index."""
    ell, q = block_map.shape
    rep: list = [None] * p
    for b in range(q):
        for a in range(ell):
            k = int(block_map[a, b])
            if k >= 0 and rep[k] is None:
                rep[k] = (a, b)
    return rep


def block(A: np.ndarray, a: int, b: int, m: int, n: int) -> np.ndarray:
    return A[a * m:(a + 1) * m, b * n:(b + 1) * n]


def struct_E(coeffs, block_map: np.ndarray, p: int) -> np.ndarray:
    """struct_E((K_k)) = sum_k E_k (x) K_k for matrices K_k (reading R2), or
    sum_k K_k E_k for scalars K_k (Theorem 'tuckerkron')."""
    E = mapping_matrices(block_map, p)
    first = np.asarray(coeffs[0])
    if first.ndim == 0:
        return sum(float(coeffs[k]) * E[k] for k in range(p))
    return sum(np.kron(E[k], np.asarray(coeffs[k])) for k in range(p))


def T_E(A: np.ndarray, block_map: np.ndarray, p: int, m: int, n: int) -> np.ndarray:
    """Matrix-to-tensor map of Section 3: slice k = sqrt(eta_k) A_k."""
    eta = multiplicities(block_map, p)
    rep = representatives(block_map, p)
    X = np.empty((m, n, p))
    for k in range(p):
        a, b = rep[k]
        X[:, :, k] = math.sqrt(eta[k]) * block(A, a, b, m, n)
    return X


def T_E_adjoint(A: np.ndarray, block_map: np.ndarray, p: int, m: int, n: int) -> np.ndarray:
    """Adjoint of M_E: slice k = sum over occurrences of A_k of A_ij/sqrt(eta_k)
    (the orthogonal projection of a possibly unstructured A onto the class)."""
    eta = multiplicities(block_map, p)
    X = np.zeros((m, n, p))
    ell, q = block_map.shape
    for a in range(ell):
        for b in range(q):
            k = int(block_map[a, b])
            if k >= 0:
                X[:, :, k] += block(A, a, b, m, n) / math.sqrt(eta[k])
    return X


def M_E(X: np.ndarray, block_map: np.ndarray) -> np.ndarray:
    """Tensor-to-matrix map of Section 3: sum_k E_k (x) X[:, :, k]."""
    p = X.shape[2]
    return struct_E([X[:, :, k] for k in range(p)], block_map, p)


# ---------------------------------------------------------------------------
# the transform M and mode products
# ---------------------------------------------------------------------------


def dct2_matrix(p: int) -> np.ndarray:
    """Reading R7: orthonormal DCT-II matrix."""
    M = np.empty((p, p))
    for k in range(p):
        a = math.sqrt(1.0 / p) if k == 0 else math.sqrt(2.0 / p)
        for j in range(p):
            M[k, j] = a * math.cos(math.pi * (2 * j + 1) * k / (2 * p))
    return M


def mode3(X: np.ndarray, M: np.ndarray) -> np.ndarray:
    """X x3 M: out[:, :, i] = sum_k M[i, k] X[:, :, k] (Section 2.1 mode product)."""
    return np.einsum("abk,ik->abi", X, M, optimize=True)


def unfold(X: np.ndarray, mode: int) -> np.ndarray:
    """Mode unfoldings of an (m, n, p) tensor in our orientation:
    mode 1: m x (n p) = [X_1, ..., X_p];  mode 2: n x (m p) = [X_1^T, ...];
    mode 3: p x (m n), row k = vec(X[:, :, k]) (column-major vec)."""
    m, n, p = X.shape
    if mode == 1:
        return np.concatenate([X[:, :, k] for k in range(p)], axis=1)
    if mode == 2:
        return np.concatenate([X[:, :, k].T for k in range(p)], axis=1)
    if mode == 3:
        return np.stack([X[:, :, k].ravel(order="F") for k in range(p)], axis=0)
    raise ValueError(mode)


# ---------------------------------------------------------------------------
# truncation rules
# ---------------------------------------------------------------------------


def truncate_global(sigmas: list[np.ndarray], rel_tol: float, normX2: float) -> np.ndarray:
    """Reading R4: ranks per slice for the global tolerance rule.

    sigmas[i] holds the singular values of slice i (any order).  Returns the
    number of retained values per slice; the retained ones are the largest of
    each slice."""
    budget = rel_tol * rel_tol * normX2
    items = []
    for i, s in enumerate(sigmas):
        for j, v in enumerate(np.sort(np.asarray(s, dtype=np.float64))[::-1]):
            items.append((float(v), i, j))
    # ascending by (sigma, slice desc, index desc) == reverse of the keep order
    items.sort(key=lambda t: (t[0], -t[1], -t[2]))
    discarded = 0.0
    ndisc = 0
    for v, _, _ in items:
        if discarded + v * v <= budget:
            discarded += v * v
            ndisc += 1
        else:
            break
    ranks = np.array([len(s) for s in sigmas], dtype=np.int64)
    for v, i, _ in items[:ndisc]:
        ranks[i] -= 1
    return ranks


def rank_for_tolerance(sig: np.ndarray, budget: float) -> int:
    """Smallest r with sum_{j >= r} sig_j^2 <= budget (sig sorted descending)."""
    sig = np.sort(np.asarray(sig, dtype=np.float64))[::-1]
    tail = 0.0
    r = len(sig)
    while r > 0 and tail + sig[r - 1] ** 2 <= budget:
        tail += sig[r - 1] ** 2
        r -= 1
    return r


def truncation_margin(sigmas: list[np.ndarray], ranks, rel_tol: float, normX2: float) -> float:
    """Relative slack of a global-tolerance decision: min over the two
    constraints (discarded energy below budget; one more discard above it),
    divided by the budget.  A perturbation of the energies smaller than
    margin*budget cannot change the retained ranks."""
    budget = rel_tol * rel_tol * normX2
    disc = 0.0
    nxt = math.inf
    for s, r in zip(sigmas, ranks):
        s = np.sort(np.asarray(s))[::-1]
        disc += float(np.sum(s[r:] ** 2))
        if r > 0:
            nxt = min(nxt, float(s[r - 1] ** 2))
    if budget <= 0:
        return 0.0
    lo = (budget - disc) / budget
    hi = (disc + nxt - budget) / budget if math.isfinite(nxt) else math.inf
    return min(lo, hi)


# ---------------------------------------------------------------------------
# step 2: t-SVDM (reading R3)
# ---------------------------------------------------------------------------


@dataclass
class TSVDM:
    M: np.ndarray                 # p x p orthogonal transform
    U: list                       # per slice, m x rho_i
    S: list                       # per slice, rho_i singular values
    V: list                       # per slice, n x rho_i
    sigma: list                   # per slice, all singular values (desc)
    ranks: np.ndarray
    normX: float
    err: float                    # sqrt(discarded energy) = ||X - T||_F
    rel_err: float

    def slice_factor(self, i: int) -> np.ndarray:
        return (self.U[i] * self.S[i][None, :]) @ self.V[i].T

    def transformed_approx(self) -> np.ndarray:
        return np.stack([self.slice_factor(i) for i in range(len(self.U))], axis=2)

    def tensor_approx(self) -> np.ndarray:
        """T = (oplus_i U_i S_i V_i^T) x3 M^T."""
        return mode3(self.transformed_approx(), self.M.T)


def tsvdm(X: np.ndarray, M: np.ndarray, rel_tol: float | None = None,
          fixed_rank: int | None = None, ranks=None) -> TSVDM:
    """t-SVDM of X (reading R3).  The retained rank of each slice comes from
    exactly one of: `ranks` (a given per-slice rank vector, each entry in
    [0, min(m, n)]: the truncation of every slice at that rank), `fixed_rank`
    (min(fixed_rank, m, n) per slice), or the global tolerance rule R4 at
    `rel_tol`."""
    m, n, p = X.shape
    Xh = mode3(X, M)
    normX2 = float(np.sum(X * X))
    Us, Ss, Vs = [], [], []
    for i in range(p):
        u, s, vt = np.linalg.svd(Xh[:, :, i], full_matrices=False)
        Us.append(u)
        Ss.append(s)
        Vs.append(vt.T)
    if ranks is not None:
        ranks = np.asarray(ranks, dtype=np.int64).ravel()
        if ranks.shape != (p,) or np.any(ranks < 0) or np.any(ranks > min(m, n)):
            raise ValueError("ranks must hold one rank in [0, min(m, n)] per slice")
        ranks = ranks.copy()
    elif fixed_rank is not None and fixed_rank > 0:
        ranks = np.array([min(fixed_rank, len(s)) for s in Ss], dtype=np.int64)
    else:
        ranks = truncate_global(Ss, float(rel_tol or 0.0), normX2)
    disc = sum(float(np.sum(Ss[i][ranks[i]:] ** 2)) for i in range(p))
    err = math.sqrt(disc)
    return TSVDM(M=M, U=[Us[i][:, :ranks[i]] for i in range(p)],
                 S=[Ss[i][:ranks[i]] for i in range(p)],
                 V=[Vs[i][:, :ranks[i]] for i in range(p)], sigma=Ss,
                 ranks=ranks, normX=math.sqrt(normX2), err=err,
                 rel_err=err / math.sqrt(normX2) if normX2 > 0 else 0.0)


# ---------------------------------------------------------------------------
# step 3: map back (Kronecker sum, block low rank)
# ---------------------------------------------------------------------------


def tsvdm_kron_terms(res: TSVDM, block_map: np.ndarray) -> list[tuple[np.ndarray, np.ndarray]]:
    """A_hat = M_E[T] = sum_i struct_E(M[i, :]) (x) U_i S_i V_i^T, one term per
    slice with rho_i > 0 (follows from T[:,:,k] = sum_i M[i,k] Xhat_i and the
    definition of M_E, as in the proof of Theorem 'tuckerkron')."""
    p = res.M.shape[0]
    terms = []
    for i in range(p):
        if res.ranks[i] == 0:
            continue
        C = struct_E(list(res.M[i, :]), block_map, p)
        terms.append((C, res.slice_factor(i)))
    return terms


def tsvdm_blr(res: TSVDM) -> tuple[np.ndarray, list, np.ndarray]:
    """Block-low-rank form A_hat = (I (x) Ut) struct_E(F_k) (I (x) Vt^T) with
    Ut = [U_1 | ... | U_p], Vt = [V_1 | ... | V_p] and F_k the diagonal matrix
    blkdiag_i(M[i, k] S_i) (the t-SVDM analogue of eq. (blockCP))."""
    p = res.M.shape[0]
    Ut = np.concatenate([res.U[i] for i in range(p)], axis=1)
    Vt = np.concatenate([res.V[i] for i in range(p)], axis=1)
    F = []
    for k in range(p):
        F.append(np.diag(np.concatenate([res.M[i, k] * res.S[i] for i in range(p)])))
    return Ut, F, Vt


def blr_dense(U: np.ndarray, F: list, W: np.ndarray, block_map: np.ndarray) -> np.ndarray:
    """(I_ell (x) U) struct_E(F_k) (I_q (x) W^T) (eq. (blockTuck) form)."""
    ell, q = block_map.shape
    p = len(F)
    mid = struct_E(F, block_map, p)
    return np.kron(np.eye(ell), U) @ mid @ np.kron(np.eye(q), W.T)


def apply_M_E(T: np.ndarray, block_map: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = M_E[T] x block by block, without forming M_E[T]: block (a, b) of
    M_E[T] is T[:, :, k] / sqrt(eta_k) for k = block_map[a, b] (Section 3,
    M_E = sum_k E_k (x) T_k), zero where block_map is -1.  x: (q*n, nrhs)."""
    m, n, p = T.shape
    ell, q = block_map.shape
    eta = multiplicities(block_map, p)
    y = np.zeros((ell * m, x.shape[1]))
    for b in range(q):
        xb = x[b * n:(b + 1) * n, :]
        for a in range(ell):
            k = int(block_map[a, b])
            if k >= 0:
                y[a * m:(a + 1) * m, :] += (T[:, :, k] / math.sqrt(eta[k])) @ xb
    return y


def kron_dense(terms) -> np.ndarray:
    return sum(np.kron(C, D) for C, D in terms)


# ---------------------------------------------------------------------------
# step 4: apply
# ---------------------------------------------------------------------------


def apply_kron(terms, x: np.ndarray) -> np.ndarray:
    """y = sum_j (C_j (x) D_j) x via vec(D X C^T) = (C (x) D) vec(X) (Section
    2.2, property 1).  x: (q*n, nrhs); returns (ell*m, nrhs)."""
    C0, D0 = terms[0]
    ell, q = C0.shape
    m, n = D0.shape
    nrhs = x.shape[1]
    Y = np.zeros((ell * m, nrhs))
    for s in range(nrhs):
        Xs = x[:, s].reshape((n, q), order="F")
        Ys = np.zeros((m, ell))
        for C, D in terms:
            Ys += D @ Xs @ C.T
        Y[:, s] = Ys.ravel(order="F")
    return Y


def apply_blr(U: np.ndarray, F: list, W: np.ndarray, block_map: np.ndarray,
              x: np.ndarray) -> np.ndarray:
    """y = (I (x) U) struct_E(F_k) (I (x) W^T) x, block by block."""
    ell, q = block_map.shape
    p = len(F)
    eta = multiplicities(block_map, p)
    m, n = U.shape[0], W.shape[0]
    nrhs = x.shape[1]
    Y = np.zeros((ell * m, nrhs))
    z = [W.T @ x[b * n:(b + 1) * n, :] for b in range(q)]
    for a in range(ell):
        acc = np.zeros((U.shape[1], nrhs))
        for b in range(q):
            k = int(block_map[a, b])
            if k >= 0:
                acc += (F[k] @ z[b]) / math.sqrt(eta[k])
        Y[a * m:(a + 1) * m, :] = U @ acc
    return Y


# ---------------------------------------------------------------------------
# Tucker / HOSVD variants (Sections 2.4, 4.2, 5.1, 6.2, 6.3)
# ---------------------------------------------------------------------------


def leading_left_singular(Y: np.ndarray, r: int | None = None,
                          budget: float | None = None) -> tuple[np.ndarray, np.ndarray, int]:
    """Leading left singular vectors of an unfolding (HOSVD factor, Section 2.4)."""
    u, s, _ = np.linalg.svd(Y, full_matrices=False)
    if r is None:
        r = rank_for_tolerance(s, float(budget or 0.0))
    r = min(r, len(s))
    return u[:, :r], s, r


@dataclass
class Tucker1Block:
    V: np.ndarray          # p x r
    G: np.ndarray          # m x n x r, G = X x3 V^T
    sigma: np.ndarray      # singular values of the block-index unfolding
    rank: int
    err: float
    rel_err: float

    def tensor_approx(self) -> np.ndarray:
        return mode3(self.G, self.V)


def tucker1_blockmode(X: np.ndarray, rel_tol: float | None = None,
                      rank: int | None = None) -> Tucker1Block:
    """Section 6.3: T = G x2 V, G = X x2 V^T with V the leading left singular
    vectors of the block-index unfolding (our mode 3)."""
    normX2 = float(np.sum(X * X))
    Y = unfold(X, 3)
    V, s, r = leading_left_singular(Y, rank, (rel_tol or 0.0) ** 2 * normX2)
    G = mode3(X, V.T)
    err = math.sqrt(max(float(np.sum(s[r:] ** 2)), 0.0))
    return Tucker1Block(V, G, s, r, err, err / math.sqrt(normX2))


def tucker1_blockmode_sketch(X: np.ndarray, Omega: np.ndarray, Psi: np.ndarray,
                             rank: int) -> Tucker1Block:
    """Section 6.3, the randomized variant used for the largest matrix of the
    Kronecker-sum experiment: V is taken from the block-index unfolding of the
    sketch Y = X x1 Omega^T x2 Psi^T (our orientation: Y[:, :, k] =
    Omega^T X[:, :, k] Psi, Omega m x s and Psi n x s Gaussian, passed in),
    keeping `rank` leading left singular vectors; the rest is the Tucker-1
    compression of X itself, G = X x3 V^T.  The error is ||X - G x3 V||_F,
    measured directly (the sketch's singular values are not those of X)."""
    normX2 = float(np.sum(X * X))
    Ysk = np.einsum("ai,abk,bj->ijk", Omega, X, Psi, optimize=True)
    V, s, r = leading_left_singular(unfold(Ysk, 3), rank)
    G = mode3(X, V.T)
    err = float(np.linalg.norm((X - mode3(G, V)).ravel()))
    return Tucker1Block(V, G, s, r, err, err / math.sqrt(normX2))


def tucker1_kron_terms(t: Tucker1Block, block_map: np.ndarray):
    """A_hat = sum_j struct_E(V[:, j]) (x) sq(G_:,j,:) (Section 6.3 / Theorem
    'tuckerkron' with U, W identities)."""
    p = t.V.shape[0]
    return [(struct_E(list(t.V[:, j]), block_map, p), t.G[:, :, j]) for j in range(t.rank)]


# ---------------------------------------------------------------------------
# CP (Kruskal) compressor: Sections 2.3, 4.1 (Theorem tildeA, Corollary
# kronsumcp) and 5 (Theorem blockCP)
# ---------------------------------------------------------------------------


@dataclass
class CPModel:
    Xf: np.ndarray         # m x r
    Yf: np.ndarray         # p x r (block index)
    Zf: np.ndarray         # n x r
    fit_err: list          # ||X - T||_F after each iteration
    err: float
    rel_err: float

    def tensor_approx(self) -> np.ndarray:
        """Frontal slice k of the Kruskal tensor: Xf diag(Yf[k, :]) Zf^T."""
        return np.einsum("aj,kj,bj->abk", self.Xf, self.Yf, self.Zf, optimize=True)


def cp_als(X: np.ndarray, Xf0: np.ndarray, Zf0: np.ndarray, iters: int) -> CPModel:
    """CP by alternating least squares (the method the paper points to for
    Section 2.3's decomposition): each factor in turn is the least-squares
    solution with the other two fixed, through the normal equations whose
    matrix is the Hadamard product of the other two factors' Gram matrices.
    Our orientation: slice k of X (m x n x p) is approximated by
    Xf diag(Yf[k, :]) Zf^T.  Order within an iteration: Yf (from the given
    Xf, Zf), then Xf, then Zf; the initial Xf, Zf are inputs, there is no
    column normalisation, and `iters` iterations are run."""
    Xf, Zf = Xf0.astype(np.float64).copy(), Zf0.astype(np.float64).copy()
    m, n, p = X.shape
    fit = []
    Yf = None
    for _ in range(iters):
        # Yf[k, j] = sum_ab X[a, b, k] Xf[a, j] Zf[b, j], then (Xf^T Xf * Zf^T Zf)^-1
        M3 = np.einsum("abk,aj,bj->kj", X, Xf, Zf, optimize=True)
        Yf = np.linalg.solve((Xf.T @ Xf) * (Zf.T @ Zf), M3.T).T
        M1 = np.einsum("abk,bj,kj->aj", X, Zf, Yf, optimize=True)
        Xf = np.linalg.solve((Zf.T @ Zf) * (Yf.T @ Yf), M1.T).T
        M2 = np.einsum("abk,aj,kj->bj", X, Xf, Yf, optimize=True)
        Zf = np.linalg.solve((Xf.T @ Xf) * (Yf.T @ Yf), M2.T).T
        T = np.einsum("aj,kj,bj->abk", Xf, Yf, Zf, optimize=True)
        fit.append(float(np.linalg.norm((X - T).ravel())))
    normX = float(np.linalg.norm(X.ravel()))
    return CPModel(Xf, Yf, Zf, fit, fit[-1], fit[-1] / normX)


def cp_kron_terms(c: CPModel, block_map: np.ndarray):
    """Corollary kronsumcp with F = Yf, G = I: A_hat = sum_j struct_E(Yf[:, j])
    (x) Xf[:, j] Zf[:, j]^T."""
    p = c.Yf.shape[0]
    return [(struct_E(list(c.Yf[:, j]), block_map, p), np.outer(c.Xf[:, j], c.Zf[:, j]))
            for j in range(c.Yf.shape[1])]


def cp_blr(c: CPModel, block_map: np.ndarray) -> np.ndarray:
    """Theorem blockCP: (I (x) Q_X) struct_E(F_k) (I (x) Q_Z^T), Xf = Q_X R_X,
    Zf = Q_Z R_Z thin QR, F_k = R_X diag(Yf[k, :]) R_Z^T (dense, for checks)."""
    QX, RX = np.linalg.qr(c.Xf)
    QZ, RZ = np.linalg.qr(c.Zf)
    p = c.Yf.shape[0]
    F = [RX @ np.diag(c.Yf[k]) @ RZ.T for k in range(p)]
    ell, q = block_map.shape
    return np.kron(np.eye(ell), QX) @ struct_E(F, block_map, p) @ np.kron(np.eye(q), QZ).T


@dataclass
class SharedU:
    U: np.ndarray          # m x r
    G: np.ndarray          # r x r x p core slices U^T X_k U
    sigma: np.ndarray      # singular values of the mode-1 unfolding
    rank: int
    err: float
    rel_err: float

    def tensor_approx(self) -> np.ndarray:
        return np.einsum("ai,ijk,bj->abk", self.U, self.G, self.U, optimize=True)


def shared_u(X: np.ndarray, rel_tol: float | None = None, rank: int | None = None) -> SharedU:
    """Section 5.1 / 6.2: two-sided compression T = G x1 U x2 U with U from the
    mode-1 unfolding (the two truncated modes share the budget, reading R5)."""
    normX2 = float(np.sum(X * X))
    U, s, r = leading_left_singular(unfold(X, 1), rank, (rel_tol or 0.0) ** 2 * normX2 / 2.0)
    G = np.einsum("ai,abk,bj->ijk", U, X, U, optimize=True)
    T = np.einsum("ai,ijk,bj->abk", U, G, U, optimize=True)
    err = float(np.linalg.norm((X - T).ravel()))
    return SharedU(U, G, s, r, err, err / math.sqrt(normX2))


# ---------------------------------------------------------------------------
# Section 5.2: preserving positive definiteness
# ---------------------------------------------------------------------------

@dataclass
class SPDApprox:
    k0: int                  # block index of the diagonal block T_0
    L: np.ndarray            # T_0 = L L^T (lower triangular, m x m)
    inner_map: np.ndarray    # map of A = sum_k E_k (x) A_k: T_0's positions empty, 0..p-2
    X: np.ndarray            # tensor of A: X[:, :, k'] = sqrt(eta_k') L^-1 T_k L^-T
    su: SharedU              # shared-U compression of X (Section 5.1)

    def inner_approx(self) -> np.ndarray:
        """M_E of the compressed tensor: the approximation of A."""
        return M_E(self.su.tensor_approx(), self.inner_map)

    def dense(self) -> np.ndarray:
        """T_hat = (I (x) L) (I + M_E[T]) (I (x) L^T)."""
        ell = self.inner_map.shape[0]
        B = np.kron(np.eye(ell), self.L)
        return B @ (np.eye(B.shape[0]) + self.inner_approx()) @ B.T


def spd_split(block_map: np.ndarray) -> tuple[int, np.ndarray]:
    """Section 5.2 writes T = I (x) T_0 + sum_k E_k (x) T_k: the block index k0
    that fills the whole diagonal (and nothing else), and the map of the
    remaining blocks renumbered 0..p-2 with T_0's positions empty."""
    ell = block_map.shape[0]
    diag = {int(block_map[a, a]) for a in range(ell)}
    if len(diag) != 1 or min(diag) < 0:
        raise ValueError("the diagonal blocks are not one distinct block")
    k0 = diag.pop()
    off = [(a, b) for a in range(ell) for b in range(block_map.shape[1])
           if a != b and block_map[a, b] == k0]
    if off:
        raise ValueError("the diagonal block also occurs off the diagonal")
    inner = np.where(block_map == k0, -1, np.where(block_map > k0, block_map - 1, block_map))
    return k0, inner.astype(block_map.dtype)


def spd_preserving(A: np.ndarray, block_map: np.ndarray, p: int, m: int,
                   rel_tol: float | None = None, rank: int | None = None) -> SPDApprox:
    """Section 5.2: Cholesky T_0 = L L^T of the diagonal block, A_k = L^-1 T_k
    L^-T for the other distinct blocks, the shared-U compression of the tensor
    of A = sum_k E_k (x) A_k (the tolerance applies to that tensor), and
    T_hat = (I (x) L)(I + M_E[T])(I (x) L^T), which is SPD when T is."""
    k0, inner = spd_split(block_map)
    reps = representatives(block_map, p)
    L = np.linalg.cholesky(block(A, *reps[k0], m, m))
    Linv = np.linalg.solve(L, np.eye(m))
    pin = p - 1
    eta = multiplicities(inner, pin)
    X = np.empty((m, m, pin))
    for k in range(p):
        if k == k0:
            continue
        kk = k - 1 if k > k0 else k
        X[:, :, kk] = math.sqrt(eta[kk]) * (Linv @ block(A, *reps[k], m, m) @ Linv.T)
    return SPDApprox(k0, L, inner, X, shared_u(X, rel_tol, rank))


@dataclass
class Tucker2:
    U: np.ndarray          # m x r1
    W: np.ndarray          # n x r3
    F: np.ndarray          # r1 x r3 x p, F_k = U^T X_k W
    err: float
    rel_err: float

    def tensor_approx(self) -> np.ndarray:
        return np.einsum("ai,ijk,bj->abk", self.U, self.F, self.W, optimize=True)


def tucker2_rows_cols(X: np.ndarray, r1: int, r3: int) -> Tucker2:
    """Eq. (blockTuck) with V = I: U from mode 1, W from mode 2 (ours)."""
    normX2 = float(np.sum(X * X))
    U, _, _ = leading_left_singular(unfold(X, 1), r1)
    W, _, _ = leading_left_singular(unfold(X, 2), r3)
    F = np.einsum("ai,abk,bj->ijk", U, X, W, optimize=True)
    T = np.einsum("ai,ijk,bj->abk", U, F, W, optimize=True)
    err = float(np.linalg.norm((X - T).ravel()))
    return Tucker2(U, W, F, err, err / math.sqrt(normX2))


@dataclass
class HOSVD3:
    factors: list          # [U1 (d1 x k1), U2, U3]
    G: np.ndarray          # k1 x k2 x k3 core
    sigmas: list
    ranks: tuple
    err: float
    rel_err: float

    def tensor_approx(self) -> np.ndarray:
        U1, U2, U3 = self.factors
        return np.einsum("ijk,ai,bj,ck->abc", self.G, U1, U2, U3, optimize=True)


def hosvd3(X: np.ndarray, rel_tol: float | None = None, ranks=None) -> HOSVD3:
    """Truncated HOSVD of a third-order tensor (Section 2.4) with each of the
    three modes given the budget tol^2 ||X||^2 / 3 (reading R5)."""
    normX2 = float(np.sum(X * X))
    budget = (rel_tol or 0.0) ** 2 * normX2 / 3.0
    d1, d2, d3 = X.shape
    Y1 = X.reshape(d1, -1)
    Y2 = np.moveaxis(X, 1, 0).reshape(d2, -1)
    Y3 = np.moveaxis(X, 2, 0).reshape(d3, -1)
    facs, sig, rk = [], [], []
    for t, Y in enumerate((Y1, Y2, Y3)):
        U, s, r = leading_left_singular(Y, None if ranks is None else ranks[t], budget)
        facs.append(U)
        sig.append(s)
        rk.append(r)
    G = np.einsum("abc,ai,bj,ck->ijk", X, *facs, optimize=True)
    T = np.einsum("ijk,ai,bj,ck->abc", G, *facs, optimize=True)
    err = float(np.linalg.norm((X - T).ravel()))
    return HOSVD3(facs, G, sig, tuple(rk), err, err / math.sqrt(normX2))


# ---------------------------------------------------------------------------
# Section 7: multilevel (three-level Toeplitz PSF with m = n = 1)
# ---------------------------------------------------------------------------


def banded_toeplitz_map(K: int, half: int) -> np.ndarray:
    """Scalar Toeplitz map of a K x K matrix with bandwidth `half`:
    entry (a, b) holds PSF index d = a - b + half when |a - b| <= half."""
    bm = -np.ones((K, K), dtype=np.int32)
    for a in range(K):
        for b in range(K):
            if abs(a - b) <= half:
                bm[a, b] = a - b + half
    return bm


def psf_tensor(P: np.ndarray, K: int) -> np.ndarray:
    """Section 7.5: X[i1, i2, i3] = sqrt(eta_i1 eta_i2 eta_i3) P[i3, i2, i1],
    level 1 the outermost (z) axis, P indexed [x, y, z]."""
    s = P.shape[0]
    half = s // 2
    eta = multiplicities(banded_toeplitz_map(K, half), s).astype(np.float64)
    w = np.sqrt(eta)
    return np.einsum("i,j,k,kji->ijk", w, w, w, P, optimize=True)


def blur_matrix(P: np.ndarray, K: int) -> np.ndarray:
    """Dense 3-level Toeplitz blur (zero boundary) on a K^3 volume, vec order
    x fastest: A = sum_{i1,i2,i3} E_i1 (x) E_i2 (x) E_i3 (x) sqrt(eta..) X..
    written out directly from the PSF (small K only)."""
    s = P.shape[0]
    half = s // 2
    N = K ** 3
    A = np.zeros((N, N))
    for z in range(K):
        for y in range(K):
            for x in range(K):
                r = x + K * (y + K * z)
                for dz in range(-half, half + 1):
                    for dy in range(-half, half + 1):
                        for dx in range(-half, half + 1):
                            zz, yy, xx = z - dz, y - dy, x - dx
                            if 0 <= zz < K and 0 <= yy < K and 0 <= xx < K:
                                c = xx + K * (yy + K * zz)
                                A[r, c] = P[dx + half, dy + half, dz + half]
    return A


def multilevel_kron_terms(h: HOSVD3, K: int, half: int):
    """Section 7.5: A_hat = sum_j G_j struct1(U[:, j1]) (x) struct2(V[:, j2])
    (x) struct3(W[:, j3]); returns (G, [C1 list], [C2 list], [C3 list])."""
    bm = banded_toeplitz_map(K, half)
    s = 2 * half + 1
    U1, U2, U3 = h.factors
    C1 = [struct_E(list(U1[:, j]), bm, s) for j in range(U1.shape[1])]
    C2 = [struct_E(list(U2[:, j]), bm, s) for j in range(U2.shape[1])]
    C3 = [struct_E(list(U3[:, j]), bm, s) for j in range(U3.shape[1])]
    return h.G, C1, C2, C3


def multilevel_apply(G, C1, C2, C3, vols: np.ndarray) -> np.ndarray:
    """y = sum_j G_j (C1_j1 (x) C2_j2 (x) C3_j3) vec(x) for volumes vols[b, x, y, z]
    (vec order x fastest, so C3 acts on x, C2 on y, C1 on z)."""
    out = np.zeros_like(vols)
    for j1 in range(len(C1)):
        for j2 in range(len(C2)):
            for j3 in range(len(C3)):
                g = G[j1, j2, j3]
                out += g * np.einsum("zc,yb,xa,nabc->nxyz", C1[j1], C2[j2], C3[j3], vols, optimize=True)
    return out


# ---------------------------------------------------------------------------
# step 5: reports
# ---------------------------------------------------------------------------


# ---------------------------------------------------------------------------
# Section 7 with two levels and m x n blocks: the (L+2)-order tensor
# ---------------------------------------------------------------------------


def product_map(map1: np.ndarray, map2: np.ndarray) -> np.ndarray:
    """The two-level structure sum_{i1,i2} E1_i1 (x) E2_i2 (x) A^(i1,i2) as a
    one-level map: level 1 outermost, so block row a1 ell2 + a2 and block
    column b1 q2 + b2 hold block index i1 + p1 i2 (-1 where either level is
    empty).  The weights multiply: eta = eta1_i1 eta2_i2."""
    l1, q1 = map1.shape
    l2, q2 = map2.shape
    p1 = int(map1.max()) + 1
    out = -np.ones((l1 * l2, q1 * q2), dtype=np.int32)
    for a1 in range(l1):
        for b1 in range(q1):
            i1 = int(map1[a1, b1])
            if i1 < 0:
                continue
            for a2 in range(l2):
                for b2 in range(q2):
                    i2 = int(map2[a2, b2])
                    if i2 >= 0:
                        out[a1 * l2 + a2, b1 * q2 + b2] = i1 + p1 * i2
    return out


def two_level_tensor(A: np.ndarray, map1: np.ndarray, map2: np.ndarray, m: int,
                     n: int) -> np.ndarray:
    """Section 7.1: the (L+2)-order tensor of a two-level structured matrix,
    X[:, :, i1, i2] = sqrt(eta1_i1 eta2_i2) A^(i1,i2) (m x n x p1 x p2; the
    paper's m x p1 x p2 x n with the block kept as the first two modes)."""
    p1, p2 = int(map1.max()) + 1, int(map2.max()) + 1
    eta1, eta2 = multiplicities(map1, p1), multiplicities(map2, p2)
    X = np.empty((m, n, p1, p2))
    for i1 in range(p1):
        a1, b1 = representatives(map1, p1)[i1]
        for i2 in range(p2):
            a2, b2 = representatives(map2, p2)[i2]
            blk = block(A, a1 * map2.shape[0] + a2, b1 * map2.shape[1] + b2, m, n)
            X[:, :, i1, i2] = math.sqrt(eta1[i1] * eta2[i2]) * blk
    return X


def two_level_matrix(X: np.ndarray, map1: np.ndarray, map2: np.ndarray) -> np.ndarray:
    """M_E of Section 7.1: sum_{i1,i2} E1_i1 (x) E2_i2 (x) X[:, :, i1, i2]."""
    p1, p2 = X.shape[2], X.shape[3]
    E1, E2 = mapping_matrices(map1, p1), mapping_matrices(map2, p2)
    return sum(np.kron(np.kron(E1[i1], E2[i2]), X[:, :, i1, i2])
               for i1 in range(p1) for i2 in range(p2))


@dataclass
class HOSVD4:
    factors: list          # [Xf (m x kx), Zf (n x kz), Y1 (p1 x k1), Y2 (p2 x k2)]
    G: np.ndarray          # kx x kz x k1 x k2
    ranks: tuple
    err: float
    rel_err: float

    def tensor_approx(self) -> np.ndarray:
        Xf, Zf, Y1, Y2 = self.factors
        return np.einsum("xzij,ax,bz,ci,dj->abcd", self.G, Xf, Zf, Y1, Y2, optimize=True)


def hosvd4(X: np.ndarray, rel_tol: float | None = None, ranks=None) -> HOSVD4:
    """Truncated HOSVD of the fourth-order tensor (eq. multiTX with L = 2):
    each factor holds leading left singular vectors of its unfolding; with a
    tolerance every one of the four modes gets tol^2 ||X||^2 / 4 (reading R5)."""
    normX2 = float(np.sum(X * X))
    budget = (rel_tol or 0.0) ** 2 * normX2 / 4.0
    facs, rk = [], []
    for t in range(4):
        Y = np.moveaxis(X, t, 0).reshape(X.shape[t], -1)
        U, _, r = leading_left_singular(Y, None if ranks is None else ranks[t], budget)
        facs.append(U)
        rk.append(r)
    G = np.einsum("abcd,ax,bz,ci,dj->xzij", X, *facs, optimize=True)
    h = HOSVD4(facs, G, tuple(rk), 0.0, 0.0)
    err = float(np.linalg.norm((X - h.tensor_approx()).ravel()))
    h.err, h.rel_err = err, err / math.sqrt(normX2)
    return h


def two_level_kron_terms(h: HOSVD4, map1: np.ndarray, map2: np.ndarray):
    """Section 7.3: sum_{j1,j2} struct1(Y1[:, j1]) (x) struct2(Y2[:, j2]) (x)
    Xf G[:, :, j1, j2] Zf^T, as (C, D) pairs with C the Kronecker product of
    the two level structures."""
    Xf, Zf, Y1, Y2 = h.factors
    p1, p2 = Y1.shape[0], Y2.shape[0]
    terms = []
    for j2 in range(Y2.shape[1]):
        for j1 in range(Y1.shape[1]):
            C = np.kron(struct_E(list(Y1[:, j1]), map1, p1), struct_E(list(Y2[:, j2]), map2, p2))
            terms.append((C, Xf @ h.G[:, :, j1, j2] @ Zf.T))
    return terms


def fro(A: np.ndarray) -> float:
    return float(np.linalg.norm(np.asarray(A).ravel()))


def storage_ratio_blr(N: int, T: int, r: int) -> float:
    """Section 6.2: (r^2 T + N r) / (N^2 T)."""
    return (r * r * T + N * r) / (N * N * T)


def trace_relerr_shared_u(blocks_diag: np.ndarray, U: np.ndarray, T: int) -> float:
    """Section 6.2: |tr C - tr C_hat| / tr C with tr C_hat = T tr(U^T C_1 U)."""
    trC = T * float(np.trace(blocks_diag))
    trCh = T * float(np.trace(U.T @ blocks_diag @ U))
    return abs(trC - trCh) / trC


def greedy_structure(A: np.ndarray, ell: int, q: int, m: int, n: int) -> np.ndarray:
    """Section 3's greedy discovery of distinct blocks (O((ell q)^2) block
    comparisons); zero blocks map to -1.  Used only as a brute-force check."""
    bm = -np.ones((ell, q), dtype=np.int32)
    distinct: list[np.ndarray] = []
    for b in range(q):
        for a in range(ell):
            B = block(A, a, b, m, n)
            if not np.any(B):
                continue
            for k, D in enumerate(distinct):
                if np.array_equal(B, D):
                    bm[a, b] = k
                    break
            else:
                bm[a, b] = len(distinct)
                distinct.append(B.copy())
    return bm
