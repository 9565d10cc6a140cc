"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the FP64 oracle, the tests and the benchmark.  It holds
no arithmetic of the approximation method itself: it draws random numbers,
builds the *user-side* description of a structured block matrix (the distinct
blocks and the integer position map that says which distinct block sits at
which block position) and, for small cases, places the blocks into a dense
array.  Multiplicities, weights, the struct_E gather, the transform, the SVDs
and everything after them are computed separately by the oracle and by the
CUDA path.

Conventions (shared by every consumer):
  * a block matrix A is (ell*m) x (q*n) with ell x q blocks of size m x n;
    block (a, b) (0-based) is A[a*m:(a+1)*m, b*n:(b+1)*n];
  * ``block_map`` is an int32 array of shape (ell, q); entry (a, b) is the
    index k in [0, p) of the distinct block at that position, or -1 for a zero
    block;
  * ``blocks`` is a float64 array of shape (p, m, n): blocks[k] is A_k;
  * every dense array is interpreted column-major (Fortran order) by the C ABI;
    numpy arrays returned here are plain C-ordered ndarrays indexed [row, col].

Seeds: numpy.random.default_rng(2105011700 + config index).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2105011700


def rng_for(cfg_index: int, salt: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + cfg_index + 1000 * salt)


# ---------------------------------------------------------------------------
# position maps (the structure descriptions of Section 3's examples)
# ---------------------------------------------------------------------------

def toeplitz_map(ell: int) -> np.ndarray:
    """Block-Toeplitz position map (Section 3, block-Toeplitz example).

    k = 0..ell-1 is the block on lag d = k below the diagonal (a - b = k);
    k = ell..2ell-2 is the block on lag d = k - ell + 1 above it (b - a).
    """
    bm = np.empty((ell, ell), dtype=np.int32)
    for a in range(ell):
        for b in range(ell):
            d = a - b
            bm[a, b] = d if d >= 0 else ell - 1 - d
    return bm


def hankel_map(s: int) -> np.ndarray:
    """Block-Hankel position map (Section 6.1): block (a, b) holds h_{a+b+1}."""
    a = np.arange(s)[:, None]
    b = np.arange(s)[None, :]
    return (a + b).astype(np.int32)


def block_diagonal_map(ell: int) -> np.ndarray:
    """Block-diagonal position map (Section 3, first example): p = ell."""
    bm = -np.ones((ell, ell), dtype=np.int32)
    for a in range(ell):
        bm[a, a] = a
    return bm


def block_banded_map(ell: int, b: int = 1) -> np.ndarray:
    """Non-symmetric block-banded map with semibandwidth b, distinct blocks
    numbered column-major over the band (b = 1: block tridiagonal, p = 3ell-2,
    the ordering of the tridiagonal example of Section 3 read column by column).
    """
    bm = -np.ones((ell, ell), dtype=np.int32)
    k = 0
    for col in range(ell):
        for row in range(ell):
            if abs(row - col) <= b:
                bm[row, col] = k
                k += 1
    return bm


def symmetric_tridiagonal_map(ell: int) -> np.ndarray:
    """Block-symmetric tridiagonal map as printed in Section 3's example:
    A_1, A_3, A_5, ... on the diagonal and A_2, A_4, ... shared by the two
    off-diagonal positions (a+1, a) and (a, a+1); p = 2ell - 1.  (The shared
    off-diagonal block appears untransposed in both positions, exactly as
    printed.)"""
    bm = -np.ones((ell, ell), dtype=np.int32)
    for a in range(ell):
        bm[a, a] = 2 * a
        if a + 1 < ell:
            bm[a + 1, a] = 2 * a + 1
            bm[a, a + 1] = 2 * a + 1
    return bm


def symmetric_banded_toeplitz_map(ell: int, half: int) -> np.ndarray:
    """Block-symmetric banded Toeplitz map: index |a - b| for |a - b| <= half
    (p = half + 1), the same block above and below the diagonal."""
    bm = -np.ones((ell, ell), dtype=np.int32)
    for a in range(ell):
        for b in range(ell):
            if abs(a - b) <= half:
                bm[a, b] = abs(a - b)
    return bm


def place_blocks(blocks: np.ndarray, block_map: np.ndarray) -> np.ndarray:
    """Dense A with blocks[block_map[a, b]] at block position (a, b)."""
    p, m, n = blocks.shape
    ell, q = block_map.shape
    A = np.zeros((ell * m, q * n), dtype=blocks.dtype)
    for a in range(ell):
        for b in range(q):
            k = int(block_map[a, b])
            if k >= 0:
                A[a * m:(a + 1) * m, b * n:(b + 1) * n] = blocks[k]
    return A


@dataclass
class Problem:
    """One structured block matrix given by its distinct blocks and map."""
    name: str
    blocks: np.ndarray          # (p, m, n) float64
    block_map: np.ndarray       # (ell, q) int32
    extra: dict = field(default_factory=dict)

    @property
    def p(self) -> int:
        return int(self.blocks.shape[0])

    @property
    def m(self) -> int:
        return int(self.blocks.shape[1])

    @property
    def n(self) -> int:
        return int(self.blocks.shape[2])

    @property
    def ell(self) -> int:
        return int(self.block_map.shape[0])

    @property
    def q(self) -> int:
        return int(self.block_map.shape[1])

    def dense(self) -> np.ndarray:
        return place_blocks(self.blocks, self.block_map)


# ---------------------------------------------------------------------------
# workload 1: planted Kronecker sum, block Toeplitz (8x8 blocks of 16x16)
# ---------------------------------------------------------------------------

def planted_kron_toeplitz(ell: int = 8, m: int = 16, terms: int = 3,
                          noise: float = 1e-8, seed_index: int = 0) -> Problem:
    """A = sum_k T_k (x) B_k (+ noise on the distinct blocks).

    T_k: ell x ell Toeplitz with its 2ell-1 defining values N(0,1);
    B_k: m x m N(0,1).  Noise N(0,1)*noise is added to each of the 2ell-1
    distinct blocks, so A stays exactly block Toeplitz.
    """
    g = rng_for(seed_index)
    p = 2 * ell - 1
    tvals = g.standard_normal((terms, p))       # value per lag index k
    B = g.standard_normal((terms, m, m))
    blocks = np.einsum("tk,tij->kij", tvals, B)
    if noise:
        blocks = blocks + noise * g.standard_normal(blocks.shape)
    return Problem("planted_kron_toeplitz", blocks, toeplitz_map(ell),
                   {"tvals": tvals, "B": B, "terms": terms, "noise": noise})


# ---------------------------------------------------------------------------
# workload 2: space-time covariance (Gneiting class), block Toeplitz in time
# ---------------------------------------------------------------------------

def gneiting(h: np.ndarray, u: float, rng_: float = 0.3, tscale: float = 5.0,
             beta: float = 0.5) -> np.ndarray:
    """Non-separable space-time covariance of the Gneiting (2002) class,
    d = 2, alpha = 1, gamma = 1/2, tau = d/2:
        psi(u) = 1 + (u/tscale)^2,
        C(h, u) = psi^-1 * exp(-|h| / (rng_ * psi^(beta/2))).
    """
    psi = 1.0 + (u / tscale) ** 2
    return np.exp(-h / (rng_ * psi ** (beta / 2.0))) / psi


def spacetime_covariance(npts: int = 256, T: int = 64, seed_index: int = 1,
                         symmetric_map: bool = False) -> Problem:
    """Block Toeplitz-in-time covariance; blocks C_u (npts x npts) at time lag
    u, points uniform in the unit square.  Non-symmetric Toeplitz map (p =
    2T-1) unless symmetric_map (then p = T with the same block above and below
    the diagonal, which is exact here because every block is symmetric)."""
    g = rng_for(seed_index)
    pts = g.random((npts, 2))
    h = np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    lag_blocks = np.stack([gneiting(h, float(u)) for u in range(T)])
    if symmetric_map:
        bm = np.empty((T, T), dtype=np.int32)
        for a in range(T):
            for b in range(T):
                bm[a, b] = abs(a - b)
        blocks = lag_blocks
    else:
        bm = toeplitz_map(T)
        blocks = np.concatenate([lag_blocks, lag_blocks[1:]], axis=0)
    return Problem("spacetime_covariance", np.ascontiguousarray(blocks), bm,
                   {"points": pts, "T": T})


# ---------------------------------------------------------------------------
# workload 3: system identification block Hankel
# ---------------------------------------------------------------------------

def lti_hankel(s: int = 64, d: int = 40, n_in: int = 32, n_out: int = 32,
               rho: float = 0.95, seed_index: int = 2) -> Problem:
    """Markov parameters h_k = C A^(k-1) B, k = 1..2s-1, of a random stable
    LTI system; block Hankel with s x s blocks of n_out x n_in."""
    g = rng_for(seed_index)
    A = g.standard_normal((d, d))
    A *= rho / np.max(np.abs(np.linalg.eigvals(A)))
    B = g.standard_normal((d, n_in))
    C = g.standard_normal((n_out, d))
    blocks = np.empty((2 * s - 1, n_out, n_in))
    P = np.eye(d)
    for k in range(2 * s - 1):
        blocks[k] = C @ P @ B
        P = P @ A
    return Problem("lti_hankel", blocks, hankel_map(s), {"A": A, "B": B, "C": C})


# ---------------------------------------------------------------------------
# workload 4: batched uneven block-tridiagonal matrices
# ---------------------------------------------------------------------------

def block_tridiag_batch(count: int = 512, ell_range=(16, 256),
                        m_choices=(8, 16, 32, 64), kmax_range=(2, 6),
                        noise: float = 1e-4, drop: float = 0.3,
                        seed_index: int = 3) -> list[Problem]:
    """Block-tridiagonal matrices whose nonzero blocks are
    sum_{k<K} c_k(i,j) (P o D_k) + noise, with one Bernoulli(drop) zero
    pattern P per matrix applied after the noise."""
    g = rng_for(seed_index)
    out = []
    for idx in range(count):
        ell = int(g.integers(ell_range[0], ell_range[1] + 1))
        m = int(m_choices[int(g.integers(0, len(m_choices)))])
        K = int(g.integers(kmax_range[0], kmax_range[1] + 1))
        out.append(_tridiag_problem(g, f"tridiag_{idx}", ell, m, K, noise, drop))
    return out


def _tridiag_problem(g: np.random.Generator, name: str, ell: int, m: int, K: int,
                     noise: float, drop: float) -> Problem:
    bm = block_banded_map(ell, 1)
    p = int(bm.max()) + 1
    D = g.standard_normal((K, m, m))
    c = g.standard_normal((p, K))
    blocks = np.einsum("pk,kij->pij", c, D) + noise * g.standard_normal((p, m, m))
    mask = (g.random((m, m)) >= drop).astype(np.float64)
    blocks *= mask[None]
    return Problem(name, blocks, bm, {"K": K, "mask": mask})


def block_tridiag_kron(ell: int, m: int, K: int = 5, noise: float = 1e-4, drop: float = 0.3,
                       seed_index: int = 3, salt: int = 6) -> Problem:
    """One block-tridiagonal matrix of the batched workload's kind with chosen
    sizes (ell blocks of m x m, Kron rank K): the stand-in for the largest
    SuiteSparse matrix of the Kronecker-sum table, compressed there with the
    randomized block-index factor."""
    return _tridiag_problem(rng_for(seed_index, salt=salt), f"tridiag_{ell}x{m}", ell, m, K,
                            noise, drop)


# ---------------------------------------------------------------------------
# workload 5: anisotropic 3-D Gaussian PSF (3-level banded Toeplitz)
# ---------------------------------------------------------------------------

def gaussian_psf3(support: int = 15, sig=(2.0, 3.0, 4.0),
                  rot_deg: float = 30.0) -> np.ndarray:
    """PSF P[ix, iy, iz] on a support^3 grid centred at 0, covariance
    R diag(sig^2) R^T with R a rotation about z; normalised to sum 1."""
    c = support // 2
    t = math.radians(rot_deg)
    R = np.array([[math.cos(t), -math.sin(t), 0.0],
                  [math.sin(t), math.cos(t), 0.0],
                  [0.0, 0.0, 1.0]])
    S = R @ np.diag(np.square(sig)) @ R.T
    Si = np.linalg.inv(S)
    ax = np.arange(support) - c
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    v = np.stack([X, Y, Z], -1)
    q = np.einsum("...i,ij,...j->...", v, Si, v)
    P = np.exp(-0.5 * q)
    return P / P.sum()


def random_volumes(count: int, K: int, seed_index: int = 4) -> np.ndarray:
    g = rng_for(seed_index, salt=1)
    return g.standard_normal((count, K, K, K))


def random_rhs(rows: int, nrhs: int, seed_index: int, salt: int = 2) -> np.ndarray:
    """nrhs right-hand sides of length rows, N(0,1); shape (rows, nrhs)."""
    g = rng_for(seed_index, salt=salt)
    return g.standard_normal((rows, nrhs))


def random_orthogonal(p: int, seed_index: int, salt: int = 3) -> np.ndarray:
    """A Haar-random orthogonal p x p matrix (for user-supplied transforms)."""
    g = rng_for(seed_index, salt=salt)
    Q, R = np.linalg.qr(g.standard_normal((p, p)))
    return Q * np.sign(np.diag(R))[None, :]


def gaussian_sketch(m: int, n: int, s: int, seed_index: int = 7,
                    salt: int = 5) -> tuple[np.ndarray, np.ndarray]:
    """Independent N(0,1) maps Omega (m x s) and Psi (n x s) for the
    randomized block-index factor (Section 6.3)."""
    g = rng_for(seed_index, salt=salt)
    return g.standard_normal((m, s)), g.standard_normal((n, s))


def planted_cp_toeplitz(ell: int = 8, m: int = 12, n: int = 10, r: int = 3,
                        noise: float = 0.0, seed_index: int = 10,
                        salt: int = 7) -> tuple[Problem, dict]:
    """Block-Toeplitz matrix whose weighted block tensor is an exact rank-r
    Kruskal tensor (plus optional noise): block k = Xf diag(Yf[k, :]) Zf^T /
    sqrt(eta_k), so X[:, :, k] = sqrt(eta_k) A_k = Xf diag(Yf[k, :]) Zf^T.
    Returns the problem and the planted factors."""
    g = rng_for(seed_index, salt=salt)
    bm = toeplitz_map(ell)
    p = 2 * ell - 1
    eta = np.zeros(p)
    for k in bm.ravel():
        eta[k] += 1
    Xf, Yf, Zf = g.standard_normal((m, r)), g.standard_normal((p, r)), g.standard_normal((n, r))
    X = np.einsum("aj,kj,bj->kab", Xf, Yf, Zf)
    if noise:
        X = X + noise * g.standard_normal(X.shape)
    blocks = X / np.sqrt(eta)[:, None, None]
    return Problem("planted_cp_toeplitz", blocks, bm, {"r": r}), {"Xf": Xf, "Yf": Yf, "Zf": Zf}


def cp_initial_factors(m: int, n: int, r: int, seed_index: int = 11,
                       salt: int = 8) -> tuple[np.ndarray, np.ndarray]:
    """N(0,1) starting factors Xf (m x r) and Zf (n x r) for CP-ALS."""
    g = rng_for(seed_index, salt=salt)
    return g.standard_normal((m, r)), g.standard_normal((n, r))


def two_level_problem(map1: np.ndarray, map2: np.ndarray, m: int, n: int, ranks=None,
                      noise: float = 0.0, seed_index: int = 12, salt: int = 9) -> Problem:
    """A two-level structured matrix (Section 7.1): level 1 outermost, the
    distinct m x n blocks A^(i1,i2) listed in the order i1 + p1 i2 over the
    one-level product map (block row a1 ell2 + a2, column b1 q2 + b2).  With
    ranks = (kx, kz, k1, k2) the weighted block tensor
    X[:, :, i1, i2] = sqrt(eta1 eta2) A^(i1,i2) has that multilinear rank
    (N(0,1) core and factors) plus optional noise; otherwise the blocks are
    N(0,1)."""
    g = rng_for(seed_index, salt=salt)
    l1, q1 = map1.shape
    l2, q2 = map2.shape
    p1, p2 = int(map1.max()) + 1, int(map2.max()) + 1
    eta1 = np.bincount(map1[map1 >= 0].ravel(), minlength=p1).astype(np.float64)
    eta2 = np.bincount(map2[map2 >= 0].ravel(), minlength=p2).astype(np.float64)
    if ranks is None:
        X = g.standard_normal((m, n, p1, p2))
    else:
        kx, kz, k1, k2 = ranks
        G = g.standard_normal((kx, kz, k1, k2))
        fs = [g.standard_normal((d, k)) for d, k in ((m, kx), (n, kz), (p1, k1), (p2, k2))]
        X = np.einsum("xzij,ax,bz,ci,dj->abcd", G, *fs)
    if noise:
        X = X + noise * g.standard_normal(X.shape)
    w = np.sqrt(np.outer(eta1, eta2))                      # [i1, i2]
    A = X / w[None, None, :, :]
    blocks = np.stack([A[:, :, i1, i2] for i2 in range(p2) for i1 in range(p1)])
    bm = -np.ones((l1 * l2, q1 * q2), dtype=np.int32)
    for a1 in range(l1):
        for b1 in range(q1):
            for a2 in range(l2):
                for b2 in range(q2):
                    i1, i2 = map1[a1, b1], map2[a2, b2]
                    if i1 >= 0 and i2 >= 0:
                        bm[a1 * l2 + a2, b1 * q2 + b2] = i1 + p1 * i2
    return Problem("two_level", blocks, bm, {"map1": map1, "map2": map2, "p1": p1, "p2": p2})


def planted_tsvdm_tensor(m: int, n: int, p: int, ranks, seed_index: int = 9,
                         salt: int = 4) -> tuple[np.ndarray, list]:
    """Random factors for a tensor whose transform-domain slices have given
    ranks: returns (Lfac, Rfac) lists with slice i = Lfac[i] @ Rfac[i]."""
    g = rng_for(seed_index, salt=salt)
    L = [g.standard_normal((m, r)) for r in ranks]
    Rf = [g.standard_normal((r, n)) for r in ranks]
    return L, Rf
