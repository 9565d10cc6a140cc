"""Shared helpers for the parity tests: run a problem through the C ABI and
through the FP64 oracle on the same seeded input."""
from __future__ import annotations

import math

import numpy as np

from oracle import sma_oracle as O
from sma_inputs import generators as G

# Tolerances (relative Frobenius) of the two precisions against the oracle.
TOL_FP64 = 1e-10
TOL_MIXED = 1e-5


def tol_for(prec):
    import paper_2105_01170_gb300 as S
    return TOL_FP64 if prec == S.SMA_FP64 else TOL_MIXED


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def input_matrix(pr: G.Problem, prec) -> np.ndarray:
    """The dense input in the precision the path takes (fp64 / fp32)."""
    import paper_2105_01170_gb300 as S
    A = pr.dense()
    return A if prec == S.SMA_FP64 else A.astype(np.float32)


def oracle_tensor(A_in: np.ndarray, pr: G.Problem) -> np.ndarray:
    return O.T_E(np.asarray(A_in, dtype=np.float64), pr.block_map, pr.p, pr.m, pr.n)


def to_dev(a: np.ndarray, dtype=None):
    import torch
    t = torch.from_numpy(np.asfortranarray(a))
    if dtype is not None:
        t = t.to(dtype)
    t = t.cuda()
    if t.dim() == 2:
        return t.t().contiguous().t()
    return t


def from_dev_colmajor(t, shape):
    """Column-major device buffer -> numpy array of `shape` (Fortran order)."""
    return t.detach().cpu().numpy().reshape(shape, order="F")


def torch_dtype(prec):
    import torch
    import paper_2105_01170_gb300 as S
    return torch.float64 if prec == S.SMA_FP64 else torch.float32


def np_dtype(prec):
    import paper_2105_01170_gb300 as S
    return np.float64 if prec == S.SMA_FP64 else np.float32


def gpu_tensor(h, which, shape, prec, i=0):
    """Export an intermediate tensor of problem i as a numpy array."""
    import torch
    import paper_2105_01170_gb300 as S
    n = h.export_size(i, which)
    dt = torch.float64 if (which == S.EXPORT_SIGMA or prec == S.SMA_FP64) else torch.float32
    buf = torch.empty(n, dtype=dt, device="cuda")
    h.export(i, which, buf)
    arr = buf.cpu().numpy().astype(np.float64)
    if shape is None:
        return arr
    return arr.reshape(shape, order="F")


def reconstruct(h, pr: G.Problem, prec, i=0):
    import torch
    rows, cols = pr.ell * pr.m, pr.q * pr.n
    Ah = torch.empty(cols, rows, dtype=torch_dtype(prec), device="cuda").t()
    h.reconstruct(i, Ah)
    return Ah.cpu().numpy().astype(np.float64)


def apply(h, pr: G.Problem, x: np.ndarray, prec, i=0):
    import torch
    X = to_dev(x.astype(np_dtype(prec)))
    Y = torch.empty(x.shape[1], pr.ell * pr.m, dtype=torch_dtype(prec), device="cuda").t()
    h.apply(i, X, Y)
    return Y.cpu().numpy().astype(np.float64)


# Every case where the mixed path's retained ranks differed from the oracle's
# (allowed only where the oracle's own decision margin is below the fp32
# perturbation); the test session prints the list in its summary.
RANK_WINDOW_HITS: list = []


def rank_window_ok(gpu_ranks, ora, rel_tol, normX2, perturb):
    """Ranks must match the oracle exactly when the oracle's decision has a
    margin larger than `perturb` (relative to the budget); otherwise the GPU
    decision must itself satisfy the tolerance and stay within the window."""
    margin = O.truncation_margin(ora.sigma, ora.ranks, rel_tol, normX2)
    if margin > perturb:
        return np.array_equal(np.asarray(gpu_ranks), np.asarray(ora.ranks)), margin
    return abs(int(np.sum(gpu_ranks)) - int(np.sum(ora.ranks))) <= max(
        8, int(0.01 * np.sum(ora.ranks))), margin


def oracle_at_gpu_ranks(gpu_ranks, ora, X, M, rel_tol, prec, where, perturb=0.2):
    """Check the GPU's retained ranks against the oracle's and return the
    oracle result that the GPU's T, M_E[T] and matvec are compared with,
    element by element, in every case.

    Identical ranks: the oracle's own truncation.  Otherwise (mixed path only,
    and only where the oracle's decision margin is below `perturb` of the
    budget, so that fp32 rounding of the energies can move the decision): the
    GPU's decision must itself meet the tolerance on the oracle's singular
    values, and the comparison is against the oracle truncated at the GPU's
    ranks (the same truncation done in fp64).  Such cases are recorded in
    RANK_WINDOW_HITS."""
    import paper_2105_01170_gb300 as S
    gpu_ranks = np.asarray(gpu_ranks, dtype=np.int64)
    if np.array_equal(gpu_ranks, np.asarray(ora.ranks)):
        return ora
    assert prec != S.SMA_FP64, (where, "fp64 ranks differ from the oracle's")
    ok, margin = rank_window_ok(gpu_ranks, ora, rel_tol, ora.normX ** 2, perturb)
    assert ok, (where, int(gpu_ranks.sum()), int(np.sum(ora.ranks)), margin)
    disc = sum(float(np.sum(np.sort(s)[::-1][r:] ** 2)) for s, r in zip(ora.sigma, gpu_ranks))
    budget = rel_tol * rel_tol * ora.normX ** 2
    assert disc <= (1.0 + perturb) * budget, (where, disc, budget)
    RANK_WINDOW_HITS.append(f"{where}: total rank {int(gpu_ranks.sum())} vs oracle "
                            f"{int(np.sum(ora.ranks))} (oracle decision margin {margin:.2e})")
    return O.tsvdm(X, M, ranks=gpu_ranks)
