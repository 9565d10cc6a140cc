"""GPU parity of the three-level path (Section 7: weighted PSF tensor of a
3-D blur, truncated HOSVD, sum of structured triple Kronecker products)
against the FP64 oracle."""
import numpy as np
import pytest

from oracle import sma_oracle as O
from sma_inputs import generators as G

from _util import TOL_MIXED, rel, to_dev

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


def setup(K, half, sig, prec, tol):
    P = G.gaussian_psf3(support=2 * half + 1, sig=sig)
    s = 2 * half + 1
    bm = O.banded_toeplitz_map(K, half)
    # distinct scalars a^(i1,i2,i3) = P[i3, i2, i1] (Section 7.5), order i1 fastest
    a = np.transpose(P, (2, 1, 0)).ravel(order="F")
    dt = np.float64 if prec == S.SMA_FP64 else np.float32
    a = a.astype(dt)
    pr = S.MultilevelProblem([bm, bm, bm], [s, s, s])
    h = S.Handle([pr], prec=prec, decomp=S.SMA_HOSVD_MULTILEVEL, layout=S.SMA_INPUT_BLOCKS,
                 rel_tol=tol)
    res = h.compress([to_dev(a)])[0]
    Pin = np.transpose(a.astype(np.float64).reshape((s, s, s), order="F"), (2, 1, 0))
    X = O.psf_tensor(Pin, K)
    return h, res, X, Pin, bm, s


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_multilevel_small_dense(prec):
    K, half, tol = 9, 2, 1e-3
    h, res, X, Pin, bm, s = setup(K, half, (1.0, 1.5, 2.0), prec, tol)
    ho = O.hosvd3(X, rel_tol=tol)
    assert tuple(res["ranks"][:3]) == ho.ranks
    assert list(h.ranks(0)) == list(ho.ranks)
    floor = (1e-13 if prec == S.SMA_FP64 else TOL_MIXED) * np.linalg.norm(X)
    assert abs(res["tensor_err"] - ho.err) <= 1e-6 * ho.err + floor
    # the dense approximation against the oracle's triple Kronecker sum
    Gc, C1, C2, C3 = O.multilevel_kron_terms(ho, K, half)
    Ao = sum(Gc[i, j, k] * np.kron(np.kron(C1[i], C2[j]), C3[k])
             for i in range(len(C1)) for j in range(len(C2)) for k in range(len(C3)))
    N = K ** 3
    Ah = torch.empty(N, N, dtype=torch.float64 if prec == S.SMA_FP64 else torch.float32,
                     device="cuda").t()
    h.reconstruct(0, Ah)
    Ah = Ah.cpu().numpy().astype(np.float64)
    tolp = 1e-10 if prec == S.SMA_FP64 else TOL_MIXED
    assert rel(Ah, Ao) < tolp
    # Lemma 2 against the dense blur operator
    A = O.blur_matrix(Pin, K)
    assert abs(np.linalg.norm(A - Ah) - res["tensor_err"]) <= tolp * np.linalg.norm(A)
    # the matvec on two volumes
    vols = G.random_volumes(2, K)
    x = np.stack([v.ravel(order="F") for v in vols], axis=1)
    dt = torch.float64 if prec == S.SMA_FP64 else torch.float32
    Xd = to_dev(x.astype(np.float64 if prec == S.SMA_FP64 else np.float32))
    Yd = torch.empty(2, N, dtype=dt, device="cuda").t()
    h.apply(0, Xd, Yd)
    y = Yd.cpu().numpy().astype(np.float64)
    assert rel(y, Ao @ x) < tolp


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_multilevel_full_psf(prec):
    """64^3 volume, 15^3 PSF (sigma 2, 3, 4, rotated 30 degrees), tol 1e-4."""
    K, half, tol = 64, 7, 1e-4
    h, res, X, Pin, bm, s = setup(K, half, (2.0, 3.0, 4.0), prec, tol)
    ho = O.hosvd3(X, rel_tol=tol)
    assert tuple(res["ranks"][:3]) == ho.ranks == (1, 6, 6)
    floor = (1e-13 if prec == S.SMA_FP64 else TOL_MIXED) * np.linalg.norm(X)
    assert abs(res["tensor_err"] - ho.err) <= 1e-6 * ho.err + floor
    Gc, C1, C2, C3 = O.multilevel_kron_terms(ho, K, half)
    vols = G.random_volumes(2, K)
    yo = O.multilevel_apply(Gc, C1, C2, C3, vols)
    x = np.stack([v.ravel(order="F") for v in vols], axis=1)
    dt = torch.float64 if prec == S.SMA_FP64 else torch.float32
    Xd = to_dev(x.astype(np.float64 if prec == S.SMA_FP64 else np.float32))
    Yd = torch.empty(2, K ** 3, dtype=dt, device="cuda").t()
    h.apply(0, Xd, Yd)
    y = Yd.cpu().numpy().astype(np.float64)
    yo2 = np.stack([v.ravel(order="F") for v in yo], axis=1)
    assert rel(y, yo2) < (1e-10 if prec == S.SMA_FP64 else TOL_MIXED)
