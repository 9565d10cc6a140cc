"""The mixed path's tensor-core matvecs scale each operand by a power of two
into fp16's range (the fp16 two-piece split): inputs far from unit size must
give the same relative accuracy.  A Kronecker-sum matvec (t-SVDM) and a
block-low-rank matvec (shared U) on inputs scaled by 2^40 and 2^-40 (with
right-hand sides scaled the other way and not at all), against the FP64
oracle at the mixed bar.  Powers of two keep the scaled fp32 inputs exact
copies of the unscaled ones."""
import numpy as np
import pytest

from oracle import sma_oracle as O
from sma_inputs import generators as G

from _util import TOL_MIXED, apply, input_matrix, oracle_tensor, rel, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
S = pytest.importorskip("paper_2105_01170_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_01170_gb300 import _build
    _build.build()


@pytest.mark.parametrize("sa", [2.0 ** 40, 2.0 ** -40])
@pytest.mark.parametrize("sx", [1.0, 2.0 ** -30, 2.0 ** 30])
def test_kron_sum_matvec_scaled_inputs(sa, sx):
    g = np.random.default_rng(5)
    bm = G.toeplitz_map(6)
    pr = G.Problem("scaled", g.standard_normal((11, 32, 24)) * sa, bm)
    A = input_matrix(pr, S.SMA_MIXED)
    h = S.Handle([pr], prec=S.SMA_MIXED, rel_tol=1e-3)
    res = h.compress([to_dev(A)])[0]
    assert res["device_status"] == 0
    X = oracle_tensor(A, pr)
    ranks = h.ranks(0)
    ora = O.tsvdm(X, O.dct2_matrix(pr.p), rel_tol=1e-3, ranks=ranks)
    x = (G.random_rhs(pr.q * pr.n, 64, 3) * sx).astype(np.float32).astype(np.float64)
    y = apply(h, pr, x, S.SMA_MIXED)
    yo = O.apply_kron(O.tsvdm_kron_terms(ora, pr.block_map), x)
    assert np.all(np.isfinite(y))
    assert rel(y, yo) < TOL_MIXED
    h.close()


@pytest.mark.parametrize("sa", [2.0 ** 40, 2.0 ** -40])
def test_shared_u_matvec_scaled_inputs(sa):
    pr0 = G.spacetime_covariance(npts=128, T=8, seed_index=2)
    pr = G.Problem("scaled", np.asarray(pr0.blocks) * sa, pr0.block_map)
    A = input_matrix(pr, S.SMA_MIXED)
    h = S.Handle([pr], prec=S.SMA_MIXED, decomp=S.SMA_TUCKER_SHARED_U, fixed_rank=24)
    res = h.compress([to_dev(A)])[0]
    assert res["device_status"] == 0
    X = oracle_tensor(A, pr).astype(np.float32).astype(np.float64)
    su = O.shared_u(X, rank=24)
    Ao = O.M_E(su.tensor_approx(), pr.block_map)
    x = G.random_rhs(pr.q * pr.n, 256, 7).astype(np.float32).astype(np.float64)
    y = apply(h, pr, x, S.SMA_MIXED)
    assert np.all(np.isfinite(y))
    assert rel(y, Ao @ x) < TOL_MIXED
    h.close()
