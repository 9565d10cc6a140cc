"""The allocation-free slice SVD (sma_slice_svd_noalloc).

It exists for callers that cannot call cudaMalloc where they need the work
done (an inference-engine plugin's execution callback, a loop whose device
memory another allocator budgeted up front) and so cannot create a handle:
its scratch lives in a fixed device array inside the library.  The test calls
it through the C ABI on the transformed slices produced by the handle path
(sma_compress) and checks, twice in a row, that its singular values match the
handle path's and that its factors rebuild the slices, with the tolerances the
other parity tests use.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from sma_inputs import generators as G

from _util import TOL_MIXED, rel, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
S = pytest.importorskip("paper_2105_01170_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_01170_gb300 import _build
    _build.build()


def handle_path(m, n, p, seed):
    """Transformed slices and their singular values from sma_compress."""
    g = np.random.default_rng(seed)
    pr = G.Problem("noalloc", g.standard_normal((p, m, n)), G.block_diagonal_map(p))
    A = pr.dense().astype(np.float32)
    h = S.Handle([pr], prec=S.SMA_MIXED, rel_tol=1e-6)
    h.compress([to_dev(A)])
    Xh = torch.empty(m * n * p, dtype=torch.float32, device="cuda")
    h.export(0, S.EXPORT_XHAT, Xh)
    rc = min(m, n)
    sig = torch.empty(rc * p, dtype=torch.float64, device="cuda")
    h.export(0, S.EXPORT_SIGMA, sig)
    h.close()
    return Xh, sig.cpu().numpy().reshape((rc, p), order="F")


def call_noalloc(Xh, m, n, p):
    mm, rc = max(m, n), min(m, n)
    W = torch.full((mm * rc * p,), float("nan"), dtype=torch.float32, device="cuda")
    V = torch.full((rc * rc * p,), float("nan"), dtype=torch.float32, device="cuda")
    sig = torch.zeros(rc * p, dtype=torch.float64, device="cuda")
    sweeps = torch.zeros(p, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = S.sma_slice_svd_noalloc(Xh.data_ptr(), m, n, p, W.data_ptr(), V.data_ptr(),
                                 sig.data_ptr(), sweeps.data_ptr(), status.data_ptr(), 0, stream)
    assert st == S.SMA_OK, S.sma_status_string(st)
    torch.cuda.synchronize()
    return (W.cpu().numpy().reshape((mm, rc, p), order="F"),
            V.cpu().numpy().reshape((rc, rc, p), order="F"),
            sig.cpu().numpy().reshape((rc, p), order="F"), sweeps.cpu().numpy(),
            int(status.item()))


@pytest.mark.parametrize("m,n,p", [(256, 256, 20),   # block mode: scratch used, two chunks
                                   (6, 11, 9)])      # transposed, fits in shared memory
def test_noalloc_matches_handle_path_twice(m, n, p):
    Xh, sig_ref = handle_path(m, n, p, seed=7)
    X = Xh.cpu().numpy().astype(np.float64).reshape((m, n, p), order="F")
    smax = float(sig_ref.max())
    for _ in range(2):                      # the second call reuses the scratch
        W, V, sig, sweeps, status = call_noalloc(Xh, m, n, p)
        assert status == 0
        assert np.all(sweeps > 0)
        assert np.max(np.abs(sig - sig_ref)) <= 2e-5 * smax
        for k in range(p):
            Wk, Vk = W[:, :, k].astype(np.float64), V[:, :, k].astype(np.float64)
            R = Wk @ Vk.T if m >= n else Vk @ Wk.T
            assert rel(R, X[:, :, k]) < TOL_MIXED
            assert np.allclose(np.linalg.norm(Wk, axis=0), sig[:, k], rtol=1e-5, atol=0)


def test_noalloc_rejects_oversized_slice_and_bad_args():
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    ptr = buf.data_ptr()
    # a 1024 x 1024 slice needs (1024 + 1024) * 1024 floats > the 8 MiB scratch
    assert S.sma_slice_svd_noalloc(ptr, 1024, 1024, 1, ptr, ptr, d.data_ptr(), 0, 0) == S.SMA_ERR_ARG
    # a 30000 x 4 slice fits the scratch ((30000 + 4) * 4 floats) but two of
    # its stacked columns do not fit in shared memory: rejected on the host
    assert S.sma_slice_svd_noalloc(ptr, 30000, 4, 1, ptr, ptr, d.data_ptr(), 0, 0) == S.SMA_ERR_ARG
    assert S.sma_slice_svd_noalloc(ptr, 0, 4, 1, ptr, ptr, d.data_ptr(), 0, 0) == S.SMA_ERR_ARG
    assert S.sma_slice_svd_noalloc(0, 4, 4, 1, ptr, ptr, d.data_ptr(), 0, 0) == S.SMA_ERR_ARG
