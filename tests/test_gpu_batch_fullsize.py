"""The batched block-tridiagonal workload at full size: 512 matrices with
block counts 16..256 and block sizes 8..64 (about 2e5 frontal slices in
total), compressed by one handle from their distinct blocks, checked against
the FP64 oracle on a sample of the problems: the smallest problem of every
block size plus two more.  Ranks (identical, or within the fp32 window and
then compared at the GPU's ranks), singular values and the error report."""
import numpy as np
import pytest

from oracle import sma_oracle as O
from sma_inputs import generators as G

from _util import oracle_at_gpu_ranks, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
S = pytest.importorskip("paper_2105_01170_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_01170_gb300 import _build
    _build.build()


def test_full_batch_sampled_against_oracle():
    prs = G.block_tridiag_batch()
    assert len(prs) == 512
    tol = 1e-3
    blocks = [np.concatenate(list(pr.blocks), axis=1).astype(np.float32) for pr in prs]
    h = S.Handle(prs, prec=S.SMA_MIXED, rel_tol=tol, layout=S.SMA_INPUT_BLOCKS)
    res = h.compress([to_dev(b) for b in blocks])
    assert all(r["device_status"] == 0 for r in res)
    nslices = sum(pr.p for pr in prs)
    assert nslices > 150000
    sample = []
    for m in (8, 16, 32, 64):
        cand = [i for i, pr in enumerate(prs) if pr.m == m]
        sample.append(min(cand, key=lambda i: prs[i].p))
    sample += [17, 300]
    for i in sample:
        pr = prs[i]
        eta = O.multiplicities(pr.block_map, pr.p)
        # block k occupies columns k n .. k n + n - 1 of the m x (n p) input
        B = blocks[i].astype(np.float64).reshape(pr.m, pr.n, pr.p, order="F")
        X = B * np.sqrt(eta)[None, None, :]
        M = O.dct2_matrix(pr.p)
        ora = O.tsvdm(X, M, rel_tol=tol)
        ranks = h.ranks(i)
        cmp = oracle_at_gpu_ranks(ranks, ora, X, M, tol, S.SMA_MIXED, f"full batch problem {i}")
        assert res[i]["tensor_err"] <= tol * ora.normX * (1 + 1e-6)
        assert abs(res[i]["tensor_err"] - cmp.err) <= 1e-5 * ora.normX
        assert abs(res[i]["norm"] - ora.normX) <= 1e-6 * ora.normX
        sig = torch.empty(min(pr.m, pr.n) * pr.p, dtype=torch.float64, device="cuda")
        h.export(i, S.EXPORT_SIGMA, sig)
        sig = sig.cpu().numpy().reshape((min(pr.m, pr.n), pr.p), order="F")
        smax = max(float(np.max(s)) for s in ora.sigma)
        diff = max(float(np.max(np.abs(sig[:, k] - ora.sigma[k]))) for k in range(pr.p))
        assert diff <= 2e-5 * smax, (i, diff / smax)
    h.close()
