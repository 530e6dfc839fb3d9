"""The allocation-free block dot, checked against the handle-based entry point.

lsg_block_dot_noalloc exists for callers that are not allowed to allocate
device memory (code inside a memory arena or pool that owns the device memory,
or a host library called where cudaMalloc/cudaFree are off limits). It must give
the same sums as lsg_block_dot, whose scratch comes from gmres_create. This file
is collected last so a run that stops at the first failure has run everything
else; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1809_05805_b300 import problems as P

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


def gamma(k):
    return k * EPS / (1 - k * EPS)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_noalloc_block_dot_matches_handle_entry_point(torch_cuda):
    torch = torch_cuda
    from paper_1809_05805_b300 import lsgmres

    lsgmres.load()
    A = P.conv_diff_7pt(23)  # 12167 rows: many tiles and a ragged last tile
    n = len(A[0]) - 1
    A_dev = tuple(torch.from_numpy(a).cuda() for a in A)
    s = lsgmres.Solver(A, m=40, tol=1e-8)
    rng = np.random.default_rng(7)
    ldv = n + 3
    # two calls in a row with different inputs and sizes; the second reuses the
    # scratch the first one left behind
    for j, use_spmv in ((17, True), (40, False)):
        Vh = rng.standard_normal((j, ldv))
        u = rng.standard_normal(n)
        w0 = rng.standard_normal(n)
        Vd = torch.from_numpy(Vh).cuda()
        ud = torch.from_numpy(u).cuda()
        w_ref = torch.from_numpy(w0).cuda()
        w_new = torch.from_numpy(w0).cuda()
        X_ref = s.block_dot(Vd, ldv, j, ud, w_ref, use_spmv)
        X_dev = torch.full((2 * j + 2,), float("nan"), dtype=torch.float64, device="cuda")
        lsgmres.block_dot_noalloc(A_dev, n, Vd, ldv, j, ud, w_new, X_dev, use_spmv)
        torch.cuda.synchronize()
        X_new = X_dev.cpu().numpy()
        w = w_ref.cpu().numpy()
        assert np.array_equal(w_new.cpu().numpy(), w)
        cols = [Vh[k, :n] for k in range(j)]
        terms = [np.abs(c * u).sum() for c in cols] + [np.abs(c * w).sum() for c in cols] + \
                [np.abs(u * u).sum(), np.abs(u * w).sum()]
        assert np.all(np.isfinite(X_new))
        assert np.all(np.abs(X_new - X_ref) <= 2 * gamma(n) * np.array(terms))


def test_noalloc_rejects_too_many_columns(torch_cuda):
    torch = torch_cuda
    from paper_1809_05805_b300 import lsgmres

    A = P.conv_diff_7pt(4)
    A_dev = tuple(torch.from_numpy(a).cuda() for a in A)
    n = 64
    V = torch.zeros((65, n), dtype=torch.float64, device="cuda")
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    X = torch.zeros(2 * 65 + 2, dtype=torch.float64, device="cuda")
    with pytest.raises(lsgmres.GmresError) as e:
        lsgmres.block_dot_noalloc(A_dev, n, V, n, 65, u, u.clone(), X)
    assert e.value.status == lsgmres.ERR_ARG and "64" in str(e.value)
