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


def _check_against_oracle(Vh, j, n, u, w_in, w_gpu, X_gpu, A, use_spmv):
    """X_gpu against the FP64 oracle's sequential sums (orc_dot) at the
    classical bound 2 gamma_n sum|terms| (any summation order), and w against
    the oracle's SpMV at gamma_k (k entries per row)."""
    import oracle

    o = oracle.get()
    if use_spmv:
        rowlen = np.diff(A[0]).max()
        assert np.all(np.abs(w_gpu - o.spmv(A, u)) <= gamma(int(rowlen)) * _abs_spmv(A, u))
    else:
        assert np.array_equal(w_gpu, w_in)
    w = w_gpu  # the sums are checked for the w the kernel used
    cols = [Vh[k, :n] for k in range(j)]
    ref = [o.dot(c, u) for c in cols] + [o.dot(c, w) for c in cols] + [o.dot(u, u), o.dot(u, w)]
    terms = [np.abs(c * u).sum() for c in cols] + [np.abs(c * w).sum() for c in cols] + \
            [np.abs(u * u).sum(), np.abs(u * w).sum()]
    assert np.all(np.isfinite(X_gpu))
    assert np.all(np.abs(X_gpu - np.array(ref)) <= 2 * gamma(n) * np.array(terms))


def _abs_spmv(A, x):
    """|A| |x| (the scale of each row's rounding error)."""
    return abs(P.to_scipy(A)) @ np.abs(x)


def test_noalloc_block_dot_matches_handle_entry_point_and_oracle(torch_cuda):
    """Calls in a row, reusing the scratch the previous call left behind: each
    against the handle entry point (whose scratch comes from gmres_create) and
    against the oracle. j = 17 with the SpMV, j = 40 with w given, j = 64 (the
    limit: every accumulator column of every warp in use), j = 0 with V = NULL
    (only u^T u and u^T w), and one call queued on a non-default stream."""
    torch = torch_cuda
    from paper_1809_05805_b300 import lsgmres

    lsgmres.load()
    A = P.conv_diff_7pt(23)  # 12167 rows: many tiles and a ragged last tile
    n = len(A[0]) - 1
    A_dev = tuple(torch.from_numpy(a).cuda() for a in A)
    s = lsgmres.Solver(A, m=64, tol=1e-8)
    rng = np.random.default_rng(7)
    ldv = n + 3
    side = torch.cuda.Stream()
    for j, use_spmv, on_side in ((17, True, False), (40, False, False), (64, True, False), (0, True, False),
                                 (33, True, True)):
        Vh = rng.standard_normal((max(j, 1), ldv))
        u = rng.standard_normal(n)
        w0 = rng.standard_normal(n)
        Vd = torch.from_numpy(Vh).cuda() if j > 0 else None
        ud = torch.from_numpy(u).cuda()
        w_ref = torch.from_numpy(w0).cuda()
        w_new = torch.from_numpy(w0).cuda()
        X_ref = s.block_dot(Vd, ldv, j, ud, w_ref, use_spmv)
        X_dev = torch.full((2 * j + 2,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        if on_side:
            lsgmres.block_dot_noalloc(A_dev, n, Vd, ldv, j, ud, w_new, X_dev, use_spmv, stream=side)
            side.synchronize()
        else:
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
        _check_against_oracle(Vh, j, n, u, w0, w_new.cpu().numpy(), X_new, A, use_spmv)


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
