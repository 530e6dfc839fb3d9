"""GPU tests of the CSR staging of the step kernel (each tile's rowptr slice,
indices and values brought into shared memory by bulk copies, completion
waited for on an mbarrier with a bounded wait).

* Matrices whose rows differ wildly in length (empty rows, one long row, a
  ragged tail) go through the staged kernel and match the oracle at the
  single-solve bar.
* The bounded wait: with the test switch on, every copy announces 16 bytes
  that never arrive, so every wait runs out (no fault, no hang: the waits are
  bounded and no copy is left in flight); the solve must come back with
  GMRES_ERR_TIMEOUT within seconds, and the same handle must solve normally
  afterwards.
"""
import time

import numpy as np
import pytest

from paper_1809_05805_b300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def lsg():
    from paper_1809_05805_b300 import lsgmres

    lsgmres.load()
    return lsgmres


def _ragged(n, seed):
    """Diagonally dominant CSR with row lengths 0..40 except every 97th row
    (length 300), and empty off-diagonal rows near the end: staged tiles of
    very different sizes."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        k = 300 if i % 97 == 5 else int(rng.integers(0, 41))
        if i > n - 40:
            k = 0
        c = np.unique(rng.integers(0, n, k))
        c = c[c != i]
        v = rng.uniform(-1, 1, len(c)) / max(len(c), 1)
        rows.extend([i] * (len(c) + 1))
        cols.extend([i, *c.tolist()])
        vals.extend([4.0, *v.tolist()])
    order = np.lexsort((np.array(cols), np.array(rows)))
    r = np.array(rows)[order]
    rp = np.zeros(n + 1, np.int32)
    np.add.at(rp, r + 1, 1)
    return np.cumsum(rp).astype(np.int32), np.array(cols, np.int32)[order], np.array(vals)[order]


@pytest.mark.parametrize("n", [1000, 5000, 40000])
def test_staged_ragged_rows_match_oracle(torch_cuda, lsg, orc, n):
    torch = torch_cuda
    A = _ragged(n, seed=n)
    b = np.random.default_rng(1).standard_normal(n)
    s = lsg.Solver(A, m=20, tol=1e-10, max_iter=400)
    s.set_persistent(0)  # per-step launches: the staged step kernel (small systems default to one launch per cycle)
    assert s.test_stall_staging(False)  # the FP64 step kernel stages this matrix
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = s.solve(torch.from_numpy(b).cuda(), x)
    r = orc.gmres(A, b, variant=1, m=20, tol=1e-10, max_iter=400)
    assert info.status == r.status and info.iters == r.iters and info.restarts == r.restarts
    hist = s.history()
    k = min(50, len(hist))
    assert np.all(np.abs(hist[:k] - r.history[:k]) <= 1e-8 * r.history[:k] + 1e-15)
    assert np.linalg.norm(x.cpu().numpy() - r.x) <= 1e-9 * np.linalg.norm(r.x)


@pytest.mark.parametrize("graph", [False, True])
def test_staging_wait_runs_out_and_reports_timeout(torch_cuda, lsg, graph):
    torch = torch_cuda
    A = P.conv_diff_7pt(24)
    n = len(A[0]) - 1
    _, b = P.rhs(A, seed=2)
    bd = torch.from_numpy(b).cuda()
    s = lsg.Solver(A, m=6, tol=1e-8, max_iter=300, stream=torch.cuda.Stream() if graph else None)
    s.set_persistent(0)  # per-step launches: the staged step kernel
    assert s.test_stall_staging(True)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    t0 = time.time()
    with pytest.raises(lsg.GmresError) as e:
        s.solve(bd, x)
    assert e.value.status == lsg.ERR_TIMEOUT
    assert time.time() - t0 < 120
    s.test_stall_staging(False)
    x.zero_()
    info = s.solve(bd, x)
    assert info.status == 0
    assert np.linalg.norm(b - P.to_scipy(A) @ x.cpu().numpy()) <= 1e-8 * np.linalg.norm(b)


def test_handles_of_different_shapes_interleave(torch_cuda, lsg):
    """Kernels are shared by all handles and their shared-memory limit is a
    process-wide attribute: a handle whose step kernel stages a large tile
    (27-point GMRES-IR at 69^3, the largest staged CSR tile) must still solve
    after handles with smaller tiles (and a smaller restart length) were made."""
    torch = torch_cuda
    big = P.aniso_27pt(69)
    _, bb = P.rhs(big, seed=3)
    s1 = lsg.Solver(big, m=40, tol=1e-8, prec="ir_fp32", max_iter=2000)
    # the same step kernel (restart 40, staged single tiles) with a 7-point tile: less shared memory
    seven = P.conv_diff_7pt(69)
    _, b7 = P.rhs(seven, seed=4)
    s2 = lsg.Solver(seven, m=40, tol=1e-8, prec="ir_fp32", max_iter=2000)
    # a shorter restart: the least-squares kernel needs less shared memory
    small = P.conv_diff_7pt(12)
    _, bs = P.rhs(small, seed=5)
    s3 = lsg.Solver(small, m=10, tol=1e-8, max_iter=2000)
    for s, A, b in ((s2, seven, b7), (s3, small, bs), (s1, big, bb), (s2, seven, b7), (s1, big, bb)):
        x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
        info = s.solve(torch.from_numpy(b).cuda(), x)
        assert info.status == 0
        assert np.linalg.norm(b - P.to_scipy(A) @ x.cpu().numpy()) <= 1e-8 * np.linalg.norm(b)


def test_dense_row_pairs_without_ring_match_oracle(torch_cuda, lsg, orc):
    """A 2D 9-point problem of 360,000 rows (1,407 tiles, enough for tile pairs
    at two CTAs per SM): its tile pair's CSR (4,608 entries, 57 KB in FP64)
    leaves no room beside it for the 48 KB column ring at two CTAs per SM, so
    the FP64 step kernel takes tile pairs without the ring (staging mode 5).
    Two cycles of GMRES(30) against the oracle, step by step."""
    torch = torch_cuda
    N = 600
    kc = np.exp(np.random.default_rng(7).uniform(np.log(0.1), np.log(10.0), (N + 1, N + 1)))
    A = P.conv_diff_9pt_2d(N, kc, 0.7, 1.0)
    n = N * N
    _, b = P.rhs(A, seed=3)
    s = lsg.Solver(A, m=30, tol=1e-14, max_iter=60)
    assert s.test_stall_staging(False)  # the FP64 step kernel stages this matrix
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = s.solve(torch.from_numpy(b).cuda(), x)
    r = orc.gmres(A, b, variant=1, m=30, tol=1e-14, max_iter=60)
    assert info.status == r.status and info.iters == r.iters == 60
    hist = s.history()
    assert np.all(np.abs(hist[:60] - r.history[:60]) <= 1e-8 * r.history[:60] + 1e-15)
    assert np.linalg.norm(x.cpu().numpy() - r.x) <= 1e-9 * np.linalg.norm(r.x)
