"""GPU tests of whole restart cycles in one cooperative launch
(gmres_set_persistent: the latency path for small systems).

* Solves with the persistent cycle match the oracle at the single-solve bar
  (identical iteration, restart and reduction counts, history 1e-8 over the
  first 50 steps, x 1e-9), for one-reduce MGS-GMRES and its L = 2 pipeline, on
  the default stream and on a non-default one, and the same as the per-step
  launches of the same handle.
* Edge cases run through it: restart length 1, a max_iter that ends inside a
  cycle, a nonzero x0, an exact breakdown (A = I), b = 0.
* The grid barrier's bounded wait: with the test switch on, the barrier waits
  for a CTA that never arrives; the solve returns GMRES_ERR_TIMEOUT within
  seconds (no fault, no hang), and the handle then solves normally.
* The automatic choice: on for a system of at most one tile per CTA, off for
  larger ones.
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


def _check(info, s, x, r, n_hist=50):
    assert info.status == r.status
    assert info.iters == r.iters and info.restarts == r.restarts and info.reductions == r.reductions
    hist = s.history()
    k = min(n_hist, len(hist))
    assert len(hist) == len(r.history)
    assert np.all(np.abs(hist[:k] - r.history[:k]) <= 1e-8 * r.history[:k] + 1e-15)
    xs = x.cpu().numpy()
    assert np.linalg.norm(xs - r.x) <= 1e-9 * max(np.linalg.norm(r.x), 1e-300)


@pytest.mark.parametrize("ortho,variant", [("one_reduce_mgs", 1), ("one_reduce_pipe2", 4)])
@pytest.mark.parametrize("N,m", [(10, 12), (32, 30)])
@pytest.mark.parametrize("use_stream", [False, True])
def test_persistent_matches_oracle(torch_cuda, lsg, orc, ortho, variant, N, m, use_stream):
    torch = torch_cuda
    A = P.conv_diff_7pt(N)
    _, b = P.rhs(A, seed=N)
    n = len(b)
    s = lsg.Solver(A, m=m, tol=1e-9, ortho=ortho, max_iter=500,
                   stream=torch.cuda.Stream() if use_stream else None)
    assert s.set_persistent(1)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    bd = torch.from_numpy(b).cuda()
    torch.cuda.synchronize()
    info = s.solve(bd, x)
    r = orc.gmres(A, b, variant=variant, m=m, tol=1e-9, max_iter=500)
    _check(info, s, x, r)
    # one launch per cycle, beside the residual, least-squares and update launches
    assert info.kernel_launches <= 4 * info.restarts + 2
    # the per-step launches of the same handle reach the same solution
    assert not s.set_persistent(0)
    x2 = torch.zeros(n, dtype=torch.float64, device="cuda")
    info2 = s.solve(bd, x2)
    assert info2.iters == info.iters and info2.kernel_launches > info.kernel_launches
    assert np.linalg.norm(x2.cpu().numpy() - x.cpu().numpy()) <= 1e-12 * np.linalg.norm(r.x)
    s.close()


@pytest.mark.parametrize("case", ["m1", "maxiter", "x0", "identity", "zero_rhs"])
def test_persistent_edge_cases(torch_cuda, lsg, orc, case):
    torch = torch_cuda
    A = P.conv_diff_7pt(12)
    m, max_iter, tol = 20, 400, 1e-10
    if case == "m1":
        m, max_iter = 1, 300
    if case == "maxiter":
        max_iter = 47  # ends inside the third cycle
    if case == "identity":
        n0 = 1500
        A = (np.arange(n0 + 1, dtype=np.int32), np.arange(n0, dtype=np.int32), np.ones(n0))
    n = len(A[0]) - 1
    _, b = P.rhs(A, seed=4)
    if case == "zero_rhs":
        b = np.zeros(n)
    x0 = np.random.default_rng(5).uniform(-1, 1, n) if case == "x0" else np.zeros(n)
    s = lsg.Solver(A, m=m, tol=tol, max_iter=max_iter)
    assert s.set_persistent(1)
    x = torch.from_numpy(x0.copy()).cuda()
    info = s.solve(torch.from_numpy(b).cuda(), x)
    if case == "zero_rhs":
        assert info.status == 0 and np.all(x.cpu().numpy() == 0.0)
        return
    r = orc.gmres(A, b, variant=1, m=m, tol=tol, max_iter=max_iter, x0=x0)
    _check(info, s, x, r)
    s.close()


@pytest.mark.parametrize("use_stream,which", [(False, 1), (True, 1), (False, 2), (True, 2)])
def test_persistent_barrier_wait_runs_out(torch_cuda, lsg, use_stream, which):
    """which = 1: the grid barrier's wait; 2: the wait for a step's epilogue."""
    torch = torch_cuda
    A = P.conv_diff_7pt(16)
    _, b = P.rhs(A, seed=2)
    bd = torch.from_numpy(b).cuda()
    s = lsg.Solver(A, m=10, tol=1e-8, max_iter=300, stream=torch.cuda.Stream() if use_stream else None)
    assert s.set_persistent(1)
    s.test_stall_barrier(which)
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    t0 = time.time()
    with pytest.raises(lsg.GmresError) as e:
        s.solve(bd, x)
    assert e.value.status == lsg.ERR_TIMEOUT
    assert time.time() - t0 < 60
    s.test_stall_barrier(False)
    x.zero_()
    info = s.solve(bd, x)
    assert info.status == 0
    assert np.linalg.norm(b - P.to_scipy(A) @ x.cpu().numpy()) <= 1e-8 * np.linalg.norm(b)
    s.close()


def test_persistent_automatic_choice(torch_cuda, lsg):
    small = lsg.Solver(P.conv_diff_7pt(32), m=30, tol=1e-8)
    assert small.set_persistent(-1)  # 128 tiles: one per CTA
    large = lsg.Solver(P.conv_diff_7pt(80), m=30, tol=1e-8)
    assert not large.set_persistent(-1)  # 2,000 tiles
    assert large.set_persistent(1)  # forced on: still possible (the grid stays resident)
    mgs = lsg.Solver(P.conv_diff_7pt(32), m=30, tol=1e-8, ortho="mgs")
    assert not mgs.set_persistent(1)  # plain MGS keeps its per-inner-product launches
    for s in (small, large, mgs):
        s.close()
