"""GPU parity of batched solves (gmres_batch_*) against the FP64 oracle run on
each system alone.

Every system of a batch follows the one-reduce MGS-GMRES of Algorithm 7 on its
own data; batching only interleaves the systems' launches and changes the order
of the partial sums of each grid reduction. So each system is held to the bar of
a single solve (iteration, restart and reduction counts equal to the oracle's,
residual history within 1e-8 relative over the first cycle, x within 1e-9
relative), whatever the grid: one CTA spanning many systems, one system spanning
many CTAs, or one tile per CTA.

The systems are the seeded 2D 9-point convection-diffusion problems of the
batched workload (log-uniform grid sides, log-uniform cell diffusion
coefficients, upwinded convection), at sides small enough for the oracle.
"""
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


def _systems(count, seed, side):
    mats, rhs = [], []
    for i, par in enumerate(P.batch_2d_params(count, seed=seed, side=side)):
        A = P.batch_2d_system(par)
        _, b = P.rhs(A, seed=seed * 1000 + i)
        mats.append(A)
        rhs.append(b)
    return mats, rhs


def _solve_batch(torch, lsg, mats, rhs, m, tol, max_iter, grid=None, stream=None, x0s=None, allow=None, rows=None):
    bs = lsg.BatchSolver(mats, m=m, tol=tol, max_iter=max_iter, stream=stream)
    if grid is not None:
        bs.set_grid(grid)
    if rows is not None:
        bs.set_rows_per_thread(rows)
    bd = [torch.from_numpy(b).cuda() for b in rhs]
    xd = [torch.zeros(len(b), dtype=torch.float64, device="cuda") if x0s is None or x0s[i] is None
          else torch.from_numpy(x0s[i]).cuda() for i, b in enumerate(rhs)]
    torch.cuda.synchronize()
    infos = bs.solve(bd, xd, allow=allow) if allow else bs.solve(bd, xd)
    return bs, infos, [x.cpu().numpy() for x in xd], [bs.history(i) for i in range(len(mats))]


def _check_against_oracle(orc, A, b, info, x, hist, m, tol, max_iter, x0=None):
    r = orc.gmres(A, b, variant=1, m=m, tol=tol, max_iter=max_iter, x0=x0)
    assert info.status == r.status
    assert info.iters == r.iters and info.restarts == r.restarts
    # the batched first residual pass carries ||b|| in the same reduction as ||r0||
    assert info.reductions == r.reductions - 1
    k = min(m, len(hist))
    assert len(hist) == len(r.history)
    assert np.all(np.abs(hist[:k] - r.history[:k]) <= 1e-8 * r.history[:k] + 1e-15)
    assert np.linalg.norm(x - r.x) <= 1e-9 * np.linalg.norm(r.x)
    return r


@pytest.mark.parametrize("grid,rows", [(None, None), (1, 1), (1, 2), (5, 2), (3, 1), ("tiles", 1)])
def test_batch_matches_oracle_per_system(torch_cuda, lsg, orc, grid, rows):
    """Nine systems of 9^2 .. 70^2 rows (ragged tiles everywhere), GMRES(20),
    for the autotuned launch shape and for pinned grids with one or two rows
    per thread (tile pairs inside a system, single tiles at odd boundaries)."""
    torch = torch_cuda
    mats, rhs = _systems(9, seed=11, side=(9, 70))
    ntiles = sum((len(A[0]) - 1 + 255) // 256 for A in mats)
    g = ntiles if grid == "tiles" else grid
    bs, infos, xs, hists = _solve_batch(torch, lsg, mats, rhs, m=20, tol=1e-8, max_iter=3000, grid=g, rows=rows)
    if g is not None:
        assert bs.grid == g
    if rows is not None:
        assert bs.rows_per_thread == rows
    for A, b, info, x, h in zip(mats, rhs, infos, xs, hists):
        assert info.status == 0
        _check_against_oracle(orc, A, b, info, x, h, 20, 1e-8, 3000)
        true = np.linalg.norm(b - P.to_scipy(A) @ x) / np.linalg.norm(b)
        assert true <= 1e-8


def test_batch_many_systems_stream_graphs(torch_cuda, lsg, orc):
    """64 systems on a non-default stream (cycles replayed as CUDA graphs), a
    grid of 7 CTAs so that every CTA covers several systems; a sample of 12
    systems is checked against the oracle, all against the true residual."""
    torch = torch_cuda
    mats, rhs = _systems(64, seed=5, side=(6, 48))
    bs, infos, xs, hists = _solve_batch(torch, lsg, mats, rhs, m=16, tol=1e-9, max_iter=4000, grid=7,
                                        stream=torch.cuda.Stream(), rows=2)
    for i in range(0, 64, 6):
        _check_against_oracle(orc, mats[i], rhs[i], infos[i], xs[i], hists[i], 16, 1e-9, 4000)
    for A, b, info, x in zip(mats, rhs, infos, xs):
        assert info.status == 0
        assert np.linalg.norm(b - P.to_scipy(A) @ x) <= 1e-9 * np.linalg.norm(b)


def test_batch_more_tiles_than_streaming_grid(torch_cuda, lsg, orc):
    """24 systems of 90^2 .. 130^2 rows: ~1,100 tiles of 256 rows, more than
    the streaming kernels' grid (4 CTAs per SM) plus the per-system Givens
    CTAs, so every CTA of every kernel covers several systems' tiles. A sample
    against the oracle, every system against the true residual."""
    torch = torch_cuda
    mats, rhs = _systems(24, seed=17, side=(90, 130))
    assert sum((len(A[0]) - 1 + 255) // 256 for A in mats) > 4 * 148 + 24
    bs, infos, xs, hists = _solve_batch(torch, lsg, mats, rhs, m=30, tol=1e-8, max_iter=5000,
                                        stream=torch.cuda.Stream())
    for i in range(0, 24, 5):
        _check_against_oracle(orc, mats[i], rhs[i], infos[i], xs[i], hists[i], 30, 1e-8, 5000)
    for A, b, info, x in zip(mats, rhs, infos, xs):
        assert info.status == 0
        assert np.linalg.norm(b - P.to_scipy(A) @ x) <= 1e-8 * np.linalg.norm(b)


def test_batch_edge_systems(torch_cuda, lsg, orc):
    """In one batch: a 1 x 1 system, a zero right-hand side, a nonzero x0, a
    dense 13 x 13 system solved exactly by GMRES(13), a system that stops at
    max_iter, and a NaN right-hand side; each keeps its own outcome."""
    torch = torch_cuda
    lsg_ = lsg
    m, tol, max_iter = 13, 1e-12, 60
    one = (np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0]))
    dense = P.from_dense(P.random_dense(13, seed=2))
    hard = P.batch_2d_system(P.batch_2d_params(1, seed=9, side=(40, 40))[0])
    plain = P.batch_2d_system(P.batch_2d_params(1, seed=3, side=(12, 12))[0])
    mats = [one, plain, plain, dense, hard, plain]
    rng = np.random.default_rng(4)
    rhs = [np.array([1.5]), np.zeros(144), rng.standard_normal(144), rng.standard_normal(13),
           P.rhs(hard, 1)[1], rng.standard_normal(144)]
    rhs[5][17] = np.nan
    x0s = [None, np.ones(144), rng.uniform(-1, 1, 144), None, None, None]
    bs, infos, xs, hists = _solve_batch(torch, lsg_, mats, rhs, m=m, tol=tol, max_iter=max_iter, x0s=x0s,
                                        allow=(lsg.OK, lsg.MAXITER, lsg.ERR_NONFINITE))
    assert infos[5].status == lsg.ERR_NONFINITE and infos[5].iters == 0
    assert infos[1].status == 0 and infos[1].iters == 0 and np.all(xs[1] == 0.0)
    assert infos[4].status == lsg.MAXITER and infos[4].iters == max_iter
    for i in (0, 2, 3, 4):
        _check_against_oracle(orc, mats[i], rhs[i], infos[i], xs[i], hists[i], m, tol, max_iter, x0=x0s[i])
    assert abs(xs[0][0] - 0.5) <= 1e-15


def test_batch_deterministic_and_graph_path(torch_cuda, lsg):
    """Fixed-order reductions: the default-stream path and the graph path of the
    same grid give bitwise identical solutions and histories, twice."""
    torch = torch_cuda
    mats, rhs = _systems(12, seed=21, side=(10, 60))
    outs = []
    for stream in (None, torch.cuda.Stream(), torch.cuda.Stream()):
        _, _, xs, hs = _solve_batch(torch, lsg, mats, rhs, m=12, tol=1e-10, max_iter=2000, grid=9, stream=stream)
        outs.append((np.concatenate(xs), np.concatenate(hs)))
    for o in outs[1:]:
        assert np.array_equal(outs[0][0], o[0]) and np.array_equal(outs[0][1], o[1])


def test_batch_results_alone_and_in_mix(torch_cuda, lsg):
    """A system solved inside a batch of 14 and in a batch of three, with
    different grids and rows per thread, gives the same result within the
    single-solve bar: identical iteration and restart counts, residual history
    within 1e-8 relative over the first cycle, x within 1e-9 relative (only the
    order of the partial sums of its reductions differs)."""
    torch = torch_cuda
    mats, rhs = _systems(14, seed=31, side=(12, 80))
    ref = None
    for grid, rows in ((None, None), (1, 1), (7, 2), (23, 1)):
        _, infos, xs, hs = _solve_batch(torch, lsg, mats, rhs, m=15, tol=1e-10, max_iter=3000, grid=grid, rows=rows)
        if ref is None:
            ref = (infos, xs, hs)
            continue
        for i in range(14):
            assert infos[i].iters == ref[0][i].iters and infos[i].restarts == ref[0][i].restarts
            assert np.linalg.norm(xs[i] - ref[1][i]) <= 1e-9 * np.linalg.norm(ref[1][i])
            assert np.all(np.abs(hs[i][:15] - ref[2][i][:15]) <= 1e-8 * ref[2][i][:15])
    pick = [3, 8, 13]
    _, infos, xs, hs = _solve_batch(torch, lsg, [mats[i] for i in pick], [rhs[i] for i in pick], m=15, tol=1e-10,
                                    max_iter=3000, grid=5, stream=torch.cuda.Stream())
    for k, i in enumerate(pick):
        assert infos[k].iters == ref[0][i].iters
        assert np.linalg.norm(xs[k] - ref[1][i]) <= 1e-9 * np.linalg.norm(ref[1][i])


def test_batch_agrees_with_single_solver(torch_cuda, lsg):
    """The batched solve of each system and a standalone Solver run of it stop
    after the same number of steps with solutions within 1e-9 relative."""
    torch = torch_cuda
    mats, rhs = _systems(5, seed=2, side=(20, 90))
    _, infos, xs, _ = _solve_batch(torch, lsg, mats, rhs, m=25, tol=1e-9, max_iter=3000)
    for A, b, info, x in zip(mats, rhs, infos, xs):
        s = lsg.Solver(A, m=25, tol=1e-9, max_iter=3000)
        xg = torch.zeros(len(b), dtype=torch.float64, device="cuda")
        si = s.solve(torch.from_numpy(b).cuda(), xg)
        assert si.iters == info.iters and si.restarts == info.restarts
        assert np.linalg.norm(xg.cpu().numpy() - x) <= 1e-9 * np.linalg.norm(x)


def test_batch_argument_checks(torch_cuda, lsg):
    torch = torch_cuda
    mats, rhs = _systems(3, seed=1, side=(8, 12))
    with pytest.raises(lsg.GmresError) as e:
        lsg.BatchSolver(mats, m=0, tol=1e-8)
    assert e.value.status == lsg.ERR_ARG
    bad = (np.array([0, 2, 1], np.int32), np.array([0, 1], np.int32), np.array([1.0, 2.0]))
    with pytest.raises(lsg.GmresError) as e:
        lsg.BatchSolver(mats + [bad], m=5, tol=1e-8)
    assert e.value.status == lsg.ERR_ARG
    bs = lsg.BatchSolver(mats, m=5, tol=1e-8)
    with pytest.raises(lsg.GmresError) as e:
        bs.set_grid(10 ** 6)
    assert e.value.status == lsg.ERR_ARG
    with pytest.raises(lsg.GmresError) as e:
        bs.set_rows_per_thread(3)
    assert e.value.status == lsg.ERR_ARG
    with pytest.raises(ValueError):
        bs.solve([torch.zeros(1, dtype=torch.float64, device="cuda")], [])


def _model_step_bytes(A, iters, m, max_iter):
    """Algorithmic bytes of the step launches of one system's solve: cycles of
    k = min(m, remaining) columns, the last one shorter; steps j = 0..k, the
    step at j = kmax reading only u and V_j."""
    n, nnz = len(A[0]) - 1, len(A[1])
    csr = 4.0 * (n + 1) + 12.0 * nnz
    total, done = 0.0, 0
    while done < iters:
        kmax = min(m, max_iter - done)
        k = min(kmax, iters - done)
        for j in range(k + 1):
            total += 8.0 * n * (j + 1) if j == kmax else csr + 8.0 * n * (j + 2)
        done += k
    return total


def test_batch_host_entry_and_profile(torch_cuda, lsg):
    """The host-buffer entry point gives the device entry point's results bit
    for bit; the profile of the graph path attributes the step launches the
    algorithmic bytes of the per-system model."""
    torch = torch_cuda
    mats, rhs = _systems(10, seed=8, side=(10, 80))
    bs, infos, xs, hs = _solve_batch(torch, lsg, mats, rhs, m=15, tol=1e-9, max_iter=3000, grid=6,
                                     stream=torch.cuda.Stream())
    bs.set_profile(True)
    xh = [np.zeros(len(b)) for b in rhs]
    infos_h = bs.solve_host([np.ascontiguousarray(b) for b in rhs], xh)
    prof = bs.profile()
    for i in range(len(mats)):
        assert np.array_equal(xh[i], xs[i]) and infos_h[i].iters == infos[i].iters
        assert np.array_equal(bs.history(i), hs[i])
    want = sum(_model_step_bytes(A, inf.iters, 15, 3000) for A, inf in zip(mats, infos_h) if inf.breakdowns == 0)
    assert all(inf.breakdowns == 0 for inf in infos_h)
    st = prof["one_reduce_step"]
    assert st["launches"] > 0 and st["ms"] > 0
    assert abs(st["bytes"] - want) <= 1e-9 * want
    assert prof["arnoldi_maxpy"]["launches"] >= st["launches"] - sum(inf.restarts for inf in infos_h) - 1
