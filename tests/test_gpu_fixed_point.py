"""GPU tests of the FP64 block dot on the integer pipes (gmres_set_block_dot).

The step kernel's full basis columns can be multiplied as exact fixed-point
integers (each FP64 value rescaled to a 58-bit integer relative to its
column's stored exponent bound, or its tile pair's for u and w, split in two
29-bit limbs; products summed exactly per tile pair, converted to FP64 once).
That changes rounding only, so:

* the standalone fused SpMV + block dot (lsg_block_dot) matches the oracle's
  sequential sums (orc_dot) at FP64 summation's classical bound
  2 gamma_n sum|terms| for vectors whose entries stay within a few binades of
  each other (zero columns, huge and tiny column scales, a ragged last tile
  pair); for entries spread over 30 decades the fixed-point form's error is
  relative to each vector's largest entry, and the test adds that documented
  term; both arithmetic forms are checked;
* whole solves with either form match the oracle's complete solve at the
  single-solve bar (identical counts, history 1e-8 over the first 50 steps, x
  1e-9), on a system large enough for the tile-pair ring kernel that carries
  the fixed-point form;
* the limb copy of the basis those kernels read is rewritten by every user
  (standalone block dots on different columns, a solve in between);
* NaN in u reaches the sums.
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


@pytest.fixture(scope="module")
def lsg():
    from paper_1809_05805_b300 import lsgmres

    lsgmres.load()
    return lsgmres


def _columns(rng, j, n, ldv, spread):
    """j basis columns whose entries vary by 2^(+-spread) within each column,
    column scales from 2^-300 to 2^300, one all-zero column, one column with a
    single nonzero entry."""
    V = np.zeros((j, ldv))
    for k in range(j):
        mag = np.exp2(rng.uniform(-spread, spread, n))
        V[k, :n] = rng.standard_normal(n) * mag * np.exp2(rng.integers(-300, 300))
    if j > 3:
        V[2, :] = 0.0
        V[3, :] = 0.0
        V[3, n // 2] = 1.5
    return V


def _fx_extra(x, y):
    """The fixed-point form's error beyond FP64 summation's: inputs rounded to
    2^-57 of their vector's largest entry (the tile pair's for u and w, which
    is no larger), and per product a dropped low-limb product below 2^-56 of
    the largest product (counted where both entries are nonzero)."""
    ax, ay = np.abs(x), np.abs(y)
    both = np.count_nonzero((ax > 0) & (ay > 0))
    return 2.0 ** -57 * (ax.max() * ay.sum() + ay.max() * ax.sum()) + 2.0 ** -56 * both * ax.max() * ay.max()


@pytest.mark.parametrize("fixed_point", [True, False])
@pytest.mark.parametrize("j,pad,spread", [(1, 6, 3), (8, 6, 3), (21, 6, 3), (50, 6, 3), (21, 5, 3), (8, 6, 50),
                                          (50, 6, 50)])
def test_block_dot_matches_oracle(torch_cuda, lsg, orc, fixed_point, j, pad, spread):
    """spread = 3: entries of a vector within 2^(+-3) of each other in
    magnitude (as in Krylov vectors): both forms within FP64 summation's
    classical bound 2 gamma_n sum|x_i y_i|. spread = 50 (entries across 30
    decades in every vector): the fixed-point form within that bound plus its
    own (_fx_extra), the FP64 form within the classical bound. pad = 5 gives an
    odd leading dimension: unaligned columns, which the library sends through
    the kernel with plain basis loads (FP64 products)."""
    torch = torch_cuda
    N = 70  # 343,000 rows: enough tile pairs per CTA for the ring kernel; ragged last pair
    A = P.conv_diff_7pt(N)
    n = len(A[0]) - 1
    rng = np.random.default_rng(j + spread)
    ldv = n + pad
    V = _columns(rng, j, n, ldv, spread)
    u = rng.standard_normal(n) * np.exp2(rng.uniform(-min(spread, 20), min(spread, 20), n)) * 2.0 ** 100
    s = lsg.Solver(A, m=50, tol=1e-8)
    active = s.set_block_dot(fixed_point)
    assert active == fixed_point  # this system runs the tile-pair ring kernel
    Vd = torch.from_numpy(V).cuda()
    ud = torch.from_numpy(u).cuda()
    wd = torch.zeros(n, dtype=torch.float64, device="cuda")
    for _ in range(2):  # twice: the exponent bounds are measured again per call
        X = s.block_dot(Vd, ldv, j, ud, wd, True)
    w = wd.cpu().numpy()
    assert np.all(np.abs(w - orc.spmv(A, u)) <= gamma(7) * (abs(P.to_scipy(A)) @ np.abs(u)))
    cols = [V[k, :n] for k in range(j)]
    ref = np.array([orc.dot(c, u) for c in cols] + [orc.dot(c, w) for c in cols] + [orc.dot(u, u), orc.dot(u, w)])
    terms = np.array([np.abs(c * u).sum() for c in cols] + [np.abs(c * w).sum() for c in cols] +
                     [np.abs(u * u).sum(), np.abs(u * w).sum()])
    assert np.all(np.isfinite(X))
    bound = 2 * gamma(n) * terms
    if fixed_point and pad % 2 == 0 and spread > 3:  # the fixed-point columns (full groups of 8)
        full = 8 * (j // 8)
        extra = np.zeros(2 * j + 2)
        for k in range(full):
            extra[k] = _fx_extra(cols[k], u)
            extra[j + k] = _fx_extra(cols[k], w)
        bound = bound + extra
    assert np.all(np.abs(X - ref) <= bound)
    if j > 3:  # the zero column gives exact zeros
        assert X[2] == 0.0 and X[j + 2] == 0.0
    s.close()


def _block_dot_checked(torch, s, orc, A, n, ldv, j, seed):
    """One standalone fused SpMV + block dot on fresh columns against the
    oracle's sums at the classical bound (entries within 2^(+-3))."""
    rng = np.random.default_rng(seed)
    V = _columns(rng, j, n, ldv, 3)
    u = rng.standard_normal(n) * np.exp2(rng.uniform(-3, 3, n))
    wd = torch.zeros(n, dtype=torch.float64, device="cuda")
    X = s.block_dot(torch.from_numpy(V).cuda(), ldv, j, torch.from_numpy(u).cuda(), wd, True)
    w = wd.cpu().numpy()
    cols = [V[k, :n] for k in range(j)]
    ref = np.array([orc.dot(c, u) for c in cols] + [orc.dot(c, w) for c in cols] + [orc.dot(u, u), orc.dot(u, w)])
    terms = np.array([np.abs(c * u).sum() for c in cols] + [np.abs(c * w).sum() for c in cols] +
                     [np.abs(u * u).sum(), np.abs(u * w).sum()])
    assert np.all(np.abs(X - ref) <= 2 * gamma(n) * terms)


def test_limb_copy_rewritten_by_each_user(torch_cuda, lsg, orc):
    """The fixed-point kernels read the basis as the limb copy (written once per
    column): two standalone block dots with different columns on one handle
    (each splits its caller's columns into the copy), then a solve (its steps
    rewrite the columns they use), then a block dot again, each against the
    oracle."""
    torch = torch_cuda
    A = P.conv_diff_7pt(70)
    n = len(A[0]) - 1
    ldv = n + 6  # even, so the columns stay 16-byte aligned for the ring kernel
    s = lsg.Solver(A, m=30, tol=1e-8, max_iter=1500)
    assert s.set_block_dot(True)
    _block_dot_checked(torch, s, orc, A, n, ldv, 21, seed=1)
    _block_dot_checked(torch, s, orc, A, n, ldv, 13, seed=2)
    _, b = P.rhs(A, seed=4)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = s.solve(torch.from_numpy(b).cuda(), x)
    r = orc.gmres(A, b, variant=1, m=30, tol=1e-8, max_iter=1500)
    assert info.status == r.status == 0 and info.iters == r.iters and info.restarts == r.restarts
    assert np.linalg.norm(x.cpu().numpy() - r.x) <= 1e-9 * np.linalg.norm(r.x)
    _block_dot_checked(torch, s, orc, A, n, ldv, 30, seed=3)
    s.close()


ORACLE_VARIANT = {"one_reduce_mgs": 1, "cgs2_lvl2": 3, "one_reduce_pipe2": 4}


@pytest.mark.parametrize("fixed_point,ortho", [(True, "one_reduce_mgs"), (False, "one_reduce_mgs"),
                                               (True, "cgs2_lvl2"), (True, "one_reduce_pipe2")])
def test_solve_matches_oracle(torch_cuda, lsg, orc, fixed_point, ortho):
    """72^3 (tile pairs, staging mode 6 when the fixed-point form is on): the
    one-reduce scheme and its two siblings, whose basis columns (and their
    stored limbs) are written by other kernels in between, at the
    single-solve bar."""
    torch = torch_cuda
    N = 72
    A = P.conv_diff_7pt(N)
    _, b = P.rhs(A, seed=3)
    n = len(b)
    stream = torch.cuda.Stream()
    s = lsg.Solver(A, m=40, tol=1e-9, max_iter=2000, stream=stream, ortho=ortho)
    assert s.set_block_dot(fixed_point) == fixed_point
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    bd = torch.from_numpy(b).cuda()
    torch.cuda.synchronize()
    info = s.solve(bd, x)
    r = orc.gmres(A, b, variant=ORACLE_VARIANT[ortho], m=40, tol=1e-9, max_iter=2000)
    assert info.status == r.status == 0
    assert info.iters == r.iters and info.restarts == r.restarts and info.reductions == r.reductions
    hist = s.history()
    assert np.all(np.abs(hist[:50] - r.history[:50]) <= 1e-8 * r.history[:50])
    assert np.linalg.norm(x.cpu().numpy() - r.x) <= 1e-9 * np.linalg.norm(r.x)
    # the same handle again, after switching the form (its cycle graphs are rebuilt)
    s.set_block_dot(not fixed_point)
    x.zero_()
    info2 = s.solve(bd, x)
    assert info2.iters == r.iters
    assert np.linalg.norm(x.cpu().numpy() - r.x) <= 1e-9 * np.linalg.norm(r.x)
    s.close()


def test_scaled_system_matches_oracle(torch_cuda, lsg, orc):
    """A right-hand side scaled by 2^400 and a matrix scaled by 2^-200: the
    stored exponent bounds follow the data, far from 1."""
    torch = torch_cuda
    A = P.conv_diff_7pt(70)
    A = (A[0], A[1], A[2] * 2.0 ** -200)
    _, b = P.rhs(A, seed=5)
    b = b * 2.0 ** 400
    s = lsg.Solver(A, m=30, tol=1e-8, max_iter=1500)
    assert s.set_block_dot(True)
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    info = s.solve(torch.from_numpy(b).cuda(), x)
    r = orc.gmres(A, b, variant=1, m=30, tol=1e-8, max_iter=1500)
    assert info.status == r.status == 0 and info.iters == r.iters
    hist = s.history()
    assert np.all(np.abs(hist[:50] - r.history[:50]) <= 1e-8 * r.history[:50])
    assert np.linalg.norm(x.cpu().numpy() - r.x) <= 1e-9 * np.linalg.norm(r.x)
    s.close()


def test_nonfinite_reaches_the_sums(torch_cuda, lsg):
    torch = torch_cuda
    A = P.conv_diff_7pt(70)
    n = len(A[0]) - 1
    s = lsg.Solver(A, m=20, tol=1e-8)
    assert s.set_block_dot(True)
    rng = np.random.default_rng(0)
    V = rng.standard_normal((16, n))
    u = rng.standard_normal(n)
    u[n // 3] = np.nan
    X = s.block_dot(torch.from_numpy(V).cuda(), n, 16, torch.from_numpy(u).cuda(),
                    torch.zeros(n, dtype=torch.float64, device="cuda"), True)
    assert np.all(np.isnan(X[:16])) and np.isnan(X[32])
    s.close()


def _batch_systems(count, seed, side):
    mats, rhs = [], []
    for i, par in enumerate(P.batch_2d_params(count, seed=seed, side=side)):
        A = P.batch_2d_system(par)
        _, b = P.rhs(A, seed=seed * 1000 + i)
        mats.append(A)
        rhs.append(b)
    return mats, rhs


@pytest.mark.parametrize("fixed_point,form", [(1, 2), (-1, 1), (0, 0)])
@pytest.mark.parametrize("grid", [None, 5, "tiles"])
def test_batch_matches_oracle(torch_cuda, lsg, orc, fixed_point, form, grid):
    """Batched FP64 solves with two rows per thread, with each form of the
    block-dot and MAXPY products (gmres_batch_set_block_dot: fixed point with
    the basis streamed through the column ring, which these 9-point systems'
    tile-pair CSR leaves room for; fixed point with direct basis loads; FP64
    FMAs), each system held to the single-solve bar against the oracle. Two systems are rescaled (the
    matrix by 2^-200 and the right-hand side by 2^300, and the right-hand side
    by 2^-400) so that their stored exponent bounds sit far from 1 and from
    each other's. grid = 'tiles' gives one tile per CTA: every unit is a single
    tile, the first or the second of its pair (masked rows in the fixed-point
    kernel); grid 5 cuts pairs at CTA boundaries."""
    torch = torch_cuda
    mats, rhs = _batch_systems(8, seed=41, side=(9, 70))
    A = mats[2]
    mats[2] = (A[0], A[1], A[2] * 2.0 ** -200)
    rhs[2] = P.rhs(mats[2], seed=7)[1] * 2.0 ** 300
    rhs[5] = rhs[5] * 2.0 ** -400
    ntiles = sum((len(A[0]) - 1 + 255) // 256 for A in mats)
    bs = lsg.BatchSolver(mats, m=20, tol=1e-8, max_iter=3000)
    if grid is not None:
        bs.set_grid(ntiles if grid == "tiles" else grid)
    bs.set_rows_per_thread(2)
    assert bs.set_block_dot(fixed_point) == form
    bd = [torch.from_numpy(b).cuda() for b in rhs]
    xd = [torch.zeros(len(b), dtype=torch.float64, device="cuda") for b in rhs]
    infos = bs.solve(bd, xd)
    for i, (A, b, info) in enumerate(zip(mats, rhs, infos)):
        r = orc.gmres(A, b, variant=1, m=20, tol=1e-8, max_iter=3000)
        assert info.status == r.status == 0
        assert info.iters == r.iters and info.restarts == r.restarts
        hist = bs.history(i)
        assert len(hist) == len(r.history)
        k = min(20, len(hist))
        assert np.all(np.abs(hist[:k] - r.history[:k]) <= 1e-8 * r.history[:k] + 1e-15 * r.history[0])
        x = xd[i].cpu().numpy()
        assert np.linalg.norm(x - r.x) <= 1e-9 * np.linalg.norm(r.x)
    # switching the form on the same handle changes rounding only
    assert bs.set_block_dot(0 if fixed_point else 1) == (0 if fixed_point else 2)
    for x in xd:
        x.zero_()
    infos2 = bs.solve(bd, xd)
    for info, info2 in zip(infos, infos2):
        assert info2.iters == info.iters
    bs.close()


def test_batch_fixed_point_off_for_single_rows(torch_cuda, lsg):
    """The fixed-point form needs two rows per thread: with one it reports
    itself inactive."""
    mats, rhs = _batch_systems(3, seed=43, side=(9, 30))
    bs = lsg.BatchSolver(mats, m=10, tol=1e-8, max_iter=500)
    bs.set_rows_per_thread(1)
    assert bs.set_block_dot(True) == 0
    bs.set_rows_per_thread(2)
    assert bs.set_block_dot(True) == 2
    assert bs.set_block_dot(-1) == 1
    bs.close()


def test_reproducible_fixed_order(torch_cuda, lsg):
    """gmres_set_reproducible(1): the fixed-point step kernel takes its tile
    pairs by a fixed stride, so two solves on one handle, and a solve on a
    second handle whose cycles replay as CUDA graphs, give bitwise identical x
    and residual histories."""
    torch = torch_cuda
    A = P.conv_diff_7pt(72)
    _, b = P.rhs(A, seed=9)
    bd = torch.from_numpy(b).cuda()
    outs = []
    for stream in (None, None, torch.cuda.Stream()):
        s = lsg.Solver(A, m=40, tol=1e-9, max_iter=2000, stream=stream)
        assert s.set_block_dot(True)
        s.set_reproducible(True)
        x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        s.solve(bd, x)
        outs.append((x.cpu().numpy(), s.history()))
        s.close()
    for o in outs[1:]:
        assert np.array_equal(outs[0][0], o[0]) and np.array_equal(outs[0][1], o[1])
