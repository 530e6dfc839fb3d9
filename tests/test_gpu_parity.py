"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances:
  * single steps (SpMV, block dot, MAXPY): the classical rounding bound
    gamma_k * sum|terms| with k the number of terms of each sum, which holds for
    any summation order (the GPU sums in a tree, the oracle sequentially);
  * Arnoldi basis and Hessenberg over one cycle: 1e-10 (rounding differences
    amplified at most by the cycle's loss of orthogonality, ~1e-11 here);
  * whole solves: residual history within 1e-8 relative over the first 50
    steps and the final x within 1e-9 relative, the bar the method is held to.
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


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


PROBLEMS = {
    "c1_32cubed": lambda: P.conv_diff_7pt(32),
    "ragged_7cubed": lambda: P.conv_diff_7pt(7),          # 343 rows: one partial tile
    "ragged_23cubed": lambda: P.conv_diff_7pt(23),        # 12167 rows: many tiles + ragged tail
    "dense_37": lambda: P.from_dense(P.random_dense(37, seed=4)),  # 37 nnz per row
}


# ------------------------------------------------------------------ single steps
@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_spmv(torch_cuda, lsg, orc, name):
    torch = torch_cuda
    A = PROBLEMS[name]()
    n = len(A[0]) - 1
    x = np.random.default_rng(1).standard_normal(n)
    s = lsg.Solver(A, m=4, tol=1e-8)
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.spmv(dev(torch, x), y)
    ref = orc.spmv(A, x)
    absA = P.to_scipy(A)
    absA.data = np.abs(absA.data)
    bound = gamma(int(np.diff(A[0]).max())) * (absA @ np.abs(x))
    assert np.all(np.abs(y.cpu().numpy() - ref) <= bound + 1e-300)


@pytest.mark.parametrize("n,j", [(343, 0), (343, 3), (12167, 9), (32768, 30), (40001, 17)])
@pytest.mark.parametrize("use_spmv", [True, False])
def test_block_dot(torch_cuda, lsg, orc, n, j, use_spmv):
    """X = [V u]^T [u w] with w = A u fused (or given), against oracle dot products."""
    torch = torch_cuda
    N = round(n ** (1 / 3))
    A = P.conv_diff_7pt(N) if N ** 3 == n else tridiag(n)  # non-cube sizes: a 3-point operator
    rng = np.random.default_rng(n + j)
    ldv = n + 5  # leading dimension larger than n
    Vh = rng.standard_normal((max(j, 1), ldv))  # row k = column k (column-major n x j)
    u = rng.standard_normal(n)
    w0 = rng.standard_normal(n)
    s = lsg.Solver(A, m=max(j, 1), tol=1e-8)
    Vd = dev(torch, Vh)
    wd = dev(torch, w0)
    X = s.block_dot(Vd, ldv, j, dev(torch, u), wd, use_spmv)
    w = orc.spmv(A, u) if use_spmv else w0
    if use_spmv:
        assert np.allclose(wd.cpu().numpy(), w, rtol=0, atol=1e-12 * np.abs(w).max())
    cols = [Vh[k, :n] for k in range(j)]
    ref = [orc.dot(c, u) for c in cols] + [orc.dot(c, w) for c in cols] + [orc.dot(u, u), orc.dot(u, w)]
    terms = [np.abs(c * u).sum() for c in cols] + [np.abs(c * w).sum() for c in cols] + \
            [np.abs(u * u).sum(), np.abs(u * w).sum()]
    for k, (a, r, t) in enumerate(zip(X, ref, terms)):
        assert abs(a - r) <= 2 * gamma(n) * t, (k, a, r)


def tridiag(n):
    import scipy.sparse as sp

    S = sp.diags([-1.0, 2.5, -1.2], [-1, 0, 1], shape=(n, n), format="csr")
    S.sort_indices()
    return S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64)


@pytest.mark.parametrize("n,K", [(1, 1), (343, 0), (1001, 5), (32768, 31), (65537, 51)])
def test_maxpy(torch_cuda, lsg, orc, n, K):
    torch = torch_cuda
    rng = np.random.default_rng(K)
    ldv = n + (n % 2)  # even leading dimension keeps 16-byte column alignment
    Vh = rng.standard_normal((max(K, 1), ldv))
    c = rng.standard_normal(K)
    y = rng.standard_normal(n)
    s = lsg.Solver(tridiag(max(n, 2)) if n > 1 else (np.array([0, 1], np.int32), np.array([0], np.int32),
                                                    np.array([2.0])), m=max(K, 1) + 1, tol=1e-8)
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.maxpy(dev(torch, Vh), ldv, c, 0.75, dev(torch, y), out)
    V = Vh[:K, :n].T if K else np.zeros((n, 0))
    ref = orc.maxpy(V, c, 0.75, y)
    bound = gamma(K + 1) * (0.75 * np.abs(y) + np.abs(V) @ np.abs(c))
    assert np.all(np.abs(out.cpu().numpy() - ref) <= bound + 1e-300)


# ------------------------------------------------------------------ one cycle
@pytest.mark.parametrize("ortho", ["mgs", "one_reduce_mgs"])
@pytest.mark.parametrize("N,k", [(7, 5), (16, 30), (32, 30)])
def test_arnoldi_cycle(torch_cuda, lsg, orc, ortho, N, k):
    torch = torch_cuda
    A = P.conv_diff_7pt(N)
    _, b = P.rhs(A, seed=3)
    s = lsg.Solver(A, m=k, tol=0.0, ortho=ortho)
    V, H, T, kk = s.arnoldi(dev(torch, b), k)
    r = orc.gmres(A, b, variant=0 if ortho == "mgs" else 1, m=k, tol=0.0, max_iter=k, capture=True)
    assert kk == r.k == k
    Vg = V.cpu().numpy()
    assert np.abs(Vg - r.V).max() <= 1e-10
    assert np.abs(H - r.H).max() <= 1e-10 * np.abs(r.H).max()
    if ortho != "mgs":
        assert np.abs(T - r.T).max() <= 1e-10
    # Arnoldi relation on the GPU's own output
    AV = P.to_scipy(A) @ Vg[:, :kk]
    assert np.linalg.norm(AV - Vg @ H) <= 1e-12 * np.linalg.norm(AV)


# ------------------------------------------------------------------ whole solves
def _solve_both(torch, lsg, orc, A, b, m, tol, max_iter, ortho, x0=None):
    n = len(A[0]) - 1
    s = lsg.Solver(A, m=m, tol=tol, ortho=ortho, max_iter=max_iter)
    x = dev(torch, np.zeros(n) if x0 is None else x0)
    info = s.solve(dev(torch, b), x)
    hist = s.history()
    r = orc.gmres(A, b, variant=0 if ortho == "mgs" else 1, m=m, tol=tol, max_iter=max_iter, x0=x0)
    return info, hist, x.cpu().numpy(), r


@pytest.mark.parametrize("ortho", ["mgs", "one_reduce_mgs"])
def test_solve_c1(torch_cuda, lsg, orc, ortho):
    """32^3 convection-diffusion, GMRES(30) to 1e-8 (the small benchmark case)."""
    A = P.conv_diff_7pt(32)
    xt, b = P.rhs(A, seed=0)
    info, hist, x, r = _solve_both(torch_cuda, lsg, orc, A, b, 30, 1e-8, 300, ortho)
    assert info.status == 0 and r.status == 0
    assert info.iters == r.iters and info.restarts == r.restarts
    assert info.reductions == r.reductions
    h50 = slice(0, min(50, len(hist)))
    assert np.all(np.abs(hist[h50] - r.history[h50]) <= 1e-8 * r.history[h50])
    assert np.linalg.norm(x - r.x) <= 1e-9 * np.linalg.norm(r.x)
    true = np.linalg.norm(b - P.to_scipy(A) @ x) / np.linalg.norm(b)
    assert true <= 1e-8 and abs(true - info.rel_resid_true) <= 1e-3 * true


@pytest.mark.parametrize("ortho", ["mgs", "one_reduce_mgs"])
@pytest.mark.parametrize("case", ["m1", "ragged_restarts", "maxiter", "x0", "direct", "exact_breakdown"])
def test_solve_edge_cases(torch_cuda, lsg, orc, ortho, case):
    torch = torch_cuda
    if case == "m1":  # GMRES(1): one column per cycle
        A = P.conv_diff_7pt(5)
        _, b = P.rhs(A, 1)
        args = dict(m=1, tol=1e-6, max_iter=400)
    elif case == "ragged_restarts":
        A = P.conv_diff_7pt(11)
        _, b = P.rhs(A, 2)
        args = dict(m=7, tol=1e-10, max_iter=500)
    elif case == "maxiter":
        A = P.conv_diff_7pt(9)
        _, b = P.rhs(A, 3)
        args = dict(m=6, tol=1e-14, max_iter=20)
    elif case == "x0":
        A = P.conv_diff_7pt(9)
        _, b = P.rhs(A, 4)
        args = dict(m=10, tol=1e-9, max_iter=300)
    elif case == "exact_breakdown":  # A = 2 I, b = e_0: u_1 = 0 exactly at step 1
        n = 300
        A = (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.full(n, 2.0))
        b = np.zeros(n)
        b[0] = 1.0
        args = dict(m=5, tol=1e-12, max_iter=50)
    else:  # GMRES(n) on a small dense system: exact termination
        M = P.random_dense(13, seed=2)
        A = P.from_dense(M)
        b = np.random.default_rng(2).standard_normal(13)
        args = dict(m=13, tol=1e-13, max_iter=13)
    n = len(A[0]) - 1
    x0 = np.random.default_rng(9).uniform(-1, 1, n) if case == "x0" else None
    info, hist, x, r = _solve_both(torch, lsg, orc, A, b, ortho=ortho, x0=x0, **args)
    assert info.status == r.status
    assert info.iters == r.iters and info.restarts == r.restarts
    k = min(50, len(hist))
    assert np.all(np.abs(hist[:k] - r.history[:k]) <= 1e-8 * r.history[:k] + 1e-15)
    assert np.linalg.norm(x - r.x) <= 1e-9 * np.linalg.norm(r.x)


def test_zero_and_nonfinite_rhs(torch_cuda, lsg):
    torch = torch_cuda
    A = P.conv_diff_7pt(6)
    s = lsg.Solver(A, m=5, tol=1e-8)
    x = torch.ones(216, dtype=torch.float64, device="cuda")
    info = s.solve(torch.zeros(216, dtype=torch.float64, device="cuda"), x)
    assert info.status == 0 and float(x.abs().max()) == 0.0
    b = torch.ones(216, dtype=torch.float64, device="cuda")
    b[7] = float("nan")
    with pytest.raises(lsg.GmresError) as e:
        s.solve(b, x)
    assert e.value.status == lsg.ERR_NONFINITE


@pytest.mark.parametrize("N,m,prec", [(20, 20, "fp64"), (32, 30, "fp64"), (69, 40, "ir_fp32"), (69, 40, "ir_bf16")])
def test_deterministic(torch_cuda, lsg, N, m, prec):
    """Fixed-order reductions: two solves give bitwise identical x and history
    (20^3: one-level grid sums; 32^3: two-level; 69^3 GMRES-IR: CSR tiles
    staged in shared memory, and with a BF16 basis its basis tiles too)."""
    torch = torch_cuda
    A = P.conv_diff_7pt(N)
    _, b = P.rhs(A, 5)
    s = lsg.Solver(A, m=m, tol=1e-9, prec=prec, max_iter=3000)
    bd = dev(torch, b)
    outs = []
    for _ in range(2):
        x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
        s.solve(bd, x)
        outs.append((x.cpu().numpy(), s.history()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_host_entry_point(torch_cuda, lsg, orc):
    """gmres_solve_host (host buffers, copies inside the call) equals the device call."""
    A = P.conv_diff_7pt(12)
    _, b = P.rhs(A, 6)
    s = lsg.Solver(A, m=15, tol=1e-9)
    xh = np.zeros(len(b))
    info = s.solve_host(np.ascontiguousarray(b), xh)
    r = orc.gmres(A, b, variant=1, m=15, tol=1e-9, max_iter=150)
    assert info.status == 0 and info.iters == r.iters
    assert np.linalg.norm(xh - r.x) <= 1e-9 * np.linalg.norm(r.x)


def test_invalid_csr_rejected(lsg):
    rowptr = np.array([0, 2, 1], dtype=np.int32)  # decreasing
    with pytest.raises(lsg.GmresError) as e:
        lsg.Solver((rowptr, np.array([0, 1], np.int32), np.ones(2)), m=2, tol=1e-8)
    assert e.value.status == lsg.ERR_ARG
    with pytest.raises(lsg.GmresError):
        lsg.Solver((np.array([0, 1, 2], np.int32), np.array([0, 5], np.int32), np.ones(2)), m=2, tol=1e-8)


@pytest.mark.parametrize("ortho", ["mgs", "one_reduce_mgs"])
def test_stream_graph_path(torch_cuda, lsg, orc, ortho):
    """On a non-default stream each cycle runs as a replayed CUDA graph. Results
    equal the oracle's and, bitwise, the kernel-by-kernel path on the default
    stream; max_iter = 70 with m = 30 also exercises a shorter last cycle."""
    torch = torch_cuda
    A = P.conv_diff_7pt(24)
    _, b = P.rhs(A, seed=11)
    n = len(b)
    bd = dev(torch, b)
    r = orc.gmres(A, b, variant=0 if ortho == "mgs" else 1, m=30, tol=1e-12, max_iter=70)
    outs = []
    for use_stream in (False, True):
        s = lsg.Solver(A, m=30, tol=1e-12, ortho=ortho, max_iter=70)
        s.set_persistent(0)  # per-step launches (graphs on the stream)
        stream = torch.cuda.Stream() if use_stream else None
        if stream is not None:
            s.set_stream(stream)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        info = s.solve(bd, x)
        outs.append((x.cpu().numpy(), s.history(), info))
    for x, hist, info in outs:
        assert info.iters == r.iters == 70 and info.restarts == r.restarts
        k = 50
        assert np.all(np.abs(hist[:k] - r.history[:k]) <= 1e-8 * r.history[:k])
        assert np.linalg.norm(x - r.x) <= 1e-9 * np.linalg.norm(r.x)
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_stream_graph_replay_twice(torch_cuda, lsg):
    """Two solves on one handle and stream (graphs replayed) give identical results."""
    torch = torch_cuda
    A = P.conv_diff_7pt(16)
    _, b = P.rhs(A, seed=12)
    s = lsg.Solver(A, m=20, tol=1e-10)
    s.set_persistent(0)  # per-step launches, so that the cycles run as replayed graphs
    stream = torch.cuda.Stream()
    s.set_stream(stream)
    bd = dev(torch, b)
    res = []
    for _ in range(2):
        with torch.cuda.stream(stream):
            x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
        stream.synchronize()
        info = s.solve(bd, x)
        res.append((x.cpu().numpy(), s.history(), info.kernel_launches))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert res[0][2] == res[1][2]
