"""GPU tests of the serving loop (gmres_server_*): continuous batching of FP64
and GMRES-IR requests of mixed sizes under a device byte budget.

Every request is checked against the oracle solving it alone at the bar of a
single solve (FP64: identical iteration and restart counts, x within 1e-9
relative; GMRES-IR: identical iteration and restart counts, x within 1e-8
relative of the oracle's GMRES-IR and of its FP64 solve), and against the same
request served alone (same counts, same x within those bars): its result must
not depend on which requests shared its launches beyond the order of partial
sums. Requests arrive from another thread while earlier ones iterate.
"""
import threading
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


def _requests(count, seed, sides=(6, 22), ir_frac=0.3):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.integers(sides[0], sides[1] + 1))
        A = P.conv_diff_7pt(N)
        _, b = P.rhs(A, seed=seed * 100 + i)
        out.append((A, b, "ir_fp32" if rng.random() < ir_frac else "fp64"))
    return out


def _serve(lsg, reqs, tol, m=20, max_iter=3000, budget=256 << 20, max_requests=8, gap_s=0.002):
    sv = lsg.Server(m=m, max_iter=max_iter, max_requests=max_requests, hbm_budget_bytes=budget, ir_share=0.4)
    xs = [np.zeros(len(b)) for _, b, _ in reqs]
    ids = [None] * len(reqs)

    def feed():
        for i, (A, b, prec) in enumerate(reqs):
            ids[i] = sv.submit(A, b, xs[i], tol=tol, prec=prec)
            time.sleep(gap_s)

    th = threading.Thread(target=feed)
    th.start()
    th.join()
    sv.drain(timeout=300)
    infos = [sv.wait(i, timeout=10) for i in ids]
    return sv, infos, xs


def test_server_mixed_requests_match_oracle_and_alone(torch_cuda, lsg, orc):
    reqs = _requests(14, seed=3)
    tol = 1e-8
    sv, infos, xs = _serve(lsg, reqs, tol)
    st = sv.stats()
    assert st["completed"][0] + st["completed"][1] == len(reqs)
    assert len(sv.latencies()) == len(reqs)
    sv.close()
    for (A, b, prec), info, x in zip(reqs, infos, xs):
        assert info.status == 0
        true = np.linalg.norm(b - P.to_scipy(A) @ x) / np.linalg.norm(b)
        assert true <= tol
        if prec == "fp64":
            r = orc.gmres(A, b, variant=1, m=20, tol=tol, max_iter=3000)
            assert info.iters == r.iters and info.restarts == r.restarts
            assert np.linalg.norm(x - r.x) <= 1e-9 * np.linalg.norm(r.x)
        else:
            r = orc.gmres(A, b, variant=2, m=20, tol=tol, max_iter=3000)
            r64 = orc.gmres(A, b, variant=1, m=20, tol=tol, max_iter=3000)
            assert info.iters == r.iters and info.restarts == r.restarts
            assert np.linalg.norm(x - r.x) <= 1e-8 * np.linalg.norm(r.x)
            assert np.linalg.norm(x - r64.x) <= 1e-8 * np.linalg.norm(r64.x)
    # each request served alone
    for k, (A, b, prec) in enumerate(reqs[:6]):
        sv1, inf1, xs1 = _serve(lsg, [(A, b, prec)], tol)
        sv1.close()
        assert inf1[0].iters == infos[k].iters and inf1[0].restarts == infos[k].restarts
        bar = 1e-9 if prec == "fp64" else 1e-8
        assert np.linalg.norm(xs1[0] - xs[k]) <= bar * np.linalg.norm(xs1[0])


def test_server_admission_by_budget(torch_cuda, lsg):
    """A budget that holds only a few of the requests at once: the rest queue
    and are admitted as earlier ones complete; the bytes occupied never exceed
    the engine's allocation; every request completes and converges."""
    reqs = [(A, b, "fp64") for A, b, _ in _requests(10, seed=5, sides=(24, 28))]
    # FP64 engine: ~18 MB (basis, its limbs, CSR) -> room for one or two 24^3..28^3 requests (m = 20)
    sv, infos, xs = _serve(lsg, reqs, 1e-8, budget=int(18e6 / 0.6), max_requests=8, gap_s=0.0)
    st = sv.stats()
    sv.close()
    assert st["completed"][0] == 10 and st["rejected"] == 0
    assert 1 <= st["peak_running"][0] < 10
    assert st["peak_bytes_in_use"][0] <= st["engine_bytes"][0]
    for (A, b, _), info, x in zip(reqs, infos, xs):
        assert info.status == 0
        assert np.linalg.norm(b - P.to_scipy(A) @ x) <= 1e-8 * np.linalg.norm(b)


def test_server_rejects_oversize_and_bad_input(torch_cuda, lsg):
    sv = lsg.Server(m=10, max_iter=200, max_requests=4, hbm_budget_bytes=8 << 20, ir_share=0.5)
    A = P.conv_diff_7pt(40)  # 64,000 rows: more than a 4 MB engine holds
    b = np.ones(len(A[0]) - 1)
    with pytest.raises(lsg.GmresError) as e:
        sv.submit(A, b, np.zeros_like(b), tol=1e-8)
    assert e.value.status == lsg.ERR_OOM
    bad = (np.array([0, 2, 1], np.int32), np.array([0, 1], np.int32), np.array([1.0, 2.0]))
    with pytest.raises(lsg.GmresError) as e:
        sv.submit(bad, np.ones(2), np.zeros(2), tol=1e-8)
    assert e.value.status == lsg.ERR_ARG
    with pytest.raises(lsg.GmresError):
        sv.submit(P.conv_diff_7pt(4), np.ones(64), np.zeros(64), tol=1e-8, max_iter=10 ** 6)
    assert sv.stats()["rejected"] == 1
    # a column index out of range is found at admission: the request completes with ERR_ARG
    rp, cl, vl = (a.copy() for a in P.conv_diff_7pt(4))
    cl[10] = 64
    rid = sv.submit((rp, cl, vl), np.ones(64), np.zeros(64), tol=1e-8)
    assert sv.wait(rid, timeout=30).status == lsg.ERR_ARG
    sv.close()


def test_server_edge_requests_and_device_buffers(torch_cuda, lsg):
    """Zero and NaN right-hand sides complete with their own status; b and
    x_out may be CUDA tensors."""
    torch = torch_cuda
    sv = lsg.Server(m=15, max_iter=500, max_requests=4, hbm_budget_bytes=64 << 20, ir_share=0.5)
    A = P.conv_diff_7pt(10)
    n = len(A[0]) - 1
    _, b = P.rhs(A, seed=1)
    bz = np.zeros(n)
    bn = b.copy()
    bn[5] = np.nan
    xz, xn = np.ones(n), np.zeros(n)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    ids = [sv.submit(A, bz, xz, tol=1e-8), sv.submit(A, bn, xn, tol=1e-8, prec="ir_fp32"),
           sv.submit(A, bd, xd, tol=1e-8)]
    sv.drain(timeout=60)
    iz, inan, idev = (sv.wait(i, timeout=5) for i in ids)
    assert iz.status == 0 and iz.iters == 0 and np.all(xz == 0.0)
    assert inan.status == lsg.ERR_NONFINITE
    assert idev.status == 0
    x = xd.cpu().numpy()
    assert np.linalg.norm(b - P.to_scipy(A) @ x) <= 1e-8 * np.linalg.norm(b)
    sv.close()
