"""GPU parity of GMRES-IR (FP32 one-reduce cycles inside FP64 restarts) against
the oracle's GMRES-IR and against its FP64 one-reduce GMRES.

Tolerances: both IR solves stop at a true relative residual <= tol = 1e-10, so
their solutions differ by at most ~kappa(A) * 2 tol (kappa of these test
problems is below 1e3): 1e-8 relative. The cycle counts must agree exactly.
Residual estimates inside the first cycle are compared to 2e-2 relative: they
come from FP32 arithmetic on both sides (the oracle's FP32 sums are sequential,
with relative error up to n * 2^-24 ~ 1e-4 per sum at these sizes, amplified
as the cycle proceeds), so only their agreement to FP32 level is meaningful.
"""
import numpy as np
import pytest

from paper_1809_05805_b300 import problems as P

pytestmark = pytest.mark.gpu

CASES = {
    "aniso27_12cubed": (lambda: P.aniso_27pt(12), 40),
    "convdiff7_16cubed": (lambda: P.conv_diff_7pt(16), 30),
    "aniso27_24cubed": (lambda: P.aniso_27pt(24), 40),
}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("use_stream", [False, True])
def test_ir_solve_matches_oracle(torch_cuda, orc, name, use_stream):
    torch = torch_cuda
    from paper_1809_05805_b300 import lsgmres

    make, m = CASES[name]
    A = make()
    xt, b = P.rhs(A, seed=0)
    n = len(b)
    tol = 1e-10
    rir = orc.gmres(A, b, variant=2, m=m, tol=tol, max_iter=3000)
    r64 = orc.gmres(A, b, variant=1, m=m, tol=tol, max_iter=3000)
    s = lsgmres.Solver(A, m=m, tol=tol, prec="ir_fp32", max_iter=3000,
                       stream=torch.cuda.Stream() if use_stream else None)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    info = s.solve(torch.from_numpy(b).cuda(), x)
    h = s.history()
    xg = x.cpu().numpy()
    assert info.status == 0 and rir.status == 0
    assert info.iters == rir.iters and info.restarts == rir.restarts
    true = np.linalg.norm(b - P.to_scipy(A) @ xg) / np.linalg.norm(b)
    assert true <= tol
    assert np.linalg.norm(xg - rir.x) <= 1e-8 * np.linalg.norm(rir.x)
    assert np.linalg.norm(xg - r64.x) <= 1e-8 * np.linalg.norm(r64.x)
    k = min(m, len(h))
    assert np.all(np.abs(h[:k] - rir.history[:k]) <= 2e-2 * rir.history[:k])


def test_ir_graph_path_equals_default_stream(torch_cuda):
    torch = torch_cuda
    from paper_1809_05805_b300 import lsgmres

    A = P.aniso_27pt(14)
    _, b = P.rhs(A, seed=4)
    out = []
    for stream in (None, torch.cuda.Stream()):
        s = lsgmres.Solver(A, m=25, tol=1e-10, prec="ir_fp32", max_iter=2000, stream=stream)
        x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        s.solve(torch.from_numpy(b).cuda(), x)
        out.append((x.cpu().numpy(), s.history()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_ir_argument_checks(torch_cuda):
    from paper_1809_05805_b300 import lsgmres

    A = P.conv_diff_7pt(6)
    s = lsgmres.Solver(A, m=5, tol=1e-8)
    for ortho, prec in (("mgs", "ir_fp32"), ("mgs", "ir_bf16"), ("cgs2_lvl2", "ir_fp32")):
        with pytest.raises(lsgmres.GmresError) as e:
            s.set(ortho=ortho, prec=prec, max_iter=10)
        assert e.value.status == lsgmres.ERR_ARG


BF16_CASES = {
    "aniso27_12cubed": (lambda: P.aniso_27pt(12), 40),
    "convdiff7_16cubed": (lambda: P.conv_diff_7pt(16), 30),
    "aniso27_23cubed": (lambda: P.aniso_27pt(23), 40),  # ragged: 12167 rows
}


@pytest.mark.parametrize("name", sorted(BF16_CASES))
@pytest.mark.parametrize("use_stream", [False, True])
def test_ir_bf16_solve(torch_cuda, orc, name, use_stream):
    """GMRES-IR with BF16 basis storage against the oracle's BF16 variant and its
    FP64 solve. The GPU rounds the unnormalized vector the MAXPY stores, the
    oracle the normalized one (one BF16 rounding per vector each), so results
    agree at BF16 level, not bit for bit: what is unique is the solution to the
    tolerance (x within 1e-8 relative of both oracle solves, true residual
    <= tol); the step count stays within 25% of the oracle's; the first four
    residual estimates (before BF16 rounding dominates the cycle) within 1%.
    Every stored basis value is a BF16 number by construction of the storage
    type."""
    torch = torch_cuda
    from paper_1809_05805_b300 import lsgmres

    make, m = BF16_CASES[name]
    A = make()
    _, b = P.rhs(A, seed=0)
    n = len(b)
    tol = 1e-10
    r16 = orc.gmres(A, b, variant=5, m=m, tol=tol, max_iter=4000)
    r64 = orc.gmres(A, b, variant=1, m=m, tol=tol, max_iter=4000)
    s = lsgmres.Solver(A, m=m, tol=tol, prec="ir_bf16", max_iter=4000,
                       stream=torch.cuda.Stream() if use_stream else None)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    info = s.solve(torch.from_numpy(b).cuda(), x)
    h = s.history()
    xg = x.cpu().numpy()
    assert info.status == 0 and r16.status == 0
    true = np.linalg.norm(b - P.to_scipy(A) @ xg) / np.linalg.norm(b)
    assert true <= tol
    assert np.linalg.norm(xg - r16.x) <= 1e-8 * np.linalg.norm(r16.x)
    assert np.linalg.norm(xg - r64.x) <= 1e-8 * np.linalg.norm(r64.x)
    assert abs(info.iters - r16.iters) <= 0.25 * r16.iters, (info.iters, r16.iters)
    assert np.all(np.abs(h[:4] - r16.history[:4]) <= 1e-2 * r16.history[:4])
