"""CPU pins of the FP64 oracle (no GPU). Each pin checks the oracle against a fact
that does not come from the oracle: closed forms, numpy/LAPACK routines, brute
force, or the paper's own qualitative statements (tests/golden/)."""
import os

import numpy as np
import pytest

import pins
from paper_1809_05805_b300 import problems as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("pin", pins.PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    pin(orc)


def test_orthogonality_slopes(orc):
    slope = pins.pin_orthogonality_slopes(orc)
    assert slope["cgs1"] > slope["mgs"] + 0.5


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_simoncini_szyld_limiting_accuracy(orc):
    """Section V-A, first problem: MGS and one-reduce MGS-GMRES behave identically,
    ||S||_2 rises to ~1 and the residual stalls near 1e-7 around iteration 80."""
    g = _golden("simoncini_szyld_e1.txt")
    runs = {v: pins.simoncini_szyld_run(orc, v) for v in (pins.MGS, pins.ONE_REDUCE)}
    for v, r in runs.items():
        h = r.history
        assert len(h) == 100
        floor = h.min()
        band = 10 ** g["stall_band_decades"]
        assert g["stall_residual"] / band <= floor <= g["stall_residual"] * band, (v, floor)
        # the stall: after the floor is first reached within 2x, no further decade of progress
        first = int(np.argmax(h <= 2 * floor))
        assert abs(first - g["stall_iteration"]) <= g["iteration_band"], (v, first)
        assert h[first:].min() >= floor
        # Paige's ||S||_2: near eps early, near one at the stall
        s_early = pins.paige_S_norm(r.V[:, :30])
        s_late = pins.paige_S_norm(r.V[:, : first + 10])
        assert s_early < 1e-6, (v, s_early)
        assert s_late > 0.5 * g["S_norm_at_stall"], (v, s_late)
    # identical convergence until orthogonality is lost
    hm, h1 = runs[pins.MGS].history, runs[pins.ONE_REDUCE].history
    pre = hm > 1e-5
    assert np.all(np.abs(hm[pre] - h1[pre]) <= 1e-6 * hm[pre])


def test_nonfinite_rhs_is_reported(orc):
    A = P.conv_diff_7pt(4)
    _, b = P.rhs(A, seed=0)
    b[3] = np.nan
    r = orc.gmres(A, b, variant=1, m=5, tol=1e-8, max_iter=10)
    assert r.status == -3


def test_zero_rhs_gives_zero(orc):
    A = P.conv_diff_7pt(4)
    r = orc.gmres(A, np.zeros(64), variant=1, m=5, tol=1e-8, max_iter=10, x0=np.ones(64))
    assert r.status == 0 and np.all(r.x == 0)


def test_maxiter_status(orc):
    A = P.conv_diff_7pt(8)
    _, b = P.rhs(A, seed=0)
    r = orc.gmres(A, b, variant=1, m=5, tol=1e-14, max_iter=12)
    assert r.status == 1 and r.iters == 12 and r.restarts == 3


def test_generator_stencil_structure():
    """The 7-point generator: nnz = 7N^3 - 6N^2, sorted columns, the upwind
    coefficients, and a diagonally dominant M-matrix sign pattern."""
    N = 6
    rowptr, col, val = P.conv_diff_7pt(N)
    assert len(col) == P.grid7_nnz(N) == rowptr[-1]
    for i in range(N ** 3):
        c = col[rowptr[i]:rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    D = P.to_scipy((rowptr, col, val)).toarray()
    assert np.allclose(np.diag(D), 6.875)
    i = 1 + N + N * N  # interior point
    assert np.isclose(D[i, i - 1], -1.5) and np.isclose(D[i, i + 1], -1.0)
    assert np.isclose(D[i, i - N], -1.25) and np.isclose(D[i, i - N * N], -1.125)
    off = D - np.diag(np.diag(D))
    assert np.all(off <= 0) and np.all(np.diag(D) >= -off.sum(axis=1))


def test_generator_27pt_equals_kronecker_definition():
    """The 27-point generator equals k_x T(x)M(x)M + k_y M(x)T(x)M + k_z M(x)M(x)T built
    with scipy's Kronecker products; it is symmetric positive definite."""
    import scipy.sparse as sp

    N = 5
    k = (1.0, 1.0, 1e-3)
    A = P.aniso_27pt(N, k)
    assert len(A[1]) == P.grid27_nnz(N)
    Tm = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(N, N))
    Mm = sp.diags([1.0, 4.0, 1.0], [-1, 0, 1], shape=(N, N)) / 6.0
    ref = (k[0] * sp.kron(sp.kron(Mm, Mm), Tm) + k[1] * sp.kron(sp.kron(Mm, Tm), Mm)
           + k[2] * sp.kron(sp.kron(Tm, Mm), Mm)).toarray()
    D = P.to_scipy(A).toarray()
    assert np.allclose(D, ref, rtol=0, atol=1e-15)
    assert np.allclose(D, D.T) and np.linalg.eigvalsh(D).min() > 0
    for i in range(N ** 3):
        c = A[1][A[0][i]:A[0][i + 1]]
        assert np.all(np.diff(c) > 0)


def test_generator_9pt_2d():
    """With kappa = 1 and no convection the 2D generator is the bilinear stiffness
    T (x) M + M (x) T (scipy Kronecker products); the full operator has at most 9
    entries per row, sorted columns, and a positive definite symmetric part."""
    import scipy.sparse as sp

    N = 6
    A = P.conv_diff_9pt_2d(N, np.ones((N + 1, N + 1)), 0.0, 0.3)
    Tm = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(N, N))
    Mm = sp.diags([1.0, 4.0, 1.0], [-1, 0, 1], shape=(N, N)) / 6.0
    ref = (sp.kron(Mm, Tm) + sp.kron(Tm, Mm)).toarray()
    assert np.allclose(P.to_scipy(A).toarray(), ref, atol=1e-15)
    par = P.batch_2d_params(3, seed=1, side=(16, 20))[0]
    B = P.batch_2d_system(par)
    assert np.diff(B[0]).max() <= 9
    D = P.to_scipy(B).toarray()
    assert np.linalg.eigvalsh(0.5 * (D + D.T)).min() > 0
    for i in range(len(B[0]) - 1):
        assert np.all(np.diff(B[1][B[0][i]:B[0][i + 1]]) > 0)
