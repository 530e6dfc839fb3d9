"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each function takes an ``oracle.Oracle`` (the real one or a mutant compiled
from an edited copy of oracle.c) and raises AssertionError when the fact fails.
The facts are mathematical (closed forms, textbook routines, invariants of the
algorithms in Sections II and III of the paper) or qualitative statements the
paper makes about its own experiment (Section V-A, tests/golden/).
"""
from __future__ import annotations

import numpy as np

from paper_1809_05805_b300 import problems as P

EPS = np.finfo(np.float64).eps
MGS, ONE_REDUCE, IR_FP32, CGS2, PIPE2, IR_BF16 = 0, 1, 2, 3, 4, 5


def _dense(A):
    return P.to_scipy(A).toarray()


# ---------------------------------------------------------------- kernels
def pin_spmv_dense(orc):
    """CSR matvec equals the dense product (numpy) on a stencil and a random matrix."""
    for A in (P.conv_diff_7pt(5), P.from_dense(P.random_dense(17, seed=3))):
        x = np.random.default_rng(1).standard_normal(len(A[0]) - 1)
        y = orc.spmv(A, x)
        yd = _dense(A) @ x
        assert np.allclose(y, yd, rtol=1e-14, atol=1e-14 * np.abs(yd).max()), "spmv != dense"


def pin_dot_maxpy(orc):
    """orc_dot and orc_maxpy equal the exactly rounded results (math.fsum) within
    the classical recursive-summation bound gamma_n * sum|terms|."""
    import math
    rng = np.random.default_rng(5)
    n = 257
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    exact = math.fsum(x * y)
    assert abs(orc.dot(x, y) - exact) <= n * EPS * np.abs(x * y).sum()
    V = rng.standard_normal((n, 5))
    c = rng.standard_normal(5)
    out = orc.maxpy(V, c, 0.5, y)
    for i in (0, 100, n - 1):
        terms = [0.5 * y[i]] + [c[k] * V[i, k] for k in range(5)]
        assert abs(out[i] - math.fsum(terms)) <= 6 * EPS * sum(abs(t) for t in terms)


# ---------------------------------------------------------------- QR kernels
def pin_qr_reconstructs(orc):
    """Q R = A to rounding for all four Gram-Schmidt variants (backward stability)."""
    A = P.tall_skinny(300, 12, 1e4, seed=2)
    for Q, R in (orc.qr_mgs(A), orc.qr_cgs(A, 1), orc.qr_cgs(A, 2), orc.qr_mgs_lvl2(A)[:2],
                 orc.qr_cgs2_lvl2(A)[:2]):
        assert np.linalg.norm(Q @ R - A) <= 1e-13 * np.linalg.norm(A), "QR != A"
        assert np.allclose(R, np.triu(R)), "R not upper triangular"
        assert np.all(np.diag(R) > 0), "R diagonal not positive"


def pin_lvl2_equals_mgs(orc):
    """Algorithm 4 produces the same Q and R as column MGS (exact arithmetic identity
    of the compact-WY form), and its T equals inv(I + L) computed from its own Q."""
    A = P.tall_skinny(400, 15, 1e3, seed=5)
    Qm, Rm = orc.qr_mgs(A)
    Q2, R2, T2 = orc.qr_mgs_lvl2(A)
    assert np.abs(Q2 - Qm).max() <= 1e-11, "lvl2 Q != MGS Q"
    assert np.abs(R2 - Rm).max() <= 1e-11 * np.abs(Rm).max(), "lvl2 R != MGS R"
    L = np.tril(Q2.T @ Q2, -1)
    Tref = np.linalg.inv(np.eye(A.shape[1]) + L)
    assert np.abs(T2 - Tref).max() <= 1e-12, "T != inv(I + L)"


def _lo(Q):
    k = Q.shape[1]
    return np.linalg.norm(np.eye(k) - Q.T @ Q, 2)


def pin_orthogonality_slopes(orc):
    """Loss of orthogonality grows like eps*kappa for MGS and Algorithm 4 and like
    eps*kappa^2 for CGS-1; CGS with one re-orthogonalization stays near eps."""
    kappas = np.logspace(2, 7, 6)
    lo = {"mgs": [], "lvl2": [], "cgs1": [], "cgs2": []}
    for kap in kappas:
        A = P.tall_skinny(1000, 30, kap, seed=11)
        lo["mgs"].append(_lo(orc.qr_mgs(A)[0]))
        lo["lvl2"].append(_lo(orc.qr_mgs_lvl2(A)[0]))
        lo["cgs1"].append(_lo(orc.qr_cgs(A, 1)[0]))
        lo["cgs2"].append(_lo(orc.qr_cgs(A, 2)[0]))
    lk = np.log10(kappas)
    slope = {k: np.polyfit(lk, np.log10(np.maximum(v, 1e-300)), 1)[0] for k, v in lo.items()}
    assert 0.7 <= slope["mgs"] <= 1.3, f"MGS slope {slope['mgs']}"
    assert 0.7 <= slope["lvl2"] <= 1.3, f"lvl2 slope {slope['lvl2']}"
    assert 1.6 <= slope["cgs1"] <= 2.4, f"CGS-1 slope {slope['cgs1']}"
    assert max(lo["cgs2"]) <= 1e-13, f"CGS-2 loss {max(lo['cgs2'])}"
    # MGS and lvl2 stay O(eps * kappa)
    for v in (lo["mgs"], lo["lvl2"]):
        assert np.all(np.array(v) <= 1e3 * EPS * kappas), "loss above O(eps kappa)"
    return slope


# ---------------------------------------------------------------- GMRES
def pin_arnoldi_relation(orc, N=10, m=25):
    """A V_k = V_{k+1} Hbar_k (Section III) for both variants, to 1e-12 relative."""
    A = P.conv_diff_7pt(N)
    _, b = P.rhs(A, seed=4)
    S = P.to_scipy(A)
    for var in (MGS, ONE_REDUCE):
        r = orc.gmres(A, b, variant=var, m=m, tol=0.0, max_iter=m, capture=True)
        assert r.k == m, "cycle shorter than m"
        AV = S @ r.V[:, : r.k]
        err = np.linalg.norm(AV - r.V @ r.H) / np.linalg.norm(AV)
        assert err <= 1e-12, f"Arnoldi relation {err} (variant {var})"
        # Arnoldi as QR of [r0, A V_m]: V_{m+1}^T r0 = ||r0|| e1 with v_0 = r0/||r0||
        assert abs(np.linalg.norm(r.V[:, 0]) - 1.0) < 1e-14
        assert np.allclose(np.triu(r.H, -1), r.H), "H not upper Hessenberg"


def pin_equivalence(orc, N=12, m=20):
    """One-reduce and MGS-GMRES coincide on a well-conditioned problem (Section V-A:
    identical convergence; exact-arithmetic identity T = I when V^T V = I)."""
    A = P.conv_diff_7pt(N)
    _, b = P.rhs(A, seed=6)
    rm = orc.gmres(A, b, variant=MGS, m=m, tol=1e-10, max_iter=200, capture=True)
    r1 = orc.gmres(A, b, variant=ONE_REDUCE, m=m, tol=1e-10, max_iter=200, capture=True)
    assert rm.iters == r1.iters and rm.restarts == r1.restarts, "iteration counts differ"
    # first cycle: relative agreement; later cycles restart from a residual ~tol*||b||,
    # so rounding in x shows up there at the ||b||*eps scale (history is relative to ||b||)
    rel = np.abs(rm.history[:m] - r1.history[:m]) / rm.history[:m]
    assert rel.max() <= 1e-12, f"first-cycle histories differ {rel.max()}"
    assert np.abs(rm.history - r1.history).max() <= 1e-14, "histories differ"
    assert np.abs(rm.V - r1.V).max() <= 1e-11, "bases differ"
    assert np.abs(rm.H - r1.H).max() <= 1e-11 * np.abs(rm.H).max(), "Hessenbergs differ"
    L = np.tril(r1.V.T @ r1.V, -1)
    Tref = np.linalg.inv(np.eye(r1.V.shape[1]) + L)
    assert np.abs(r1.T - Tref).max() <= 1e-13, "T != inv(I + L)"
    assert np.linalg.norm(rm.x - r1.x) <= 1e-8 * np.linalg.norm(rm.x)


def pin_compact_wy_coefficients(orc, m=60):
    """Compact-WY identity (Section II): for a basis with unit columns, the product
    of MGS rank-1 projectors equals I - V T V^T with T = inv(I + L). So each
    Hessenberg column must equal the coefficients of a sequential MGS sweep of
    A v_j over the same computed basis, even after V has lost orthogonality.
    Checked on the ill-conditioned Simoncini-Szyld matrix, where a projection that
    skips T (classical GS) visibly departs from MGS."""
    A, b = P.simoncini_szyld(100, seed=0)
    M = _dense(A)
    for var in (MGS, ONE_REDUCE):
        r = orc.gmres(A, b, variant=var, m=m, tol=0.0, max_iter=m, capture=True)
        V, H = r.V, r.H
        worst = 0.0
        for j in range(r.k):
            z = M @ V[:, j]
            h = np.zeros(j + 1)
            for k in range(j + 1):
                h[k] = V[:, k] @ z
                z = z - h[k] * V[:, k]
            worst = max(worst, np.abs(h - H[: j + 1, j]).max() / np.abs(H[: j + 2, j]).max())
        assert worst <= 1e-13, f"variant {var}: Hessenberg != MGS coefficients ({worst})"


def pin_direct_solve(orc):
    """GMRES(n) on an n x n system is a direct solve: x equals numpy's LU solve."""
    for n, seed in ((6, 1), (13, 2), (20, 3)):
        M = P.random_dense(n, seed=seed)
        A = P.from_dense(M)
        b = np.random.default_rng(seed).standard_normal(n)
        xref = np.linalg.solve(M, b)
        kap = np.linalg.cond(M)
        for var in (MGS, ONE_REDUCE, CGS2, PIPE2):
            r = orc.gmres(A, b, variant=var, m=n, tol=1e-15, max_iter=n)
            err = np.linalg.norm(r.x - xref) / np.linalg.norm(xref)
            assert err <= 1e-12 * kap, f"n={n} var={var} err={err}"


def pin_krylov_minimum(orc):
    """After k steps the residual equals min over x in K_k of ||b - A x|| (the
    definition of GMRES), computed by brute-force least squares over an
    orthonormalized Krylov matrix [b, Ab, ..., A^{k-1} b] (numpy QR + lstsq)."""
    n, kmax = 40, 8
    M = P.random_dense(n, seed=8, shift=3.0)
    A = P.from_dense(M)
    b = np.random.default_rng(9).standard_normal(n)
    K = np.empty((n, kmax))
    v = b / np.linalg.norm(b)
    for k in range(kmax):
        K[:, k] = v
        v = M @ v
        v /= np.linalg.norm(v)
    ref = []
    for k in range(1, kmax + 1):
        Qk, _ = np.linalg.qr(K[:, :k])
        y, *_ = np.linalg.lstsq(M @ Qk, b, rcond=None)
        ref.append(np.linalg.norm(b - M @ (Qk @ y)) / np.linalg.norm(b))
    ref = np.array(ref)
    for var in (MGS, ONE_REDUCE, CGS2, PIPE2):
        r = orc.gmres(A, b, variant=var, m=kmax, tol=0.0, max_iter=kmax)
        assert np.allclose(r.history[:kmax], ref, rtol=1e-9, atol=1e-15), f"var {var}: {r.history} vs {ref}"
        # the solution after the cycle realizes the last minimum
        assert abs(np.linalg.norm(b - M @ r.x) / np.linalg.norm(b) - ref[-1]) <= 1e-9 * ref[-1] + 1e-15


def pin_finite_termination(orc):
    """A diagonalizable matrix with d distinct eigenvalues has a minimal polynomial
    of degree d, so GMRES reaches the solution after d steps."""
    M = P.distinct_eigs(40, [1.0, 2.5, 4.0], seed=2)
    A = P.from_dense(M)
    b = np.random.default_rng(3).standard_normal(40)
    for var in (MGS, ONE_REDUCE, CGS2, PIPE2):
        r = orc.gmres(A, b, variant=var, m=10, tol=1e-12, max_iter=10)
        assert r.iters == 3, f"var {var}: {r.iters} steps"
        assert r.history[1] > 1e-6 and r.rel_resid_true <= 1e-12


def pin_explicit_residual(orc, N=16):
    """At exit the reported true residual is ||b - A x|| / ||b|| (numpy) and below tol."""
    A = P.conv_diff_7pt(N)
    xt, b = P.rhs(A, seed=0)
    S = P.to_scipy(A)
    for var in (MGS, ONE_REDUCE):
        r = orc.gmres(A, b, variant=var, m=30, tol=1e-8, max_iter=300)
        true = np.linalg.norm(b - S @ r.x) / np.linalg.norm(b)
        assert r.status == 0 and true <= 1e-8
        assert abs(true - r.rel_resid_true) <= 1e-12 * max(true, 1e-300) + 1e-18


def pin_reduction_counts(orc):
    """Global reductions: MGS-GMRES makes i+1 inner products plus a norm at step i
    (Section IV); the one-reduce variant makes one per step plus one per cycle tail.
    Both add one norm for ||b|| and one per true-residual check."""
    A = P.conv_diff_7pt(8)
    _, b = P.rhs(A, seed=1)
    m, it = 7, 20  # cycles of 7, 7, 6 steps with tol = 0
    rm = orc.gmres(A, b, variant=MGS, m=m, tol=0.0, max_iter=it)
    r1 = orc.gmres(A, b, variant=ONE_REDUCE, m=m, tol=0.0, max_iter=it)
    cycles = [7, 7, 6]
    base = 1 + (len(cycles) + 1)  # ||b||, one true residual per cycle start + the final one
    exp_mgs = base + sum(sum(i + 2 for i in range(k)) for k in cycles)
    exp_1r = base + sum(k + 1 for k in cycles)
    assert rm.iters == r1.iters == 20
    assert rm.reductions == exp_mgs, (rm.reductions, exp_mgs)
    assert r1.reductions == exp_1r, (r1.reductions, exp_1r)


def pin_ir_refines_to_fp64_accuracy(orc):
    """GMRES-IR (FP32 cycles, FP64 residual and update) reaches a true relative
    residual of 1e-12 -- far below FP32 rounding -- and its x equals a dense LU
    solve (numpy) within the conditioning bound."""
    for A in (P.aniso_27pt(7), P.conv_diff_7pt(7)):
        xt, b = P.rhs(A, seed=2)
        D = _dense(A)
        xref = np.linalg.solve(D, b)
        kap = np.linalg.cond(D)
        r = orc.gmres(A, b, variant=IR_FP32, m=30, tol=1e-12, max_iter=2000)
        assert r.status == 0
        true = np.linalg.norm(b - D @ r.x) / np.linalg.norm(b)
        assert true <= 1e-12, true
        assert np.linalg.norm(r.x - xref) <= 10 * kap * 1e-12 * np.linalg.norm(xref)


def pin_ir_cycle_is_fp32(orc):
    """The IR cycle runs in FP32: its first-cycle residual estimates and Arnoldi
    relation agree with the FP64 one-reduce cycle at FP32 level (well above
    FP64 rounding, well below the quantities themselves)."""
    A = P.aniso_27pt(8)
    _, b = P.rhs(A, seed=3)
    m = 20
    r64 = orc.gmres(A, b, variant=ONE_REDUCE, m=m, tol=0.0, max_iter=m, capture=True)
    r32 = orc.gmres(A, b, variant=IR_FP32, m=m, tol=0.0, max_iter=m, capture=True)
    rel = np.abs(r32.history - r64.history) / r64.history
    assert 1e-10 < rel.max() < 1e-3, rel.max()
    S = P.to_scipy(A)
    AV = S @ r32.V[:, : r32.k]
    err = np.linalg.norm(AV - r32.V @ r32.H) / np.linalg.norm(AV)
    assert 1e-10 < err < 1e-5, err


def pin_cgs2_lvl2_qr(orc):
    """Algorithm 5 (iterated CGS with lagged normalization): the paper states its
    columns are orthogonal to machine precision; so ||I - Q^T Q|| stays O(eps)
    for kappa up to 1e12 while MGS loses eps*kappa. Q R = A to rounding; on a
    well-conditioned matrix Q and R equal column MGS's (exact-arithmetic
    identity of the two projections), and T = inv(I + L) is the identity to
    rounding because the re-orthogonalized columns are orthogonal."""
    for kap in (1e2, 1e6, 1e10, 1e12):
        A = P.tall_skinny(1000, 30, kap, seed=11)
        Q, R, T = orc.qr_cgs2_lvl2(A)
        assert _lo(Q) <= 1e-13, f"kappa {kap}: loss {_lo(Q)}"
        assert np.linalg.norm(Q @ R - A) <= 1e-13 * np.linalg.norm(A)
        assert np.abs(T - np.eye(30)).max() <= 1e-12
    assert _lo(orc.qr_mgs(P.tall_skinny(1000, 30, 1e12, seed=11))[0]) >= 1e-6  # the contrast
    A = P.tall_skinny(400, 15, 1e3, seed=5)
    Qm, Rm = orc.qr_mgs(A)
    Q2, R2, _ = orc.qr_cgs2_lvl2(A)
    assert np.abs(Q2 - Qm).max() <= 1e-11 and np.abs(R2 - Rm).max() <= 1e-11 * np.abs(Rm).max()


def pin_cgs2_gmres(orc):
    """GMRES with Algorithm 5's two-reduction orthogonalization: on the
    Simoncini-Szyld problem, where one-reduce loses orthogonality completely by
    step 80, its basis stays orthonormal to 1e-13, its Hessenberg equals
    V^T A V_k (the Galerkin identity of an orthonormal Arnoldi basis) and the
    Arnoldi relation holds; on a well-conditioned problem it coincides with
    MGS-GMRES; a cycle of k steps makes 2k + 1 reductions."""
    A, b = P.simoncini_szyld(100, seed=0)
    M = _dense(A)
    r = orc.gmres(A, b, variant=CGS2, m=80, tol=0.0, max_iter=80, capture=True)
    r1 = orc.gmres(A, b, variant=ONE_REDUCE, m=80, tol=0.0, max_iter=80, capture=True)
    V = r.V[:, : r.k]
    assert _lo(V) <= 1e-13, _lo(V)
    assert _lo(r1.V[:, : r1.k]) >= 1e-3  # the contrast
    G = r.V.T @ M @ V
    assert np.abs(G - r.H).max() <= 1e-13 * np.abs(r.H).max()
    assert np.linalg.norm(M @ V - r.V @ r.H) <= 1e-12 * np.linalg.norm(M @ V)
    A = P.conv_diff_7pt(12)
    _, b = P.rhs(A, seed=6)
    rm = orc.gmres(A, b, variant=MGS, m=20, tol=1e-10, max_iter=200)
    rc = orc.gmres(A, b, variant=CGS2, m=20, tol=1e-10, max_iter=200)
    assert rm.iters == rc.iters and rm.restarts == rc.restarts
    assert np.all(np.abs(rm.history[:20] - rc.history[:20]) <= 1e-12 * rm.history[:20])
    A = P.conv_diff_7pt(8)
    _, b = P.rhs(A, seed=1)
    rc = orc.gmres(A, b, variant=CGS2, m=7, tol=0.0, max_iter=20)
    cycles = [7, 7, 6]
    assert rc.reductions == 1 + (len(cycles) + 1) + sum(2 * k + 1 for k in cycles), rc.reductions


def pin_pipeline(orc):
    """The L = 2 pipeline (Algorithm 8) changes only when the Givens rotations
    are applied: with a fixed step count its basis, Hessenberg, T and residual
    estimates are bit for bit those of one-reduce; with a tolerance it sees
    convergence only after an even column (or column 0), so a single-cycle
    solve that one-reduce ends after k steps ends after k steps when k - 1 is
    even and after k + 1 steps otherwise."""
    A = P.conv_diff_7pt(10)
    _, b = P.rhs(A, seed=4)
    r1 = orc.gmres(A, b, variant=ONE_REDUCE, m=25, tol=0.0, max_iter=25, capture=True)
    rp = orc.gmres(A, b, variant=PIPE2, m=25, tol=0.0, max_iter=25, capture=True)
    for a, c in ((r1.V, rp.V), (r1.H, rp.H), (r1.T, rp.T), (r1.history, rp.history)):
        assert np.array_equal(a, c), "pipeline changed the arithmetic"
    seen_odd = False
    for seed in range(8):
        A = P.conv_diff_7pt(9)
        _, b = P.rhs(A, seed=seed)
        tol = 10.0 ** (-4 - seed % 4)
        r1 = orc.gmres(A, b, variant=ONE_REDUCE, m=200, tol=tol, max_iter=200)
        rp = orc.gmres(A, b, variant=PIPE2, m=200, tol=tol, max_iter=200)
        assert r1.restarts == rp.restarts == 1
        k1 = r1.iters
        want = k1 if (k1 - 1) % 2 == 0 or k1 == 1 else k1 + 1
        seen_odd |= want != k1
        assert rp.iters == want, (seed, k1, rp.iters)
        assert rp.rel_resid_true <= tol
    assert seen_odd, "no case where the pipeline needs the extra step"


def pin_bf16_rounding(orc):
    """The oracle's FP32 -> BF16 rounding equals torch's (round to nearest,
    ties to even) on random values, exact ties, powers of two and values near
    the largest finite BF16."""
    import torch

    rng = np.random.default_rng(13)
    x = np.concatenate([rng.standard_normal(4000).astype(np.float32) * np.float32(10.0) ** rng.integers(-8, 8, 4000),
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 2.0 ** -126, 0.0,
                                  3.3895e38, -1.5], dtype=np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    got = orc.round_bf16(x)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), "BF16 rounding differs"


def pin_ir_bf16(orc):
    """GMRES-IR with the basis stored in BF16: every stored basis value is a
    BF16 number (low 16 bits of its FP32 word zero); the solve still reaches a
    true relative residual of 1e-10 with x equal to a dense LU solve within
    the conditioning bound; and the first steps' residual estimates agree with
    FP64 at BF16 level (well above FP32 rounding, below 1%)."""
    A = P.aniso_27pt(8)
    _, b = P.rhs(A, seed=3)
    m = 20
    r64 = orc.gmres(A, b, variant=ONE_REDUCE, m=m, tol=0.0, max_iter=m, capture=True)
    r16 = orc.gmres(A, b, variant=IR_BF16, m=m, tol=0.0, max_iter=m, capture=True)
    V = r16.V.astype(np.float32)
    assert np.array_equal(V.astype(np.float64), r16.V), "basis not FP32-representable"
    assert np.all((V.view(np.uint32) & 0xFFFF) == 0), "basis value not a BF16 number"
    # over the first 8 steps (before BF16 rounding in the basis dominates the
    # small residual): above FP32 rounding (~1e-6 here), below 1%
    rel = np.abs(r16.history[:8] - r64.history[:8]) / r64.history[:8]
    assert 2e-5 < rel.max() < 1e-2, rel.max()
    for A in (P.aniso_27pt(7), P.conv_diff_7pt(7)):
        _, b = P.rhs(A, seed=2)
        D = _dense(A)
        xref = np.linalg.solve(D, b)
        r = orc.gmres(A, b, variant=IR_BF16, m=30, tol=1e-10, max_iter=3000)
        assert r.status == 0
        assert np.linalg.norm(b - D @ r.x) / np.linalg.norm(b) <= 1e-10
        assert np.linalg.norm(r.x - xref) <= 10 * np.linalg.cond(D) * 1e-10 * np.linalg.norm(xref)


def simoncini_szyld_run(orc, variant):
    A, b = P.simoncini_szyld(100, seed=0)
    return orc.gmres(A, b, variant=variant, m=100, tol=0.0, max_iter=100, capture=True)


def paige_S_norm(V):
    """Paige's loss-of-orthogonality measure ||S||_2, S = (I + L^T)^{-1} L^T, with L
    the strictly lower part of V^T V (Section II)."""
    k = V.shape[1]
    L = np.tril(V.T @ V, -1)
    S = np.linalg.solve(np.eye(k) + L.T, L.T)
    return np.linalg.norm(S, 2)


PINS = [
    pin_spmv_dense,
    pin_dot_maxpy,
    pin_qr_reconstructs,
    pin_lvl2_equals_mgs,
    pin_arnoldi_relation,
    pin_equivalence,
    pin_compact_wy_coefficients,
    pin_direct_solve,
    pin_krylov_minimum,
    pin_finite_termination,
    pin_explicit_residual,
    pin_reduction_counts,
    pin_ir_refines_to_fp64_accuracy,
    pin_ir_cycle_is_fp32,
    pin_cgs2_lvl2_qr,
    pin_cgs2_gmres,
    pin_pipeline,
    pin_bf16_rounding,
    pin_ir_bf16,
]
