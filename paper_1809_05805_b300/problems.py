"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module builds problem data only: CSR matrices of the stencil problems,
right-hand sides, and small dense test matrices. It contains none of the
solver's arithmetic (no Gram-Schmidt, Arnoldi, Givens or least squares), and it
imports neither the CUDA library nor the oracle, so both sides can consume the
same inputs without sharing code.

All CSR matrices are ``(rowptr int32[n+1], col int32[nnz], val float64[nnz])``
with columns sorted ascending inside each row.

The stencil problems stand in for the paper's CFD matrices (Nalu V27, ~11
nonzeros per row; parabolic_fem, ~7 per row), which are not available here.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

CSR = tuple  # (rowptr, col, val)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# 3D 7-point convection-diffusion
# --------------------------------------------------------------------------
def conv_diff_7pt(N: int, peclet=(0.5, 0.25, 0.125)) -> CSR:
    """Upwinded 3D convection-diffusion on the N^3 interior points of a unit cube.

    The equation -Laplace(u) + b . grad(u) = f is scaled by h^2 (diffusion 1).
    First-order upwinding of a velocity with positive components and per-axis
    cell Peclet numbers ``p_a = b_a h`` gives, along each axis, the coefficients
    ``-(1 + p_a)`` for the upwind (lower-index) neighbour, ``-1`` for the
    downwind neighbour and ``2 + p_a`` on the diagonal. The default velocity
    direction (1, 0.5, 0.25) at cell Peclet 0.5 gives p = (0.5, 0.25, 0.125).
    Dirichlet boundary values are eliminated, so there are N^3 unknowns and
    7 N^3 - 6 N^2 nonzeros. Unknowns are ordered x fastest, then y, then z.
    """
    N = int(N)
    n = N ** 3
    px, py, pz = (float(p) for p in peclet)
    idx = np.arange(n, dtype=np.int64)
    ix = idx % N
    iy = (idx // N) % N
    iz = idx // (N * N)
    # entries in ascending column order: -N^2, -N, -1, 0, +1, +N, +N^2
    offs = np.array([-N * N, -N, -1, 0, 1, N, N * N], dtype=np.int64)
    vals = np.array([-(1 + pz), -(1 + py), -(1 + px), 6.0 + px + py + pz, -1.0, -1.0, -1.0])
    valid = np.empty((n, 7), dtype=bool)
    valid[:, 0] = iz > 0
    valid[:, 1] = iy > 0
    valid[:, 2] = ix > 0
    valid[:, 3] = True
    valid[:, 4] = ix < N - 1
    valid[:, 5] = iy < N - 1
    valid[:, 6] = iz < N - 1
    del ix, iy, iz
    counts = valid.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    cols = (idx[:, None] + offs[None, :])[valid].astype(np.int32)
    v = np.broadcast_to(vals, (n, 7))[valid].astype(np.float64)
    return rowptr.astype(np.int32), cols, v


def grid7_nnz(N: int) -> int:
    return 7 * N ** 3 - 6 * N ** 2


# --------------------------------------------------------------------------
# 3D 27-point anisotropic diffusion (trilinear finite elements)
# --------------------------------------------------------------------------
def aniso_27pt(N: int, k=(1.0, 1.0, 1e-3)) -> CSR:
    """Stiffness matrix of -div(diag(k) grad u) with trilinear (Q1) elements on a
    uniform N^3 interior grid of the unit cube, Dirichlet boundary eliminated:

        A = k_x T (x) M (x) M + k_y M (x) T (x) M + k_z M (x) M (x) T

    (x fastest), with the 1D stiffness T = tridiag(-1, 2, -1) and the 1D mass
    M = tridiag(1, 4, 1) / 6, the common factor h dropped. Symmetric positive
    definite, 27 nonzeros per interior row, (3N - 2)^3 nonzeros in total.
    """
    N = int(N)
    n = N ** 3
    kx, ky, kz = (float(v) for v in k)
    T = {-1: -1.0, 0: 2.0, 1: -1.0}
    M = {-1: 1.0 / 6.0, 0: 4.0 / 6.0, 1: 1.0 / 6.0}
    idx = np.arange(n, dtype=np.int64)
    ix = idx % N
    iy = (idx // N) % N
    iz = idx // (N * N)
    offs, vals, masks = [], [], []
    for dz in (-1, 0, 1):  # ascending column order: dz, then dy, then dx
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                offs.append(dz * N * N + dy * N + dx)
                vals.append(kx * T[dx] * M[dy] * M[dz] + ky * M[dx] * T[dy] * M[dz] + kz * M[dx] * M[dy] * T[dz])
                ok = np.ones(n, dtype=bool)
                for d, i in ((dx, ix), (dy, iy), (dz, iz)):
                    if d < 0:
                        ok &= i > 0
                    elif d > 0:
                        ok &= i < N - 1
                masks.append(ok)
    del ix, iy, iz
    valid = np.stack(masks, axis=1)
    del masks
    counts = valid.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    cols = (idx[:, None] + np.array(offs, dtype=np.int64)[None, :])[valid].astype(np.int32)
    v = np.broadcast_to(np.array(vals), (n, 27))[valid].astype(np.float64)
    return rowptr.astype(np.int32), cols, v


def grid27_nnz(N: int) -> int:
    return (3 * N - 2) ** 3


# --------------------------------------------------------------------------
# 2D 9-point variable-coefficient convection-diffusion (batched workload)
# --------------------------------------------------------------------------
# Bilinear (Q1) element stiffness of -div(kappa grad u) on a unit square cell
# with constant kappa, corners ordered (0,0), (1,0), (1,1), (0,1).
_Q1_K = np.array([[4.0, -1.0, -2.0, -1.0],
                  [-1.0, 4.0, -1.0, -2.0],
                  [-2.0, -1.0, 4.0, -1.0],
                  [-1.0, -2.0, -1.0, 4.0]]) / 6.0


def conv_diff_9pt_2d(N: int, kappa_cells: np.ndarray, peclet: float, theta: float) -> CSR:
    """-div(kappa grad u) + b . grad(u) on the N x N interior nodes of a uniform
    grid of the unit square, Dirichlet boundary eliminated. Diffusion: bilinear
    (Q1) elements with one kappa per cell ((N+1) x (N+1) cells, kappa_cells[cy, cx]),
    giving a 9-point stencil. Convection: first-order upwinding of a constant
    velocity with cell Peclet number `peclet` in direction theta, added as
    (|p_a|) on the diagonal and -|p_a| on the upwind neighbour along each axis,
    p = peclet * (cos theta, sin theta). Nodes are ordered x fastest."""
    import scipy.sparse as sparse

    N = int(N)
    n = N * N
    kc = np.asarray(kappa_cells, dtype=np.float64)
    assert kc.shape == (N + 1, N + 1)
    cy, cx = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")
    cx, cy, kk = cx.ravel(), cy.ravel(), kc.ravel()
    # node coordinates (0..N+1) of the 4 corners, interior nodes are 1..N
    corners = [(cx, cy), (cx + 1, cy), (cx + 1, cy + 1), (cx, cy + 1)]
    rows, cols, vals = [], [], []
    for a in range(4):
        xa, ya = corners[a]
        ia_ok = (xa >= 1) & (xa <= N) & (ya >= 1) & (ya <= N)
        ia = (ya - 1) * N + (xa - 1)
        for b in range(4):
            xb, yb = corners[b]
            ok = ia_ok & (xb >= 1) & (xb <= N) & (yb >= 1) & (yb <= N)
            ib = (yb - 1) * N + (xb - 1)
            rows.append(ia[ok])
            cols.append(ib[ok])
            vals.append(kk[ok] * _Q1_K[a, b])
    # upwind convection
    px, py = peclet * np.cos(theta), peclet * np.sin(theta)
    idx = np.arange(n)
    ix, iy = idx % N, idx // N
    rows.append(idx)
    cols.append(idx)
    vals.append(np.full(n, abs(px) + abs(py)))
    for p, shift, pos in ((px, 1, ix), (py, N, iy)):
        if p > 0:  # flow in +axis: upwind neighbour is the lower one
            ok = pos > 0
            rows.append(idx[ok]); cols.append(idx[ok] - shift); vals.append(np.full(ok.sum(), -abs(p)))
        elif p < 0:
            ok = pos < N - 1
            rows.append(idx[ok]); cols.append(idx[ok] + shift); vals.append(np.full(ok.sum(), -abs(p)))
    S = sparse.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    S.sum_duplicates()
    S.sort_indices()
    return S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64)


def batch_2d_params(count: int, seed: int = 0, side=(32, 256)):
    """Seeded parameters of the batched workload: per system a grid side
    log-uniform in `side`, cell diffusion coefficients log-uniform in [0.1, 10],
    a cell Peclet number U[0, 2] and a flow direction U[0, 2 pi)."""
    rng = _rng(seed)
    out = []
    for _ in range(count):
        N = int(round(np.exp(rng.uniform(np.log(side[0]), np.log(side[1])))))
        out.append(dict(N=N, kseed=int(rng.integers(1 << 31)), peclet=float(rng.uniform(0.0, 2.0)),
                        theta=float(rng.uniform(0.0, 2 * np.pi))))
    return out


def batch_2d_system(par) -> CSR:
    N = par["N"]
    kc = np.exp(_rng(par["kseed"]).uniform(np.log(0.1), np.log(10.0), (N + 1, N + 1)))
    return conv_diff_9pt_2d(N, kc, par["peclet"], par["theta"])


# --------------------------------------------------------------------------
# right-hand sides and generic helpers
# --------------------------------------------------------------------------
def to_scipy(A: CSR) -> sp.csr_matrix:
    rowptr, col, val = A
    n = len(rowptr) - 1
    return sp.csr_matrix((val, col, rowptr), shape=(n, n))


def from_dense(M: np.ndarray) -> CSR:
    S = sp.csr_matrix(np.asarray(M, dtype=np.float64))
    S.sort_indices()
    return S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64)


def x_true(n: int, seed: int = 0) -> np.ndarray:
    """x_true ~ U[-1, 1] from PCG64(seed)."""
    return _rng(seed).uniform(-1.0, 1.0, n)


def rhs(A: CSR, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """(x_true, b = A x_true) with x_true ~ U[-1, 1] from PCG64(seed)."""
    rowptr = A[0]
    xt = x_true(len(rowptr) - 1, seed)
    b = to_scipy(A) @ xt
    return xt, b


# --------------------------------------------------------------------------
# small test problems
# --------------------------------------------------------------------------
def simoncini_szyld(n: int = 100, seed: int = 0) -> tuple[CSR, np.ndarray]:
    """A = diag(1e-8, 2, 3, ..., n) and a normalized Gaussian b (kappa = 1e10)."""
    d = np.arange(1, n + 1, dtype=np.float64)
    d[0] = 1e-8
    A = (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    b = _rng(seed).standard_normal(n)
    return A, b / np.linalg.norm(b)


def random_dense(n: int, seed: int = 0, shift: float = 4.0) -> np.ndarray:
    """Well-conditioned nonsymmetric dense matrix: shift * I + G / sqrt(n), G Gaussian."""
    G = _rng(seed).standard_normal((n, n))
    return shift * np.eye(n) + G / np.sqrt(n)


def distinct_eigs(n: int, eigs, seed: int = 0) -> np.ndarray:
    """Nonsymmetric diagonalizable S diag(lambda) S^{-1} whose spectrum takes only
    the values in `eigs` (so its minimal polynomial has degree len(eigs))."""
    rng = _rng(seed)
    lam = np.resize(np.asarray(eigs, dtype=np.float64), n)
    S = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    return S @ np.diag(lam) @ np.linalg.inv(S)


def tall_skinny(n: int, p: int, kappa: float, seed: int = 0) -> np.ndarray:
    """U diag(sigma) W^T with orthonormal U (n x p), orthogonal W (p x p) and
    singular values log-spaced from 1 down to 1/kappa."""
    rng = _rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, p)))
    W, _ = np.linalg.qr(rng.standard_normal((p, p)))
    sigma = np.logspace(0.0, -np.log10(kappa), p)
    return (U * sigma) @ W.T
