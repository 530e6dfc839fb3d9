"""FP64 CPU oracle for one-reduce and plain MGS-GMRES (arXiv:1809.05805).

Test infrastructure only. Importers: ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference arm of ``bench.py``. The product library
(``paper_1809_05805_b300``) never imports this package, and this package
imports nothing from it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, sequential loops, compiled
with ``-O2 -ffp-contract=off``). This module only compiles it on demand and
marshals numpy arrays through ``ctypes``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ORC_OK, ORC_MAXITER, ORC_BREAKDOWN = 0, 1, 2
ORC_ERR_ARG, ORC_ERR_NONFINITE, ORC_ERR_OOM = -1, -3, -4
MGS, ONE_REDUCE, IR_FP32, CGS2, PIPE2, IR_BF16 = 0, 1, 2, 3, 4, 5

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c99"]


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
OMP_FLAGS = ["-fopenmp", "-DORC_OMP"]


def build(src: str = _SRC, out: str = _LIB, extra: list[str] | None = None) -> str:
    """Compile oracle.c into a shared library (idempotent; rebuilds when stale)."""
    fresh = os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src)
    if fresh and (not extra or out == _LIB_OMP):
        return out
    cmd = ["gcc", *CFLAGS, *(extra or []), src, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(out + ".tmp", out)
    return out


class _OrcInfo(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("restarts", ctypes.c_int),
        ("status", ctypes.c_int),
        ("breakdowns", ctypes.c_int),
        ("rel_resid_true", ctypes.c_double),
        ("rel_resid_est", ctypes.c_double),
        ("reductions", ctypes.c_int64),
    ]


_P = ctypes.c_void_p


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """ctypes view of one compiled oracle library (the default one, or a mutant)."""

    def __init__(self, path: str | None = None):
        self.path = path or build()
        lib = ctypes.CDLL(self.path)
        lib.orc_spmv.argtypes = [ctypes.c_int64, _P, _P, _P, _P, _P]
        lib.orc_spmv.restype = None
        lib.orc_dot.argtypes = [ctypes.c_int64, _P, _P]
        lib.orc_dot.restype = ctypes.c_double
        lib.orc_maxpy.argtypes = [ctypes.c_int64, ctypes.c_int, _P, ctypes.c_int64, _P, ctypes.c_double, _P, _P]
        lib.orc_maxpy.restype = None
        lib.orc_qr_mgs.argtypes = [ctypes.c_int64, ctypes.c_int, _P, _P, _P]
        lib.orc_qr_cgs.argtypes = [ctypes.c_int64, ctypes.c_int, _P, _P, _P, ctypes.c_int]
        lib.orc_qr_mgs_lvl2.argtypes = [ctypes.c_int64, ctypes.c_int, _P, _P, _P, _P]
        lib.orc_qr_cgs2_lvl2.argtypes = [ctypes.c_int64, ctypes.c_int, _P, _P, _P, _P]
        for f in (lib.orc_qr_mgs, lib.orc_qr_cgs, lib.orc_qr_mgs_lvl2, lib.orc_qr_cgs2_lvl2):
            f.restype = ctypes.c_int
        lib.orc_gmres.argtypes = [
            ctypes.c_int64, _P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
            ctypes.c_int, _P, ctypes.c_int, ctypes.POINTER(_OrcInfo), _P, _P, _P,
            ctypes.POINTER(ctypes.c_int),
        ]
        lib.orc_gmres.restype = ctypes.c_int
        lib.orc_threads.argtypes = []
        lib.orc_threads.restype = ctypes.c_int
        self.threads = lib.orc_threads()
        lib.orc_round_bf16.argtypes = [ctypes.c_float]
        lib.orc_round_bf16.restype = ctypes.c_float
        self.lib = lib

    # -- kernels -----------------------------------------------------------
    def spmv(self, A, x: np.ndarray) -> np.ndarray:
        rowptr, col, val = _csr(A)
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(len(rowptr) - 1, dtype=np.float64)
        self.lib.orc_spmv(len(y), _ptr(rowptr), _ptr(col), _ptr(val), _ptr(x), _ptr(y))
        return y

    def dot(self, x: np.ndarray, y: np.ndarray) -> float:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        return self.lib.orc_dot(len(x), _ptr(x), _ptr(y))

    def maxpy(self, V: np.ndarray, c: np.ndarray, alpha: float, y: np.ndarray) -> np.ndarray:
        """alpha * y + V @ c with V (n x K) column-major."""
        V = np.asfortranarray(V, dtype=np.float64)
        c = np.ascontiguousarray(c, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        out = np.empty_like(y)
        n, K = V.shape
        self.lib.orc_maxpy(n, K, _ptr(V), n, _ptr(c), alpha, _ptr(y), _ptr(out))
        return out

    def _qr(self, fn, A: np.ndarray, *extra, with_T=False):
        A = np.asfortranarray(A, dtype=np.float64)
        n, p = A.shape
        Q = np.zeros((n, p), dtype=np.float64, order="F")
        R = np.zeros((p, p), dtype=np.float64, order="F")
        if with_T:
            T = np.zeros((p, p), dtype=np.float64, order="F")
            st = fn(n, p, _ptr(A), _ptr(Q), _ptr(R), _ptr(T))
            _check(st)
            return Q, R, T
        st = fn(n, p, _ptr(A), _ptr(Q), _ptr(R), *extra)
        _check(st)
        return Q, R

    def qr_mgs(self, A):
        """Column MGS QR (Algorithm 2)."""
        return self._qr(self.lib.orc_qr_mgs, A)

    def qr_cgs(self, A, passes: int = 1):
        """Classical GS QR with `passes` sweeps (Algorithm 1)."""
        return self._qr(self.lib.orc_qr_cgs, A, ctypes.c_int(passes))

    def qr_mgs_lvl2(self, A):
        """Level-2 compact-WY MGS with lagged normalization (Algorithm 4); returns Q, R, T."""
        return self._qr(self.lib.orc_qr_mgs_lvl2, A, with_T=True)

    def qr_cgs2_lvl2(self, A):
        """Level-2 iterated CGS with lagged normalization (Algorithm 5); returns Q, R, T."""
        return self._qr(self.lib.orc_qr_cgs2_lvl2, A, with_T=True)

    def round_bf16(self, x: np.ndarray) -> np.ndarray:
        """The oracle's FP32 -> BF16 rounding (as FP32 values), element by element."""
        return np.array([self.lib.orc_round_bf16(float(v)) for v in np.asarray(x, dtype=np.float32)],
                        dtype=np.float32)

    # -- solver ------------------------------------------------------------
    def gmres(self, A, b, *, variant: int, m: int, tol: float, max_iter: int, x0=None,
              capture: bool = False) -> "OracleResult":
        rowptr, col, val = _csr(A)
        n = len(rowptr) - 1
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        hist = np.zeros(max(max_iter, 1), dtype=np.float64)
        info = _OrcInfo()
        mm = min(m, max_iter) if max_iter > 0 else m
        V1 = H1 = T1 = None
        k1 = ctypes.c_int(0)
        if capture:
            V1 = np.zeros((n, mm + 1), dtype=np.float64, order="F")
            H1 = np.zeros((mm + 1, mm), dtype=np.float64, order="F")
            T1 = np.zeros((mm + 1, mm + 1), dtype=np.float64, order="F")
        st = self.lib.orc_gmres(n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(b), _ptr(x),
                                variant, m, tol, max_iter, _ptr(hist), len(hist),
                                ctypes.byref(info), _ptr(V1), _ptr(H1), _ptr(T1),
                                ctypes.byref(k1))
        res = OracleResult(
            x=x, status=st, iters=info.iters, restarts=info.restarts,
            breakdowns=info.breakdowns, rel_resid_true=info.rel_resid_true,
            rel_resid_est=info.rel_resid_est, reductions=info.reductions,
            history=hist[: min(info.iters, len(hist))].copy(),
        )
        if capture:
            k = k1.value
            res.V = V1[:, : k + 1]
            res.H = H1[: k + 1, :k]
            res.T = T1[: k + 1, : k + 1]
            res.k = k
        return res


@dataclass
class OracleResult:
    x: np.ndarray
    status: int
    iters: int
    restarts: int
    breakdowns: int
    rel_resid_true: float
    rel_resid_est: float
    reductions: int
    history: np.ndarray
    V: np.ndarray | None = None
    H: np.ndarray | None = None
    T: np.ndarray | None = None
    k: int = 0
    extra: dict = field(default_factory=dict)


def _csr(A):
    rowptr, col, val = A
    return (np.ascontiguousarray(rowptr, dtype=np.int32), np.ascontiguousarray(col, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float64))


def _check(st: int):
    if st != ORC_OK:
        raise RuntimeError(f"oracle status {st}")


_DEFAULT: Oracle | None = None


def get() -> Oracle:
    """The oracle compiled from this directory's oracle.c."""
    global _DEFAULT
    if _DEFAULT is None:
        _DEFAULT = Oracle()
    return _DEFAULT


_OMP = None


def get_omp() -> Oracle:
    """The same oracle.c built with OpenMP (-DORC_OMP -fopenmp): its vector
    loops run on all host cores (OMP_NUM_THREADS, default all). For timing the
    CPU baseline only; its sums are reordered, so it is never the checker."""
    global _OMP
    if _OMP is None:
        _OMP = Oracle(build(out=_LIB_OMP, extra=OMP_FLAGS))
    return _OMP
