"""ctypes binding of the C ABI in include/lsgmres.h (argument marshalling only).

Every numerical step runs in the CUDA library ``liblsgmres.so`` built from
``csrc/lsgmres.cu``; this module converts torch tensors and numpy arrays to
pointers and status codes to exceptions. There is no CPU fallback: importing
fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblsgmres.so")

OK, MAXITER, BREAKDOWN_EXACT = 0, 1, 2
ERR_ARG, ERR_CUDA, ERR_NONFINITE, ERR_OOM, ERR_TIMEOUT = -1, -2, -3, -4, -5
MGS, ONE_REDUCE_MGS, CGS2_LVL2, ONE_REDUCE_PIPE2 = 0, 1, 2, 3
FP64, IR_FP32, IR_BF16 = 0, 1, 2
ORTHO = {"mgs": MGS, "one_reduce_mgs": ONE_REDUCE_MGS, "one_reduce": ONE_REDUCE_MGS, "cgs2_lvl2": CGS2_LVL2,
         "one_reduce_pipe2": ONE_REDUCE_PIPE2}
PREC = {"fp64": FP64, "ir_fp32": IR_FP32, "ir_bf16": IR_BF16}
STATUS_NAMES = {0: "OK", 1: "MAXITER", 2: "BREAKDOWN_EXACT", -1: "ERR_ARG", -2: "ERR_CUDA",
                -3: "ERR_NONFINITE", -4: "ERR_OOM", -5: "ERR_TIMEOUT"}


class GmresError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class _Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("on_device", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("status", ctypes.c_int),
                ("breakdowns", ctypes.c_int), ("rel_resid_true", ctypes.c_double),
                ("rel_resid_est", ctypes.c_double), ("reductions", ctypes.c_int64),
                ("grid_syncs", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("seconds", ctypes.c_double)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("m_restart", ctypes.c_int), ("max_iter", ctypes.c_int), ("max_requests", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_int64), ("ir_share", ctypes.c_double),
                ("nnz_per_row_hint", ctypes.c_int64)]


_I64x2 = ctypes.c_int64 * 2


class _ServerCounters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("rejected", ctypes.c_int64), ("admitted", _I64x2),
                ("completed", _I64x2), ("queued", _I64x2), ("running", _I64x2), ("peak_running", _I64x2),
                ("cycles", _I64x2), ("engine_bytes", _I64x2), ("peak_bytes_in_use", _I64x2),
                ("arena_rows", _I64x2), ("kernel_launches", _I64x2), ("busy_seconds", ctypes.c_double * 2),
                ("wall_seconds", ctypes.c_double)]


class _ProbeResult(ctypes.Structure):
    _fields_ = [("ops_per_clk_per_sm", ctypes.c_double), ("ops_per_s", ctypes.c_double), ("sm_mhz", ctypes.c_double),
                ("seconds", ctypes.c_double), ("sms", ctypes.c_int)]


PROBE_OPS = ["dfma", "dadd", "ffma", "imad", "imad_wide", "imad_hi", "iadd", "lop3", "shf", "i2f_f64", "f2i_f64",
             "f2f_f32_f64", "i2f_f32", "flo"]


@dataclass
class SolveInfo:
    status: int
    iters: int
    restarts: int
    breakdowns: int
    rel_resid_true: float
    rel_resid_est: float
    reductions: int
    grid_syncs: int
    kernel_launches: int
    seconds: float


EXPORTS = ["gmres_create", "gmres_set", "gmres_set_tol", "gmres_set_stream", "gmres_solve",
           "gmres_solve_host", "gmres_history", "gmres_destroy", "gmres_last_error", "lsg_spmv",
           "lsg_block_dot", "lsg_maxpy", "gmres_arnoldi", "gmres_set_profile", "gmres_profile", "gmres_test_stall_staging", "gmres_set_block_dot", "gmres_set_reproducible", "gmres_set_persistent",
           "gmres_test_stall_barrier",
           "lsg_block_dot_noalloc", "gmres_batch_create", "gmres_batch_set_grid", "gmres_batch_get_grid",
           "gmres_batch_set_rows_per_thread", "gmres_batch_get_rows_per_thread", "gmres_batch_set_block_dot",
           "gmres_batch_set_stream", "gmres_batch_solve",
           "gmres_batch_solve_host", "gmres_batch_set_profile", "gmres_batch_profile", "gmres_batch_launch_log",
           "gmres_batch_history", "gmres_batch_destroy", "gmres_batch_last_error", "gmres_server_create",
           "gmres_server_submit", "gmres_server_poll", "gmres_server_wait", "gmres_server_drain",
           "gmres_server_release", "gmres_server_stats", "gmres_server_latencies", "gmres_server_destroy",
           "gmres_server_last_error", "gmres_server_set_profile", "gmres_server_profile", "lsg_probe_pipe",
           "lsg_probe_last_error"]

PROFILE_CLASSES = ["one_reduce_step", "arnoldi_maxpy", "mgs_spmv_dot", "mgs_axpy_dot", "residual",
                   "least_squares", "x_update", "noop", "reorth_dot", "reorth_maxpy", "persistent_cycle"]

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not built; run `python -m paper_1809_05805_b300.build`")
    lib = ctypes.CDLL(path)
    P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "gmres_create": ([ctypes.POINTER(_Csr), I, D, ctypes.POINTER(P)], I),
        "gmres_set": ([P, I, I, I], I),
        "gmres_set_tol": ([P, D], I),
        "gmres_set_stream": ([P, P], I),
        "gmres_solve": ([P, P, P, ctypes.POINTER(_Info)], I),
        "gmres_solve_host": ([P, P, P, ctypes.POINTER(_Info)], I),
        "gmres_history": ([P, P, I, ctypes.POINTER(I)], I),
        "gmres_destroy": ([P], I),
        "gmres_last_error": ([P], ctypes.c_char_p),
        "lsg_spmv": ([P, P, P], I),
        "lsg_block_dot": ([P, P, I64, I, P, P, I, P], I),
        "lsg_maxpy": ([P, P, I64, I, P, D, P, P], I),
        "gmres_arnoldi": ([P, P, I, P, P, P, ctypes.POINTER(I)], I),
        "gmres_set_profile": ([P, I], I),
        "gmres_test_stall_staging": ([P, I, ctypes.POINTER(I)], I),
        "gmres_set_block_dot": ([P, I, ctypes.POINTER(I)], I),
        "gmres_set_reproducible": ([P, I], I),
        "gmres_set_persistent": ([P, I, ctypes.POINTER(I)], I),
        "gmres_test_stall_barrier": ([P, I], I),
        "lsg_block_dot_noalloc": ([P, P, P, I64, P, I64, I, P, P, I, P, P], I),
        "gmres_profile": ([P, I, ctypes.POINTER(D), ctypes.POINTER(I64), ctypes.POINTER(D),
                           ctypes.POINTER(D)], I),
        "gmres_batch_create": ([ctypes.POINTER(_Csr), I, I, D, I, ctypes.POINTER(P)], I),
        "gmres_batch_set_stream": ([P, P], I),
        "gmres_batch_set_grid": ([P, I], I),
        "gmres_batch_get_grid": ([P, ctypes.POINTER(I)], I),
        "gmres_batch_set_rows_per_thread": ([P, I], I),
        "gmres_batch_get_rows_per_thread": ([P, ctypes.POINTER(I)], I),
        "gmres_batch_set_block_dot": ([P, I, ctypes.POINTER(I)], I),
        "gmres_batch_solve": ([P, P, P, ctypes.POINTER(_Info)], I),
        "gmres_batch_history": ([P, I, P, I, ctypes.POINTER(I)], I),
        "gmres_batch_solve_host": ([P, P, P, ctypes.POINTER(_Info)], I),
        "gmres_batch_set_profile": ([P, I], I),
        "gmres_batch_launch_log": ([P, I, P, P, P, P, P, ctypes.POINTER(I)], I),
        "gmres_batch_profile": ([P, I, ctypes.POINTER(D), ctypes.POINTER(I64), ctypes.POINTER(D),
                                 ctypes.POINTER(D)], I),
        "gmres_batch_destroy": ([P], I),
        "gmres_batch_last_error": ([P], ctypes.c_char_p),
        "gmres_server_create": ([ctypes.POINTER(_ServerConfig), ctypes.POINTER(P)], I),
        "gmres_server_submit": ([P, ctypes.POINTER(_Csr), P, P, P, D, I, I, ctypes.POINTER(I64)], I),
        "gmres_server_poll": ([P, I64, ctypes.POINTER(I), ctypes.POINTER(_Info)], I),
        "gmres_server_wait": ([P, I64, D, ctypes.POINTER(_Info)], I),
        "gmres_server_drain": ([P, D], I),
        "gmres_server_release": ([P, I64], I),
        "gmres_server_stats": ([P, ctypes.POINTER(_ServerCounters)], I),
        "gmres_server_latencies": ([P, P, I, ctypes.POINTER(I)], I),
        "gmres_server_destroy": ([P], I),
        "gmres_server_last_error": ([P], ctypes.c_char_p),
        "gmres_server_set_profile": ([P, I], I),
        "gmres_server_profile": ([P, I, I, ctypes.POINTER(D), ctypes.POINTER(I64), ctypes.POINTER(D),
                                  ctypes.POINTER(D)], I),
        "lsg_probe_pipe": ([I, I, I, ctypes.POINTER(_ProbeResult)], I),
        "lsg_probe_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes, f.restype = args, res
    _lib = lib
    return lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()  # torch tensor


def _dev_f64(t, n: int, name: str):
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} elements, need {n}")
    return t


class Solver:
    """Restarted GMRES(m) on one GPU through the C ABI (gmres_create/solve/...)."""

    def __init__(self, A, m: int, tol: float, *, ortho: str = "one_reduce_mgs", max_iter: int | None = None,
                 stream=None, prec: str | int = "fp64"):
        lib = load()
        self.lib = lib
        rowptr, col, val = A
        on_dev = not isinstance(rowptr, np.ndarray)
        if not on_dev:
            rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
            col = np.ascontiguousarray(col, dtype=np.int32)
            val = np.ascontiguousarray(val, dtype=np.float64)
        self.n = int(len(rowptr) - 1 if not on_dev else rowptr.numel() - 1)
        self.nnz = int(len(col) if not on_dev else col.numel())
        self.m = m
        csr = _Csr(self.n, self.nnz, _ptr(rowptr), _ptr(col), _ptr(val), int(on_dev))
        h = ctypes.c_void_p()
        st = lib.gmres_create(ctypes.byref(csr), m, tol, ctypes.byref(h))
        if st != OK:
            raise GmresError(st, lib.gmres_last_error(None).decode())
        self.h = h
        self.set(ortho=ortho, max_iter=max_iter if max_iter is not None else 10 * m, prec=prec)
        if stream is not None:
            self.set_stream(stream)

    def _check(self, st: int, allow=(OK,)):
        if st not in allow:
            raise GmresError(st, self.lib.gmres_last_error(self.h).decode())
        return st

    def set(self, *, ortho: str | int = "one_reduce_mgs", prec: str | int = FP64, max_iter: int = 300):
        o = ORTHO[ortho] if isinstance(ortho, str) else int(ortho)
        pr = PREC[prec] if isinstance(prec, str) else int(prec)
        self._check(self.lib.gmres_set(self.h, o, pr, max_iter))
        self.ortho, self.prec, self.max_iter = o, pr, max_iter

    def set_tol(self, tol: float):
        self._check(self.lib.gmres_set_tol(self.h, tol))

    def set_stream(self, stream):
        self._check(self.lib.gmres_set_stream(self.h, ctypes.c_void_p(int(stream.cuda_stream))))

    def solve(self, b, x, *, raise_on_maxiter: bool = False) -> SolveInfo:
        """b, x: float64 CUDA tensors (x holds x0 on entry, the solution on exit)."""
        _dev_f64(b, self.n, "b")
        _dev_f64(x, self.n, "x")
        info = _Info()
        st = self.lib.gmres_solve(self.h, _ptr(b), _ptr(x), ctypes.byref(info))
        self._check(st, (OK,) if raise_on_maxiter else (OK, MAXITER))
        return _info(info)

    def solve_host(self, b: np.ndarray, x: np.ndarray) -> SolveInfo:
        """b, x: float64 numpy arrays (host); copies in, solves, copies x back."""
        assert b.dtype == np.float64 and x.dtype == np.float64 and b.flags.c_contiguous and x.flags.c_contiguous
        info = _Info()
        st = self.lib.gmres_solve_host(self.h, _ptr(b), _ptr(x), ctypes.byref(info))
        self._check(st, (OK, MAXITER))
        return _info(info)

    def history(self) -> np.ndarray:
        n = ctypes.c_int(0)
        self._check(self.lib.gmres_history(self.h, None, 0, ctypes.byref(n)))
        buf = np.zeros(n.value, dtype=np.float64)
        self._check(self.lib.gmres_history(self.h, _ptr(buf), n.value, ctypes.byref(n)))
        return buf

    # -- single steps, for parity tests ------------------------------------
    def spmv(self, x, y):
        self._check(self.lib.lsg_spmv(self.h, _ptr(x), _ptr(y)))

    def block_dot(self, V, ldv: int, j: int, u, w, use_spmv: bool = True) -> np.ndarray:
        X = np.zeros(2 * j + 2, dtype=np.float64)
        self._check(self.lib.lsg_block_dot(self.h, _ptr(V), ldv, j, _ptr(u), _ptr(w), int(use_spmv), _ptr(X)))
        return X

    def maxpy(self, V, ldv: int, c: np.ndarray, alpha: float, y_in, y_out):
        c = np.ascontiguousarray(c, dtype=np.float64)
        self._check(self.lib.lsg_maxpy(self.h, _ptr(V), ldv, len(c), _ptr(c), alpha, _ptr(y_in), _ptr(y_out)))

    def arnoldi(self, r0, k: int):
        """k Arnoldi steps from r0 (CUDA tensor). Returns (V torch n x (k'+1), H (k'+1) x k', T, k')."""
        import torch

        V = torch.zeros((k + 1, self.n), dtype=torch.float64, device=r0.device)  # column-major n x (k+1)
        H = np.zeros((k + 1, k), dtype=np.float64, order="F")
        T = np.zeros((k + 1, k + 1), dtype=np.float64, order="F")
        kd = ctypes.c_int(0)
        self._check(self.lib.gmres_arnoldi(self.h, _ptr(r0), k, _ptr(V), _ptr(H), _ptr(T), ctypes.byref(kd)))
        kk = kd.value
        return V[: kk + 1].T, H[: kk + 1, :kk], T[: kk + 1, : kk + 1], kk

    def set_profile(self, on: bool):
        self._check(self.lib.gmres_set_profile(self.h, int(on)))

    def set_block_dot(self, fixed_point: bool) -> bool:
        """gmres_set_block_dot: FP64 block dot with exact fixed-point products on
        the integer pipes (True, the default) or FP64 FMAs; returns whether the
        handle's step kernel uses the fixed-point form."""
        active = ctypes.c_int(0)
        self._check(self.lib.gmres_set_block_dot(self.h, int(fixed_point), ctypes.byref(active)))
        return bool(active.value)

    def set_reproducible(self, on: bool):
        """gmres_set_reproducible: tile pairs of the fixed-point step kernel by a
        fixed stride (bitwise reproducible results) instead of from a counter."""
        self._check(self.lib.gmres_set_reproducible(self.h, int(bool(on))))

    def set_persistent(self, mode: int) -> bool:
        """gmres_set_persistent: one launch per restart cycle (1), per-step
        launches (0) or automatic (-1, the default); returns whether the next
        solve runs whole cycles in one launch."""
        active = ctypes.c_int(0)
        self._check(self.lib.gmres_set_persistent(self.h, int(mode), ctypes.byref(active)))
        return bool(active.value)

    def test_stall_barrier(self, on):
        """Make a wait of the persistent cycle run out (testing): on = 1 (or
        True) its grid barrier waits for a CTA that never arrives, on = 2 its
        epilogue wait for an epilogue that never comes; the solve returns
        GMRES_ERR_TIMEOUT after ~1 s. 0 (False) restores normal operation."""
        self._check(self.lib.gmres_test_stall_barrier(self.h, int(on)))

    def test_stall_staging(self, on: bool) -> bool:
        """Make the bounded waits of the CSR staging run out (testing); returns
        whether the FP64 step kernel stages its CSR at all."""
        staged = ctypes.c_int(0)
        self._check(self.lib.gmres_test_stall_staging(self.h, int(on), ctypes.byref(staged)))
        return bool(staged.value)

    def profile(self) -> dict:
        """Per kernel class of the last solve: device ms, launches, algorithmic bytes and flops."""
        out = {}
        for c, name in enumerate(PROFILE_CLASSES):
            ms, cnt, by, fl = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
            self._check(self.lib.gmres_profile(self.h, c, ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(by),
                                               ctypes.byref(fl)))
            out[name] = dict(ms=ms.value, launches=cnt.value, bytes=by.value, flops=fl.value)
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.gmres_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def block_dot_noalloc(A_dev, n: int, V, ldv: int, j: int, u, w, X, use_spmv: bool = True, stream=None):
    """lsg_block_dot_noalloc: the fused SpMV + block dot without a handle or any
    allocation by the library. A_dev = (rowptr, col, val) as CUDA tensors; V, u,
    w, X CUDA float64 tensors (X receives 2j+2 sums). Queued on `stream`
    (a torch.cuda.Stream, default: the legacy default stream); not synchronized."""
    lib = load()
    rowptr, col, val = A_dev
    st = lib.lsg_block_dot_noalloc(_ptr(rowptr), _ptr(col), _ptr(val), n, _ptr(V), ldv, j, _ptr(u), _ptr(w),
                                   int(use_spmv), _ptr(X), None if stream is None else int(stream.cuda_stream))
    if st != OK:
        raise GmresError(st, lib.gmres_last_error(None).decode())


def probe_pipe(op: str, ctas_per_sm: int = 2, iters: int = 4096) -> dict:
    """lsg_probe_pipe: measured rate of one instruction kind on the current
    device (thread instructions per SM clock and per second, the SM clock)."""
    lib = load()
    r = _ProbeResult()
    st = lib.lsg_probe_pipe(PROBE_OPS.index(op), ctas_per_sm, iters, ctypes.byref(r))
    if st != OK:
        raise GmresError(st, lib.lsg_probe_last_error().decode())
    return {"op": op, "ops_per_clk_per_sm": r.ops_per_clk_per_sm, "ops_per_s": r.ops_per_s, "sm_mhz": r.sm_mhz,
            "seconds": r.seconds, "sms": r.sms}


class BatchSolver:
    """Many independent systems solved together (gmres_batch_*): one-reduce
    MGS-GMRES(m) in FP64, lock-step cycles, one launch per Arnoldi step."""

    def __init__(self, mats, m: int, tol: float, *, max_iter: int | None = None, stream=None):
        lib = load()
        self.lib = lib
        self._keep = []
        csrs = (_Csr * len(mats))()
        self.n = []
        for i, (rowptr, col, val) in enumerate(mats):
            rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
            col = np.ascontiguousarray(col, dtype=np.int32)
            val = np.ascontiguousarray(val, dtype=np.float64)
            self._keep += [rowptr, col, val]
            n = len(rowptr) - 1
            csrs[i] = _Csr(n, len(col), _ptr(rowptr), _ptr(col), _ptr(val), 0)
            self.n.append(n)
        self.count, self.m = len(mats), m
        self.max_iter = max_iter if max_iter is not None else 10 * m
        h = ctypes.c_void_p()
        st = lib.gmres_batch_create(csrs, len(mats), m, tol, self.max_iter, ctypes.byref(h))
        self._keep = None
        if st != OK:
            raise GmresError(st, lib.gmres_batch_last_error(None).decode())
        self.h = h
        if stream is not None:
            self.set_stream(stream)

    def _check(self, st: int, allow=(OK,)):
        if st not in allow:
            raise GmresError(st, self.lib.gmres_batch_last_error(self.h).decode())
        return st

    def set_stream(self, stream):
        self._check(self.lib.gmres_batch_set_stream(self.h, ctypes.c_void_p(int(stream.cuda_stream))))

    @property
    def grid(self) -> int:
        g = ctypes.c_int(0)
        self._check(self.lib.gmres_batch_get_grid(self.h, ctypes.byref(g)))
        return g.value

    def set_grid(self, ctas: int):
        """Pin the grid of the batched kernels (0: autotune grid and rows per thread again)."""
        self._check(self.lib.gmres_batch_set_grid(self.h, int(ctas)))

    @property
    def rows_per_thread(self) -> int:
        r = ctypes.c_int(0)
        self._check(self.lib.gmres_batch_get_rows_per_thread(self.h, ctypes.byref(r)))
        return r.value

    def set_rows_per_thread(self, rows: int):
        self._check(self.lib.gmres_batch_set_rows_per_thread(self.h, int(rows)))

    def set_block_dot(self, fixed_point) -> int:
        """gmres_batch_set_block_dot: fixed-point block-dot and MAXPY products
        (True / 1, the default; -1: without the column ring) or FP64 FMAs
        (False / 0); returns the form the next solve uses: 0 FP64 FMAs, 1 fixed
        point with direct basis loads, 2 fixed point with the column ring
        (FP64 batches with two rows per thread)."""
        active = ctypes.c_int(0)
        self._check(self.lib.gmres_batch_set_block_dot(self.h, int(fixed_point), ctypes.byref(active)))
        return active.value

    def solve(self, bs, xs, *, allow=(OK, MAXITER)) -> list[SolveInfo]:
        """bs, xs: lists of float64 CUDA tensors (xs hold x0 on entry, solutions on exit)."""
        if len(bs) != self.count or len(xs) != self.count:
            raise ValueError(f"need {self.count} right-hand sides and solution vectors")
        for i in range(self.count):
            _dev_f64(bs[i], self.n[i], f"b[{i}]")
            _dev_f64(xs[i], self.n[i], f"x[{i}]")
        bp = (ctypes.c_void_p * self.count)(*[_ptr(t) for t in bs])
        xp = (ctypes.c_void_p * self.count)(*[_ptr(t) for t in xs])
        infos = (_Info * self.count)()
        self._check(self.lib.gmres_batch_solve(self.h, bp, xp, infos), allow)
        return [_info(i) for i in infos]

    def solve_host(self, bs, xs, *, allow=(OK, MAXITER)) -> list[SolveInfo]:
        """bs, xs: lists of float64 numpy arrays (host; pinned for speed); x holds x0 on entry."""
        if len(bs) != self.count or len(xs) != self.count:
            raise ValueError(f"need {self.count} right-hand sides and solution vectors")
        for i in range(self.count):
            for a, nm in ((bs[i], "b"), (xs[i], "x")):
                if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
                        and a.size >= self.n[i]):
                    raise TypeError(f"{nm}[{i}] must be a contiguous float64 numpy array of {self.n[i]} entries")
        bp = (ctypes.c_void_p * self.count)(*[_ptr(a) for a in bs])
        xp = (ctypes.c_void_p * self.count)(*[_ptr(a) for a in xs])
        infos = (_Info * self.count)()
        self._check(self.lib.gmres_batch_solve_host(self.h, bp, xp, infos), allow)
        return [_info(i) for i in infos]

    def set_profile(self, on: bool):
        self._check(self.lib.gmres_batch_set_profile(self.h, int(on)))

    def profile(self) -> dict:
        """Per kernel class of the last batch solve: device ms, launches, algorithmic bytes and flops."""
        out = {}
        for c, name in enumerate(PROFILE_CLASSES):
            ms, cnt, by, fl = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
            self._check(self.lib.gmres_batch_profile(self.h, c, ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(by),
                                                     ctypes.byref(fl)))
            out[name] = dict(ms=ms.value, launches=cnt.value, bytes=by.value, flops=fl.value)
        return out

    def launch_log(self) -> dict:
        """Per launch of the last profiled solve: class name, step j, listed tiles, ms, algorithmic flops."""
        cnt = ctypes.c_int(0)
        self._check(self.lib.gmres_batch_launch_log(self.h, 0, None, None, None, None, None, ctypes.byref(cnt)))
        k = cnt.value
        cls = np.zeros(k, np.int32)
        step = np.zeros(k, np.int32)
        tiles = np.zeros(k, np.int64)
        ms = np.zeros(k, np.float32)
        fl = np.zeros(k, np.float64)
        self._check(self.lib.gmres_batch_launch_log(self.h, k, _ptr(cls), _ptr(step), _ptr(tiles), _ptr(ms),
                                                    _ptr(fl), ctypes.byref(cnt)))
        return dict(cls=np.array(PROFILE_CLASSES)[cls] if k else np.array([], dtype=str), step=step, tiles=tiles,
                    ms=ms, flops=fl)

    def history(self, i: int) -> np.ndarray:
        n = ctypes.c_int(0)
        self._check(self.lib.gmres_batch_history(self.h, i, None, 0, ctypes.byref(n)))
        buf = np.zeros(n.value, dtype=np.float64)
        self._check(self.lib.gmres_batch_history(self.h, i, _ptr(buf), n.value, ctypes.byref(n)))
        return buf

    def close(self):
        if getattr(self, "h", None):
            self.lib.gmres_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching solve server (gmres_server_*): requests of any size,
    FP64 or GMRES-IR, are admitted at cycle boundaries under a device byte
    budget and iterate together; one worker thread and CUDA stream per
    precision."""

    def __init__(self, *, m: int = 30, max_iter: int = 3000, max_requests: int = 256,
                 hbm_budget_bytes: int = 16 << 30, ir_share: float = 0.3, nnz_per_row_hint: int = 7):
        lib = load()
        self.lib = lib
        cfg = _ServerConfig(m, max_iter, max_requests, int(hbm_budget_bytes), float(ir_share), int(nnz_per_row_hint))
        h = ctypes.c_void_p()
        st = lib.gmres_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != OK:
            raise GmresError(st, lib.gmres_server_last_error(None).decode())
        self.h = h
        self.m, self.max_iter = m, max_iter
        self._refs = {}

    def _check(self, st: int, allow=(OK,)):
        if st not in allow:
            raise GmresError(st, self.lib.gmres_server_last_error(self.h).decode())
        return st

    def submit(self, A, b, x_out, *, tol: float, prec: str | int = "fp64", max_iter: int | None = None,
               x0=None) -> int:
        """A = (rowptr, col, val) host arrays; b, x0, x_out float64 numpy arrays or CUDA tensors. The arrays
        are kept referenced here until the request is waited for or released."""
        rowptr = np.ascontiguousarray(A[0], dtype=np.int32)
        col = np.ascontiguousarray(A[1], dtype=np.int32)
        val = np.ascontiguousarray(A[2], dtype=np.float64)
        n = len(rowptr) - 1
        for a, nm in ((b, "b"), (x_out, "x_out"), (x0, "x0")):
            if a is None:
                continue
            if isinstance(a, np.ndarray):
                if not (a.dtype == np.float64 and a.flags.c_contiguous and a.size >= n):
                    raise TypeError(f"{nm} must be a contiguous float64 array of {n} entries")
            else:
                _dev_f64(a, n, nm)
        csr = _Csr(n, len(col), _ptr(rowptr), _ptr(col), _ptr(val), 0)
        pr = PREC[prec] if isinstance(prec, str) else int(prec)
        rid = ctypes.c_int64(0)
        self._check(self.lib.gmres_server_submit(self.h, ctypes.byref(csr), _ptr(b), _ptr(x0), _ptr(x_out), tol, pr,
                                                 self.max_iter if max_iter is None else int(max_iter),
                                                 ctypes.byref(rid)))
        self._refs[rid.value] = (rowptr, col, val, b, x0, x_out)
        return rid.value

    def poll(self, rid: int):
        done = ctypes.c_int(0)
        info = _Info()
        self._check(self.lib.gmres_server_poll(self.h, rid, ctypes.byref(done), ctypes.byref(info)))
        return bool(done.value), (_info(info) if done.value else None)

    def wait(self, rid: int, timeout: float = 600.0) -> SolveInfo:
        info = _Info()
        st = self.lib.gmres_server_wait(self.h, rid, timeout, ctypes.byref(info))
        if st == ERR_TIMEOUT:
            raise TimeoutError(f"request {rid} not done after {timeout} s")
        return _info(info)

    def drain(self, timeout: float = 600.0):
        if self.lib.gmres_server_drain(self.h, timeout) == ERR_TIMEOUT:
            raise TimeoutError(f"requests still in flight after {timeout} s")

    def release(self, rid: int):
        self._check(self.lib.gmres_server_release(self.h, rid))
        self._refs.pop(rid, None)

    def stats(self) -> dict:
        c = _ServerCounters()
        self._check(self.lib.gmres_server_stats(self.h, ctypes.byref(c)))
        out = {}
        for name, _ in _ServerCounters._fields_:
            v = getattr(c, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out

    def set_profile(self, on: bool):
        self._check(self.lib.gmres_server_set_profile(self.h, int(on)))

    def profile(self, engine: int) -> dict:
        """Per kernel class since profiling was switched on: device ms, launches, algorithmic bytes and flops."""
        out = {}
        for c, name in enumerate(PROFILE_CLASSES):
            ms, cnt, by, fl = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
            self._check(self.lib.gmres_server_profile(self.h, engine, c, ctypes.byref(ms), ctypes.byref(cnt),
                                                      ctypes.byref(by), ctypes.byref(fl)))
            out[name] = dict(ms=ms.value, launches=cnt.value, bytes=by.value, flops=fl.value)
        return out

    def latencies(self) -> np.ndarray:
        n = ctypes.c_int(0)
        self._check(self.lib.gmres_server_latencies(self.h, None, 0, ctypes.byref(n)))
        buf = np.zeros(n.value, dtype=np.float64)
        self._check(self.lib.gmres_server_latencies(self.h, _ptr(buf), n.value, ctypes.byref(n)))
        return buf[: n.value]

    def close(self):
        if getattr(self, "h", None):
            self.lib.gmres_server_destroy(self.h)
            self.h = None
            self._refs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _info(i: _Info) -> SolveInfo:
    return SolveInfo(i.status, i.iters, i.restarts, i.breakdowns, i.rel_resid_true, i.rel_resid_est,
                     i.reductions, i.grid_syncs, i.kernel_launches, i.seconds)
