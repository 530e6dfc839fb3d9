#!/usr/bin/env python
"""Time-to-solve of one-reduce MGS-GMRES against plain MGS-GMRES on B300.

Default workload: FP64 3D 7-point upwinded convection-diffusion on a 256^3
grid (n = 16,777,216, nnz = 117,047,296), GMRES(50), relative residual 1e-8,
x_true ~ U[-1, 1] from PCG64(0), b = A x_true, x0 = 0. One step is one
complete solve (every Arnoldi step, restart and solution update on the GPU).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload 256|128|32|192|144|256ir|batch512|batch64|serve|serve_small]
                  [--no-mgs] [--no-cpu-baseline]

--workload batch512: 512 independent 2D 9-point variable-coefficient
convection-diffusion systems (grid side log-uniform in 32..256, cell diffusion
log-uniform in [0.1, 10], cell Peclet U[0, 2], seeded), GMRES(30) to 1e-8, all
solved together by the batched solver against the same systems solved one
after another.

--workload serve: 256 requests arriving as a Poisson stream at 2000 req/s
(3D 7-point convection-diffusion, n log-uniform in 4k..2M, 70% FP64 / 30%
GMRES-IR, each to 1e-8) served by one continuous-batching server; reports
solves/s and p50/p99 latency, a run at half the measured capacity, and the
same requests one at a time on the single-system solver.

The default run (256^3, one GPU) then measures the other configurations in the
same process and reports each under "legs", with its own timing, roofline,
clocks and CPU baseline: 32^3 GMRES(30) (latency-bound), the 192^3 27-point
GMRES-IR solve (FP32 and BF16 basis, FP64 one-reduce beside them, errors
against the FP64 oracle's stored solve), batch512, and the serving loop with a
sweep of sustained arrival rates (--no-legs skips them).

The FP64 kernels' roofline is the FP64 pipe's rate measured by the library's
instruction-throughput probe (lsg_probe_pipe) in the same run; the CPU
baselines time the oracle on one host thread and on all host cores.

Prints one JSON line (rank 0). With N > 1 (torchrun) every rank solves its own
replica of the system (no data-path collective); the time is the maximum
over ranks. The reference arm (--impl reference) times the FP64 CPU oracle on
a bounded sample of the same workload and scales it to a whole solve.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1809_05805_b300 import problems as P  # noqa: E402

WORKLOADS = {
    # 7-point convection-diffusion, FP64 one-reduce against plain MGS on the same kernels
    256: dict(N=256, m=50, tol=1e-8, max_iter=3000, stencil="7pt", prec="fp64", compare="mgs"),
    128: dict(N=128, m=50, tol=1e-8, max_iter=3000, stencil="7pt", prec="fp64", compare="mgs"),  # profiling size
    32: dict(N=32, m=30, tol=1e-8, max_iter=300, stencil="7pt", prec="fp64", compare="mgs"),
    # 27-point anisotropic diffusion, GMRES-IR (FP32 cycles) against FP64 one-reduce
    192: dict(N=192, m=40, tol=1e-10, max_iter=5000, stencil="27pt", prec="ir_fp32", compare="fp64",
              golden_fp64="c3_fp64"),
    144: dict(N=144, m=40, tol=1e-10, max_iter=5000, stencil="27pt", prec="ir_fp32", compare="fp64"),  # profiling
    # the 256^3 7-point problem of the headline, solved by GMRES-IR (FP32 cycles)
    "256ir": dict(N=256, m=50, tol=1e-8, max_iter=3000, stencil="7pt", prec="ir_fp32", compare="fp64"),
    "128ir": dict(N=128, m=50, tol=1e-8, max_iter=3000, stencil="7pt", prec="ir_fp32", compare="fp64"),  # profiling
}
# batched uneven solves: 2D 9-point variable-coefficient convection-diffusion
# systems, grid side log-uniform in `side`, all solved together
BATCH_WORKLOADS = {
    "batch512": dict(count=512, side=(32, 256), m=30, tol=1e-8, max_iter=20000, seed=0),
    "batch64": dict(count=64, side=(32, 256), m=30, tol=1e-8, max_iter=20000, seed=0),  # profiling size
}
METRIC_BATCH = "time-to-solve (1e-8 rel. resid) of a batch of uneven systems, batched one-reduce MGS-GMRES"
# serving: Poisson arrivals of 3D 7-point convection-diffusion solves, n
# log-uniform in n_range (cube side rounded onto `sides` log-spaced values),
# 70% FP64 / 30% GMRES-IR, each to 1e-8, one continuous-batching server
SERVE_WORKLOADS = {
    "serve": dict(rate=2000.0, requests=256, n_range=(4096, 2_000_000), sides=16, ir_frac=0.3, m=30, tol=1e-8,
                  max_iter=3000, budget=64 << 30, max_requests=256, seed=0,
                  sweep=(0.25, 0.5, 0.75, 1.0, 1.25), sweep_s=10.0),
    "serve_small": dict(rate=2000.0, requests=48, n_range=(4096, 262_144), sides=8, ir_frac=0.3, m=30, tol=1e-8,
                        max_iter=3000, budget=16 << 30, max_requests=64, seed=0,
                        sweep=(0.5, 1.0), sweep_s=2.0),  # profiling size
}
METRIC_SERVE = "solves/s at 2000 req/s offered (1e-8 rel. resid each), continuous-batching serving loop; p50/p99 latency"
METRIC = "time-to-solve (1e-8 rel. resid), one-reduce MGS-GMRES"
METRIC_IR = "time-to-solve ({tol} rel. resid), GMRES-IR: one-reduce cycles in FP32, FP64 restarts"


def make_problem(w):
    return P.conv_diff_7pt(w["N"]) if w["stencil"] == "7pt" else P.aniso_27pt(w["N"])
FP64_DFMA_PER_CLK_SM = 2  # B300: 1.25 TFLOP/s nominal FP64 = 148 SMs x 2 DFMA/clk x 2 flop x ~2.1 GHz
# DRAM bytes per step launch / algorithmic bytes, from ncu captures of the
# step kernels (dram__bytes_read.sum + dram__bytes_write.sum over the launch's
# algorithmic bytes): the FP64 kernel with staged tile pairs on the 128^3
# 7-point workload at j = 8 and 9; the FP32 kernels, per stencil: single
# tiles on the 144^3 27-point GMRES-IR workload at j = 18 and 19, tile pairs
# with the column ring on the 128^3 7-point one at j = 20 and 21. Valid only
# for the kernel builds those captures measured; set to None when a kernel
# changes.
STEP_TRAFFIC_RATIO = 1.048
# The same ratio for the FP64 step with fixed-point products (staging mode 6,
# the basis read as stored limbs; the limbs of u, 8n bytes, written on top):
# 128^3 7-point at j = 10 and 11.
STEP6_TRAFFIC_RATIO = 1.035
STEP32_TRAFFIC_RATIO = {"27pt": 1.014, "7pt": 1.005}


def _rank_device(dist):
    """Device of the collective tensors: CUDA under NCCL, the host under gloo."""
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def rank_barrier(dist):
    """All ranks meet, then this rank's device work is done (the timing rule's
    synchronization on both sides of the timed region)."""
    import torch

    if dist is not None:
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def rank_max(dist, v):
    """Largest v over all ranks (a replicated step is as slow as its slowest rank)."""
    if dist is None:
        return v
    import torch

    t = torch.tensor([float(v)], dtype=torch.float64, device=_rank_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_name(w):
    N = w["N"]
    if w["stencil"] == "27pt":
        return (f"3D 27-point anisotropic diffusion k=(1,1,1e-3) {N}^3 (n={N ** 3}, nnz={P.grid27_nnz(N)}), "
                f"GMRES-IR: one-reduce GMRES({w['m']}) cycles in FP32 (FP32 basis, SpMV, dots, MAXPY) inside "
                f"FP64 restarts, vs FP64 one-reduce, tol {w['tol']:g}, x0=0")
    if w["prec"] == "ir_fp32":
        return (f"3D 7-point convection-diffusion {N}^3 (n={N ** 3}, nnz={P.grid7_nnz(N)}), GMRES-IR: one-reduce "
                f"GMRES({w['m']}) cycles in FP32 inside FP64 restarts, vs FP64 one-reduce, tol {w['tol']:g}, x0=0")
    return (f"3D 7-point convection-diffusion {N}^3 (n={N ** 3}, nnz={P.grid7_nnz(N)}), FP64 CSR, "
            f"GMRES({w['m']}) one-reduce MGS vs plain MGS, tol {w['tol']:g}, x0=0")


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"lsgmres_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    p = [t.strip() for t in line.split(",")]
                    if len(p) >= 9 and p[1].isdigit():
                        rows.append(p)
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = np.array([float(r[1]) for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][2]), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                "reasons": reasons}


# ----------------------------------------------------------------------------- helpers
def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


_FP64_PEAK = None


def fp64_peak():
    """The FP64 pipe's measured rate on this device (lsg_probe_pipe: DFMA chains
    on every SM, nothing else issued; the best of a few launch shapes), as
    TFLOP/s (2 flops per DFMA), with the derived nominal figure beside it."""
    global _FP64_PEAK
    if _FP64_PEAK is None:
        from paper_1809_05805_b300 import lsgmres

        best = None
        for cps in (2, 4):
            r = lsgmres.probe_pipe("dfma", ctas_per_sm=cps, iters=4096)
            if best is None or r["ops_per_s"] > best["ops_per_s"]:
                best = r
        peaks = load_peaks()
        _FP64_PEAK = {
            "tflops": 2 * best["ops_per_s"] / 1e12, "dfma_per_clk_per_sm": best["ops_per_clk_per_sm"],
            "probe_sm_mhz": best["sm_mhz"],
            "nominal_tflops": best["sms"] * FP64_DFMA_PER_CLK_SM * 2 * float(peaks.get("sm_max_mhz", 2032.0)) / 1e6,
            "source": "measured: lsg_probe_pipe DFMA (independent fma.rn.f64 chains on every SM, CUDA events; "
                      "best of 2 and 4 CTAs/SM); nominal = SMs x 2 DFMA/clk x 2 flop x max SM clock",
        }
    return _FP64_PEAK


def cycle_profile(total_iters, m):
    """Columns per cycle of a solve with `total_iters` steps and restart m (all cycles full but the last)."""
    ks = [m] * (total_iters // m)
    if total_iters % m:
        ks.append(total_iters % m)
    return ks


def oracle_step_bytes(n, nnz, j):
    """Bytes the (unfused, sequential) CPU oracle moves in one-reduce step j of a cycle:
    SpMV, 2j+2 separate dot products, the normalization, and the MAXPY as j+1 axpys."""
    spmv = 12.0 * nnz + 4.0 * n + 16.0 * n
    if j == 0:
        return spmv + 16.0 * n + 16.0 * n + 24.0 * n
    return spmv + 16.0 * n * (2 * j + 2) + 32.0 * n + 24.0 * n * (j + 1)


def oracle_solve_bytes(n, nnz, ks):
    tot = 0.0
    for k in ks:
        tot += sum(oracle_step_bytes(n, nnz, j) for j in range(k)) + 16.0 * n * (k + 2)  # steps + tail
        tot += 12.0 * nnz + 4.0 * n + 40.0 * n + 24.0 * n * k  # residual, its norm, x update
    return tot


def cpu_baseline(A, b, w, ks_full, sample_iters):
    """Time the FP64 oracle (1 thread) on the first `sample_iters` steps of the same
    solve and scale to the whole solve by a model of the oracle's own memory traffic
    (checked against one complete 256^3 oracle solve: the scaled 12-step sample came
    within 13% of the measured 1650.7 s)."""
    import oracle

    n, nnz = len(A[0]) - 1, len(A[1])
    variant = oracle.IR_FP32 if w["prec"] == "ir_fp32" else oracle.ONE_REDUCE
    scale = oracle_solve_bytes(n, nnz, ks_full) / oracle_solve_bytes(n, nnz, [min(sample_iters, sum(ks_full))])
    out = None
    for o in (oracle.get(), oracle.get_omp()):
        t0 = time.perf_counter()
        r = o.gmres(A, b, variant=variant, m=w["m"], tol=0.0, max_iter=sample_iters)
        dt = time.perf_counter() - t0
        entry = {"value": dt * scale, "unit": "s", "cores": o.threads, "kind": "oracle",
                 "sample": (f"first {r.iters} Arnoldi steps (+ tail, residual, update) of "
                            f"{'GMRES-IR' if w['prec'] == 'ir_fp32' else 'one-reduce GMRES'}({w['m']}) "
                            f"on the same {w['N']}^3 system, FP64 C oracle on {o.threads} host thread(s), "
                            f"{dt:.2f} s, scaled to the full solve ({sum(ks_full)} steps, {len(ks_full)} cycles) "
                            f"by a model of the oracle's memory traffic"),
                 "sample_seconds": dt}
        if out is None:
            out = entry
        else:
            entry["build"] = "oracle.c with -DORC_OMP -fopenmp (its vector loops on all host cores; timing only)"
            out["all_cores"] = entry
    return out


def _oracle_solve_job(job):
    """Worker of the all-core CPU baseline: one complete oracle solve (1 thread)."""
    from oracle import Oracle

    A, b, variant, m, tol, max_iter = job
    r = Oracle().gmres(A, b, variant=variant, m=m, tol=tol, max_iter=max_iter)
    return r.iters


def pool_oracle_solves(jobs):
    """Wall time of the independent oracle solves `jobs` run on all host cores
    (one spawned process per core, each solve on one thread; spawn, so no
    process forks after the CUDA context exists). Returns (seconds, cores)."""
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_solve_job, jobs[:1])  # workers started and warm before timing
        t0 = time.perf_counter()
        pool.map(_oracle_solve_job, jobs, chunksize=1)
        dt = time.perf_counter() - t0
    return dt, cores


def golden_profile(name):
    path = os.path.join(ROOT, "tests", "golden", f"oracle_profile_{name}.txt")
    if not os.path.exists(path):
        return None
    out = {}
    with open(path) as f:
        for line in f:
            f_ = line.split()
            if line.startswith("#") or len(f_) != 2:  # comments and the vector entries (history, x samples)
                continue
            out[f_[0]] = float(f_[1])
    return out


def golden_vectors(name):
    """All entries of an oracle profile, vectors (history, x samples) as arrays; None if absent."""
    path = os.path.join(ROOT, "tests", "golden", f"oracle_profile_{name}.txt")
    if not os.path.exists(path):
        return None
    out = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split(" ", 1)
            out[k] = np.array([float(t) for t in v.split()])
    return out


def oracle_sample_error(gold, x):
    """Relative 2-norm error of x against the FP64 oracle's solution over the
    profile's sampled entries (None without a profile)."""
    if gold is None or "x_sample" not in gold:
        return None
    idx = gold["x_sample_idx"].astype(np.int64)
    return float(np.linalg.norm(x[idx] - gold["x_sample"]) / np.linalg.norm(gold["x_sample"]))


# ----------------------------------------------------------------------------- reference arm
def single_config(w, n, nnz, world=1):
    """The `config` object of a single-system workload (both arms print the same one)."""
    ir = w["prec"] == "ir_fp32"
    return {"workload": workload_name(w), "n": n, "nnz": nnz, "m": w["m"], "tol": w["tol"],
            "parallelism": "replicas" if world > 1 else "1 GPU",
            "l2": (("inputs larger than L2 (Krylov basis %.1f GB >> 126 MB), no flush"
                    % ((4 if ir else 8) * n * (w["m"] + 1) / 1e9)) if (8 * n * (w["m"] + 1) > 126e6) else
                   ("L2-resident by design (Krylov basis %.1f MB < 126 MB: the latency-bound case), no flush"
                    % ((4 if ir else 8) * n * (w["m"] + 1) / 1e6)))}


def run_reference(args, w, rank, world):
    """The oracle as it stands (sequential FP64 C, one host thread) on the same
    workload. Every timed step is a bounded sample -- the first `sample`
    Arnoldi steps of the same solve, with the cycle tail, residual and update --
    and `value` scales the sample to a whole solve by a model of the oracle's
    own memory traffic and its recorded iteration profile (checked against one
    complete 256^3 oracle solve: within 13%). `ms_per_step` is the measured wall
    time of one sample, so steps x ms_per_step is the time actually spent."""
    if rank != 0:
        return None
    A = make_problem(w)
    _, b = P.rhs(A, seed=0)
    n, nnz = len(A[0]) - 1, len(A[1])
    if w["prec"] == "ir_fp32" and w["N"] >= 192:
        return {"impl": "reference", "unavailable": "no complete run of the oracle's GMRES-IR at this size "
                "to scale a sample by (at 192^3 27-point its sequential FP32 sums stall it: true residual "
                "1.43e-10 after 5000 steps, tol 1e-10)"}
    prof = golden_profile({256: "c2_one_reduce", 32: "c1"}.get(w["N"], "none"))
    if prof is None:
        return {"impl": "reference", "unavailable": "oracle iteration profile for this workload "
                "(tests/golden/oracle_profile_*.txt) has not been written"}
    import oracle

    ks = cycle_profile(int(prof["iters"]), w["m"])
    sample = 6 if w["N"] >= 128 else w["max_iter"]
    variant = oracle.IR_FP32 if w["prec"] == "ir_fp32" else oracle.ONE_REDUCE
    o = oracle.get()
    walls, iters = [], 0
    for s_ in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = o.gmres(A, b, variant=variant, m=w["m"], tol=0.0 if w["N"] >= 128 else w["tol"], max_iter=sample)
        dt = time.perf_counter() - t0
        iters = r.iters
        if s_ >= args.warmup:
            walls.append(dt)
    sample_s = float(np.mean(walls))
    full = iters >= int(prof["iters"])  # the sample is the whole solve
    v = sample_s if full else sample_s * oracle_solve_bytes(n, nnz, ks) / oracle_solve_bytes(n, nnz, [iters])
    what = ("the complete solve" if full else
            f"first {iters} Arnoldi steps (+ tail, residual, update) of the same solve, scaled to the whole solve "
            f"({sum(ks)} steps, {len(ks)} cycles, the oracle's own profile) by a model of its memory traffic")
    # the same sample once more on all host cores (timing build of the same source)
    om = oracle.get_omp()
    t0 = time.perf_counter()
    r2 = om.gmres(A, b, variant=variant, m=w["m"], tol=0.0 if w["N"] >= 128 else w["tol"], max_iter=sample)
    dt_all = time.perf_counter() - t0
    v_all = dt_all if full else dt_all * oracle_solve_bytes(n, nnz, ks) / oracle_solve_bytes(n, nnz, [r2.iters])
    metric = METRIC_IR.format(tol=("%.0e" % w["tol"]).replace("e-0", "e-")) if w["prec"] == "ir_fp32" else METRIC
    return {
        "impl": "reference", "metric": metric, "value": v, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sample_s, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded stencil, x_true ~ U[-1,1])",
        "config": single_config(w, n, nnz, world),
        "value_basis": ("measured" if full else "extrapolated") + ": each timed step runs " + what
                       + "; ms_per_step is the measured wall time of one such sample",
        "sample_seconds": sample_s,
        "cpu_baseline": {"value": v, "unit": "s", "cores": o.threads, "kind": "oracle",
                         "sample": what + f", FP64 C oracle on {o.threads} host thread, {sample_s:.2f} s per sample",
                         "all_cores": {"value": v_all, "unit": "s", "cores": om.threads, "kind": "oracle",
                                       "sample": f"the same sample once on {om.threads} host threads "
                                                 f"(oracle.c built with -DORC_OMP -fopenmp): {dt_all:.2f} s"}},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ----------------------------------------------------------------------------- our arm
def timed_solves(torch, s, bd, x, steps, warmup, stream):
    """K timed solves (CUDA events on the solver's stream, no per-kernel timing
    inside), then one more solve, untimed, with per-kernel timing for the
    roofline (its graphs with timing nodes are captured by a warm-up solve)."""
    infos = []
    s.set_profile(False)
    for _ in range(warmup):
        x.zero_()
        s.solve(bd, x)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ms = 0.0
    for _ in range(steps):
        with torch.cuda.stream(stream):
            x.zero_()
        torch.cuda.synchronize()
        e0.record(stream)
        infos.append(s.solve(bd, x))
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    s.set_profile(True)
    for _ in range(2):  # the first profiled solve captures the timed graphs
        with torch.cuda.stream(stream):
            x.zero_()
        s.solve(bd, x)
    prof = s.profile()
    s.set_profile(False)
    return ms / steps, infos, prof


def run_ours(args, w, rank, world, dist):
    import torch

    from paper_1809_05805_b300 import lsgmres

    lsgmres.load()  # fails loudly when the CUDA library is missing
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    A = make_problem(w)
    _, b = P.rhs(A, seed=0)
    n, nnz = len(A[0]) - 1, len(A[1])
    peaks = load_peaks()
    ir = w["prec"] == "ir_fp32"

    def barrier():
        rank_barrier(dist)

    def max_over_ranks(v):
        return rank_max(dist, v)

    bd = torch.from_numpy(b).cuda()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    s = lsgmres.Solver(A, m=w["m"], tol=w["tol"], ortho="one_reduce_mgs", max_iter=w["max_iter"], stream=stream,
                       prec=w["prec"])
    # FP64 cycles: the block dot and MAXPY products on the integer pipes (the
    # library's default where the tile-pair ring kernel runs); small systems run
    # each restart cycle in one launch (the library's default where it applies)
    fx = s.set_block_dot(True)
    persistent = s.set_persistent(-1)

    barrier()
    with ClockSampler(local) as clk:
        ms, infos, prof = timed_solves(torch, s, bd, x, args.steps, args.warmup, stream)
        barrier()
    clocks = clk.summary()
    ms = max_over_ranks(ms)
    info = infos[-1]
    xs = x.cpu().numpy()
    true_rel = float(np.linalg.norm(b - P.to_scipy(A) @ xs) / np.linalg.norm(b))
    hist_1r = s.history()

    # the comparison leg on the same kernels: plain MGS (FP64 workloads) or the
    # FP64 one-reduce solve (GMRES-IR workload, which also gives IR's error)
    mgs = None
    fp64 = None
    if not args.no_mgs and w["compare"] == "fp64":
        s.set(ortho="one_reduce_mgs", prec="fp64", max_iter=w["max_iter"])
        ms_f, infos_f, prof_f = timed_solves(torch, s, bd, x, max(1, min(args.steps, 2)), 1, stream)
        ms_f = max_over_ranks(ms_f)
        i64 = infos_f[-1]
        x64 = x.cpu().numpy()
        gold = golden_vectors(w["golden_fp64"]) if w.get("golden_fp64") else None
        fp64 = {"time_to_solve_s": ms_f / 1e3, "iters": i64.iters, "restarts": i64.restarts,
                "rel_resid_true": i64.rel_resid_true,
                "ir_rel_error_vs_fp64": float(np.linalg.norm(xs - x64) / np.linalg.norm(x64)),
                # against the CPU oracle's complete FP64 one-reduce solve (64 sampled entries)
                "ir_rel_error_vs_fp64_oracle": oracle_sample_error(gold, xs),
                "fp64_rel_error_vs_fp64_oracle": oracle_sample_error(gold, x64),
                "oracle_profile": ("tests/golden/oracle_profile_%s.txt" % w["golden_fp64"]) if gold else None,
                "step_tflops_fp64": prof_f["one_reduce_step"]["flops"] / (prof_f["one_reduce_step"]["ms"] * 1e9)
                if prof_f["one_reduce_step"]["ms"] else None}
        # BF16 basis storage (FP32 arithmetic): the other GMRES-IR storage option
        s.set(ortho="one_reduce_mgs", prec="ir_bf16", max_iter=w["max_iter"])
        ms_b, infos_b, prof_b = timed_solves(torch, s, bd, x, max(1, min(args.steps, 2)), 1, stream)
        ib16 = infos_b[-1]
        xb = x.cpu().numpy()
        fp64["ir_bf16"] = {"time_to_solve_s": max_over_ranks(ms_b) / 1e3, "iters": ib16.iters,
                           "restarts": ib16.restarts, "rel_resid_true": ib16.rel_resid_true,
                           "rel_error_vs_fp64": float(np.linalg.norm(xb - x64) / np.linalg.norm(x64)),
                           "rel_error_vs_fp64_oracle": oracle_sample_error(gold, xb),
                           "step_hbm_gbs": prof_b["one_reduce_step"]["bytes"] / (prof_b["one_reduce_step"]["ms"] * 1e6)
                           if prof_b["one_reduce_step"]["ms"] else None,
                           "maxpy_hbm_gbs": prof_b["arnoldi_maxpy"]["bytes"] / (prof_b["arnoldi_maxpy"]["ms"] * 1e6)
                           if prof_b["arnoldi_maxpy"]["ms"] else None}
        s.set(ortho="one_reduce_mgs", prec=w["prec"], max_iter=w["max_iter"])
    if not args.no_mgs and w["compare"] == "mgs":
        s.set(ortho="mgs", max_iter=w["max_iter"])
        ms_m, infos_m, prof_m = timed_solves(torch, s, bd, x, max(1, min(args.steps, 2)), 1, stream)
        ms_m = max_over_ranks(ms_m)
        im = infos_m[-1]
        mgs = {"time_to_solve_s": ms_m / 1e3, "iters": im.iters, "restarts": im.restarts,
               "reductions": im.reductions, "kernel_launches": im.kernel_launches,
               "rel_resid_true": im.rel_resid_true,
               "alg_gbs": sum(v["bytes"] for v in prof_m.values()) / (sum(v["ms"] for v in prof_m.values()) * 1e6)
               if prof_m else None}
        s.set(ortho="one_reduce_mgs", max_iter=w["max_iter"])

    # small systems: the same solve with one launch per step and MAXPY, for comparison
    per_step = None
    if persistent and not args.no_mgs:
        s.set_persistent(0)
        ms_p, infos_p, _ = timed_solves(torch, s, bd, x, max(1, min(args.steps, 10)), 3, stream)
        ip = infos_p[-1]
        per_step = {"time_to_solve_s": max_over_ranks(ms_p) / 1e3, "iters": ip.iters,
                    "us_per_arnoldi_step": ms_p * 1e3 / max(ip.iters, 1), "kernel_launches": ip.kernel_launches,
                    "rel_resid_true": ip.rel_resid_true}
        s.set_persistent(-1)

    # the same solve with every FP64 product on the FP64 pipe (FMAs), for comparison
    dfma = None
    if fx and not ir and not args.no_mgs:
        s.set_block_dot(False)
        ms_d, infos_d, prof_d = timed_solves(torch, s, bd, x, max(1, min(args.steps, 2)), 1, stream)
        idd = infos_d[-1]
        std = prof_d["one_reduce_step"]
        dfma = {"time_to_solve_s": max_over_ranks(ms_d) / 1e3, "iters": idd.iters, "restarts": idd.restarts,
                "rel_resid_true": idd.rel_resid_true,
                "step_launch_avg_ms": std["ms"] / max(std["launches"], 1),
                "step_tflops": std["flops"] / (std["ms"] * 1e9) if std["ms"] else None,
                "maxpy_launch_avg_ms": prof_d["arnoldi_maxpy"]["ms"] / max(prof_d["arnoldi_maxpy"]["launches"], 1)}
        s.set_block_dot(True)

    # the paper's sibling schemes on the same kernels (Algorithm 5: two reductions
    # per step; Algorithm 8: Givens rotations on column pairs)
    siblings = None
    if not args.no_mgs and w["compare"] == "mgs":
        siblings = {}
        for ortho in ("cgs2_lvl2", "one_reduce_pipe2"):
            s.set(ortho=ortho, max_iter=w["max_iter"])
            ms_s, infos_s, prof_s = timed_solves(torch, s, bd, x, 1, 1, stream)
            isb = infos_s[-1]
            siblings[ortho] = {"time_to_solve_s": max_over_ranks(ms_s) / 1e3, "iters": isb.iters,
                               "restarts": isb.restarts, "reductions": isb.reductions,
                               "rel_resid_true": isb.rel_resid_true}
        s.set(ortho="one_reduce_mgs", max_iter=w["max_iter"])

    # end to end through the host-buffer entry point (copies inside the call)
    bh = torch.from_numpy(b).pin_memory().numpy()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
    s.set_profile(False)
    e2e_ms = 0.0
    e2e_steps = max(1, min(args.steps, 2))
    s.solve_host(bh, xh)  # warm the staging buffers
    for _ in range(e2e_steps):
        xh[:] = 0.0
        t0 = time.perf_counter()
        s.solve_host(bh, xh)
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_ms = max_over_ranks(e2e_ms / e2e_steps)

    # roofline of the dominant kernel (the fused SpMV + block-dot step)
    st = prof["one_reduce_step"]
    mx = prof["arnoldi_maxpy"]
    clk_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
    step_avg_ms = st["ms"] / max(st["launches"], 1)
    step_tflops = st["flops"] / (st["ms"] * 1e-3) / 1e12 if st["ms"] else None
    step_gbs = st["bytes"] / (st["ms"] * 1e-3) / 1e9 if st["ms"] else None
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    if persistent and not ir:  # one launch per cycle: the cycle kernel is the only one that matters
        cy = prof["persistent_cycle"]
        cy_gbs = cy["bytes"] / (cy["ms"] * 1e-3) / 1e9 if cy["ms"] else None
        roofline = {
            "kernel": "k_cycle_persistent (every Arnoldi step of a restart cycle in one cooperative launch)",
            "bound": "hbm", "achieved": cy_gbs, "peak": hbm, "unit": "GB/s",
            "frac": cy_gbs / hbm if cy_gbs else None,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth, of measured)",
            "note": "latency-bound by design: the working set (%.1f MB) is L2-resident, so the fraction of HBM "
                    "bandwidth is low; us_per_arnoldi_step and grid_syncs_per_step are the figures of merit"
                    % ((8 * n * (w["m"] + 2) + 12 * nnz) / 1e6),
            "traffic": None,
            "launch_avg_ms": cy["ms"] / max(cy["launches"], 1), "launches": cy["launches"],
            "alg_bytes_per_launch": cy["bytes"] / max(cy["launches"], 1),
            "fp64_tflops": cy["flops"] / (cy["ms"] * 1e9) if cy["ms"] else None,
        }
    elif ir:  # FP32 cycles: the step kernel streams at FP32 rates, HBM is the bound
        roofline = {
            "kernel": "k_one_reduce_step<float> (fused FP32 CSR SpMV + block dot + epilogue)",
            "bound": "hbm", "achieved": step_gbs, "peak": hbm, "unit": "GB/s",
            "frac": step_gbs / hbm if step_gbs else None,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth, of measured)",
            "traffic": ((STEP32_TRAFFIC_RATIO[w["stencil"]] * st["bytes"] / max(st["launches"], 1))
                        if STEP32_TRAFFIC_RATIO and w["prec"] == "ir_fp32" else None),
            "traffic_source": ("ncu dram bytes / algorithmic bytes of the FP32 step "
                               + ("(single tiles) at 144^3 27-point" if w["stencil"] == "27pt"
                                  else "(tile pairs, column ring) at 128^3 7-point")
                               + " (same kernel build), times this run's algorithmic bytes per launch"),
            "launch_avg_ms": step_avg_ms, "launches": st["launches"],
            "alg_bytes_per_launch": st["bytes"] / max(st["launches"], 1),
            "fp32_tflops": step_tflops,
            "maxpy": {"launch_avg_ms": mx["ms"] / max(mx["launches"], 1),
                      "hbm_gbs": mx["bytes"] / (mx["ms"] * 1e-3) / 1e9 if mx["ms"] else None,
                      "hbm_frac_of_measured": (mx["bytes"] / (mx["ms"] * 1e-3) / 1e9) / hbm if mx["ms"] else None},
        }
    elif fx:  # FP64 cycles with fixed-point products: HBM is the bound again
        pk = fp64_peak()
        survey_bytes = st["bytes"] - 8.0 * n * max(st["launches"] - info.restarts, 0)
        roofline = {
            "kernel": "k_one_reduce_step<., double, double, 6> (fused CSR SpMV + block dot [V u]^T[u w] with the "
                      "basis columns' products as exact fixed-point integers + epilogue)",
            "bound": "hbm", "achieved": step_gbs, "peak": hbm, "unit": "GB/s",
            "frac": step_gbs / hbm if step_gbs else None,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth, of measured)",
            "alg_bytes_formula": "4(n+1) + 12 nnz + 8n(j+1) + 8n (CSR, u and V_j read, w written; the basis "
                                 "is read as stored limbs, 8 bytes per entry, and the limbs of u, 8n, written "
                                 "on top are not counted)",
            "hbm_frac_of_measured_survey_bytes": (survey_bytes / (st["ms"] * 1e-3) / 1e9) / hbm if st["ms"] else None,
            "traffic": (STEP6_TRAFFIC_RATIO * st["bytes"] / max(st["launches"], 1)) if STEP6_TRAFFIC_RATIO else None,
            "traffic_source": "ncu dram bytes / algorithmic bytes of the fixed-point step at 128^3 (same kernel build), "
                              "times this run's algorithmic bytes per launch",
            "launch_avg_ms": step_avg_ms, "launches": st["launches"],
            "alg_bytes_per_launch": st["bytes"] / max(st["launches"], 1),
            "fp64_method_tflops": step_tflops,
            "fp64_pipe_peak_tflops": pk["tflops"], "fp64_pipe_peak_source": pk["source"],
            "maxpy": {"kernel": "k_maxpy_fx", "launch_avg_ms": mx["ms"] / max(mx["launches"], 1),
                      "hbm_gbs": mx["bytes"] / (mx["ms"] * 1e-3) / 1e9 if mx["ms"] else None,
                      "hbm_frac_of_measured": (mx["bytes"] / (mx["ms"] * 1e-3) / 1e9) / hbm if mx["ms"] else None},
        }
    else:
        pk = fp64_peak()
        # the method's own byte count per step (12 nnz + 4n + 8n(j+1): CSR, u and
        # V_j read) -- the library's count without the 8n of w written by each
        # launch that ran the SpMV (all but the cycle tails)
        survey_bytes = st["bytes"] - 8.0 * n * max(st["launches"] - info.restarts, 0)
        roofline = {
            "kernel": "k_one_reduce_step (fused CSR SpMV + block dot [V u]^T[u w] + epilogue)",
            "bound": "alu", "achieved": step_tflops, "peak": pk["tflops"], "unit": "TFLOP/s",
            "frac": step_tflops / pk["tflops"] if step_tflops else None,
            "peak_source": pk["source"] + " (of measured)",
            "peak_nominal": pk["nominal_tflops"],
            "frac_of_nominal": step_tflops / pk["nominal_tflops"] if step_tflops else None,
            "hbm_frac_of_measured_survey_bytes": (survey_bytes / (st["ms"] * 1e-3) / 1e9) / hbm if st["ms"] else None,
            "traffic": (STEP_TRAFFIC_RATIO * st["bytes"] / max(st["launches"], 1)) if STEP_TRAFFIC_RATIO else None,
            "traffic_source": "ncu dram bytes / algorithmic bytes at 128^3 (same kernel build), times this run's "
                              "algorithmic bytes per launch",
            "launch_avg_ms": step_avg_ms, "launches": st["launches"],
            "alg_flops_per_launch": st["flops"] / max(st["launches"], 1),
            "alg_bytes_per_launch": st["bytes"] / max(st["launches"], 1),
            "hbm_gbs": step_gbs, "hbm_frac_of_measured": step_gbs / hbm if step_gbs else None,
            "maxpy": {"launch_avg_ms": mx["ms"] / max(mx["launches"], 1),
                      "tflops": mx["flops"] / (mx["ms"] * 1e-3) / 1e12 if mx["ms"] else None,
                      "hbm_gbs": mx["bytes"] / (mx["ms"] * 1e-3) / 1e9 if mx["ms"] else None},
        }
    total_bytes = sum(v["bytes"] for v in prof.values())
    total_ms_prof = sum(v["ms"] for v in prof.values())

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ks = cycle_profile(info.iters, w["m"])
        sample = 12 if w["N"] >= 128 else w["max_iter"]
        cpu = cpu_baseline(A, b, w, ks, sample)

    line = {
        "metric": METRIC_IR.format(tol=("%.0e" % w["tol"]).replace("e-0", "e-")) if ir else METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 cycles / f64 restarts" if ir else "f64",
        "data": "synthetic (seeded stencil, x_true ~ U[-1,1])",
        "config": single_config(w, n, nnz, world),
        "fixed_point_products": bool(fx) and not ir,
        "iters": info.iters, "restarts": info.restarts, "reductions": info.reductions,
        "grid_syncs": info.grid_syncs, "rel_resid_true": true_rel,
        "us_per_arnoldi_step": ms * 1e3 / max(info.iters, 1),
        "grid_syncs_per_step": info.grid_syncs / max(info.iters, 1),
        "solves_per_s": world / (ms / 1e3),
        "alg_hbm_gbs_whole_solve": total_bytes / (total_ms_prof * 1e6) if total_ms_prof else None,
        "mgs": mgs,
        "speedup_vs_mgs": (mgs["time_to_solve_s"] / (ms / 1e3)) if mgs else None,
        "one_launch_per_cycle": bool(persistent),
        "per_step_launches": per_step,
        "speedup_vs_per_step_launches": (per_step["time_to_solve_s"] / (ms / 1e3)) if per_step else None,
        "fma_products": dfma,
        "speedup_vs_fma_products": (dfma["time_to_solve_s"] / (ms / 1e3)) if dfma else None,
        "siblings": siblings,
        "fp64_one_reduce": fp64,
        "speedup_vs_fp64": (fp64["time_to_solve_s"] / (ms / 1e3)) if fp64 else None,
        "e2e": {"value": e2e_ms / 1e3, "unit": "s", "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 8 * n},
        "gpu_launches": int(sum(i.kernel_launches for i in infos)),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "history_first": [float(h) for h in hist_1r[:3]],
    }
    s.close()
    return line


# ----------------------------------------------------------------------------- batched workload
def batch_problem(w):
    pars = P.batch_2d_params(w["count"], seed=w["seed"], side=w["side"])
    mats, rhs = [], []
    for i, par in enumerate(pars):
        A = P.batch_2d_system(par)
        mats.append(A)
        rhs.append(P.rhs(A, seed=i)[1])
    return pars, mats, rhs


def batch_workload_name(w, mats):
    n = sum(len(A[0]) - 1 for A in mats)
    nnz = sum(len(A[1]) for A in mats)
    return (f"{w['count']} independent 2D 9-point variable-coefficient convection-diffusion systems, grid side "
            f"log-uniform {w['side'][0]}..{w['side'][1]} (total n={n}, nnz={nnz}), kappa log-uniform [0.1,10], "
            f"cell Peclet U[0,2], FP64 CSR, batched one-reduce GMRES({w['m']}) vs the same systems solved one "
            f"after another, tol {w['tol']:g}, x0=0")


def batch_cpu_baseline(mats, rhs, w, iters, budget_s=20.0):
    """Time the FP64 oracle (1 thread) on complete solves of a sample of the
    systems (every 16th, in order, until `budget_s`), scaled to the whole batch
    by the ratio of sum(n_i * iters_i) over all systems to that over the sample."""
    from oracle import Oracle

    orc = Oracle()
    t_tot, work_s, names = 0.0, 0.0, []
    for i in range(0, len(mats), 16):
        t0 = time.perf_counter()
        r = orc.gmres(mats[i], rhs[i], variant=1, m=w["m"], tol=w["tol"], max_iter=w["max_iter"])
        t_tot += time.perf_counter() - t0
        work_s += (len(mats[i][0]) - 1) * r.iters
        names.append(i)
        if t_tot >= budget_s:
            break
    work_all = sum((len(A[0]) - 1) * k for A, k in zip(mats, iters))
    v = t_tot * work_all / work_s
    # all host cores: the systems are independent, so the same sample solved by
    # one process per core
    dt, cores = pool_oracle_solves([(mats[i], rhs[i], 1, w["m"], w["tol"], w["max_iter"]) for i in names])
    return {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": f"complete oracle solves of {len(names)} of the {len(mats)} systems (every 16th), "
                      f"{t_tot:.1f} s, scaled by sum(n_i * iters_i) over all systems / over the sample",
            "all_cores": {"value": dt * work_all / work_s, "unit": "s", "cores": cores, "kind": "oracle",
                          "sample": f"the same {len(names)} solves on {cores} spawned processes (one per core, "
                                    f"1 thread each): {dt:.1f} s wall, scaled the same way"}}


def run_batch_reference(args, w, rank):
    if rank != 0:
        return None
    _, mats, rhs = batch_problem(w)
    from oracle import Oracle

    orc = Oracle()
    # every 32nd system per step (sizes are drawn independently, so the sample
    # is representative), scaled to the batch by total n / sample n
    vals = []
    for s in range(args.warmup + args.steps):
        t_tot, work_s, cnt = 0.0, 0.0, 0
        for i in range(0, len(mats), 32):
            t0 = time.perf_counter()
            r = orc.gmres(mats[i], rhs[i], variant=1, m=w["m"], tol=w["tol"], max_iter=w["max_iter"])
            t_tot += time.perf_counter() - t0
            work_s += len(mats[i][0]) - 1
            cnt += 1
            if t_tot >= 8.0:
                break
        v = t_tot * sum(len(A[0]) - 1 for A in mats) / work_s
        if s >= args.warmup:
            vals.append(v)
    v = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC_BATCH, "value": v, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * v, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": batch_workload_name(w, mats), "m": w["m"], "tol": w["tol"]},
        "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": f"complete oracle solves of {cnt} systems (every 32nd) per step, scaled by "
                                   f"total n / sample n"},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return line


def run_batch(args, w, rank, world, dist):
    import torch

    from paper_1809_05805_b300 import lsgmres

    lsgmres.load()  # fails loudly when the CUDA library is missing
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    pars, mats, rhs = batch_problem(w)
    S = len(mats)
    ntot = sum(len(A[0]) - 1 for A in mats)
    peaks = load_peaks()

    def barrier():
        rank_barrier(dist)

    def max_over_ranks(v):
        return rank_max(dist, v)

    t0 = time.perf_counter()
    bs = lsgmres.BatchSolver(mats, m=w["m"], tol=w["tol"], max_iter=w["max_iter"], stream=stream)
    create_s = time.perf_counter() - t0
    bd = [torch.from_numpy(b).cuda() for b in rhs]
    xd = [torch.zeros(len(b), dtype=torch.float64, device="cuda") for b in rhs]
    bs.set_profile(False)  # timed without per-launch timing nodes; profiled after
    if getattr(args, "batch_shape", None):
        ctas, rows = (int(v) for v in args.batch_shape.split(","))
        bs.set_grid(ctas)
        bs.set_rows_per_thread(rows)
    fx = bs.set_block_dot(True)  # the default: fixed-point products on FP64 tile pairs (autotuned rows per thread)

    def one_solve():
        with torch.cuda.stream(stream):
            for x in xd:
                x.zero_()
        return bs.solve(bd, xd)

    for _ in range(args.warmup):
        one_solve()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ms, prof, launches = 0.0, None, 0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0.record(stream)
            infos = one_solve()
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            launches += infos[0].kernel_launches
        barrier()
    clocks = clk.summary()
    # per-kernel timing of one more solve, untimed (the first captures its graphs)
    bs.set_profile(True)
    one_solve()
    one_solve()
    prof = bs.profile()
    ms = max_over_ranks(ms / args.steps)
    xs = [x.cpu().numpy() for x in xd]
    true_rel = [float(np.linalg.norm(b - P.to_scipy(A) @ x) / np.linalg.norm(b)) for A, b, x in zip(mats, rhs, xs)]
    iters = [i.iters for i in infos]

    # the comparison leg: the same systems solved one after another by the
    # single-system solver (same kernels, graphs on the same stream)
    seq = None
    if not args.no_mgs:
        seq_ms, seq_iters = 0.0, []
        for A, b in zip(mats, bd):
            s1 = lsgmres.Solver(A, m=w["m"], tol=w["tol"], ortho="one_reduce_mgs", max_iter=w["max_iter"],
                                stream=stream)
            x1 = torch.zeros(len(b), dtype=torch.float64, device="cuda")
            s1.solve(b, x1)  # captures its graphs
            x1.zero_()
            torch.cuda.synchronize()
            e0.record(stream)
            inf1 = s1.solve(b, x1)
            e1.record(stream)
            e1.synchronize()
            seq_ms += e0.elapsed_time(e1)
            seq_iters.append(inf1.iters)
            s1.close()
        seq = {"time_to_solve_s": seq_ms / 1e3, "iters_equal_to_batched": int(sum(a == b for a, b in
                                                                                 zip(seq_iters, iters))),
               "systems": S}

    # end to end through the host-buffer entry point (copies inside the call)
    bh = [torch.from_numpy(b).pin_memory().numpy() for b in rhs]
    xh = [torch.zeros(len(b), dtype=torch.float64).pin_memory().numpy() for b in rhs]
    bs.set_profile(False)
    bs.solve_host(bh, xh)
    e2e_steps = max(1, min(args.steps, 2))
    e2e_ms = 0.0
    for _ in range(e2e_steps):
        for x in xh:
            x[:] = 0.0
        t0 = time.perf_counter()
        bs.solve_host(bh, xh)
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_ms = max_over_ranks(e2e_ms / e2e_steps)

    st = prof["one_reduce_step"]
    mx = prof["arnoldi_maxpy"]
    pk = fp64_peak()
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    step_tflops = st["flops"] / (st["ms"] * 1e-3) / 1e12 if st["ms"] else None
    step_gbs = st["bytes"] / (st["ms"] * 1e-3) / 1e9 if st["ms"] else None
    kname = ("ke_step (batched fused CSR SpMV + block dot, per-(CTA, system) partial sums, per-system epilogue"
             + ("; tile pairs, the basis products as exact fixed-point integers"
                + (", basis streamed through the per-warp cp.async column ring)" if fx == 2 else ")") if fx else ")"))
    if fx:  # the FP64 pipe no longer bounds it: HBM does
        bound = {"bound": "hbm", "achieved": step_gbs, "peak": hbm, "unit": "GB/s",
                 "frac": step_gbs / hbm if step_gbs else None,
                 "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth, of measured)",
                 "fp64_method_tflops": step_tflops, "fp64_pipe_peak_tflops": pk["tflops"]}
    else:
        bound = {"bound": "alu", "achieved": step_tflops, "peak": pk["tflops"], "unit": "TFLOP/s",
                 "frac": step_tflops / pk["tflops"] if step_tflops else None,
                 "peak_source": pk["source"] + " (of measured)", "peak_nominal": pk["nominal_tflops"]}
    roofline = {
        "kernel": kname, **bound,
        "fixed_point_products": bool(fx), "column_ring": fx == 2,
        "traffic": None,
        "launch_avg_ms": st["ms"] / max(st["launches"], 1), "launches": st["launches"],
        "alg_flops_per_launch": st["flops"] / max(st["launches"], 1),
        "alg_bytes_per_launch": st["bytes"] / max(st["launches"], 1),
        "hbm_gbs": step_gbs, "hbm_frac_of_measured": step_gbs / hbm if step_gbs else None,
        "noop_launches": prof["noop"]["launches"],
        "maxpy": {"launch_avg_ms": mx["ms"] / max(mx["launches"], 1),
                  "tflops": mx["flops"] / (mx["ms"] * 1e-3) / 1e12 if mx["ms"] else None,
                  "hbm_gbs": mx["bytes"] / (mx["ms"] * 1e-3) / 1e9 if mx["ms"] else None},
    }
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = batch_cpu_baseline(mats, rhs, w, iters)
    line = {
        "metric": METRIC_BATCH, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded 2D stencils, x_true ~ U[-1,1])",
        "config": {"workload": batch_workload_name(w, mats), "systems": S, "n_total": ntot, "m": w["m"],
                   "tol": w["tol"], "grid_ctas": bs.grid, "create_s": create_s,
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 (batch Krylov basis %.1f GB >> 126 MB), no flush"
                         % (8 * ntot * (w["m"] + 1) / 1e9)},
        "iters_max": max(iters), "iters_median": float(np.median(iters)),
        "all_converged": all(i.status == 0 for i in infos), "max_rel_resid_true": max(true_rel),
        "solves_per_s": world * S / (ms / 1e3),
        "sequential": seq,
        "speedup_vs_sequential": (seq["time_to_solve_s"] / (ms / 1e3)) if seq else None,
        "e2e": {"value": e2e_ms / 1e3, "unit": "s", "h2d_bytes_per_step": 16 * ntot, "d2h_bytes_per_step": 8 * ntot},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    bs.close()
    return line


# ----------------------------------------------------------------------------- serving workload
def serve_requests(w):
    """Seeded request stream: arrival times, cube sides, precisions, and the
    systems (one matrix per distinct side, b = A x_true per request)."""
    rng = np.random.default_rng(w["seed"])
    k = w["requests"]
    arrivals = np.cumsum(rng.exponential(1.0 / w["rate"], k))
    arrivals -= arrivals[0]
    lo, hi = w["n_range"]
    n = np.exp(rng.uniform(np.log(lo), np.log(hi), k))
    grid = np.unique(np.round(np.exp(np.linspace(np.log(lo ** (1 / 3)), np.log(hi ** (1 / 3)), w["sides"]))))
    sides = grid[np.abs(np.log(grid)[None, :] - np.log(np.cbrt(n))[:, None]).argmin(axis=1)].astype(int)
    precs = np.where(rng.random(k) < w["ir_frac"], "ir_fp32", "fp64")
    mats = {N: P.conv_diff_7pt(int(N)) for N in np.unique(sides)}
    reqs = []
    for i in range(k):
        A = mats[int(sides[i])]
        reqs.append(dict(A=A, b=P.rhs(A, seed=1000 + i)[1], prec=str(precs[i]), t=float(arrivals[i]),
                         n=int(sides[i]) ** 3))
    return reqs


def serve_trace(reqs, rate, duration, seed):
    """A finite Poisson trace of `duration` seconds of arrivals at `rate`/s,
    each request drawn (seeded) from the pool `reqs` (same sizes, precisions
    and systems as the stream)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            return out
        out.append(dict(reqs[int(rng.integers(len(reqs)))], t=t))


def serve_run(lsgmres, sv, reqs, w, time_scale=1.0):
    """Submit the requests at their arrival times (multiplied by time_scale)
    from one thread, wait for all; returns wall time, latencies and the
    solutions."""
    import threading

    xs = [np.zeros(r["n"]) for r in reqs]
    ids = [None] * len(reqs)
    slip = np.zeros(len(reqs))
    t0 = time.perf_counter()

    def feed():
        for i, r in enumerate(reqs):
            due = t0 + r["t"] * time_scale
            dt = due - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            slip[i] = max(0.0, time.perf_counter() - due)
            ids[i] = sv.submit(r["A"], r["b"], xs[i], tol=w["tol"], prec=r["prec"], max_iter=w["max_iter"])

    th = threading.Thread(target=feed)
    th.start()
    th.join()
    sv.drain(timeout=900)
    wall = time.perf_counter() - t0
    infos = [sv.wait(i, timeout=10) for i in ids]
    # latency from the scheduled arrival: the submit thread's delay plus the
    # server's submit-to-completion time
    lat = np.array([i.seconds for i in infos]) + slip
    for i in ids:
        sv.release(i)
    return wall, lat, infos, xs


def run_serve(args, w, rank, world, dist):
    import torch

    from paper_1809_05805_b300 import lsgmres

    lsgmres.load()  # fails loudly when the CUDA library is missing
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    peaks = load_peaks()
    reqs = serve_requests(w)
    k = len(reqs)
    sv = lsgmres.Server(m=w["m"], max_iter=w["max_iter"], max_requests=w["max_requests"],
                        hbm_budget_bytes=w["budget"], ir_share=w["ir_frac"])
    # warm-up: graph capture of the cycle shapes and first-touch costs
    for _ in range(max(1, args.warmup)):
        serve_run(lsgmres, sv, reqs[: min(16, k)], w)
    with ClockSampler(local) as clk:  # timed without per-launch timing nodes
        walls, lats, all_infos, xs_last = [], [], None, None
        for _ in range(args.steps):
            wall, lat, infos, xs = serve_run(lsgmres, sv, reqs, w)
            walls.append(wall)
            lats.append(lat)
            all_infos, xs_last = infos, xs
    clocks = clk.summary()
    st = sv.stats()
    # per-kernel timing of the engines over one more run of the stream, untimed
    sv.set_profile(True)
    serve_run(lsgmres, sv, reqs, w)
    prof = [sv.profile(0), sv.profile(1)]
    lat = np.concatenate(lats)
    wall = float(np.mean(walls))
    thr = k / wall
    # replicas: every rank serves its own copy of the stream; the job's throughput
    # is all ranks' requests over the slowest rank's makespan
    job_thr = world * k / rank_max(dist, wall)
    true_rel = [float(np.linalg.norm(r["b"] - P.to_scipy(r["A"]) @ x) / np.linalg.norm(r["b"]))
                for r, x in zip(reqs, xs_last)]
    # sustained service: finite Poisson traces of sweep_s seconds at fractions of
    # the capacity the burst measured, requests drawn from the same stream
    sv.set_profile(False)
    sweep = []
    for i, f in enumerate(w.get("sweep", ())):
        rate = f * thr
        trace = serve_trace(reqs, rate, w["sweep_s"], seed=w["seed"] + 17 + i)
        wall_t, lat_t, infos_t, _ = serve_run(lsgmres, sv, trace, w)
        last_arrival = trace[-1]["t"] if trace else 0.0
        sweep.append({"fraction_of_burst_capacity": f, "offered_rate": rate, "requests": len(trace),
                      "arrivals_s": last_arrival, "solves_per_s": len(trace) / wall_t,
                      "latency_p50_s": float(np.percentile(lat_t, 50)),
                      "latency_p99_s": float(np.percentile(lat_t, 99)),
                      "latency_max_s": float(np.max(lat_t)),
                      "drain_after_last_arrival_s": wall_t - last_arrival,
                      "all_converged": all(x.status == 0 for x in infos_t)})
    sv.close()

    # baseline: the same requests one at a time in arrival order by the
    # single-system solver (FIFO queue simulated from the measured solve times)
    seq = None
    if not args.no_mgs:
        stream = torch.cuda.Stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        solo = []
        cache = {}
        for r in reqs:
            key = (r["n"], r["prec"])
            if key not in cache:
                cache[key] = lsgmres.Solver(r["A"], m=w["m"], tol=w["tol"], max_iter=w["max_iter"], stream=stream,
                                            prec=r["prec"])
            s1 = cache[key]
            bd = torch.from_numpy(r["b"]).cuda()
            x1 = torch.zeros(r["n"], dtype=torch.float64, device="cuda")
            s1.solve(bd, x1)  # graph capture for this shape
            x1.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s1.solve(bd, x1)
            x1.cpu()
            solo.append(time.perf_counter() - t0)
        for s1 in cache.values():
            s1.close()
        arr = np.array([r["t"] for r in reqs])
        end = 0.0
        lat_q = []
        for a, d in zip(arr, solo):
            end = max(end, a) + d
            lat_q.append(end - a)
        seq = {"solves_per_s": k / end, "latency_p50_s": float(np.percentile(lat_q, 50)),
               "latency_p99_s": float(np.percentile(lat_q, 99)), "solo_solve_s_sum": float(np.sum(solo)),
               "note": "each request alone on the single-system solver (graphs on one stream), FIFO in arrival "
                       "order; queueing simulated from the measured solve times"}

    st0, st1 = prof[0]["one_reduce_step"], prof[1]["one_reduce_step"]
    pk = fp64_peak()
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    tf0 = st0["flops"] / (st0["ms"] * 1e-3) / 1e12 if st0["ms"] else None
    gbs1 = st1["bytes"] / (st1["ms"] * 1e-3) / 1e9 if st1["ms"] else None
    gbs0 = st0["bytes"] / (st0["ms"] * 1e-3) / 1e9 if st0["ms"] else None
    roofline = {
        # the server's FP64 engine runs tile pairs with fixed-point block-dot and MAXPY products
        "kernel": "ke_step<double> (FP64 engine: fused CSR SpMV + block dot with the basis products as exact "
                  "fixed-point integers + per-request epilogue)",
        "bound": "hbm", "achieved": gbs0, "peak": hbm, "unit": "GB/s",
        "frac": gbs0 / hbm if gbs0 else None,
        "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth, of measured)",
        "fp64_method_tflops": tf0, "fp64_pipe_peak_tflops": pk["tflops"],
        "traffic": None, "launch_avg_ms": st0["ms"] / max(st0["launches"], 1), "launches": st0["launches"],
        "ir_engine_step": {"kernel": "ke_step<float>", "bound": "hbm", "achieved_gbs": gbs1, "peak_gbs": hbm,
                           "frac": gbs1 / hbm if gbs1 else None, "launches": st1["launches"]},
    }
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import Oracle

        orc = Oracle()
        t_tot, work_s, cnt = 0.0, 0.0, 0
        for i in range(0, k, 4):
            r = reqs[i]
            if r["n"] > 300_000:  # keep the sample to seconds; the scaling below accounts for size
                continue
            t0 = time.perf_counter()
            ro = orc.gmres(r["A"], r["b"], variant=1 if r["prec"] == "fp64" else 2, m=w["m"], tol=w["tol"],
                           max_iter=w["max_iter"])
            t_tot += time.perf_counter() - t0
            work_s += r["n"] * ro.iters
            cnt += 1
            if t_tot >= 15.0:
                break
        work_all = sum(r["n"] * i.iters for r, i in zip(reqs, all_infos))
        cpu_s = t_tot * work_all / work_s
        cpu = {"value": k / cpu_s, "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": f"complete oracle solves of {cnt} requests (every 4th with n <= 300k, until 15 s: "
                         f"{t_tot:.1f} s), scaled to all {k} requests by sum(n_i * iters_i)"}
        # all host cores: the same sample, one spawned process per core
        picked = [r for r in reqs[0:k:4] if r["n"] <= 300_000][:cnt]
        dt, cores = pool_oracle_solves([(r["A"], r["b"], 1 if r["prec"] == "fp64" else 2, w["m"], w["tol"],
                                         w["max_iter"]) for r in picked])
        cpu["all_cores"] = {"value": k / (dt * work_all / work_s), "unit": "solves/s", "cores": cores,
                            "kind": "oracle", "sample": f"the same {cnt} solves on {cores} spawned processes "
                                                        f"(1 thread each): {dt:.1f} s wall, scaled the same way"}
    ntot = sum(r["n"] for r in reqs)
    line = {
        "metric": METRIC_SERVE, "value": job_thr, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * world * k / job_thr, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 / f32 cycles (GMRES-IR)",
        "data": "synthetic (seeded 3D 7-point stencils, x_true ~ U[-1,1], Poisson arrivals)",
        "config": {"workload": (f"{k} requests, Poisson arrivals at {w['rate']:g}/s, 3D 7-point convection-diffusion, "
                                f"n log-uniform {w['n_range'][0]}..{w['n_range'][1]} (cube side on {w['sides']} "
                                f"log-spaced values), {int(100 * (1 - w['ir_frac']))}% FP64 / "
                                f"{int(100 * w['ir_frac'])}% GMRES-IR, GMRES({w['m']}) to {w['tol']:g} each"),
                   "requests": k, "total_unknowns": ntot, "hbm_budget_bytes": w["budget"],
                   "max_requests_per_engine": w["max_requests"], "parallelism": "1 GPU, 2 engines / streams",
                   "l2": "each engine's arena and bases exceed L2; no flush",
                   "timing": "host wall clock from the first arrival to the last completion (requests from host "
                             "buffers, solutions back to host buffers)"},
        "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
        "makespan_s": wall,
        "sustained_sweep": sweep,
        "sustained_capacity_solves_per_s": max((p["solves_per_s"] for p in sweep), default=None),
        "sustained_note": ("each sweep point is a finite Poisson trace of about sweep_s seconds of arrivals at the "
                           "given fraction of the burst's measured throughput, drawn from the same request "
                           "distribution; latency from each scheduled arrival to its solution in host memory"),
        "all_converged": all(i.status == 0 for i in all_infos), "max_rel_resid_true": max(true_rel),
        "server": {"peak_running": st["peak_running"], "cycles": st["cycles"], "engine_bytes": st["engine_bytes"],
                   "peak_bytes_in_use": st["peak_bytes_in_use"]},
        "sequential": seq,
        "speedup_vs_sequential": (thr / seq["solves_per_s"]) if seq else None,
        "e2e": {"value": job_thr, "unit": "solves/s", "h2d_bytes_per_step": int(sum(8 * r["n"] + 12 * len(r["A"][1])
                                                                            for r in reqs)),
                "d2h_bytes_per_step": int(8 * ntot)},
        "gpu_launches": int(sum(st["kernel_launches"])),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    return line


def run_serve_reference(args, w, rank):
    if rank != 0:
        return None
    reqs = serve_requests(w)
    from oracle import Oracle

    orc = Oracle()
    vals = []
    cnt = 0
    for s in range(args.warmup + args.steps):
        t_tot, n_s = 0.0, 0.0
        cnt = 0
        for i in range(0, len(reqs), 16):
            r = reqs[i]
            t0 = time.perf_counter()
            orc.gmres(r["A"], r["b"], variant=1 if r["prec"] == "fp64" else 2, m=w["m"], tol=w["tol"],
                      max_iter=w["max_iter"])
            t_tot += time.perf_counter() - t0
            n_s += r["n"]
            cnt += 1
            if t_tot >= 8.0:
                break
        total_s = t_tot * sum(r["n"] for r in reqs) / n_s
        if s >= args.warmup:
            vals.append(len(reqs) / total_s)
    v = float(np.mean(vals))
    return ({
        "impl": "reference", "metric": METRIC_SERVE, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * len(reqs) / v, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{len(reqs)} requests of the serving stream, solved one after another by the oracle"},
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": f"complete oracle solves of {cnt} requests (every 16th) per step, scaled by "
                                   f"total n / sample n"},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    })


# ----------------------------------------------------------------------------- the other configurations
SERVE_LEG = dict(SERVE_WORKLOADS["serve"], sweep_s=6.0)


def run_legs(args, rank, world, dist):
    """The other benchmark configurations, each measured in the same run after
    the headline and reported under its own key with its own timing, roofline,
    clocks and CPU baseline: 32^3 (latency-bound, one-reduce vs plain MGS),
    192^3 27-point GMRES-IR (FP32 and BF16 basis vs FP64 one-reduce, errors
    against the FP64 oracle's stored solve), 512 uneven 2D systems batched, and
    the serving loop (a 2000 req/s burst and a sweep of sustained arrival
    rates). Steps are capped per leg so the whole run stays within minutes."""
    import copy

    def sub(cap, warm=3):
        a = copy.copy(args)
        a.steps, a.warmup = max(1, min(args.steps, cap)), warm
        return a

    legs = {}
    for name, fn in (("c1_32cubed", lambda: run_ours(sub(20), WORKLOADS[32], rank, world, dist)),
                     ("c3_192cubed_gmres_ir", lambda: run_ours(sub(3), WORKLOADS[192], rank, world, dist)),
                     ("c4_batch512", lambda: run_batch(sub(3), BATCH_WORKLOADS["batch512"], rank, world, dist)),
                     ("c5_serve", lambda: run_serve(sub(1), SERVE_LEG, rank, world, dist))):
        t0 = time.perf_counter()
        line = fn()
        if line is not None:
            line.pop("history_first", None)
            line["leg_wall_s"] = time.perf_counter() - t0
        legs[name] = line
    return legs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=[str(k) for k in sorted(WORKLOADS, key=str)] + sorted(BATCH_WORKLOADS)
                    + sorted(SERVE_WORKLOADS), default="256")
    ap.add_argument("--no-mgs", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-shape", default=None, metavar="CTAS,ROWS",
                    help="batch workloads: pin the launch shape (grid CTAs, rows per thread) instead of the "
                         "autotuner's choice, e.g. to profile the shape a plain run chose")
    ap.add_argument("--no-legs", action="store_true",
                    help="default workload: skip the other configurations measured after the headline")
    args = ap.parse_args()
    batch = args.workload in BATCH_WORKLOADS
    serve = args.workload in SERVE_WORKLOADS
    w = (BATCH_WORKLOADS[args.workload] if batch else SERVE_WORKLOADS[args.workload] if serve
         else WORKLOADS[int(args.workload) if args.workload.isdigit() else args.workload])
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        if args.impl == "reference":
            dist = None  # the reference arm runs on rank 0 only
        else:
            import torch

            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            dist_mod.init_process_group("nccl")
            dist = dist_mod
    try:
        if serve:
            line = (run_serve_reference(args, w, rank) if args.impl == "reference"
                    else run_serve(args, w, rank, world, dist))
        elif batch:
            line = (run_batch_reference(args, w, rank) if args.impl == "reference"
                    else run_batch(args, w, rank, world, dist))
        elif args.impl == "reference":
            line = run_reference(args, w, rank, world)
        else:
            line = run_ours(args, w, rank, world, dist)
            if args.workload == "256" and world == 1 and not args.no_legs:
                line["legs"] = run_legs(args, rank, world, dist)
        if rank == 0 and line is not None:
            print(json.dumps(line))
        return 0
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
