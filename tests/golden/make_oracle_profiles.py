"""Write tests/golden/oracle_profile_<name>.txt by running the oracle (only).

For each benchmark workload the file records the oracle's iteration count,
restart count, reduction count, final true residual and its per-step residual
history. The GPU solve of the same seeded inputs is compared against these
files, and bench.py's reference arm scales its bounded oracle sample by the
recorded step profile. Nothing here touches the CUDA library.

Usage:  python tests/golden/make_oracle_profiles.py [c1] [c2_one_reduce] [c2_mgs] [c3_ir] [c3_fp64]
(c2 and c3 run the full 256^3 / 192^3 solves single-threaded: tens of minutes.)
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1809_05805_b300 import problems as P  # noqa: E402

WORKLOADS = {
    "c1": dict(N=32, m=30, tol=1e-8, max_iter=300, variant=oracle.ONE_REDUCE),
    "c1_mgs": dict(N=32, m=30, tol=1e-8, max_iter=300, variant=oracle.MGS),
    "c2_one_reduce": dict(N=256, m=50, tol=1e-8, max_iter=3000, variant=oracle.ONE_REDUCE),
    "c2_mgs": dict(N=256, m=50, tol=1e-8, max_iter=3000, variant=oracle.MGS),
    # GMRES-IR (FP32 cycles inside FP64 restarts) on the 192^3 27-point problem
    "c3_ir": dict(N=192, m=40, tol=1e-10, max_iter=5000, variant=2, stencil="27pt"),
    # the same 192^3 27-point system solved by FP64 one-reduce MGS-GMRES (Algorithm 7):
    # the fixed point against which the GMRES-IR solutions' error is stated
    "c3_fp64": dict(N=192, m=40, tol=1e-10, max_iter=5000, variant=oracle.ONE_REDUCE, stencil="27pt"),
}
VARIANT_NAMES = {0: "mgs", 1: "one_reduce", 2: "ir_fp32"}


def run(name):
    w = WORKLOADS[name]
    A = P.aniso_27pt(w["N"]) if w.get("stencil") == "27pt" else P.conv_diff_7pt(w["N"])
    _, b = P.rhs(A, seed=0)
    t0 = time.time()
    r = oracle.get().gmres(A, b, variant=w["variant"], m=w["m"], tol=w["tol"], max_iter=w["max_iter"])
    dt = time.time() - t0
    path = os.path.join(HERE, f"oracle_profile_{name}.txt")
    with open(path, "w") as f:
        f.write(f"# written by tests/golden/make_oracle_profiles.py from the oracle only\n")
        stencil = "27-point anisotropic diffusion" if w.get("stencil") == "27pt" else "7-point convection-diffusion"
        f.write(f"# workload: {stencil} N={w['N']} (n={w['N'] ** 3}), x_true ~ U[-1,1] "
                f"PCG64(0), b = A x_true, x0 = 0, GMRES(m={w['m']}), tol={w['tol']}, "
                f"variant={VARIANT_NAMES[w['variant']]}\n")
        f.write(f"# oracle wall time {dt:.1f} s (1 thread)\n")
        f.write(f"status {r.status}\niters {r.iters}\nrestarts {r.restarts}\nreductions {r.reductions}\n")
        f.write(f"rel_resid_true {r.rel_resid_true!r}\n")
        f.write("history " + " ".join(repr(float(h)) for h in r.history) + "\n")
        idx = np.sort(np.random.default_rng(123).choice(len(b), size=64, replace=False))
        f.write("x_sample_idx " + " ".join(str(int(i)) for i in idx) + "\n")
        f.write("x_sample " + " ".join(repr(float(r.x[i])) for i in idx) + "\n")
    print(name, r.status, r.iters, r.restarts, r.rel_resid_true, f"{dt:.1f}s", flush=True)


def load(name):
    vals = {}
    with open(os.path.join(HERE, f"oracle_profile_{name}.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split(" ", 1)
            vals[k] = np.array([float(t) for t in v.split()]) if k in ("history", "x_sample_idx", "x_sample") \
                else float(v)
    return vals


if __name__ == "__main__":
    for name in sys.argv[1:] or ["c1", "c1_mgs"]:
        run(name)
