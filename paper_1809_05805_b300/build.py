"""Build the CUDA library in-tree for sm_103a (B300).

``python -m paper_1809_05805_b300.build`` compiles the translation units of
``csrc/`` with nvcc, in parallel, and links them into one ``liblsgmres.so``
beside this file:

* ``lsgmres.cu``: the single-system solver (host side and its other kernels);
* ``step_<type>_s<stage>.cu``: the instantiations of its step kernel
  (``step.cuh``), one per arithmetic / storage type and CSR staging mode;
* ``batch.cu``: the batched engine and the serving loop;
* ``engine_step_f64.cu``, ``engine_step_f32.cu``: the engine's step kernel
  (``engine_step.cuh``);

all on the device code of ``common.cuh``. The result travels with the source
tree; nothing is installed into site-packages or a JIT cache.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRCS = [os.path.join(HERE, "csrc", f) for f in (
    "lsgmres.cu", *(f"step_{t}_s{s}.cu" for t in ("f64", "f32", "bf16") for s in (0, 1, 2)),
    "step_bf16_s3.cu", "step_bf16_s4.cu",
    *(f"step_{t}_s5.cu" for t in ("f64", "f32", "bf16")), "step_f64_s6.cu",
    "batch.cu", "engine_step_f64.cu", "engine_step_f32.cu", "probe.cu")]
OBJ_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblsgmres.so")
INCLUDE = os.path.join(ROOT, "include")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-lineinfo", "-O3", "-std=c++17",
    "-Xcompiler", "-fPIC",
]


def sources() -> list[str]:
    csrc = os.path.join(HERE, "csrc")
    return [os.path.join(csrc, f) for f in sorted(os.listdir(csrc)) if f.endswith((".cu", ".cuh", ".h"))] + [
        os.path.join(INCLUDE, f) for f in sorted(os.listdir(INCLUDE)) if f.endswith(".h")
    ]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in sources())


def _run(cmd: list[str]) -> subprocess.CompletedProcess:
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
    return p


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(OBJ_DIR, exist_ok=True)
    objs = [os.path.join(OBJ_DIR, os.path.basename(src)[:-3] + ".o") for src in SRCS]
    cmds = []
    for src, obj in zip(SRCS, objs):
        cmd = [nvcc, *NVCC_FLAGS, f"-I{INCLUDE}", "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        cmds.append(cmd)
    with ThreadPoolExecutor(max_workers=max(1, min(len(cmds), os.cpu_count() or 1))) as ex:
        results = list(ex.map(_run, cmds))
    if verbose:
        for p in results:
            sys.stderr.write(p.stderr)
    _run([nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", *objs, "-o", LIB + ".tmp"])
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
