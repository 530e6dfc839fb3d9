"""Planted mistakes in the oracle must be caught by the pins.

Each mutant is a copy of oracle/oracle.c with one plausible slip (a dropped term,
a wrong sign or index, a transposed operand, a missing scale). It is compiled into
a temporary directory and the pins of tests/pins.py run against it in a child
process; at least one pin must fail. Mutants only touch arithmetic, never loop
bounds that could index outside a buffer.
"""
import os
import subprocess
import sys
import tempfile

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    # one-reduce Arnoldi step (Algorithm 7 on Algorithm 4)
    "s_last_one_beta": ("ws->s[j] = d / (beta * beta);", "ws->s[j] = d / beta;"),
    "T_row_sign": ("TL(ws, j, k) = -t;", "TL(ws, j, k) = t;"),
    "T_transposed": ("t += TL(ws, i, k) * ws->s[k];", "t += TL(ws, k, i) * ws->s[k];"),
    "c_unscaled": ("ws->s[i] = ws->c[i] / beta;", "ws->s[i] = ws->c[i];"),
    "ell_unscaled": ("for (int i = 0; i < j; ++i) ws->a[i] /= beta;",
                     "for (int i = 0; i < j; ++i) ws->a[i] /= 1.0;"),
    "w_unscaled": ("un[l] = ws->w[l] / beta;", "un[l] = ws->w[l];"),
    "H_sub_sigma": ("HH(ws, j, j - 1) = beta;", "HH(ws, j, j - 1) = sigma;"),
    "maxpy_drop_last": ("for (int i = 0; i <= j; ++i) axpy(n, -ws->r[i], VCOL(ws, i), un);",
                        "for (int i = 0; i < j; ++i) axpy(n, -ws->r[i], VCOL(ws, i), un);"),
    "T_recurrence_drop": ("for (int i = k; i < j; ++i) t += ws->a[i] * TL(ws, i, k);",
                          "for (int i = k + 1; i < j; ++i) t += ws->a[i] * TL(ws, i, k);"),
    "step0_sign": ("axpy(n, -d0, VCOL(ws, 0), u1);", "axpy(n, d0, VCOL(ws, 0), u1);"),
    # Givens / least squares
    "givens_rot_sign": ("RR(ws, i + 1, j) = -ws->sn[i] * RR(ws, i, j) + ws->cs[i] * RR(ws, i + 1, j);",
                        "RR(ws, i + 1, j) = ws->sn[i] * RR(ws, i, j) + ws->cs[i] * RR(ws, i + 1, j);"),
    "g_sign": ("ws->g[j + 1] = -ws->sn[j] * ws->g[j];", "ws->g[j + 1] = ws->sn[j] * ws->g[j];"),
    "backsub_transposed": ("t -= RR(ws, i, l) * y[l];", "t -= RR(ws, l, i) * y[l];"),
    "update_sign": ("for (int i = 0; i < k; ++i) axpy(ws->n, y[i], VCOL(ws, i), x);",
                    "for (int i = 0; i < k; ++i) axpy(ws->n, -y[i], VCOL(ws, i), x);"),
    # MGS-GMRES (Algorithm 6)
    "mgs_axpy_sign": ("axpy(n, -h, VCOL(ws, k), w);", "axpy(n, h, VCOL(ws, k), w);"),
    "mgs_H_index": ("HH(ws, k, i) = h;", "HH(ws, i, k) = h;"),
    # kernels and QR variants
    "spmv_gather": ("s += val[p] * x[col[p]];", "s += val[p] * x[i];"),
    "lvl2_z_unscaled": ("sv[j - 1] = z / beta;", "sv[j - 1] = z;"),
    "lvl2_T_sign": ("TT(j - 1, k) = -t;", "TT(j - 1, k) = t;"),
    "cgs_R_overwrite": ("R[i + (size_t)j * p] += s[i];", "R[i + (size_t)j * p] = s[i];"),
    "maxpy_alpha": ("double t = alpha * y_in[i];", "double t = y_in[i];"),
    # GMRES-IR (FP32 cycle)
    "ir_v0_unnormalized": ("V32COL(0)[l] = (float)(VCOL(ws, 0)[l] / beta0);", "V32COL(0)[l] = (float)VCOL(ws, 0)[l];"),
    "ir_maxpy_sign": ("for (int64_t l = 0; l < n; ++l) un[l] -= ri * vi[l];",
                      "for (int64_t l = 0; l < n; ++l) un[l] += ri * vi[l];"),
    "ir_w_unscaled": ("for (int64_t l = 0; l < n; ++l) un[l] = w32[l] / fb;",
                      "for (int64_t l = 0; l < n; ++l) un[l] = w32[l];"),
    "ir_cycle_fp64_spmv": ("if (!tail) spmv_f32(n, ws->rowptr, ws->col, val32, u, w32);",
                           "if (!tail) spmv_f32(n, ws->rowptr, ws->col, val32, u, w32), w32[0] *= 1.5f;"),
    # Algorithm 5 (second projection) and the L = 2 pipeline (Algorithm 8). Dropping
    # the second-pass coefficients from H / R is not planted: they are of the size
    # of the rounding in H itself (eps ||A v_j||), invisible to any pin.
    "cgs2_reorth_sign": ("axpy(n, -ws->a[i], VCOL(ws, i), un);", "axpy(n, ws->a[i], VCOL(ws, i), un);"),
    "qr_cgs2_second_pass_sign": ("for (int i = 0; i < j; ++i) axpy(n, -s2[i], QCOL(i), uj);",
                                 "for (int i = 0; i < j; ++i) axpy(n, s2[i], QCOL(i), uj);"),
    "pipe_pairs_shifted": ("c == 0 || c % 2 == 0 || tail || brk;", "c == 0 || c % 2 == 1 || tail || brk;"),
    "pipe_skip_pending": ("for (int q = rotated; q <= c; ++q) {", "for (int q = c; q <= c; ++q) {"),
    # GMRES-IR with BF16 basis storage
    "bf16_no_tie_even": ("const uint32_t lsb = (u >> 16) & 1u;", "const uint32_t lsb = 0u;"),
    "bf16_truncate": ("u = (u + 0x7fffu + lsb) & 0xffff0000u;", "u = u & 0xffff0000u;"),
    "bf16_normalized_unrounded": ("    for (int64_t l = 0; l < n; ++l) u[l] *= ib; /* v_j */\n    round_bf16_vec(n, u, bf16);",
                                  "    for (int64_t l = 0; l < n; ++l) u[l] *= ib; /* v_j */"),
    "dot_square": ("double orc_dot(int64_t n, const double* x, const double* y) { return dot(n, x, y); }",
                   "double orc_dot(int64_t n, const double* x, const double* y) { return dot(n, x, x); }"),
}

RUNNER = r"""
import sys, traceback
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle, pins
o = oracle.Oracle({lib!r})
failed = []
for pin in pins.PINS + [pins.pin_orthogonality_slopes]:
    try:
        pin(o)
    except AssertionError as e:
        failed.append(pin.__name__)
    except Exception as e:
        failed.append(pin.__name__ + ":" + type(e).__name__)
print("FAILED_PINS", ",".join(failed))
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    # a site that also appears in the FP32 (GMRES-IR) copy of the cycle is mutated
    # at its first occurrence, which is the FP64 cycle (defined earlier in the file)
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    with tempfile.TemporaryDirectory() as d:
        msrc = os.path.join(d, "oracle_mut.c")
        with open(msrc, "w") as f:
            f.write(src.replace(old, new, 1))
        lib = oracle.build(msrc, os.path.join(d, "liboracle_mut.so"), extra=["-DORC_MUTANT"])
        code = RUNNER.format(root=ROOT, tests=os.path.dirname(__file__), lib=lib)
        p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    line = [ln for ln in p.stdout.splitlines() if ln.startswith("FAILED_PINS")]
    assert p.returncode == 0 and line, f"runner failed for {name}: {p.stderr[-2000:]}"
    caught = line[0].split(" ", 1)[1].strip()
    assert caught, f"mutant {name} passed every pin"
