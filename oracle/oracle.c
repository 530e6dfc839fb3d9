/*
 * FP64 CPU oracle for "Low synchronization GMRES algorithms"
 * (Swirydowicz, Langou, Ananthan, Yang, Thomas, arXiv:1809.05805).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously-correct statement
 * of what the GPU path computes. It may be loaded only by tests/, by the
 * smoke check in __graft_entry__.py and by the CPU-baseline / reference arm of
 * bench.py. The product path never links, imports or calls it, and it shares
 * no code, header, table or constant with the CUDA library.
 *
 * Style rules that keep it checkable by eye against the paper:
 *   - every vector operation is a plain sequential loop in FP64;
 *   - no blocking, fusion or reordering beyond what the algorithm states;
 *   - compiled with -O2 -ffp-contract=off (no fused multiply-add), single thread.
 *
 * Contents, each citing the passage it follows:
 *   orc_spmv          y = A x for CSR A (Section IV, CSR matvec)
 *   orc_dot, orc_maxpy  the mass inner product and MAXPY of Section IV, one
 *                     column at a time
 *   orc_qr_mgs        column MGS QR (Algorithm 2, one column at a time)
 *   orc_qr_cgs        classical GS QR, 1 or 2 passes (Algorithm 1)
 *   orc_qr_mgs_lvl2   Level-2 compact-WY MGS with lagged normalization
 *                     (Algorithm 4, with the T recurrence of Section II)
 *   orc_qr_cgs2_lvl2  Level-2 iterated CGS with lagged normalization
 *                     (Algorithm 5): Algorithm 4's step, then a second
 *                     classical projection with a second reduction [A16]
 *   orc_gmres         restarted GMRES(m) with
 *                       variant 0: MGS-GMRES (Algorithm 6)
 *                       variant 1: one-synchronization MGS-GMRES with lagged
 *                                  normalization (Algorithm 7 built on Algorithm 4)
 *                       variant 2: variant 1 with each cycle's vectors in FP32
 *                                  inside FP64 restarts (GMRES-IR) [A13]
 *                       variant 3: variant 1 with the second (re-orthogonalizing)
 *                                  projection of Algorithm 5: two reductions
 *                                  per step [A16]
 *                       variant 4: variant 1 with the Givens rotations applied
 *                                  two columns at a time, the L = 2 pipeline
 *                                  of Algorithm 8 [A17]
 *                       variant 5: variant 2 with the basis stored in BF16
 *                                  (FP32 arithmetic and accumulation) [A18]
 *
 * Parity unpinned at rounding level: the second-pass coefficients that
 * orc_qr_cgs2_lvl2 and variant 3 add to R and H are of the size of the rounding
 * in those entries (eps ||a_j||), so no pin can tell whether they are added.
 *
 * What pins each function (tests/test_oracle_*.py, all CPU-only):
 *   the Arnoldi relation A V_k = V_{k+1} Hbar_k (Section III); the MGS /
 *   one-reduce equivalence on well-conditioned problems (Section V-A); T equal
 *   to inv(I + L) from the computed basis (Section II); Q R = A and the
 *   O(eps)kappa vs O(eps)kappa^2 loss-of-orthogonality slopes (Section I);
 *   GMRES(n) on n x n systems equal to an LU solve; the residual after k steps
 *   equal to a brute-force least-squares minimum over the Krylov space; exact
 *   termination after d steps for a matrix with d distinct eigenvalues; the
 *   limiting-accuracy stall of the Simoncini-Szyld diagonal problem
 *   (Section V-A); and source-level mutants of this file that each pin catches.
 *
 * Readings of passages that are ambiguous or garbled in the paper (and of the
 * extensions beyond it) are listed where they are used, tagged [A1]..[A18].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_MAXITER 1
#define ORC_BREAKDOWN 2
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NONFINITE (-3)
#define ORC_ERR_OOM (-4)

#define ORC_VARIANT_MGS 0
#define ORC_VARIANT_ONE_REDUCE 1
#define ORC_VARIANT_IR_FP32 2
#define ORC_VARIANT_CGS2 3
#define ORC_VARIANT_PIPE2 4
#define ORC_VARIANT_IR_BF16 5

/* Timing build only: compiled with -DORC_OMP -fopenmp, the plain vector loops
 * below are shared out over the host's cores (each sum by an OpenMP
 * reduction, so its order changes), to time the oracle on all cores for the
 * CPU baseline. The checker is built without ORC_OMP: these macros are then
 * empty and every loop stays sequential. */
#ifdef ORC_OMP
#include <omp.h>
#define ORC_PAR_FOR _Pragma("omp parallel for schedule(static)")
#define ORC_PAR_SUM_S _Pragma("omp parallel for schedule(static) reduction(+ : s)")
#else
#define ORC_PAR_FOR
#define ORC_PAR_SUM_S
#endif

/* Host threads the vector loops use (1 unless built with ORC_OMP). */
int orc_threads(void) {
#ifdef ORC_OMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Breakdown threshold factor [A6]: the new direction is declared exhausted
 * when its norm is below BREAKDOWN_FACTOR * eps * ||Hbar(:, j)||. */
#define BREAKDOWN_FACTOR 16.0

/* ------------------------------------------------------------------------- */
/* Level-1 building blocks: plain loops.                                      */
/* ------------------------------------------------------------------------- */

/* y = A x, A in compressed-sparse-row form (rowptr[n+1], col[nnz], val[nnz]). */
void orc_spmv(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
              const double* x, double* y) {
  ORC_PAR_FOR
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s += val[p] * x[col[p]];
    y[i] = s;
  }
}

static double dot(int64_t n, const double* x, const double* y) {
  double s = 0.0;
  ORC_PAR_SUM_S
  for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
  return s;
}

static double nrm2(int64_t n, const double* x) { return sqrt(dot(n, x, x)); }

/* Inner product x^T y, sequential (the plain definition behind the mass inner
 * product of Section IV: one such sum per column). */
double orc_dot(int64_t n, const double* x, const double* y) { return dot(n, x, y); }

/* MAXPY of Section IV: y_out = alpha y_in + sum_{k<K} c[k] V(:, k), V column-major
 * with leading dimension ldv, written term by term in column order. */
void orc_maxpy(int64_t n, int K, const double* V, int64_t ldv, const double* c, double alpha,
               const double* y_in, double* y_out) {
  ORC_PAR_FOR
  for (int64_t i = 0; i < n; ++i) {
    double t = alpha * y_in[i];
    for (int k = 0; k < K; ++k) t += c[k] * V[i + (size_t)k * ldv];
    y_out[i] = t;
  }
}

/* y = y + alpha x */
static void axpy(int64_t n, double alpha, const double* x, double* y) {
  ORC_PAR_FOR
  for (int64_t i = 0; i < n; ++i) y[i] += alpha * x[i];
}

/* x = alpha x */
static void scal(int64_t n, double alpha, double* x) {
  ORC_PAR_FOR
  for (int64_t i = 0; i < n; ++i) x[i] *= alpha;
}

/* Plane rotation G = [c s; -s c] with G [a; b] = [rho; 0], rho = hypot(a, b). [A7] */
static void givens(double a, double b, double* c, double* s) {
  if (b == 0.0) {
    *c = 1.0;
    *s = 0.0;
  } else {
    double rho = hypot(a, b);
    *c = a / rho;
    *s = b / rho;
  }
}

/* ------------------------------------------------------------------------- */
/* QR factorizations of a tall n x p matrix (column-major), Section II.       */
/* ------------------------------------------------------------------------- */

/* Column MGS, Algorithm 2: each new column a is reduced by p rank-1 updates
 * s_i = q_i^T a, a = a - q_i s_i, then normalized. Q (n x p), R (p x p, upper). */
int orc_qr_mgs(int64_t n, int p, const double* A, double* Q, double* R) {
  if (n <= 0 || p <= 0 || p > n) return ORC_ERR_ARG;
  memset(R, 0, sizeof(double) * (size_t)p * p);
  for (int j = 0; j < p; ++j) {
    double* a = Q + (size_t)j * n;
    memcpy(a, A + (size_t)j * n, sizeof(double) * n);
    for (int i = 0; i < j; ++i) {
      const double* qi = Q + (size_t)i * n;
      double s = dot(n, qi, a);
      axpy(n, -s, qi, a);
      R[i + (size_t)j * p] = s;
    }
    double r = nrm2(n, a);
    R[j + (size_t)j * p] = r;
    scal(n, 1.0 / r, a);
  }
  return ORC_OK;
}

/* Classical Gram-Schmidt, Algorithm 1 with `passes` projection sweeps
 * (passes = 1: CGS-1; passes = 2: CGS with one re-orthogonalization).
 * Each sweep projects against all previous columns at once: s = Q^T a,
 * r += s, a = a - Q s. */
int orc_qr_cgs(int64_t n, int p, const double* A, double* Q, double* R, int passes) {
  if (n <= 0 || p <= 0 || p > n || passes < 1) return ORC_ERR_ARG;
  memset(R, 0, sizeof(double) * (size_t)p * p);
  double* s = (double*)malloc(sizeof(double) * (size_t)p);
  if (!s) return ORC_ERR_OOM;
  for (int j = 0; j < p; ++j) {
    double* a = Q + (size_t)j * n;
    memcpy(a, A + (size_t)j * n, sizeof(double) * n);
    for (int k = 0; k < passes; ++k) {
      for (int i = 0; i < j; ++i) s[i] = dot(n, Q + (size_t)i * n, a);
      for (int i = 0; i < j; ++i) {
        axpy(n, -s[i], Q + (size_t)i * n, a);
        R[i + (size_t)j * p] += s[i];
      }
    }
    double r = nrm2(n, a);
    R[j + (size_t)j * p] = r;
    scal(n, 1.0 / r, a);
  }
  free(s);
  return ORC_OK;
}

/* Level-2 compact-WY MGS with lagged normalization, Algorithm 4, run over the
 * columns of A. T (p x p) is returned lower triangular: T = (I + L)^{-1}, where
 * L is the strictly lower part of Q^T Q built one row per column [A2]; the
 * paper's upper-triangular T of the Malard-Paige recurrence is its transpose.
 *
 * When column j (0-based, j >= 1) arrives, column j-1 is orthogonalized but not
 * yet normalized (u_{j-1}). One block reduction gives
 *   x = Q_{j-2}^T u_{j-1},  sigma = u_{j-1}^T u_{j-1},
 *   y = Q_{j-2}^T a_j,      z = u_{j-1}^T a_j,
 * then: beta = sqrt(sigma) = R(j-1,j-1), q_{j-1} = u_{j-1}/beta (the lag);
 * ell = x / beta is the new row of L; the new row of T is -ell^T T;
 * the projections of a_j onto Q_{j-1} are s = [y; z / beta] [A1];
 * r = T s is column j of R; u_j = a_j - Q_{j-1} r.
 * After the last column one more reduction normalizes it. */
int orc_qr_mgs_lvl2(int64_t n, int p, const double* A, double* Q, double* R, double* T) {
  if (n <= 0 || p <= 0 || p > n) return ORC_ERR_ARG;
  memset(R, 0, sizeof(double) * (size_t)p * p);
  memset(T, 0, sizeof(double) * (size_t)p * p);
  double* x = (double*)malloc(sizeof(double) * (size_t)p);
  double* y = (double*)malloc(sizeof(double) * (size_t)p);
  double* sv = (double*)malloc(sizeof(double) * (size_t)p);
  double* r = (double*)malloc(sizeof(double) * (size_t)p);
  if (!x || !y || !sv || !r) {
    free(x); free(y); free(sv); free(r);
    return ORC_ERR_OOM;
  }
#define QCOL(i) (Q + (size_t)(i) * n)
#define TT(i, k) T[(i) + (size_t)(k) * p]
  memcpy(QCOL(0), A, sizeof(double) * n); /* u_0 = a_0 */
  TT(0, 0) = 1.0;
  for (int j = 1; j <= p; ++j) {
    /* at j == p only the lagged norm (and the last row of T) remain */
    const int last = (j == p);
    double* u = QCOL(j - 1);
    const double* a = last ? NULL : A + (size_t)j * n;
    /* the single block reduction */
    for (int i = 0; i < j - 1; ++i) x[i] = dot(n, QCOL(i), u);
    double sigma = dot(n, u, u);
    if (!last) {
      for (int i = 0; i < j - 1; ++i) y[i] = dot(n, QCOL(i), a);
    }
    double z = last ? 0.0 : dot(n, u, a);
    /* lagged normalization of column j-1 */
    double beta = sqrt(sigma);
    R[(j - 1) + (size_t)(j - 1) * p] = beta;
    scal(n, 1.0 / beta, u);
    /* new row of T = (I + L)^{-1}: T(j-1, k) = -sum_{i=k}^{j-2} ell_i T(i, k) */
    for (int i = 0; i < j - 1; ++i) x[i] /= beta; /* ell */
    for (int k = 0; k < j - 1; ++k) {
      double t = 0.0;
      for (int i = k; i < j - 1; ++i) t += x[i] * TT(i, k);
      TT(j - 1, k) = -t;
    }
    TT(j - 1, j - 1) = 1.0;
    if (last) break;
    /* projections of a_j onto q_0..q_{j-1}, then r = T s */
    for (int i = 0; i < j - 1; ++i) sv[i] = y[i];
    sv[j - 1] = z / beta;
    for (int i = 0; i < j; ++i) {
      double t = 0.0;
      for (int k = 0; k <= i; ++k) t += TT(i, k) * sv[k];
      r[i] = t;
      R[i + (size_t)j * p] = t;
    }
    /* u_j = a_j - Q_{j-1} r */
    double* uj = QCOL(j);
    memcpy(uj, a, sizeof(double) * n);
    for (int i = 0; i < j; ++i) axpy(n, -r[i], QCOL(i), uj);
  }
#undef QCOL
#undef TT
  free(x); free(y); free(sv); free(r);
  return ORC_OK;
}

/* Level-2 iterated classical Gram-Schmidt with lagged normalization,
 * Algorithm 5, over the columns of A [A16]. When column j arrives, the first
 * synchronization is exactly Algorithm 4's: one block reduction gives
 * Q_{j-2}^T u_{j-1}, ||u_{j-1}||^2, Q_{j-2}^T a_j and u_{j-1}^T a_j; column j-1
 * is normalized (the lag), the row of T is formed and the first projection
 * r = T s gives u_j = a_j - Q_{j-1} r. The second synchronization is the
 * re-orthogonalization of classical Gram-Schmidt applied twice:
 * s2 = Q_{j-1}^T u_j, u_j = u_j - Q_{j-1} s2, and column j of R is r + s2.
 * After the last column one more reduction normalizes it. T is returned as in
 * orc_qr_mgs_lvl2. */
int orc_qr_cgs2_lvl2(int64_t n, int p, const double* A, double* Q, double* R, double* T) {
  if (n <= 0 || p <= 0 || p > n) return ORC_ERR_ARG;
  memset(R, 0, sizeof(double) * (size_t)p * p);
  memset(T, 0, sizeof(double) * (size_t)p * p);
  double* x = (double*)malloc(sizeof(double) * (size_t)p);
  double* y = (double*)malloc(sizeof(double) * (size_t)p);
  double* sv = (double*)malloc(sizeof(double) * (size_t)p);
  double* r = (double*)malloc(sizeof(double) * (size_t)p);
  double* s2 = (double*)malloc(sizeof(double) * (size_t)p);
  if (!x || !y || !sv || !r || !s2) {
    free(x); free(y); free(sv); free(r); free(s2);
    return ORC_ERR_OOM;
  }
#define QCOL(i) (Q + (size_t)(i) * n)
#define TT(i, k) T[(i) + (size_t)(k) * p]
  memcpy(QCOL(0), A, sizeof(double) * n);
  TT(0, 0) = 1.0;
  for (int j = 1; j <= p; ++j) {
    const int last = (j == p);
    double* u = QCOL(j - 1);
    const double* a = last ? NULL : A + (size_t)j * n;
    /* first synchronization: Algorithm 4's block reduction */
    for (int i = 0; i < j - 1; ++i) x[i] = dot(n, QCOL(i), u);
    double sigma = dot(n, u, u);
    if (!last) {
      for (int i = 0; i < j - 1; ++i) y[i] = dot(n, QCOL(i), a);
    }
    double z = last ? 0.0 : dot(n, u, a);
    double beta = sqrt(sigma);
    R[(j - 1) + (size_t)(j - 1) * p] = beta;
    scal(n, 1.0 / beta, u);
    for (int i = 0; i < j - 1; ++i) x[i] /= beta;
    for (int k = 0; k < j - 1; ++k) {
      double t = 0.0;
      for (int i = k; i < j - 1; ++i) t += x[i] * TT(i, k);
      TT(j - 1, k) = -t;
    }
    TT(j - 1, j - 1) = 1.0;
    if (last) break;
    for (int i = 0; i < j - 1; ++i) sv[i] = y[i];
    sv[j - 1] = z / beta;
    for (int i = 0; i < j; ++i) {
      double t = 0.0;
      for (int k = 0; k <= i; ++k) t += TT(i, k) * sv[k];
      r[i] = t;
    }
    double* uj = QCOL(j);
    memcpy(uj, a, sizeof(double) * n);
    for (int i = 0; i < j; ++i) axpy(n, -r[i], QCOL(i), uj);
    /* second synchronization: re-orthogonalize against q_0 .. q_{j-1} */
    for (int i = 0; i < j; ++i) s2[i] = dot(n, QCOL(i), uj);
    for (int i = 0; i < j; ++i) axpy(n, -s2[i], QCOL(i), uj);
    for (int i = 0; i < j; ++i) R[i + (size_t)j * p] = r[i] + s2[i];
  }
#undef QCOL
#undef TT
  free(x); free(y); free(sv); free(r); free(s2);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Restarted GMRES(m), Section III.                                          */
/* ------------------------------------------------------------------------- */

typedef struct {
  int iters;              /* Arnoldi columns completed, all cycles */
  int restarts;           /* cycles run */
  int status;             /* ORC_OK / ORC_MAXITER / ORC_ERR_* */
  int breakdowns;         /* cycles ended by a vanishing new direction */
  double rel_resid_true;  /* ||b - A x|| / ||b|| at exit */
  double rel_resid_est;   /* last Givens estimate |g_{k+1}| / ||b|| */
  int64_t reductions;     /* global reductions: one per inner product, norm or block */
} orc_info;

/* Workspace of one cycle. H is kept unrotated (for the Arnoldi relation);
 * Rg is the Givens-rotated copy used for the least-squares problem. */
typedef struct {
  int64_t n;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
  int m;
  double* V;   /* n x (m+1): normalized basis v_0..v_m (u_j before normalization) */
  double* w;   /* n */
  double* H;   /* (m+1) x m, column-major, unrotated Hessenberg */
  double* Rg;  /* (m+1) x m, rotated */
  double* cs;  /* m */
  double* sn;  /* m */
  double* g;   /* m+1 */
  double* T;   /* (m+1) x (m+1) lower: (I + L)^{-1}, one-reduce only */
  double* a;   /* m+1: block-dot column 1 (V^T u) */
  double* c;   /* m+1: block-dot column 2 (V^T w) */
  double* s;   /* m+1 */
  double* r;   /* m+1 */
} cycle_ws;

#define VCOL(ws, k) ((ws)->V + (size_t)(k) * (ws)->n)
#define HH(ws, i, j) ((ws)->H[(i) + (size_t)(j) * ((ws)->m + 1)])
#define RR(ws, i, j) ((ws)->Rg[(i) + (size_t)(j) * ((ws)->m + 1)])
#define TL(ws, i, j) ((ws)->T[(i) + (size_t)(j) * ((ws)->m + 1)])

/* Column j of H is complete: rotate a copy of it by the stored rotations,
 * form rotation j, and update g. Returns |g_{j+1}|, the residual norm of the
 * least-squares problem with j+1 columns (Algorithm 6, "apply Givens rotations"). */
static double rotate_column(cycle_ws* ws, int j) {
  for (int i = 0; i <= j + 1; ++i) RR(ws, i, j) = HH(ws, i, j);
  for (int i = 0; i < j; ++i) {
    double t = ws->cs[i] * RR(ws, i, j) + ws->sn[i] * RR(ws, i + 1, j);
    RR(ws, i + 1, j) = -ws->sn[i] * RR(ws, i, j) + ws->cs[i] * RR(ws, i + 1, j);
    RR(ws, i, j) = t;
  }
  givens(RR(ws, j, j), RR(ws, j + 1, j), &ws->cs[j], &ws->sn[j]);
  RR(ws, j, j) = ws->cs[j] * RR(ws, j, j) + ws->sn[j] * RR(ws, j + 1, j);
  RR(ws, j + 1, j) = 0.0;
  ws->g[j + 1] = -ws->sn[j] * ws->g[j];
  ws->g[j] = ws->cs[j] * ws->g[j];
  return fabs(ws->g[j + 1]);
}

/* ||Hbar(0:j+1, j)||_2 for the breakdown test [A6]. */
static double hcol_norm(cycle_ws* ws, int j) {
  double s = 0.0;
  for (int i = 0; i <= j + 1; ++i) s += HH(ws, i, j) * HH(ws, i, j);
  return sqrt(s);
}

/* x = x + V_k y with R(0:k,0:k) y = g(0:k) solved by back substitution. */
static void update_solution(cycle_ws* ws, int k, double* x) {
  double* y = ws->s; /* reuse */
  for (int i = k - 1; i >= 0; --i) {
    double t = ws->g[i];
    for (int l = i + 1; l < k; ++l) t -= RR(ws, i, l) * y[l];
    y[i] = t / RR(ws, i, i);
  }
  for (int i = 0; i < k; ++i) axpy(ws->n, y[i], VCOL(ws, i), x);
}

typedef struct {
  int k;          /* columns used */
  int breakdown;  /* 1 if the cycle stopped on a vanishing direction */
  double est;     /* last |g_{k}| */
} cycle_out;

/* One cycle of MGS-GMRES, Algorithm 6. On entry V column 0 holds r0 and
 * beta0 = ||r0||. The i-th step makes i+1 inner products and one norm, each a
 * separate global reduction. MGS uses the updated w in every inner product
 * (the modified, not the classical, order) [A8]. */
static cycle_out cycle_mgs(cycle_ws* ws, int kmax, double beta0, double bnorm, double tol,
                           double* hist, int* hlen, int hcap, int64_t* nred) {
  cycle_out out = {0, 0, 0.0};
  const int64_t n = ws->n;
  scal(n, 1.0 / beta0, VCOL(ws, 0));
  memset(ws->g, 0, sizeof(double) * (size_t)(ws->m + 1));
  ws->g[0] = beta0;
  for (int i = 0; i < kmax; ++i) {
    double* w = VCOL(ws, i + 1);
    orc_spmv(n, ws->rowptr, ws->col, ws->val, VCOL(ws, i), w); /* z = A v_i */
    for (int k = 0; k <= i; ++k) {
      double h = dot(n, w, VCOL(ws, k));
      *nred += 1;
      HH(ws, k, i) = h;
      axpy(n, -h, VCOL(ws, k), w);
    }
    double hn = nrm2(n, w);
    *nred += 1;
    HH(ws, i + 1, i) = hn;
    double est = rotate_column(ws, i) / bnorm;
    if (*hlen < hcap) hist[*hlen] = est;
    *hlen += 1;
    out.k = i + 1;
    out.est = est;
    if (hn <= BREAKDOWN_FACTOR * 2.220446049250313e-16 * hcol_norm(ws, i)) {
      out.breakdown = 1;
      if (hn != 0.0) scal(n, 1.0 / hn, w);
      break;
    }
    scal(n, 1.0 / hn, w); /* v_{i+1} */
    if (est <= tol) break;
  }
  return out;
}

/* One cycle of one-synchronization MGS-GMRES with lagged normalization,
 * Algorithm 7, whose orthogonalization is Algorithm 4 applied to the Arnoldi
 * vectors. The reading used here [A1, A3, A8, A9]:
 *
 * step 0 (v_0 = r0 / beta0 is normalized): w = A v_0; one reduction
 *   d = v_0^T w; T = [1]; H(0,0) = d; u_1 = w - d v_0.
 * step j >= 1 (u_j orthogonalized, not yet normalized):
 *   w = A u_j (the unnormalized vector);
 *   one reduction: a = V_{j-1}^T u_j, sigma = u_j^T u_j,
 *                  c = V_{j-1}^T w,   d = u_j^T w;
 *   beta = sqrt(sigma); H(j, j-1) = beta completes column j-1 (the lag),
 *   which is rotated, giving the residual estimate of step j-1;
 *   v_j = u_j / beta; ell = a / beta is row j of L; row j of T is -ell^T T;
 *   s = [c / beta; d / beta^2] are the projections of A v_j = w / beta onto
 *   V_j (the entry against u_j carries beta twice [A1]);
 *   r = T s is column j of H; u_{j+1} = w / beta - V_j r.
 * after the last step one extra reduction gives beta = ||u_kmax||, which
 *   completes column kmax-1 (the cycle's tail).
 * Only the tail pays a reduction that is not shared with a block product, so
 * a cycle of k steps makes k+1 reductions.
 *
 * reorth (variant 3, Algorithm 5 in Arnoldi form [A16]): after u_{j+1} is
 * formed, a second reduction s2 = V_{j+1}^T u_{j+1} and the projection
 * u_{j+1} -= V_{j+1} s2 re-orthogonalize it, and H(0:j, j) = r + s2; a cycle
 * of k steps makes 2k+1 reductions.
 * pairs (variant 4, the L = 2 pipeline of Algorithm 8 [A17]): column 0 is
 * rotated when it completes; afterwards columns are rotated two at a time,
 * the odd column c-1 together with the even column c once c completes, and
 * the convergence test runs only after a rotation. The cycle's tail and a
 * breakdown rotate whatever is pending. V, H and every rotation are those of
 * variant 1; only the step at which convergence is seen can come one later. */
static cycle_out cycle_one_reduce(cycle_ws* ws, int kmax, double beta0, double bnorm, double tol,
                                  double* hist, int* hlen, int hcap, int64_t* nred, int reorth, int pairs) {
  cycle_out out = {0, 0, 0.0};
  const int64_t n = ws->n;
  const int ld = ws->m + 1;
  scal(n, 1.0 / beta0, VCOL(ws, 0));
  memset(ws->g, 0, sizeof(double) * (size_t)ld);
  ws->g[0] = beta0;
  memset(ws->T, 0, sizeof(double) * (size_t)ld * ld);

  /* step 0 */
  orc_spmv(n, ws->rowptr, ws->col, ws->val, VCOL(ws, 0), ws->w);
  double d0 = dot(n, VCOL(ws, 0), ws->w);
  *nred += 1;
  TL(ws, 0, 0) = 1.0;
  HH(ws, 0, 0) = d0;
  {
    double* u1 = VCOL(ws, 1);
    memcpy(u1, ws->w, sizeof(double) * n);
    axpy(n, -d0, VCOL(ws, 0), u1);
    if (reorth) {
      double s2 = dot(n, VCOL(ws, 0), u1);
      *nred += 1;
      axpy(n, -s2, VCOL(ws, 0), u1);
      HH(ws, 0, 0) += s2;
    }
  }

  int rotated = 0; /* columns rotated so far */
  for (int j = 1; j <= kmax; ++j) {
    const int tail = (j == kmax);
    double* u = VCOL(ws, j);
    if (!tail) orc_spmv(n, ws->rowptr, ws->col, ws->val, u, ws->w);
    /* the single global reduction of this step */
    for (int i = 0; i < j; ++i) ws->a[i] = dot(n, VCOL(ws, i), u);
    double sigma = dot(n, u, u);
    double d = 0.0;
    if (!tail) {
      for (int i = 0; i < j; ++i) ws->c[i] = dot(n, VCOL(ws, i), ws->w);
      d = dot(n, u, ws->w);
    }
    *nred += 1;

    /* lagged norm completes column j-1 */
    double beta = sqrt(sigma);
    HH(ws, j, j - 1) = beta;
    const int brk = beta <= BREAKDOWN_FACTOR * 2.220446049250313e-16 * hcol_norm(ws, j - 1);
    const int c = j - 1;
    const int rotate_now = !pairs || c == 0 || c % 2 == 0 || tail || brk;
    double est = out.est;
    if (rotate_now) {
      for (int q = rotated; q <= c; ++q) {
        est = rotate_column(ws, q) / bnorm;
        if (*hlen < hcap) hist[*hlen] = est;
        *hlen += 1;
      }
      rotated = c + 1;
    }
    out.k = j;
    out.est = est;
    if (brk) {
      out.breakdown = 1;
      if (beta != 0.0) scal(n, 1.0 / beta, u);
      break;
    }
    scal(n, 1.0 / beta, u); /* v_j */

    /* row j of T = (I + L)^{-1} from ell = a / beta (Section II recurrence) */
    for (int i = 0; i < j; ++i) ws->a[i] /= beta;
    for (int k = 0; k < j; ++k) {
      double t = 0.0;
      for (int i = k; i < j; ++i) t += ws->a[i] * TL(ws, i, k);
      TL(ws, j, k) = -t;
    }
    TL(ws, j, j) = 1.0;
    if (tail || (rotate_now && est <= tol)) break;

    /* s = [c / beta; d / beta^2], r = T s, H(0:j, j) = r */
    for (int i = 0; i < j; ++i) ws->s[i] = ws->c[i] / beta;
    ws->s[j] = d / (beta * beta);
    for (int i = 0; i <= j; ++i) {
      double t = 0.0;
      for (int k = 0; k <= i; ++k) t += TL(ws, i, k) * ws->s[k];
      ws->r[i] = t;
      HH(ws, i, j) = t;
    }
    /* u_{j+1} = w / beta - V_j r */
    double* un = VCOL(ws, j + 1);
    for (int64_t l = 0; l < n; ++l) un[l] = ws->w[l] / beta;
    for (int i = 0; i <= j; ++i) axpy(n, -ws->r[i], VCOL(ws, i), un);
    if (reorth) { /* second reduction: s2 = V_j^T u_{j+1} (a is free now) */
      for (int i = 0; i <= j; ++i) ws->a[i] = dot(n, VCOL(ws, i), un);
      *nred += 1;
      for (int i = 0; i <= j; ++i) {
        axpy(n, -ws->a[i], VCOL(ws, i), un);
        HH(ws, i, j) += ws->a[i];
      }
    }
  }
  return out;
}


/* ------------------------------------------------------------------------- */
/* GMRES-IR: the one-reduce cycle in FP32 inside FP64 restarts [A13].        */
/* ------------------------------------------------------------------------- */
/* Mixed-precision iterative refinement (an extension; the paper is FP64
 * throughout). Every n-vector of a cycle -- the basis, A u with the matrix
 * values rounded to FP32, the block inner products and the MAXPY -- is FP32,
 * summed sequentially in FP32. The small dense arithmetic (beta, T, Givens,
 * least squares) is FP64, and so are the restart residual b - A x, its norm and
 * the correction x += V y (the FP32 basis widened exactly to FP64). */

static void spmv_f32(int64_t n, const int32_t* rowptr, const int32_t* col, const float* val32,
                     const float* x, float* y) {
  ORC_PAR_FOR
  for (int64_t i = 0; i < n; ++i) {
    float s = 0.0f;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s += val32[p] * x[col[p]];
    y[i] = s;
  }
}

static float dot_f32(int64_t n, const float* x, const float* y) {
  float s = 0.0f;
  ORC_PAR_SUM_S
  for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
  return s;
}

/* Round an FP32 value to the nearest BF16 value (8 significant bits, ties to
 * even), returned as the FP32 number it represents [A18]. BF16 is the upper
 * half of an FP32 word; NaN stays NaN. */
static float round_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return f; /* Inf / NaN */
  const uint32_t lsb = (u >> 16) & 1u;
  u = (u + 0x7fffu + lsb) & 0xffff0000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

/* Exported for the pin that compares the rounding with an independent BF16 conversion. */
float orc_round_bf16(float f) { return round_bf16(f); }

static void round_bf16_vec(int64_t n, float* x, int on) {
  if (!on) return;
  for (int64_t i = 0; i < n; ++i) x[i] = round_bf16(x[i]);
}

/* One cycle of cycle_one_reduce's steps with FP32 vectors. With bf16 set, each
 * basis vector v_j is stored in BF16: rounded once, when it is normalized
 * (v_0 when it is formed) [A18]. On entry V column 0
 * (FP64) holds r0 = b - A x and beta0 = ||r0|| (FP64). On exit the cycle's FP32
 * basis, widened, is in V (FP64) for the correction, and H, T, g as in FP64. */
static cycle_out cycle_one_reduce_f32(cycle_ws* ws, float* V32, float* w32, const float* val32, int kmax,
                                      double beta0, double bnorm, double tol, double* hist, int* hlen,
                                      int hcap, int64_t* nred, int bf16) {
  cycle_out out = {0, 0, 0.0};
  const int64_t n = ws->n;
  const int ld = ws->m + 1;
#define V32COL(k) (V32 + (size_t)(k) * n)
  for (int64_t l = 0; l < n; ++l) V32COL(0)[l] = (float)(VCOL(ws, 0)[l] / beta0); /* v_0 */
  round_bf16_vec(n, V32COL(0), bf16);
  memset(ws->g, 0, sizeof(double) * (size_t)ld);
  ws->g[0] = beta0;
  memset(ws->T, 0, sizeof(double) * (size_t)ld * ld);

  /* step 0 */
  spmv_f32(n, ws->rowptr, ws->col, val32, V32COL(0), w32);
  double d0 = (double)dot_f32(n, V32COL(0), w32);
  *nred += 1;
  TL(ws, 0, 0) = 1.0;
  HH(ws, 0, 0) = d0;
  for (int64_t l = 0; l < n; ++l) V32COL(1)[l] = w32[l] - (float)d0 * V32COL(0)[l];

  int kcols = 0;
  for (int j = 1; j <= kmax; ++j) {
    const int tail = (j == kmax);
    float* u = V32COL(j);
    if (!tail) spmv_f32(n, ws->rowptr, ws->col, val32, u, w32);
    for (int i = 0; i < j; ++i) ws->a[i] = (double)dot_f32(n, V32COL(i), u);
    double sigma = (double)dot_f32(n, u, u);
    double d = 0.0;
    if (!tail) {
      for (int i = 0; i < j; ++i) ws->c[i] = (double)dot_f32(n, V32COL(i), w32);
      d = (double)dot_f32(n, u, w32);
    }
    *nred += 1;

    double beta = sqrt(sigma);
    HH(ws, j, j - 1) = beta;
    double est = rotate_column(ws, j - 1) / bnorm;
    if (*hlen < hcap) hist[*hlen] = est;
    *hlen += 1;
    out.k = j;
    out.est = est;
    kcols = j;
    if (beta <= BREAKDOWN_FACTOR * 2.220446049250313e-16 * hcol_norm(ws, j - 1)) {
      out.breakdown = 1;
      break;
    }
    const float ib = (float)(1.0 / beta);
    for (int64_t l = 0; l < n; ++l) u[l] *= ib; /* v_j */
    round_bf16_vec(n, u, bf16);

    for (int i = 0; i < j; ++i) ws->a[i] /= beta;
    for (int k = 0; k < j; ++k) {
      double t = 0.0;
      for (int i = k; i < j; ++i) t += ws->a[i] * TL(ws, i, k);
      TL(ws, j, k) = -t;
    }
    TL(ws, j, j) = 1.0;
    if (tail || est <= tol) break;

    for (int i = 0; i < j; ++i) ws->s[i] = ws->c[i] / beta;
    ws->s[j] = d / (beta * beta);
    for (int i = 0; i <= j; ++i) {
      double t = 0.0;
      for (int k = 0; k <= i; ++k) t += TL(ws, i, k) * ws->s[k];
      ws->r[i] = t;
      HH(ws, i, j) = t;
    }
    float* un = V32COL(j + 1);
    const float fb = (float)beta;
    for (int64_t l = 0; l < n; ++l) un[l] = w32[l] / fb;
    for (int i = 0; i <= j; ++i) {
      const float ri = (float)ws->r[i];
      const float* vi = V32COL(i);
      for (int64_t l = 0; l < n; ++l) un[l] -= ri * vi[l];
    }
  }
  /* widen the used basis for the FP64 correction (exact) */
  for (int k = 0; k <= kcols && k <= ws->m; ++k)
    for (int64_t l = 0; l < n; ++l) VCOL(ws, k)[l] = (double)V32COL(k)[l];
#undef V32COL
  return out;
}

static int all_finite(int64_t n, const double* v) {
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(v[i])) return 0;
  return 1;
}

/* Restarted GMRES(m) for A x = b. x holds x0 on entry and the solution on exit.
 * Convergence is ||r|| / ||b|| <= tol [A5]: a cycle stops early when the Givens
 * estimate reaches tol; the true residual b - A x is then computed, and a new
 * cycle starts from it unless it is below tol or max_iter steps are spent.
 *
 * hist[k] (k < hist_cap) receives the Givens estimate after Arnoldi column k
 * completes, over all cycles [A8]. If V1/H1/T1/k1 are non-NULL they receive
 * the first cycle's normalized basis (n x (m+1)), unrotated Hessenberg
 * ((m+1) x m), T ((m+1) x (m+1), one-reduce only) and its column count. */
int orc_gmres(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
              const double* b, double* x, int variant, int m, double tol, int max_iter,
              double* hist, int hist_cap, orc_info* info,
              double* V1, double* H1, double* T1, int* k1) {
  if (n <= 0 || m <= 0 || max_iter < 0 || !(tol >= 0.0) || !b || !x || !info) return ORC_ERR_ARG;
  if (variant != ORC_VARIANT_MGS && variant != ORC_VARIANT_ONE_REDUCE && variant != ORC_VARIANT_IR_FP32 &&
      variant != ORC_VARIANT_CGS2 && variant != ORC_VARIANT_PIPE2 && variant != ORC_VARIANT_IR_BF16)
    return ORC_ERR_ARG;
  memset(info, 0, sizeof(*info));
  if (!all_finite(n, b) || !all_finite(n, x)) {
    info->status = ORC_ERR_NONFINITE;
    return ORC_ERR_NONFINITE;
  }
  /* the basis needs no more columns than the iterations allowed */
  const int mm = (max_iter > 0 && max_iter < m) ? max_iter : m;
  cycle_ws ws;
  memset(&ws, 0, sizeof(ws));
  ws.n = n;
  ws.rowptr = rowptr;
  ws.col = col;
  ws.val = val;
  ws.m = mm;
  const size_t ld = (size_t)mm + 1;
  ws.V = (double*)malloc(sizeof(double) * (size_t)n * ld);
  ws.w = (double*)malloc(sizeof(double) * (size_t)n);
  ws.H = (double*)calloc(ld * mm, sizeof(double));
  ws.Rg = (double*)calloc(ld * mm, sizeof(double));
  ws.cs = (double*)calloc(ld, sizeof(double));
  ws.sn = (double*)calloc(ld, sizeof(double));
  ws.g = (double*)calloc(ld, sizeof(double));
  ws.T = (double*)calloc(ld * ld, sizeof(double));
  ws.a = (double*)calloc(ld, sizeof(double));
  ws.c = (double*)calloc(ld, sizeof(double));
  ws.s = (double*)calloc(ld, sizeof(double));
  ws.r = (double*)calloc(ld, sizeof(double));
  double* res = (double*)malloc(sizeof(double) * (size_t)n);
  float* V32 = NULL;
  float* w32 = NULL;
  float* val32 = NULL;
  int status = ORC_OK;
  if (variant == ORC_VARIANT_IR_FP32 || variant == ORC_VARIANT_IR_BF16) {
    const int64_t nnz = rowptr[n];
    V32 = (float*)malloc(sizeof(float) * (size_t)n * ld);
    w32 = (float*)malloc(sizeof(float) * (size_t)n);
    val32 = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    if (!V32 || !w32 || !val32) {
      status = ORC_ERR_OOM;
      goto done;
    }
    for (int64_t p = 0; p < nnz; ++p) val32[p] = (float)val[p];
  }
  if (!ws.V || !ws.w || !ws.H || !ws.Rg || !ws.cs || !ws.sn || !ws.g || !ws.T || !ws.a ||
      !ws.c || !ws.s || !ws.r || !res) {
    status = ORC_ERR_OOM;
    goto done;
  }

  const double bnorm = nrm2(n, b);
  info->reductions += 1;
  if (bnorm == 0.0) {
    memset(x, 0, sizeof(double) * n);
    info->rel_resid_true = 0.0;
    goto done;
  }
  int hlen = 0;
  int first = 1;
  for (;;) {
    /* true residual r = b - A x: also the next cycle's r0 */
    orc_spmv(n, rowptr, col, val, x, res);
    for (int64_t i = 0; i < n; ++i) res[i] = b[i] - res[i];
    double beta0 = nrm2(n, res);
    info->reductions += 1;
    info->rel_resid_true = beta0 / bnorm;
    if (!isfinite(beta0)) {
      status = ORC_ERR_NONFINITE;
      break;
    }
    if (beta0 / bnorm <= tol) {
      status = ORC_OK;
      break;
    }
    if (info->iters >= max_iter) {
      status = ORC_MAXITER;
      break;
    }
    int kmax = max_iter - info->iters;
    if (kmax > mm) kmax = mm;
    memcpy(VCOL(&ws, 0), res, sizeof(double) * n);
    memset(ws.H, 0, sizeof(double) * ld * mm);
    cycle_out co;
    if (variant == ORC_VARIANT_MGS)
      co = cycle_mgs(&ws, kmax, beta0, bnorm, tol, hist, &hlen, hist_cap, &info->reductions);
    else if (variant == ORC_VARIANT_ONE_REDUCE || variant == ORC_VARIANT_CGS2 || variant == ORC_VARIANT_PIPE2)
      co = cycle_one_reduce(&ws, kmax, beta0, bnorm, tol, hist, &hlen, hist_cap, &info->reductions,
                            variant == ORC_VARIANT_CGS2, variant == ORC_VARIANT_PIPE2);
    else
      co = cycle_one_reduce_f32(&ws, V32, w32, val32, kmax, beta0, bnorm, tol, hist, &hlen, hist_cap,
                                &info->reductions, variant == ORC_VARIANT_IR_BF16);
    if (first) {
      if (V1) memcpy(V1, ws.V, sizeof(double) * (size_t)n * ld);
      if (H1) memcpy(H1, ws.H, sizeof(double) * ld * mm);
      if (T1) memcpy(T1, ws.T, sizeof(double) * ld * ld);
      if (k1) *k1 = co.k;
      first = 0;
    }
    update_solution(&ws, co.k, x);
    info->iters += co.k;
    info->restarts += 1;
    info->breakdowns += co.breakdown;
    info->rel_resid_est = co.est;
  }
done:
  info->status = status;
  free(ws.V); free(ws.w); free(ws.H); free(ws.Rg); free(ws.cs); free(ws.sn); free(ws.g);
  free(ws.T); free(ws.a); free(ws.c); free(ws.s); free(ws.r); free(res);
  free(V32); free(w32); free(val32);
  return status;
}
