/*
 * lsgmres.h: C ABI of the B300-native low-synchronization GMRES library.
 *
 * Solves A x = b for a square sparse A in CSR form with restarted GMRES(m)
 * (Saad and Schultz), in one of four orthogonalization schemes:
 *
 *   GMRES_MGS             MGS-GMRES, Algorithm 6 of Swirydowicz, Langou,
 *                         Ananthan, Yang and Thomas, "Low synchronization GMRES
 *                         algorithms" (arXiv:1809.05805). Step i makes i+1
 *                         inner products and one norm, each a separate
 *                         grid-wide reduction (Section IV).
 *   GMRES_ONE_REDUCE_MGS  one-synchronization MGS-GMRES with lagged
 *                         normalization, Algorithm 7 built on the Level-2
 *                         compact-WY MGS of Algorithm 4 (Sections II-III). Each
 *                         step makes one grid-wide reduction: the block inner
 *                         product [V_{j-1} u_j]^T [u_j  A u_j], which also
 *                         carries the lagged norm of u_j.
 *   GMRES_CGS2_LVL2       two-synchronization GMRES on the Level-2 iterated
 *                         classical Gram-Schmidt of Algorithm 5: the one-reduce
 *                         step, then a second block reduction V_{j+1}^T u_{j+1}
 *                         and projection that re-orthogonalize the new vector
 *                         (basis orthogonal to machine precision).
 *   GMRES_ONE_REDUCE_PIPE2  the one-reduce scheme with the Givens rotations
 *                         applied two columns at a time (the L = 2 pipeline of
 *                         Algorithm 8); the same basis and Hessenberg, the
 *                         convergence test after every second column.
 *
 * All schemes run on the same kernels (CSR SpMV, multi-column dot, MAXPY) on
 * one GPU. All arithmetic on the solve path is FP64, except in the GMRES-IR
 * precisions (GMRES_IR_FP32, GMRES_IR_BF16), whose restart cycles run in FP32.
 *
 * Conventions for every entry point:
 *   - Every call returns a gmres_status; no call aborts or exits. After an
 *     error, gmres_last_error(h) describes it.
 *   - "device" pointers are CUDA global-memory addresses on the handle's device
 *     (for example torch.Tensor.data_ptr() of a CUDA tensor); "host" pointers
 *     are ordinary CPU memory. Vectors are contiguous FP64 arrays of length n.
 *   - Work is ordered on the handle's stream (gmres_set_stream; default: the
 *     legacy default stream). Calls that return results to the host
 *     synchronize that stream before returning.
 *   - The library owns its copy of A and all Krylov workspace; the caller owns
 *     b and x and every buffer it passes in. No call retains a caller pointer.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef LSGMRES_H
#define LSGMRES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GMRES_OK = 0,              /* converged: ||b - A x|| / ||b|| <= tol */
  GMRES_MAXITER = 1,         /* max_iter Arnoldi steps spent before convergence */
  GMRES_BREAKDOWN_EXACT = 2, /* reserved: a vanishing Krylov direction ends a cycle; the
                                solve restarts from the true residual, so it is not returned */
  GMRES_ERR_ARG = -1,        /* invalid argument or invalid CSR structure */
  GMRES_ERR_CUDA = -2,       /* a CUDA runtime call failed */
  GMRES_ERR_NONFINITE = -3,  /* NaN or Inf in b, x0 or a reduction */
  GMRES_ERR_OOM = -4,        /* device or pinned-host allocation failed */
  GMRES_ERR_TIMEOUT = -5     /* a bounded device-side wait gave up, or a host wait timed out */
} gmres_status;

typedef enum { GMRES_MGS = 0, GMRES_ONE_REDUCE_MGS = 1, GMRES_CGS2_LVL2 = 2, GMRES_ONE_REDUCE_PIPE2 = 3 } gmres_ortho;

/* Arithmetic of the Krylov loop.
 *   GMRES_FP64     everything in FP64.
 *   GMRES_IR_FP32  GMRES-IR: every restart cycle runs the one-reduce Arnoldi
 *                  steps with FP32 vectors (basis, A u with FP32 matrix values,
 *                  block inner products and MAXPY, FP32 accumulation), while the
 *                  residual b - A x, the small dense algebra and the correction
 *                  x += V y stay FP64, so the solve still reaches FP64 residuals.
 *                  One-reduce scheme only; gmres_set allocates the FP32 copies
 *                  ((m+1) n + n + nnz floats, n doubles) on first use.
 *   GMRES_IR_BF16  GMRES_IR_FP32 with the basis stored in BF16: each new basis
 *                  vector is rounded to BF16 (nearest, ties to even) as the
 *                  MAXPY stores it, and widened exactly on every load; all
 *                  arithmetic and accumulation stay FP32 (w and the matrix
 *                  values too). Halves the basis traffic of the cycles; each
 *                  cycle reduces the residual less, so a solve takes more
 *                  steps. One-reduce scheme only; gmres_set allocates
 *                  (m+1) n BF16 values plus the FP32 copies on first use. */
typedef enum { GMRES_FP64 = 0, GMRES_IR_FP32 = 1, GMRES_IR_BF16 = 2 } gmres_prec;

typedef struct gmres_ctx* gmres_handle;

/* Square CSR matrix: row i holds entries rowptr[i] .. rowptr[i+1]-1 of col/val.
 * rowptr[0] = 0, rowptr nondecreasing, rowptr[n] = nnz, 0 <= col < n.
 * on_device = 0: the three arrays are host memory; 1: device memory.
 * Either way gmres_create copies them; the caller may free them afterwards. */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
  int on_device;
} gmres_csr;

typedef struct {
  int iters;              /* Arnoldi steps (Hessenberg columns) over all cycles */
  int restarts;           /* cycles run */
  int status;             /* the gmres_status of the solve */
  int breakdowns;         /* cycles ended by a vanishing new direction */
  double rel_resid_true;  /* ||b - A x|| / ||b|| at exit, recomputed from x */
  double rel_resid_est;   /* last Givens estimate |g_{k+1}| / ||b|| */
  int64_t reductions;     /* grid-wide reductions executed on the device */
  int64_t grid_syncs;     /* kernel boundaries that did work (one grid-wide sync each) */
  int64_t kernel_launches;/* kernels launched by the solve */
  double seconds;         /* wall time of the solve */
} gmres_info;

/* Create a solver for A with restart length m_restart (1 <= m <= 128) and
 * relative tolerance tol >= 0. Validates A on the host (structure above; n > 0;
 * nnz < 2^31), copies it to the device and allocates the Krylov basis
 * ((m+1) columns of n doubles) and the small dense state; when the fixed-point
 * block dot is active (gmres_set_block_dot; the default for matrices that take
 * the tile-pair kernel) also a second copy of the basis as fixed-point limbs
 * (8 bytes per entry), written once per column and read by the later steps'
 * block dots and MAXPYs; when that copy does not fit, the handle starts with
 * FP64 products instead (see gmres_set_block_dot). Defaults:
 * GMRES_ONE_REDUCE_MGS, GMRES_FP64, max_iter = 10 * m, legacy default stream.
 * Errors: GMRES_ERR_ARG, GMRES_ERR_OOM, GMRES_ERR_CUDA; *out is NULL then. */
gmres_status gmres_create(const gmres_csr* A, int m_restart, double tol, gmres_handle* out);

/* Select the orthogonalization scheme, the arithmetic and the iteration limit
 * (max_iter >= 0 Arnoldi steps over all cycles). GMRES_ERR_ARG for an unknown
 * scheme, GMRES_IR_FP32 or GMRES_IR_BF16 with a scheme other than
 * GMRES_ONE_REDUCE_MGS, or max_iter < 0;
 * GMRES_ERR_OOM if the FP32 copies cannot be allocated. */
gmres_status gmres_set(gmres_handle h, gmres_ortho ortho, gmres_prec prec, int max_iter);

/* Change the tolerance (tol >= 0). */
gmres_status gmres_set_tol(gmres_handle h, double tol);

/* Order all later work of h on cuda_stream (a cudaStream_t; NULL = legacy default). */
gmres_status gmres_set_stream(gmres_handle h, void* cuda_stream);

/* Solve A x = b. b: device, n doubles, read only. x: device, n doubles, holds
 * x0 on entry and the solution on exit. A cycle ends when the Givens residual
 * estimate reaches tol; the solve ends when the recomputed true residual
 * ||b - A x|| / ||b|| <= tol (GMRES_OK) or after max_iter steps
 * (GMRES_MAXITER). b = 0 gives x = 0. info may be NULL. Synchronizes the stream.
 * Errors: GMRES_ERR_ARG (NULL or misaligned pointer: b and x must be 8-byte
 * aligned), GMRES_ERR_NONFINITE, GMRES_ERR_CUDA, GMRES_ERR_TIMEOUT (a bounded
 * wait of the step kernel for the bulk copies that stage its CSR and basis
 * tiles in shared memory gave up after about a second; see
 * gmres_test_stall_staging). */
gmres_status gmres_solve(gmres_handle h, const double* b, double* x, gmres_info* info);

/* As gmres_solve with b and x in host memory: copies b and x0 to the device,
 * solves, and copies x back (the copies are part of the call). */
gmres_status gmres_solve_host(gmres_handle h, const double* b_host, double* x_host,
                              gmres_info* info);

/* Copy the residual-estimate history of the last solve (one entry per
 * Arnoldi step: |g_{k+1}| / ||b|| after column k completes) into host_buf
 * (capacity cap). *len receives the full history length. */
gmres_status gmres_history(gmres_handle h, double* host_buf, int cap, int* len);

/* Release all device and host memory of h. NULL is accepted. */
gmres_status gmres_destroy(gmres_handle h);

/* Description of the last error on h. With h = NULL: the last error of a call
 * that has no handle (a failed gmres_create, lsg_block_dot_noalloc) made by
 * the calling host thread; each host thread has its own such message. The
 * string is owned by the library and stays valid until the next failing call
 * on the same handle (or, for NULL, by the same thread). */
const char* gmres_last_error(gmres_handle h);

/* Per-kernel timing. With on = 1, later solves bracket every kernel launch
 * with CUDA events on the handle's stream (a few microseconds of host work
 * per launch) and gmres_profile reports, per kernel class, the summed device
 * time, the launch count and the algorithmic bytes and flops of the launches
 * that did work (launches that found their cycle already finished are counted
 * separately). Counters reset at the start of every solve.
 * Classes: 0 one-reduce step (fused SpMV + block dot + epilogue), 1 Arnoldi
 * MAXPY, 2 MGS SpMV + first dot, 3 MGS axpy + next dot, 4 residual / norm,
 * 5 least squares, 6 solution update (MAXPY), 7 launches that did no work,
 * 8 second (re-orthogonalizing) block reduction of GMRES_CGS2_LVL2, 9 its
 * in-place MAXPY, 10 whole cycles in one launch (gmres_set_persistent; their
 * bytes and flops are the cycle's steps and MAXPYs). */
#define GMRES_PROFILE_CLASSES 11
gmres_status gmres_set_profile(gmres_handle h, int on);
gmres_status gmres_profile(gmres_handle h, int cls, double* total_ms, int64_t* launches,
                           double* alg_bytes, double* alg_flops);

/* Arithmetic of the FP64 block inner product [V_{j-1} u_j]^T [u_j  A u_j] of
 * the one-reduce step (Algorithm 4's single reduction; Section IV's mass inner
 * product). fixed_point = 1 (the default): where the step kernel stages tile
 * pairs with its column ring, the products of the basis columns run on the
 * integer pipes as exact fixed-point products -- each FP64 value rescaled by
 * a power of two to a 58-bit integer (relative to its column's largest
 * exponent, or its tile pair's for u and w), split in two 29-bit limbs,
 * multiplied and summed exactly in 64-bit integers over each tile pair, then
 * converted to FP64 once -- while the slow FP64 pipe of this GPU is spent on
 * the SpMV, the norms and the few remainder columns only. Each product's
 * inputs are exact to 2^-58 of their vector's largest entry and the integer
 * sums are exact, so a sum x^T y is off by at most about 2^-57 (max|x| sum|y_i|
 * + max|y| sum|x_i|) before its last FP64 roundings: below FP64 summation's
 * classical bound gamma_n sum|x_i y_i| unless the largest entries of one
 * vector sit where the other is many orders of magnitude smaller. fixed_point = 0: FP64 fused
 * multiply-adds throughout. *active (may be NULL) receives whether this
 * handle's step kernel uses the fixed-point form (it needs staging mode 2:
 * large enough matrices whose tile-pair CSR fits the shared memory). The
 * choice changes rounding only. Turning the form on allocates the limb copy of
 * the basis (see gmres_create) if the handle has none; GMRES_ERR_OOM or
 * GMRES_ERR_CUDA if that fails, and the FP64 form stays in use. */
gmres_status gmres_set_block_dot(gmres_handle h, int fixed_point, int* active);

/* Run-to-run reproducibility of the fixed-point step kernel (the one
 * gmres_set_block_dot reports active). By default (on = 0) its CTAs take the
 * 512-row tile pairs from a counter, so that CTAs that run faster take more;
 * which CTA sums which pair, and so the order of the FP64 additions of the
 * pairs' exact sums, then varies from run to run, and results can differ in
 * the last bits between identical solves (each within the same bounds). on = 1
 * assigns pair p to CTA p mod P (P the reduction grid): every sum in a fixed
 * order, results bitwise reproducible for a given device and grid, about 2%
 * slower at 256^3. Every other kernel of the library sums in a fixed
 * order always. Never errors on a valid handle. */
gmres_status gmres_set_reproducible(gmres_handle h, int on);

/* One launch per restart cycle, for small systems whose steps are bound by
 * launch and synchronization latency rather than by memory or arithmetic.
 * The kernel keeps every CTA resident (a cooperative launch) and runs all
 * Arnoldi steps of the cycle (Algorithm 7): per step the fused SpMV + block
 * dot with its single grid reduction and the epilogue in the last CTA, a wait
 * for that epilogue, the MAXPY beside the Givens rotation of the previous
 * column, and a software grid barrier -- one grid reduction and one barrier
 * per step, without kernel boundaries. Arithmetic as the per-step launches of
 * the unstaged kernel (FP64 fused multiply-adds).
 * mode = 1: use it whenever it applies (FP64, GMRES_ONE_REDUCE_MGS or
 * GMRES_ONE_REDUCE_PIPE2, and the grid fits on the device at once); 0: never;
 * -1 (the default): when it applies and the system has at most one 256-row
 * tile per CTA of the reduction grid (n <= 2 x SMs x 256). *active (may be
 * NULL) receives whether the handle's next solve uses it. Every wait of the
 * launch is bounded (about one second of SM clocks); a wait that gives up
 * ends the cycle and the solve returns GMRES_ERR_TIMEOUT. Never errors on a
 * valid handle. */
gmres_status gmres_set_persistent(gmres_handle h, int mode, int* active);

/* Testing the bounded waits of the persistent cycle: with on = 1 its grid
 * barrier waits for one CTA more than the grid has; with on = 2 the wait for
 * each step's epilogue waits for one epilogue more than there is. Either way
 * the first such wait runs out (no fault, no hang: about one second), the
 * kernel returns and the solve reports GMRES_ERR_TIMEOUT; on = 0 restores
 * normal operation. Other values: GMRES_ERR_ARG. */
gmres_status gmres_test_stall_barrier(gmres_handle h, int on);

/* Testing the bounded waits of the CSR staging. The step kernel brings each
 * tile's CSR into shared memory with bulk copies whose completion it waits for
 * on an mbarrier, for at most ~2^31 SM clocks (about one second); a wait that
 * runs out marks the solve stalled, the kernel stops using staged data and
 * returns, and the solve (or gmres_arnoldi) returns GMRES_ERR_TIMEOUT. With
 * on = 1, later FP64 solves of this handle announce 16 bytes per copy that no
 * copy delivers, so every such wait runs out (each step launch then takes about
 * two seconds); on = 0 restores normal operation. *staged (may be NULL)
 * receives whether the handle's FP64 step kernel stages its CSR at all (a
 * matrix whose largest tile does not fit the shared memory is read from global
 * memory, with no waits). Never errors on a valid handle. */
gmres_status gmres_test_stall_staging(gmres_handle h, int on, int* staged);

/* ------------------------------------------------------------------------
 * Batched solves: many independent systems, one launch per Arnoldi step.
 * ------------------------------------------------------------------------
 * The paper defines the method for one system (Algorithm 7, Sections III-IV);
 * batching is this library's addition and changes no system's arithmetic.
 * A batch holds `count` square CSR systems of any sizes. Its solve runs
 * restarted one-reduce MGS-GMRES(m) (FP64) on all of them in lock-step cycles:
 * each system's rows occupy a region of a shared row arena (padded to whole
 * 512-row tile pairs) in every Krylov basis column, with its own CSR, and each
 * Arnoldi step of the cycle is one fused SpMV + block-inner-product launch and
 * one MAXPY launch for every system still iterating, with a grid reduction and
 * an epilogue per system. A system's results match a solve of it alone up to
 * the order of the partial sums of its reductions (which depends on the grid
 * and on the other systems sharing the launches; for a given batch and grid it
 * is fixed, so results are bitwise reproducible). A system leaves its cycle when its own residual
 * estimate reaches tol and the batch when its true residual does (or after
 * max_iter steps). Its first residual pass carries ||b|| in the same
 * reduction as ||r0||, so a batched solve reports one reduction fewer than the
 * single-system solver. The launch shape (grid, rows per thread) is chosen by
 * a timing autotuner at create.
 */
typedef struct gmres_batch_ctx* gmres_batch;

/* Create a batch from `count` >= 1 host CSR matrices (A[i].on_device must be
 * 0; the arrays are copied), restart length 1 <= m <= 128, tol >= 0,
 * max_iter >= 0 steps per system. The row arena holds the m + 1 basis columns
 * twice, as FP64 values and as the fixed-point limbs the engine's block dot
 * and MAXPY read (8 bytes per entry each). Errors: GMRES_ERR_ARG, GMRES_ERR_OOM,
 * GMRES_ERR_CUDA (details in gmres_batch_last_error(NULL)). */
gmres_status gmres_batch_create(const gmres_csr* A, int count, int m_restart, double tol, int max_iter,
                                gmres_batch* out);

/* Order the batch's work on cuda_stream (cudaStream_t; NULL = legacy default;
 * a non-default stream lets each cycle run as a replayed CUDA graph). */
gmres_status gmres_batch_set_stream(gmres_batch bt, void* cuda_stream);

/* Grid of the batched reduction kernels (CTAs; CTA c takes the contiguous
 * range [c Ta / P, (c+1) Ta / P) of the Ta 256-row tiles of the systems still
 * iterating, P = min(ctas, Ta)). ctas = 0 re-runs the autotuner; otherwise
 * 1 <= ctas <= 8 x the SM count, else GMRES_ERR_ARG. The grid changes only
 * the order of the partial sums. */
gmres_status gmres_batch_set_grid(gmres_batch bt, int ctas);
gmres_status gmres_batch_get_grid(gmres_batch bt, int* ctas);

/* Rows per thread of the batched step kernel: 1 (one 256-row tile per CTA
 * iteration) or 2 (two consecutive tiles of one system together, so the CSR
 * loads of two rows are in flight at once; the same sums in the same order);
 * chosen by the autotuner with the grid (gmres_batch_set_grid(bt, 0)). Other
 * values: GMRES_ERR_ARG. */
gmres_status gmres_batch_set_rows_per_thread(gmres_batch bt, int rows);
gmres_status gmres_batch_get_rows_per_thread(gmres_batch bt, int* rows);

/* FP64 products of the batched block dot [V_{j-1} u_j]^T [u_j  A u_j] and of
 * the Arnoldi MAXPY as exact fixed-point integers on the integer pipes, as
 * gmres_set_block_dot for one system: each basis value becomes a 58-bit
 * integer relative to its system's column exponent bound (kept per system by
 * the kernels that write the column), u and w relative to their tile pair's
 * largest entry; products are summed exactly per tile pair (per row in the
 * MAXPY) and rounded to FP64 once. fixed_point = 1 (the default) uses them
 * for FP64 batches with two rows per thread, the step kernel streaming the
 * basis through a per-warp ring of column slices in shared memory when the
 * listed systems' tile-pair CSR fits the staging capacity left beside the
 * ring, else loading it directly; -1 uses them with direct loads always; 0
 * uses FP64 fused multiply-adds. *active (may be NULL) receives the form the
 * next solve uses for the systems listed now: 0 FP64 FMAs, 1 fixed point
 * with direct loads, 2 fixed point with the ring. The choice changes rounding
 * only (bound as gmres_set_block_dot states). Never errors on a valid
 * handle. */
gmres_status gmres_batch_set_block_dot(gmres_batch bt, int fixed_point, int* active);

/* Solve all systems: b[i] and x[i] are device pointers (host array of `count`
 * pointers) to system i's right-hand side and its x0 / solution. info may be
 * NULL or a host array of `count` entries (per system). Returns GMRES_OK if
 * every system converged, GMRES_MAXITER if some hit max_iter, or the first
 * error. Errors: GMRES_ERR_ARG (NULL arrays, a NULL or not 8-byte-aligned
 * pointer), GMRES_ERR_CUDA; a system whose b or x0 holds NaN/Inf reports
 * GMRES_ERR_NONFINITE in its info entry while the others are solved.
 * The b[i] are read-only; each x[i] is written once, at the end. Synchronizes
 * the stream. */
gmres_status gmres_batch_solve(gmres_batch bt, const double* const* b, double* const* x, gmres_info* info);

/* As gmres_batch_solve with b[i] and x[i] in host memory (pinned or
 * pageable): the copies into and out of the device are part of the call. */
gmres_status gmres_batch_solve_host(gmres_batch bt, const double* const* b_host, double* const* x_host,
                                    gmres_info* info);

/* Per-launch timing of batch solves (as gmres_set_profile / gmres_profile;
 * classes 0, 1, 4, 5, 6 and 7 occur). Each launch's algorithmic bytes and
 * flops are summed over the systems it did work for. */
gmres_status gmres_batch_set_profile(gmres_batch bt, int on);
gmres_status gmres_batch_profile(gmres_batch bt, int cls, double* total_ms, int64_t* launches,
                                 double* alg_bytes, double* alg_flops);

/* Launch-by-launch record of the last profiled batch solve, in launch order:
 * class (as gmres_profile), step index j (step and MAXPY launches; 1 for the
 * residual launches), 256-row tiles listed at the launch, device ms,
 * algorithmic flops. Any output may be NULL; at most cap entries are written;
 * *count receives the total. */
gmres_status gmres_batch_launch_log(gmres_batch bt, int cap, int* cls, int* step, int64_t* active_tiles,
                                    float* ms, double* alg_flops, int* count);

/* Residual-estimate history of system i in the last batch solve (as gmres_history). */
gmres_status gmres_batch_history(gmres_batch bt, int i, double* host_buf, int cap, int* len);

gmres_status gmres_batch_destroy(gmres_batch bt);

/* Description of the last error on bt (or, with NULL, of the calling host
 * thread's last failed gmres_batch_create). */
const char* gmres_batch_last_error(gmres_batch bt);

/* ------------------------------------------------------------------------
 * Serving loop: continuous batching of independent solves.
 * ------------------------------------------------------------------------
 * Not in the paper (which defines the method for one system); each request is
 * solved by the paper's one-reduce MGS-GMRES (Algorithm 7), FP64 or with FP32
 * cycles inside FP64 restarts (GMRES_IR_FP32), exactly as a batch would.
 * A server owns two batched engines, one per precision, each with its own
 * CUDA stream and host worker thread, so their launches overlap on the
 * device. Each engine's device memory (Krylov bases, for FP64 also as
 * fixed-point limbs, and vectors for a fixed
 * number of arena rows, a CSR pool, per-request state) is allocated once at
 * create from its share of hbm_budget_bytes. A worker runs lock-step restart
 * cycles over its iterating requests; at every cycle boundary it completes
 * the requests whose true residual reached their tol (copying x to x_out) and,
 * while the next cycle runs, admits queued requests first come first served
 * as long as arena rows, CSR pool space and a request slot are free. A request
 * thus starts at the next cycle boundary of its engine after room frees up,
 * and its Krylov basis stays on the device until it completes. Results equal a
 * solve of the request alone up to the order of the partial sums of its
 * reductions (which depends on the requests sharing its launches). */
typedef struct gmres_server_ctx* gmres_server;

typedef struct {
  int m_restart;             /* restart length of every request, 1..128 */
  int max_iter;              /* largest per-request max_iter accepted (sizes the histories) */
  int max_requests;          /* request slots per engine (requests iterating at once) */
  int64_t hbm_budget_bytes;  /* device bytes of both engines together */
  double ir_share;           /* fraction of the budget for the GMRES_IR_FP32 engine, 0..1 */
  int64_t nnz_per_row_hint;  /* expected nonzeros per row: splits an engine's bytes between arena rows and CSR */
} gmres_server_config;

typedef struct {
  int64_t submitted, rejected;       /* all requests; rejected at submit (too large for their engine) */
  int64_t admitted[2], completed[2]; /* per engine: [0] FP64, [1] GMRES_IR_FP32 */
  int64_t queued[2], running[2], peak_running[2], cycles[2];
  int64_t engine_bytes[2];           /* device bytes the engine holds (arena + CSR pool) */
  int64_t peak_bytes_in_use[2];      /* largest arena + CSR bytes occupied by admitted requests */
  int64_t arena_rows[2];
  int64_t kernel_launches[2];        /* engine kernel launches since create */
  double busy_seconds[2];            /* worker time with requests in flight */
  double wall_seconds;               /* since create */
} gmres_server_counters;

/* Create a server on the current device and start its workers. Errors:
 * GMRES_ERR_ARG (a field out of range), GMRES_ERR_OOM (the budget does not fit
 * on the device), GMRES_ERR_CUDA; details in gmres_server_last_error(NULL). */
gmres_status gmres_server_create(const gmres_server_config* cfg, gmres_server* out);

/* Queue a request (O(1): the full CSR check runs when the request is admitted,
 * and a request failing it completes with GMRES_ERR_ARG): A is a host CSR,
 * b and x0 (may be NULL:
 * zero) host or device vectors of A->n doubles, x_out where the solution is
 * written at completion (host or device). A, b, x0 and x_out are borrowed:
 * they must stay valid and unchanged until the request completes. prec is
 * GMRES_FP64 or GMRES_IR_FP32; 0 <= max_iter <= cfg.max_iter. *id receives the
 * request's id. Errors: GMRES_ERR_ARG, GMRES_ERR_OOM (larger than its
 * engine's whole share of the budget: the request is rejected). */
gmres_status gmres_server_submit(gmres_server sv, const gmres_csr* A, const double* b, const double* x0,
                                 double* x_out, double tol, int prec, int max_iter, int64_t* id);

/* Completion of request id: *done = 1 when x_out holds its result; then info
 * (may be NULL) receives its counts, status and info.seconds = its latency
 * from submit to completion. */
gmres_status gmres_server_poll(gmres_server sv, int64_t id, int* done, gmres_info* info);

/* Block until request id completes (returns its status if negative, else
 * GMRES_OK) or timeout_s passes (GMRES_ERR_TIMEOUT). */
gmres_status gmres_server_wait(gmres_server sv, int64_t id, double timeout_s, gmres_info* info);

/* Block until every submitted request has completed (or GMRES_ERR_TIMEOUT). */
gmres_status gmres_server_drain(gmres_server sv, double timeout_s);

/* Forget a completed request (its id becomes unknown). */
gmres_status gmres_server_release(gmres_server sv, int64_t id);

gmres_status gmres_server_stats(gmres_server sv, gmres_server_counters* st);

/* Per-launch timing of the engines' kernels (as gmres_set_profile /
 * gmres_profile; engine 0 = FP64, 1 = GMRES_IR_FP32). Switching is allowed
 * only while no request is queued or running (GMRES_ERR_ARG otherwise) and
 * resets the totals. */
gmres_status gmres_server_set_profile(gmres_server sv, int on);
gmres_status gmres_server_profile(gmres_server sv, int engine, int cls, double* total_ms, int64_t* launches,
                                  double* alg_bytes, double* alg_flops);

/* Latencies (seconds, submit to completion) of the completed requests, in
 * completion order; at most cap written, *len receives the total. */
gmres_status gmres_server_latencies(gmres_server sv, double* buf, int cap, int* len);

/* Stop: queued requests are dropped (never complete); requests already
 * admitted run to completion first. */
gmres_status gmres_server_destroy(gmres_server sv);

/* Description of the last error on sv (or, with NULL, of the calling host
 * thread's last failed gmres_server_create). */
const char* gmres_server_last_error(gmres_server sv);

/* ------------------------------------------------------------------------
 * Single steps of the solve path, exposed for parity tests.
 * ------------------------------------------------------------------------ */

/* y = A x (device x, y; n doubles each). The CSR SpMV of the Arnoldi step
 * (Section IV: the matvec partitions by rows). */
gmres_status lsg_spmv(gmres_handle h, const double* x, double* y);

/* The fused SpMV + block inner product of one one-reduce step (Algorithm 4's
 * single reduction, Section IV's mass inner product): with V the first j
 * columns of a column-major device array (leading dimension ldv >= n) and
 * u a device vector, computes w = A u (written to device w) and the 2j+2 sums
 *   X[0:j]   = V^T u,   X[j:2j] = V^T w,   X[2j] = u^T u,   X[2j+1] = u^T w
 * into host X. If use_spmv is 0, w is an input (not overwritten) and the
 * SpMV is skipped (the standalone QR form of Algorithm 4). 0 <= j <= m. */
gmres_status lsg_block_dot(gmres_handle h, const double* V, int64_t ldv, int j,
                           const double* u, double* w, int use_spmv, double* X);

/* lsg_block_dot_noalloc: the fused SpMV + block inner product of lsg_block_dot
 * for callers that cannot allocate device memory -- for example code running
 * under a memory pool or arena that owns all device memory, a process whose
 * allocator is locked for the duration of a solve, or a host library that may
 * not call cudaMalloc/cudaFree in its calling context. It needs no handle and
 * makes no allocation: the reduction scratch lives in a fixed array compiled
 * into this library (about 300 KB, present on every device that loads the
 * library until the process exits). The paper has no counterpart; it is an
 * interface convenience.
 *
 * Inputs (all device memory, caller-owned): the CSR arrays rowptr/col/val of an
 * n x n matrix (used when use_spmv != 0), V (first j columns of a column-major
 * array, leading dimension ldv >= n), u (n doubles), w (n doubles: written
 * with A u when use_spmv != 0, read otherwise). Output: X (device, 2j+2
 * doubles) = [V^T u, V^T w, u^T u, u^T w], as in lsg_block_dot.
 * Limits: 0 <= j <= 64 and 1 <= n < 2^31; larger j returns GMRES_ERR_ARG with
 * the limit in gmres_last_error(NULL). Work is queued on cuda_stream (a
 * cudaStream_t, NULL = legacy default) and the call does not synchronize.
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture. All calls share the one scratch array, so calls that
 * could run at the same time on the GPU (different streams, threads) race and
 * must be serialized by the caller. Errors are described by
 * gmres_last_error(NULL). */
gmres_status lsg_block_dot_noalloc(const int32_t* rowptr, const int32_t* col, const double* val, int64_t n,
                                   const double* V, int64_t ldv, int j, const double* u, double* w,
                                   int use_spmv, double* X, void* cuda_stream);

/* MAXPY (Section IV): y_out = alpha * y_in + sum_{k<K} c[k] * V[:, k] for
 * device V (leading dimension ldv >= n, 16-byte aligned columns), device
 * y_in and y_out (may alias), host c (K values), 0 <= K <= m + 1. */
gmres_status lsg_maxpy(gmres_handle h, const double* V, int64_t ldv, int K, const double* c,
                       double alpha, const double* y_in, double* y_out);

/* Run one GMRES cycle of k Arnoldi steps (1 <= k <= m) from the device vector
 * r0, with no convergence test, using the selected scheme and precision (a
 * GMRES-IR handle runs one inner cycle from r0 / ||r0|| rounded to its basis
 * type, as gmres_solve does; its basis is exported widened to FP64 and its
 * Hessenberg is that of the unit right-hand side). Returns the
 * normalized basis V_out (device, n x (k+1), leading dimension n), the
 * unrotated Hessenberg H_out (host, (k+1) x k, column-major) and, for the
 * one-reduce scheme, T_out = (I + L)^{-1} (host, (k+1) x (k+1), lower;
 * zeros for MGS). Any output pointer may be NULL. *k_done receives the
 * number of columns completed (< k only after a breakdown). */
gmres_status gmres_arnoldi(gmres_handle h, const double* r0, int k, double* V_out,
                           double* H_out, double* T_out, int* k_done);

/* ------------------------------------------------------------------------
 * Instruction-throughput probe (measurement only).
 * ------------------------------------------------------------------------
 * The paper has no counterpart. On B300 the FP64 Arnoldi step is bound by the
 * FP64 pipe rather than by HBM, so the roofline it is reported against is a
 * measured instruction rate; these calls measure it, and the rates of the
 * integer and conversion instructions an FP64 product can be emulated with.
 * lsg_probe_pipe launches ctas_per_sm x (SM count) CTAs of 256 threads on the
 * current device (legacy default stream; it synchronizes), each thread
 * running 8 independent chains of `iters` x 4 instructions of kind `op` and
 * nothing else, and reports per-SM and whole-GPU rates. It allocates and
 * frees a few KB of device memory per call. 1 <= ctas_per_sm <= 8,
 * 1 <= iters <= 2^24. Errors: GMRES_ERR_ARG, GMRES_ERR_CUDA, described by
 * lsg_probe_last_error() (per host thread). */
typedef enum {
  LSG_PROBE_DFMA = 0,        /* fma.rn.f64 */
  LSG_PROBE_DADD = 1,        /* add.rn.f64 */
  LSG_PROBE_FFMA = 2,        /* fma.rn.f32 */
  LSG_PROBE_IMAD = 3,        /* mad.lo.u32 */
  LSG_PROBE_IMAD_WIDE = 4,   /* mad.wide.u32: 32 x 32 + 64 -> 64 bits */
  LSG_PROBE_IMAD_HI = 5,     /* mad.hi.u32 */
  LSG_PROBE_IADD = 6,        /* add.u32 */
  LSG_PROBE_LOP3 = 7,        /* lop3.b32 */
  LSG_PROBE_SHF = 8,         /* shf.l.wrap.b32 (funnel shift) */
  LSG_PROBE_I2F_F64 = 9,     /* cvt.rn.f64.s64 */
  LSG_PROBE_F2I_F64 = 10,    /* cvt.rni.s64.f64 */
  LSG_PROBE_F2F_F32_F64 = 11,/* cvt.rn.f32.f64 */
  LSG_PROBE_I2F_F32 = 12,    /* cvt.rn.f32.s32 */
  LSG_PROBE_FLO = 13         /* clz.b32 */
} lsg_probe_op;

typedef struct {
  double ops_per_clk_per_sm; /* thread instructions retired per SM clock (from clock64 stamps) */
  double ops_per_s;          /* thread instructions per second, whole GPU (CUDA events) */
  double sm_mhz;             /* SM clock during the run: clock64 cycles / event time */
  double seconds;            /* device time of the timed launch */
  int sms;                   /* SM count */
} lsg_probe_result;

gmres_status lsg_probe_pipe(int op, int ctas_per_sm, int iters, lsg_probe_result* out);
const char* lsg_probe_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LSGMRES_H */
