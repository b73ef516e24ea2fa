/*
 * hqr.h -- C ABI of the GB300 hierarchical tile Householder QR library.
 *
 * Method: Dongarra, Faverge, Herault, Langou, Robert, "Hierarchical QR
 * factorization algorithms for multi-core cluster systems" (arXiv 1110.1553).
 * A tile QR of an m x n tile matrix (tiles b x b, M = m b, N = n b) is fully
 * determined by its elimination list (Sec. 2, Alg. 1); each elimination is
 * carried out by the tile kernels GEQRT, TSQRT/TTQRT and UNMQR, TSMQR/TTMQR
 * (Alg. 2). HQR builds the list from TS domains of a tiles, a low-level tree
 * inside each of p virtual domains and a high-level tree over the domains
 * (Sec. 4.1-4.2). Q is applied by replaying the trees (Sec. 5.1).
 *
 * Conventions shared by every call:
 *  - Matrices passed by the caller are column-major with a leading dimension
 *    (LAPACK style). "d" pointers are device pointers, "h" pointers host
 *    pointers. The caller owns every buffer it passes; the library never
 *    frees or keeps them.
 *  - The library copies A into its own tile-major workspace (zero padded to
 *    whole tiles, Sec. 2 assumes M and N are multiples of b); the caller's A
 *    is never written.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). All device
 *    work of a call is ordered on it; calls that return a host result
 *    synchronize the stream first, and say so.
 *  - Return value: 0 on success; -k when argument k (1-based) is invalid;
 *    a positive HQR_ERR_* code otherwise. No call aborts the process and no
 *    kernel traps: device-side waits have a time limit and report
 *    HQR_ERR_TIMEOUT. hqr_strerror() turns a code into text; for
 *    HQR_ERR_CUDA, hqr_last_error() gives the CUDA error text.
 */
#ifndef HQR_H
#define HQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Reduction tree shapes (Sec. 3.1-3.3): FLAT and BINARY of Sec. 3.1, GREEDY
 * of Sec. 3.2 (Table 4), FIBONACCI = the Modi-Clarke order-1 scheme named in
 * Sec. 3.3 (its definition is not printed in the paper; see hqr_elim_list). */
typedef enum { HQR_FLAT = 0, HQR_BINARY = 1, HQR_GREEDY = 2, HQR_FIBONACCI = 3 } hqr_tree_t;

/* Kernel kind of an elimination (Sec. 2, Alg. 2). */
typedef enum { HQR_KIND_TS = 0, HQR_KIND_TT = 1 } hqr_kind_t;

/* One elimination elim(i, killer, k) of Sec. 2: tile (i, k) is zeroed by
 * tile (killer, k). level: 0 = TS level, 1 = low level, 2 = coupling
 * ("domino") level, only in lists from hqr_elim_list_domino, 3 = high level
 * (Sec. 4.2). step: time step of the unit-time model of Sec. 3.1-3.2.
 * 24 bytes, no padding surprises. */
typedef struct {
  int32_t k;
  int32_t i;
  int32_t killer;
  int32_t kind;
  int32_t level;
  int32_t step;
} hqr_elim_t;

/* Arithmetic of the factorization. HQR_FP64: FP64 storage and arithmetic
 * everywhere (the paper's setting, Sec. 5.1). HQR_FP32: FP32 storage and
 * FP32 arithmetic (panel norms with a scaled second pass on under- or
 * overflow); device buffers passed with it hold float. HQR_FP32_BF16X3:
 * FP32 storage; tiles of nb = 128 run the updates (UNMQR, TSMQR, TTMQR) on
 * the tensor cores (tcgen05) with every FP32 operand split into three BF16
 * pieces (six BF16 products per step, FP32 accumulation: about FP32
 * accuracy) and one full 128 x 128 T per tile (ib is taken as nb); other
 * tile sizes fall back to HQR_FP32 arithmetic. hqr_geqrf requires nb = 128
 * with it. */
typedef enum { HQR_FP64 = 0, HQR_FP32 = 1, HQR_FP32_BF16X3 = 2 } hqr_prec_t;

enum {
  HQR_SUCCESS = 0,
  HQR_ERR_CUDA = 1,      /* a CUDA runtime call failed; see hqr_last_error() */
  HQR_ERR_TIMEOUT = 2,   /* a device-side wait reached its time limit */
  HQR_ERR_NOMEM = 3,     /* device or host allocation failed */
  HQR_ERR_CAPACITY = 4,  /* output array too small; *count holds the size needed */
  HQR_ERR_INVALID_LIST = 5, /* elimination list breaks a rule of Sec. 2 */
  HQR_ERR_SINGULAR = 6,  /* exact zero on the diagonal of R (hqr_gels) */
  HQR_ERR_INTERNAL = 7,  /* internal consistency check failed */
  HQR_ERR_TOO_LARGE = 8, /* problem exceeds the fixed limits of hqr_geqrf_r_noalloc */
  HQR_ERR_BUSY = 9,      /* server: no slot, memory or pool space free right now; retry later */
  HQR_ERR_BUDGET = 10,   /* server: the request can never fit the server's budget */
  HQR_ERR_NOCONV = 11    /* refinement did not reach the tolerance within its rounds */
};

/* Opaque factorization: owns the tile workspace (V and R), the T factors,
 * a copy of the elimination list and the device task graphs. */
typedef struct hqr_factors hqr_factors;

/*
 * hqr_elim_list -- HQR elimination list (Sec. 4.1-4.2, trees of Sec. 3.1-3.3).
 * Host only, integer only, deterministic.
 *   m, n      tile rows and tile columns, m >= n >= 1.
 *   a         TS domain size (a = 1: no TS kernels), a >= 1.
 *   p         number of virtual domains; tile row i is in domain i mod p.
 *   low_tree  tree over the TS heads of each domain (level 1).
 *   high_tree tree over the p domain tops (level 3).
 *   out, cap  caller array of cap records (out may be NULL when cap == 0).
 *   count     receives the number of records, sum_{k<n} (m-k-1).
 * Records are written sorted by (k, step, i). If cap is too small nothing is
 * written, *count is set and HQR_ERR_CAPACITY is returned.
 * Where the paper leaves a rule open (Sec. 3.3 names FIBONACCI without
 * defining it; Sec. 4.1 refers to a lost figure for the TS domain alignment),
 * this library reads it as follows: heads are every a-th active row counted
 * from the domain top; GREEDY takes readiness into account
 * (a row is a candidate at step t once its last elimination is before t);
 * FIBONACCI cuts the leaves below the survivor into groups of 1, 2, 3, ...
 * killed by the same number of leaves right above them, bottom group first.
 */
int hqr_elim_list(int m, int n, int a, int p, int low_tree, int high_tree,
                  hqr_elim_t *out, size_t cap, size_t *count);

/*
 * hqr_elim_list_domino -- hqr_elim_list with the coupling level of Sec. 4.2
 * (level 2, "domino"): in panel k, the TS domains and the low-level tree of
 * domain c reduce only its rows on and below its local diagonal (local index
 * k, tile row k p + c), to that diagonal row; the rows between the domain's
 * top and its local diagonal (the diagonal row included) are then killed by
 * the top, one after the other in ascending order, with TT kernels (records
 * with level 2); the high-level tree reduces the tops as before. With p = 1
 * the list equals hqr_elim_list's. Same arguments and returns.
 */
int hqr_elim_list_domino(int m, int n, int a, int p, int low_tree, int high_tree,
                         hqr_elim_t *out, size_t cap, size_t *count);

/*
 * hqr_validate_list -- check a list against the validity rules of Sec. 2:
 * every tile (i, k), i > k, killed exactly once; both rows ready (zeroed in
 * every earlier panel before this record); the killer not yet zeroed in this
 * panel; a TS kill only of a square tile (a row that has not killed before in
 * this panel) and no kill by a TS-zeroed row. Host only.
 * Returns 0 if valid, HQR_ERR_INVALID_LIST otherwise, -k for bad arguments.
 */
int hqr_validate_list(int m, int n, const hqr_elim_t *list, size_t count);

/*
 * hqr_task_graph -- a task graph the library builds for an m x n tile
 * matrix and a valid list (Alg. 2 expansion and its dependencies, with the
 * current slab widths and panel split setting), for inspection. Host only,
 * no device work.
 *   nb, ib, prec  as in hqr_geqrf.
 *   kind     0: the factorization (hqr_geqrf); 1: Q^T applied to a right-
 *            hand side of `param` column slabs (hqr_apply_q, trans = 1);
 *            2: Q applied (trans = 0); 3: a least-squares problem of a plan
 *            with `param` refinement rounds (0: QR solve); 4: the same as a
 *            server request (packing tasks first); 5: a problem of a plan
 *            from hqr_ls_plan_create_tol with at most `param` rounds (round
 *            tasks carry trans = 2 and k = the round; op 18 is a round's
 *            convergence check, op 19 a round's gate; op 20 joins a round's
 *            residual rows before its A^T r tasks); 6: the graph of
 *            hqr_geqrf_r_noalloc (FP64 only, its limits apply:
 *            HQR_ERR_TOO_LARGE beyond them; built in the static storage that
 *            entry point uses, so not concurrently with it).
 *   tasks    caller array of 10 int32 per task: op (0 GEQRT, 1 UNMQR,
 *            2 TSQRT, 3 TSMQR, 4 TTQRT, 5 TTMQR, 6.. the vector tasks of
 *            least-squares graphs), blk (0: the whole panel / every block;
 *            q + 1: block q of a split panel), i, r, k, j, c0, cw, trans,
 *            tgt (fields of the device task record); tasks are in a
 *            topological order.
 *   succ_ptr caller array of ntasks + 1 offsets into succ (CSR successors;
 *            with priority policy 1, each task's successors in the order the
 *            device graph lists them: decreasing bottom level).
 *   succ     caller array of nedges successor ids.
 * With tasks == NULL only *ntasks and *nedges are set (HQR_ERR_CAPACITY
 * when buffers were given but are too small). Returns
 * HQR_ERR_INVALID_LIST for an invalid list, -k for bad arguments.
 */
int hqr_task_graph(int m, int n, int nb, int ib, int prec, const hqr_elim_t *list, size_t count, int kind,
                   int param, int32_t *tasks, int64_t task_cap, int64_t *succ_ptr, int32_t *succ, int64_t succ_cap,
                   int64_t *ntasks, int64_t *nedges);

/*
 * hqr_geqrf -- tile QR factorization A = Q R driven by an elimination list
 * (Alg. 1 with the eliminations of Alg. 2), executed by a persistent device
 * kernel that starts each tile task as soon as its inputs are final
 * (Sec. 4.2, "Execution scheme").
 *   dA      device, M x N column-major, lda >= M; read only.
 *   M, N    matrix size, M >= N >= 1. Padded with zeros to whole tiles.
 *   prec    hqr_prec_t.
 *   nb      tile size b: multiple of 8, 8 <= nb <= 256.
 *   ib      inner block of the compact-WY T factors: divides nb, at most 16
 *           or exactly 32, a multiple of 2 (FP64) or 4 (FP32).
 *   list    host array of `count` records for m = ceil(M/nb), n = ceil(N/nb)
 *           tiles, or NULL for the default list (flat TS domains of a = 4,
 *           p = 1, greedy low tree).
 *   F       receives the new factorization (free with hqr_factors_free).
 * The stream is synchronized before return (the device reports its status).
 */
int hqr_geqrf(const void *dA, int M, int N, int lda, int prec, int nb, int ib,
              const hqr_elim_t *list, size_t count, hqr_factors **F, void *stream);

/*
 * hqr_refactor -- factor a new matrix of the same shape with an existing
 * factorization object (same list, tile size and task graph; no allocation).
 * Used for repeated factorizations. Synchronizes the stream.
 */
int hqr_refactor(hqr_factors *F, const void *dA, int lda, void *stream);

/*
 * hqr_refactor_async -- as hqr_refactor but does not synchronize: the device
 * status is left in the factorization and read by hqr_status(). No host
 * synchronization, so it can be captured in a CUDA graph.
 */
int hqr_refactor_async(hqr_factors *F, const void *dA, int lda, void *stream);

/* hqr_status -- synchronize `stream` and return the device status of the
 * last asynchronous call on F (0, HQR_ERR_TIMEOUT or HQR_ERR_INTERNAL). */
int hqr_status(hqr_factors *F, void *stream);

/*
 * hqr_get_r -- copy the N x N upper triangular factor R into dR (device,
 * column-major, ldr >= N). The strict lower part of dR is set to zero.
 */
int hqr_get_r(const hqr_factors *F, void *dR, int ldr, void *stream);

/*
 * hqr_get_tiles -- copy the factored tile workspace, Mp x Np (padded sizes,
 * see hqr_factors_info), into dOut (device, column-major, ld >= Mp): R in the
 * upper triangles of the tiles on the diagonal and above, GEQRT V below the
 * diagonal of each triangle tile, TSQRT V2 in TS-killed tiles, TTQRT V2 in
 * the upper triangle of TT-killed tiles (Sec. 2 storage of the kernels).
 */
int hqr_get_tiles(const hqr_factors *F, void *dOut, int ld, void *stream);

/*
 * hqr_get_t -- copy all T factors into dT (device). Layout: for tile (i, k)
 * of the m x n tile grid and which = 0 (GEQRT T) or 1 (TSQRT/TTQRT T), an
 * ib x nb column-major array at element offset ((k*m + i)*2 + which)*ib*nb.
 * Block q of reflectors owns columns q*ib .. q*ib+ib-1 (an upper triangle).
 */
int hqr_get_t(const hqr_factors *F, void *dT, void *stream);

/* hqr_kernel_ms -- device time (CUDA events on the call's stream) of the
 * persistent task kernel of the last factorization or apply-Q run on F.
 * Waits for that kernel to finish. */
int hqr_kernel_ms(hqr_factors *F, float *ms);

/* hqr_kernel_times -- device times (CUDA events on each run's stream) of
 * the persistent task kernel of every factorization or apply-Q run on F
 * since the previous call (at most the last 64 runs), oldest first, into
 * ms[0 .. *count). Waits for the last of those kernels. cap too small:
 * HQR_ERR_CAPACITY with *count = the number needed. */
int hqr_kernel_times(hqr_factors *F, float *ms, int cap, int *count);

/*
 * hqr_trace -- per-task timing of the persistent kernel (for analysis).
 * enable = 1: record from the next run on (allocates a device buffer of
 * 3 x 8 bytes per task); 0: stop and free it; -1: copy the last run's
 * records to `host` (cap >= 3 * *count entries): per task its start and end
 * (%globaltimer, ns) and (CTA index << 32 | SM id). *count = tasks traced.
 */
int hqr_trace(hqr_factors *F, int enable, uint64_t *host, size_t cap, size_t *count);

/* hqr_factors_info -- sizes of a factorization: padded rows/cols, tiles,
 * tile size, inner block, number of tasks in the factorization graph. */
int hqr_factors_info(const hqr_factors *F, int *Mp, int *Np, int *m, int *n,
                     int *nb, int *ib, int64_t *ntasks);

/*
 * hqr_apply_q -- B <- Q^T B (trans = 1) or B <- Q B (trans = 0), replaying
 * the elimination list forward or in reverse (Sec. 5.1: Q is formed by
 * applying the reverse trees to the identity).
 *   dB      device, M x nrhs column-major (M = the factorization's rows),
 *           ldb >= M; overwritten with the result.
 */
int hqr_apply_q(hqr_factors *F, int trans, void *dB, int ldb, int nrhs, void *stream);

/*
 * hqr_gels_qr -- least squares min ||b - A x||_2 for M >= N, full rank, in
 * the storage precision, for many right-hand sides and a given list:
 * factor, c = Q^T b, x = R^{-1} c[0:N] (problem of Sec. 2 with the
 * application of Sec. 5.1).
 *   db      device, M x nrhs, ldb >= M; read only.
 *   dx      device, N x nrhs, ldx >= N; receives x.
 *   list    as in hqr_geqrf (NULL = default).
 * Returns HQR_ERR_SINGULAR if a diagonal entry of R is exactly zero.
 */
int hqr_gels_qr(const void *dA, int M, int N, int lda, const void *db, int ldb, int nrhs,
                void *dx, int ldx, int prec, int nb, int ib, const hqr_elim_t *list,
                size_t count, void *stream);

/* Outcome of hqr_gels. */
typedef struct {
  int iters;               /* refinement rounds applied (0 when max_iter = 0) */
  int converged;           /* 1: the tolerance was met (always 1 when max_iter = 0) */
  double rel_correction;   /* ||d||_2 / ||x||_2 of the last applied correction d; -1 without refinement */
  double backward_error;   /* ||b - A x||_2 / (||A||_F ||x||_2 + ||b||_2), FP64 on the device */
  double normal_residual;  /* ||A^T (b - A x)||_2 / (||A||_F ||b - A x||_2): near rounding level at a
                              least-squares solution even when b - A x itself is large */
  int64_t singular_index;  /* first column with an exact zero on R's diagonal, -1 if none */
} hqr_gels_info;

/*
 * hqr_gels -- least squares min ||b - A x||_2 for one M x N matrix, M >= N,
 * solved through the tile QR (the problem of Sec. 2; Q^T applied by
 * replaying the trees, Sec. 5.1), with the tolerance-stopped refinement of
 * hqr_ls_plan_create_tol.
 *   dA, lda   device, column-major, lda >= M, in the storage precision of
 *             `prec` (double for HQR_FP64, float otherwise); read only.
 *   db        device, M doubles; read only.
 *   dx        device, N doubles; receives x.
 *   prec      HQR_FP64: FP64 tile QR. HQR_FP32 / HQR_FP32_BF16X3: the
 *             mixed-precision solve: FP32 tile QR (tiles of 128 on the tensor
 *             cores with BF16X3), FP64 only in the refinement (residual,
 *             A^T r, triangular solves with the low-precision R).
 *   tol       stop the refinement at the first compensated round whose
 *             correction has ||d||_2 <= tol ||x||_2 (tol >= 0); see
 *             hqr_ls_plan_create_tol for the other stop.
 *   max_iter  refinement rounds at most, 0 <= max_iter <= 64. With 0, x is
 *             the plain QR solve R^{-1} (Q^T b)[0:N] in the storage precision.
 *   info      NULL, or receives the outcome (also on HQR_ERR_NOCONV and
 *             HQR_ERR_SINGULAR).
 * Tile configuration: the autotuner table (hqr_set_tuning / hqr_autotune)
 * or the built-in heuristic. Allocates and frees its own workspace and
 * synchronizes `stream`. Returns HQR_ERR_NOCONV when max_iter rounds did not
 * meet tol (x is then the last iterate) and HQR_ERR_SINGULAR when R has an
 * exact zero on its diagonal (info->singular_index names the column).
 */
int hqr_gels(const void *dA, int M, int N, int lda, const double *db, double *dx, int prec, double tol,
             int max_iter, hqr_gels_info *info, void *stream);

/*
 * hqr_debug_block_task -- testing aid for the device-side time limits: add
 * `extra` never-satisfied inputs to task `task` of F's factorization graph,
 * so the next hqr_refactor cannot finish and must return HQR_ERR_TIMEOUT
 * (after hqr_set_timeout_ms) instead of hanging. extra = 0 restores it.
 */
int hqr_debug_block_task(hqr_factors *F, int64_t task, int extra);

/*
 * hqr_geqrf_r_noalloc -- the R factor of A with no memory allocation at all.
 * The paper has no counterpart: this is an operational variant of hqr_geqrf
 * for callers that may not allocate device memory (the device memory belongs
 * to another allocator's pool, or cudaMalloc's implicit synchronization is
 * not acceptable at that point) or may not grow the host heap.
 *   dA, M, N, lda  device input, as in hqr_geqrf (read only).
 *   nb, ib         as in hqr_geqrf, with nb <= 64.
 *   list, count    elimination list for ceil(M/nb) x ceil(N/nb) tiles
 *                  (required; e.g. from hqr_elim_list called beforehand).
 *   dR, ldr        device output: the N x N upper triangular R (strict
 *                  lower part set to zero), ldr >= N.
 * Limits: at most 64 x 16 tile rows x columns and 256 tiles, at most 16384
 * tasks, and everything (tiles, T factors, task graph) within one 16 MiB
 * scratch array that is a static device variable of the library: it is
 * reserved on every GPU that loads the library until the process exits.
 * Larger problems return HQR_ERR_TOO_LARGE before any device work.
 * The schedule is a simpler one than hqr_geqrf's: fixed priority classes
 * (panels, then updates of the next tile column, then the rest) and whole
 * panel tasks (no split panels); the arithmetic of each task is the same.
 * An invalid list returns -7 (argument 7, as every -k code names argument k).
 * No cudaMalloc, cudaFree or other allocating call is made. The first call
 * on each device looks up that device's scratch address (a one-time set-up).
 * The call cannot be part of a CUDA graph: it copies its task graph from
 * static host memory and synchronizes `stream`, so a stream that is being
 * captured returns -11 (argument 11) before any work. All calls share the one
 * scratch array and the library's static host staging, so calls that
 * overlap (on the GPU, or from several host threads) race; the array keeps
 * the last call's contents and every call rewrites all it reads. The call
 * synchronizes `stream` and returns the device status.
 */
int hqr_geqrf_r_noalloc(const void *dA, int M, int N, int lda, int nb, int ib,
                        const hqr_elim_t *list, size_t count, void *dR, int ldr, void *stream);

/* ------------------------------------------------------------------------
 * Least-squares plans: one or many independent problems min ||b - A x||
 * (M >= N each, shapes may differ) solved by ONE persistent launch over the
 * merged task graph of all problems (Sec. 4.2 execution scheme applied to a
 * batch). Two solve modes:
 *  - refine_iters > 0 (mixed precision with HQR_FP32 storage): the tile QR
 *    gives R only; x comes from corrected semi-normal equations
 *    (Bjorck 1987): x0 = 0, then refine_iters times r = b - A x,
 *    g = A^T r (both FP64, compensated products and sums), R^T R d = g
 *    (FP64 triangular solves with the low-precision R), x += d.
 *  - refine_iters == 0: x = R^{-1} (Q^T b)[0:N] (Q^T b by replaying the
 *    list, Sec. 5.1), in the storage precision.
 * ------------------------------------------------------------------------ */
typedef struct {
  int M, N;          /* M >= N >= 1 */
  const void *dA;    /* device, column-major, storage precision of the plan */
  int lda;           /* >= M */
  const double *db;  /* device, M entries (FP64) */
  double *dx;        /* device, N entries (FP64); receives x */
} hqr_ls_problem_t;

/* Tile configuration of one problem; nb = 0 asks the plan to choose
 * (the autotuner table when set with hqr_set_tuning, else a heuristic). */
typedef struct {
  int nb, ib, a, p, low_tree, high_tree;
} hqr_tile_config_t;

typedef struct hqr_ls_plan hqr_ls_plan;

/*
 * hqr_ls_plan_create -- build the merged task graph and workspaces for
 * `count` problems. cfg: NULL or `count` entries. prec: HQR_FP64/HQR_FP32.
 * The problems' pointers are kept and used by every run; their buffers
 * must stay valid while the plan runs. No device work is started.
 */
int hqr_ls_plan_create(int count, const hqr_ls_problem_t *probs, const hqr_tile_config_t *cfg, int prec,
                       int refine_iters, hqr_ls_plan **plan);

/*
 * hqr_ls_plan_create_tol -- as hqr_ls_plan_create with refinement rounds
 * that stop at a tolerance (corrected semi-normal equations as above,
 * started from the QR solution x0 = R^{-1} (Q^T b)[0:N] computed in the
 * storage precision instead of x0 = 0): at
 * most max_iter rounds (1 .. 64); each problem stops after the first round
 * whose correction d has ||d||_2 <= tol ||x||_2 and whose residual and A^T r
 * were compensated (tolerance met), or after two compensated rounds in a row
 * whose corrections did not shrink by 10 % (no more progress: the attainable
 * accuracy with this R is reached; reported as not met). Rounds start with
 * plain FP64 sums and switch to compensated ones when the corrections, below
 * 1e-6, stop halving from round to round or reach tol (decided on the
 * device, two rounds ahead). The rounds after a problem's last one are
 * skipped on the device. A problem that does not meet tol reports
 * HQR_ERR_NOCONV (hqr_ls_plan_status); see hqr_ls_plan_refine_info.
 */
int hqr_ls_plan_create_tol(int count, const hqr_ls_problem_t *probs, const hqr_tile_config_t *cfg, int prec,
                           int max_iter, double tol, hqr_ls_plan **plan);

/* hqr_ls_plan_refine_info -- outcome of problem idx after a run of a plan
 * from hqr_ls_plan_create_tol: rounds applied, the last applied correction
 * ||d||_2 / ||x||_2, whether tol was met, how many of the applied rounds had
 * compensated residuals, and the first column with an exact zero on R's
 * diagonal (-1: none). Plans from hqr_ls_plan_create report their fixed
 * round count, -1, 0, their compensated round count and -1. Any output may
 * be NULL. Synchronizes `stream`. */
int hqr_ls_plan_refine_info(hqr_ls_plan *plan, int idx, int *iters, double *rel_correction, int *converged,
                            int *compensated, int64_t *singular_index, void *stream);

/* hqr_ls_plan_run -- solve all problems (asynchronous on `stream`): one
 * preparation kernel (tile packing, b, x = 0), the persistent task kernel,
 * one kernel copying every x out. If hqr_ls_plan_capture was called, the
 * captured CUDA graph is launched instead. */
int hqr_ls_plan_run(hqr_ls_plan *plan, void *stream);

/* hqr_ls_plan_capture -- capture one run on `stream` (not the legacy
 * default stream) into a CUDA graph used by later runs. A plan that splits
 * its launch (hqr_set_split_launch) keeps the SM share it has at capture:
 * run it a few times first so that the share is set from measured times. */
int hqr_ls_plan_capture(hqr_ls_plan *plan, void *stream);

/* hqr_ls_plan_status -- synchronize `stream`; 0, the device status of the
 * last run, HQR_ERR_SINGULAR if a problem's R had an exact zero diagonal
 * (that problem's x is then not meaningful), or HQR_ERR_NOCONV if a problem
 * of a tolerance plan did not meet its tolerance (the first problem's code
 * when several failed). */
int hqr_ls_plan_status(hqr_ls_plan *plan, void *stream);

/* hqr_ls_plan_correction -- size of the last refinement correction of
 * problem idx after a run: *rel = max_i |d_i| / max_i |x_i|, d the
 * correction the last CSNE round added to x (plans from
 * hqr_ls_plan_create_tol: ||d||_2 / ||x||_2 of the last applied round, the
 * measure their stop uses). A small value says the refinement has
 * converged; -1 when the plan has no refinement rounds. Synchronizes
 * `stream` (the one the plan ran on). */
int hqr_ls_plan_correction(hqr_ls_plan *plan, int idx, double *rel, void *stream);

/* hqr_ls_plan_info -- tasks of the merged graph, the paper's QR flop count
 * sum of 2 M N^2 - 2/3 N^3, and the device time of the last run (the task
 * kernel alone; the whole captured graph when it was launched). */
int hqr_ls_plan_info(hqr_ls_plan *plan, int64_t *ntasks, double *qr_flops, float *kernel_ms);

/* hqr_ls_plan_config -- the tile configuration chosen for problem `idx`. */
int hqr_ls_plan_config(const hqr_ls_plan *plan, int idx, hqr_tile_config_t *cfg);

/* hqr_ls_plan_trace -- per-task timing of the plan's task kernel, as
 * hqr_trace (enable 1 / 0 / -1 = read) but 4 words per task: start, end,
 * CTA << 32 | SM id, opcode << 24 | problem index. Must be enabled before
 * hqr_ls_plan_capture to be recorded by captured runs. */
int hqr_ls_plan_trace(hqr_ls_plan *plan, int enable, uint64_t *host, size_t cap, size_t *count);

void hqr_ls_plan_free(hqr_ls_plan *plan);

/*
 * hqr_set_tuning -- install an autotuner table: `count` entries, entry e
 * applies to problems with floor(log2 M) == keys[2e] and floor(log2 N) ==
 * keys[2e+1]. Host only; copied. count = 0 clears it.
 */
int hqr_set_tuning(int count, const int *keys, const hqr_tile_config_t *cfgs);

/*
 * hqr_critical_path -- unit-cost model of the factorization of an m x n tile
 * matrix by a list (host only): every task of the library's graph costs its
 * Sec. 2 weight (GEQRT 4, TSQRT 6, TTQRT 2, UNMQR 6, TSMQR 12, TTMQR 6 units
 * of b^3 / 3; column slabs and split-panel blocks their share). Returns the
 * longest chain of costs (the time on unbounded processors; the paper's
 * coarse model of Sec. 3 counts steps instead) and their sum (the time on
 * one processor). nb, ib, prec as in hqr_geqrf; -k for a bad argument k,
 * HQR_ERR_INVALID_LIST for an invalid list.
 */
int hqr_critical_path(int m, int n, int nb, int ib, int prec, const hqr_elim_t *list, size_t count,
                      double *critical_path, double *work);

/*
 * hqr_autotune -- measured autotuner for least-squares plans. For every
 * shape class (floor(log2 M), floor(log2 N)) among the `count` shapes
 * (Ms[q] x Ns[q]), times candidate tile configurations on `reps` random
 * problems of the class's geometric-mean shape solved in one plan (prec,
 * refine_iters as in hqr_ls_plan_create), in two stages: (1) nb in {32, 64,
 * 128} x TS domains a in {1, 4, 16} with greedy trees, or one flat TS
 * domain, with p = 1; (2) for the winner, p in {2, 4, 8, 16} x high-level
 * trees {greedy, Fibonacci, binary, flat}, ranked by the unit-cost model of
 * hqr_critical_path (the larger of the critical path and the work over the
 * resident CTAs), of which the best three are timed. Installs the fastest
 * per class with hqr_set_tuning. The chosen table is also copied to
 * keys_out (2 ints per class) / cfg_out when cap is large enough;
 * *nout = number of classes. Synchronizes `stream`; allocates and frees its
 * own random test matrices.
 */
int hqr_autotune(int count, const int *Ms, const int *Ns, int prec, int refine_iters, int reps,
                 int *keys_out, hqr_tile_config_t *cfg_out, int cap, int *nout, void *stream);

/* ------------------------------------------------------------------------
 * Least-squares server (continuous batching). One resident persistent task
 * kernel serves requests for its whole lifetime: a request submitted while
 * others are running is admitted as soon as a slot, workspace memory within
 * the HBM budget and task-pool space are free, its task graph (packing,
 * tile QR, solve as in hqr_ls_plan_create) is copied into the device pools
 * and announced through an inbox that the kernel polls, and its tasks then
 * run interleaved with those of every other live request. Each request's
 * tiles, T factors and vectors stay resident in its own workspace until it
 * completes. Completion is published in host-mapped memory.
 * ------------------------------------------------------------------------ */
typedef struct {
  int prec;            /* HQR_FP32 or HQR_FP32_BF16X3 (mixed precision), or HQR_FP64 */
  int refine_iters;    /* as in hqr_ls_plan_create */
  int max_live;        /* requests in flight at most */
  size_t hbm_budget;   /* bytes of request workspace (tiles, T, vectors) */
  int64_t task_pool;   /* task records in the device pool */
  int64_t edge_pool;   /* successor entries in the device pool */
} hqr_server_opts;

typedef struct hqr_server hqr_server;

/* hqr_server_create -- allocate the pools and the workspace arena
 * (hbm_budget bytes); nothing runs yet. */
int hqr_server_create(const hqr_server_opts *opts, hqr_server **server);

/* hqr_server_start -- launch the resident task kernel on the server's own
 * stream; returns at once. The kernel leaves by itself after about one
 * second without work (so an idle or forgotten server does not hold the
 * GPU); submit, poll and stop relaunch it whenever work is owed. */
int hqr_server_start(hqr_server *server);

/* hqr_server_submit -- admit one request (pointers as in hqr_ls_problem_t;
 * the caller keeps A, b and x valid until the request completes). Returns 0
 * and a ticket, HQR_ERR_BUSY when it does not fit right now (poll, then
 * retry), or HQR_ERR_BUDGET when it can never fit. The tile configuration
 * comes from the tuning table (hqr_set_tuning / hqr_autotune) or the
 * heuristic, with nb <= 128. */
int hqr_server_submit(hqr_server *server, const hqr_ls_problem_t *problem, int64_t *ticket);

/* hqr_server_poll -- collect requests completed since the last poll
 * (their tickets into done[0 .. min(cap, *count)) ) and free their
 * resources. Returns the kernel's status (0 while healthy). */
int hqr_server_poll(hqr_server *server, int64_t *done, int cap, int *count);

/* hqr_server_stats -- requests submitted / completed, live requests, bytes
 * of the budget in use. */
int hqr_server_stats(const hqr_server *server, int64_t *submitted, int64_t *completed, int *live,
                     size_t *bytes_in_use);

/* hqr_server_counters -- device-side counters for monitoring: out[0] inbox
 * entries claimed, out[1] inbox entries posted, out[2] stop flag, out[3]
 * tasks outstanding (approximate while running), out[4] 1 if the resident
 * kernel is running. cap >= 5. */
int hqr_server_counters(const hqr_server *server, uint32_t *out, int cap);

/* hqr_server_progress -- tasks completed and tasks in total of the live
 * request `ticket` (a snapshot read from the device; *done may lag). Returns
 * HQR_ERR_INTERNAL when no live request has that ticket. */
int hqr_server_progress(const hqr_server *server, int64_t ticket, int *done, int *total);

/* hqr_server_stop -- let the kernel finish all admitted work and exit;
 * returns its status. */
int hqr_server_stop(hqr_server *server);

void hqr_server_free(hqr_server *server);

/* hqr_factors_free -- release a factorization (NULL is allowed). */
void hqr_factors_free(hqr_factors *F);

/* Process-wide settings (hqr_set_slab_widths, hqr_set_panel_split,
 * hqr_set_split_launch, hqr_set_priority_policy, hqr_set_timeout_ms,
 * hqr_set_tuning): read when a
 * factorization, plan or server request is created (the time limit: when a
 * kernel is launched). They are plain globals: set them before, not while,
 * other threads create work. */

/* hqr_set_slab_widths -- engine tuning for factorizations and plans created
 * afterwards: column-slab width of an update task (w), of the trailing
 * update inside a panel task (wt), and V columns staged per chunk (vc,
 * must divide ib). 0 restores the built-in choice; values are even.
 * Larger slabs mean fewer, longer tasks and more shared memory per CTA. */
int hqr_set_slab_widths(int w, int wt, int vc);

/* hqr_set_panel_split -- panels of factorizations, plans and server requests
 * created afterwards whose tiles have nb >= min_nb (CUDA-core kernels, at
 * least two ib blocks per tile) run as one task per ib block plus the
 * updates of the panel's own trailing columns with that block, so that a
 * panel's trailing work spreads over several CTAs. 0 keeps whole panel tasks
 * everywhere; default 64. Returns -1 for min_nb < 0. */
int hqr_set_panel_split(int min_nb);

/* hqr_set_split_launch -- least-squares plans created afterwards that hold
 * both tensor-core problems (HQR_FP32_BF16X3 tiles of 128) and CUDA-core
 * ones run them as two persistent launches side by side: the tensor-core
 * kernel (one CTA per SM) on a share of the SMs and the CUDA-core kernel
 * (two CTAs per SM) on the rest, the share set from the parts' QR flops and
 * rebalanced from the two kernels' times after every timed run (not inside a
 * captured graph, which keeps the share it was captured with). 1 (default):
 * on; 0: one launch of the tensor-core kernel for every problem. */
int hqr_set_split_launch(int on);

/* hqr_set_priority_policy -- ready-queue priorities of task graphs created
 * afterwards (factorizations, plans, server requests): 1 (default) by the
 * length of the longest chain of estimated task costs that still follows
 * each task (critical path first); 0 panel kernels first, then updates of
 * the next panel's column, then the rest (a look-ahead order; cf. the
 * priority function of Sec. 4.3). */
int hqr_set_priority_policy(int policy);

/* hqr_set_timeout_ms -- time limit of every device-side wait (default 20000). */
void hqr_set_timeout_ms(int64_t ms);

/* hqr_fp64_pipe_rates -- measured FP64 rates of the current GPU (TFLOP/s,
 * a multiply-add counted as 2 flops): DFMA instructions and DMMA
 * (mma.sync m8n8k4 f64) instructions, each from independent register
 * chains in every warp of 4 CTAs per SM (no memory traffic); best of three
 * timed launches after a warm-up. A reference for the FP64 kernels'
 * roofline; the paper has no counterpart. Synchronizes the device. */
int hqr_fp64_pipe_rates(double *dfma_tflops, double *dmma_tflops);

/* hqr_widen_f32 -- y[i] = x[i] widened exactly from FP32 to FP64, i < n, on
 * `stream` (device pointers; asynchronous). The same integer-pipe widening
 * the refinement kernels apply to FP32 matrices (A, R) before their FP64
 * products: the FP32 -> FP64 conversion instruction runs at the FP64 rate
 * on this GPU. Equal bit for bit to the conversion instruction, except that a
 * signalling NaN stays signalling. Returns -1 / -2 for a null x / y with
 * n > 0, -3 for n < 0, HQR_ERR_CUDA if the launch fails. */
int hqr_widen_f32(const float *x, double *y, long long n, void *stream);

/* hqr_strerror -- static text of a status code. */
const char *hqr_strerror(int status);

/* hqr_last_error -- text of the last CUDA error seen by this thread. */
const char *hqr_last_error(void);

/* hqr_last_launch -- kernel launches made by the last factorization or apply
 * call on this thread (for launch accounting). */
int64_t hqr_last_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* HQR_H */
