// Internal declarations shared by the host task-graph builder and the CUDA
// engine. Not part of the public ABI.
#pragma once

#include <cstdint>
#include <vector>

#include "../../include/hqr.h"

namespace hqr {

// Tile task opcodes (Alg. 2). The update opcodes also serve Q / Q^T
// application to a right-hand side (Sec. 5.1).
enum Op : int8_t {
  OP_GEQRT = 0,
  OP_UNMQR = 1,
  OP_TSQRT = 2,
  OP_TSMQR = 3,
  OP_TTQRT = 4,
  OP_TTMQR = 5,
  // FP64 vector tasks of least-squares solves (per tile of the vectors)
  OP_RESID = 6,    // partial sums of A(i, column chunk j) x, compensated (row tile i)
  OP_ATR = 7,      // partial sums of A(rows of chunk i, j)^T r, compensated (column tile j, row chunk i)
  OP_TRSV_TD = 8,  // g_i <- R_ii^{-T} g_i (with the inverse from OP_TRINV)
  OP_TRSV_TU = 9,  // g_j -= R(i,j)^T g_i, j > i
  OP_TRSV_D = 10,  // g_i <- R_ii^{-1} g_i (with the inverse from OP_TRINV)
  OP_TRSV_U = 11,  // g_j -= R(j,i) g_i, j < i
  OP_XUPD = 12,    // x_j += g_j
  OP_BTOG = 13,    // g_i = first column of the right-hand-side block of row tile i
  OP_PACK = 14,    // tile column j of the workspace from the caller's matrix (j = 0 also b, x = 0)
  OP_ATRR = 15,    // g_j = sum over row chunks of the OP_ATR partial sums
  OP_TRINV = 16,   // inverse of the diagonal R tile i (FP64), used by OP_TRSV_TD / OP_TRSV_D
  OP_RESR = 17,    // r_i = b_i - sum over column chunks of the OP_RESID partial sums
  OP_RCHK = 18,    // convergence check of one refinement round (tolerance-stopped plans)
  OP_RGATE = 19,   // gate of refinement round k >= 2 (tolerance-stopped plans): cancels rounds >= k
  OP_RJOIN = 20,   // join of a round's residual rows before its A^T r tasks (no work)
};

// Refinement rounds of a least-squares graph at most.
constexpr int kMaxRounds = 64;

// Per-problem state of a tolerance-stopped refinement (device memory, zeroed
// before every run). Round r's x-update task of tile j leaves sum d_i^2 and
// sum x_i^2 over its tile in a per-problem array (two doubles per tile);
// round r's check task (after all of them) adds them up in tile order into
// cval[r] = ||d||_2 / ||x||_2, decides whether round r + 2 computes its
// residuals compensated, and whether to stop: at the first compensated round
// with cval <= tol (met = 1), or at a compensated round that no longer
// shrinks the correction (cval > 0.9 cval of the compensated round before:
// the attainable accuracy of the low-precision R is reached, met = 0). The
// tasks of the rounds after the stop do nothing.
struct RefineState {
  double cval[kMaxRounds];  // ||d||_2 / ||x||_2 of round r
  int mode[kMaxRounds];     // 1: round r's residual and A^T r compensated (Dot2)
  int conv;                 // rounds applied when the refinement stopped (0: running)
  int met;                  // 1: it stopped because the tolerance was met
  unsigned sing;            // ~c for the first column c with a zero diagonal entry of R (0: none)
  int pad_;
};
static_assert(sizeof(RefineState) % 8 == 0, "RefineState layout");

// Row tiles per chunk of the A^T r partial sums, column tiles per chunk of
// the residual partial sums.
constexpr int kAtrChunk = 8;
constexpr int kResChunk = 8;
inline int atr_chunks(int m) { return (m + kAtrChunk - 1) / kAtrChunk; }
inline int res_chunks(int n) { return (n + kResChunk - 1) / kResChunk; }

// Scheduling classes, highest first: panel kernels (on the critical path),
// updates of the next panel's column (look-ahead), other updates.
constexpr int kNumQueues = 4;

// One task of the device task graph. For update tasks, columns
// [c0, c0 + cw) of the target tiles are updated (a column slab).
struct Task {
  int8_t op;
  int8_t prio;
  int8_t trans;   // apply Q^T (1) or Q (0); factorization tasks use 1
  int8_t tgt;     // update target: 0 = tiles of the matrix, 1 = right-hand-side blocks
  int32_t i;      // killed row (TS/TT), or the row of GEQRT/UNMQR
  int32_t r;      // killer row (TS/TT); equals i for GEQRT/UNMQR
  int32_t k;      // panel
  int32_t j;      // target tile column (updates) or right-hand-side block
  int16_t c0;     // first column of the slab inside the target block
  int16_t cw;     // slab width
  int16_t blk;    // 0: every ib block of the panel; q + 1: only block q (a panel split into block
                  // tasks: the panel task factors block q, an update task on the panel's own
                  // tiles applies block q to the trailing slab [c0, c0 + cw))
  int16_t pad_;
  int32_t pid;    // problem index (several problems can share one graph)
  int32_t succ_begin, succ_end;  // successor range in the CSR array
};
static_assert(sizeof(Task) == 40, "Task layout");

// A task graph ready for upload: tasks in a topological order, successor
// lists (CSR), in-degrees and per-queue initial ready lists.
struct Graph {
  std::vector<Task> tasks;
  std::vector<int32_t> succ;
  std::vector<int32_t> indeg;
  int64_t nedges = 0;
};

// One step of the factorization in execution order, replayed by apply-Q.
struct PanelOp {
  int8_t kind;  // 0 geqrt(row i), 1 ts(i, r), 2 tt(i, r)
  int32_t k, i, r;
};

// Operation sequence of Alg. 1/Alg. 2 for a validated list, one panel after
// the other: a GEQRT the first time a row acts as a triangle in a panel, then
// the TS or TT elimination. A panel without eliminations gets GEQRT(k, k).
std::vector<PanelOp> expand_ops(const hqr_elim_t *list, size_t count, int m, int n);

// Factorization graph: every op expanded into its panel task and its update
// tasks over the tile columns j > k, each split into column slabs of width w.
// With split_ib > 0 (dividing nb) every panel becomes nb /
// split_ib block tasks, block q followed by the updates of the panel's own
// trailing slabs with block q, so that a panel's trailing work spreads over
// several CTAs and the next block starts as soon as its own slabs are done.
Graph build_factor_graph(const std::vector<PanelOp> &ops, int m, int n, int nb, int w, int pid = 0,
                         int split_ib = 0);

// Q^T (trans = 1) or Q (trans = 0) applied to a right-hand side split into
// row tiles and `nslab` column slabs of width w: the update kernels replayed
// forward or backwards.
Graph build_apply_graph(const std::vector<PanelOp> &ops, int m, int nslab, int w, int trans, int pid = 0);

// Least-squares task graph for one problem of m x n tiles (tile size nb, true
// column count N): the factorization, then either `iters` rounds of
// corrected semi-normal equations (x0 = 0; r = b - A x, g = A^T r,
// R^T R d = g, x += d; all FP64) or, with iters = 0, Q^T b applied to the
// right-hand-side block followed by R x = (Q^T b)[0:N].
// With `pack`, the graph starts with one OP_PACK task per tile column that
// copies the caller's matrix into the workspace (for runs where no separate
// preparation kernel can be launched).
//
// With tol_mode, the refinement starts from the QR solution x0 = R^{-1}
// (Q^T b)[0:N] (the iters = 0 tasks, in the storage precision), `iters` is
// the largest number of rounds and the rounds stop at a tolerance: every
// task of round r (residual, A^T r, solve steps, x
// update) carries trans = 2 and k = r; round r ends with an OP_RCHK task after
// all its x updates, and round r + 1's x updates follow that check, so a round
// whose check found the tolerance met leaves x as it was (its other tasks may
// still run on scratch vectors: harmless). Which rounds compensate their
// residuals is decided at run time (RefineState::mode), not by `tgt`. Every
// round r >= 2 starts with an OP_RGATE task (after check r - 2 and gate
// r - 1; before the round's residual tasks, which every other task of the
// round and of later rounds follows); its `j` holds the number of tasks
// after it in the graph (rounds >= r). A gate that finds the refinement
// stopped at round r - 2 or earlier releases no successor and counts those
// tasks as done, so the cancelled rounds cost nothing.
Graph build_ls_graph(const std::vector<PanelOp> &ops, int m, int n, int nb, int w, int iters, int pid,
                     bool pack = false, int split_ib = 0, bool tol_mode = false);

// Priorities from the critical path: every task gets its bottom level (its
// own estimated cost plus the longest chain of estimated costs after it)
// and the queue 0 (longest remaining chain) .. kNumQueues-1 of its quantile.
// Replaces the default classes (panel kernels, next-column updates, rest).
void critical_path_priorities(Graph &g, int nb);

// Longest chain of estimated task costs (units of b^3 / 3, Sec. 2 weights) of
// a graph, and the sum of all its task costs: a unit-cost model of the time
// on unbounded and on one processor.
double critical_path_length(const Graph &g, int nb);
double total_cost(const Graph &g, int nb);

// Append graph g to `into` (its task ids and successor lists renumbered);
// the two graphs stay independent.
void append_graph(Graph &into, const Graph &g);

}  // namespace hqr
