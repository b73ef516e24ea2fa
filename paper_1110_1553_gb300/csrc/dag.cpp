// Host construction of the tile task graphs (Alg. 1 and Alg. 2 expanded into
// tasks with data dependencies). Each task lists the pieces of tile storage
// it reads and writes; an edge is added for every read-after-write,
// write-after-write and write-after-read between tasks taken in the
// sequential order of Alg. 1, so any order the device scheduler picks gives
// the same arithmetic as the sequential algorithm (Sec. 4.2 "Execution
// scheme": tasks fire as soon as their dependencies are met).
#include <algorithm>
#include <stdexcept>

#include "hqr_internal.h"

namespace hqr {

std::vector<PanelOp> expand_ops(const hqr_elim_t *list, size_t count, int m, int n) {
  std::vector<PanelOp> ops;
  const int K = std::min(m, n);
  // records grouped by panel, keeping the list order inside a panel
  std::vector<std::vector<size_t>> by_panel(K);
  for (size_t q = 0; q < count; ++q) by_panel[list[q].k].push_back(q);
  std::vector<int> triangle(m, -1);  // panel in which the row last got GEQRT
  for (int k = 0; k < K; ++k) {
    for (size_t q : by_panel[k]) {
      const hqr_elim_t &e = list[q];
      if (triangle[e.killer] != k) {
        ops.push_back({0, k, e.killer, e.killer});
        triangle[e.killer] = k;
      }
      if (e.kind == HQR_KIND_TT && triangle[e.i] != k) {
        ops.push_back({0, k, e.i, e.i});
        triangle[e.i] = k;
      }
      ops.push_back({(int8_t)(e.kind == HQR_KIND_TS ? 1 : 2), k, e.i, e.killer});
    }
    if (by_panel[k].empty()) ops.push_back({0, k, k, k});
  }
  return ops;
}

namespace {

// Last writer and readers-since-last-write per storage piece.
class Tracker {
 public:
  explicit Tracker(size_t nres) : writer_(nres, -1), readers_(nres) {}
  void read(size_t res, std::vector<int32_t> &deps) {
    if (writer_[res] >= 0) deps.push_back(writer_[res]);
    pending_reads_.push_back(res);
  }
  void write(size_t res, std::vector<int32_t> &deps) {
    if (writer_[res] >= 0) deps.push_back(writer_[res]);
    for (int32_t r : readers_[res]) deps.push_back(r);
    pending_writes_.push_back(res);
  }
  // Record the task's accesses after all its dependencies were collected.
  void commit(int32_t task) {
    for (size_t res : pending_writes_) {
      writer_[res] = task;
      readers_[res].clear();
    }
    for (size_t res : pending_reads_) readers_[res].push_back(task);
    pending_reads_.clear();
    pending_writes_.clear();
  }

 private:
  std::vector<int32_t> writer_;
  std::vector<std::vector<int32_t>> readers_;
  std::vector<size_t> pending_reads_, pending_writes_;
};

class Builder {
 public:
  explicit Builder(size_t nres) : tr_(nres) {}
  Tracker &tr() { return tr_; }
  std::vector<int32_t> &deps() { return deps_; }
  int32_t next_id() const { return (int32_t)g_.tasks.size(); }
  void add(const Task &t) {
    const int32_t id = (int32_t)g_.tasks.size();
    std::sort(deps_.begin(), deps_.end());
    deps_.erase(std::unique(deps_.begin(), deps_.end()), deps_.end());
    for (int32_t d : deps_) edges_.push_back({d, id});
    g_.indeg.push_back((int32_t)deps_.size());
    g_.tasks.push_back(t);
    tr_.commit(id);
    deps_.clear();
  }
  Graph finish() {
    const size_t nt = g_.tasks.size();
    std::vector<int32_t> cnt(nt + 1, 0);
    for (auto &e : edges_) cnt[e.first + 1]++;
    for (size_t q = 0; q < nt; ++q) cnt[q + 1] += cnt[q];
    g_.succ.assign(edges_.size(), 0);
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
    for (auto &e : edges_) g_.succ[fill[e.first]++] = e.second;
    for (size_t q = 0; q < nt; ++q) {
      g_.tasks[q].succ_begin = cnt[q];
      g_.tasks[q].succ_end = cnt[q + 1];
    }
    g_.nedges = (int64_t)edges_.size();
    return std::move(g_);
  }

 private:
  Tracker tr_;
  std::vector<int32_t> deps_;
  std::vector<std::pair<int32_t, int32_t>> edges_;
  Graph g_;
};

Task make_task(int op, int prio, int i, int r, int k, int j, int c0, int cw, int trans, int tgt, int pid) {
  Task t;
  t.op = (int8_t)op;
  t.prio = (int8_t)prio;
  t.trans = (int8_t)trans;
  t.tgt = (int8_t)tgt;
  t.pid = pid;
  t.i = i;
  t.r = r;
  t.k = k;
  t.j = j;
  t.c0 = (int16_t)c0;
  t.cw = (int16_t)cw;
  t.blk = 0;
  t.pad_ = 0;
  t.succ_begin = t.succ_end = 0;
  return t;
}

// Storage pieces of the tile workspace for dependency tracking: for every
// tile (i, j) and column slab s (w columns), its upper part (rows <= column:
// R, or TTQRT's V) and its strict lower part (GEQRT's V). Updates write whole
// slabs; a panel's V and R are parts of all its slabs (or of one block's).
struct TilePieces {
  int m, S;
  size_t count(int n) const { return (size_t)m * n * S * 2; }
  size_t u(int i, int j, int s) const { return (((size_t)j * m + i) * S + s) * 2; }
  size_t l(int i, int j, int s) const { return u(i, j, s) + 1; }
};

// The factorization part of a graph (panels and their updates, Alg. 2).
void add_factor_tasks(Builder &b, const std::vector<PanelOp> &ops, const TilePieces &P, int n, int nb, int w,
                      int pid, int split_ib) {
  Tracker &tr = b.tr();
  std::vector<int32_t> &d = b.deps();
  const int S = P.S;
  const bool split = split_ib > 0;
  const int nq = split ? nb / split_ib : 1;
  auto slab_of = [&](int col) { return col / w; };
  auto wr_u = [&](int i, int j, int s) { tr.write(P.u(i, j, s), d); };
  auto wr_slab = [&](int i, int j, int s) {
    tr.write(P.u(i, j, s), d);
    tr.write(P.l(i, j, s), d);
  };
  for (const PanelOp &o : ops) {
    const int k = o.k, kind = o.kind;
    const int pop = kind == 0 ? OP_GEQRT : (kind == 1 ? OP_TSQRT : OP_TTQRT);
    const int uop = kind == 0 ? OP_UNMQR : (kind == 1 ? OP_TSMQR : OP_TTMQR);
    // what the panel (or its block) writes in slabs [s0, s1) of column k
    auto panel_writes = [&](int s0, int s1) {
      for (int s = s0; s < s1; ++s) {
        if (kind == 0) {
          wr_slab(o.i, k, s);
        } else if (kind == 1) {
          wr_u(o.r, k, s);
          wr_slab(o.i, k, s);
        } else {
          wr_u(o.r, k, s);
          wr_u(o.i, k, s);
        }
      }
    };
    // the reflectors of slabs [s0, s1): GEQRT's V below the diagonal, TSQRT's the whole tile,
    // TTQRT's the upper part
    auto v_reads = [&](int s0, int s1) {
      for (int s = s0; s < s1; ++s) {
        if (kind != 2) tr.read(P.l(o.i, k, s), d);
        if (kind != 0) tr.read(P.u(o.i, k, s), d);
      }
    };
    if (!split) {
      panel_writes(0, S);
      b.add(make_task(pop, 0, o.i, o.r, k, k, 0, nb, 1, 0, pid));
    } else {
      // block q covers columns [q0, q1); its trailing columns [q1, nb) go in pieces no wider than
      // a slab and never across one (slab s0 of a block wider than its block ends the first piece)
      for (int q = 0; q < nq; ++q) {
        const int q0 = q * split_ib, q1 = q0 + split_ib;
        const int s0 = slab_of(q0), s1 = slab_of(q1 - 1) + 1;  // slabs holding block q
        panel_writes(s0, s1);
        Task tp = make_task(pop, 0, o.i, o.r, k, k, q0, split_ib, 1, 0, pid);
        tp.blk = (int16_t)(q + 1);
        b.add(tp);
        for (int c = q1; c < nb;) {  // block q applied to trailing columns [c, ce)
          const int s = slab_of(c), ce = std::min(nb, (s + 1) * w);
          v_reads(s0, s1);
          panel_writes(s, s + 1);
          Task tu = make_task(uop, 0, o.i, o.r, k, k, c, ce - c, 1, 0, pid);
          tu.blk = (int16_t)(q + 1);
          b.add(tu);
          c = ce;
        }
      }
    }
    for (int j = k + 1; j < n; ++j)
      for (int s = 0; s < S; ++s) {
        v_reads(0, S);
        if (kind != 0) wr_slab(o.r, j, s);
        wr_slab(o.i, j, s);
        b.add(make_task(uop, j == k + 1 ? 1 : 2, o.i, o.r, k, j, s * w, std::min(w, nb - s * w), 1, 0, pid));
      }
  }
}

}  // namespace

Graph build_factor_graph(const std::vector<PanelOp> &ops, int m, int n, int nb, int w, int pid, int split_ib) {
  const TilePieces P{m, (nb + w - 1) / w};
  Builder b(P.count(n));
  add_factor_tasks(b, ops, P, n, nb, w, pid, split_ib);
  return b.finish();
}

Graph build_apply_graph(const std::vector<PanelOp> &ops, int m, int nslab, int w, int trans, int pid) {
  // storage pieces: (row tile, column slab) of the right-hand side
  auto piece = [&](int r, int s) { return (size_t)r * nslab + (size_t)s; };
  Builder b((size_t)m * nslab);
  Tracker &tr = b.tr();
  std::vector<int32_t> &d = b.deps();
  const size_t nops = ops.size();
  for (size_t q = 0; q < nops; ++q) {
    const PanelOp &o = trans ? ops[q] : ops[nops - 1 - q];
    for (int s = 0; s < nslab; ++s) {
      if (o.kind == 0) {
        tr.write(piece(o.i, s), d);
        b.add(make_task(OP_UNMQR, 1, o.i, o.i, o.k, s, 0, w, trans, 1, pid));
      } else {
        tr.write(piece(o.r, s), d);
        tr.write(piece(o.i, s), d);
        b.add(make_task(o.kind == 1 ? OP_TSMQR : OP_TTMQR, 1, o.i, o.r, o.k, s, 0, w, trans, 1, pid));
      }
    }
  }
  return b.finish();
}

Graph build_ls_graph(const std::vector<PanelOp> &ops, int m, int n, int nb, int w, int iters, int pid,
                     bool pack, int split_ib, bool tol_mode) {
  const int S = (nb + w - 1) / w;
  const TilePieces P{m, S};
  const size_t ntile_res = P.count(n);
  // vector pieces: x (n tiles), r (m tiles), g (n tiles), rhs block (m tiles)
  auto xres = [&](int j) { return ntile_res + (size_t)j; };
  auto rres = [&](int i) { return ntile_res + (size_t)n + (size_t)i; };
  auto gres = [&](int j) { return ntile_res + (size_t)n + (size_t)m + (size_t)j; };
  auto bres = [&](int i) { return ntile_res + (size_t)2 * n + (size_t)m + (size_t)i; };
  const int nch = atr_chunks(m), nrc = res_chunks(n);
  size_t nres = ntile_res + 2 * (size_t)n + 2 * (size_t)m;
  const size_t pres0 = nres;
  nres += (size_t)nch * n;
  const size_t qres0 = nres;  // residual partial sums (row tile, column chunk)
  nres += (size_t)m * nrc;
  const size_t ires0 = nres;  // inverses of the diagonal R tiles
  nres += (size_t)n;
  const size_t jres = nres++;  // a round's residual join
  auto pres = [&](int c, int j) { return pres0 + (size_t)c * n + (size_t)j; };
  auto qres = [&](int i, int c) { return qres0 + (size_t)i * nrc + (size_t)c; };
  auto ires = [&](int i) { return ires0 + (size_t)i; };
  Builder b(nres);
  Tracker &tr = b.tr();
  std::vector<int32_t> &d = b.deps();
  if (pack) {
    for (int j = 0; j < n; ++j) {
      for (int i = 0; i < m; ++i)
        for (int s = 0; s < S; ++s) {
          tr.write(P.u(i, j, s), d);
          tr.write(P.l(i, j, s), d);
        }
      if (j == 0) {
        for (int i = 0; i < m; ++i) tr.write(bres(i), d);
        for (int jj = 0; jj < n; ++jj) tr.write(xres(jj), d);
      }
      b.add(make_task(OP_PACK, 0, 0, 0, 0, j, 0, 0, 1, 0, pid));
    }
  }
  add_factor_tasks(b, ops, P, n, nb, w, pid, split_ib);
  // R tiles (i, j), j >= i, are final after their last writers
  auto read_r = [&](int i, int j) {
    for (int s = 0; s < S; ++s) {
      tr.read(P.u(i, j, s), d);
      tr.read(P.l(i, j, s), d);
    }
  };
  // tasks of refinement round `round` (-1: not a round task) carry k = round and, with
  // tol_mode, trans = 2 (see the header)
  int round = -1;
  auto rmark = [&](Task t) {
    if (round >= 0) {
      t.k = round;
      if (tol_mode) t.trans = 2;
    }
    return t;
  };
  auto vtask = [&](int op, int i, int j) { return rmark(make_task(op, 1, i, i, 0, j, 0, 0, 1, 0, pid)); };
  int32_t check = -1;  // the previous round's check task (tol_mode)
  std::vector<int32_t> xupd;  // this round's x updates
  bool inverted = false;
  auto solve_r = [&](bool transposed_first) {
    if (!inverted) {  // inverses of the diagonal tiles, once per factorization
      const int rsave = round;
      round = -1;
      for (int i = 0; i < n; ++i) {
        read_r(i, i);
        tr.write(ires(i), d);
        b.add(vtask(OP_TRINV, i, i));
      }
      round = rsave;
      inverted = true;
    }
    // The update of the next diagonal tile's vector is its last writer before the inverse is
    // applied, so that task applies the inverse too (tgt = 1): one task and one hop less per step
    // of the chain. Tile 0 (forward) and n - 1 (backward) have their own inverse task.
    auto ftask = [&](int op, int i, int j, int fused) {
      return rmark(make_task(op, 1, i, i, 0, j, 0, 0, 1, fused, pid));
    };
    if (transposed_first) {  // R^T y = g, forward
      tr.read(ires(0), d);
      tr.write(gres(0), d);
      b.add(vtask(OP_TRSV_TD, 0, 0));
      for (int i = 0; i < n; ++i) {
        for (int j = n - 1; j > i; --j) {  // the next tile's update last, when the others are done
          const int fused = j == i + 1;
          read_r(i, j);
          tr.read(gres(i), d);
          if (fused) tr.read(ires(j), d);
          tr.write(gres(j), d);
          b.add(ftask(OP_TRSV_TU, i, j, fused));
        }
      }
    }
    tr.read(ires(n - 1), d);  // R d = y, backward
    tr.write(gres(n - 1), d);
    b.add(vtask(OP_TRSV_D, n - 1, n - 1));
    for (int i = n - 1; i >= 0; --i) {
      for (int j = 0; j < i; ++j) {
        const int fused = j == i - 1;
        read_r(j, i);
        tr.read(gres(i), d);
        if (fused) tr.read(ires(j), d);
        tr.write(gres(j), d);
        b.add(ftask(OP_TRSV_U, i, j, fused));
      }
    }
    xupd.clear();
    for (int j = 0; j < n; ++j) {
      tr.read(gres(j), d);
      tr.write(xres(j), d);
      if (tol_mode && check >= 0) d.push_back(check);  // applied only if no earlier round met the tolerance
      xupd.push_back(b.next_id());
      b.add(vtask(OP_XUPD, j, j));
    }
    if (tol_mode && round >= 0) {  // the round's check, after all its x updates
      for (int32_t u : xupd) d.push_back(u);
      if (check >= 0) d.push_back(check);
      check = b.next_id();
      b.add(vtask(OP_RCHK, 0, 0));
    }
  };
  if (iters == 0 || tol_mode) {
    // Q^T b on the right-hand-side block, replaying the factorization forward (with tol_mode:
    // the starting point x0 = R^{-1} (Q^T b)[0:N] of the refinement, in place of x0 = 0)
    for (const PanelOp &o : ops) {
      if (o.kind == 0) {
        for (int s = 0; s < S; ++s) tr.read(P.l(o.i, o.k, s), d);
        tr.write(bres(o.i), d);
        b.add(make_task(OP_UNMQR, 1, o.i, o.i, o.k, 0, 0, 1, 1, 1, pid));
      } else {
        for (int s = 0; s < S; ++s) {
          tr.read(P.u(o.i, o.k, s), d);
          if (o.kind == 1) tr.read(P.l(o.i, o.k, s), d);
        }
        tr.write(bres(o.r), d);
        tr.write(bres(o.i), d);
        b.add(make_task(o.kind == 1 ? OP_TSMQR : OP_TTMQR, 1, o.i, o.r, o.k, 0, 0, 1, 1, 1, pid));
      }
    }
    for (int i = 0; i < n; ++i) {
      tr.read(bres(i), d);
      tr.write(gres(i), d);
      b.add(vtask(OP_BTOG, i, i));
    }
    solve_r(false);
  }
  // Residuals and A^T r of the last rounds are compensated (Dot2); the earlier rounds, whose
  // corrections are still far above the FP64 rounding level, use plain FP64 sums (1 FMA per
  // element instead of ~10 FP64 operations). Vector tasks carry the choice in `tgt`.
  const int ncomp = std::min(iters, std::max(4, (2 * iters + 4) / 5));
  std::vector<int32_t> checks, gates;  // tol_mode: each round's check; the gates (ids)
  int32_t gate = -1;
  for (int it = 0; it < iters; ++it) {
    round = it;
    const int comp = (!tol_mode && it >= iters - ncomp) ? 1 : 0;
    auto rtask = [&](int op, int i, int j) { return rmark(make_task(op, 1, i, i, 0, j, 0, 0, 1, comp, pid)); };
    if (tol_mode && it >= 2) {  // the round's gate: after check it - 2 and the previous gate
      d.push_back(checks[it - 2]);
      if (gate >= 0) d.push_back(gate);
      gate = b.next_id();
      gates.push_back(gate);
      b.add(vtask(OP_RGATE, 0, 0));
    }
    for (int i = 0; i < m; ++i) {
      for (int c = 0; c < nrc; ++c) {
        for (int j = c * kResChunk; j < std::min(n, (c + 1) * kResChunk); ++j) tr.read(xres(j), d);
        tr.write(qres(i, c), d);
        if (tol_mode && it >= 2) d.push_back(gate);
        b.add(rtask(OP_RESID, i, c));
      }
      for (int c = 0; c < nrc; ++c) tr.read(qres(i, c), d);
      tr.write(rres(i), d);
      b.add(vtask(OP_RESR, i, i));
    }
    // The round's join, after every residual row: its release hands out all A^T r tasks at once in
    // decreasing bottom level (the row chunks of column tile 0 first, which the forward solve
    // needs first), where each row chunk's last residual would release them chunk by chunk and
    // column tile 0 would be complete only at the end.
    for (int i = 0; i < m; ++i) tr.read(rres(i), d);
    tr.write(jres, d);
    b.add(vtask(OP_RJOIN, 0, 0));
    for (int j = 0; j < n; ++j) {
      for (int c = 0; c < nch; ++c) {
        for (int i = c * kAtrChunk; i < std::min(m, (c + 1) * kAtrChunk); ++i) tr.read(rres(i), d);
        tr.read(jres, d);
        tr.write(pres(c, j), d);
        b.add(rtask(OP_ATR, c, j));
      }
      for (int c = 0; c < nch; ++c) tr.read(pres(c, j), d);
      tr.write(gres(j), d);
      b.add(vtask(OP_ATRR, j, j));
    }
    solve_r(true);
    if (tol_mode) checks.push_back(check);
  }
  Graph g = b.finish();
  for (int32_t q : gates) g.tasks[q].j = (int32_t)g.tasks.size() - q - 1;  // tasks after the gate
  return g;
}

// Estimated cost of a task in units of b^3/3 (Sec. 2 weights), updates scaled by slab width;
// the FP64 vector tasks of least-squares graphs by their relative durations (a compensated
// residual or A^T r chunk costs about a GEQRT, a plain one a fifth of it, a triangular-solve
// step a few percent, twice that when it also applies the next diagonal inverse), so that the
// solve chains keep their place ahead of the next round's residuals and the step that carries
// the chain is its predecessor's most critical successor.
static double task_cost(const Task &t, int nb) {
  const double slab = t.cw > 0 ? (double)t.cw / nb : 1.0;
  // a block task of a split panel: about one block's share of its panel (or of one update slab)
  const double part = t.blk > 0 ? 0.125 : 1.0;
  switch (t.op) {
    case OP_GEQRT: return 4.0 * part;
    case OP_TSQRT: return 6.0 * part;
    case OP_TTQRT: return 2.0 * part;
    case OP_UNMQR: return 6.0 * slab * part;
    case OP_TSMQR: return 12.0 * slab * part;
    case OP_TTMQR: return 6.0 * slab * part;
    case OP_RESID:
    case OP_ATR: return t.tgt ? 3.5 : 0.7;
    case OP_TRINV: return 12.0;
    case OP_TRSV_TD:
    case OP_TRSV_TU:
    case OP_TRSV_D:
    case OP_TRSV_U: return t.tgt ? 0.4 : 0.2;  // a fused step also applies the next inverse
    default: return 0.1;
  }
}

// Bottom level of every task: its cost plus the longest chain of costs after it.
static std::vector<double> bottom_levels(const Graph &g, int nb) {
  const size_t nt = g.tasks.size();
  std::vector<double> bl(nt, 0.0);
  for (size_t q = nt; q-- > 0;) {  // tasks are in a topological order
    double best = 0.0;
    for (int32_t e = g.tasks[q].succ_begin; e < g.tasks[q].succ_end; ++e) best = std::max(best, bl[g.succ[e]]);
    bl[q] = task_cost(g.tasks[q], nb) + best;
  }
  return bl;
}

double critical_path_length(const Graph &g, int nb) {
  double cp = 0.0;
  for (double v : bottom_levels(g, nb)) cp = std::max(cp, v);
  return cp;
}

double total_cost(const Graph &g, int nb) {
  double w = 0.0;
  for (const Task &t : g.tasks) w += task_cost(t, nb);
  return w;
}

void critical_path_priorities(Graph &g, int nb) {
  const size_t nt = g.tasks.size();
  if (nt == 0) return;
  const std::vector<double> bl = bottom_levels(g, nb);
  // successors in decreasing bottom level: the most critical ones are released first
  for (size_t q = 0; q < nt; ++q) {
    const Task &t = g.tasks[q];
    std::stable_sort(g.succ.begin() + t.succ_begin, g.succ.begin() + t.succ_end,
                     [&](int32_t a, int32_t b) { return bl[a] > bl[b]; });
  }
  std::vector<double> sorted(bl);
  std::sort(sorted.begin(), sorted.end());
  double cut[kNumQueues];
  for (int c = 0; c < kNumQueues; ++c) cut[c] = sorted[(size_t)((double)(kNumQueues - 1 - c) / kNumQueues * (nt - 1))];
  for (size_t q = 0; q < nt; ++q) {
    int c = kNumQueues - 1;
    while (c > 0 && bl[q] >= cut[c - 1]) --c;
    g.tasks[q].prio = (int8_t)c;
  }
}

void append_graph(Graph &into, const Graph &g) {
  const int32_t toff = (int32_t)into.tasks.size();
  const int32_t eoff = (int32_t)into.succ.size();
  for (Task t : g.tasks) {
    t.succ_begin += eoff;
    t.succ_end += eoff;
    into.tasks.push_back(t);
  }
  for (int32_t s : g.succ) into.succ.push_back(s + toff);
  into.indeg.insert(into.indeg.end(), g.indeg.begin(), g.indeg.end());
  into.nedges += g.nedges;
}

}  // namespace hqr
