"""CPU tests of the task-graph builder (the Alg. 2 expansion of a list into
tile tasks, and their dependencies), through hqr_task_graph. No device work.

The race check derives every task's reads and writes from what each kernel
touches -- per tile, column and part of the column (rows on and above the
diagonal, "U": R or a TT reflector; rows below it, "L": a GEQRT reflector) --
written here from the kernels' definitions (Sec. 2, Alg. 2), not from the
builder. Any two tasks that touch the same (tile, column, part), at least one
of them writing, must be ordered by a path of the graph."""
import itertools

import numpy as np
import pytest

from oracle.elim_list import BINARY, FIBONACCI, FLAT, GREEDY, hqr_elim_list

hqr = pytest.importorskip("paper_1110_1553_gb300.hqr")

GEQRT, UNMQR, TSQRT, TSMQR, TTQRT, TTMQR = range(6)
RESID, ATR, TRSV_TD, TRSV_TU, TRSV_D, TRSV_U, XUPD, BTOG, PACK, ATRR, TRINV, RESR, RCHK, RGATE, RJOIN = range(6, 21)
WEIGHT = {GEQRT: 4, UNMQR: 6, TSQRT: 6, TSMQR: 12, TTQRT: 2, TTMQR: 6}  # units of b^3 / 3 (Sec. 2)
CHUNK = 8  # tiles per chunk of the residual / A^T r partial sums


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1110_1553_gb300 import _build
    _build.build()
    hqr.load()
    yield
    hqr.set_panel_split(64)
    hqr.set_slab_widths(0, 0, 0)


def tile(row, col, nb):
    """Every (column, part) piece of one tile."""
    return {(row, col, c, part) for c in range(nb) for part in "UL"}


def accesses(task, nb, ib, m=0, n=0):
    """(reads, writes) of one task: tile pieces (row tile, tile column, column, part), right-hand-side
    blocks ("rhs", row, slab) and the least-squares vectors ("x" / "r" / "g" / "inv", tile),
    ("res", row tile, column chunk), ("atr", row chunk, column tile)."""
    op, blk, i, r, k, j, c0, cw, trans, tgt = (int(x) for x in task)
    reads, writes = set(), set()
    if op >= RESID:  # vector tasks of a least-squares graph
        nrc, nch = -(-n // CHUNK), -(-m // CHUNK)
        if op == RESID:  # partial sums of A x over row tile i and column chunk j
            reads = {("x", q) for q in range(j * CHUNK, min(n, (j + 1) * CHUNK))}
            writes = {("res", i, j)}
        elif op == RESR:  # r_i = b_i - sum over the chunks
            reads, writes = {("res", i, c) for c in range(nrc)}, {("r", i)}
        elif op == ATR:  # partial sums of A^T r over row chunk i for column tile j
            reads = {("r", q) for q in range(i * CHUNK, min(m, (i + 1) * CHUNK))}
            writes = {("atr", i, j)}
        elif op == ATRR:
            reads, writes = {("atr", c, j) for c in range(nch)}, {("g", j)}
        elif op == TRINV:  # inverse of the diagonal R tile
            reads, writes = tile(i, i, nb), {("inv", i)}
        elif op in (TRSV_TD, TRSV_D):
            reads, writes = {("inv", i), ("g", i)}, {("g", i)}
        elif op in (TRSV_TU, TRSV_U):  # g_j -= R(i,j)^T g_i (TU) or R(j,i) g_i (U); fused: then X_j
            reads = (tile(i, j, nb) if op == TRSV_TU else tile(j, i, nb)) | {("g", i)}
            if tgt:
                reads.add(("inv", j))
            writes = {("g", j)}
        elif op == XUPD:
            reads, writes = {("g", j)}, {("x", j)}
        elif op == RGATE:  # round k's gate: acts on the stop decisions of the checks up to round k - 2
            reads = {("conv", k - 2)}
        elif op == RJOIN:  # a join of the round's residual rows: no data of its own
            pass
        elif op == RCHK:  # round k's convergence check (tolerance plans): its stop decision ("conv", k)
            reads = {("stat", k), ("cval", k - 1), ("mode", k), ("mode", k + 1), ("conv", k - 1)}
            writes = {("conv", k), ("cval", k), ("mode", k + 2)}
        elif op == BTOG:
            reads, writes = {("rhs", i, 0)}, {("g", i)}
        elif op == PACK:  # tile column j from the caller's matrix; column 0 also b and x = 0
            writes = set().union(*(tile(row, j, nb) for row in range(m)))
            if j == 0:
                writes |= {("rhs", row, 0) for row in range(m)} | {("x", q) for q in range(n)}
        else:
            raise AssertionError("unexpected task %d" % op)
        if trans == 2:  # a round of a tolerance-stopped refinement (round k)
            if op in (RESID, ATR):  # plain or compensated sums, as decided two rounds before
                reads.add(("mode", k))
            if op == XUPD:  # applied only if no earlier round stopped the refinement
                reads.add(("conv", k - 1))
            # every round task also reads the stop flag to skip work, but only x updates and
            # checks act on it in an order that matters: the others write scratch vectors only
        return reads, writes
    block = range((blk - 1) * ib, blk * ib) if blk > 0 else range(nb)
    if op in (GEQRT, TSQRT, TTQRT):  # a panel (or one block of it)
        for c in block:
            if op == GEQRT:
                writes |= {(i, k, c, "U"), (i, k, c, "L")}
            elif op == TSQRT:  # R of the killer, the whole killed tile
                writes |= {(r, k, c, "U"), (i, k, c, "U"), (i, k, c, "L")}
            else:  # R of the killer, the triangle of the killed tile
                writes |= {(r, k, c, "U"), (i, k, c, "U")}
        return reads, writes
    for c in block:  # the reflectors applied
        if op != TTMQR:
            reads.add((i, k, c, "L"))
        if op != UNMQR:
            reads.add((i, k, c, "U"))
    rows = (i,) if op == UNMQR else (r, i)
    if tgt:  # a right-hand-side slab
        writes |= {("rhs", row, j) for row in rows}
        return reads, writes
    for c in range(c0, c0 + cw):
        if blk > 0:  # a panel block applied to the panel's own trailing columns
            if op == UNMQR:
                writes |= {(i, k, c, "U"), (i, k, c, "L")}
            elif op == TSMQR:
                writes |= {(r, k, c, "U"), (i, k, c, "U"), (i, k, c, "L")}
            else:
                writes |= {(r, k, c, "U"), (i, k, c, "U")}
        else:  # whole target slabs of tile column j
            for row in rows:
                writes |= {(row, j, c, "U"), (row, j, c, "L")}
    return reads, writes


def accumulates(task):
    """Commutative accumulations of a task (atomic maxima): x updates of a
    tolerance round fold max |d| and max |x| into that round's statistics."""
    op, k, trans = int(task[0]), int(task[4]), int(task[8])
    return {("stat", k)} if (op == XUPD and trans == 2) else set()


def check_no_races(tasks, ptr, succ, nb, ib, m=0, n=0):
    nt = len(tasks)
    preds = [[] for _ in range(nt)]
    for a in range(nt):
        for b in succ[ptr[a]:ptr[a + 1]]:
            assert b > a, "task ids are not a topological order"
            preds[b].append(a)
    anc = [0] * nt
    last_w, readers, accs = {}, {}, {}
    for t in range(nt):
        before = 0  # bit q set: task q is an ancestor of t
        for p in preds[t]:
            before |= anc[p] | (1 << p)
        anc[t] = before
        rd, wr = accesses(tasks[t], nb, ib, m, n)
        ac = accumulates(tasks[t])
        for x in rd | wr | ac:
            w = last_w.get(x)
            assert w is None or (before >> w) & 1, ("unordered with the last writer", t, w, x)
        for x in wr | ac:
            for q in readers.get(x, ()):
                assert q == t or (before >> q) & 1, ("write unordered with an earlier read", t, q, x)
        for x in rd | wr:  # accumulations commute with each other, not with reads or writes
            for q in accs.get(x, ()):
                assert (before >> q) & 1, ("unordered with an accumulation", t, q, x)
        for x in rd - wr:
            readers.setdefault(x, []).append(t)
        for x in ac:
            accs.setdefault(x, []).append(t)
        for x in wr:
            last_w[x] = t
            readers[x] = []
            accs[x] = []


TREE_CASES = [(FLAT, FLAT, 6, 1), (GREEDY, FIBONACCI, 2, 2), (BINARY, GREEDY, 1, 3), (FIBONACCI, BINARY, 3, 2),
              (GREEDY, GREEDY, 1, 1)]


@pytest.mark.parametrize("low,high,a,p", TREE_CASES)
@pytest.mark.parametrize("nb,ib,split", [(64, 16, 64), (64, 8, 64), (64, 16, 0), (256, 32, 64)])
def test_graph_has_no_races(low, high, a, p, nb, ib, split):
    """nb 64 / ib 8: blocks narrower than the 16-column update slabs."""
    m, n = (6, 3) if nb == 64 else (4, 2)
    recs = hqr_elim_list(m, n, a, p, low, high)
    hqr.set_panel_split(split)
    tasks, ptr, succ = hqr.task_graph(m, n, nb, ib, recs)
    check_no_races(tasks, ptr, succ, nb, ib)


def test_race_check_catches_a_dropped_edge():
    """The check itself: removing one edge between a panel and its update is reported."""
    recs = hqr_elim_list(4, 2, 2, 1, GREEDY, GREEDY)
    hqr.set_panel_split(0)
    tasks, ptr, succ = hqr.task_graph(4, 2, 64, 16, recs)
    a = next(t for t in range(len(tasks)) if tasks[t, 0] == GEQRT)
    kept = [int(b) for b in succ[ptr[a]:ptr[a + 1]] if tasks[b, 0] != UNMQR]
    succ2 = np.concatenate([succ[:ptr[a]], np.array(kept, dtype=np.int32), succ[ptr[a + 1]:]])
    ptr2 = ptr.copy()
    ptr2[a + 1:] -= ptr[a + 1] - ptr[a] - len(kept)
    with pytest.raises(AssertionError):
        check_no_races(tasks, ptr2, succ2, 64, 16)


@pytest.mark.parametrize("low,high", list(itertools.product((FLAT, BINARY, GREEDY, FIBONACCI), repeat=2)))
def test_flop_weights_of_the_expansion(low, high):
    """Whole panels and slab updates: sum of the kernel weights x covered columns / nb is
    6 m n^2 - 2 n^3 (Sec. 2), for every tree pair."""
    m, n, nb = 7, 4, 32
    hqr.set_panel_split(0)
    for a, p in ((1, 1), (2, 2), (m, 1)):
        tasks, _, _ = hqr.task_graph(m, n, nb, 8, hqr_elim_list(m, n, a, p, low, high))
        total = sum(WEIGHT[int(t[0])] * (int(t[7]) / nb if t[0] in (UNMQR, TSMQR, TTMQR) else 1) for t in tasks)
        assert total == pytest.approx(6 * m * n * n - 2 * n ** 3)


@pytest.mark.parametrize("nb,ib", [(64, 16), (64, 8), (256, 32)])
def test_split_panel_structure(nb, ib):
    """A split panel is nb / ib block tasks; block q is followed by update tasks on its own
    tile column that cover exactly the columns [(q + 1) ib, nb), cut at the 16-column update
    slabs; the updates of later tile columns are the same as with whole panels."""
    m, n = 5, 3
    recs = hqr_elim_list(m, n, 2, 2, GREEDY, FIBONACCI)
    hqr.set_panel_split(0)
    whole, _, _ = hqr.task_graph(m, n, nb, ib, recs)
    hqr.set_panel_split(64)
    split, _, _ = hqr.task_graph(m, n, nb, ib, recs)
    nq, w = nb // ib, 16
    panels = [t for t in whole if t[0] in (GEQRT, TSQRT, TTQRT)]
    blocks = [t for t in split if t[0] in (GEQRT, TSQRT, TTQRT)]
    assert all(t[1] == 0 for t in panels) and len(blocks) == nq * len(panels)
    own = [t for t in split if t[0] in (UNMQR, TSMQR, TTMQR) and t[1] > 0]
    for (op, blk, i, r, k, j, c0, cw, _, _) in own:
        assert j == k and c0 >= blk * ib and c0 // w == (c0 + cw - 1) // w
    for (op, i, r, k) in {(int(t[0]), int(t[2]), int(t[3]), int(t[4])) for t in blocks}:
        for q in range(1, nq + 1):
            cols = sorted(c for t in own if (t[0], t[2], t[3], t[4], t[1]) == (op + 1, i, r, k, q)
                          for c in range(t[6], t[6] + t[7]))
            assert cols == list(range(q * ib, nb))
    later = lambda g: sorted(tuple(int(x) for x in t) for t in g if t[0] in (UNMQR, TSMQR, TTMQR) and t[1] == 0)
    assert later(whole) == later(split)


@pytest.mark.parametrize("low,high,a,p", TREE_CASES[:3])
@pytest.mark.parametrize("iters,split,kind", [(0, 64, "ls"), (3, 64, "ls"), (3, 0, "ls"), (2, 64, "request")])
def test_least_squares_graph_has_no_races(low, high, a, p, iters, split, kind):
    """A plan's graph: the factorization, then Q^T b and the triangular solve (iters = 0) or
    CSNE rounds (residual and A^T r partial sums, inverses of the diagonal tiles, fused solve
    steps, x updates); a server request's graph packs the caller's matrix first."""
    m, n, nb, ib = 9, 9, 64, 16
    hqr.set_panel_split(split)
    tasks, ptr, succ = hqr.task_graph(m, n, nb, ib, hqr_elim_list(m, n, a, p, low, high), kind=kind,
                                      param=iters)
    assert ((tasks[:, 0] == PACK).sum() == n) == (kind == "request")
    check_no_races(tasks, ptr, succ, nb, ib, m, n)
    ops = tasks[:, 0]
    assert (ops == XUPD).sum() == n * max(iters, 1)
    if iters:
        assert (ops == RESID).sum() == iters * m * -(-n // CHUNK)
        # one fused solve step per tile pair of the chain (next tile) in each direction
        assert ((ops == TRSV_TU) & (tasks[:, 9] == 1)).sum() == iters * (n - 1)
        assert ((ops == TRSV_U) & (tasks[:, 9] == 1)).sum() == iters * (n - 1)


@pytest.mark.parametrize("low,high,a,p", TREE_CASES[:3])
def test_apply_graphs_replay_the_factorization(low, high, a, p):
    """Q^T and Q on a right-hand side of 3 slabs: no races, and on every slab the updates
    replay the factorization's panels in their order (Q^T) or in reverse (Q), Sec. 5.1."""
    m, n, nb, ib = 7, 4, 64, 16
    recs = hqr_elim_list(m, n, a, p, low, high)
    hqr.set_panel_split(0)
    fac, _, _ = hqr.task_graph(m, n, nb, ib, recs)
    panels = [(int(t[0]) + 1, int(t[2]), int(t[3]), int(t[4])) for t in fac if t[0] in (GEQRT, TSQRT, TTQRT)]
    for kind, trans in (("qt", 1), ("q", 0)):
        tasks, ptr, succ = hqr.task_graph(m, n, nb, ib, recs, kind=kind, param=3)
        check_no_races(tasks, ptr, succ, nb, ib)
        assert (tasks[:, 8] == trans).all() and (tasks[:, 9] == 1).all()
        for slab in range(3):
            seq = [(int(t[0]), int(t[2]), int(t[3]), int(t[4])) for t in tasks if t[5] == slab]
            assert seq == (panels if trans else panels[::-1])


def test_race_check_catches_a_dropped_refinement_edge():
    """The vector-task model: without the edges out of an x update, the next round's residual
    reads x unordered, and the check reports it."""
    m, n, nb, ib = 9, 9, 64, 16
    tasks, ptr, succ = hqr.task_graph(m, n, nb, ib, hqr_elim_list(m, n, 2, 2, GREEDY, FIBONACCI), kind="ls",
                                      param=2)
    check_no_races(tasks, ptr, succ, nb, ib, m, n)
    a = next(t for t in range(len(tasks)) if tasks[t, 0] == XUPD)
    succ2 = np.concatenate([succ[:ptr[a]], succ[ptr[a + 1]:]])
    ptr2 = ptr.copy()
    ptr2[a + 1:] -= ptr[a + 1] - ptr[a]
    with pytest.raises(AssertionError):
        check_no_races(tasks, ptr2, succ2, nb, ib, m, n)


@pytest.mark.parametrize("prec,nb,ib,split", [
    (hqr.FP64, 64, 16, True), (hqr.FP64, 256, 32, True), (hqr.FP64, 32, 8, False),  # FP64 from nb 64
    (hqr.FP32, 128, 16, False), (hqr.FP32, 256, 32, True),  # FP32: only blocks spanning whole slabs
    (hqr.FP32_BF16X3, 128, 128, False),  # tensor-core tiles keep whole panels (one block)
])
def test_panel_split_policy(prec, nb, ib, split):
    recs = hqr_elim_list(3, 2, 2, 1, GREEDY, GREEDY)
    hqr.set_panel_split(64)
    tasks, _, _ = hqr.task_graph(3, 2, nb, ib, recs, prec=prec)
    assert (tasks[:, 1] > 0).any() == split
    hqr.set_panel_split(0)
    tasks, _, _ = hqr.task_graph(3, 2, nb, ib, recs, prec=prec)
    assert not (tasks[:, 1] > 0).any()
    hqr.set_panel_split(64)


def test_task_graph_arguments():
    import ctypes
    lib = hqr.load()
    recs = hqr.to_array(hqr_elim_list(4, 2, 2, 1, GREEDY, GREEDY))
    nt, ne = ctypes.c_int64(0), ctypes.c_int64(0)

    def call(m=4, n=2, nb=64, ib=16, prec=0, lst=recs, kind=0, param=0, tasks=None, cap=0, ptr=None, succ=None,
             scap=0):
        return lib.hqr_task_graph(m, n, nb, ib, prec, lst.ctypes.data if len(lst) else None, len(lst), kind, param,
                                  tasks, cap, ptr, succ, scap, ctypes.byref(nt), ctypes.byref(ne))
    assert call() == 0 and nt.value > 0 and ne.value > 0
    assert call(m=0) == -1 and call(n=5) == -2 and call(nb=12) == -3 and call(ib=5) == -4
    assert call(kind=7) == -8 and call(kind=1, param=0) == -9
    bad = recs.copy()
    bad[0]["killer"] = bad[0]["i"]  # a row cannot kill itself
    assert call(lst=bad) == hqr.ERR_INVALID_LIST
    small = np.zeros((1, 10), dtype=np.int32)
    ptr = np.zeros(2, dtype=np.int64)
    succ = np.zeros(1, dtype=np.int32)
    assert call(tasks=small.ctypes.data, cap=1, ptr=ptr.ctypes.data, succ=succ.ctypes.data, scap=1) == \
        hqr.ERR_CAPACITY


@pytest.mark.parametrize("split", [64, 0])
def test_graph_with_coupling_level_has_no_races(split):
    """Lists with the coupling (domino) level: level-2 TT kills by the domain tops."""
    m, n, nb, ib = 10, 5, 64, 16
    hqr.set_panel_split(split)
    for low, high, a, p in ((GREEDY, FIBONACCI, 2, 3), (FLAT, BINARY, 1, 4)):
        recs = hqr_elim_list(m, n, a, p, low, high, domino=True)
        assert any(r[4] == 2 for r in recs)
        tasks, ptr, succ = hqr.task_graph(m, n, nb, ib, recs)
        check_no_races(tasks, ptr, succ, nb, ib)


@pytest.mark.parametrize("low,high,a,p", TREE_CASES[:3])
@pytest.mark.parametrize("iters,split", [(1, 64), (4, 64), (5, 0)])
def test_tolerance_graph_has_no_races(low, high, a, p, iters, split):
    """A plan from hqr_ls_plan_create_tol: the QR solution as starting point,
    then rounds whose tasks carry trans = 2 and k = the round, one
    convergence check per round after all its x updates, and the next round's
    x updates after that check."""
    m, n, nb, ib = 9, 9, 64, 16
    hqr.set_panel_split(split)
    try:
        tasks, ptr, succ = hqr.task_graph(m, n, nb, ib, hqr_elim_list(m, n, a, p, low, high), kind="ls_tol",
                                          param=iters)
    finally:
        hqr.set_panel_split(64)
    check_no_races(tasks, ptr, succ, nb, ib, m, n)
    ops, ks, trans = tasks[:, 0], tasks[:, 4], tasks[:, 8]
    assert (ops == RCHK).sum() == iters
    assert sorted(ks[ops == RCHK]) == list(range(iters))
    assert sorted(ks[ops == RJOIN]) == list(range(iters))  # one join per round, before its A^T r tasks
    for q in np.nonzero(ops == RJOIN)[0]:  # it releases every A^T r task of its round
        atr = np.nonzero((ops == ATR) & (ks == ks[q]) & (trans == 2))[0]
        assert len(atr) and set(atr.tolist()) <= set(succ[ptr[q]:ptr[q + 1]].tolist())
    rnd = np.isin(ops, [RESID, RESR, ATR, ATRR, TRSV_TD, TRSV_TU, TRSV_D, TRSV_U, XUPD, RCHK, RGATE, RJOIN])
    assert rnd[trans == 2].all()  # only round tasks are marked
    assert (trans[np.isin(ops, [RESID, RESR, ATR, ATRR, RCHK])] == 2).all()
    # the starting point x0 = R^{-1} (Q^T b)[0:N]: Q^T b, its first N entries, one backward solve
    assert (ops == BTOG).sum() == n
    assert ((ops == XUPD) & (trans != 2)).sum() == n and ((ops == XUPD) & (trans == 2)).sum() == iters * n
    # gates of rounds >= 2: after check k - 2 and gate k - 1, before every residual task of round k;
    # j = the number of tasks after the gate, all of rounds >= k and all its descendants
    gidx = np.nonzero(ops == RGATE)[0]
    assert sorted(ks[gidx]) == list(range(2, iters))
    for q in gidx:
        k = ks[q]
        assert tasks[q, 5] == len(tasks) - q - 1
        assert (ks[q + 1:][trans[q + 1:] == 2] >= k).all() and (trans[q + 1:] == 2).all()
        assert q in succ[ptr[int(np.nonzero((ops == RCHK) & (ks == k - 2))[0][0])]:ptr[int(np.nonzero((ops == RCHK) & (ks == k - 2))[0][0]) + 1]]
        for u in np.nonzero((ops == RESID) & (ks == k) & (trans == 2))[0]:
            assert u in succ[ptr[q]:ptr[q + 1]]
        # every later task descends from the gate (a cancelled gate releases nothing, so none of them runs)
        desc = np.zeros(len(tasks), bool)
        desc[q] = True
        for t in range(q, len(tasks)):
            if desc[t]:
                desc[succ[ptr[t]:ptr[t + 1]]] = True
        assert desc[q + 1:].all()
    # every check follows all x updates of its round; every x update of round k + 1 follows check k
    for q in np.nonzero(ops == RCHK)[0]:
        k = ks[q]
        for u in np.nonzero((ops == XUPD) & (ks == k) & (trans == 2))[0]:
            assert q in succ[ptr[u]:ptr[u + 1]]
        for u in np.nonzero((ops == XUPD) & (ks == k + 1) & (trans == 2))[0]:
            assert u in succ[ptr[q]:ptr[q + 1]]


def test_race_check_catches_a_missing_check_edge():
    """Dropping the edge from a round's check to the next round's x update
    must be reported (that x update could apply a correction after the
    tolerance was met)."""
    m, n, nb, ib = 5, 5, 64, 16
    tasks, ptr, succ = hqr.task_graph(m, n, nb, ib, hqr_elim_list(m, n, 2, 2, GREEDY, FIBONACCI), kind="ls_tol",
                                      param=3)
    ops, ks, trans = tasks[:, 0], tasks[:, 4], tasks[:, 8]
    q = int(np.nonzero((ops == RCHK) & (ks == 0))[0][0])
    u = int(np.nonzero((ops == XUPD) & (ks == 1) & (trans == 2))[0][0])
    s2 = list(succ[ptr[q]:ptr[q + 1]])
    s2.remove(u)
    succ2 = np.concatenate([succ[:ptr[q]], np.array(s2, dtype=succ.dtype), succ[ptr[q + 1]:]])
    ptr2 = ptr.copy()
    ptr2[q + 1:] -= 1
    # the x update may still be ordered after the check through another path: only a
    # missing path counts
    with pytest.raises(AssertionError):
        check_no_races(tasks, ptr2, succ2, nb, ib, m, n)


@pytest.mark.parametrize("low,high", [(FLAT, FLAT), (GREEDY, FIBONACCI), (BINARY, GREEDY), (FIBONACCI, BINARY)])
def test_critical_path_model(low, high):
    """hqr_critical_path: with whole panels the work is the Sec. 2 weight sum
    6 m n^2 - 2 n^3 (units of b^3 / 3) for every list; the critical path lies
    between the longest single task and the work."""
    m, n, nb, ib = 12, 5, 64, 16
    hqr.set_panel_split(0)
    try:
        for a, p in ((1, 1), (2, 3), (m, 1)):
            cp, work = hqr.critical_path(m, n, nb, ib, hqr_elim_list(m, n, a, p, low, high))
            assert work == pytest.approx(6 * m * n * n - 2 * n ** 3, rel=1e-12)
            assert 12.0 / 4 <= cp <= work  # a TSMQR slab (16 of 64 columns) is the smallest full task
    finally:
        hqr.set_panel_split(64)


def test_critical_path_orders_trees_on_a_tall_matrix():
    """On a tall-skinny tile matrix the flat tree (one TS domain) has the
    longest critical path and a tree over single tiles a much shorter one
    (Sec. 3: the flat tree's panel is a chain of m - 1 kills)."""
    m, n, nb, ib = 64, 4, 64, 16
    cp_flat, _ = hqr.critical_path(m, n, nb, ib, hqr_elim_list(m, n, m, 1, FLAT, FLAT))
    cp_greedy, _ = hqr.critical_path(m, n, nb, ib, hqr_elim_list(m, n, 1, 1, GREEDY, GREEDY))
    cp_hier, _ = hqr.critical_path(m, n, nb, ib, hqr_elim_list(m, n, 4, 4, GREEDY, FIBONACCI))
    assert cp_greedy < cp_hier < cp_flat
    assert cp_flat > 4 * cp_greedy


@pytest.mark.parametrize("nb,ib", [(16, 4), (32, 8), (64, 16)])
@pytest.mark.parametrize("low,high,a,p,domino", [(FLAT, FLAT, 4, 1, False), (GREEDY, FIBONACCI, 2, 2, False),
                                                 (BINARY, GREEDY, 1, 3, False), (GREEDY, FLAT, 2, 3, True),
                                                 (FIBONACCI, BINARY, 1, 4, True)])
def test_noalloc_graph_has_no_races(nb, ib, low, high, a, p, domino):
    """The allocation-free entry point builds its own task graph in static
    storage (coarser dependency pieces than the main builder: slab, upper and
    lower part per tile); the same independent race check applies to it, for
    TS and TT lists and lists with the coupling level."""
    m, n = 12, 5
    recs = hqr_elim_list(m, n, a, p, low, high, domino=domino)
    tasks, ptr, succ = hqr.task_graph(m, n, nb, ib, recs, kind="noalloc")
    check_no_races(tasks, ptr, succ, nb, ib, m, n)
    # one panel task per op of the expansion and one update per (op, later column, slab)
    S = -(-nb // min(16, nb))
    nops = (tasks[:, 0] % 2 == 0).sum()
    assert len(tasks) == nops + S * sum(n - 1 - t[4] for t in tasks if t[0] % 2 == 0 and t[0] <= 4)


def test_noalloc_graph_limits():
    recs = hqr_elim_list(65, 1, 1, 1, FLAT, FLAT)
    with pytest.raises(hqr.HQRError) as e:
        hqr.task_graph(65, 1, 16, 4, recs, kind="noalloc")
    assert e.value.status == hqr.ERR_TOO_LARGE


@pytest.mark.parametrize("kind", ["ls", "ls_tol"])
def test_fused_solve_steps_lead_their_predecessors_successors(kind):
    """The scheduler lets a CTA keep the first successor (in list order) that a
    finished triangular-solve step makes ready and run it next. Successor
    lists are sorted by decreasing bottom level, and the cost model weights a
    fused step (an update that also applies the next diagonal inverse) twice a
    plain one, so the step that carries each solve chain is listed first among
    the successors of the previous fused step."""
    m = n = 9
    nb, ib = 64, 16
    tasks, ptr, succ = hqr.task_graph(m, n, nb, ib, hqr_elim_list(m, n, 2, 1, GREEDY, FIBONACCI), kind=kind,
                                      param=3)
    ops, ii, jj, tgt = tasks[:, 0], tasks[:, 2], tasks[:, 5], tasks[:, 9]
    checked = 0
    for op in (TRSV_TU, TRSV_U):
        step = 1 if op == TRSV_TU else -1
        fused = np.where((ops == op) & (tgt == 1))[0]
        by_pos = {(int(ii[q]), int(jj[q]), int(q)): q for q in fused}
        for q in fused:
            # the next fused step of the same chain: row i + step, applying the inverse of tile j + step
            nxt = [r for (i, j, r) in by_pos if i == ii[q] + step and j == jj[q] + step and r > q]
            if not nxt:
                continue
            r = min(nxt)  # the same round: the first such step after q
            lst = succ[ptr[q]:ptr[q + 1]]
            assert r in lst, (op, q, r)
            assert lst[0] == r, (op, int(q), int(r), [int(x) for x in lst[:4]])
            checked += 1
    assert checked >= 2 * 3 * (n - 2)  # every round's two chains
