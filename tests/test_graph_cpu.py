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
WEIGHT = {GEQRT: 4, UNMQR: 6, TSQRT: 6, TSMQR: 12, TTQRT: 2, TTMQR: 6}  # units of b^3 / 3 (Sec. 2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1110_1553_gb300 import _build
    _build.build()
    hqr.load()
    yield
    hqr.set_panel_split(64)
    hqr.set_slab_widths(0, 0, 0)


def accesses(task, nb, ib):
    """(reads, writes) of one task as sets of (row tile, tile column, column, part)."""
    op, blk, i, r, k, j, c0, cw = (int(x) for x in task)
    block = range((blk - 1) * ib, blk * ib) if blk > 0 else range(nb)
    reads, writes = set(), set()
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
    for c in range(c0, c0 + cw):
        if blk > 0:  # a panel block applied to the panel's own trailing columns
            if op == UNMQR:
                writes |= {(i, k, c, "U"), (i, k, c, "L")}
            elif op == TSMQR:
                writes |= {(r, k, c, "U"), (i, k, c, "U"), (i, k, c, "L")}
            else:
                writes |= {(r, k, c, "U"), (i, k, c, "U")}
        else:  # whole target slabs of tile column j
            rows = (i,) if op == UNMQR else (r, i)
            for row in rows:
                writes |= {(row, j, c, "U"), (row, j, c, "L")}
    return reads, writes


def check_no_races(tasks, ptr, succ, nb, ib):
    nt = len(tasks)
    preds = [[] for _ in range(nt)]
    for a in range(nt):
        for b in succ[ptr[a]:ptr[a + 1]]:
            assert b > a, "task ids are not a topological order"
            preds[b].append(a)
    anc = [0] * nt
    last_w, readers = {}, {}
    for t in range(nt):
        m = 0
        for p in preds[t]:
            m |= anc[p] | (1 << p)
        anc[t] = m
        rd, wr = accesses(tasks[t], nb, ib)
        for x in rd | wr:
            w = last_w.get(x)
            assert w is None or (m >> w) & 1, ("unordered with the last writer", t, w, x)
        for x in wr:
            for q in readers.get(x, ()):
                assert q == t or (m >> q) & 1, ("write unordered with an earlier read", t, q, x)
        for x in rd - wr:
            readers.setdefault(x, []).append(t)
        for x in wr:
            last_w[x] = t
            readers[x] = []


@pytest.mark.parametrize("low,high,a,p", [(FLAT, FLAT, 6, 1), (GREEDY, FIBONACCI, 2, 2), (BINARY, GREEDY, 1, 3),
                                          (FIBONACCI, BINARY, 3, 2), (GREEDY, GREEDY, 1, 1)])
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
    for (op, blk, i, r, k, j, c0, cw) in own:
        assert j == k and c0 >= blk * ib and c0 // w == (c0 + cw - 1) // w
    for (op, i, r, k) in {(int(t[0]), int(t[2]), int(t[3]), int(t[4])) for t in blocks}:
        for q in range(1, nq + 1):
            cols = sorted(c for t in own if (t[0], t[2], t[3], t[4], t[1]) == (op + 1, i, r, k, q)
                          for c in range(t[6], t[6] + t[7]))
            assert cols == list(range(q * ib, nb))
    later = lambda g: sorted(tuple(int(x) for x in t) for t in g if t[0] in (UNMQR, TSMQR, TTMQR) and t[1] == 0)
    assert later(whole) == later(split)
