"""Oracle: HQR elimination-list generator and the list validity rules.

Test infrastructure only (see the package docstring). Integer work, plain
Python, written to be checked against the paper by eye.

A record is ``(k, i, killer, kind, level, step)``:

* ``k``      -- panel (tile column) index;
* ``i``      -- the tile row that is zeroed ("killed") in panel k;
* ``killer`` -- the tile row that kills it; ``elim(i, killer, k)`` of Sec. 2
                (the paper writes elim(killed, killer, panel) in Sec. 2 and
                Sec. 4.2; the killer-first order used in Sec. 3.1 is read as
                the same operation);
* ``kind``   -- 0 = TS (a triangle kills a square), 1 = TT (a triangle kills a
                triangle), Sec. 2 and Alg. 2;
* ``level``  -- 0 = TS level, 1 = low level (intra-domain tree), 2 = coupling
                level ("domino", only when asked for), 3 = high level (tree
                over the p virtual domains), Sec. 4.1-4.2;
* ``step``   -- the time step of the coarse unit-time model of Sec. 3.1-3.2
                (every elimination takes one time unit).

Hierarchy (Sec. 4.1, Sec. 4.2; where the paper is silent, the reading taken
is stated with the rule):

* tile row i belongs to virtual domain ``i mod p`` (cyclic distribution);
* in panel k the active rows of a domain are its rows ``>= k``, ascending, and
  its top is the first of them;
* TS level: counting from the domain's top, every a-th active row is a head
  that kills, with TS kernels and in ascending order, the a-1 rows below it;
* low level: a TT reduction tree of the chosen shape over the heads of the
  domain, whose survivor is the domain's top;
* high level: a TT reduction tree of the chosen shape over the tops of all
  domains, whose survivor is row k.

With the coupling level (Sec. 4.2, "Working out an example"): levels 0 and 1
of domain c reduce only its rows on and below its local diagonal, the row of
local index k (global row k p + c), to that row; level 2 then kills the rows
between the top (excluded) and the local diagonal (included) with the top as
killer, in ascending order, TT kernels; level 3 is unchanged.

Tree shapes over an ordered leaf list x0 < x1 < ... (survivor x0):

* FLAT (Sec. 3.1, Table 1): x0 kills x1, x2, ... in order;
* BINARY (Sec. 3.1): at round l, x_j kills x_{j+2^l} for j = 0 mod 2^(l+1);
* GREEDY (Sec. 3.2, Table 4): at each time step, of the z' leaves that are
  alive and ready, the bottom floor(z'/2) are killed by the floor(z'/2) leaves
  right above them, paired in natural order;
* FIBONACCI (Modi-Clarke order-1 scheme, named in Sec. 3.3 but not defined in
  the paper): x is the least integer with x(x+1)/2 >= R-1; the leaves x1 ...
  x_{R-1} are cut from the top into consecutive groups of 1, 2, 3, ... leaves
  (the bottom group truncated); group g is killed at planned step x-g+1 by as
  many leaves as it holds, taken right above it, paired in natural order.

Steps: ``busy[r]`` is the step of the last elimination row r took part in.
A fixed-shape tree's eliminations are visited in the tree's order and get
``step = max(busy[i], busy[killer]) + 1``. GREEDY runs the time loop itself and
the step is the loop time. Levels are processed in the order 0, 1, 2, 3 and the
records of a panel are sorted by (step, i).
"""

FLAT, BINARY, GREEDY, FIBONACCI = 0, 1, 2, 3
TS, TT = 0, 1
TREE_NAMES = {FLAT: "flat", BINARY: "binary", GREEDY: "greedy", FIBONACCI: "fibonacci"}


def flat_pairs(leaves):
    """FLAT tree (Sec. 3.1, Table 1): the first leaf kills every other one, top
    to bottom. Returns (killed, killer) pairs in the order they happen."""
    return [(x, leaves[0]) for x in leaves[1:]]


def binary_pairs(leaves):
    """BINARY tree (Sec. 3.1): rounds l = 0, 1, ...; at round l leaf j kills
    leaf j + 2^l for every j that is a multiple of 2^(l+1)."""
    R = len(leaves)
    pairs = []
    d = 1
    while d < R:
        for j in range(0, R, 2 * d):
            if j + d < R:
                pairs.append((leaves[j + d], leaves[j]))
        d *= 2
    return pairs


def fibonacci_pairs(leaves):
    """FIBONACCI (Modi-Clarke order-1) tree, in order of planned step.

    Let x be the least integer with x(x+1)/2 >= R-1. Positions 1..R-1 are cut
    into consecutive groups of nominal sizes 1, 2, 3, ... from the top; the last
    group holds what is left. A group of s leaves that starts at position q is
    killed by the s leaves at positions q-s .. q-1, pairing in natural order,
    at planned step x-g+1. Returned bottom group first (planned step 1)."""
    R = len(leaves)
    if R <= 1:
        return []
    x = 0
    while x * (x + 1) // 2 < R - 1:
        x += 1
    groups = []
    start, g = 1, 1
    while start < R:
        end = min(start + g, R)
        groups.append((g, start, end))
        start, g = end, g + 1
    pairs = []
    for g, start, end in sorted(groups, key=lambda t: x - t[0] + 1):
        s = end - start
        for t in range(s):
            pairs.append((leaves[start + t], leaves[start - s + t]))
    return pairs


def greedy_pairs(leaves, busy):
    """GREEDY (Sec. 3.2, Table 4) with readiness.

    At time t the candidates are the leaves still alive whose busy step is
    < t, ascending. With z' candidates, the bottom z = floor(z'/2) are killed
    at step t by the z candidates right above them (first with first). Every
    row involved becomes busy until t. Runs until one leaf is left. Updates
    ``busy`` in place and returns (killed, killer, step) triples."""
    alive = list(leaves)
    out = []
    if len(alive) <= 1:
        return out
    t = min(busy[r] for r in alive) + 1
    while len(alive) > 1:
        cand = [r for r in alive if busy[r] < t]
        z = len(cand) // 2
        if z > 0:
            killed = cand[len(cand) - z:]
            killers = cand[len(cand) - 2 * z:len(cand) - z]
            for kd, kr in zip(killed, killers):
                out.append((kd, kr, t))
                busy[kd] = t
                busy[kr] = t
            gone = set(killed)
            alive = [r for r in alive if r not in gone]
        t += 1
    return out


def _tree(tree, leaves, busy):
    """Eliminations of one reduction tree over ``leaves`` as
    (killed, killer, step) triples, updating ``busy``."""
    if tree == GREEDY:
        return greedy_pairs(leaves, busy)
    if tree == FLAT:
        pairs = flat_pairs(leaves)
    elif tree == BINARY:
        pairs = binary_pairs(leaves)
    elif tree == FIBONACCI:
        pairs = fibonacci_pairs(leaves)
    else:
        raise ValueError("unknown tree %r" % (tree,))
    out = []
    for kd, kr in pairs:
        step = max(busy[kd], busy[kr]) + 1
        busy[kd] = step
        busy[kr] = step
        out.append((kd, kr, step))
    return out


def hqr_elim_list(m, n, a, p, low, high, domino=False):
    """Elimination list of HQR for an m x n tile matrix (m >= n), TS domains of
    a tiles, p virtual domains, low-level tree ``low`` and high-level tree
    ``high`` (Sec. 4.1-4.2), with the coupling level if ``domino``. Returns
    records (k, i, killer, kind, level, step) sorted by (k, step, i)."""
    if m < 1 or n < 1 or m < n:
        raise ValueError("need m >= n >= 1")
    if a < 1 or p < 1:
        raise ValueError("need a >= 1 and p >= 1")
    busy = [0] * m
    records = []
    for k in range(min(m, n)):
        panel = []
        tops = []
        for c in range(p):
            rows = [i for i in range(k, m) if i % p == c]
            if not rows:
                continue
            top = rows[0]
            # the local reduction starts at the local diagonal (local index k) with the
            # coupling level, at the top without it
            diag = k * p + c if domino else top
            local = [i for i in rows if i >= diag]
            coupled = [i for i in rows if top < i < diag]
            if local and local[0] != top:
                coupled.append(local[0])
            heads = local[::a]
            # level 0: each head kills the a-1 rows below it with TS kernels
            for h in range(0, len(local), a):
                head = local[h]
                for i in local[h + 1:h + a]:
                    step = max(busy[i], busy[head]) + 1
                    busy[i] = step
                    busy[head] = step
                    panel.append((k, i, head, TS, 0, step))
            # level 1: tree over the heads; survivor = the local diagonal (the top
            # without the coupling level)
            for kd, kr, step in _tree(low, heads, busy):
                panel.append((k, kd, kr, TT, 1, step))
            # level 2 (domino): the top kills the coupled rows one after the other
            for i in coupled:
                step = max(busy[i], busy[top]) + 1
                busy[i] = step
                busy[top] = step
                panel.append((k, i, top, TT, 2, step))
            tops.append(top)
        tops.sort()
        # level 3: tree over the domain tops; survivor = row k
        for kd, kr, step in _tree(high, tops, busy):
            panel.append((k, kd, kr, TT, 3, step))
        panel.sort(key=lambda r: (r[5], r[1]))
        records.extend(panel)
    return records


def validate(records, m, n):
    """Validity rules of Sec. 2 for an elimination list, plus the tile-state
    rule of Sec. 2 that only a square tile may be killed by a TS kernel.
    Returns None when the list is valid, else a message naming the first
    broken rule."""
    seen = {}
    for pos, (k, i, killer, kind, level, step) in enumerate(records):
        if not (0 <= k < min(m, n)):
            return "record %d: panel %d out of range" % (pos, k)
        if not (k < i < m):
            return "record %d: killed row %d not below the diagonal of panel %d" % (pos, i, k)
        if not (k <= killer < m) or killer == i:
            return "record %d: bad killer %d" % (pos, killer)
        if (i, k) in seen:
            return "record %d: tile (%d,%d) killed twice" % (pos, i, k)
        seen[(i, k)] = pos
    for k in range(min(m, n)):
        for i in range(k + 1, m):
            if (i, k) not in seen:
                return "tile (%d,%d) never killed" % (i, k)
    pos_of = seen
    for pos, (k, i, killer, kind, level, step) in enumerate(records):
        for kp in range(k):
            for r in (i, killer):
                if r > kp and pos_of[(r, kp)] > pos:
                    return "record %d: row %d not ready (panel %d later)" % (pos, r, kp)
        if killer > k and pos_of[(killer, k)] < pos:
            return "record %d: killer %d already zeroed in panel %d" % (pos, killer, k)
    # tile states: a TS kill needs a square victim (never a killer before)
    for k in range(min(m, n)):
        was_killer = set()
        for pos, (kk, i, killer, kind, level, step) in enumerate(records):
            if kk != k:
                continue
            if kind == TS and i in was_killer:
                return "record %d: TS kill of a triangle (row %d)" % (pos, i)
            was_killer.add(killer)
    # a TS-killed row may not kill afterwards (it is zero)
    for k in range(min(m, n)):
        ts_dead = set()
        for pos, (kk, i, killer, kind, level, step) in enumerate(records):
            if kk != k:
                continue
            if killer in ts_dead:
                return "record %d: killer %d is already zero" % (pos, killer)
            if kind == TS:
                ts_dead.add(i)
    return None


# weights in units of b^3/3 (Sec. 2)
W_GEQRT, W_UNMQR, W_TSQRT, W_TSMQR, W_TTQRT, W_TTMQR = 4, 6, 6, 12, 2, 6


def triangle_rows(records, k, m, n):
    """Rows that are triangles in panel k (they get a GEQRT, Alg. 2): every
    killer and every TT-killed row; with no elimination at all, row k."""
    rows = set()
    for (kk, i, killer, kind, level, step) in records:
        if kk != k:
            continue
        rows.add(killer)
        if kind == TT:
            rows.add(i)
    if not rows:
        rows.add(k)
    return rows


def total_weight(records, m, n):
    """Sum of the task weights of Alg. 2 for the list, in units of b^3/3."""
    w = 0
    for k in range(min(m, n)):
        c = n - k - 1
        w += len(triangle_rows(records, k, m, n)) * (W_GEQRT + c * W_UNMQR)
        for (kk, i, killer, kind, level, step) in records:
            if kk != k:
                continue
            if kind == TS:
                w += W_TSQRT + c * W_TSMQR
            else:
                w += W_TTQRT + c * W_TTMQR
    return w
