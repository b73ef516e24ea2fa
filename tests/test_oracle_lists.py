"""Pins for the oracle's elimination-list generator (not the CUDA library).

Pinned against: the worked tables of Sec. 3.1-3.2 (fixtures under
tests/golden/), a hand-worked Fibonacci tree, the validity rules of Sec. 2
checked by brute force over every small shape, and the constant total weight
6mn^2 - 2n^3 of Sec. 2.
"""
import itertools
import os

import pytest

from oracle.elim_list import (BINARY, FIBONACCI, FLAT, GREEDY, TS, TT, fibonacci_pairs,
                              hqr_elim_list, total_weight, validate, triangle_rows)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TREES = (FLAT, BINARY, GREEDY, FIBONACCI)


def load_table(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].split()
            if not line:
                continue
            r = int(line[0])
            cols = line[1:]
            rows[r] = [(None if cols[2 * q] == "-" else int(cols[2 * q]),
                        None if cols[2 * q + 1] == "-" else int(cols[2 * q + 1]))
                       for q in range(len(cols) // 2)]
    return rows


def by_panel(records):
    out = {}
    for (k, i, killer, kind, level, step) in records:
        out[(k, i)] = (killer, step)
    return out


def test_table1_flat_panel0():
    t = load_table("table1_flat_panel0.txt")
    got = by_panel(hqr_elim_list(12, 1, 1, 1, FLAT, FLAT))
    for r, cols in t.items():
        if cols[0][0] is not None:
            assert got[(0, r)] == cols[0]


@pytest.mark.parametrize("a", [1, 12])
def test_table2_flat_3panels(a):
    # a=1: flat TT tree; a=12: one TS domain (PLASMA flat tree) -- same list
    t = load_table("table2_flat_3panels.txt")
    L = hqr_elim_list(12, 3, a, 1, FLAT, FLAT)
    got = by_panel(L)
    for r, cols in t.items():
        for k, (killer, step) in enumerate(cols):
            if killer is not None:
                assert got[(k, r)] == (killer, step), (k, r)
    assert all(rec[3] == (TS if a == 12 else TT) for rec in L)


def test_table3_binary_killers_and_panel0_steps():
    t = load_table("table3_binary_3panels.txt")
    got = by_panel(hqr_elim_list(12, 3, 1, 1, BINARY, FLAT))
    for r, cols in t.items():
        for k, (killer, step) in enumerate(cols):
            if killer is None:
                continue
            assert got[(k, r)][0] == killer, (k, r)
            if k == 0:
                assert got[(k, r)][1] == step, (k, r)


def test_table4_greedy_3panels():
    t = load_table("table4_greedy_3panels.txt")
    got = by_panel(hqr_elim_list(12, 3, 1, 1, GREEDY, FLAT))
    unpinned = {(2, 5), (2, 6)}
    for r, cols in t.items():
        for k, (killer, step) in enumerate(cols):
            if killer is None or (k, r) in unpinned:
                continue
            assert got[(k, r)] == (killer, step), (k, r)
    # the two contradictory entries follow the Greedy rule instead
    assert got[(2, 5)] == (3, 6) and got[(2, 6)] == (4, 6)


def test_greedy_single_panel_halving():
    # Sec. 3.2: z = floor(z'/2) bottom rows killed by the z rows right above
    got = by_panel(hqr_elim_list(12, 1, 1, 1, GREEDY, FLAT))
    assert [got[(0, r)] for r in range(6, 12)] == [(r - 6, 1) for r in range(6, 12)]
    assert [got[(0, r)] for r in (3, 4, 5)] == [(0, 2), (1, 2), (2, 2)]
    assert got[(0, 2)] == (1, 3) and got[(0, 1)] == (0, 4)


def test_fibonacci_hand_example():
    # R = 12 leaves, x = 5: groups {1}, {2,3}, {4,5,6}, {7,...,10}, {11}
    pairs = fibonacci_pairs(list(range(12)))
    assert pairs == [(11, 10), (7, 3), (8, 4), (9, 5), (10, 6), (4, 1), (5, 2), (6, 3),
                     (2, 0), (3, 1), (1, 0)]
    # R = 16 (the 16 virtual domains of the tall-skinny workload): x = 5
    pairs = fibonacci_pairs(list(range(16)))
    killed = sorted(kd for kd, _ in pairs)
    assert killed == list(range(1, 16))
    # every killer is alive when it kills (it dies later in the sequence)
    dead = set()
    for kd, kr in pairs:
        assert kr not in dead and kd not in dead
        dead.add(kd)


def test_binary_last_elimination_distance():
    # Sec. 3.1: the last elimination of the binary tree is row 0 killing
    # row 2^(ceil(log2 m) - 1)
    for m in range(2, 40):
        L = hqr_elim_list(m, 1, 1, 1, BINARY, FLAT)
        last = max(L, key=lambda r: r[5])
        lg = (m - 1).bit_length()
        assert (last[1], last[2]) == (2 ** (lg - 1), 0)


def _check_structure(L, m, n, a, p):
    assert validate(L, m, n) is None
    # canonical order and strictly increasing steps per row
    assert L == sorted(L, key=lambda r: (r[0], r[5], r[1]))
    last = {}
    for (k, i, killer, kind, level, step) in L:
        for r in (i, killer):
            assert last.get(r, 0) < step
            last[r] = step
    for k in range(n):
        recs = [r for r in L if r[0] == k]
        killed = {r[1] for r in recs}
        assert k not in killed and killed == set(range(k + 1, m))
        nts = 0
        for c in range(p):
            rows = [i for i in range(k, m) if i % p == c]
            if rows:
                nts += len(rows) - len(rows[::a])
        assert sum(1 for r in recs if r[3] == TS) == nts
        for (kk, i, killer, kind, level, step) in recs:
            if level in (0, 1):
                assert i % p == killer % p
            if level == 0:
                assert kind == TS
            else:
                assert kind == TT
            if level == 3:
                assert i == min(r for r in range(k, m) if r % p == i % p)
    assert total_weight(L, m, n) == 6 * m * n * n - 2 * n ** 3


def test_bruteforce_small_shapes():
    count = 0
    for m in range(1, 8):
        for n in range(1, m + 1):
            for a in range(1, m + 1):
                for p in range(1, m + 1):
                    for low, high in itertools.product(TREES, TREES):
                        _check_structure(hqr_elim_list(m, n, a, p, low, high), m, n, a, p)
                        count += 1
    assert count > 10000


@pytest.mark.parametrize("m,n,a,p", [(24, 10, 2, 3), (40, 8, 4, 4), (64, 8, 4, 16), (33, 5, 3, 5)])
def test_structure_medium(m, n, a, p):
    for low, high in itertools.product(TREES, TREES):
        _check_structure(hqr_elim_list(m, n, a, p, low, high), m, n, a, p)


def test_tall_skinny_counts():
    # 512 x 8 tiles, a = 4, p = 16: panel 0 has 384 TS, 112 low-level and 15
    # high-level eliminations; 8*511 - 28 records in all
    L = hqr_elim_list(512, 8, 4, 16, GREEDY, FIBONACCI)
    assert len(L) == 8 * 511 - 28
    p0 = [r for r in L if r[0] == 0]
    assert sum(r[4] == 0 for r in p0) == 384
    assert sum(r[4] == 1 for r in p0) == 112
    assert sum(r[4] == 3 for r in p0) == 15


def _mutations(L):
    """Lists that break one rule each."""
    L = list(L)
    yield "dup", L + [L[-1]]
    yield "drop", L[:-1]
    # killer zeroed before it kills: move a killer's own elimination earlier
    for q, (k, i, killer, kind, level, step) in enumerate(L):
        if killer > k:
            dq = next(t for t, r in enumerate(L) if r[0] == k and r[1] == killer)
            if dq > q:
                M = L[:q] + [L[dq]] + L[q:dq] + L[dq + 1:]
                yield "dead killer", M
                break
    # a row used before it is ready: swap the first record of panel 1 into panel 0
    q1 = next(t for t, r in enumerate(L) if r[0] == 1)
    M = [L[q1]] + L[:q1] + L[q1 + 1:]
    yield "not ready", M
    # TS kill of a triangle
    for q, r in enumerate(L):
        if r[3] == TT and r[4] == 1:
            M = list(L)
            M[q] = (r[0], r[1], r[2], TS, r[4], r[5])
            yield "ts on triangle", M
            break


def test_validator_rejects_broken_lists():
    L = hqr_elim_list(16, 4, 2, 2, BINARY, BINARY)
    assert validate(L, 16, 4) is None
    names = set()
    for name, M in _mutations(L):
        assert validate(M, 16, 4) is not None, name
        names.add(name)
    assert names == {"dup", "drop", "dead killer", "not ready", "ts on triangle"}


def test_triangle_rows():
    L = hqr_elim_list(8, 8, 8, 1, FLAT, FLAT)
    for k in range(8):
        assert triangle_rows(L, k, 8, 8) == {k}


# ----------------------------------------------------- coupling level --
# Sec. 4.2 ("Working out an example", m = 24, n = 10, p = 3, a = 2): tiles
# (4, 1) and (5, 1) are level-2 ("domino") tiles killed by their clusters' top
# tiles (1, 1) and (2, 1), after the inter-cluster eliminations elim(1, 0, 0)
# and elim(2, 0, 0) updated those tops; the last local killer of cluster P0 in
# panel 2 is its local diagonal tile (6, 2).

def _domino_structure(L, m, n, a, p):
    assert validate(L, m, n) is None
    assert L == sorted(L, key=lambda r: (r[0], r[5], r[1]))
    last = {}
    for (k, i, killer, kind, level, step) in L:
        for r in (i, killer):
            assert last.get(r, 0) < step
            last[r] = step
    for k in range(n):
        recs = [r for r in L if r[0] == k]
        assert {r[1] for r in recs} == set(range(k + 1, m))
        for c in range(p):
            rows = [i for i in range(k, m) if i % p == c]
            if not rows:
                continue
            top, diag = rows[0], k * p + c
            local = [i for i in rows if i >= diag]
            mine = [r for r in recs if r[1] % p == c and r[4] in (0, 1, 2)]
            for (kk, i, killer, kind, level, step) in mine:
                if level == 2:  # coupled rows: between the top and the local diagonal, killed by the top
                    assert killer == top and kind == TT and top < i <= diag
                else:  # local rows: on or below the local diagonal, reduced to it
                    assert i > diag and killer >= diag and killer % p == c
            coupled = sorted(r[1] for r in mine if r[4] == 2)
            assert coupled == [i for i in rows if top < i < diag] + ([local[0]] if local and local[0] != top else [])
            steps = [r[5] for r in sorted((r for r in mine if r[4] == 2), key=lambda r: r[1])]
            assert steps == sorted(steps)  # ascending, one after the other
    assert total_weight(L, m, n) == 6 * m * n * n - 2 * n ** 3


@pytest.mark.parametrize("high", [FLAT, BINARY])
def test_domino_example_facts(high):
    for low in TREES:
        L = hqr_elim_list(24, 10, 2, 3, low, high, domino=True)
        rec = {(r[0], r[1], r[2]): r for r in L}
        assert rec[(1, 4, 1)][4] == 2 and rec[(1, 5, 2)][4] == 2
        assert rec[(0, 1, 0)][4] == 3 and rec[(0, 2, 0)][4] == 3
        assert rec[(1, 4, 1)][5] > rec[(0, 1, 0)][5]
        assert rec[(1, 5, 2)][5] > rec[(0, 2, 0)][5]
        local = [r for r in L if r[0] == 2 and r[1] % 3 == 0 and r[4] in (0, 1)]
        assert max(local, key=lambda r: r[5])[2] == 6
        assert all(r[1] != 6 for r in local)
        _domino_structure(L, 24, 10, 2, 3)


def test_domino_with_one_domain_is_the_plain_list():
    for m, n, a in ((8, 8, 1), (9, 4, 3), (16, 5, 16)):
        for low, high in itertools.product(TREES, TREES):
            assert hqr_elim_list(m, n, a, 1, low, high, domino=True) == hqr_elim_list(m, n, a, 1, low, high)


def test_domino_bruteforce_small_shapes():
    count = 0
    for m in range(1, 8):
        for n in range(1, m + 1):
            for a in range(1, m + 1):
                for p in range(1, m + 1):
                    for low, high in itertools.product(TREES, TREES):
                        _domino_structure(hqr_elim_list(m, n, a, p, low, high, domino=True), m, n, a, p)
                        count += 1
    assert count > 10000


def test_domino_medium_and_level_counts():
    m, n, a, p = 64, 8, 4, 16
    L = hqr_elim_list(m, n, a, p, GREEDY, FIBONACCI, domino=True)
    _domino_structure(L, m, n, a, p)
    # the number of coupled rows grows with the panel: k - (local index of the top) per domain
    for k in range(n):
        want = 0
        for c in range(p):
            rows = [i for i in range(k, m) if i % p == c]
            if rows:
                want += len([i for i in rows if rows[0] < i <= k * p + c])
        assert sum(1 for r in L if r[0] == k and r[4] == 2) == want
    assert not any(r[4] == 2 for r in hqr_elim_list(m, n, a, p, GREEDY, FIBONACCI))
