"""Planted mistakes in the oracle: each must be caught by the committed pins.

The oracle is pinned to the paper's tables, closed forms and library routines
(tests/test_oracle_lists.py, tests/test_oracle_qr.py). A pin is only worth
something if a plausible slip in the oracle makes it fail, so every test here
rewrites one line of one oracle function in memory (the source file is never
touched), runs the pins that should notice, requires at least one of them to
fail, and restores the function.

Mistakes planted (one per test):
  transposed T in the block application, Householder sign rule flipped,
  sign of the T recursion flipped, the killer's row dropped from a TSQRT
  product, wrong diagonal offset of the TTQRT reflector triangle, Greedy
  killers paired in reverse, TS heads spaced one row too wide, coupling-level
  (domino) rows killed in descending order, the forward
  and backward replays of Q swapped, the TwoProduct error term dropped from
  the compensated residual.
"""
import inspect
import sys
import textwrap

import pytest

import oracle.elim_list as EL
import oracle.kernels as K
import oracle.lstsq as LS
import oracle.tile_qr as TQ
from tests import test_oracle_lists as TL
from tests import test_oracle_qr as TQR


def _plant(monkeypatch, module, fname, old, new):
    """Replace function `fname` of `module` by a copy whose source has `old`
    replaced by `new` (exactly one occurrence). Every already-imported test
    module that bound the original object by name gets the copy too."""
    orig = getattr(module, fname)
    src = textwrap.dedent(inspect.getsource(orig))
    assert src.count(old) == 1, (fname, old)
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), module.__file__, "exec"), ns)
    mutant = ns[fname]
    monkeypatch.setattr(module, fname, mutant)
    for name, mod in list(sys.modules.items()):
        if mod is None or not (name.startswith("tests.") or name.startswith("test_")):
            continue
        for attr, val in list(vars(mod).items()):
            if val is orig:
                monkeypatch.setattr(mod, attr, mutant)


def _caught(pins):
    """True if at least one pin (callable, kwargs) fails."""
    for fn, kw in pins:
        try:
            fn(**kw)
        except (AssertionError, ValueError, IndexError, KeyError, FloatingPointError):
            return True
    return False


MUTATIONS = [
    # (id, module, function, old text, new text, pins that must notice)
    ("transposed_T", K, "unmqr", "W = (Tb.T if trans else Tb) @ W", "W = (Tb if trans else Tb.T) @ W",
     [(TQR.test_geqrt_unmqr, dict(b=16, ib=4))]),
    ("householder_sign", K, "householder", "beta = -nrm if alpha >= 0.0 else nrm",
     "beta = nrm if alpha >= 0.0 else -nrm", [(TQR.test_householder_reflector, {})]),
    ("t_recursion_sign", K, "_t_column", "T[:j, j] = -tau * (T", "T[:j, j] = tau * (T",
     [(TQR.test_geqrt_unmqr, dict(b=16, ib=4))]),
    ("tsqrt_dropped_term", K, "tsqrt", "wv = R[j, cols] + v2 @ A[:, cols]", "wv = v2 @ A[:, cols]",
     [(TQR.test_tsqrt_tsmqr, dict(b=16, ib=4))]),
    ("ttqrt_triangle_offset", K, "ttqrt_v", "R2f[:j0 + w, j0:j0 + w], -j0)", "R2f[:j0 + w, j0:j0 + w], 0)",
     [(TQR.test_ttqrt_ttmqr, dict(b=16, ib=4))]),
    ("greedy_pairing", EL, "greedy_pairs", "zip(killed, killers)", "zip(killed, killers[::-1])",
     [(TL.test_table4_greedy_3panels, {}), (TL.test_greedy_single_panel_halving, {})]),
    ("head_spacing", EL, "hqr_elim_list", "heads = local[::a]", "heads = local[::a + 1]",
     [(TL.test_bruteforce_small_shapes, {}), (TL.test_structure_medium, dict(m=24, n=10, a=2, p=3))]),
    ("replay_swap", TQ, "apply_q", "seq = F.ops if trans else F.ops[::-1]", "seq = F.ops[::-1] if trans else F.ops",
     [(TQR.test_backward_error_and_orthogonality, dict(low=EL.GREEDY, high=EL.FIBONACCI, a=2, p=3))]),
    ("domino_order", EL, "hqr_elim_list", "for i in coupled:", "for i in coupled[::-1]:",
     [(TL.test_domino_example_facts, dict(high=EL.FLAT)), (TL.test_domino_bruteforce_small_shapes, {})]),
    ("dot2_dropped_twoproduct_error", LS, "dot2_residual", "c += e1 + e2", "c += e2",
     [(TQR.test_dot2_exact_rational, {})]),
]


@pytest.mark.parametrize("mid,module,fname,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, mid, module, fname, old, new, pins):
    # the pins pass on the real oracle
    assert not _caught(pins), mid
    _plant(monkeypatch, module, fname, old, new)
    assert _caught(pins), "planted mistake %s was not caught" % mid


def test_planting_leaves_the_oracle_intact():
    # the mutations above are undone by monkeypatch: the source on disk and the
    # module functions are the originals
    for _, module, fname, old, _, _ in MUTATIONS:
        assert old in inspect.getsource(getattr(module, fname))
