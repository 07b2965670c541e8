"""Pins for the oracle hp-AMR driving strategy (Algorithm 4, smooth-pred):
hand-worked marking and decisions, a hand-worked 2:1 balance cascade, and
the tiling / 2:1 invariants through the oracle mesh constructor (which
rejects a leaf set that does not tile the box or is not 2:1 balanced)."""
import math

import numpy as np
import pytest

from oracle import hpamr
from oracle.mesh import Mesh
from paper_1907_01572_gb300 import inputs

H, P, N = hpamr.H_REFINE, hpamr.P_REFINE, hpamr.NONE


def test_mark_fraction_ties_to_lower_index():
    eta = [1.0, 5.0, 3.0, 5.0, 0.5]
    assert hpamr.mark(eta, 'fraction', 0.4) == [False, True, False, True, False]
    assert hpamr.mark(eta, 'fraction', 0.5) == [False, True, True, True, False]
    assert hpamr.mark(eta, 'fraction', 0.2) == [False, True, False, False, False]
    assert hpamr.mark([], 'fraction', 0.5) == []


def test_mark_mean():
    eta = [1.0, 2.0, 3.0, 6.0]     # mean 3
    assert hpamr.mark(eta, 'mean', 1.0) == [False, False, False, True]
    assert hpamr.mark(eta, 'mean', 0.5) == [False, True, True, True]


def test_smooth_pred_decisions_and_predictions():
    eta = [4.0, 4.0, 1.0, 2.0, 7.0]
    pred = [math.inf, 1.0, 8.0, 0.0, 0.0]
    p = [2, 3, 8, 8, 4]
    level = [1, 1, 1, 15, 2]
    marked = [True, True, True, True, False]
    act, nxt = hpamr.smooth_pred(eta, pred, p, level, marked, gamma_h=0.25, gamma_p=0.1)
    # e0: no prediction yet -> p; e1: above its prediction -> h; e2: below, but
    # p = p_max -> h; e3: above, deepest level and p_max -> nothing; e4: unmarked
    assert act == [P, H, H, N, N]
    assert nxt[0] == pytest.approx(0.4, rel=1e-15)
    assert nxt[1] == 0.25 / 8 / 4 ** 3 * 4.0
    assert nxt[2] == 0.25 / 8 / 4 ** 8 * 1.0
    assert nxt[3] == 0.0 and nxt[4] == 0.0


def test_literal_zero_prediction_refines_h_first():
    act, _ = hpamr.smooth_pred([1.0], [0.0], [3], [2], [True], 0.25, 0.1)
    assert act == [H]
    act, _ = hpamr.smooth_pred([1.0], [math.inf], [3], [2], [True], 0.25, 0.1)
    assert act == [P]


def _check_tiles_and_balanced(out, p_of=None):
    leaves = sorted(out)
    vol = sum(8.0 ** -lf[0] for lf in leaves)
    assert vol == pytest.approx(1.0, abs=1e-15)
    Mesh((0, 0, 0), (1, 1, 1), leaves, [out[lf][0] for lf in leaves])   # raises if not 2:1 / not tiling


def test_balance_cascade_by_hand():
    """Refining the level-2 child that touches x = 0 next to the unrefined
    level-1 cube (1,1,0,0) forces that cube to level 2; nothing else moves."""
    lv = inputs.refine(inputs.uniform_leaves(1), lambda lf: lf[1:] == (0, 0, 0))
    n = len(lv)
    target = lv.index((2, 1, 0, 0))
    act = [H if e == target else N for e in range(n)]
    out = hpamr.refine(lv, [3] * n, act, [7.0] * n, pred_init=math.inf)
    assert len(out) == n - 1 + 8 - 1 + 8
    forced = lv.index((1, 1, 0, 0))
    assert (1, 1, 0, 0) not in out
    for c in range(8):
        kid = (2, 2 + (c & 1), (c >> 1) & 1, (c >> 2) & 1)
        assert out[kid] == (3, math.inf, forced)
        kid3 = (3, 2 + (c & 1), (c >> 1) & 1, (c >> 2) & 1)
        assert out[kid3] == (3, 7.0, target)
    _check_tiles_and_balanced(out)


def test_p_refinement_raises_degree_only():
    lv = inputs.uniform_leaves(1)
    act = [P if e == 2 else N for e in range(8)]
    out = hpamr.refine(lv, [4] * 8, act, [0.5] * 8, pred_init=0.0)
    assert len(out) == 8 and out[tuple(lv[2])] == (5, 0.5, 2) and out[tuple(lv[3])] == (4, 0.5, 3)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_refinement_sequences_stay_balanced(seed):
    rng = np.random.default_rng(seed)
    lv = [tuple(x) for x in inputs.uniform_leaves(1)]
    p = [2] * len(lv)
    pred = [math.inf] * len(lv)
    for step in range(3):
        n = len(lv)
        eta = rng.random(n)
        marked = hpamr.mark(eta, 'fraction', 0.15)
        level = [lf[0] for lf in lv]
        act, nxt = hpamr.smooth_pred(eta, pred, p, level, marked, 0.25, 0.1, p_max=4)
        out = hpamr.refine(lv, p, act, nxt, pred_init=math.inf)
        _check_tiles_and_balanced(out)
        for e in range(n):
            if act[e] == H:
                assert tuple(lv[e]) not in out
        lv = sorted(out)
        p = [out[lf][0] for lf in lv]
        pred = [out[lf][1] for lf in lv]
        assert max(p) <= 4


def test_balance_across_a_turned_block_interface_by_hand():
    """Two unit boxes glued at x = 1, the second turned (rotation 5): the
    block-0 family next to (1, 0, 0) is at level 2; splitting its four
    children on the interface puts level-3 cells against the level-1 cell
    [1, 1.5] x [0, 0.5]^2 of block 1 across the interface and against the
    level-1 cells (1, 1, 1, 0) and (1, 1, 0, 1) of block 0 itself: those
    three, and nothing else, must split."""
    from oracle.blockmesh import BlockMesh, block_map
    d = inputs.block_pair_mesh(rot=5, level=1, refine_block=0, seed=1)
    lv, eb, p = np.asarray(d["leaves"]), np.asarray(d["elem_block"]), np.asarray(d["p"])
    n = len(p)
    act = [H if (eb[e] == 0 and lv[e][0] == 2 and lv[e][1] == 3) else N for e in range(n)]
    assert act.count(H) == 4
    out = hpamr.refine_blocks(d["blocks"], eb, lv, p, act, [1.0] * n, pred_init=math.inf)
    split = [k for k in out if k[0] == 1 and k[1] == 2]
    assert len(split) == 8
    for k in split:
        c = block_map(d["blocks"][1], (-1.0 + (2.0 * np.array(k[2:]) + 1.0) / 4.0)[None])[0]
        assert 1.0 < c[0] < 1.5 and 0.0 < c[1] < 0.5 and 0.0 < c[2] < 0.5
        assert out[k][1] == math.inf
    assert (0, 1, 1, 1, 0) not in out and (0, 1, 1, 0, 1) not in out
    assert len(out) == n - 4 + 32 - 3 + 24
    keys = sorted(out)
    BlockMesh(d["blocks"], [k[0] for k in keys], [k[1:] for k in keys], [out[k][0] for k in keys])
