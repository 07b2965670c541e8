"""The library's host hp-AMR calls (dg_hp_mark, dg_hp_refine; Algorithm 4 and
2:1 balancing) against the oracle (oracle/hpamr.py): decisions, predictions
and leaf sets bit-identical on random inputs (no GPU needed)."""
import math

import numpy as np
import pytest

from oracle import hpamr
from oracle.mesh import Mesh
from paper_1907_01572_gb300 import dgell, inputs

CRIT = {'fraction': dgell.DG_MARK_FRACTION, 'mean': dgell.DG_MARK_MEAN}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_01572_gb300 import build
    build.build()


@pytest.mark.parametrize("crit,theta", [("fraction", 0.1), ("fraction", 0.37), ("fraction", 1.0),
                                        ("mean", 1.0), ("mean", 2.5)])
@pytest.mark.parametrize("seed", [0, 1])
def test_mark_and_decisions_match_oracle(crit, theta, seed):
    rng = np.random.default_rng(seed)
    n = 500
    eta = np.exp(rng.normal(size=n) * 3)
    eta[::17] = eta[3]                       # ties
    pred = np.where(rng.random(n) < 0.3, np.inf, np.exp(rng.normal(size=n) * 3))
    pred[::11] = 0.0
    p = rng.integers(1, 9, size=n)
    level = rng.integers(0, 16, size=n)
    act, nxt = dgell.hp_mark(eta, pred, p, level, CRIT[crit], theta, 0.25, 0.1)
    marked = hpamr.mark(list(eta), crit, theta)
    a_ref, n_ref = hpamr.smooth_pred(list(eta), list(pred), list(p), list(level), marked, 0.25, 0.1)
    assert act.tolist() == a_ref
    assert np.array_equal(nxt, np.array(n_ref))      # bit-identical, inf included


def _as_dict(L, P, Q, R):
    return {tuple(int(v) for v in L[i]): (int(P[i]), float(Q[i]), int(R[i])) for i in range(len(P))}


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_refine_and_balance_match_oracle(seed):
    rng = np.random.default_rng(seed)
    lv = [tuple(x) for x in inputs.uniform_leaves(1)]
    p = [2] * len(lv)
    pred = [math.inf] * len(lv)
    for step in range(3):
        n = len(lv)
        act = rng.choice([0, 0, 0, 1, 2], size=n).astype(np.int32)
        act[np.array(p) >= 8] = 0
        nxt = rng.random(n)
        L, P, Q, R = dgell.hp_refine(lv, p, act, nxt, pred_init=math.inf)
        got = _as_dict(L, P, Q, R)
        ref = hpamr.refine(lv, p, list(act), list(nxt), pred_init=math.inf)
        assert got == ref
        assert len(got) == len(L)
        Mesh((0, 0, 0), (1, 1, 1), L.tolist(), P.tolist())      # 2:1 balanced and tiling
        lv, p, pred = [tuple(x) for x in L.tolist()], P.tolist(), Q.tolist()


def test_refine_order_children_in_place_and_errors():
    lv = inputs.uniform_leaves(1)
    act = np.zeros(8, dtype=np.int32)
    act[1] = dgell.DG_AMR_H_REFINE
    L, P, Q, R = dgell.hp_refine(lv, [3] * 8, act, np.zeros(8))
    assert L.shape == (15, 4)
    assert L[:1].tolist() == [list(lv[0])]
    x, y, z = lv[1][1:]
    assert L[1:9].tolist() == [[2, 2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + ((c >> 2) & 1)] for c in range(8)]
    assert R.tolist() == [0] + [1] * 8 + list(range(2, 8))
    with pytest.raises(dgell.DgError):
        dgell.hp_refine([(15, 0, 0, 0)], [3], [dgell.DG_AMR_H_REFINE], [0.0])
    with pytest.raises(dgell.DgError):
        dgell.hp_refine([(0, 0, 0, 0)], [8], [dgell.DG_AMR_P_REFINE], [0.0])
    with pytest.raises(dgell.DgError):
        dgell.hp_refine([(1, 2, 0, 0)], [3], [0], [0.0])


def test_mark_rejects_bad_theta():
    eta = np.ones(4)
    z = np.zeros(4)
    p = np.full(4, 2)
    for crit, th in ((dgell.DG_MARK_FRACTION, 0.0), (dgell.DG_MARK_FRACTION, 1.5), (dgell.DG_MARK_FRACTION, math.nan),
                     (dgell.DG_MARK_MEAN, -1.0), (dgell.DG_MARK_MEAN, math.inf), (dgell.DG_MARK_MEAN, math.nan)):
        with pytest.raises(dgell.DgError):
            dgell.hp_mark(eta, z, p, p, crit, th)
    for crit, th in (('fraction', 0.0), ('fraction', 1.5), ('mean', -1.0), ('mean', math.inf)):
        with pytest.raises(ValueError):
            hpamr.mark(list(eta), crit, th)


def _block_dict(out, Q, R):
    return {(int(b),) + tuple(int(v) for v in lf): (int(pp), float(q), int(r))
            for b, lf, pp, q, r in zip(out["elem_block"], out["leaves"], out["p"], Q, R)}


@pytest.mark.parametrize("case", ["pair5", "pair13", "pair23", "sphere"])
def test_block_mesh_refinement_matches_oracle(case):
    """dg_hp_refine_mesh on multi-block meshes (block connectivity and
    orientation codes) against the oracle's physical point location, over
    two random refinement steps; the result builds as an oracle block mesh
    (2:1 across every interface, tiling every block)."""
    from oracle.blockmesh import BlockMesh
    if case == "sphere":
        d = inputs.cubed_sphere_mesh(level=1, a=1.0, r=3.0, r_out=30.0, refine_wedge=(2, 3), pmin=2, pmax=4)
    else:
        d = inputs.block_pair_mesh(rot=int(case[4:]), level=1, refine_block=0, seed=1)
    rng = np.random.default_rng(len(case))
    for step in range(2):
        n = len(d["p"])
        act = rng.choice([0, 0, 0, 1, 2], size=n).astype(np.int32)
        act[np.asarray(d["p"]) >= 8] = 0
        nxt = rng.random(n)
        out, Q, R = dgell.hp_refine_mesh(d, act, nxt, pred_init=math.inf)
        ref = hpamr.refine_blocks(d["blocks"], d["elem_block"], d["leaves"], d["p"], list(act), list(nxt), math.inf)
        assert _block_dict(out, Q, R) == ref
        BlockMesh(d["blocks"], out["elem_block"], out["leaves"], out["p"])
        d = out


def test_refine_mesh_single_box_equals_refine():
    d = inputs.sweep_mesh(level=1, seed=3)
    n = len(d["p"])
    rng = np.random.default_rng(9)
    act = rng.choice([0, 1, 2], size=n).astype(np.int32)
    nxt = rng.random(n)
    out, Q, R = dgell.hp_refine_mesh(d, act, nxt)
    L, P, Q2, R2 = dgell.hp_refine(d["leaves"], d["p"], act, nxt)
    assert np.array_equal(out["leaves"], L) and np.array_equal(out["p"], P)
    assert np.array_equal(Q, Q2) and np.array_equal(R, R2)
    assert out["lo"] == d["lo"] and out.get("warp") == d.get("warp")
