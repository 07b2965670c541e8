"""hp-AMR driving strategy (oracle; test infrastructure only).

Sec. II.D (driving strategy), Algorithm 4 (smooth-pred): elements with a
large eta^2(e) are refined; an element whose eta^2(e) exceeds the error
predicted for it at the previous step, eta^2_pred(e), is h-refined and its
children are given eta^2_pred = gamma_h (1/2)^d (1/2)^(2 p_e) eta^2(e);
otherwise it is p-refined and eta^2_pred(e) = gamma_p eta^2(e).

Which elements count as "large" (the conditional of Algorithm 4), both
criteria of Sec. II.D:
 * 'fraction': the ceil(theta n) elements with the largest eta^2 (ties to
   the lower element index);
 * 'mean': eta^2(e) > theta * mean(eta^2) (the mean summed in element order).

Readings (where the paper leaves the choice open or disagrees with itself):
 * Initial prediction: the text says every element is first p-refined,
   while Algorithm 4 with eta^2_pred = 0 h-refines first.  Elements start
   with a caller-chosen eta^2_pred; +inf gives the text's p-first start,
   0 the listing's literal one.
 * Limits: a p-refinement at p = p_max becomes an h-refinement; an
   h-refinement at the deepest level becomes a p-refinement, and nothing
   when p = p_max as well.
 * h-refined children keep the parent's degree.  After the marked
   refinements, leaves are refined further until no two face neighbours
   differ by more than one level (2:1 balance); children of such
   balance-only refinements keep the degree and start with the initial
   prediction.

Multi-block meshes (refine_blocks): the same actions, and 2:1 balance
across block interfaces found physically: the point just outside the centre
of each leaf face is mapped with the leaf's block map and located in every
block by Newton's method on that block's map; the leaf of that block
covering the point is the face neighbour to compare with.

Pins: hand-worked marking, decisions and balance cascades (one box, and
across a turned block interface); the 2:1 and tiling invariants through the
oracle mesh constructors (tests/test_oracle_hpamr.py).
"""
import math

import numpy as np

NONE, P_REFINE, H_REFINE = 0, 1, 2


def mark(eta2, criterion, theta):
    """Booleans: which elements Algorithm 4 treats as having a large eta^2."""
    n = len(eta2)
    if criterion == 'fraction' and not 0.0 < theta <= 1.0:
        raise ValueError("the fraction criterion takes theta in (0, 1]")
    if criterion == 'mean' and not (theta >= 0.0 and math.isfinite(theta)):
        raise ValueError("the mean criterion takes a finite theta >= 0")
    if n == 0:
        return []
    if criterion == 'fraction':
        k = int(math.ceil(theta * n))
        order = sorted(range(n), key=lambda e: (-float(eta2[e]), e))
        chosen = set(order[:k])
        return [e in chosen for e in range(n)]
    if criterion == 'mean':
        s = 0.0
        for v in eta2:
            s += float(v)
        mean = s / n
        return [float(v) > theta * mean for v in eta2]
    raise ValueError("criterion is 'fraction' or 'mean'")


def smooth_pred(eta2, pred, p, level, marked, gamma_h, gamma_p, p_max=8, level_max=15, d=3):
    """Algorithm 4 for every element.  Returns (action, pred_next): action is
    NONE / P_REFINE / H_REFINE; pred_next is the prediction the element (for
    P_REFINE / NONE) or each of its children (for H_REFINE) carries on."""
    action, nxt = [], []
    for e in range(len(eta2)):
        a = NONE
        if marked[e]:
            a = H_REFINE if float(eta2[e]) > float(pred[e]) else P_REFINE
            if a == P_REFINE and p[e] >= p_max:
                a = H_REFINE
            if a == H_REFINE and level[e] >= level_max:
                a = P_REFINE if p[e] < p_max else NONE
        if a == H_REFINE:
            v = gamma_h * 0.5 ** d * 0.5 ** (2 * int(p[e])) * float(eta2[e])
        elif a == P_REFINE:
            v = gamma_p * float(eta2[e])
        else:
            v = float(pred[e])
        action.append(a)
        nxt.append(v)
    return action, nxt


def _children(leaf):
    L, ix, iy, iz = leaf
    return [(L + 1, 2 * ix + (c & 1), 2 * iy + ((c >> 1) & 1), 2 * iz + ((c >> 2) & 1)) for c in range(8)]


def _box(leaf, depth):
    """Integer box of a leaf on the uniform grid of level `depth`."""
    L, ix, iy, iz = leaf
    s = 1 << (depth - L)
    return [(ix * s, (ix + 1) * s), (iy * s, (iy + 1) * s), (iz * s, (iz + 1) * s)]


def _face_neighbours(a, b, depth):
    """True when leaves a and b share part of a face (positive area)."""
    A, B = _box(a, depth), _box(b, depth)
    touch = 0
    for k in range(3):
        if A[k][1] == B[k][0] or B[k][1] == A[k][0]:
            touch += 1
        elif min(A[k][1], B[k][1]) <= max(A[k][0], B[k][0]):
            return False
    return touch == 1


def refine(leaves, p, action, pred_next, pred_init):
    """Applies the actions, then 2:1-balances by brute force over all leaf
    pairs.  Returns {leaf: (p, pred, parent)} (parent: the old element the
    new leaf lies in)."""
    out = {}
    for e, lf in enumerate(leaves):
        lf = tuple(int(v) for v in lf)
        if action[e] == H_REFINE:
            for c in _children(lf):
                out[c] = (int(p[e]), float(pred_next[e]), e)
        elif action[e] == P_REFINE:
            out[lf] = (int(p[e]) + 1, float(pred_next[e]), e)
        else:
            out[lf] = (int(p[e]), float(pred_next[e]), e)
    while True:
        keys = list(out)
        depth = max(k[0] for k in keys)
        coarse = set()
        for i, a in enumerate(keys):
            for b in keys[i + 1:]:
                if abs(a[0] - b[0]) >= 2 and _face_neighbours(a, b, depth):
                    coarse.add(a if a[0] < b[0] else b)
        if not coarse:
            return out
        for lf in coarse:
            pe, _, parent = out.pop(lf)
            for c in _children(lf):
                out[c] = (pe, float(pred_init), parent)


def _locate(blocks, x, tol=1e-9, iters=60):
    """(block, reference point) of each physical point x (P, 3), or (-1, None)
    outside every block: Newton's method on each block map from its centre."""
    from .blockmesh import block_jacobian, block_map
    P = len(x)
    where = np.full(P, -1)
    ref = np.zeros((P, 3))
    for b, blk in enumerate(blocks):
        todo = np.nonzero(where < 0)[0]
        if len(todo) == 0:
            break
        xi = np.zeros((len(todo), 3))
        for _ in range(iters):
            r = block_map(blk, xi) - x[todo]
            step = np.linalg.solve(block_jacobian(blk, xi), r[:, :, None])[:, :, 0]
            xi = np.clip(xi - step, -3.0, 3.0)
            if np.abs(step).max() < 1e-14:
                break
        ok = (np.abs(block_map(blk, xi) - x[todo]).max(axis=1) <= 1e-10 * np.maximum(1.0, np.abs(x[todo]).max(axis=1))) \
            & (np.abs(xi).max(axis=1) <= 1.0 + tol)
        where[todo[ok]] = b
        ref[todo[ok]] = xi[ok]
    return where, ref


def refine_blocks(blocks, elem_block, leaves, p, action, pred_next, pred_init):
    """refine() for a multi-block mesh: returns {(block, level, ix, iy, iz):
    (p, pred, parent)}."""
    from .blockmesh import block_map
    out = {}
    for e, lf in enumerate(leaves):
        b = int(elem_block[e])
        L, ix, iy, iz = (int(v) for v in lf)
        if action[e] == H_REFINE:
            for c in _children((L, ix, iy, iz)):
                out[(b,) + c] = (int(p[e]), float(pred_next[e]), e)
        elif action[e] == P_REFINE:
            out[(b, L, ix, iy, iz)] = (int(p[e]) + 1, float(pred_next[e]), e)
        else:
            out[(b, L, ix, iy, iz)] = (int(p[e]), float(pred_next[e]), e)
    while True:
        keys = list(out)
        pts, src = [], []
        for k in keys:
            b, L, ix, iy, iz = k
            for f in range(6):
                d, s = divmod(f, 2)
                xi = -1.0 + (2.0 * np.array([ix, iy, iz], dtype=np.float64) + 1.0) / (1 << L)
                xi[d] = -1.0 + (2.0 * [ix, iy, iz][d] + (2.0 if s else 0.0)) / (1 << L) + (1e-7 if s else -1e-7)
                pts.append(block_map(blocks[b], xi[None])[0])
                src.append(k)
        where, ref = _locate(blocks, np.array(pts))
        coarse = set()
        for k, b2, r in zip(src, where, ref):
            if b2 < 0:
                continue
            L = k[1]
            for l in range(L, -1, -1):
                cell = tuple(int(min(max(np.floor((r[i] + 1.0) / 2.0 * (1 << l)), 0), (1 << l) - 1)) for i in range(3))
                if (int(b2), l) + cell in out:
                    if l < L - 1:
                        coarse.add((int(b2), l) + cell)
                    break
        if not coarse:
            return out
        for k in coarse:
            pe, _, parent = out.pop(k)
            for c in _children(k[1:]):
                out[(k[0],) + c] = (pe, float(pred_init), parent)
