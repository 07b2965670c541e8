"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds mesh *descriptions* (octree leaves, per-element degrees,
block-map parameters), seeded random vectors and source parameters only.
It contains none of the DG method's arithmetic: both the CUDA library and the
oracle turn these descriptions into geometry, operators and right-hand sides
with their own code.

Leaf format: (level, ix, iy, iz) of a single box block; level-L cells have
width (hi - lo) / 2^L.  Leaves are emitted in Morton (z-curve) order.
"""
import numpy as np


def _morton_key(L, ix, iy, iz, maxL):
    s = maxL - L
    x, y, z = ix << s, iy << s, iz << s
    key = 0
    for b in range(maxL):
        key |= ((x >> b) & 1) << (3 * b) | ((y >> b) & 1) << (3 * b + 1) | ((z >> b) & 1) << (3 * b + 2)
    return key


def morton_sort(leaves):
    leaves = [tuple(int(v) for v in lf) for lf in leaves]
    maxL = max(lf[0] for lf in leaves)
    return sorted(leaves, key=lambda lf: (_morton_key(lf[0], lf[1], lf[2], lf[3], maxL), lf[0]))


def uniform_leaves(level):
    m = 1 << level
    return morton_sort([(level, i, j, k) for k in range(m) for j in range(m) for i in range(m)])


def refine(leaves, predicate):
    """Replace every leaf for which predicate(leaf) holds by its 8 children."""
    out = []
    for lf in leaves:
        L, i, j, k = lf
        if predicate(lf):
            for c in range(8):
                out.append((L + 1, 2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + ((c >> 2) & 1)))
        else:
            out.append(tuple(lf))
    return out


def balance_2to1(leaves):
    """Refine leaves until every face neighbour differs by at most one level."""
    leaves = [tuple(lf) for lf in leaves]
    while True:
        S = set(leaves)
        maxL = max(lf[0] for lf in leaves)
        bad = set()
        for (L, i, j, k) in leaves:
            for d in range(3):
                for sgn in (-1, 1):
                    c = [i, j, k]
                    c[d] += sgn
                    if c[d] < 0 or c[d] >= (1 << L):
                        continue
                    # a neighbour two levels finer exists iff some level L+2 leaf lies in the
                    # adjacent level-L cell: check all deeper levels.
                    for L2 in range(L + 2, maxL + 1):
                        sh = L2 - L
                        lo = [v << sh for v in c]
                        found = False
                        span = 1 << sh
                        # only cells touching our face matter
                        rng = [range(lo[t], lo[t] + span) for t in range(3)]
                        rng[d] = [lo[d] + (span - 1 if sgn < 0 else 0)]
                        for a in rng[0]:
                            for b in rng[1]:
                                for cc in rng[2]:
                                    if (L2, a, b, cc) in S:
                                        found = True
                                        break
                                if found:
                                    break
                            if found:
                                break
                        if found:
                            bad.add((L, i, j, k))
                            break
        if not bad:
            return morton_sort(leaves)
        leaves = refine(leaves, lambda lf: lf in bad)


def config1_mesh():
    """Poisson on [-1,1]^3, 4x4x4 affine elements, uniform p = 3."""
    leaves = uniform_leaves(2)
    return dict(lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), leaves=np.array(leaves, dtype=np.int32),
                p=np.full(len(leaves), 3, dtype=np.int32), warp=None)


def sweep_mesh(level=5, seed=0, pmin=2, pmax=7, curved=True, refine_octant=True, h=1.0 / 16.0):
    """Operator-apply sweep mesh: 2^level per axis on [-1,1]^3, the octant
    x, y, z < 0 h-refined once (2:1 non-conforming faces), per-element p drawn
    uniformly from {pmin..pmax}, node positions curved by the seeded sine warp
    with amplitude 0.1 h and k_i drawn from {1,2,3}.  h is the coarse element
    width of the full 32^3 workload (1/16) at every level, so smaller test
    meshes carry the same physical block map.  level = 5 gives the full
    workload (61,440 elements)."""
    rng = np.random.default_rng(seed)
    half = 1 << (level - 1)
    leaves = uniform_leaves(level)
    if refine_octant:
        leaves = refine(leaves, lambda lf: lf[1] < half and lf[2] < half and lf[3] < half)
    leaves = morton_sort(leaves)
    p = rng.integers(pmin, pmax + 1, size=len(leaves)).astype(np.int32)
    warp = None
    if curved:
        k = tuple(int(v) for v in rng.integers(1, 4, size=3))
        warp = (0.1 * h, k)
    return dict(lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), leaves=np.array(leaves, dtype=np.int32),
                p=p, warp=warp)


def random_vector(n, seed=1):
    """i.i.d. N(0, 1) input vector in FP64."""
    return np.random.default_rng(seed).standard_normal(n)


def oracle_mesh_args(desc):
    """Positional/keyword arguments for the oracle's Mesh constructor."""
    return (desc['lo'], desc['hi'], desc['leaves'], desc['p']), dict(warp=desc['warp'])
