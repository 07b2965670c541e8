"""Pins for the oracle mesh and mortar set (Sec. II.A.1, mortar figure)."""
import numpy as np

from oracle.mesh import Mesh
from paper_1907_01572_gb300 import inputs


def _mesh(desc):
    a, k = inputs.oracle_mesh_args(desc)
    return Mesh(*a, **k)


def test_config1_counts():
    m = _mesh(inputs.config1_mesh())
    nb = sum(1 for mm in m.mortars if mm.eB is None)
    assert m.n_elems == 64 and m.n_dofs == 4096
    assert len(m.mortars) - nb == 144 and nb == 96


def test_two_to_one_mortars():
    """4^3 mesh with the x,y,z<0 octant refined: each coarse face on the
    refinement interface is covered by four fine mortars."""
    m = _mesh(inputs.sweep_mesh(level=2, seed=0))
    assert m.n_elems == 56 + 64
    coarse_faces = 0
    for e in range(m.n_elems):
        for f in range(6):
            k = len(m.elem_mortars[e][f])
            assert k in (1, 4)
            if k == 4:
                coarse_faces += 1
                for mi in m.elem_mortars[e][f]:
                    mm = m.mortars[mi]
                    assert mm.eB == e and mm.posB != (0, 0) and mm.posA == (0, 0)
                    assert m.leaves[mm.eA][0] == m.leaves[e][0] + 1
    # the refined octant (2x2x2 coarse cells) has 3 interface planes of 2x2 coarse faces
    assert coarse_faces == 3 * 4
    # every element face is covered by its mortars exactly once in area
    for e in range(m.n_elems):
        for f in range(6):
            areas = 0.0
            for mi in m.elem_mortars[e][f]:
                mm = m.mortars[mi]
                pos = mm.posA if mm.eA == e else mm.posB
                areas += np.prod([1.0 if p == 0 else 0.5 for p in pos])
            assert abs(areas - 1.0) < 1e-15


def test_mortar_degree_rule():
    """Mortar degree = max(p+, p-): the mortar figure's p=4 | (p=3, p=6) example."""
    leaves = [(1, 0, 0, 0)]
    leaves += [(2, 2 + a, b, c) for c in range(2) for b in range(2) for a in range(2)]
    leaves += [(1, 0, 1, 0), (1, 1, 1, 0), (1, 0, 0, 1), (1, 1, 0, 1), (1, 0, 1, 1), (1, 1, 1, 1)]
    p = [4] + [3, 3, 6, 6, 3, 3, 6, 6] + [2] * 6
    m = Mesh((0, 0, 0), (1, 1, 1), leaves, p)
    degs = sorted(m.mortars[mi].pm for mi in m.elem_mortars[0][1])
    assert degs == [4, 4, 6, 6]
