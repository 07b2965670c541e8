"""Pins for the oracle's metric terms (eqs. Jacobian, Surface-Jacobian, normal)
on curved isoparametric elements."""
import numpy as np

from oracle import sipg, tables
from oracle.mesh import Mesh
from paper_1907_01572_gb300 import inputs


def _curved(level=1, warp=(0.03, (1, 2, 1))):
    lv = inputs.uniform_leaves(level)
    return Mesh((-1, -1, -1), (1, 1, 1), lv, [4] * len(lv), warp=warp)


def test_stiffness_of_coordinate_function_is_volume():
    """u = x_1 is represented exactly by its nodal values on an isoparametric
    element, so u^T K_e u = int |grad x_1|^2 = |e| = sum w det J."""
    m = _curved()
    for e in range(m.n_elems):
        K = sipg.element_stiffness(m, e, extra=3)
        X = m.node_coords(e)
        _, w, _, detJ, _ = sipg.volume_geometry(m, e, extra=3)
        vol = np.sum(w * detJ)
        for d in range(3):
            assert abs(X[:, d] @ K @ X[:, d] - vol) < 1e-12 * vol
        assert abs(X[:, 0] @ K @ X[:, 1]) < 1e-12


def test_divergence_theorem_on_curved_element():
    """3 |e| = sum over faces int x . n dS (exact with enough GL points);
    pins det J, S^m and the normal's orientation and sign."""
    m = _curved(level=0, warp=(0.05, (1, 1, 2)))
    e = 0
    n = int(m.n[e])
    q = 3 * n
    _, w, _, detJ, _ = sipg.volume_geometry(m, e, extra=q - n)
    vol = np.sum(w * detJ)
    s, ws = tables.gl_nodes_weights(q)
    s1, s2 = np.tile(s, q), np.repeat(s, q)
    wt = np.tile(ws, q) * np.repeat(ws, q)
    flux = 0.0
    for f in range(6):
        d, sg = divmod(f, 2)
        xi = m.face_ref_points(f, (0, 0), s1, s2)
        J = m.jacobian_at(e, xi)
        Jinv = np.linalg.inv(J)
        g = Jinv[:, d, :]
        nrm = np.linalg.norm(g, axis=1)
        S = np.linalg.det(J) * nrm
        nvec = (1 if sg else -1) * g / nrm[:, None]
        x = m.position_at(e, xi)
        flux += np.sum(wt * S * np.einsum('pi,pi->p', x, nvec))
    assert abs(flux - 3 * vol) < 1e-12
    # the warp keeps the cube: volume is 8 when integrated exactly
    assert abs(vol - 8.0) < 1e-12


def test_positive_jacobian_on_sweep_map():
    d = inputs.sweep_mesh(level=2, seed=0)
    a, k = inputs.oracle_mesh_args(d)
    m = Mesh(*a, **k)
    for e in range(0, m.n_elems, 7):
        _, _, _, detJ, _ = sipg.volume_geometry(m, e)
        assert detJ.min() > 0
