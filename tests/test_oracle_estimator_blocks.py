"""Pins of the oracle's estimator on multi-block meshes (Sec. II.D with the
exact block maps) and of its fiducial-grid form (Sec. II.D, fiducial-grid
paragraph; Problem C): the block maps' second derivatives against differences
of their Jacobians, the chain-rule Laplacian of an interpolated smooth field
against the field's own Laplacian on curved elements, and the exact scaling of
each estimator term under a uniformly scaled fiducial grid."""
import numpy as np
import pytest

from oracle import estimator, tables
from oracle.blockmesh import BlockMesh, block_hessian, block_jacobian
from paper_1907_01572_gb300 import inputs


def _blocks():
    hexb = dict(kind="hex8", corners=[[-1.0 + 0.1 * c, -1.0 + 0.2 * (c >> 1 & 1) + 2.0 * (c >> 1 & 1),
                                        -1.0 + 2.0 * (c >> 2 & 1) - 0.15 * (c & 1) * (c >> 2 & 1)] for c in range(8)])
    for c in range(8):
        hexb["corners"][c][0] += 2.0 * (c & 1) + 0.3 * (c >> 1 & 1) * (c >> 2 & 1)
    return [hexb, dict(kind="wedge", face=1, a=1.0, r=3.0), dict(kind="wedge", face=4, a=2.0, r=10.0),
            dict(kind="shell", face=3, r1=10.0, r2=1e3), dict(kind="shell", face=0, r1=2.0, r2=5.0)]


def test_block_hessians_against_jacobian_differences():
    rng = np.random.default_rng(4)
    xi = rng.uniform(-0.9, 0.9, (6, 3))
    h = 1e-5
    for b in _blocks():
        H = block_hessian(b, xi)
        for m in range(3):
            e = np.zeros(3)
            e[m] = h
            dJ = (block_jacobian(b, xi + e) - block_jacobian(b, xi - e)) / (2 * h)
            scale = max(1.0, np.abs(dJ).max())
            assert np.abs(H[:, :, :, m] - dJ).max() < 1e-6 * scale, (b["kind"], m)
        assert np.allclose(H, np.swapaxes(H, 2, 3))


def _wedge_shell_mesh(p, level=1):
    blocks = inputs.cubed_sphere_blocks(a=1.0, r=3.0, r_out=9.0)
    lv = inputs.uniform_leaves(level)
    leaves = [lf for b in range(len(blocks)) for lf in lv]
    eb = [b for b in range(len(blocks)) for _ in lv]
    return BlockMesh(blocks, eb, leaves, [p] * len(leaves))


def test_laplacian_of_interpolated_field_on_curved_blocks():
    """u_h = the p = 8 interpolant of U = sin(x/2) cos(0.3 y) + 0.2 z^2 on wedge
    and shell elements (every block at level 2): the estimator's Lap u_h (exact
    map with its second derivatives) matches Lap U to interpolation accuracy
    (errors of 2e-6 to 2e-5); dropping the map's second derivatives (a
    plausible mistake) is off by 0.1 to 1."""
    m = _wedge_shell_mesh(8, level=2)
    U = lambda X: np.sin(0.5 * X[:, 0]) * np.cos(0.3 * X[:, 1]) + 0.2 * X[:, 2] ** 2
    LU = lambda X: -0.34 * np.sin(0.5 * X[:, 0]) * np.cos(0.3 * X[:, 1]) + 0.4
    from oracle.sipg import volume_points
    for e in (64, 64 * 5 + 3, 64 * 9 + 6):      # elements of two wedges and a shell
        ue = U(m.node_coords(e))
        lap, uq, wd = estimator.laplacian_at_gl(m, e, ue)
        xq = volume_points(m, e)
        err = np.abs(lap - LU(xq)).max()
        assert err < 1e-4, (e, err)
        hes = m.hessian_at
        try:
            m.hessian_at = lambda ee, xi: 0.0 * hes(ee, xi)
            lap0, _, _ = estimator.laplacian_at_gl(m, e, ue)
        finally:
            del m.hessian_at
        assert np.abs(lap0 - LU(xq)).max() > 100 * err, e


def _scaled(b, s):
    b = dict(b)
    if b["kind"] == "hex8":
        b["corners"] = [[s * v for v in c] for c in b["corners"]]
    elif b["kind"] == "wedge":
        b["a"], b["r"] = s * b["a"], s * b["r"]
    else:
        b["r1"], b["r2"] = s * b["r1"], s * b["r2"]
    return b


def test_fiducial_grid_weights_scale_exactly():
    """A fiducial grid equal to the physical one changes nothing; one scaled by
    s multiplies the volume term by s^5 (h_e^2 s^2, w det J s^3), the flux-jump
    term by s^3 (h_m s, w S s^2) and the value-jump terms by s^0 (sigma / h_m
    s^-2, w S s^2) -- each ingredient taken from the right grid."""
    m = _wedge_shell_mesh(3)
    u = inputs.random_vector(m.n_dofs, seed=9)
    gD = lambda X: 0.1 * X[:, 0]
    base, vol, mort = estimator.estimate(m, u, gD_fn=gD, parts=True)
    same = estimator.estimate(m, u, gD_fn=gD, fiducial=m.with_blocks(m.blocks))
    assert np.allclose(same, base, rtol=1e-13)
    s = 1.7
    f = m.with_blocks([_scaled(b, s) for b in m.blocks])
    tot, vol_f, mort_f = estimator.estimate(m, u, gD_fn=gD, parts=True, fiducial=f)
    assert np.allclose(vol_f, s ** 5 * vol, rtol=1e-11)
    m1 = np.zeros(m.n_elems)
    m23 = np.zeros(m.n_elems)
    for mi, mm in enumerate(m.mortars):
        t1, t23 = estimator._mortar_terms(m, mi, u, gD, 10.0)
        for e in (mm.eA, mm.eB):
            if e is not None:
                m1[e] += t1
                m23[e] += t23
    assert np.allclose(mort, m1 + m23, rtol=1e-12)
    assert np.allclose(mort_f, s ** 3 * m1 + m23, rtol=1e-11)
    with pytest.raises(ValueError):
        estimator.estimate(m, u, fiducial=_wedge_shell_mesh(2))
