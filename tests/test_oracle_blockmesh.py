"""Pins of the oracle's multi-block mesh (oracle/blockmesh.py) against
closed forms and invariants that do not depend on the oracle itself."""
import itertools

import numpy as np
import pytest

from oracle import blockmesh, sipg, tables


def rotations():
    """The 24 proper rotations of the reference cube (signed permutation matrices, det +1)."""
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((-1, 1), repeat=3):
            R = np.zeros((3, 3))
            for i in range(3):
                R[i, perm[i]] = signs[i]
            if np.linalg.det(R) > 0:
                out.append(R)
    return out


def box_corners(lo, hi, R=np.eye(3)):
    """hex8 corners of the box [lo, hi] whose reference frame is rotated by R."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    C = []
    for c in range(8):
        xi = np.array([2 * (c & 1) - 1, 2 * ((c >> 1) & 1) - 1, 2 * ((c >> 2) & 1) - 1], float)
        y = R @ xi
        C.append(lo + 0.5 * (y + 1.0) * (hi - lo))
    return C


def uniform(level, block):
    m = 1 << level
    return [(block, (level, i, j, k)) for k in range(m) for j in range(m) for i in range(m)]


def refine(leaves, target):
    out = []
    for b, lf in leaves:
        if (b, lf) == target:
            L, i, j, k = lf
            for c in range(8):
                out.append((b, (L + 1, 2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + ((c >> 2) & 1))))
        else:
            out.append((b, lf))
    return out


def ball_blocks(a=1.0, r=3.0, shell=None):
    blocks = [dict(kind="hex8", corners=box_corners([-a] * 3, [a] * 3))]
    blocks += [dict(kind="wedge", face=f, a=a, r=r) for f in range(6)]
    if shell:
        blocks += [dict(kind="shell", face=f, r1=r, r2=shell) for f in range(6)]
    return blocks


def mesh_of(blocks, leaves, p):
    eb = [b for b, _ in leaves]
    lv = [lf for _, lf in leaves]
    return blockmesh.BlockMesh(blocks, eb, lv, p)


def volume(mesh):
    tot = 0.0
    for e in range(mesh.n_elems):
        _, w, _, detJ, _ = sipg.volume_geometry(mesh, e, extra=2)
        assert np.all(detJ > 0)
        tot += np.sum(w * detJ)
    return tot


def test_ball_mortar_counts_and_volume():
    blocks = ball_blocks(1.0, 3.0)
    leaves = sum((uniform(0, b) for b in range(7)), [])
    m = mesh_of(blocks, leaves, [6] * len(leaves))
    inter = sum(1 for mo in m.mortars if mo.eB is not None)
    bnd = sum(1 for mo in m.mortars if mo.eB is None)
    assert (inter, bnd) == (18, 6)         # 6 cube-wedge + 12 wedge-wedge faces; 6 outer faces
    assert abs(volume(m) - 4.0 / 3.0 * np.pi * 27.0) / (4.0 / 3.0 * np.pi * 27.0) < 2e-3


def test_ball_volume_converges_and_surface_area():
    blocks = ball_blocks(1.0, 3.0)
    errs = []
    for p in (3, 5, 7):
        leaves = sum((uniform(1, b) for b in range(7)), [])
        m = mesh_of(blocks, leaves, [p] * len(leaves))
        errs.append(abs(volume(m) / (4.0 / 3.0 * np.pi * 27.0) - 1.0))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-6
    leaves = sum((uniform(1, b) for b in range(7)), [])
    m = mesh_of(blocks, leaves, [7] * len(leaves))
    area = 0.0
    for mi, mo in enumerate(m.mortars):
        if mo.eB is None:
            area += sipg.MortarData(m, mi, 10.0).W.sum()
    assert abs(area / (4 * np.pi * 9.0) - 1.0) < 1e-6


def test_shell_volume_inverse_radius_map():
    blocks = ball_blocks(1.0, 2.0, shell=4.0)
    leaves = sum((uniform(1, b) for b in range(13)), [])
    m = mesh_of(blocks, leaves, [7] * len(leaves))
    assert abs(volume(m) / (4.0 / 3.0 * np.pi * 64.0) - 1.0) < 1e-5
    # the shell's radial coordinate follows 1/r linearly: the midpoint of a radial line
    x = blockmesh.block_map(blocks[7], np.array([[0.3, -0.2, 0.0]]))
    assert abs(np.linalg.norm(x) - 1.0 / (0.5 / 2.0 + 0.5 / 4.0)) < 1e-12


def patch_residual(mesh):
    u = lambda X: X[:, 0] ** 2 + X[:, 1] ** 2 - 2 * X[:, 2] ** 2 + X[:, 0] * X[:, 1]
    A = sipg.assemble(mesh, C=10.0)
    F = sipg.rhs(mesh, lambda X: np.zeros(len(X)), u, C=10.0)
    uI = sipg.interpolate(mesh, u)
    return np.linalg.norm(A @ uI - F) / np.linalg.norm(F), A


@pytest.mark.parametrize("ri", range(0, 24, 5))
def test_patch_test_across_rotated_blocks(ri):
    """Two affine blocks, the second with its reference frame rotated; 2:1 and
    p-jump faces on the block interface: SIPG consistency makes L u_I = F for
    quadratic u (p >= 2), and L is symmetric positive definite."""
    R = rotations()[ri]
    blocks = [dict(kind="hex8", corners=box_corners([0, 0, 0], [1, 1, 1])),
              dict(kind="hex8", corners=box_corners([1, 0, 0], [2, 1, 1], R))]
    leaves = uniform(1, 0) + uniform(1, 1)
    leaves = refine(leaves, (0, (1, 1, 0, 0)))      # block 0 element touching the interface
    rng = np.random.default_rng(ri)
    p = rng.integers(2, 4, size=len(leaves))
    m = mesh_of(blocks, leaves, p)
    res, A = patch_residual(m)
    assert res < 1e-10
    Ad = A.toarray()
    assert np.abs(Ad - Ad.T).max() / np.abs(Ad).max() < 1e-12
    assert np.linalg.eigvalsh(Ad).min() > 0


def test_patch_test_coarse_side_in_rotated_block():
    R = rotations()[13]
    blocks = [dict(kind="hex8", corners=box_corners([0, 0, 0], [1, 1, 1])),
              dict(kind="hex8", corners=box_corners([0, 1, 0], [1, 2, 1], R))]
    leaves = uniform(1, 0) + uniform(1, 1)
    # refine the element of block 1 that touches the interface y = 1 at its lowest corner
    tgt = None
    for b, lf in leaves:
        if b == 1:
            L, i, j, k = lf
            centre = -1.0 + (2.0 * np.array([i, j, k], float) + 1.0) / 2.0 ** L
            c = blockmesh.block_map(blocks[1], centre[None, :])[0]
            if c[1] < 1.5 and c[0] < 0.5 and c[2] < 0.5:
                tgt = (b, lf)
    leaves = refine(leaves, tgt)
    m = mesh_of(blocks, leaves, [3] * len(leaves))
    assert any(mo.eB is not None and np.abs(np.abs(mo.mapB[0]).sum() - 1.0) < 1e-12 for mo in m.mortars)
    res, _ = patch_residual(m)
    assert res < 1e-10


def test_wedge_and_shell_frames_right_handed():
    for f in range(6):
        for blk in (dict(kind="wedge", face=f, a=1.0, r=3.0), dict(kind="shell", face=f, r1=3.0, r2=9.0)):
            xi = np.array([[0.1, -0.2, 0.3]])
            h = 1e-6
            J = np.column_stack([(blockmesh.block_map(blk, xi + h * np.eye(3)[k]) -
                                  blockmesh.block_map(blk, xi - h * np.eye(3)[k]))[0] / (2 * h) for k in range(3)])
            assert np.linalg.det(J) > 0
            # the third reference axis points outward along the cube face normal
            d, s = divmod(f, 2)
            assert J[d, 2] * (1 if s else -1) > 0


def test_block_jacobians_match_finite_differences():
    blocks = [dict(kind="wedge", face=f, a=1.5, r=7.0) for f in range(6)]
    blocks += [dict(kind="shell", face=f, r1=7.0, r2=1e6) for f in range(6)]
    blocks += [dict(kind="hex8", corners=box_corners([0, 1, 2], [2, 2, 5], rotations()[9]))]
    rng = np.random.default_rng(0)
    xi = rng.uniform(-0.9, 0.9, size=(5, 3))
    for blk in blocks:
        J = blockmesh.block_jacobian(blk, xi)
        for k in range(3):
            h = 1e-6
            fd = (blockmesh.block_map(blk, xi + h * np.eye(3)[k]) - blockmesh.block_map(blk, xi - h * np.eye(3)[k])) / (2 * h)
            assert np.abs(J[:, :, k] - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())


def test_far_shell_keeps_positive_jacobian_and_exact_volume():
    """Shell to r2 = 1e9 in a single element per block at p = 2: the exact map
    keeps det J > 0 (an interpolated map would fold), and the shell volume
    between r1 and r2' matches 4/3 pi (r2'^3 - r1^3) for a moderate r2'."""
    blocks = ball_blocks(1.0, 3.0, shell=1e9)
    leaves = sum((uniform(0, b) for b in range(13)), [])
    m = mesh_of(blocks, leaves, [2] * len(leaves))
    for e in range(m.n_elems):
        _, _, _, detJ, _ = sipg.volume_geometry(m, e)
        assert np.all(detJ > 0)
    blocks = ball_blocks(1.0, 3.0, shell=6.0)
    m = mesh_of(blocks, leaves, [6] * len(leaves))
    shell = sum(np.sum(sipg.volume_geometry(m, e, extra=4)[1] * sipg.volume_geometry(m, e, extra=4)[3])
                for e in range(7, 13))
    assert abs(shell / (4.0 / 3.0 * np.pi * (216.0 - 27.0)) - 1.0) < 1e-6
