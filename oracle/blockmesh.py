"""Multi-block octree mesh for the oracle (test infrastructure only).

Sec. II.A.1 (mesh): the domain is a union of macro-elements (blocks), each
the image of the reference cube under its own map; every block is refined as
an octree and the leaves carry their own polynomial degree.  Blocks meet
face to face with arbitrary relative orientation.  The mortar set is built
as in the single-block mesh (oracle.mesh): one mortar per conforming face
pair, per 2:1 interface piece and per boundary face.

Block maps (Sec. III: the cubed-sphere domains of the test problems):
 * 'hex8'  : trilinear map through 8 corner points, corner (i, j, k) in
             {0, 1}^3 at index i + 2 j + 4 k (a box or any parallelepiped);
 * 'wedge' : one of the six blocks between the cube of half-width a and the
             sphere of radius r: the cube-face point and its central
             projection onto the sphere, blended linearly in the radial
             reference coordinate;
 * 'shell' : one of the six blocks of the spherical shell r1 < r < r2 with
             the inverse-radius map 1/r = (1 - t)/r1 + t/r2 (t = (xi_2 + 1)/2)
             along the central projection of the cube face.
Wedge and shell frames: for cube face (axis d, sign sg) the reference axes
0, 1, 2 point along e_{t1}, e_{t2} and outward, with (t1, t2) = (d+1, d+2)
(mod 3) for sg = +1 and (d+2, d+1) for sg = -1 (right-handed frames).

Element geometry on block meshes is exact: x and J = dx/dxi come from the
block map itself composed with the element's linear map into its block
(Sec. II.A.5, the Jacobian of the mapping phi_e), so shell blocks reaching
r2 >> r1 keep a positive Jacobian at any degree and block interfaces are
watertight.  The block-map Jacobians here are derived symbolically (sympy)
from the formulas above.

How neighbours across block boundaries are found (independent of the
library's block connectivity and orientation codes): faces are matched by
the physical positions of their centres and corners under the exact block
maps; side B's face coordinates of the mortar points come from the affine
map fixed by where side A's four face corners fall on side B's face
(lattice {-1, 0, 1}^2 of B's face coordinates, so a quarter of a coarse face
is found as well).

Parity pinned by tests/test_oracle_blockmesh.py: polynomial patch test and
symmetry / positive definiteness on affine blocks glued in every relative
orientation with 2:1 and p-jump faces across the block interfaces, volume
and surface area of the cubed-sphere ball against 4/3 pi r^3 and 4 pi r^2,
mortar counts.
"""
import numpy as np
from scipy.spatial import cKDTree

from . import tables
from .mesh import Mesh, Mortar, subface_map, tangential_dims


def wedge_axes(face):
    d, s = divmod(int(face), 2)
    if s == 1:
        return d, 1.0, (d + 1) % 3, (d + 2) % 3
    return d, -1.0, (d + 2) % 3, (d + 1) % 3


def block_map(block, xi):
    """Physical points of block reference points xi (P, 3) in [-1, 1]^3."""
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    kind = block["kind"]
    if kind == "hex8":
        C = np.asarray(block["corners"], dtype=np.float64).reshape(8, 3)
        x = np.zeros((len(xi), 3))
        for c in range(8):
            bits = (c & 1, (c >> 1) & 1, (c >> 2) & 1)
            w = np.ones(len(xi))
            for k in range(3):
                w = w * (0.5 * (1.0 + xi[:, k]) if bits[k] else 0.5 * (1.0 - xi[:, k]))
            x += w[:, None] * C[c]
        return x
    d, sg, t1, t2 = wedge_axes(block["face"])
    v = np.zeros((len(xi), 3))
    v[:, d] = sg
    v[:, t1] = xi[:, 0]
    v[:, t2] = xi[:, 1]
    t = 0.5 * (xi[:, 2] + 1.0)
    length = np.linalg.norm(v, axis=1)
    if kind == "wedge":
        a, r = float(block["a"]), float(block["r"])
        cube = a * v
        sph = r * v / length[:, None]
        return (1.0 - t)[:, None] * cube + t[:, None] * sph
    if kind == "shell":
        r1, r2 = float(block["r1"]), float(block["r2"])
        rad = 1.0 / ((1.0 - t) / r1 + t / r2)
        return rad[:, None] * v / length[:, None]
    raise ValueError("unknown block kind " + str(kind))


_JAC = {}


def _jacobian_fn(kind, face):
    """numpy function (xi0, xi1, xi2, params...) -> 3 x 3 entries of d x / d xi, from sympy."""
    key = (kind, face)
    if key in _JAC:
        return _JAC[key]
    import sympy
    xi = sympy.symbols("xi0 xi1 xi2", real=True)
    if kind == "hex8":
        C = sympy.symbols("c0:24", real=True)
        x = [0, 0, 0]
        for c in range(8):
            w = 1
            for k in range(3):
                w = w * ((1 + xi[k]) / 2 if (c >> k) & 1 else (1 - xi[k]) / 2)
            for i in range(3):
                x[i] = x[i] + w * C[3 * c + i]
        params = C
    else:
        d, sg, t1, t2 = wedge_axes(face)
        v = [0, 0, 0]
        v[d] = sympy.Integer(int(sg))
        v[t1] = xi[0]
        v[t2] = xi[1]
        length = sympy.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
        t = (xi[2] + 1) / 2
        if kind == "wedge":
            a, r = sympy.symbols("a r", positive=True)
            x = [(1 - t) * a * v[i] + t * r * v[i] / length for i in range(3)]
            params = (a, r)
        else:
            r1, r2 = sympy.symbols("r1 r2", positive=True)
            R = 1 / ((1 - t) / r1 + t / r2)
            x = [R * v[i] / length for i in range(3)]
            params = (r1, r2)
    J = [[sympy.diff(x[i], xi[l]) for l in range(3)] for i in range(3)]
    H = [[[sympy.diff(x[i], xi[l], xi[m]) for m in range(3)] for l in range(3)] for i in range(3)]
    fn = sympy.lambdify(tuple(xi) + tuple(params), J, "numpy")
    fh = sympy.lambdify(tuple(xi) + tuple(params), H, "numpy")
    _JAC[key] = fn
    _HES[key] = fh
    return fn


_HES = {}


def block_hessian(block, xi):
    """d^2 x_i / dxi_l dxi_m of the block map at reference points xi (P, 3):
    (P, 3, 3, 3), from the same symbolic map as block_jacobian."""
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    kind = block["kind"]
    if kind == "hex8":
        params = np.asarray(block["corners"], dtype=np.float64).reshape(24)
        key = ("hex8", None)
    elif kind == "wedge":
        params = (float(block["a"]), float(block["r"]))
        key = ("wedge", int(block["face"]))
    else:
        params = (float(block["r1"]), float(block["r2"]))
        key = ("shell", int(block["face"]))
    _jacobian_fn(*key)
    vals = _HES[key](xi[:, 0], xi[:, 1], xi[:, 2], *params)
    H = np.zeros((len(xi), 3, 3, 3))
    for i in range(3):
        for l in range(3):
            for m in range(3):
                H[:, i, l, m] = np.broadcast_to(np.asarray(vals[i][l][m], dtype=np.float64), (len(xi),))
    return H


def block_jacobian(block, xi):
    """d x / d xi of the block map at reference points xi (P, 3): (P, 3, 3)."""
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    kind = block["kind"]
    if kind == "hex8":
        params = np.asarray(block["corners"], dtype=np.float64).reshape(24)
        fn = _jacobian_fn("hex8", None)
    elif kind == "wedge":
        params = (float(block["a"]), float(block["r"]))
        fn = _jacobian_fn("wedge", int(block["face"]))
    else:
        params = (float(block["r1"]), float(block["r2"]))
        fn = _jacobian_fn("shell", int(block["face"]))
    J = np.zeros((len(xi), 3, 3))
    vals = fn(xi[:, 0], xi[:, 1], xi[:, 2], *params)
    for i in range(3):
        for l in range(3):
            J[:, i, l] = np.broadcast_to(np.asarray(vals[i][l], dtype=np.float64), (len(xi),))
    return J


class BlockMortar(Mortar):
    __slots__ = ("mapB",)

    def __init__(self, eA, fA, eB, fB, pm, mapB):
        super().__init__(eA, fA, (0, 0), eB, fB, None, pm)
        self.mapB = mapB     # (M 2x2, c 2): side B face coordinates = M s + c


class BlockMesh(Mesh):
    """Octree leaves (level, ix, iy, iz) of several blocks; element e lies in block elem_block[e]."""

    def __init__(self, blocks, elem_block, leaves, p):
        self.blocks = [dict(b) for b in blocks]
        self.elem_block = np.asarray(elem_block, dtype=np.int64).ravel()
        self.leaves = np.asarray(leaves, dtype=np.int64).reshape(-1, 4)
        self.p = np.asarray(p, dtype=np.int64).ravel()
        if not (len(self.p) == len(self.leaves) == len(self.elem_block)):
            raise ValueError("one block index and one degree per leaf")
        self.warp = None
        self.n_elems = len(self.leaves)
        self.n = self.p + 1
        self.dof_off = np.concatenate([[0], np.cumsum(self.n ** 3)])
        self.n_dofs = int(self.dof_off[-1])
        self.key = {(int(b),) + tuple(int(v) for v in lf): e
                    for e, (b, lf) in enumerate(zip(self.elem_block, self.leaves))}
        if len(self.key) != self.n_elems:
            raise ValueError("duplicate leaf")
        self._block_faces()
        self._build_mortars()

    # ---- geometry -------------------------------------------------------
    def block_ref(self, e, xi):
        """Block reference coordinates of element reference points xi (P, 3)."""
        L, ix, iy, iz = (int(v) for v in self.leaves[e])
        idx = np.array([ix, iy, iz], dtype=np.float64)
        return -1.0 + (2.0 * idx + np.asarray(xi) + 1.0) / (2.0 ** L)

    def exact_point(self, e, xi):
        return block_map(self.blocks[int(self.elem_block[e])], self.block_ref(e, xi))

    def node_coords(self, e):
        n = int(self.n[e])
        xl, _ = tables.lgl_nodes_weights(n)
        return self.exact_point(e, tables.tensor_points(xl))

    def position_at(self, e, xi):
        return self.exact_point(e, xi)

    def jacobian_at(self, e, xi):
        """J[p, i, l] = d x_i / d xi_l of phi_e: the block map's Jacobian times 2^-level."""
        L = int(self.leaves[e][0])
        return block_jacobian(self.blocks[int(self.elem_block[e])], self.block_ref(e, xi)) / (2.0 ** L)

    def hessian_at(self, e, xi):
        """X[p, i, l, m] = d^2 x_i / dxi_l dxi_m of phi_e: the block map's
        second derivatives times 4^-level."""
        L = int(self.leaves[e][0])
        return block_hessian(self.blocks[int(self.elem_block[e])], self.block_ref(e, xi)) / (4.0 ** L)

    def with_blocks(self, blocks):
        """The same leaves, degrees and block indices on other block maps (a
        fiducial grid of identical structure and connectivity)."""
        return BlockMesh(blocks, self.elem_block, self.leaves, self.p)

    def face_point_ref(self, f, b1, b2):
        d, s = divmod(f, 2)
        t1, t2 = tangential_dims(d)
        xi = np.zeros((np.size(b1), 3))
        xi[:, d] = 1.0 if s == 1 else -1.0
        xi[:, t1] = b1
        xi[:, t2] = b2
        return xi

    # ---- connectivity ---------------------------------------------------
    def _block_faces(self):
        """Block faces whose four corners coincide with another block face's are interior."""
        cents, ids = [], []
        for b, blk in enumerate(self.blocks):
            for f in range(6):
                d, s = divmod(f, 2)
                t1, t2 = tangential_dims(d)
                xi = np.zeros((4, 3))
                xi[:, d] = 1.0 if s == 1 else -1.0
                xi[:, t1] = [-1, 1, -1, 1]
                xi[:, t2] = [-1, -1, 1, 1]
                cents.append(block_map(blk, xi).mean(axis=0))
                ids.append((b, f))
        cents = np.array(cents)
        scale = np.maximum(np.linalg.norm(cents, axis=1), 1.0)
        tree = cKDTree(cents)
        self.block_face_interior = {}
        for k, (b, f) in enumerate(ids):
            hits = [j for j in tree.query_ball_point(cents[k], 1e-9 * scale[k]) if j != k]
            self.block_face_interior[(b, f)] = len(hits) > 0

    def _face_center(self, b, L, idx, f):
        d, s = divmod(f, 2)
        xi = np.zeros((1, 3))
        xi[0, d] = 1.0 if s == 1 else -1.0
        bref = -1.0 + (2.0 * np.asarray(idx, dtype=np.float64) + xi[0] + 1.0) / (2.0 ** L)
        return block_map(self.blocks[b], bref[None, :])[0]

    def _affine_to(self, eA, fA, eB, fB):
        """(M, c) with side B face coordinates = M s + c for side A face coordinates s."""
        sA = np.array([[-1, -1], [1, -1], [-1, 1], [1, 1]], dtype=np.float64)
        PA = self.exact_point(eA, self.face_point_ref(fA, sA[:, 0], sA[:, 1]))
        lat = np.array([(u, v) for v in (-1.0, 0.0, 1.0) for u in (-1.0, 0.0, 1.0)])
        PB = self.exact_point(eB, self.face_point_ref(fB, lat[:, 0], lat[:, 1]))
        scale = max(1.0, float(np.abs(PA).max()))
        bB = []
        for k in range(4):
            dist = np.linalg.norm(PB - PA[k], axis=1)
            j = int(np.argmin(dist))
            if dist[j] > 1e-8 * scale:
                raise ValueError(f"faces ({eA},{fA}) and ({eB},{fB}) do not match")
            bB.append(lat[j])
        bB = np.array(bB)
        M = np.column_stack([(bB[1] - bB[0]) / 2.0, (bB[2] - bB[0]) / 2.0])
        c = bB[0] + M @ np.array([1.0, 1.0])
        if np.abs(M @ sA[3] + c - bB[3]).max() > 1e-12:
            raise ValueError("face corner correspondence is not affine")
        return M, c

    def _build_mortars(self):
        self.mortars = []
        self.elem_mortars = [[[] for _ in range(6)] for _ in range(self.n_elems)]
        bf_keys, bf_cent, bf_level = [], [], []
        for e in range(self.n_elems):
            b = int(self.elem_block[e])
            L, ix, iy, iz = (int(v) for v in self.leaves[e])
            idx = [ix, iy, iz]
            for f in range(6):
                d, s = divmod(f, 2)
                if idx[d] + (1 if s == 1 else -1) in (-1, 1 << L):
                    bf_keys.append((e, f))
                    bf_cent.append(self._face_center(b, L, idx, f))
                    bf_level.append(L)
        tree = cKDTree(np.array(bf_cent)) if bf_cent else None
        bf_index = {k: i for i, k in enumerate(bf_keys)}

        def find(center, level):
            tol = 1e-9 * max(1.0, float(np.linalg.norm(center)))
            return [bf_keys[j] for j in tree.query_ball_point(center, tol) if bf_level[j] == level]

        for e in range(self.n_elems):
            b = int(self.elem_block[e])
            L, ix, iy, iz = (int(v) for v in self.leaves[e])
            idx = [ix, iy, iz]
            for f in range(6):
                d, s = divmod(f, 2)
                fo = 2 * d + (1 - s)
                j = list(idx)
                j[d] += 1 if s == 1 else -1
                t1, t2 = tangential_dims(d)
                pe = int(self.p[e])
                if 0 <= j[d] < (1 << L):             # inside the block: integer neighbours
                    k = (b, L, j[0], j[1], j[2])
                    if k in self.key:
                        o = self.key[k]
                        if o < e:
                            continue
                        m = BlockMortar(e, f, o, fo, max(pe, int(self.p[o])), (np.eye(2), np.zeros(2)))
                    else:
                        kc = (b, L - 1, j[0] >> 1, j[1] >> 1, j[2] >> 1)
                        if L > 0 and kc in self.key:
                            o = self.key[kc]
                            pos = (1 + (idx[t1] & 1), 1 + (idx[t2] & 1))
                            M = np.diag([0.5, 0.5])
                            c = np.array([-0.5 if pos[0] == 1 else 0.5, -0.5 if pos[1] == 1 else 0.5])
                            m = BlockMortar(e, f, o, fo, max(pe, int(self.p[o])), (M, c))
                        else:
                            for b2 in range(2):
                                for b1 in range(2):
                                    cc = [2 * j[0], 2 * j[1], 2 * j[2]]
                                    cc[d] = 2 * j[d] + (0 if s == 1 else 1)
                                    cc[t1] += b1
                                    cc[t2] += b2
                                    if (b, L + 1, cc[0], cc[1], cc[2]) not in self.key:
                                        raise ValueError(f"mesh is not 2:1 balanced at element {e} face {f}")
                            continue
                elif not self.block_face_interior[(b, f)]:
                    m = BlockMortar(e, f, None, None, pe, None)
                else:                                 # across a block interface: physical matching
                    cen = bf_cent[bf_index[(e, f)]]
                    same = [(o, fb) for (o, fb) in find(cen, L) if o != e]
                    if same:
                        o, fb = same[0]
                        if o < e:
                            continue
                        m = BlockMortar(e, f, o, fb, max(pe, int(self.p[o])), self._affine_to(e, f, o, fb))
                    else:
                        coarse = find(self._face_center(b, L - 1, [v >> 1 for v in idx], f), L - 1) if L > 0 else []
                        if coarse:
                            o, fb = coarse[0]
                            m = BlockMortar(e, f, o, fb, max(pe, int(self.p[o])), self._affine_to(e, f, o, fb))
                        else:
                            fine = 0
                            for b2 in range(2):
                                for b1 in range(2):
                                    cc = [2 * v for v in idx]
                                    cc[d] += 1 if s == 1 else 0
                                    cc[t1] += b1
                                    cc[t2] += b2
                                    fine += len(find(self._face_center(b, L + 1, cc, f), L + 1))
                            if fine != 4:
                                raise ValueError(f"block interface not matched at element {e} face {f}")
                            continue
                self.mortars.append(m)
        for mi, m in enumerate(self.mortars):
            self.elem_mortars[m.eA][m.fA].append(mi)
            if m.eB is not None:
                self.elem_mortars[m.eB][m.fB].append(mi)

    def side_ref_points(self, m, side, s1, s2):
        if side == 0:
            return self.face_point_ref(m.fA, s1, s2)
        M, c = m.mapB
        bb = M @ np.vstack([s1, s2]) + c[:, None]
        return self.face_point_ref(m.fB, bb[0], bb[1])
