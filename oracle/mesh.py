"""Single-block octree mesh for the oracle (test infrastructure only).

Sec. II.A.1 (mesh): the macro-element is the box [lo, hi]^3 (image of the
reference cube); fine elements are octree leaves (level, ix, iy, iz), each
with the map Phi_e that is linear in the block's reference coordinates
(eq. Phi_e) composed with the block map.  Faces of adjacent leaves differ by
at most 2:1.  The mortar set M = M_I u M_B is built from the leaf faces; a
mortar joins at most two elements.

Readings (where the paper leaves the choice open):
 * Element geometry is isoparametric: the block map is sampled at the
   element's own LGL nodes and interpolated with its degree-p basis.
 * Curved block map ("sine warp"): x_i <- x_i + a sin(2 pi k_i x_i)
   sin(2 pi k_{i+1} x_{i+1}) (cyclic i), evaluated on the unwarped point.
 * Mortar '-' side (geometry side, A): the finer element; on conforming
   faces the lower element index.  Normals and surface Jacobian come from A.
 * Mortar degree p_m = max(p^+, p^-) (mortar figure caption), with p_m + 1
   GL points per direction.
 * Face tangential axes are the two remaining reference axes in increasing
   order.  Sub-face position codes: 0 full face, 1 lower half, 2 upper half.

Parity pinned by the mesh/mortar count and mortar-degree tests
(tests/test_oracle_mesh.py) and the geometry identities in
tests/test_oracle_geometry.py.
"""
import numpy as np

from . import tables


def tangential_dims(d):
    return [k for k in range(3) if k != d]


def subface_map(pos, s):
    """Map a mortar coordinate s in [-1, 1] to the face coordinate of a side."""
    if pos == 0:
        return s
    if pos == 1:
        return (s - 1.0) / 2.0
    return (s + 1.0) / 2.0


class Mortar:
    __slots__ = ("eA", "fA", "posA", "eB", "fB", "posB", "pm")

    def __init__(self, eA, fA, posA, eB, fB, posB, pm):
        self.eA, self.fA, self.posA = eA, fA, posA
        self.eB, self.fB, self.posB = eB, fB, posB
        self.pm = pm

    @property
    def boundary(self):
        return self.eB is None


class Mesh:
    """Octree leaves of one box block, each with its own polynomial degree."""

    def __init__(self, lo, hi, leaves, p, warp=None):
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)
        self.leaves = np.asarray(leaves, dtype=np.int64).reshape(-1, 4)
        self.p = np.asarray(p, dtype=np.int64).ravel()
        if len(self.p) != len(self.leaves):
            raise ValueError("one polynomial degree per leaf")
        self.warp = warp  # None or (amp, (k0, k1, k2))
        self.n_elems = len(self.leaves)
        self.n = self.p + 1
        self.dof_off = np.concatenate([[0], np.cumsum(self.n ** 3)])
        self.n_dofs = int(self.dof_off[-1])
        self.key = {tuple(int(v) for v in lf): e for e, lf in enumerate(self.leaves)}
        if len(self.key) != self.n_elems:
            raise ValueError("duplicate leaf")
        self._build_mortars()

    # ---- geometry -------------------------------------------------------
    def element_bounds(self, e):
        L, ix, iy, iz = self.leaves[e]
        size = (self.hi - self.lo) / (2.0 ** L)
        a = self.lo + size * np.array([ix, iy, iz], dtype=np.float64)
        return a, a + size

    def block_map(self, x):
        """Block map applied to unwarped physical points x (P, 3)."""
        x = np.asarray(x, dtype=np.float64)
        if self.warp is None:
            return x.copy()
        amp, k = self.warp
        y = x.copy()
        for i in range(3):
            j = (i + 1) % 3
            y[:, i] = x[:, i] + amp * np.sin(2 * np.pi * k[i] * x[:, i]) * np.sin(2 * np.pi * k[j] * x[:, j])
        return y

    def node_coords(self, e):
        """Physical coordinates of element e's LGL nodes, (n^3, 3)."""
        n = int(self.n[e])
        xl, _ = tables.lgl_nodes_weights(n)
        ref = tables.tensor_points(xl)
        a, b = self.element_bounds(e)
        x = a + (ref + 1.0) * 0.5 * (b - a)
        return self.block_map(x)

    def jacobian_at(self, e, xi):
        """J[p, i, l] = d x_i / d xi_l of the isoparametric map at reference points xi."""
        n = int(self.n[e])
        xl, _ = tables.lgl_nodes_weights(n)
        X = self.node_coords(e)
        _, dPsi = tables.basis3d(xl, xi)
        J = np.einsum('lpa,ai->pil', dPsi, X)
        return J

    def position_at(self, e, xi):
        n = int(self.n[e])
        xl, _ = tables.lgl_nodes_weights(n)
        Psi, _ = tables.basis3d(xl, xi)
        return Psi @ self.node_coords(e)

    # ---- connectivity ---------------------------------------------------
    def _neighbor(self, e, f):
        """('bnd',) | ('conf', nb) | ('coarse_nb', nb) | ('fine_nbs', [nb...])."""
        L, ix, iy, iz = (int(v) for v in self.leaves[e])
        idx = [ix, iy, iz]
        d, s = divmod(f, 2)
        j = list(idx)
        j[d] += 1 if s == 1 else -1
        if j[d] < 0 or j[d] >= (1 << L):
            return ('bnd',)
        k = (L, j[0], j[1], j[2])
        if k in self.key:
            return ('conf', self.key[k])
        if L > 0:
            kc = (L - 1, j[0] >> 1, j[1] >> 1, j[2] >> 1)
            if kc in self.key:
                return ('coarse_nb', self.key[kc])
        t1, t2 = tangential_dims(d)
        nbs = []
        for b2 in range(2):
            for b1 in range(2):
                c = [2 * j[0], 2 * j[1], 2 * j[2]]
                c[d] = 2 * j[d] + (0 if s == 1 else 1)
                c[t1] += b1
                c[t2] += b2
                kf = (L + 1, c[0], c[1], c[2])
                if kf not in self.key:
                    raise ValueError(f"mesh is not 2:1 balanced or does not cover the block at element {e} face {f}")
                nbs.append(self.key[kf])
        return ('fine_nbs', nbs)

    def _build_mortars(self):
        self.mortars = []
        self.elem_mortars = [[[] for _ in range(6)] for _ in range(self.n_elems)]
        for e in range(self.n_elems):
            L, ix, iy, iz = (int(v) for v in self.leaves[e])
            idx = [ix, iy, iz]
            for f in range(6):
                d, s = divmod(f, 2)
                fo = 2 * d + (1 - s)
                nb = self._neighbor(e, f)
                if nb[0] == 'bnd':
                    m = Mortar(e, f, (0, 0), None, None, None, int(self.p[e]))
                elif nb[0] == 'conf':
                    o = nb[1]
                    if o < e:
                        continue
                    m = Mortar(e, f, (0, 0), o, fo, (0, 0), int(max(self.p[e], self.p[o])))
                elif nb[0] == 'coarse_nb':
                    o = nb[1]
                    t1, t2 = tangential_dims(d)
                    posB = (1 + (idx[t1] & 1), 1 + (idx[t2] & 1))
                    m = Mortar(e, f, (0, 0), o, fo, posB, int(max(self.p[e], self.p[o])))
                else:
                    continue
                self.mortars.append(m)
        for mi, m in enumerate(self.mortars):
            self.elem_mortars[m.eA][m.fA].append(mi)
            if m.eB is not None:
                self.elem_mortars[m.eB][m.fB].append(mi)

    def side_ref_points(self, m, side, s1, s2):
        """Reference coordinates on mortar m's side (0 = A, 1 = B) of its points (s1, s2)."""
        if side == 0:
            return self.face_ref_points(m.fA, m.posA, s1, s2)
        return self.face_ref_points(m.fB, m.posB, s1, s2)

    def face_ref_points(self, f, pos, s1, s2):
        """Reference coordinates on face f of mortar points (s1, s2) for sub-face pos."""
        d, s = divmod(f, 2)
        t1, t2 = tangential_dims(d)
        xi = np.zeros((len(s1), 3))
        xi[:, d] = 1.0 if s == 1 else -1.0
        xi[:, t1] = subface_map(pos[0], s1)
        xi[:, t2] = subface_map(pos[1], s2)
        return xi
